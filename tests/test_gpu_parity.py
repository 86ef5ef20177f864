"""GPU parity: every hot-path step through the C ABI against the FP64 CPU
oracle on the same seeded inputs.

Tolerances: the FP64 path is held to 1e-10 relative on the probabilities
and on p; the mixed FP32 + FP64-refinement path to 1e-4 relative on
P_EELS, P_CL (and P_ext, P_abs) and 1e-4 in relative 2-norm on p.
Single steps: K0/K1 1e-13, fields 1e-12, FP64 matvec 1e-12, FP32 matvec
2e-5 (relative 2-norm; the FP32 FFT rounding grows like eps32 * log M)."""
import numpy as np
import pytest

from oracle import green, run
from oracle.constants import NM
from paper_2208_01348_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2208_01348_gb300 import eelsdda
    return eelsdda


@pytest.fixture(scope="module")
def ctx(dd):
    h = dd.eels_create(0)
    yield h
    dd.eels_destroy(h)


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ------------------------------------------------------------------ K0, K1
def test_bessel_k01_device_matches_scipy(dd):
    import torch
    from scipy.special import kv
    mags = np.geomspace(1e-3, 40.0, 41)
    args = np.linspace(-np.pi / 2, 0.0, 13)
    z = (mags[:, None] * np.exp(1j * args[None, :])).ravel()
    z = np.concatenate([z, [2.0, 2.0000001, -2j, 1.999 - 0.01j, 0.013, 3.1 * np.exp(-1.558j)]])
    zt = torch.from_numpy(z.astype(np.complex128)).cuda()
    k0 = torch.empty_like(zt)
    k1 = torch.empty_like(zt)
    dd.eels_bessel_k01_dev(zt.data_ptr(), k0.data_ptr(), k1.data_ptr(), len(z), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    g0, g1 = k0.cpu().numpy(), k1.cpu().numpy()
    r0, r1 = kv(0, z), kv(1, z)
    assert np.max(np.abs(g0 - r0) / np.abs(r0)) < 1e-13
    assert np.max(np.abs(g1 - r1) / np.abs(r1)) < 1e-13


# ------------------------------------------------------------------ fields
@pytest.mark.parametrize("eps_h,ekin,e_eV,beam", [
    (1.0, 100.0, 2.4, (15.0, 0.0)), (2.1025, 120.0, 3.7, (17.0, -4.0)), (4.0 + 0.05j, 200.0, 2.2, (13.0, 6.0)),
    (4.0, 200.0, 1.6, (0.0, 14.0))])
def test_incident_and_auxiliary_field(dd, ctx, eps_h, ekin, e_eV, beam):
    w = I.config_small_sphere()
    g = w.grid
    dd.eels_set_grid(ctx, g.occ, g.d_nm)
    E, Ea = dd.eels_incident_field(ctx, ekin, e_eV, eps_h, beam)
    pt = run.setup(g.nx, g.ny, g.nz, g.d_nm, g.occ, e_eV, [1.0], eps_h, beam, ekin_keV=ekin)
    assert rel(E, pt.E_inc) < 1e-12
    assert rel(Ea, pt.E_a) < 1e-12


# ------------------------------------------------------------------ matvec
def _random_grid(dims, seed, frac=0.7, nmat=1):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    occ = (rng.random((nz, ny, nx)) < frac).astype(np.uint8)
    if nmat > 1:
        occ *= rng.integers(1, nmat + 1, size=occ.shape).astype(np.uint8)
    occ.flat[0] = 1
    return occ


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 2, 2), (3, 4, 5), (7, 3, 2), (5, 9, 6), (12, 12, 12), (13, 6, 17),
                                  (32, 5, 3), (31, 4, 6), (64, 3, 2),
                                  # padded x lengths 64 and 128 with Mz a multiple of 16 / 8: the
                                  # register-resident FP32 x pass (full and ragged x lines)
                                  (32, 3, 8), (31, 5, 8), (64, 2, 4), (64, 3, 8)])
def test_matvec_equals_dense_oracle(dd, ctx, dims):
    nx, ny, nz = dims
    nmat = 2 if nx * ny * nz > 8 else 1
    occ = _random_grid(dims, seed=nx * 100 + ny * 10 + nz, nmat=nmat)
    d_nm = 2.0
    dd.eels_set_grid(ctx, occ, d_nm)
    eps_p = [I.drude(2.3), 3.0 + 0.4j][:nmat]
    eps_h = 2.0 + 0.1j
    pt = run.setup(nx, ny, nz, d_nm, occ, 2.3, eps_p, eps_h, (100.0, 100.0), ekin_keV=100.0)
    A = green.dense_matrix(pt.r, pt.k, pt.alpha)
    x = I.random_complex((3, len(pt.r), 3), seed=5)
    ref = np.stack([(A @ xi.reshape(-1)).reshape(-1, 3) for xi in x])
    y64 = dd.eels_apply_matrix(ctx, dd.EELS_FP64, 2.3, eps_p, eps_h, x)
    y32 = dd.eels_apply_matrix(ctx, dd.EELS_MIXED, 2.3, eps_p, eps_h, x)
    for i in range(3):
        assert rel(y64[i], ref[i]) < 1e-12
        assert rel(y32[i], ref[i]) < 2e-5


@pytest.mark.parametrize("dims", [(4, 32, 31), (3, 31, 32), (6, 32, 32), (2, 64, 64), (3, 64, 64), (32, 32, 32),
                                  (31, 32, 30), (64, 12, 24), (64, 64, 64)])
def test_matvec_64_point_transforms_equal_fft_oracle(dd, ctx, dims):
    """Lattices whose y and z transforms are 64 or 128 points long (the FP32
    path then uses the register-resident slab kernels); the oracle is its own
    FFT convolution (period 2N), itself pinned to the dense matrix."""
    nx, ny, nz = dims
    occ = _random_grid(dims, seed=7 * nx + ny + nz, nmat=2)
    d_nm = 1.5
    dd.eels_set_grid(ctx, occ, d_nm)
    mx, my, mz = dd.eels_padded_dims(ctx)
    assert (my, mz) in ((64, 64), (128, 128)) or mx in (64, 128)
    eps_p = [I.drude(2.0), 2.5 + 0.3j]
    eps_h = 2.1025 + 0j
    pt = run.setup(nx, ny, nz, d_nm, occ, 2.0, eps_p, eps_h, (100.0, 100.0), ekin_keV=120.0)
    op = green.FFTOperator(pt.idx, pt.n_axes, pt.d, pt.k, pt.alpha)
    x = I.random_complex((2, len(pt.r), 3), seed=11)
    ref = np.stack([op.matvec(xi) for xi in x])
    y32 = dd.eels_apply_matrix(ctx, dd.EELS_MIXED, 2.0, eps_p, eps_h, x)
    y64 = dd.eels_apply_matrix(ctx, dd.EELS_FP64, 2.0, eps_p, eps_h, x)
    for i in range(2):
        assert rel(y64[i], ref[i]) < 1e-12
        assert rel(y32[i], ref[i]) < 2e-5


@pytest.mark.parametrize("n,two_mat", [(32, False), (32, True), (64, False), (64, True), (31, True)])
def test_matvec_sphere_lattices_equal_fft_oracle(dd, ctx, n, two_mat):
    """Sphere lattices (every column's occupied cells contiguous: the slab
    kernels address dipoles through the per-column table), with one material
    or a core and shell of two, at the padded sizes of the 64- and 128-point
    register kernels; the oracle is its own FFT convolution."""
    occ = I.sphere_occupancy(n, 1.0 * n)
    if two_mat:
        c = (np.arange(n) + 0.5) - n / 2.0
        z, y, x = np.meshgrid(c, c, c, indexing="ij")
        occ = np.where(x * x + y * y + z * z <= (0.3 * n) ** 2, 2, occ).astype(np.uint8)
    d_nm = 1.0
    dd.eels_set_grid(ctx, occ, d_nm)
    eps_p = [I.drude(2.0), 2.5 + 0.3j][:2 if two_mat else 1]
    eps_h = 4.0 + 0.05j
    pt = run.setup(n, n, n, d_nm, occ, 2.0, eps_p, eps_h, (100.0, 100.0), ekin_keV=200.0)
    op = green.FFTOperator(pt.idx, pt.n_axes, pt.d, pt.k, pt.alpha)
    x = I.random_complex((1, len(pt.r), 3), seed=13)
    ref = op.matvec(x[0])
    y32 = dd.eels_apply_matrix(ctx, dd.EELS_MIXED, 2.0, eps_p, eps_h, x)
    y64 = dd.eels_apply_matrix(ctx, dd.EELS_FP64, 2.0, eps_p, eps_h, x)
    assert rel(y64[0], ref) < 1e-12
    assert rel(y32[0], ref) < 2e-5


# ------------------------------------------------------------------ solve
def _solve(dd, ctx, w, precision, energies=None, beams=None, n_dir=2562, want_p=True, eps=1e-10, max_batch=0):
    g = w.grid
    dd.eels_set_grid(ctx, g.occ, g.d_nm)
    ie = np.arange(len(w.energies_eV)) if energies is None else np.asarray(energies)
    bm = w.beams_nm if beams is None else np.asarray(beams)
    o = dd.eels_default_opts(ekin_keV=w.ekin_keV, precision=precision, eps_it=eps, n_dir=n_dir, max_batch=max_batch)
    return dd.eels_solve(ctx, o, w.energies_eV[ie], w.eps_p[ie], w.eps_h[ie], bm, want_p=want_p)


def _oracle(w, ie, ib, beams=None):
    bm = w.beams_nm if beams is None else beams
    g = w.grid
    return run.solve_point(g.nx, g.ny, g.nz, g.d_nm, g.occ, w.energies_eV[ie], w.eps_p[ie], w.eps_h[ie], bm[ib],
                           ekin_keV=w.ekin_keV)


def _check_point(res, ie, ib, o, tol_p, tol_vec):
    for key, got in (("P_EELS", res.p_eels), ("P_CL", res.p_cl), ("P_ext", res.p_ext), ("P_abs", res.p_abs)):
        assert abs(got[ie, ib] - o[key]) <= tol_p * abs(o[key]), (key, got[ie, ib], o[key])
    if res.p is not None:
        assert rel(res.p[ie, ib], o["p"]) < tol_vec


def test_small_sphere_fp64_matches_lu(dd, ctx):
    w = I.config_small_sphere()
    res = _solve(dd, ctx, w, dd.EELS_FP64, eps=1e-12)
    assert res.converged.all() and res.residual.max() <= 1e-12
    _check_point(res, 0, 0, _oracle(w, 0, 0), 1e-10, 1e-10)


def test_small_sphere_mixed_matches_lu(dd, ctx):
    w = I.config_small_sphere()
    res = _solve(dd, ctx, w, dd.EELS_MIXED, eps=1e-8)
    assert res.converged.all()
    _check_point(res, 0, 0, _oracle(w, 0, 0), 1e-4, 1e-4)


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_reduced_spectrum_glass_host(dd, ctx, prec):
    """32^3 sphere config on a 12^3 lattice: same particle, host, electron; 5 energies."""
    w = I.reduced(I.config_spectrum(), 12 / 32, n_energy=5)
    p = getattr(dd, "EELS_" + prec)
    res = _solve(dd, ctx, w, p, eps=1e-12 if prec == "FP64" else 1e-8)
    tol = 1e-10 if prec == "FP64" else 1e-4
    for ie in (0, 2, 4):
        _check_point(res, ie, 0, _oracle(w, ie, 0), tol, tol)
    # below the Cherenkov threshold the particle loss equals extinction (Sec. 2.4)
    assert np.allclose(res.p_eels, res.p_ext, rtol=1e-9 if prec == "FP64" else 1e-6, atol=0)
    # ... so the total emission of Eq. 41 reduces to P_CL (Sec. 2.6)
    assert np.all(np.abs(res.p_cl_tot - res.p_cl) <= (1e-9 if prec == "FP64" else 1e-6) * np.abs(res.p_eels))


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_reduced_cherenkov_absorbing_host(dd, ctx, prec):
    """100 nm silver sphere in eps_h = 4 + 0.05i at 200 keV (beta_h > 1) on 12^3."""
    w = I.reduced(I.config_cherenkov(), 12 / 64, n_energy=3)
    p = getattr(dd, "EELS_" + prec)
    res = _solve(dd, ctx, w, p, eps=1e-12 if prec == "FP64" else 1e-8)
    tol = 1e-10 if prec == "FP64" else 1e-4
    for ie in range(3):
        o = _oracle(w, ie, 0)
        _check_point(res, ie, 0, o, tol, tol)
        assert abs(o["P_EELS"] - o["P_ext"]) > 1e-3 * abs(o["P_ext"])


def test_reduced_rod_map_block_of_beams(dd, ctx):
    """Rod 40x40x120 nm on 4x4x12 cells, 2 energies x 6 beams solved as one batch."""
    w = I.reduced(I.config_rod_map(), 4 / 24, n_energy=2)
    beams = I.rod_raster_beams(3, 2, pitch=9.0)
    res = _solve(dd, ctx, w, dd.EELS_FP64, beams=beams, eps=1e-12)
    for ie in range(2):
        for ib in (0, 3, 5):
            _check_point(res, ie, ib, _oracle(w, ie, ib, beams), 1e-10, 1e-10)


def test_32_beams_of_one_energy_match_lu_and_solo_solves(dd, ctx):
    """A spherical gold shell in a 17^3 box (padded 64 x 36 x 36: the mixed
    path's FP32 rounds and the register x pass, which reuses one staged D-hat
    tile over up to 16 beams): 32 beams of one energy in one batch against
    the oracle's LU solve, and bit-identical to the beams solved alone."""
    n = 17
    c = (np.arange(n) + 0.5) - n / 2.0
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    rr = np.sqrt(x * x + y * y + z * z)
    occ = ((rr >= 6.5) & (rr <= 8.5)).astype(np.uint8)
    d_nm, e_eV = 2.0, 2.4
    dd.eels_set_grid(ctx, occ, d_nm)
    assert dd.eels_padded_dims(ctx) == (64, 36, 36)
    ang = np.linspace(0.0, 2.0 * np.pi, 32, endpoint=False)
    beams = np.stack([24.0 * np.cos(ang), 24.0 * np.sin(ang)], axis=1)
    o = dd.eels_default_opts(ekin_keV=100.0, precision=dd.EELS_MIXED, eps_it=1e-10)
    eps_p, eps_h = [[I.drude(e_eV)]], [2.1025]
    res = dd.eels_solve(ctx, o, [e_eV], eps_p, eps_h, beams, want_p=True)
    assert res.converged.all()
    pts = [run.setup(n, n, n, d_nm, occ, e_eV, eps_p[0], eps_h[0], beams[ib], ekin_keV=100.0) for ib in (0, 7, 16, 31)]
    A = green.dense_matrix(pts[0].r, pts[0].k, pts[0].alpha)
    for ib, pt in zip((0, 7, 16, 31), pts):
        p_t = np.linalg.solve(A, pt.E_inc.reshape(-1)).reshape(-1, 3)
        ref = run.observables(pt, p_t)
        for key, got in (("P_EELS", res.p_eels), ("P_CL", res.p_cl), ("P_ext", res.p_ext), ("P_abs", res.p_abs)):
            assert abs(got[0, ib] - ref[key]) <= 1e-4 * abs(ref[key]), (key, ib, got[0, ib], ref[key])
        assert rel(res.p[0, ib], run.p_si(pt, p_t)) < 1e-4
    for ib in (3, 16):
        solo = dd.eels_solve(ctx, o, [e_eV], eps_p, eps_h, beams[ib:ib + 1], want_p=True)
        assert solo.p_eels[0, 0] == res.p_eels[0, ib] and solo.p_cl[0, 0] == res.p_cl[0, ib]
        assert np.array_equal(solo.p[0, 0], res.p[0, ib])


def test_batch_composition_does_not_change_results(dd, ctx):
    """A point solved alone and inside a larger batch gives identical bits."""
    w = I.reduced(I.config_spectrum(), 10 / 32, n_energy=4)
    full = _solve(dd, ctx, w, dd.EELS_MIXED, want_p=False, eps=1e-8)
    alone = _solve(dd, ctx, w, dd.EELS_MIXED, energies=[2], want_p=False, eps=1e-8)
    split = _solve(dd, ctx, w, dd.EELS_MIXED, want_p=False, eps=1e-8, max_batch=1)
    assert full.p_eels[2, 0] == alone.p_eels[0, 0]
    assert full.p_cl[2, 0] == alone.p_cl[0, 0]
    assert np.array_equal(full.p_eels, split.p_eels)


def test_single_dipole_and_ragged_lattice(dd, ctx):
    occ = np.ones((1, 1, 1), dtype=np.uint8)
    w = I.Workload("one", I.Grid(1, 1, 1, 4.0, occ), 100.0, np.array([2.2]), I.drude(np.array([2.2]))[:, None],
                   np.array([2.1025 + 0j]), np.array([[10.0, 0.0]]))
    res = _solve(dd, ctx, w, dd.EELS_FP64, eps=1e-13)
    _check_point(res, 0, 0, _oracle(w, 0, 0), 1e-10, 1e-10)
    occ = _random_grid((5, 7, 3), seed=3)
    w2 = I.Workload("ragged", I.Grid(5, 7, 3, 1.5, occ), 150.0, np.array([1.9, 3.3]),
                    I.drude(np.array([1.9, 3.3]), I.DRUDE_AG)[:, None], np.array([1.7 + 0j, 1.7 + 0j]),
                    np.array([[9.0, 2.0], [-1.0, 8.0]]))
    res = _solve(dd, ctx, w2, dd.EELS_FP64, eps=1e-12)
    for ie in range(2):
        for ib in range(2):
            _check_point(res, ie, ib, _oracle(w2, ie, ib), 1e-10, 1e-10)


def test_invalid_inputs_raise(dd, ctx):
    w = I.config_small_sphere()
    g = w.grid
    dd.eels_set_grid(ctx, g.occ, g.d_nm)
    o = dd.eels_default_opts(ekin_keV=100.0)
    with pytest.raises(dd.EelsError) as e:        # beam through the particle
        dd.eels_solve(ctx, o, [2.4], [[I.drude(2.4)]], [1.0], [[0.3, 0.2]])
    assert e.value.code == dd.EELS_E_BEAM_INSIDE
    with pytest.raises(dd.EelsError) as e:        # active host
        dd.eels_solve(ctx, o, [2.4], [[I.drude(2.4)]], [1.0 - 0.1j], [[15.0, 0.0]])
    assert e.value.code == dd.EELS_E_INVALID_ARG
    from oracle.physics import electron_speed
    from oracle.constants import C_LIGHT
    m = C_LIGHT / electron_speed(100.0)
    with pytest.raises(dd.EelsError) as e:        # exactly at the Cherenkov threshold
        dd.eels_solve(ctx, o, [2.4], [[I.drude(2.4)]], [m * m], [[15.0, 0.0]])
    assert e.value.code == dd.EELS_E_THRESHOLD
    with pytest.raises(dd.EelsError) as e:
        dd.eels_set_grid(ctx, np.zeros((3, 3, 3), np.uint8), 1.0)
    assert e.value.code == dd.EELS_E_INVALID_ARG


@pytest.mark.parametrize("solver", ["BICGSTAB", "QMR"])
@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_other_solvers_match_lu(dd, ctx, prec, solver):
    """The BiCGStab and three-term QMR inner solvers reach the same solution
    as LU (Cherenkov absorbing host replica, 3 energies, and the small gold
    sphere); the default two-term QMR is covered by every other solve."""
    for w in (I.reduced(I.config_cherenkov(), 12 / 64, n_energy=3), I.config_small_sphere()):
        g = w.grid
        dd.eels_set_grid(ctx, g.occ, g.d_nm)
        o = dd.eels_default_opts(ekin_keV=w.ekin_keV, precision=getattr(dd, "EELS_" + prec), solver=getattr(dd, "EELS_" + solver),
                                 eps_it=1e-12 if prec == "FP64" else 1e-8)
        res = dd.eels_solve(ctx, o, w.energies_eV, w.eps_p, w.eps_h, w.beams_nm, want_p=True)
        assert res.converged.all()
        tol = 1e-10 if prec == "FP64" else 1e-4
        for ie in range(len(w.energies_eV)):
            _check_point(res, ie, 0, _oracle(w, ie, 0), tol, tol)


def test_async_solve_matches_blocking_solve(dd, ctx):
    """eels_solve_async gives the same bits as eels_solve on the same context."""
    w = I.reduced(I.config_spectrum(), 10 / 32, n_energy=3)
    ref = _solve(dd, ctx, w, dd.EELS_MIXED, want_p=True, eps=1e-8)
    o = dd.eels_default_opts(ekin_keV=w.ekin_keV, precision=dd.EELS_MIXED, eps_it=1e-8)
    job = dd.eels_solve_async(ctx, o, w.energies_eV, w.eps_p, w.eps_h, w.beams_nm, want_p=True)
    import time
    t_end = time.time() + 120.0
    while not job.poll() and time.time() < t_end:
        time.sleep(0.01)
    res = job.wait()
    for a, b in ((res.p_eels, ref.p_eels), (res.p_cl, ref.p_cl), (res.p_ext, ref.p_ext), (res.p, ref.p)):
        assert np.array_equal(a, b)



@pytest.mark.parametrize("direction,origin,shift", [
    ((0.0, 0.0, 1.0), (3.0, -2.0, 5.0), True),      # z electron: beams shift by (ox, oy), phase by oz
    ((1.0, 1.0, 1.0), (4.0, 4.0, 4.0), False),      # origin along the direction: phase only
])
def test_grid_origin_translates_the_beams(dd, ctx, direction, origin, shift):
    """A lattice centred at origin_nm is the centred lattice with every
    trajectory moved by -origin_nm: the same probabilities, and dipole moments
    times exp(i w s / v), s the move of the phase reference point along the
    electron (FP64 path; LU-checked centred solves elsewhere pin the rest)."""
    from oracle import physics
    w = I.reduced(I.config_spectrum(), 10 / 32, n_energy=2)
    o = dd.eels_default_opts(ekin_keV=w.ekin_keV, precision=dd.EELS_FP64, eps_it=1e-10, n_dir=162,
                             beam_dir=direction)
    beams = np.asarray(w.beams_nm, dtype=float)
    org = np.asarray(origin)
    dd.eels_set_grid(ctx, w.grid.occ, w.grid.d_nm, origin_nm=origin)
    moved = dd.eels_solve(ctx, o, w.energies_eV, w.eps_p, w.eps_h, beams + (org[:2] if shift else 0.0),
                          want_p=True)
    dd.eels_set_grid(ctx, w.grid.occ, w.grid.d_nm)
    ref = dd.eels_solve(ctx, o, w.energies_eV, w.eps_p, w.eps_h, beams, want_p=True)
    for a, b in ((moved.p_eels, ref.p_eels), (moved.p_cl, ref.p_cl), (moved.p_ext, ref.p_ext),
                 (moved.p_abs, ref.p_abs)):
        assert np.allclose(a, b, rtol=1e-9, atol=0)
    n = np.asarray(direction) / np.linalg.norm(direction)
    s_m = float(org @ n) * 1e-9
    v = physics.electron_speed(w.ekin_keV)
    for e, E in enumerate(w.energies_eV):
        ph = np.exp(1j * physics.omega_of(E) * s_m / v)
        pm, pr = moved.p[e], ref.p[e]
        assert np.linalg.norm(pm - ph * pr) <= 1e-8 * np.linalg.norm(pr)


@pytest.mark.parametrize("solver", ["QMR2", "QMR", "BICGSTAB"])
def test_device_loop_matches_host_loop(dd, ctx, solver):
    """Inner solves as one graph launch with a WHILE node (device_loop = 1)
    give the same bits as host-driven bursts of graph replays: systems that
    have converged stop changing, so where the loop ends does not matter.
    FP32 rounds (padded grid above the FP64-inner size) and FP64 solves."""
    nx, ny, nz, d_nm = 16, 16, 36, 1.5
    dd.eels_set_grid(ctx, I.box_occupancy(nx, ny, nz), d_nm)
    e = np.array([1.9, 2.6, 3.2])
    eps_p = I.drude(e)[:, None]
    eps_h = np.full(3, 2.1025 + 0j)
    beams = np.array([[nx * d_nm / 2 + 6.0, 0.0], [nx * d_nm / 2 + 9.0, 3.0]])
    for prec in (dd.EELS_MIXED, dd.EELS_FP64):
        res = []
        for loop in (0, 1):
            o = dd.eels_default_opts(ekin_keV=100.0, precision=prec, eps_it=1e-8,
                                     solver=getattr(dd, "EELS_" + solver), n_dir=162, device_loop=loop)
            r = dd.eels_solve(ctx, o, e, eps_p, eps_h, beams, want_p=True, want_cl=True)
            assert r.converged.all()
            res.append(r)
        for a, b in ((res[0].p_eels, res[1].p_eels), (res[0].p_cl, res[1].p_cl), (res[0].p_ext, res[1].p_ext),
                     (res[0].p, res[1].p), (res[0].residual, res[1].residual)):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("solver", ["QMR2", "QMR"])
def test_mixed_fp32_rounds_match_oracle_above_fp64_threshold(dd, ctx, solver):
    """A lattice whose padded grid (32 x 32 x 72) is above the size where the
    mixed path switches to FP64 inner solves, so FP32 QMR rounds with FP64
    refinement run (two-term and three-term QMR); the oracle solves the same
    points with its own FFT operator and GMRES."""
    nx, ny, nz, d_nm = 16, 16, 36, 1.5
    occ = I.box_occupancy(nx, ny, nz)
    dd.eels_set_grid(ctx, occ, d_nm)
    assert np.prod(dd.eels_padded_dims(ctx)) > 65536
    e = np.array([2.6, 3.2])          # where the oracle's GMRES is quick
    eps_p = I.drude(e)[:, None]
    eps_h = np.full(2, 2.1025 + 0j)
    beam = np.array([[nx * d_nm / 2 + 6.0, 0.0]])
    o = dd.eels_default_opts(ekin_keV=100.0, precision=dd.EELS_MIXED, eps_it=1e-8,
                             solver=getattr(dd, "EELS_" + solver))
    res = dd.eels_solve(ctx, o, e, eps_p, eps_h, beam)
    assert res.converged.all()
    for ie in range(2):
        ref = run.solve_point(nx, ny, nz, d_nm, occ, e[ie], eps_p[ie], eps_h[ie], beam[0], ekin_keV=100.0,
                              method="fft", rtol=1e-11)
        for key, got in (("P_EELS", res.p_eels), ("P_CL", res.p_cl), ("P_ext", res.p_ext), ("P_abs", res.p_abs)):
            assert abs(got[ie, 0] - ref[key]) <= 1e-4 * abs(ref[key]), (key, got[ie, 0], ref[key])


@pytest.mark.parametrize("dims", [(13, 9, 11), (20, 9, 16), (40, 6, 8)])
def test_tile_autotuning_keeps_matvec_bits(dd, dims):
    """The first solve on a grid times the x-pass tile widths (and, for x
    lengths 64 and 128, how U moves and how many systems a block takes);
    matvecs before and after the choice are bit-identical (the choices only
    regroup the same arithmetic), and setting a grid of the same shape again
    restores the choices and their timings instead of timing again."""
    ctx = dd.eels_create(0)
    try:
        _autotuning_case(dd, ctx, dims)
    finally:
        dd.eels_destroy(ctx)


def _autotuning_case(dd, ctx, dims):
    occ = _random_grid(dims, seed=21, nmat=2)
    dd.eels_set_grid(ctx, occ, 1.7)
    assert dd.eels_tile_widths(ctx) == (0, 0)
    assert dd.eels_tuned_xpass(ctx) == (0, 0)
    assert dd.eels_xpass_timings(ctx) == []
    eps_p, eps_h = [I.drude(2.2), 2.0 + 0.5j], 1.9 + 0j
    x = I.random_complex((2, dd.eels_num_dipoles(ctx), 3), seed=8)
    y_before = [dd.eels_apply_matrix(ctx, pr, 2.2, eps_p, eps_h, x) for pr in (dd.EELS_FP64, dd.EELS_MIXED)]
    o = dd.eels_default_opts(ekin_keV=100.0, eps_it=1e-6)
    dd.eels_solve(ctx, o, [2.2, 2.9], [eps_p, eps_p], [eps_h, eps_h], [[50.0, 0.0]])
    w32, w64 = dd.eels_tile_widths(ctx)
    assert w32 in (8, 16, 32) and w64 in (8, 16, 32)
    mode, spb = dd.eels_tuned_xpass(ctx)
    timings = dd.eels_xpass_timings(ctx)
    if dd.eels_padded_dims(ctx)[0] in (64, 128):
        assert mode in (1, 2) and spb == 1
        assert timings and all(t[2] > 0 for t in timings)
        best = min(timings, key=lambda t: t[2])
        assert (best[0], best[1]) == (mode, spb)
    else:
        assert (mode, spb) == (0, 0) and timings == []
    y_after = [dd.eels_apply_matrix(ctx, pr, 2.2, eps_p, eps_h, x) for pr in (dd.EELS_FP64, dd.EELS_MIXED)]
    for a, b in zip(y_before, y_after):
        assert np.array_equal(a, b)
    dd.eels_set_grid(ctx, occ, 1.7)
    assert dd.eels_tile_widths(ctx) == (w32, w64)
    assert dd.eels_tuned_xpass(ctx) == (mode, spb)
    assert dd.eels_xpass_timings(ctx) == timings


# ------------------------------------------------------------------ electron direction
@pytest.mark.parametrize("direction,eps_h", [((1.0, 2.0, 2.0), 2.1025), ((0.0, 0.0, -1.0), 4.0 + 0.05j),
                                             ((1.0, 0.0, 0.0), 1.0), ((0.3, -0.2, 0.9), 4.0)])
def test_incident_field_along_a_direction(dd, ctx, direction, eps_h):
    w = I.config_small_sphere()
    g = w.grid
    dd.eels_set_grid(ctx, g.occ, g.d_nm)
    beam = (16.0, 3.0)
    E, Ea = dd.eels_incident_field(ctx, 150.0, 2.6, eps_h, beam, beam_dir=direction)
    pt = run.setup(g.nx, g.ny, g.nz, g.d_nm, g.occ, 2.6, [1.0], eps_h, beam, ekin_keV=150.0, direction=direction)
    assert rel(E, pt.E_inc) < 1e-12
    assert rel(Ea, pt.E_a) < 1e-12


def test_oblique_electron_solves_match_lu_and_rotations_agree(dd, ctx):
    """An electron along (1, 1, 1) against the oracle's LU solve (FP64 and
    mixed), and electrons along x and z with the same (x0, y0) past the
    lattice sphere give the same probabilities (a quarter turn maps one onto
    the other); an oblique line through the particle is refused."""
    w = I.config_small_sphere()
    g = w.grid
    dd.eels_set_grid(ctx, g.occ, g.d_nm)
    beam = np.array([[15.0, 2.0]])
    for prec, eps, tol in ((dd.EELS_FP64, 1e-12, 1e-10), (dd.EELS_MIXED, 1e-8, 1e-4)):
        o = dd.eels_default_opts(ekin_keV=100.0, precision=prec, eps_it=eps, beam_dir=(1.0, 1.0, 1.0))
        res = dd.eels_solve(ctx, o, w.energies_eV, w.eps_p, w.eps_h, beam, want_p=True)
        ref = run.solve_point(g.nx, g.ny, g.nz, g.d_nm, g.occ, w.energies_eV[0], w.eps_p[0], w.eps_h[0], beam[0],
                              ekin_keV=100.0, direction=(1.0, 1.0, 1.0))
        _check_point(res, 0, 0, ref, tol, tol)
    out = {}
    for n in ((0.0, 0.0, 1.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0)):
        o = dd.eels_default_opts(ekin_keV=100.0, precision=dd.EELS_FP64, eps_it=1e-12, beam_dir=n)
        out[n] = dd.eels_solve(ctx, o, w.energies_eV, w.eps_p, w.eps_h, beam)
    for n in ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0)):
        for a, b in ((out[n].p_eels, out[(0.0, 0.0, 1.0)].p_eels), (out[n].p_cl, out[(0.0, 0.0, 1.0)].p_cl)):
            assert np.allclose(a, b, rtol=1e-9, atol=0)
    o = dd.eels_default_opts(ekin_keV=100.0, beam_dir=(1.0, 1.0, 0.0))
    with pytest.raises(dd.EelsError) as e:
        dd.eels_solve(ctx, o, w.energies_eV, w.eps_p, w.eps_h, [[0.0, 1.0]])
    assert e.value.code == dd.EELS_E_BEAM_INSIDE


def test_vacuum_equivalent_problems_reproduce_host_probabilities(dd, ctx):
    """Sec. 2.7 through the library: a gold sphere in glass (eps_h = 2.1025)
    and the vacuum problems eels_vacuum_equivalent gives for it (Eq. 45:
    loss energy times m_h; Eq. 46: lengths times m_h, probabilities / m_h)
    give the same probabilities; the host solve itself matches the oracle's
    LU solve."""
    w = I.config_small_sphere()
    g = w.grid
    eps_h, ek = 2.1025, 100.0
    energies = np.array([1.9, 2.4])
    eps_p = np.array([[I.drude(e)] for e in energies])
    beam = np.array([[15.0, 2.0]])
    opts = dict(precision=dd.EELS_FP64, eps_it=1e-12)
    dd.eels_set_grid(ctx, g.occ, g.d_nm)
    host = dd.eels_solve(ctx, dd.eels_default_opts(ekin_keV=ek, **opts), energies, eps_p,
                         np.full(len(energies), eps_h, dtype=complex), beam)
    assert host.converged.all()
    ref = run.solve_point(g.nx, g.ny, g.nz, g.d_nm, g.occ, energies[1], eps_p[1], eps_h, beam[0], ekin_keV=ek)
    for key, got in (("P_EELS", host.p_eels), ("P_CL", host.p_cl)):
        assert abs(got[1, 0] - ref[key]) <= 1e-10 * abs(ref[key]), key
    for rule in (dd.EELS_SCALE_ENERGY, dd.EELS_SCALE_LENGTH):
        maps = [dd.eels_vacuum_equivalent(ek, eps_h, e, rule) for e in energies]
        s = maps[0]["length_scale"]
        dd.eels_set_grid(ctx, g.occ, g.d_nm * s)
        vac = dd.eels_solve(ctx, dd.eels_default_opts(ekin_keV=maps[0]["ekin_keV"], **opts),
                            np.array([m["energy_eV"] for m in maps]), eps_p * maps[0]["eps_p_scale"],
                            np.ones(len(energies), dtype=complex), beam * s)
        assert vac.converged.all()
        for a, b in ((vac.p_eels, host.p_eels), (vac.p_cl, host.p_cl), (vac.p_ext, host.p_ext),
                     (vac.p_abs, host.p_abs)):
            assert np.allclose(maps[0]["p_scale"] * a, b, rtol=1e-9, atol=0), rule


# ------------------------------------------------------------------ Krylov solve on the prepared operator
def _scaled_operator(pt):
    """A' = a^1/2 (alpha~^-1 - G~) a^1/2 d^3 with a = alpha~ / d^3 (lattice units),
    the operator eels_prepare_operator sets up, in the oracle's dipole order."""
    A = green.dense_matrix(pt.r, pt.k, pt.alpha)
    sa = np.repeat(np.sqrt(pt.alpha / pt.d ** 3), 3)
    return sa[:, None] * A * sa[None, :] * pt.d ** 3


def _internal_perm(pt):
    """internal dipole i (cells sorted by ix, iy, iz) -> oracle dipole (x-fastest order)."""
    idx = pt.idx
    return np.lexsort((idx[:, 2], idx[:, 1], idx[:, 0]))


def _to_internal(v, perm):       # [N][3] oracle order -> [3][N] internal order
    return np.ascontiguousarray(v[perm].T)


def _from_internal(v, perm):     # [3][N] internal -> [N][3] oracle order
    out = np.empty((v.shape[1], 3), dtype=v.dtype)
    out[perm] = v.T
    return out


@pytest.mark.parametrize("solver", ["QMR2", "QMR", "BICGSTAB"])
@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_krylov_solve_dev_matches_dense_solve(dd, ctx, solver, prec):
    """eels_krylov_solve_dev on the prepared operator against LU of the same
    Jacobi-scaled matrix (oracle dense assembly), for a random right-hand side."""
    import torch
    dims = (6, 5, 7)
    occ = _random_grid(dims, seed=41, nmat=2)
    d_nm, e_eV = 2.0, 2.3
    eps_p, eps_h = [I.drude(e_eV), 3.0 + 0.4j], 2.0 + 0.1j
    dd.eels_set_grid(ctx, occ, d_nm)
    dd.eels_prepare_operator(ctx, [e_eV], [eps_p], [eps_h])
    pt = run.setup(*dims, d_nm, occ, e_eV, eps_p, eps_h, (100.0, 100.0), ekin_keV=100.0)
    perm = _internal_perm(pt)
    b = I.random_complex((len(pt.r), 3), seed=17)
    ref = np.linalg.solve(_scaled_operator(pt), b.reshape(-1)).reshape(-1, 3)
    dt = torch.complex128 if prec == "FP64" else torch.complex64
    bt = torch.from_numpy(_to_internal(b, perm)).to(dt).cuda()
    xt = torch.zeros_like(bt)
    eps = 1e-12 if prec == "FP64" else 1e-6
    status, iters = dd.eels_krylov_solve_dev(ctx, getattr(dd, "EELS_" + prec), getattr(dd, "EELS_" + solver),
                                             bt.data_ptr(), xt.data_ptr(), 1, eps, 5000,
                                             torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert status[0] == 1 and iters[0] > 0
    x = _from_internal(xt.cpu().numpy().astype(np.complex128), perm)
    assert rel(x, ref) < (1e-9 if prec == "FP64" else 1e-4)


@pytest.mark.parametrize("solver", ["QMR2", "QMR"])
@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_qmr_reports_breakdown_when_b_transpose_b_vanishes(dd, ctx, solver, prec):
    """b = u + i w with u orthogonal to w and |u| = |w| has b^T b = 0: the
    complex-symmetric Lanczos process breaks down at its start.  The solver
    must report a breakdown (status 3) with x = 0, not a convergence."""
    import torch
    dims = (6, 5, 7)
    occ = _random_grid(dims, seed=41, nmat=2)
    d_nm, e_eV = 2.0, 2.3
    eps_p, eps_h = [I.drude(e_eV), 3.0 + 0.4j], 2.0 + 0.1j
    dd.eels_set_grid(ctx, occ, d_nm)
    dd.eels_prepare_operator(ctx, [e_eV], [eps_p], [eps_h])
    n = dd.eels_num_dipoles(ctx)
    rng = np.random.default_rng(5)
    u = rng.standard_normal(3 * n)
    w = rng.standard_normal(3 * n)
    w -= (w @ u) / (u @ u) * u
    w *= np.linalg.norm(u) / np.linalg.norm(w)
    b = (u + 1j * w).reshape(3, n)
    assert abs(np.sum(b * b)) < 1e-12 * np.sum(np.abs(b) ** 2)
    dt = torch.complex128 if prec == "FP64" else torch.complex64
    bt = torch.from_numpy(b).to(dt).cuda()
    xt = torch.full_like(bt, 7.0)
    status, iters = dd.eels_krylov_solve_dev(ctx, getattr(dd, "EELS_" + prec), getattr(dd, "EELS_" + solver),
                                             bt.data_ptr(), xt.data_ptr(), 1, 1e-6, 100,
                                             torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert status[0] == 3 and iters[0] == 1
    assert torch.count_nonzero(xt).item() == 0


# ------------------------------------------------------------------ device-buffer solve
def test_solve_dev_is_bit_identical_to_host_solve(dd, ctx):
    """eels_solve_dev with torch device buffers and the current stream gives
    the same bits as eels_solve with host buffers."""
    import ctypes
    import torch
    w = I.config_small_sphere()
    g = w.grid
    dd.eels_set_grid(ctx, g.occ, g.d_nm)
    energies = np.array([2.0, 2.4, 2.9])
    eps_p = np.array([[I.drude(e)] for e in energies])
    eps_h = np.full(len(energies), 1.0 + 0j)
    beams = np.array([[15.0, 0.0], [0.0, 13.0]])
    o = dd.eels_default_opts(ekin_keV=w.ekin_keV, eps_it=1e-8)
    host = dd.eels_solve(ctx, o, energies, eps_p, eps_h, beams, want_p=True)
    dev = dict(device="cuda")
    ne, nb, n = len(energies), len(beams), dd.eels_num_dipoles(ctx)
    et = torch.tensor(energies, dtype=torch.float64, **dev)
    ept = torch.tensor(eps_p, dtype=torch.complex128, **dev)
    eht = torch.tensor(eps_h, dtype=torch.complex128, **dev)
    bt = torch.tensor(beams, dtype=torch.float64, **dev)
    out = {k: torch.zeros(ne, nb, dtype=torch.float64, **dev) for k in ("eels", "cl", "ext", "abs")}
    pt = torch.zeros(ne, nb, n, 3, dtype=torch.complex128, **dev)
    st = torch.zeros(ne * nb * ctypes.sizeof(dd.eels_point_stats), dtype=torch.uint8, **dev)
    code = dd.eels_solve_dev(ctx, o, et, ept, eht, bt, out["eels"], out["cl"], out["ext"], out["abs"], pt, st,
                             stream=torch.cuda.current_stream().cuda_stream)
    assert code == dd.EELS_OK
    assert np.array_equal(out["eels"].cpu().numpy(), host.p_eels)
    assert np.array_equal(out["cl"].cpu().numpy(), host.p_cl)
    assert np.array_equal(out["ext"].cpu().numpy(), host.p_ext)
    assert np.array_equal(out["abs"].cpu().numpy(), host.p_abs)
    assert np.array_equal(pt.cpu().numpy(), host.p)
    sts = (dd.eels_point_stats * (ne * nb)).from_buffer_copy(st.cpu().numpy().tobytes())
    assert [s.iters for s in sts] == host.iters.ravel().tolist()
    # a host buffer where device memory is required is refused before any work
    with pytest.raises(dd.EelsError) as e:
        dd.eels_solve_dev(ctx, o, et.cpu(), ept, eht, bt, out["eels"])
    assert e.value.code == dd.EELS_E_INVALID_ARG


# ------------------------------------------------------------------ several materials, extrapolation
@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_three_material_particle_solve_matches_lu(dd, ctx, prec):
    """A 12^3 sphere of three concentric materials (Drude gold core, a
    dielectric shell, Drude silver outside) in glass: every probability and
    p against the oracle's LU solve."""
    n, diam = 12, 24.0
    c = ((np.arange(n) + 0.5) - n / 2.0) * (diam / n)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    rr = np.sqrt(x * x + y * y + z * z)
    occ = np.where(rr <= 5.0, 1, np.where(rr <= 8.0, 2, np.where(rr <= diam / 2, 3, 0))).astype(np.uint8)
    assert set(np.unique(occ)) == {0, 1, 2, 3}
    e_eV = 2.6
    eps_p = [I.drude(e_eV), 2.25 + 0.1j, I.drude(e_eV, I.DRUDE_AG)]
    eps_h, beam = 2.1025, (18.0, 3.0)
    dd.eels_set_grid(ctx, occ, diam / n)
    o = dd.eels_default_opts(ekin_keV=120.0, precision=getattr(dd, "EELS_" + prec), eps_it=1e-12 if prec == "FP64" else 1e-9)
    res = dd.eels_solve(ctx, o, [e_eV], [eps_p], [eps_h], [beam], want_p=True)
    ref = run.solve_point(n, n, n, diam / n, occ, e_eV, eps_p, eps_h, beam, ekin_keV=120.0)
    tol = 1e-10 if prec == "FP64" else 1e-4
    for key, got in (("P_EELS", res.p_eels), ("P_CL", res.p_cl), ("P_ext", res.p_ext), ("P_abs", res.p_abs)):
        assert abs(got[0, 0] - ref[key]) <= tol * abs(ref[key]), (key, got[0, 0], ref[key])
    assert rel(res.p[0, 0], ref["p"]) < tol


def test_library_extrapolation_to_zero_dipole_size_matches_oracle_and_mie(dd, ctx):
    """Sec. 3.2 through the library: a 20 nm absorbing dielectric sphere in
    vacuum on nine volume-corrected lattices (10^3 to 32^3 cells), each solved
    on the GPU (FP64) and by the oracle, extrapolated to d = 0 with
    eels_extrapolate: per-lattice and extrapolated values agree with the
    oracle's, and the extrapolated P_EELS and P_CL lie within their 95 %
    intervals of the Lorenz-Mie solution."""
    from oracle import mie_eels, physics
    from oracle.extrapolate import extrapolate_to_zero
    ek, diam, b, e_eV, eps_p, eps_h = 100.0, 20.0, 25.0, 2.5, 2.25 + 0.5j, 1.0
    coef = mie_eels.electron_coefficients(eps_h, e_eV, b * NM, physics.electron_speed(ek), 16, 17.5 * NM)
    exact = mie_eels.eels_cl_from(coef, diam / 2 * NM, eps_p, eps_h)
    ds, gpu, ora = [], [], []
    o = dd.eels_default_opts(ekin_keV=ek, precision=dd.EELS_FP64, eps_it=1e-11)
    for n in (10, 12, 14, 16, 18, 20, 24, 28, 32):
        occ = I.sphere_occupancy(n, diam)
        d = (np.pi * diam ** 3 / 6 / int(occ.sum())) ** (1 / 3)
        dd.eels_set_grid(ctx, occ, d)
        r = dd.eels_solve(ctx, o, [e_eV], [[eps_p]], [eps_h], [(b, 0.0)])
        ref = run.solve_point(n, n, n, d, occ, e_eV, [eps_p], eps_h, (b, 0.0), ekin_keV=ek, method="fft", rtol=1e-11)
        ds.append(d)
        gpu.append((r.p_eels[0, 0], r.p_cl[0, 0]))
        ora.append((ref["P_EELS"], ref["P_CL"]))
    for j in (0, 1):
        g = np.array([v[j] for v in gpu])
        y = np.array([v[j] for v in ora])
        assert np.max(np.abs(g - y) / np.abs(y)) < 1e-8
        v0, ci = dd.eels_extrapolate(ds, g)
        r0, rci = extrapolate_to_zero(np.array(ds), y)
        assert abs(v0 - r0) <= 1e-7 * abs(r0) and abs(ci - rci) <= 1e-5 * rci
        assert abs(v0 - exact[j]) <= ci, (j, v0 / exact[j] - 1, ci / exact[j])


# ------------------------------------------------------------------ igt_so (Sec. S5)
@pytest.mark.parametrize("dims", [(5, 4, 6), (7, 3, 9), (32, 3, 8), (13, 6, 17)])
def test_igt_so_matvec_equals_dense_oracle(dd, ctx, dims):
    """The cell-integrated interaction and polarizability (igt_so) through
    eels_apply_matrix, FP64 and FP32, against the oracle's dense matrix."""
    nx, ny, nz = dims
    occ = _random_grid(dims, seed=nx + 3 * ny + 7 * nz, nmat=2)
    d_nm, e_eV = 2.0, 2.3
    eps_p, eps_h = [I.drude(e_eV), 3.0 + 0.4j], 2.0 + 0.1j
    dd.eels_set_grid(ctx, occ, d_nm)
    dd.eels_set_interaction(ctx, dd.EELS_INT_IGT_SO, dd.EELS_POL_IGT_SO)
    try:
        pt = run.setup(nx, ny, nz, d_nm, occ, e_eV, eps_p, eps_h, (100.0, 100.0), ekin_keV=100.0,
                       interaction="igt_so", polarizability="igt_so")
        A = run.system_matrix(pt)
        x = I.random_complex((2, len(pt.r), 3), seed=9)
        ref = np.stack([(A @ xi.reshape(-1)).reshape(-1, 3) for xi in x])
        y64 = dd.eels_apply_matrix(ctx, dd.EELS_FP64, e_eV, eps_p, eps_h, x)
        y32 = dd.eels_apply_matrix(ctx, dd.EELS_MIXED, e_eV, eps_p, eps_h, x)
    finally:
        dd.eels_set_interaction(ctx, dd.EELS_INT_POINT, dd.EELS_POL_CM)
    for i in range(2):
        assert rel(y64[i], ref[i]) < 1e-12
        assert rel(y32[i], ref[i]) < 2e-5


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_igt_so_solve_matches_lu(dd, ctx, prec):
    """A 12^3 high-index sphere (eps = 15 + i) in glass with the igt_so
    interaction and polarizability: probabilities and p against the oracle's
    LU solve of the same model."""
    w = I.config_small_sphere()
    g = w.grid
    e_eV, eps_p, eps_h, beam = 2.5, 15.0 + 1.0j, 2.1025, (16.0, 2.0)
    dd.eels_set_grid(ctx, g.occ, g.d_nm)
    o = dd.eels_default_opts(ekin_keV=120.0, precision=getattr(dd, "EELS_" + prec),
                             eps_it=1e-12 if prec == "FP64" else 1e-9,
                             interaction=dd.EELS_INT_IGT_SO, polarizability=dd.EELS_POL_IGT_SO)
    res = dd.eels_solve(ctx, o, [e_eV], [[eps_p]], [eps_h], [beam], want_p=True)
    ref = run.solve_point(g.nx, g.ny, g.nz, g.d_nm, g.occ, e_eV, [eps_p], eps_h, beam, ekin_keV=120.0,
                          interaction="igt_so", polarizability="igt_so")
    pnt = run.solve_point(g.nx, g.ny, g.nz, g.d_nm, g.occ, e_eV, [eps_p], eps_h, beam, ekin_keV=120.0)
    tol = 1e-10 if prec == "FP64" else 1e-4
    for key, got in (("P_EELS", res.p_eels), ("P_CL", res.p_cl), ("P_ext", res.p_ext), ("P_abs", res.p_abs)):
        assert abs(got[0, 0] - ref[key]) <= tol * abs(ref[key]), (key, got[0, 0], ref[key])
    assert rel(res.p[0, 0], ref["p"]) < tol
    # the model differs from point dipoles by far more than the tolerance
    assert abs(pnt["P_EELS"] / ref["P_EELS"] - 1.0) > 1e-3
