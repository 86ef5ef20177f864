"""Parity at the workloads' full sizes, in the launch configuration bench.py
uses (mixed path, eps_it 1e-8, inner 1e-5 restarted every 2000 iterations).

At these sizes a dense oracle solve is out of reach, so each sampled point is
checked by the oracle in two independent ways:
  * residual certificate: the oracle's own FP64 FFT operator (period 2N,
    scipy.fft) evaluates the relative residual of the Jacobi-scaled system at
    the GPU dipoles, ||a^1/2 (E_inc - A p)|| / ||a^1/2 E_inc||;
  * the oracle recomputes P_EELS, P_ext, P_abs (Eq. 32, 17, 18) and P_CL
    (Eq. 42) from the GPU dipoles with its own incident field.
Where the oracle's Krylov solve is cheap (high loss energies) it also solves
the point itself and the probabilities are compared directly (1e-4)."""
import numpy as np
import pytest

from oracle import green, run
from oracle.constants import EPS0
from paper_2208_01348_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2208_01348_gb300 import eelsdda
    return eelsdda


def _gpu(dd, w, ie, beams=None, precision=None):
    ctx = dd.eels_create(0)
    try:
        g = w.grid
        dd.eels_set_grid(ctx, g.occ, g.d_nm)
        o = dd.eels_default_opts(ekin_keV=w.ekin_keV, eps_it=1e-8, eps_inner=1e-5,
                                 precision=dd.EELS_MIXED if precision is None else precision)
        bm = w.beams_nm if beams is None else beams
        return dd.eels_solve(ctx, o, w.energies_eV[ie], w.eps_p[ie], w.eps_h[ie], bm, want_p=True)
    finally:
        dd.eels_destroy(ctx)


def _certify(w, ie, ib, res, k, beams=None, p_tol=1e-10, cl_tol=1e-5):
    """Residual and observables of GPU point (k, ib) with the oracle's operator."""
    g = w.grid
    bm = w.beams_nm if beams is None else beams
    pt = run.setup(g.nx, g.ny, g.nz, g.d_nm, g.occ, w.energies_eV[ie], w.eps_p[ie], w.eps_h[ie], bm[ib],
                   ekin_keV=w.ekin_keV)
    op = green.FFTOperator(pt.idx, pt.n_axes, pt.d, pt.k, pt.alpha)
    p_t = res.p[k, ib] / (4 * np.pi * EPS0 * pt.eps_h)
    sa = np.sqrt(pt.alpha)[:, None]
    r = sa * (pt.E_inc - op.matvec(p_t))
    rel = np.linalg.norm(r) / np.linalg.norm(sa * pt.E_inc)
    assert rel <= 2e-8, rel
    obs = run.observables(pt, p_t)
    for key, got, tol in (("P_EELS", res.p_eels, p_tol), ("P_ext", res.p_ext, p_tol), ("P_abs", res.p_abs, p_tol),
                          ("P_CL", res.p_cl, cl_tol)):
        assert abs(got[k, ib] - obs[key]) <= tol * abs(obs[key]), (key, got[k, ib], obs[key])
    return pt, op


def test_spectrum_full_size_certified_across_the_spectrum(dd):
    """32^3 sphere (17,256 dipoles, 64^3 FFT): low, resonant and high energies."""
    w = I.config_spectrum()
    ie = np.array([0, 60, 100, 199])
    res = _gpu(dd, w, ie)
    assert res.converged.all()
    for k, e in enumerate(ie):
        _certify(w, e, 0, res, k)


def test_spectrum_full_size_matches_oracle_solve_at_high_energy(dd):
    w = I.config_spectrum()
    ie = np.array([185, 199])
    res = _gpu(dd, w, ie)
    for k, e in enumerate(ie):
        o = run.solve_workload_point(w, e, 0, method="fft", rtol=1e-11)
        for key, got in (("P_EELS", res.p_eels), ("P_CL", res.p_cl), ("P_ext", res.p_ext), ("P_abs", res.p_abs)):
            assert abs(got[k, 0] - o[key]) <= 1e-4 * abs(o[key]), (key, got[k, 0], o[key])
        assert np.linalg.norm(res.p[k, 0] - o["p"]) <= 1e-4 * np.linalg.norm(o["p"])


def test_rod_map_full_size_block_of_beams_certified(dd):
    """24x24x72 rod (41,472 dipoles, 48x48x144 FFT): one energy, four raster
    beams solved as one block sharing D-hat."""
    w = I.config_rod_map(n_energy=64)
    beams = w.beams_nm[[0, 33, 517, 1023]]
    ie = np.array([31])
    res = _gpu(dd, w, ie, beams=beams)
    assert res.converged.all()
    for ib in range(len(beams)):
        _certify(w, 31, ib, res, 0, beams=beams)


def test_rod_map_full_size_block_of_32_beams(dd):
    """One energy of the rod map with 32 raster beams in one batch (the FFT x
    pass reuses each staged D-hat tile over 16 beams): six beams certified by
    the oracle, and two of them bit-identical to solving them alone."""
    w = I.config_rod_map(n_energy=64)
    pick = np.arange(0, 1024, 32)                 # one beam per raster row
    beams = w.beams_nm[pick]
    ie = np.array([40])
    res = _gpu(dd, w, ie, beams=beams)
    assert res.converged.all()
    for ib in (0, 5, 13, 21, 28, 31):
        _certify(w, 40, ib, res, 0, beams=beams)
    for ib in (0, 21):
        solo = _gpu(dd, w, ie, beams=beams[ib:ib + 1])
        assert solo.p_eels[0, 0] == res.p_eels[0, ib]
        assert solo.p_cl[0, 0] == res.p_cl[0, ib]
        assert np.array_equal(solo.p[0, 0], res.p[0, ib])


def test_cherenkov_full_size_certified(dd):
    """64^3 silver sphere (137,376 dipoles, 128^3 FFT) in eps_h = 4 + 0.05i at
    200 keV (beta_h > 1)."""
    w = I.config_cherenkov()
    ie = np.array([20, 80])
    res = _gpu(dd, w, ie)
    assert res.converged.all()
    for k, e in enumerate(ie):
        pt, _ = _certify(w, e, 0, res, k)
        assert pt.beta_h.real > 1
        assert abs(res.p_eels[k, 0] - res.p_ext[k, 0]) > 1e-3 * abs(res.p_ext[k, 0])
