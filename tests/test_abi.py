"""The C-ABI library loads, exports every symbol include/eelsdda.h declares,
and its host-only logic behaves (no GPU compute here)."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "eelsdda.h")
LIB = os.path.join(ROOT, "paper_2208_01348_gb300", "libeelsdda.so")


@pytest.fixture(scope="module")
def lib():
    from paper_2208_01348_gb300 import build
    build.build()
    from paper_2208_01348_gb300 import eelsdda
    return eelsdda


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eels_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("eels_create", "eels_destroy", "eels_set_grid", "eels_solve", "eels_query_footprint",
              "eels_last_error", "eels_bessel_k01_dev", "eels_incident_field", "eels_apply_matrix"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (eels_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    assert set(lib.EXPORTED) <= exported


def test_default_opts(lib):
    o = lib.eels_default_opts()
    assert o.precision == lib.EELS_MIXED and o.solver == lib.EELS_QMR2
    assert o.eps_it == 1e-8 and o.eps_inner == 1e-5 and o.n_dir == 2562


def test_host_direction_grid_matches_oracle(lib):
    from oracle.icosphere import icosphere
    d, w = lib.eels_directions(2562)
    V, wo = icosphere(4)
    assert d.shape == (2562, 3)
    # same construction -> same vertices (up to rounding order)
    assert np.allclose(d, V, atol=1e-15, rtol=0)
    assert np.allclose(w, wo, atol=1e-15, rtol=0)
    with pytest.raises(lib.EelsError):
        lib.eels_directions(100)


def test_footprint_grows_with_systems(lib):
    from paper_2208_01348_gb300 import inputs as I
    occ = I.sphere_occupancy(32, 30.0)
    o = lib.eels_default_opts()
    a = lib.eels_query_footprint(occ, 30 / 32, o, 1)
    b = lib.eels_query_footprint(occ, 30 / 32, o, 200)
    assert 0 < a < b
    o64 = lib.eels_default_opts(precision=lib.EELS_FP64)
    assert lib.eels_query_footprint(occ, 30 / 32, o64, 200) > b


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="checks the no-GPU error path")
def test_create_without_gpu_fails_loudly(lib):
    with pytest.raises(lib.EelsError) as e:
        lib.eels_create(0)
    assert e.value.code == lib.EELS_E_CUDA


def test_package_import_has_no_fallback():
    # the product path imports only the CUDA binding; it never touches the oracle
    pkg = os.path.join(ROOT, "paper_2208_01348_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert "import oracle" not in src and "from oracle" not in src, f


def test_host_utilities_eq29_eq41_match_oracle():
    """Host-side utilities of the library (no GPU work): the Frank-Tamm loss
    per unit length (Eq. 29) and P_CL^tot (Eq. 41) against the oracle."""
    import numpy as np
    from oracle import losses, physics
    from paper_2208_01348_gb300 import eelsdda as dd
    for ek, eps_h in ((200.0, 4.0), (100.0, 4.0), (100.0, 2.1025), (300.0, 2.25)):
        ref = losses.frank_tamm_rate(physics.electron_speed(ek), np.sqrt(eps_h))
        got = dd.eels_frank_tamm(ek, eps_h)
        assert (got == 0.0 and ref == 0.0) or abs(got - ref) <= 1e-12 * abs(ref)
    with pytest.raises(dd.EelsError):
        dd.eels_frank_tamm(200.0, 4.0 + 0.05j)
    rng = np.random.default_rng(3)
    a, b, c = rng.random((3, 7, 2))
    assert np.allclose(dd.eels_cl_total(a, b, c), losses.p_cl_tot(a, b, c), rtol=0, atol=1e-15)


def test_extrapolation_utility_matches_oracle():
    """eels_extrapolate (Sec. 3.2) against the oracle on exact and noisy data."""
    import numpy as np
    from oracle.extrapolate import extrapolate_to_zero
    from paper_2208_01348_gb300 import eelsdda as dd
    d = 30.0 / np.array([128, 108, 91, 76, 64, 54, 45, 38, 32])
    rng = np.random.default_rng(9)
    for noise in (0.0, 1e-4, 1e-2):
        y = 1.7 + 0.4 * d - 0.05 * d * d + noise * d ** 3 * rng.standard_normal(len(d))
        v, ci = dd.eels_extrapolate(d, y)
        rv, rci = extrapolate_to_zero(d, y)
        assert v == pytest.approx(rv, rel=1e-12)
        assert ci == pytest.approx(rci, rel=1e-7, abs=1e-9)   # noiseless: both are rounding-level
    with pytest.raises(dd.EelsError):
        dd.eels_extrapolate([1.0, 2.0], [1.0, 2.0])


def test_vacuum_equivalent_utility_matches_oracle():
    """eels_vacuum_equivalent (Sec. 2.7, Eq. 45-47, Eq. S16) against the
    oracle's map; the library takes the kinetic energy of speed m_h v directly,
    the oracle by Eq. 47, so the two routes check each other."""
    import math
    from oracle import physics
    from paper_2208_01348_gb300 import eelsdda as dd
    cases = [(100.0, 2.1025, 2.3), (60.0, 1.69, 1.1), (300.0, 1.21, 3.9), (200.0, 1.44, 2.0)]
    for ek, eps_h, e in cases:
        for rule in (dd.EELS_SCALE_ENERGY, dd.EELS_SCALE_LENGTH):
            got = dd.eels_vacuum_equivalent(ek, eps_h, e, rule)
            ref = physics.vacuum_equivalent(ek, eps_h, e, length_rule=rule == dd.EELS_SCALE_LENGTH)
            for key in ("ekin_keV", "energy_eV", "length_scale", "eps_p_scale", "p_scale"):
                assert got[key] == pytest.approx(ref[key], rel=1e-12), (ek, eps_h, rule, key)
            with pytest.raises(dd.EelsError):
                dd.eels_vacuum_equivalent(ek, eps_h, e, rule | dd.EELS_SCALE_ULTRAREL)
    for ek, eps_h, e in ((200.0, 4.0, 2.0), (100.0, 6.25, 3.0)):
        for rule in (dd.EELS_SCALE_ENERGY, dd.EELS_SCALE_LENGTH):
            got = dd.eels_vacuum_equivalent(ek, eps_h, e, rule | dd.EELS_SCALE_ULTRAREL)
            ref = physics.vacuum_equivalent(ek, eps_h, e, length_rule=rule == dd.EELS_SCALE_LENGTH,
                                            ultrarelativistic=True)
            assert math.isinf(got["ekin_keV"]) and math.isinf(ref["ekin_keV"])
            for key in ("energy_eV", "length_scale", "eps_p_scale", "p_scale"):
                assert got[key] == pytest.approx(ref[key], rel=1e-12), (ek, eps_h, rule, key)
            with pytest.raises(dd.EelsError):
                dd.eels_vacuum_equivalent(ek, eps_h, e, rule)
    for bad in ((0.0, 2.0, 2.0, 0), (100.0, 0.0, 2.0, 0), (100.0, 2.0, -1.0, 0), (100.0, 2.0, 2.0, 4)):
        with pytest.raises(dd.EelsError):
            dd.eels_vacuum_equivalent(bad[0], bad[1], bad[2], bad[3])
