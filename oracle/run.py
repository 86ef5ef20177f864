"""One (energy, beam) point of the DDA end to end, in the paper's order:
host and electron factors (Eq. 24), incident field (Eq. 25), auxiliary field
(Eq. 34), polarizabilities, the dipole system, then the losses (Eq. 32/37,
17/48, 18, 42).

Readings: lattice centred at the origin, z0 = 0, q = -e (the sign of q does
not change any probability, only the sign of p), beam along +z at (x0, y0).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import scipy.sparse.linalg as spla

from . import field, green, losses, physics
from .constants import C_LIGHT, EPS0, NM
from .icosphere import icosphere


def lattice(nx, ny, nz, d_nm, occ):
    """Occupied cells in x-fastest linear order: idx [N,3] = (ix,iy,iz),
    positions r [N,3] in metres, material index (1-based) [N]."""
    occ = np.asarray(occ).reshape(nz, ny, nx)
    iz, iy, ix = np.nonzero(occ)
    idx = np.stack([ix, iy, iz], axis=1)
    n = np.array([nx, ny, nz], dtype=np.float64)
    r = ((idx + 0.5) - n / 2.0) * d_nm * NM
    return idx, r, occ[iz, iy, ix].astype(int)


@dataclasses.dataclass
class Point:
    omega: float
    k: complex
    m_h: complex
    beta_h: complex
    gamma_h: complex
    v: float
    idx: np.ndarray
    r: np.ndarray
    alpha: np.ndarray          # alpha~ per dipole (CM + radiative reaction)
    alpha_cm: np.ndarray
    E_inc: np.ndarray
    E_a: np.ndarray
    eps_h: complex
    n_axes: tuple
    d: float
    interaction: str = "point"     # "point" (Eq. 5 at the cell centres) or "igt_so" (oracle/igt.py)


def setup(nx, ny, nz, d_nm, occ, energy_eV, eps_p, eps_h, beam_nm, ekin_keV=None, v=None, direction=None,
          interaction="point", polarizability="cm"):
    """interaction / polarizability: "point" / "cm" (point dipoles, Clausius-
    Mossotti with radiative reaction) or "igt_so" / "igt_so" (the cell-
    integrated Green's tensor to second order in kd, Sec. S5; oracle/igt.py)."""
    if v is None:
        v = physics.electron_speed(ekin_keV)
    omega = float(physics.omega_of(energy_eV))
    m_h = physics.host_index(eps_h)
    beta, gamma = physics.beta_gamma_h(v, m_h)
    k = m_h * omega / C_LIGHT                       # k = m_h k0 (Eq. 4)
    idx, r, mat = lattice(nx, ny, nz, d_nm, occ)
    d = d_nm * NM
    m2 = np.asarray(eps_p, dtype=np.complex128)[mat - 1] / complex(eps_h)   # m = m_p / m_h (Eq. 2)
    a_cm = physics.polarizability_cm(m2, d)
    if polarizability == "igt_so":
        from . import igt
        a = igt.polarizability_igt_so(a_cm, k, d)
    else:
        a = physics.polarizability_rr(a_cm, k)
    x0, y0 = beam_nm[0] * NM, beam_nm[1] * NM
    if direction is None:
        E = field.incident_field(r, omega, v, m_h, gamma, x0, y0)
        Ea = field.auxiliary_field(r, omega, v, m_h, gamma, x0, y0)
    else:
        E, Ea = field.fields_along(r, omega, v, m_h, gamma, x0, y0, direction)
    return Point(omega, k, m_h, beta, gamma, v, idx, r, a, a_cm, E, Ea, complex(eps_h), (nx, ny, nz), d, interaction)


def system_matrix(pt: Point):
    """The dense 3N x 3N matrix of the point's interaction model."""
    if pt.interaction == "igt_so":
        from . import igt
        return igt.dense_matrix_so(pt.idx, pt.k, pt.alpha, pt.d)
    return green.dense_matrix(pt.r, pt.k, pt.alpha)


def solve_lu(pt: Point):
    return np.linalg.solve(system_matrix(pt), pt.E_inc.reshape(-1)).reshape(-1, 3)


def solve_fft(pt: Point, rtol=1e-12, restart=200, maxiter=20000, workers=-1, x0=None):
    """Library GMRES on the lattice FFT operator, Jacobi-scaled:
    (alpha^1/2 A alpha^1/2) y = alpha^1/2 E, p = alpha^1/2 y."""
    op = green.FFTOperator(pt.idx, pt.n_axes, pt.d, pt.k, pt.alpha, workers=workers, interaction=pt.interaction)
    sq = np.sqrt(pt.alpha)
    n3 = 3 * len(pt.r)

    def mv(y):
        y = y.reshape(-1, 3)
        return (sq[:, None] * op.matvec(sq[:, None] * y)).reshape(-1)

    L = spla.LinearOperator((n3, n3), matvec=mv, dtype=np.complex128)
    b = (sq[:, None] * pt.E_inc).reshape(-1)
    y0 = None if x0 is None else (x0 / sq[:, None]).reshape(-1)
    y, info = spla.gmres(L, b, x0=y0, rtol=rtol, atol=0.0, restart=restart, maxiter=maxiter)
    if info != 0:
        raise RuntimeError(f"oracle GMRES did not converge (info={info})")
    return (sq[:, None] * y.reshape(-1, 3)), op


def residual(pt: Point, p, op: Optional[green.FFTOperator] = None):
    """||E_inc - A p|| / ||E_inc|| with the oracle's own FFT operator."""
    if op is None:
        op = green.FFTOperator(pt.idx, pt.n_axes, pt.d, pt.k, pt.alpha, interaction=pt.interaction)
    r = pt.E_inc - op.matvec(p)
    return float(np.linalg.norm(r) / np.linalg.norm(pt.E_inc))


_ICO = {}


def directions(level=4):
    if level not in _ICO:
        _ICO[level] = icosphere(level)
    return _ICO[level]


def observables(pt: Point, p_t, want_cl=True, want_img=False, level=4):
    out = dict(
        P_EELS=losses.p_eels(pt.E_a, p_t, pt.eps_h, pt.omega),
        P_ext=losses.p_ext(pt.E_inc, p_t, pt.eps_h, pt.omega),
        P_abs=losses.p_abs(p_t, pt.alpha_cm, pt.eps_h, pt.omega),
    )
    if want_cl:
        dirs, w = directions(level)
        out["P_CL"] = losses.p_cl(pt.r, p_t, pt.k, pt.m_h, pt.omega, dirs, w)
    if want_img:
        out["P_sca_img"] = losses.p_sca_img(pt.r, p_t, pt.k, pt.eps_h, pt.omega)
    return out


def p_si(pt: Point, p_t):
    """Dipole moments in SI (C m s): p = 4 pi eps0 eps_h,rel p~."""
    return 4.0 * np.pi * EPS0 * pt.eps_h * p_t


def solve_point(nx, ny, nz, d_nm, occ, energy_eV, eps_p, eps_h, beam_nm, ekin_keV=None, v=None,
                method="lu", want_cl=True, want_img=False, rtol=1e-12, direction=None, interaction="point",
                polarizability="cm"):
    pt = setup(nx, ny, nz, d_nm, occ, energy_eV, eps_p, eps_h, beam_nm, ekin_keV=ekin_keV, v=v, direction=direction,
               interaction=interaction, polarizability=polarizability)
    if method == "lu":
        p_t = solve_lu(pt)
    else:
        p_t, _ = solve_fft(pt, rtol=rtol)
    out = observables(pt, p_t, want_cl=want_cl, want_img=want_img)
    out["p_t"] = p_t
    out["p"] = p_si(pt, p_t)
    out["point"] = pt
    return out


def solve_workload_point(w, ie: int, ib: int, **kw):
    g = w.grid
    return solve_point(g.nx, g.ny, g.nz, g.d_nm, g.occ, w.energies_eV[ie], w.eps_p[ie], w.eps_h[ie],
                       w.beams_nm[ib], ekin_keV=w.ekin_keV, **kw)


# --------------------------------------------------------------------------
# Plane-wave excitation (used only by the Lorenz-Mie pin of the DDA core).
# --------------------------------------------------------------------------
def plane_wave_cross_sections(nx, ny, nz, d_nm, occ, m_rel2, k):
    """x-polarised plane wave along +z in a real host (E0 = 1):
    C_ext = 4 pi k Im sum E^* . p~, C_abs = 4 pi k sum |p~|^2 (-Im 1/alpha~_CM)
    (Eq. 17-19 with I0 of Eq. 19)."""
    idx, r, mat = lattice(nx, ny, nz, d_nm, occ)
    d = d_nm * NM
    a_cm = physics.polarizability_cm(np.full(len(r), m_rel2), d)
    a = physics.polarizability_rr(a_cm, k)
    E = np.zeros((len(r), 3), dtype=np.complex128)
    E[:, 0] = np.exp(1j * k * r[:, 2])
    A = green.dense_matrix(r, k, a)
    p = np.linalg.solve(A, E.reshape(-1)).reshape(-1, 3)
    c_ext = 4.0 * np.pi * k * np.imag(np.sum(np.conj(E) * p))
    c_abs = 4.0 * np.pi * k * np.sum(np.sum(np.abs(p) ** 2, axis=1) * (-np.imag(1.0 / a_cm)))
    return float(np.real(c_ext)), float(np.real(c_abs))
