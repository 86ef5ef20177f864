"""Lorenz-Mie EELS and CL of a homogeneous sphere in a non-absorbing host,
below the Cherenkov threshold: the exact solution the paper compares its DDA
spectra with (Sec. 3.2, Figs. 3-7), used here only to pin the oracle's DDA
as the lattice is refined.  Test infrastructure, like the rest of oracle/.

The paper cites the multipole solution (its refs. [5], [47]) without
formulas; this module obtains the same solution by a route that needs only
textbook Mie theory:

 1. Inside the cylinder rho < b around the trajectory the electron's field
    has no sources, so it expands in regular vector spherical waves about the
    sphere's centre,
        E_inc = sum_nm [c^M_nm j_n(kr) X_nm + c^N_nm curl(j_n(kr) X_nm) / k],
    X_nm = L Y_nm / sqrt(n(n+1)) (L = -i r x grad, Y_nm orthonormal).  Since
    r . curl(f X_nm) = i sqrt(n(n+1)) f Y_nm and X_nm has no radial part,
        r^.E = sum i sqrt(n(n+1)) j_n(kr)/(kr) c^N_nm Y_nm,
        r^.H = sum (k / (w mu0)) sqrt(n(n+1)) j_n(kr)/(kr) c^M_nm Y_nm,
    with H = curl(E)/(i w mu0).  Projecting r^.E and r^.H on a sphere of
    radius R (a < R < b) onto Y_nm gives c^N and c^M.  E_inc is Eq. 25;
    H = curl(I1 e_z) with I1 of Eq. 23 (E = i w mu0 (1 + grad d_z / k^2) I1 e_z,
    Eq. 22).
 2. The sphere scatters each term into the outgoing wave of the same (n, m)
    (h_n^(1) in place of j_n) with s^N = -a_n c^N, s^M = -b_n c^M (Mie
    coefficients a_n, b_n of oracle/mie.py).
 3. With orthonormal X_nm the outgoing flux of a term c j_n + s h_n is
    (Re(c^* s) + |s|^2) / (2 Z k^2), Z = Z0 / m_h, so
        W_sca = sum |s|^2 / (2 Z k^2),   W_ext = -sum Re(c^* s) / (2 Z k^2).
 4. P_EELS = P_ext = 2 W_ext / (pi hbar^2 w) and P_CL = 2 W_sca / (pi hbar^2 w)
    (Eq. 37 and Eq. 42 with E_a = -E_inc^* for real gamma_h, Sec. 2.4), in
    eV^-1.

The same projection applied to a plane wave reproduces the textbook cross
sections (a pin of steps 1-3); the electron's H against the curl of Eq. 25
by finite differences pins step 1's magnetic field.
"""
from __future__ import annotations

import numpy as np
from scipy.special import kv, spherical_jn, sph_harm_y

from . import field, physics
from .constants import C_LIGHT, E_CHARGE, HBAR, MU0, Q_ELECTRON
from .mie import mie_coefficients


def sphere_grid(n_theta: int, n_phi: int):
    """Gauss-Legendre nodes in cos(theta) times uniform phi: directions [P,3]
    and weights [P] (sum 4 pi), with theta, phi."""
    x, wx = np.polynomial.legendre.leggauss(n_theta)
    th = np.arccos(x)
    ph = 2.0 * np.pi * np.arange(n_phi) / n_phi
    T, F = np.meshgrid(th, ph, indexing="ij")
    W = np.repeat(wx[:, None], n_phi, axis=1) * (2.0 * np.pi / n_phi)
    u = np.stack([np.sin(T) * np.cos(F), np.sin(T) * np.sin(F), np.cos(T)], axis=-1)
    return u.reshape(-1, 3), W.reshape(-1), T.reshape(-1), F.reshape(-1)


def regular_coefficients(E_fn, H_fn, k: float, Z: float, R: float, n_max: int, n_theta=None, n_phi=None):
    """c^M_nm, c^N_nm (arrays [n_max][2 n_max + 1], m = -n..n at column m + n_max)
    of a source-free field given by callables E_fn(r[P,3]), H_fn(r[P,3])
    (complex [P,3]) on the sphere |r| = R (step 1 above)."""
    n_theta = n_theta or 2 * n_max + 16
    n_phi = n_phi or 2 * n_theta
    u, w, th, ph = sphere_grid(n_theta, n_phi)
    r = R * u
    er = np.sum(u * E_fn(r), axis=1)
    hr = np.sum(u * H_fn(r), axis=1)
    cM = np.zeros((n_max, 2 * n_max + 1), dtype=np.complex128)
    cN = np.zeros_like(cM)
    kr = k * R
    for n in range(1, n_max + 1):
        jn = spherical_jn(n, kr)
        s = np.sqrt(n * (n + 1.0))
        for m in range(-n, n + 1):
            y = np.conj(sph_harm_y(n, m, th, ph))
            pe = np.sum(w * y * er)
            ph_ = np.sum(w * y * hr)
            cN[n - 1, m + n_max] = pe * kr / (1j * s * jn)
            cM[n - 1, m + n_max] = ph_ * Z * kr / (s * jn)          # k / (w mu0) = 1 / Z
    return cM, cN


def powers(cM, cN, m_rel: complex, k: float, a: float, Z: float):
    """(W_ext, W_sca) of the sphere of radius a in the regular field (cM, cN)."""
    n_max = cM.shape[0]
    an, bn = mie_coefficients(m_rel, k * a, n_max)
    sM = -bn[:, None] * cM
    sN = -an[:, None] * cN
    f = 1.0 / (2.0 * Z * k * k)
    w_ext = -f * float(np.sum(np.real(np.conj(cM) * sM) + np.real(np.conj(cN) * sN)))
    w_sca = f * float(np.sum(abs(sM) ** 2 + abs(sN) ** 2))
    return w_ext, w_sca


def electron_H(r, omega, v, gamma_h, x0, y0, z0=0.0, q=Q_ELECTRON):
    """H = curl(I1 e_z) = (d_y I1, -d_x I1, 0), I1 = q/(2 pi) exp(i w (z - z0)/v) K0(w b/(gamma_h v))
    (Eq. 22-23); d_b K0(u) = -K1(u) du/db."""
    dx = r[:, 0] - x0
    dy = r[:, 1] - y0
    b = np.hypot(dx, dy)
    kap = omega / (gamma_h * v)
    g = q / (2.0 * np.pi) * np.exp(1j * omega * (r[:, 2] - z0) / v) * (-kv(1, kap * b) * kap)
    h = np.zeros((len(r), 3), dtype=np.complex128)
    h[:, 0] = g * dy / b
    h[:, 1] = -g * dx / b
    return h


def electron_coefficients(eps_h: float, energy_eV: float, b: float, v: float, n_max: int, R: float):
    """Regular-wave coefficients (cM, cN) of the electron's field about the
    origin (electron along +z through (b, 0), host eps_h real, beta_h < 1),
    projected on the sphere |r| = R < b, with (k, Z, omega)."""
    m_h = float(np.sqrt(eps_h))
    omega = float(physics.omega_of(energy_eV))
    k = m_h * omega / C_LIGHT
    beta, gamma = physics.beta_gamma_h(v, m_h)
    if not beta.real < 1.0:
        raise ValueError("the Mie EELS solution here needs beta_h < 1")
    if not 0.0 < R < b:
        raise ValueError("the projection sphere must lie inside the trajectory's cylinder")
    Z = MU0 * C_LIGHT / m_h

    def E_fn(r):
        return field.incident_field(r, omega, v, m_h, gamma, b, 0.0)

    def H_fn(r):
        return electron_H(r, omega, v, gamma, b, 0.0)

    cM, cN = regular_coefficients(E_fn, H_fn, k, Z, R, n_max)
    return cM, cN, k, Z, omega


def eels_cl_from(coef, a: float, eps_p: complex, eps_h: float):
    """P_EELS and P_CL (eV^-1) of a sphere of radius a (m, a < R) in the field
    whose coefficients electron_coefficients returned."""
    cM, cN, k, Z, omega = coef
    w_ext, w_sca = powers(cM, cN, np.sqrt(complex(eps_p) / eps_h), k, a, Z)
    f = 2.0 / (np.pi * HBAR ** 2 * omega) * E_CHARGE
    return f * w_ext, f * w_sca


def eels_cl_sphere(a: float, eps_p: complex, eps_h: float, energy_eV: float, b: float, v: float,
                   n_max: int = 30, R=None):
    """P_EELS and P_CL (eV^-1) of a sphere of radius a (m) centred at the
    origin, electron along +z through (b, 0) (b > a, m), host eps_h real with
    beta_h < 1.  R: radius of the projection sphere (default (a + b)/2)."""
    R = 0.5 * (a + b) if R is None else R
    return eels_cl_from(electron_coefficients(eps_h, energy_eV, b, v, n_max, R), a, eps_p, eps_h)
