"""Plane-wave Lorenz-Mie cross sections of a homogeneous sphere in a
non-absorbing host (the classical solution the paper cites in Sec. 3.2,
ref. [46]; coefficients in the textbook Riccati-Bessel form).  Used only to
pin the oracle's DDA core (Green's tensor, polarizability, solve) against an
exact solution as the lattice is refined.

  a_n = [m psi_n(mx) psi_n'(x) - psi_n(x) psi_n'(mx)] / [m psi_n(mx) xi_n'(x) - xi_n(x) psi_n'(mx)]
  b_n = [psi_n(mx) psi_n'(x) - m psi_n(x) psi_n'(mx)] / [psi_n(mx) xi_n'(x) - m xi_n(x) psi_n'(mx)]
  C_ext = (2 pi / k^2) sum (2n+1) Re(a_n + b_n)
  C_sca = (2 pi / k^2) sum (2n+1) (|a_n|^2 + |b_n|^2)

psi_n(z) = z j_n(z), xi_n(z) = z h_n^(1)(z); x = k a, m = relative index.
"""
from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def _psi(n, z):
    return z * spherical_jn(n, z)


def _dpsi(n, z):
    return spherical_jn(n, z) + z * spherical_jn(n, z, derivative=True)


def _xi(n, x):
    return x * (spherical_jn(n, x) + 1j * spherical_yn(n, x))


def _dxi(n, x):
    h = spherical_jn(n, x) + 1j * spherical_yn(n, x)
    dh = spherical_jn(n, x, derivative=True) + 1j * spherical_yn(n, x, derivative=True)
    return h + x * dh


def mie_coefficients(m_rel: complex, x: float, n_max: int):
    """Arrays a_n, b_n (n = 1..n_max) for size parameter x = k a."""
    mx = m_rel * x
    an = np.empty(n_max, dtype=np.complex128)
    bn = np.empty(n_max, dtype=np.complex128)
    for n in range(1, n_max + 1):
        ps_x, dps_x = _psi(n, x), _dpsi(n, x)
        ps_m, dps_m = _psi(n, mx), _dpsi(n, mx)
        xi_x, dxi_x = _xi(n, x), _dxi(n, x)
        an[n - 1] = (m_rel * ps_m * dps_x - ps_x * dps_m) / (m_rel * ps_m * dxi_x - xi_x * dps_m)
        bn[n - 1] = (ps_m * dps_x - m_rel * ps_x * dps_m) / (ps_m * dxi_x - m_rel * xi_x * dps_m)
    return an, bn


def mie_cross_sections(m_rel: complex, k: float, a: float, n_max=None):
    x = k * a
    if n_max is None:
        n_max = int(np.ceil(x + 4.0 * x ** (1.0 / 3.0) + 2.0)) + 2
    an, bn = mie_coefficients(m_rel, x, n_max)
    n = np.arange(1, n_max + 1)
    f = 2.0 * np.pi / k ** 2
    return f * float(np.sum((2 * n + 1) * np.real(an + bn))), f * float(np.sum((2 * n + 1) * (abs(an) ** 2 + abs(bn) ** 2)))
