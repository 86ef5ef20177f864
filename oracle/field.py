"""Fast-electron incident field and the auxiliary field of conjugate sources.

K0 and K1 of complex argument come from scipy.special.kv (AMOS).  The
argument omega b / (gamma_h v) lies in the fourth quadrant (arg in
[-pi/2, 0]) because gamma_h lies in the first one (Sec. 2.2).
"""
from __future__ import annotations

import numpy as np
from scipy.special import kv

from .constants import EPS0, Q_ELECTRON


def _transverse(r, x0, y0):
    dx = r[:, 0] - x0
    dy = r[:, 1] - y0
    b = np.hypot(dx, dy)
    if np.any(b == 0.0):
        raise ValueError("impact parameter b = 0 at a dipole: the field of Eq. 25 is singular")
    return dx, dy, b


def incident_field(r, omega, v, m_h, gamma_h, x0, y0, z0=0.0, q=Q_ELECTRON):
    """E_inc at points r [N,3] (m), Eq. 25:
    E = q w / (2 pi eps0 m_h^2 v^2 gamma_h) exp(i w (z - z0)/v)
        * ((x-x0)/b K1(a), (y-y0)/b K1(a), -(i/gamma_h) K0(a)),  a = w b/(gamma_h v).
    Units: V s / m (frequency-domain field).  Returns complex [N,3]."""
    dx, dy, b = _transverse(r, x0, y0)
    a = omega * b / (gamma_h * v)
    k0 = kv(0, a)
    k1 = kv(1, a)
    pref = q * omega / (2.0 * np.pi * EPS0 * m_h ** 2 * v ** 2 * gamma_h)
    ph = np.exp(1j * omega * (r[:, 2] - z0) / v)
    e = np.empty((len(r), 3), dtype=np.complex128)
    e[:, 0] = pref * ph * dx / b * k1
    e[:, 1] = pref * ph * dy / b * k1
    e[:, 2] = pref * ph * (-1j / gamma_h) * k0
    return e


def auxiliary_field(r, omega, v, m_h, gamma_h, x0, y0, z0=0.0, q=Q_ELECTRON):
    """E_a, the incident field of the conjugate sources, first line of Eq. 34:
    E_a = -q w / (2 pi eps0 m_h^2 v^2 gamma_h) exp(-i w (z - z0)/v)
          * ((x-x0)/b K1, (y-y0)/b K1, (i/gamma_h) K0)."""
    dx, dy, b = _transverse(r, x0, y0)
    a = omega * b / (gamma_h * v)
    k0 = kv(0, a)
    k1 = kv(1, a)
    pref = -q * omega / (2.0 * np.pi * EPS0 * m_h ** 2 * v ** 2 * gamma_h)
    ph = np.exp(-1j * omega * (r[:, 2] - z0) / v)
    e = np.empty((len(r), 3), dtype=np.complex128)
    e[:, 0] = pref * ph * dx / b * k1
    e[:, 1] = pref * ph * dy / b * k1
    e[:, 2] = pref * ph * (1j / gamma_h) * k0
    return e


def line_integral_I1(r, omega, v, gamma_h, x0, y0, z0=0.0, q=Q_ELECTRON, conjugate=False):
    """I1 of Eq. 23 (Eq. S14): q/(2 pi) exp(i w (z-z0)/v) K0(w b/(gamma_h v)).
    With conjugate=True the source is J_s^* (Eq. 33), which flips the sign of
    the phase (Sec. 2.4, before Eq. 34)."""
    dx, dy, b = _transverse(r, x0, y0)
    sgn = -1.0 if conjugate else 1.0
    return q / (2.0 * np.pi) * np.exp(sgn * 1j * omega * (r[:, 2] - z0) / v) * kv(0, omega * b / (gamma_h * v))


def beam_frame(direction):
    """Orthonormal frame (e1, e2, n) of an electron moving along `direction`:
    the rotation that takes z to n by the smallest angle (about the axis
    z x n; a half turn about x when n = -z) applied to (x, y, z).  For n = z
    it is the lattice frame, so (x0, y0) keep their meaning."""
    n = np.asarray(direction, dtype=np.float64)
    n = n / np.linalg.norm(n)
    z = np.array([0.0, 0.0, 1.0])
    axis = np.cross(z, n)
    s = np.linalg.norm(axis)
    c = float(n[2])
    if s < 1e-15:
        Rm = np.eye(3) if c > 0 else np.diag([1.0, -1.0, -1.0])
    else:
        k = axis / s
        K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
        Rm = np.eye(3) + s * K + (1 - c) * (K @ K)      # Rodrigues' rotation formula
    return Rm[:, 0], Rm[:, 1], Rm[:, 2]


def fields_along(r, omega, v, m_h, gamma_h, x0, y0, direction, q=Q_ELECTRON):
    """E_inc and E_a for an electron moving along `direction` through the
    point x0 e1 + y0 e2 of its frame (beam_frame), phase reference there:
    Eq. 25 and the first line of Eq. 34 evaluated in the frame (e1, e2, n)
    and rotated back to the lattice frame.  Returns two complex [N,3]."""
    e1, e2, n = beam_frame(direction)
    Rm = np.stack([e1, e2, n], axis=1)            # columns: frame axes in lattice coordinates
    rp = (r - (x0 * e1 + y0 * e2)) @ Rm           # coordinates in the beam frame
    E = incident_field(rp, omega, v, m_h, gamma_h, 0.0, 0.0, q=q) @ Rm.T
    Ea = auxiliary_field(rp, omega, v, m_h, gamma_h, 0.0, 0.0, q=q) @ Rm.T
    return E, Ea
