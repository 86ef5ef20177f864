"""Integrated-Green's-tensor interaction and polarizability, to second order
in kd: the options the paper recommends in Sec. S5 ("-int igt_so",
"-pol igt_so"), whose formulas it does not give.

Test infrastructure only (see oracle/__init__.py).

Reading (written out here from the definitions, not from any program):

* Interaction.  Dipole j stands for its cubic cell of edge d uniformly
  polarised, so the field it makes at dipole i is the Green's tensor of
  Eq. 5 averaged over the source cell,

      G_int(R) = d^-3 integral over the cell of G~(R - s) d^3 s,   R = r_i - r_j != 0

  (`cell_average`, by tensor-product Gauss-Legendre cubature).  With
  rho = R - s, G~(rho) = exp(ik rho) [k^2 A - B + ik C], where
  A = (I - rr)/rho, B = (I - 3 rr)/rho^3, C = (I - 3 rr)/rho^2.  The
  second-order ("so") form expands the exponential around the cell centre,
  exp(ik rho) = exp(ikR) (1 + ik delta - k^2 delta^2 / 2 + ...),
  delta = rho - R, keeps every term up to k^2 and integrates the geometric
  tensors exactly:

      G_so(R) = exp(ikR) [ -<B> + ik <C - delta B> + k^2 <A - delta C + delta^2 B / 2> ],

  <.> the cell average (`so_tables`).  It differs from G_int by O((kd)^3)
  and tends to G~(R) far from the cell.  It is used for lattice offsets of
  max-norm <= L_NEAR; beyond them the cell average and the point tensor
  differ by O((d/R)^4) (the second-order Taylor term of the cell average is
  (d^2/24) Laplacian G~ = -(kd)^2/24 G~), and the point tensor is used.

* Polarizability.  The field of a cell at its own centre is the principal
  value (a spherical hole) of the same cell integral; the static part of
  its integrand, -B, integrates to zero over a cube by symmetry, and the
  Clausius-Mossotti relation already holds the Lorentz field of the hole.
  Expanding exp(ik rho) in powers of k rho, the k^1 terms cancel, the k^2
  terms sum to (k^2 / 2 rho)(I + rr) and the k^3 terms to (2/3) i k^3 I, so

      M = d^-3 PV integral of G~ = (2/3) (c1 k^2 / d + i k^3) I + O(k^4 d),
      c1 = integral over [-1/2, 1/2]^3 of |u|^-1 d^3 u = 3 ln(2 + sqrt 3) - pi / 2,

  and 1/alpha~_so = 1/alpha~_CM - M: the radiative reaction of
  physics.polarizability_rr plus the k^2 term of the cell.
"""
from __future__ import annotations

import math

import numpy as np

from .green import PAIRS, green_tilde

L_NEAR = 3                 # lattice offsets of max-norm <= L_NEAR take the cell-averaged form
C1 = 3.0 * math.log(2.0 + math.sqrt(3.0)) - math.pi / 2.0


def _cell_nodes(n: int):
    """Gauss-Legendre nodes and weights on [-1/2, 1/2]^3 (unit cell), n per axis."""
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * x
    w = 0.5 * w
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]
    return np.stack([X, Y, Z], axis=-1).reshape(-1, 3), W.reshape(-1)


def cell_average(R, k, d, n: int = 24):
    """d^-3 times the integral of G~(R - s) over the cell s in [-d/2, d/2]^3
    (R [3] in metres, not inside the cell), by n^3-point cubature."""
    s, w = _cell_nodes(n)
    G = green_tilde(np.asarray(R, dtype=np.float64)[None, :] - d * s, k)
    return np.tensordot(w, G, axes=(0, 0))


def so_tables(offset, n: int = 24):
    """Cell averages <B>, <C - delta B>, <A - delta C + delta^2 B / 2> for the
    lattice offset (i, j, l) != 0, in lattice units (lengths in d): returns
    three real [3, 3] tensors (units d^-3, d^-2, d^-1)."""
    R = np.asarray(offset, dtype=np.float64)
    s, w = _cell_nodes(n)
    rho = R[None, :] - s
    rn = np.linalg.norm(rho, axis=1)
    rh = rho / rn[:, None]
    rr = rh[:, :, None] * rh[:, None, :]
    eye = np.eye(3)[None]
    A = (eye - rr) / rn[:, None, None]
    B = (eye - 3.0 * rr) / rn[:, None, None] ** 3
    C = (eye - 3.0 * rr) / rn[:, None, None] ** 2
    delta = (rn - np.linalg.norm(R))[:, None, None]
    T0 = np.tensordot(w, B, axes=(0, 0))
    T1 = np.tensordot(w, C - delta * B, axes=(0, 0))
    T2 = np.tensordot(w, A - delta * C + 0.5 * delta ** 2 * B, axes=(0, 0))
    return T0, T1, T2


_TABLES = {}


def _tables(offset):
    key = tuple(int(v) for v in offset)
    if key not in _TABLES:
        _TABLES[key] = so_tables(key)
    return _TABLES[key]


def green_so(offset, k, d):
    """Interaction tensor for the lattice offset (integers) at spacing d (m):
    G_so of the module docstring for max-norm <= L_NEAR, G~(offset d) beyond."""
    off = np.asarray(offset)
    if np.max(np.abs(off)) > L_NEAR:
        return green_tilde(off * d, k)
    T0, T1, T2 = _tables(off)
    R = np.linalg.norm(off) * d
    return np.exp(1j * k * R) * (-T0 / d ** 3 + 1j * k * T1 / d ** 2 + k ** 2 * T2 / d)


def self_term(k, d):
    """Second-order self term M of the cell (a scalar times I), SI."""
    return (2.0 / 3.0) * (C1 * k ** 2 / d + 1j * k ** 3)


def polarizability_igt_so(alpha_cm, k, d):
    """1 / (1/alpha~_CM - M): the cell's self term to second order in kd."""
    a = np.asarray(alpha_cm, dtype=np.complex128)
    return 1.0 / (1.0 / a - self_term(k, d))


def green_lattice(offsets, k, d):
    """G_so for integer offsets [..., 3] (none zero)."""
    off = np.asarray(offsets)
    flat = off.reshape(-1, 3)
    out = np.empty((len(flat), 3, 3), dtype=np.complex128)
    far = np.max(np.abs(flat), axis=1) > L_NEAR
    if np.any(far):
        out[far] = green_tilde(flat[far] * d, k)
    for i in np.nonzero(~far)[0]:
        out[i] = green_so(flat[i], k, d)
    return out.reshape(off.shape[:-1] + (3, 3))


def dense_matrix_so(idx, k, alpha, d):
    """A = diag(alpha~^{-1}) - G_so over the lattice cells idx [N, 3]
    (integers), size 3N x 3N, dipole-major."""
    idx = np.asarray(idx)
    n = len(idx)
    off = idx[:, None, :] - idx[None, :, :]
    mask = ~np.eye(n, dtype=bool)
    G = np.zeros((n, n, 3, 3), dtype=np.complex128)
    G[mask] = green_lattice(off[mask], k, d)
    A = -G.transpose(0, 2, 1, 3).reshape(3 * n, 3 * n)
    A[np.arange(3 * n), np.arange(3 * n)] += np.repeat(1.0 / np.asarray(alpha), 3)
    return A


def symmetric_components(G):
    """[..., 3, 3] -> [6, ...] in the order of PAIRS."""
    return np.stack([G[..., a, b] for a, b in PAIRS])
