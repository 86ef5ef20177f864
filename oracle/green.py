"""Green's tensor, the dense DDA matrix and a plain FFT convolution.

Normalisation.  With p = 4 pi eps_h p~ (eps_h absolute) and
G~(R) = 4 pi k^2 G(R), the discrete form of Eq. 8 (point dipoles, field at
dipole i excluding its own) reads

    alpha~_i^{-1} p~_i - sum_{j != i} G~(r_i - r_j) p~_j = E_inc(r_i),

because omega^2 mu0 G / (4 pi ...) p = G~ p~ (omega^2 mu0 = k^2 / eps_h).
For R != 0, Eq. 5 gives

    G~(R) = exp(ikR)/R [ k^2 (I - RR/R^2) - (1 - ikR)/R^2 (I - 3 RR/R^2) ].

Component order for symmetric tensors: xx, xy, xz, yy, yz, zz.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

PAIRS = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))


def green_tilde(R, k):
    """G~ for separation vectors R [...,3] (m), complex k; returns [...,3,3].
    R must be non-zero."""
    R = np.asarray(R, dtype=np.float64)
    rn = np.linalg.norm(R, axis=-1)
    rh = R / rn[..., None]
    rr = rh[..., :, None] * rh[..., None, :]
    eye = np.eye(3)
    ph = np.asarray(np.exp(1j * k * rn) / rn)
    t1 = k ** 2 * (eye - rr)
    t2 = np.asarray((1.0 - 1j * k * rn) / rn ** 2)[..., None, None] * (eye - 3.0 * rr)
    return ph[..., None, None] * (t1 - t2)


def dense_matrix(r, k, alpha):
    """A = diag(alpha~^{-1}) - G~, size 3N x 3N, dipole-major (row 3i + a)."""
    n = len(r)
    R = r[:, None, :] - r[None, :, :]
    off = ~np.eye(n, dtype=bool)
    G = np.zeros((n, n, 3, 3), dtype=np.complex128)
    G[off] = green_tilde(R[off], k)
    A = -G.transpose(0, 2, 1, 3).reshape(3 * n, 3 * n)
    A[np.arange(3 * n), np.arange(3 * n)] += np.repeat(1.0 / np.asarray(alpha), 3)
    return A


def dense_matrix_loops(r, k, alpha):
    """The same matrix written with explicit loops (tiny N only)."""
    n = len(r)
    A = np.zeros((3 * n, 3 * n), dtype=np.complex128)
    for i in range(n):
        for a in range(3):
            A[3 * i + a, 3 * i + a] = 1.0 / alpha[i]
        for j in range(n):
            if i == j:
                continue
            g = green_tilde(r[i] - r[j], k)
            for a in range(3):
                for b in range(3):
                    A[3 * i + a, 3 * j + b] = -g[a, b]
    return A


class FFTOperator:
    """y = A x by zero-padded circular convolution on the lattice.

    Dipoles sit on lattice cells idx [N,3] (integers, 0 <= idx < n) with
    spacing d.  The separations (i - j) d with |i - j| < n per axis fit in a
    period of m = 2 n per axis, so a circular convolution of length m
    reproduces the dense sum exactly (G~ is set to 0 at zero separation and
    at the unused wrap index n)."""

    def __init__(self, idx, n_axes, d, k, alpha, workers=-1, interaction="point"):
        self.idx = np.asarray(idx)
        self.n = tuple(int(v) for v in n_axes)
        self.m = tuple(2 * v for v in self.n)
        self.k = k
        self.alpha = np.asarray(alpha, dtype=np.complex128)
        self.workers = workers
        grids = []
        for nv, mv in zip(self.n, self.m):
            s = np.arange(mv, dtype=np.float64)
            s[s > nv] -= mv          # indices 0..n-1 -> +, n+1..m-1 -> negative
            grids.append(s * d)
        X, Y, Z = np.meshgrid(*grids, indexing="ij")
        R = np.stack([X, Y, Z], axis=-1)
        rn = np.linalg.norm(R, axis=-1)
        valid = rn > 0
        for ax, nv in enumerate(self.n):
            sl = [slice(None)] * 3
            sl[ax] = nv
            valid[tuple(sl)] = False
        G = np.zeros(self.m + (3, 3), dtype=np.complex128)
        if interaction == "igt_so":
            from . import igt
            offsets = np.rint(R[valid] / d).astype(int)
            G[valid] = igt.green_lattice(offsets, k, d)
        else:
            G[valid] = green_tilde(R[valid], k)
        self.D = np.stack([sfft.fftn(G[..., a, b], workers=workers) for a, b in PAIRS])

    def conv(self, x):
        """sum_{j != i} G~(r_i - r_j) x_j for x [N,3]."""
        X = np.zeros((3,) + self.m, dtype=np.complex128)
        ii = tuple(self.idx.T)
        for a in range(3):
            X[a][ii] = x[:, a]
        Xf = np.stack([sfft.fftn(X[a], workers=self.workers) for a in range(3)])
        D = self.D
        full = {}
        for c, (a, b) in enumerate(PAIRS):
            full[(a, b)] = D[c]
            full[(b, a)] = D[c]
        out = np.empty((len(x), 3), dtype=np.complex128)
        for a in range(3):
            Yf = full[(a, 0)] * Xf[0] + full[(a, 1)] * Xf[1] + full[(a, 2)] * Xf[2]
            out[:, a] = sfft.ifftn(Yf, workers=self.workers)[ii]
        return out

    def matvec(self, x):
        """A x = alpha~^{-1} x - conv(x), x [N,3]."""
        return x / self.alpha[:, None] - self.conv(x)
