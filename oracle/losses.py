"""Loss and emission probabilities from the dipoles p~ (p = 4 pi eps_h p~).

Volume integrals become sums over dipoles (midpoint rule, P(r) d^3 = p).
All probabilities are returned in eV^-1: P [1/J] * e [J/eV].

  W_enh = -(w/2) Im sum E_a . p                         (Eq. 32, unconjugated dot)
  W_ext = -(w/2) Im sum E_inc . p^*                     (Eq. 17)
  W_abs = (w/2) 4 pi eps0 Re(eps_h) sum |p~|^2 (-Im 1/alpha~_CM)   (Eq. 18, discrete)
  W_sca = (1/2) Re(m_h) eps0 c |k|^4 int |F(n)|^2 dOmega,
          F(n) = sum_j (I - nn) p~_j exp(-i k n . r_j)  (far field of the dipoles)
  P_X   = (2/pi) W_X / (hbar^2 w)                       (Eq. 37, 42, 48)

Discrete readings: W_abs in the Draine form (the absorbed part of
Im(E_exc^* . p) with the radiative-reaction term removed), which closes the
energy budget exactly for a real host; in an absorbing host Re(eps_h) is
used and the value is reported only (Sec. 2.1 calls it ambiguous there).
W_sca in an absorbing host keeps the complex k in the phase and |k|^4, and
drops the path attenuation (Sec. 2.6 says Eq. 42 is qualitative there).
"""
from __future__ import annotations

import numpy as np

from .constants import C_LIGHT, E_CHARGE, EPS0, HBAR
from .green import green_tilde


def _to_prob(W, omega):
    return 2.0 / np.pi * W / (HBAR ** 2 * omega) * E_CHARGE


def p_eels(E_a, p_t, eps_h, omega):
    W = -(omega / 2.0) * 4.0 * np.pi * EPS0 * np.imag(eps_h * np.sum(E_a * p_t))
    return _to_prob(W, omega)


def p_ext(E_inc, p_t, eps_h, omega):
    W = -(omega / 2.0) * 4.0 * np.pi * EPS0 * np.imag(np.sum(E_inc * np.conj(eps_h * p_t)))
    return _to_prob(W, omega)


def p_abs(p_t, alpha_cm, eps_h, omega):
    per = np.sum(np.abs(p_t) ** 2, axis=1) * (-np.imag(1.0 / np.asarray(alpha_cm)))
    W = (omega / 2.0) * 4.0 * np.pi * EPS0 * np.real(eps_h) * np.sum(per)
    return _to_prob(W, omega)


def far_field_amplitude(r, p_t, k, dirs):
    """F(n) [n_dir,3] = sum_j (I - n n) p~_j exp(-i k n.r_j)."""
    ph = np.exp(-1j * k * (dirs @ r.T))          # [n_dir, N]
    s = ph @ p_t                                  # [n_dir, 3]
    return s - dirs * np.sum(dirs * s, axis=1)[:, None]


def p_cl(r, p_t, k, m_h, omega, dirs, weights):
    F = far_field_amplitude(r, p_t, k, dirs)
    W = 0.5 * np.real(m_h) * EPS0 * C_LIGHT * np.abs(k) ** 4 * np.sum(weights * np.sum(np.abs(F) ** 2, axis=1))
    return _to_prob(W, omega)


def p_sca_img(r, p_t, k, eps_h, omega):
    """Scattered power from the induced dipoles by Eq. 12-15 (real k only):
    W_sca = (w/2) 4 pi eps0 eps_h sum_ij p~_i^* Im G~_ij p~_j, with the
    self term Im G~_ii = (2/3) k^3 I (Eq. 15 times 4 pi k^2)."""
    if abs(np.imag(k)) > 0 or abs(np.imag(eps_h)) > 0:
        raise ValueError("the Im-G form needs a non-absorbing host")
    k = float(np.real(k))
    n = len(r)
    R = r[:, None, :] - r[None, :, :]
    off = ~np.eye(n, dtype=bool)
    ImG = np.zeros((n, n, 3, 3))
    ImG[off] = np.imag(green_tilde(R[off], k))
    ImG[~off] = (2.0 / 3.0) * k ** 3 * np.eye(3)
    q = np.einsum("ia,ijab,jb->", np.conj(p_t), ImG, p_t)
    W = (omega / 2.0) * 4.0 * np.pi * EPS0 * np.real(eps_h) * np.real(q)
    return _to_prob(W, omega)


def p_cl_tot(P_EELS, P_ext, P_CL):
    """Particle-related total emission probability P_CL^tot (Eq. 41), in its
    second form: the prefactor of Eq. 37 and 42 times (C_enh - C_ext + C_sca),
    i.e. P_EELS - P_ext + P_CL.  Meaningful in a non-absorbing host (Sec. 2.6);
    it equals P_CL below the Cherenkov threshold, where P_EELS = P_ext."""
    return P_EELS - P_ext + P_CL


def frank_tamm_rate(v: float, m_h: float) -> float:
    """Free-space (particle-free) loss of the electron per unit path length,
    as a probability density in eV^-1 m^-1: Eq. 29 for dW0/dz, turned into a
    probability by the (2/pi) / (hbar^2 w) of Eq. 37, times e.  The omega of
    Eq. 29 cancels: (mu0 q^2 / (4 pi hbar^2)) (1 - c^2 / (v^2 m_h^2)).  Zero at
    and below the threshold beta_h = v m_h / c <= 1 (Eq. 28).  Real host
    index only (W0 diverges in an absorbing host, Sec. 2.5)."""
    from .constants import MU0, Q_ELECTRON
    beta_h = v * m_h / C_LIGHT
    if beta_h <= 1.0:
        return 0.0
    dW0_dz_over_w = MU0 / 8.0 * Q_ELECTRON ** 2 * (1.0 - 1.0 / beta_h ** 2)
    return 2.0 / np.pi * dW0_dz_over_w / HBAR ** 2 * E_CHARGE
