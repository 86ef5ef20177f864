"""Kinematics, host-medium factors and the dipole polarizability.

Readings of the paper used here:
  * time dependence exp(-i omega t): Eq. 1 (curl E = i omega mu0 H) and the
    passive-medium assumption Im eps >= 0 (Sec. 2.1) fix it;
  * m_h = sqrt(eps_h) on the principal branch, 0 <= arg m_h < pi/2 (Sec. 2.1);
  * gamma_h = (1 - beta_h^2)^(-1/2) in the first quadrant (Sec. 2.2, after
    Eq. 24); for real beta_h > 1 this is the limit Im eps_h -> 0+, i.e.
    gamma_h = +i / sqrt(beta_h^2 - 1).
"""
from __future__ import annotations

import numpy as np

from .constants import C_LIGHT, E_CHARGE, HBAR, ME_C2_KEV


def electron_speed(ekin_keV: float) -> float:
    """Relativistic speed for kinetic energy E: gamma = 1 + E / (m_e c^2)."""
    gamma = 1.0 + ekin_keV / ME_C2_KEV
    return C_LIGHT * np.sqrt(1.0 - 1.0 / gamma ** 2)


def kinetic_energy(v: float) -> float:
    """Inverse of electron_speed (keV)."""
    return ME_C2_KEV * (1.0 / np.sqrt(1.0 - (v / C_LIGHT) ** 2) - 1.0)


def omega_of(energy_eV):
    """Angular frequency of a loss energy hbar*omega given in eV."""
    return np.asarray(energy_eV) * E_CHARGE / HBAR


def host_index(eps_h) -> complex:
    """m_h = sqrt(eps_h), principal branch (Sec. 2.1)."""
    return complex(np.sqrt(complex(eps_h)))


def one_over_gamma_h(beta_h: complex) -> complex:
    """s = sqrt(1 - beta_h^2) = 1/gamma_h with gamma_h in the first quadrant
    (Eq. 24 and the branch rule after it).  1 - beta_h^2 has Im <= 0 for
    0 <= arg beta_h < pi/2, so the principal root lies in the fourth
    quadrant; on the real negative axis the root is taken as -i sqrt(|.|)
    (the limit from Im eps_h -> 0+)."""
    a = 1.0 - complex(beta_h) ** 2
    if a.imag == 0.0 and a.real < 0.0:
        return -1j * np.sqrt(-a.real)
    return complex(np.sqrt(a))


def beta_gamma_h(v: float, m_h: complex):
    """beta_h = v m_h / c and gamma_h (Eq. 24)."""
    beta = v / C_LIGHT * complex(m_h)
    s = one_over_gamma_h(beta)
    if abs(s) < 1e-6:
        raise ValueError("beta_h = 1: gamma_h is singular (Eq. 24)")
    return beta, 1.0 / s


def polarizability_cm(m_rel2, d: float):
    """Clausius-Mossotti polarizability in the normalisation alpha~ =
    alpha / (4 pi eps_h): (3/(4 pi)) d^3 (m^2 - 1)/(m^2 + 2), where m is the
    refractive index relative to the host (Eq. 2), m^2 = eps_p / eps_h."""
    m2 = np.asarray(m_rel2, dtype=np.complex128)
    return 3.0 / (4.0 * np.pi) * d ** 3 * (m2 - 1.0) / (m2 + 2.0)


def polarizability_rr(alpha_cm, k: complex):
    """Radiative-reaction correction: alpha~ = alpha~_CM / (1 - (2/3) i k^3
    alpha~_CM), k the (possibly complex) host wavenumber of Eq. 4.  The
    (2/3) k^3 is the self term of Im G~ (the limit of Eq. 15, scaled by
    4 pi k^2)."""
    a = np.asarray(alpha_cm, dtype=np.complex128)
    return a / (1.0 - (2.0 / 3.0) * 1j * k ** 3 * a)


def scaled_kinetic_energy(ekin_keV: float, eps_h: float) -> float:
    """Eq. 47: kinetic energy whose speed is m_h times the speed at ekin."""
    e0 = ME_C2_KEV
    e = ekin_keV
    return e0 * ((e + e0) / np.sqrt(e0 ** 2 - (eps_h - 1.0) * e * (2.0 * e0 + e)) - 1.0)


def vacuum_equivalent(ekin_keV: float, eps_h: float, energy_eV: float, length_rule: bool = False,
                      ultrarelativistic: bool = False) -> dict:
    """Sec. 2.7: a vacuum problem whose probabilities give those of a particle
    in a real host eps_h.  Eq. 43-44 rescale the indices by eta and every
    length by xi (k by 1/xi); then omega -> xi eta omega, v -> eta v and
    P -> P / xi.  With eta = m_h the host becomes vacuum:
      * xi = 1 (Eq. 45): same lattice, loss energy m_h hbar omega;
      * xi = 1/m_h (Eq. 46): lengths times m_h, same loss energy, P / m_h.
    The particle permittivity becomes eps_p(omega) / eps_h (m_p -> m_p / eta,
    taken at the original frequency) and the kinetic energy follows Eq. 47.
    Both need beta_h < 1.  For beta_h > 1, Eq. S16 (approximate, from the
    quasi-static field of Eq. S15) sets v = c in the vacuum problem and
    divides its probabilities by beta_h^2.
    Returns ekin_keV (inf for v = c), energy_eV, length_scale, eps_p_scale
    and p_scale with P_host = p_scale * P_vacuum."""
    if not (eps_h > 0 and ekin_keV > 0 and energy_eV > 0):
        raise ValueError("vacuum equivalence needs a real positive eps_h")
    m_h = float(np.sqrt(eps_h))
    beta_h = electron_speed(ekin_keV) * m_h / C_LIGHT
    eta = m_h
    xi = 1.0 / m_h if length_rule else 1.0
    out = {"energy_eV": xi * eta * energy_eV, "length_scale": 1.0 / xi, "eps_p_scale": 1.0 / eta ** 2,
           "p_scale": xi}
    if ultrarelativistic:
        if not beta_h > 1.0:
            raise ValueError("Eq. S16 applies above the Cherenkov threshold")
        out["ekin_keV"] = float("inf")
        out["p_scale"] = xi / beta_h ** 2
    else:
        if not beta_h < 1.0:
            raise ValueError("no vacuum equivalent at or above the Cherenkov threshold (v m_h >= c)")
        out["ekin_keV"] = float(scaled_kinetic_energy(ekin_keV, eps_h))
    return out
