"""Physical constants, SI (CODATA 2018; e, hbar-derived and c exact)."""
E_CHARGE = 1.602176634e-19        # C
HBAR = 1.054571817e-34            # J s
C_LIGHT = 299792458.0             # m / s
EPS0 = 8.8541878128e-12           # F / m
MU0 = 1.0 / (EPS0 * C_LIGHT ** 2)  # H / m
ME_C2_KEV = 510.99895000          # electron rest energy, keV
Q_ELECTRON = -E_CHARGE            # the moving charge q of Sec. 2.2
NM = 1e-9
