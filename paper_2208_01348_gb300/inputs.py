"""Seeded synthetic inputs shaped like the paper's workloads.

This module only *describes* problems: occupancy grids, dipole spacing,
electron energy, beam positions, loss energies and the permittivity tables
that stand in for the paper's tabulated optical data (the Drude model used
here is an input model, not part of the DDA method).  It holds none of the
method's arithmetic (no fields, no Green's tensor, no solve, no losses), so
both the CUDA path and the CPU oracle may import it.

Geometry convention (shared by every consumer): a lattice of nx*ny*nz cubic
cells of edge d, centred at the origin, x fastest in the occupancy array.
Cell (ix, iy, iz) has its centre at ((ix + 1/2) - nx/2) * d along x (and the
same along y, z).  An occupancy value of 0 means empty; k > 0 means the cell
holds material k (1-based index into the permittivity table).

The workloads follow the shapes the paper simulates: spheres scanned in loss
energy (Sec. 3.2-3.3, Figs. 2-8), a rod-like particle in a glass-like host
scanned with the beam (Sec. 3.4, Fig. 10) and a dense Cherenkov host
(Sec. 3.3-3.4, Figs. 8-9).  The paper's optical data tables are not
available, so Drude permittivities stand in for gold and silver.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# ---------------------------------------------------------------------------
# Material models (inputs).  eps(E) = eps_inf - Ep^2 / (E (E + i G)), with
# energies in eV.  Im eps > 0 for E > 0 under the exp(-i omega t) convention.
# ---------------------------------------------------------------------------
DRUDE_AU = (9.5, 8.95, 0.069)      # eps_inf, hbar*omega_p [eV], hbar*gamma [eV]
DRUDE_AG = (3.7, 9.1, 0.018)


def drude(energy_eV, params=DRUDE_AU) -> np.ndarray:
    eps_inf, ep, g = params
    e = np.asarray(energy_eV, dtype=np.float64)
    return eps_inf - ep * ep / (e * (e + 1j * g))


# ---------------------------------------------------------------------------
# Geometry inputs
# ---------------------------------------------------------------------------
def _centres(n: int, d: float) -> np.ndarray:
    return ((np.arange(n) + 0.5) - n / 2.0) * d


def sphere_occupancy(n: int, diameter_nm: float, material: int = 1) -> np.ndarray:
    """n^3 cells of edge diameter/n; a cell is occupied when its centre lies
    inside the sphere.  Returns uint8 [nz][ny][nx] (x fastest)."""
    d = diameter_nm / n
    c = _centres(n, d)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    inside = x * x + y * y + z * z <= (diameter_nm / 2.0) ** 2
    return (inside * material).astype(np.uint8)


def box_occupancy(nx: int, ny: int, nz: int, material: int = 1) -> np.ndarray:
    return np.full((nz, ny, nx), material, dtype=np.uint8)


@dataclasses.dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    d_nm: float
    occ: np.ndarray                     # uint8 [nz][ny][nx]

    @property
    def n_occupied(self) -> int:
        return int(np.count_nonzero(self.occ))


@dataclasses.dataclass
class Workload:
    """One EELS/CL job: a particle, a host, an electron and the points to
    solve (energies x beams)."""
    name: str
    grid: Grid
    ekin_keV: float
    energies_eV: np.ndarray             # [n_energy]
    eps_p: np.ndarray                   # complex [n_energy][n_mat]
    eps_h: np.ndarray                   # complex [n_energy]
    beams_nm: np.ndarray                # [n_beam][2] = (x0, y0); electron along +z, z0 = 0
    eps_it: float = 1e-8
    n_dir: int = 2562

    @property
    def n_points(self) -> int:
        return len(self.energies_eV) * len(self.beams_nm)


def _const_host(eps_h: complex, n: int) -> np.ndarray:
    return np.full(n, complex(eps_h), dtype=np.complex128)


def config_small_sphere() -> Workload:
    """12^3 sphere, D = 20 nm, Drude gold, vacuum, 100 keV, b = 15 nm, 2.4 eV."""
    occ = sphere_occupancy(12, 20.0)
    e = np.array([2.4])
    return Workload("sphere12_au_vacuum_2.4eV", Grid(12, 12, 12, 20.0 / 12, occ), 100.0, e,
                    drude(e)[:, None], _const_host(1.0, 1), np.array([[15.0, 0.0]]), 1e-8)


def config_spectrum(n_energy: int = 200) -> Workload:
    """32^3 sphere, D = 30 nm, Drude gold in n = 1.45, 120 keV, b = 20 nm,
    200 energies 1.0-4.0 eV (an EELS spectrum, Figs. 2-7)."""
    occ = sphere_occupancy(32, 30.0)
    e = np.linspace(1.0, 4.0, n_energy)
    return Workload("sphere32_au_n1.45_spectrum", Grid(32, 32, 32, 30.0 / 32, occ), 120.0, e,
                    drude(e)[:, None], _const_host(1.45 ** 2, n_energy),
                    np.array([[20.0, 0.0]]), 1e-8)


def rod_raster_beams(nbx: int = 32, nby: int = 32, pitch: float = 2.0,
                     x_start: float = 22.0, y_start: float = -31.0) -> np.ndarray:
    bx = x_start + pitch * np.arange(nbx)
    by = y_start + pitch * np.arange(nby)
    xx, yy = np.meshgrid(bx, by, indexing="ij")
    return np.stack([xx.ravel(), yy.ravel()], axis=1)


def config_rod_map(n_energy: int = 64, nbx: int = 32, nby: int = 32) -> Workload:
    """24x24x72 box (40x40x120 nm) of Drude gold in n = 1.45, 100 keV,
    32x32 beams on a 2 nm raster beside the rod, 64 energies 1.2-2.6 eV
    (a plasmon map, Fig. 10)."""
    occ = box_occupancy(24, 24, 72)
    e = np.linspace(1.2, 2.6, n_energy)
    return Workload("rod24x24x72_au_n1.45_map", Grid(24, 24, 72, 40.0 / 24, occ), 100.0, e,
                    drude(e)[:, None], _const_host(1.45 ** 2, n_energy),
                    rod_raster_beams(nbx, nby), 1e-8)


def config_cherenkov(n_energy: int = 100) -> Workload:
    """64^3 sphere, D = 100 nm, Drude silver in eps_h = 4 + 0.05i, 200 keV
    (beta_h > 1), b = 60 nm, 100 energies 1.5-4.0 eV (Figs. 8-9)."""
    occ = sphere_occupancy(64, 100.0)
    e = np.linspace(1.5, 4.0, n_energy)
    return Workload("sphere64_ag_cherenkov", Grid(64, 64, 64, 100.0 / 64, occ), 200.0, e,
                    drude(e, DRUDE_AG)[:, None], _const_host(4.0 + 0.05j, n_energy),
                    np.array([[60.0, 0.0]]), 1e-8)


def reduced(w: Workload, n_scale: float, n_energy: Optional[int] = None,
            beams: Optional[np.ndarray] = None) -> Workload:
    """Same physics on a coarser lattice (same particle size, fewer cells)."""
    g = w.grid
    nx, ny, nz = (max(2, int(round(v * n_scale))) for v in (g.nx, g.ny, g.nz))
    size = (g.nx * g.d_nm, g.ny * g.d_nm, g.nz * g.d_nm)
    d = size[0] / nx
    if np.all(g.occ > 0):
        occ = box_occupancy(nx, ny, nz)
    else:
        occ = sphere_occupancy(nx, size[0])
    e = w.energies_eV if n_energy is None else w.energies_eV[np.linspace(0, len(w.energies_eV) - 1, n_energy).astype(int)]
    idx = np.searchsorted(w.energies_eV, e)
    return dataclasses.replace(w, name=w.name + f"_reduced{nx}", grid=Grid(nx, ny, nz, d, occ),
                               energies_eV=e, eps_p=w.eps_p[idx], eps_h=w.eps_h[idx],
                               beams_nm=w.beams_nm if beams is None else beams)


# ---------------------------------------------------------------------------
# Serving stream (Poisson arrivals), seeded.
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Request:
    t_arrival_s: float
    workload: Workload


def serving_stream(n_requests: int = 200, rate_per_s: float = 20.0, seed: int = 20261203,
                   n_min: int = 16, n_max: int = 96, beams_max: int = 256,
                   energies_min: int = 8, energies_max: int = 128) -> List[Request]:
    """Requests with exponential inter-arrival times; each picks a sphere or a
    rod (ceil(n/3) x ceil(n/3) x n box), gold or silver, a host from
    {1.0, 2.1, 4.0+0.05i}, 1..beams_max beams placed 2-20 nm outside the
    particle and energies_min..energies_max loss energies in 1.0-4.0 eV."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    d = 1.25
    hosts = [1.0 + 0j, 2.1 + 0j, 4.0 + 0.05j]
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        n = int(rng.integers(n_min, n_max + 1))
        shape = "sphere" if rng.random() < 0.5 else "rod"
        mat = DRUDE_AU if rng.random() < 0.5 else DRUDE_AG
        eps_h = hosts[int(rng.integers(0, 3))]
        nb = int(rng.integers(1, beams_max + 1))
        ne = int(rng.integers(energies_min, energies_max + 1))
        if shape == "sphere":
            grid = Grid(n, n, n, d, sphere_occupancy(n, n * d))
            half_x = n * d / 2.0
        else:
            m = -(-n // 3)
            grid = Grid(m, m, n, d, box_occupancy(m, m, n))
            half_x = m * d / 2.0
        gap = rng.uniform(2.0, 20.0, size=nb)
        yoff = rng.uniform(-half_x, half_x, size=nb) if shape == "rod" else np.zeros(nb)
        if shape == "rod":
            beams = np.stack([half_x + gap, yoff], axis=1)
        else:
            ang = rng.uniform(0, 2 * math.pi, size=nb)
            rad = half_x + gap
            beams = np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)
        e = np.linspace(1.0, 4.0, ne)
        w = Workload(f"req{i}_{shape}{n}", grid, 100.0, e, drude(e, mat)[:, None],
                     _const_host(eps_h, ne), beams, 1e-8)
        out.append(Request(t, w))
    return out


def random_complex(shape: Sequence[int], seed: int, dtype=np.complex128) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(dtype)
