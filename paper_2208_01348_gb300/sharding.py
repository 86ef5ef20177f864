"""Partition of independent (energy, beam) points across ranks.

Every (energy, beam) point is an independent dipole system, so ranks never
exchange data on the solve path: each rank takes a contiguous block of
energies (all beams of an energy stay together, since they share one
D-hat) and solves it alone.  Only timing and results travel between ranks.
"""
from __future__ import annotations

from typing import List, Tuple


def energy_block(n_energy: int, rank: int, world: int) -> Tuple[int, int]:
    """[start, stop) of the energies owned by `rank`: contiguous blocks whose
    sizes differ by at most one."""
    if world <= 0 or not (0 <= rank < world):
        raise ValueError("rank must be in [0, world)")
    base, extra = divmod(n_energy, world)
    start = rank * base + min(rank, extra)
    stop = start + base + (1 if rank < extra else 0)
    return start, stop


def weak_scaling_beams(base_beams, rank: int, shift_nm: float = 0.5) -> List[Tuple[float, float]]:
    """Weak scaling: every rank solves a full workload of its own; rank r's
    beams are shifted by r * shift_nm along y, so the ranks' points are
    distinct while the per-rank work stays the same."""
    return [(float(x), float(y) + rank * shift_nm) for x, y in base_beams]
