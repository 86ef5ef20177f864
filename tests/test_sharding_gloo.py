"""Multi-rank host logic on CPU (gloo, world size 2): the energy blocks of
all ranks cover every energy exactly once, the weak-scaling beam sets are
distinct per rank, and a spectrum split by energy blocks (each rank solving
its block with the oracle) gathers to the single-rank result.  No GPU and no
data-path collective are involved: only results travel between ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2208_01348_gb300 import sharding


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n_energy, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    a, b = sharding.energy_block(n_energy, rank, world)
    beams = sharding.weak_scaling_beams([(20.0, 0.0), (25.0, 1.0)], rank)
    got = [None] * world
    dist.all_gather_object(got, (a, b, beams))
    if rank == 0:
        out.put(got)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("n_energy", [200, 7, 1])
def test_energy_blocks_cover_once_across_two_ranks(n_energy):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n_energy, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    covered = []
    for a, b, _ in got:
        covered += list(range(a, b))
    assert covered == list(range(n_energy))
    assert got[0][2] != got[1][2]


def _solve_block(rank, world, port, out):
    import numpy as np
    from oracle import run
    from paper_2208_01348_gb300 import inputs as I
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = I.reduced(I.config_spectrum(), 4 / 32, n_energy=5)
    a, b = sharding.energy_block(len(w.energies_eV), rank, world)
    mine = {ie: run.solve_workload_point(w, ie, 0, want_cl=False)["P_EELS"] for ie in range(a, b)}
    got = [None] * world
    dist.all_gather_object(got, mine)
    if rank == 0:
        merged = {}
        for g in got:
            merged.update(g)
        out.put([float(np.real(merged[ie])) for ie in sorted(merged)])
    dist.barrier()
    dist.destroy_process_group()


def test_energy_split_gathers_to_the_single_rank_spectrum():
    import numpy as np
    from oracle import run
    from paper_2208_01348_gb300 import inputs as I
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_solve_block, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    split = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    w = I.reduced(I.config_spectrum(), 4 / 32, n_energy=5)
    whole = [float(np.real(run.solve_workload_point(w, ie, 0, want_cl=False)["P_EELS"]))
             for ie in range(len(w.energies_eV))]
    assert split == whole


def test_block_sizes_balanced():
    for n in (0, 1, 5, 200):
        for w in (1, 2, 3, 8):
            sizes = [b - a for a, b in (sharding.energy_block(n, r, w) for r in range(w))]
            assert sum(sizes) == n and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharding.energy_block(10, 2, 2)
