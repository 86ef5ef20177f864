"""Benchmark: EELS/CL (energy, beam) points per second on one GB300.

Default workload: the 30 nm Drude-gold sphere on a 32^3 lattice (17,256
dipoles, 64^3 padded FFT) in an n = 1.45 host, 120 keV electron at b = 20 nm,
200 loss energies 1.0-4.0 eV -- one EELS + CL spectrum per step, solved in
the mixed path (FP32 QMR to 1e-5 inside FP64 refinement to 1e-8; FP64
incident field and loss sums; CL far field on 2562 directions).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload ...]

A step is one eels_solve over every point of the workload.  `value` is
device-timed (CUDA events on the library's stream, the lattice already set);
`e2e` adds the host->device copy of the inputs (eels_set_grid + host input
arrays) and the device->host copy of the outputs through the same C ABI.
Under torchrun every rank solves its own copy of the workload (weak scaling,
no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2208_01348_gb300 import inputs as I  # noqa: E402

METRIC = "EELS points/s at rel.err≤1e-4 vs FP64 oracle; matvec HBM-roofline %; p50/p99 ms"

WORKLOADS = {
    "spectrum": lambda: I.config_spectrum(),
    "small": lambda: I.config_small_sphere(),
    "cherenkov": lambda: I.config_cherenkov(),
    "rod": lambda: I.config_rod_map(n_energy=8, nbx=32, nby=32),
}
# a bounded oracle sample per workload: (energy index, beam index)
CPU_SAMPLE = {"spectrum": (100, 0), "small": (0, 0), "cherenkov": (50, 0), "rod": (4, 0)}

# ncu DRAM traffic (read + write bytes) of one matvec launch set, per system,
# measured on the 64^3-FFT kernels of the spectrum workload whose sources hash
# to TRAFFIC_SRC_HASH; reported as null for other workloads (other FFT sizes,
# other kernels) and when the kernel sources differ from the measured ones.
TRAFFIC_BYTES_PER_SYSTEM = 13_713_772       # profiles/fft_matvec_sphere32_64systems.md
TRAFFIC_SRC_HASH = "730a9a2c5c0e6dec"
TRAFFIC_WORKLOAD = "spectrum"


def kernel_src_hash() -> str:
    h = hashlib.sha256()
    for f in ("k_fft.cu", "fft.cuh", "kernels.h", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2208_01348_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(wname: str, w):
    """The oracle (FP64, scipy FFT convolution + GMRES to 1e-8) on one point."""
    from oracle import run
    ie, ib = CPU_SAMPLE[wname]
    t0 = time.perf_counter()
    g = w.grid
    pt = run.setup(g.nx, g.ny, g.nz, g.d_nm, g.occ, w.energies_eV[ie], w.eps_p[ie], w.eps_h[ie], w.beams_nm[ib],
                   ekin_keV=w.ekin_keV)
    p, _ = run.solve_fft(pt, rtol=1e-8)
    run.observables(pt, p)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": "points/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"1 point of {w.name}: energy {w.energies_eV[ie]:.3f} eV (index {ie}), beam {ib}; "
                      f"oracle per-point time varies strongly with energy (GMRES iterations)",
            "seconds": dt}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import run
    ie, ib = CPU_SAMPLE[args.workload]
    g = w.grid

    def step():
        pt = run.setup(g.nx, g.ny, g.nz, g.d_nm, g.occ, w.energies_eV[ie], w.eps_p[ie], w.eps_h[ie], w.beams_nm[ib],
                       ekin_keV=w.ekin_keV)
        p, _ = run.solve_fft(pt, rtol=1e-8)
        run.observables(pt, p)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    v = 1.0 / dt
    sample = f"1 point per step of {w.name}: energy {w.energies_eV[ie]:.3f} eV (index {ie}), beam {ib}"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "points/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "oracle": "FP64 numpy/scipy: FFT convolution + GMRES to 1e-8"},
        "cpu_baseline": {"value": v, "unit": "points/s", "cores": os.cpu_count(), "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_matvec_only(args):
    """The FFT matvec alone (the dominant kernel set) on S systems of the
    workload, energies spread over its spectrum; used for ncu captures."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2208_01348_gb300 import eelsdda as dd
    w = WORKLOADS[args.workload]()
    S = args.matvec_only
    stream = torch.cuda.current_stream()
    ctx = dd.eels_create(0, stream.cuda_stream)
    dd.eels_set_grid(ctx, w.grid.occ, w.grid.d_nm)
    idx = np.linspace(0, len(w.energies_eV) - 1, S).astype(int)
    dd.eels_prepare_operator(ctx, w.energies_eV[idx], w.eps_p[idx], w.eps_h[idx])
    n = dd.eels_num_dipoles(ctx)
    mx, my, mz = dd.eels_padded_dims(ctx)
    prec = dd.EELS_MIXED if args.precision == "mixed" else dd.EELS_FP64
    dt = torch.complex64 if prec == dd.EELS_MIXED else torch.complex128
    x = torch.randn(S, 3, n, dtype=dt, device="cuda")
    y = torch.empty_like(x)
    for _ in range(4):
        dd.eels_matvec_dev(ctx, prec, x.data_ptr(), y.data_ptr(), S, stream.cuda_stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.matvec_reps):
        dd.eels_matvec_dev(ctx, prec, x.data_ptr(), y.data_ptr(), S, stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.matvec_reps
    s = 8 if prec == dd.EELS_MIXED else 16
    M, Mr = mx * my * mz, (mx // 2 + 1) * (my // 2 + 1) * (mz // 2 + 1)
    alg = S * (6 * M + 6 * Mr + 6 * n) * s
    peak, kind = measured_peaks()
    print(json.dumps({"workload": w.name, "systems": S, "precision": args.precision, "ms_per_matvec": ms,
                      "alg_bytes": alg, "achieved_gbs": alg / (ms * 1e-3) / 1e9, "peak_gbs": peak, "peak_kind": kind,
                      "frac": alg / (ms * 1e-3) / 1e9 / peak}))
    dd.eels_destroy(ctx)


SERVE_STREAM = dict(rate_per_s=20.0, seed=20261203, n_min=12, n_max=32, beams_max=4, energies_min=4, energies_max=16)



def run_serve(args):
    """Serving stream: seeded Poisson arrivals (mean 20/s) of sphere / rod
    requests (Drude gold or silver, host from {1.0, 2.1, 4.0+0.05i}) admitted
    by footprint and run concurrently; bounded to args.serve_requests
    requests with lattices 12-32 cells, 1-4 beams and 4-16 energies so a
    pass ends within minutes."""
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable":
                              "the serving stream has no CPU reference beyond the per-point oracle"}))
        return
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2208_01348_gb300 import eelsdda as dd
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    reqs = I.serving_stream(n_requests=args.serve_requests, **SERVE_STREAM)
    warm = I.serving_stream(n_requests=3, **dict(SERVE_STREAM, seed=7))

    def one_pass(stream):
        srv = dd.eels_server_create(device=local, max_concurrent=args.serve_concurrency)
        t0 = time.perf_counter()
        ids = []
        for r in stream:
            dt = r.t_arrival_s - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            w = r.workload
            o = dd.eels_default_opts(ekin_keV=w.ekin_keV, eps_it=1e-8, n_dir=w.n_dir)
            ids.append((dd.eels_server_submit(srv, w.grid.occ, w.grid.d_nm, o, w.energies_eV, w.eps_p, w.eps_h,
                                              w.beams_nm), w))
        lat, pts, t_first, t_last = [], 0, None, 0.0
        for j, w in ids:
            code, out, info = dd.eels_server_wait(srv, j, len(w.energies_eV), len(w.beams_nm))
            assert code in (dd.EELS_OK, dd.EELS_E_NOT_CONVERGED), code
            lat.append((info["t_end"] - info["t_submit"]) * 1e3)
            pts += w.n_points
            t_first = info["t_submit"] if t_first is None else min(t_first, info["t_submit"])
            t_last = max(t_last, info["t_end"])
        stats = dd.eels_server_stats(srv)
        dd.eels_server_destroy(srv)
        return pts, t_last - t_first, lat, stats

    for _ in range(max(1, args.warmup)):
        one_pass(warm)
    l0 = dd.eels_kernel_launches()
    with ClockSampler(local) as clk:
        pts, span, lat, stats = one_pass(reqs)
    launches = dd.eels_kernel_launches() - l0
    if rank != 0:
        return
    value = pts / span
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": 1, "steps": 1, "warmup": args.warmup,
        "ms_per_step": span * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic seeded request stream",
        "config": {"workload": f"serving stream: {len(reqs)} requests, Poisson 20/s, lattices 12-32, "
                               f"1-4 beams, 4-16 energies, {pts} points", "concurrency": args.serve_concurrency,
                   "running_max": stats["running_max"]},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(np.max(lat))},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                "note": "requests enter and leave through host buffers; the value above is already end to end"},
        "gpu_launches": int(launches), "clocks": clk.summary(),
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="spectrum", choices=sorted(WORKLOADS) + ["serve"])
    ap.add_argument("--matvec-only", type=int, default=0,
                    help="time only the FFT matvec on this many systems of the workload (profiling)")
    ap.add_argument("--serve-requests", type=int, default=16)
    ap.add_argument("--serve-concurrency", type=int, default=8)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--solver", default="qmr2", choices=["qmr2", "qmr", "bicgstab"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-sample", type=int, default=5,
                    help="energies of the plain FP64 single-system comparison (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--matvec-reps", type=int, default=20)
    args = ap.parse_args()
    if args.workload == "serve":
        run_serve(args)
        return
    if args.matvec_only:
        run_matvec_only(args)
        return
    w = WORKLOADS[args.workload]()
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2208_01348_gb300 import eelsdda as dd

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist

    def barrier():
        if dist:
            dist.barrier()

    if world > 1:
        # weak scaling: every rank solves a full workload of its own (distinct
        # beam positions, same amount of work); no data moves between ranks
        from paper_2208_01348_gb300 import sharding
        w.beams_nm = np.array(sharding.weak_scaling_beams(w.beams_nm, rank))
    stream = torch.cuda.current_stream()
    ctx = dd.eels_create(local, stream.cuda_stream)
    g = w.grid
    prec = dd.EELS_MIXED if args.precision == "mixed" else dd.EELS_FP64
    opts = dd.eels_default_opts(ekin_keV=w.ekin_keV, precision=prec, eps_it=1e-8, eps_inner=1e-5, n_dir=w.n_dir,
                                solver={"qmr2": dd.EELS_QMR2, "qmr": dd.EELS_QMR, "bicgstab": dd.EELS_BICGSTAB}[args.solver])
    dd.eels_set_grid(ctx, g.occ, g.d_nm)

    def step():
        return dd.eels_solve(ctx, opts, w.energies_eV, w.eps_p, w.eps_h, w.beams_nm, want_cl=True)

    for _ in range(args.warmup):
        res = step()
    assert res.converged.all(), "warm-up solve did not converge"
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = dd.eels_kernel_launches()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            res = step()
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = dd.eels_kernel_launches() - l0
    barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    pts = w.n_points * world
    value = pts / (ms * 1e-3)
    clocks = clk.summary()

    # end to end through the host API: lattice upload + host inputs + host outputs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        dd.eels_set_grid(ctx, g.occ, g.d_nm)
        r2 = step()
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.e2e_steps
    if dist:
        t = torch.tensor([e2e_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    h2d = g.occ.nbytes + w.energies_eV.nbytes + w.eps_p.nbytes + w.eps_h.nbytes + w.beams_nm.nbytes
    d2h = 4 * w.n_points * 8 + w.n_points * 24

    # roofline of the FFT matvec (the dominant kernel set) on this workload's systems
    S = len(w.energies_eV)
    tiles = dd.eels_tile_widths(ctx)
    dd.eels_prepare_operator(ctx, w.energies_eV, w.eps_p, w.eps_h)
    n = dd.eels_num_dipoles(ctx)
    mx, my, mz = dd.eels_padded_dims(ctx)
    x = torch.randn(S, 3, n, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    for _ in range(3):
        dd.eels_matvec_dev(ctx, dd.EELS_MIXED, x.data_ptr(), y.data_ptr(), S, stream.cuda_stream)
    torch.cuda.synchronize()
    m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    m0.record(stream)
    for _ in range(args.matvec_reps):
        dd.eels_matvec_dev(ctx, dd.EELS_MIXED, x.data_ptr(), y.data_ptr(), S, stream.cuda_stream)
    m1.record(stream)
    torch.cuda.synchronize()
    mv_ms = m0.elapsed_time(m1) / args.matvec_reps
    M = mx * my * mz
    Mr = (mx // 2 + 1) * (my // 2 + 1) * (mz // 2 + 1)
    alg_bytes = S * (6 * M + 6 * Mr + 6 * n) * 8      # complex64, one beam per energy (B = 1)
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (mv_ms * 1e-3) / 1e9
    traffic = None
    if (TRAFFIC_BYTES_PER_SYSTEM is not None and args.workload == TRAFFIC_WORKLOAD
            and TRAFFIC_SRC_HASH == kernel_src_hash()):
        traffic = TRAFFIC_BYTES_PER_SYSTEM * S

    # the plain FP64 path, one system per solve, on a sample of the energies
    # (first beam): its points/s, and how far the mixed results are from it
    fp64_cmp = None
    if prec == dd.EELS_MIXED and world == 1 and args.fp64_sample > 0:
        idx = np.unique(np.linspace(0, len(w.energies_eV) - 1, args.fp64_sample).round().astype(int))
        o64 = dd.eels_default_opts(ekin_keV=w.ekin_keV, precision=dd.EELS_FP64, eps_it=1e-8, n_dir=w.n_dir,
                                   max_batch=1)
        dd.eels_set_grid(ctx, g.occ, g.d_nm)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r64 = dd.eels_solve(ctx, o64, w.energies_eV[idx], w.eps_p[idx], w.eps_h[idx], w.beams_nm[:1], want_cl=True)
        torch.cuda.synchronize()
        v64 = len(idx) / (time.perf_counter() - t0)
        rel_e = np.abs(res.p_eels[idx, 0] - r64.p_eels[:, 0]) / np.abs(r64.p_eels[:, 0])
        rel_c = np.abs(res.p_cl[idx, 0] - r64.p_cl[:, 0]) / np.abs(r64.p_cl[:, 0])
        fp64_cmp = {"value": v64, "unit": "points/s",
                    "sample": f"energies {idx.tolist()} of {w.name}, beam 0, one system per solve, eps 1e-8",
                    "mixed_over_fp64": value / v64, "p_eels_max_rel_diff": float(rel_e.max()),
                    "p_cl_max_rel_diff": float(rel_c.max())}
    dd.eels_destroy(ctx)

    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec == dd.EELS_MIXED else "f64",
        "data": "synthetic (Drude permittivities stand in for tabulated optical data)",
        "config": {"workload": w.name, "points_per_gpu": w.n_points, "dipoles": n, "fft": [mx, my, mz],
                   "precision": args.precision, "solver": args.solver, "x_tile": list(tiles), "eps_it": 1e-8, "eps_inner": 1e-5, "n_dir": w.n_dir,
                   "l2": "working set of a step > L2 (several GB of per-system vectors)",
                   "iters_mean": float(np.mean(res.iters)), "residual_max": float(np.max(res.residual))},
        "e2e": {"value": pts / (e2e_ms * 1e-3), "unit": "points/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms},
        "roofline": {"bound": "hbm", "kernel": (f"fft_matvec (3 launches: slab forward, x pass, slab inverse; {mx}x{my}x{mz} FFT"
                               + (", k_slab_fwd64 / k_xpassc<float,16,64> / k_slab_inv64)" if (mx, my, mz) == (64, 64, 64) else ")")),
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "traffic": traffic, "ms_per_matvec": mv_ms, "systems": S,
                     "alg_bytes": alg_bytes},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if fp64_cmp:
        out["fp64_single_rhs"] = fp64_cmp
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, w)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
