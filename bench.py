"""Benchmark: EELS/CL (energy, beam) points per second on one GB300.

Default workload: the 100 nm Drude-silver sphere on a 64^3 lattice (137,376
dipoles, 128^3 padded FFT) in the absorbing Cherenkov host eps_h = 4 + 0.05i,
200 keV electron (beta_h > 1) at b = 60 nm, 100 loss energies 1.5-4.0 eV,
CL far field on 2562 directions -- the largest single-GPU workload.  The
mixed path: FP32 QMR inside FP64 refinement to 1e-8, FP64 incident field
and loss sums.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload ...]

A step is one eels_solve over one batch of the workload: 25 energies of the
Cherenkov spectrum (the steps cycle through its four batches, so K = 20
covers it five times), all 200 energies of the 32^3 spectrum.  `value` is
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
    "cherenkov": lambda: I.config_cherenkov(),
    "spectrum": lambda: I.config_spectrum(),
    "small": lambda: I.config_small_sphere(),
    "rod": lambda: I.config_rod_map(n_energy=8, nbx=32, nby=32),
}
# energies per step (one batch of the workload; the steps cycle through the spectrum)
STEP_ENERGIES = {"cherenkov": 25, "spectrum": 200, "small": 1, "rod": 1}

# The oracle sample of the CPU baseline, per workload: the point (energy
# index, beam index); None, or the GMRES iterations timed and the direction
# stride of the far field timed (the oracle at full size takes tens of
# minutes per point on a host: its point time is modelled from the timed
# parts, see oracle_point()), with the GMRES matvecs the oracle needs for
# that point (bench.py --oracle-iterations prints them).
CPU_SAMPLE = {"spectrum": (100, 0, None), "small": (0, 0, None),
              "cherenkov": (50, 0, dict(iters=30, cl_stride=8, matvecs=1937)),
              "rod": (4, 0, dict(iters=30, cl_stride=8, matvecs=897))}

# ncu DRAM traffic (read + write bytes) of one matvec launch set, per system,
# measured on the workload TRAFFIC_WORKLOAD with kernel sources that hash to
# TRAFFIC_SRC_HASH; reported as null for other workloads (other FFT sizes,
# other kernels) and when the kernel sources differ from the measured ones.
TRAFFIC_BYTES_PER_SYSTEM = 115_766_848   # 1,852,269,568 B over 16 systems, 128^3 FFT
TRAFFIC_SRC_HASH = "1ee292d212c5f1ea"
TRAFFIC_WORKLOAD = "cherenkov"


def kernel_src_hash() -> str:
    h = hashlib.sha256()
    for f in ("k_fft.cu", "k_xreg.cu", "fft.cuh", "fft_warp.cuh", "kernels.h", "common.cuh"):
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


def oracle_point(wname: str, w):
    """One point of the workload through the FP64 oracle on the host cores.
    Small workloads: the full solve (scipy FFT convolution + GMRES(200) to
    1e-8) and every loss.  Full-size Cherenkov sphere and rod map: the same
    setup (fields, D-hat), the first `iters` GMRES(200) iterations, the
    P_EELS / P_ext / P_abs sums and the far field on every cl_stride-th
    direction are timed, and the point time is modelled as setup +
    matvecs x (time per timed iteration) + losses + cl_stride x far field.
    The first iterations of a restart cycle orthogonalise against fewer
    vectors than the average one, so the modelled time is a lower bound
    and the CPU figure an upper bound."""
    import scipy.sparse.linalg as spla
    from oracle import green, losses, run
    ie, ib, smp = CPU_SAMPLE[wname]
    g = w.grid
    point = f"{w.name} energy {w.energies_eV[ie]:.3f} eV (index {ie}), beam {ib}"
    t0 = time.perf_counter()
    pt = run.setup(g.nx, g.ny, g.nz, g.d_nm, g.occ, w.energies_eV[ie], w.eps_p[ie], w.eps_h[ie], w.beams_nm[ib],
                   ekin_keV=w.ekin_keV)
    if smp is None:
        p, _ = run.solve_fft(pt, rtol=1e-8)
        run.observables(pt, p)
        dt = time.perf_counter() - t0
        return {"seconds": dt, "cpu_seconds": dt, "sample": f"1 point of {point}, solved in full"}
    op = green.FFTOperator(pt.idx, pt.n_axes, pt.d, pt.k, pt.alpha)
    t_setup = time.perf_counter() - t0
    sq = np.sqrt(pt.alpha)
    n3 = 3 * len(pt.r)
    count = [0]

    class _Enough(Exception):
        pass

    def mv(y):
        if count[0] >= smp["iters"] + 1:          # the initial residual and `iters` iterations
            raise _Enough
        count[0] += 1
        y = y.reshape(-1, 3)
        return (sq[:, None] * op.matvec(sq[:, None] * y)).reshape(-1)

    L = spla.LinearOperator((n3, n3), matvec=mv, dtype=np.complex128)
    b = (sq[:, None] * pt.E_inc).reshape(-1)
    t1 = time.perf_counter()
    try:
        spla.gmres(L, b, rtol=1e-8, atol=0.0, restart=200, maxiter=20000)
    except _Enough:
        pass
    t_iter = (time.perf_counter() - t1) / count[0]
    p = np.zeros_like(pt.E_inc)                   # the timed sums do not depend on the values
    t2 = time.perf_counter()
    losses.p_eels(pt.E_a, p, pt.eps_h, pt.omega)
    losses.p_ext(pt.E_inc, p, pt.eps_h, pt.omega)
    losses.p_abs(p, pt.alpha_cm, pt.eps_h, pt.omega)
    t3 = time.perf_counter()
    dirs, wts = run.directions()
    st = smp["cl_stride"]
    losses.p_cl(pt.r, p, pt.k, pt.m_h, pt.omega, dirs[::st], wts[::st])
    t4 = time.perf_counter()
    n_mv = smp["matvecs"] or 1000
    seconds = t_setup + n_mv * t_iter + (t3 - t2) + st * (t4 - t3)
    return {"seconds": seconds, "cpu_seconds": t4 - t0,
            "sample": (f"1 point of {point}: setup, {count[0]} of the {n_mv} GMRES(200) matvecs it needs"
                       + ("" if smp["matvecs"] else " (assumed)")
                       + f", the loss sums and 1/{st} of the far-field directions timed; point time modelled as "
                         f"setup + {n_mv} x time per timed iteration + losses + {st} x far field (a lower bound: "
                         f"early iterations of a restart cycle are the cheapest)")}


def cpu_baseline(wname: str, w):
    """The oracle (FP64) on a bounded sample of the workload (oracle_point)."""
    r = oracle_point(wname, w)
    return {"value": 1.0 / r["seconds"], "unit": "points/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": r["sample"], "seconds_per_point": r["seconds"], "cpu_seconds": r["cpu_seconds"]}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_point(args.workload, w)
    t0 = time.perf_counter()
    secs = []
    for _ in range(args.steps):
        r = oracle_point(args.workload, w)
        secs.append(r["seconds"])
    wall = (time.perf_counter() - t0) / args.steps
    v = 1.0 / float(np.mean(secs))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "points/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "oracle": "FP64 numpy/scipy: FFT convolution + GMRES(200) to 1e-8"},
        "cpu_baseline": {"value": v, "unit": "points/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "per step: " + r["sample"]},
        "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_oracle_iterations(args, w):
    """Runs the oracle's GMRES(200) on the CPU-baseline point of the workload
    to 1e-8 and prints how many matvecs it needed (the constant of CPU_SAMPLE)."""
    import scipy.sparse.linalg as spla
    from oracle import green, run
    ie, ib, _ = CPU_SAMPLE[args.workload]
    g = w.grid
    pt = run.setup(g.nx, g.ny, g.nz, g.d_nm, g.occ, w.energies_eV[ie], w.eps_p[ie], w.eps_h[ie], w.beams_nm[ib],
                   ekin_keV=w.ekin_keV)
    op = green.FFTOperator(pt.idx, pt.n_axes, pt.d, pt.k, pt.alpha)
    sq = np.sqrt(pt.alpha)
    count = [0]

    def mv(y):
        count[0] += 1
        y = y.reshape(-1, 3)
        return (sq[:, None] * op.matvec(sq[:, None] * y)).reshape(-1)

    n3 = 3 * len(pt.r)
    L = spla.LinearOperator((n3, n3), matvec=mv, dtype=np.complex128)
    _, info = spla.gmres(L, (sq[:, None] * pt.E_inc).reshape(-1), rtol=1e-8, atol=0.0, restart=200, maxiter=20000)
    print(json.dumps({"workload": w.name, "energy_index": ie, "beam_index": ib, "info": int(info),
                      "matvecs": count[0]}))


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


def serve_requests(n_requests: int, rate: float, n_energy: int, n_beam: int):
    """The seeded request stream of the serving workload at its stated ranges
    (lattices 16^3-96^3 spheres and rods, gold or silver, host from {1.0,
    2.1, 4.0+0.05i}, 1-256 beams, 8-128 energies, Poisson arrivals at `rate`):
    its first n_requests requests, each cut to n_energy of its energies
    (spread over its spectrum) and its first n_beam beams.  Changing the
    rate rescales the arrival times only (the draws are the same)."""
    reqs = I.serving_stream(n_requests=n_requests, rate_per_s=rate)
    for r in reqs:
        w = r.workload
        ie = np.unique(np.linspace(0, len(w.energies_eV) - 1, min(n_energy, len(w.energies_eV))).round().astype(int))
        w.energies_eV, w.eps_p, w.eps_h = w.energies_eV[ie], w.eps_p[ie], w.eps_h[ie]
        w.beams_nm = w.beams_nm[:n_beam]
    return reqs


def run_serve(args):
    """Serving: the request stream (serve_requests) submitted at its arrival
    times to the library's serving loop (admission by device-memory
    footprint, concurrent requests on per-worker streams), at the stated
    mean rate of 20 requests/s and at 5/s; points/s and p50/p99 latency
    (submit to completion) of each pass."""
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

    def one_pass(stream):
        srv = dd.eels_server_create(device=local, max_concurrent=args.serve_concurrency)
        t0 = time.perf_counter()
        ids = []
        for r in stream:
            dt = r.t_arrival_s - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            w = r.workload
            o = dd.eels_default_opts(ekin_keV=w.ekin_keV, eps_it=1e-8, n_dir=w.n_dir, device_loop=int(args.device_loop))
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

    warm = serve_requests(3, 20.0, 1, 1)
    for r in warm:
        r.workload.grid = I.Grid(16, 16, 16, 1.25, I.sphere_occupancy(16, 20.0))
        r.workload.beams_nm = np.array([[15.0, 0.0]])
    for _ in range(max(1, args.warmup)):
        one_pass(warm)
    passes = {}
    l0 = dd.eels_kernel_launches()
    with ClockSampler(local) as clk:
        for rate in (20.0, 5.0):
            reqs = serve_requests(args.serve_requests, rate, args.serve_energies, args.serve_beams)
            pts, span, lat, stats = one_pass(reqs)
            passes[rate] = dict(points=pts, seconds=span, points_per_s=pts / span,
                                p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                                max_ms=float(np.max(lat)), running_max=stats["running_max"],
                                lattices=sorted({f"{r.workload.grid.nx}x{r.workload.grid.ny}x{r.workload.grid.nz}"
                                                 for r in reqs}))
    launches = dd.eels_kernel_launches() - l0
    if rank != 0:
        return
    main_pass = passes[20.0]
    print(json.dumps({
        "metric": METRIC, "value": main_pass["points_per_s"], "unit": "points/s", "n_gpus": 1, "steps": 1,
        "warmup": args.warmup, "ms_per_step": main_pass["seconds"] * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic seeded request stream",
        "config": {"workload": (f"serving stream (seed 20261203, lattices 16^3-96^3 spheres/rods, Au/Ag, three hosts, "
                                f"1-256 beams, 8-128 energies): first {args.serve_requests} requests, each cut to "
                                f"{args.serve_energies} energies x its first {args.serve_beams} beams"),
                   "concurrency": args.serve_concurrency,
                   "inner_loop": "device" if args.device_loop else "host bursts"},
        "latency_ms": {"p50": main_pass["p50_ms"], "p99": main_pass["p99_ms"], "max": main_pass["max_ms"]},
        "passes": {f"{int(r)}/s": v for r, v in passes.items()},
        "e2e": {"value": main_pass["points_per_s"], "unit": "points/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0,
                "note": "requests enter and leave through host buffers; the value above is already end to end"},
        "gpu_launches": int(launches), "clocks": clk.summary(),
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cherenkov", choices=sorted(WORKLOADS) + ["serve"])
    ap.add_argument("--step-energies", type=int, default=0,
                    help="energies per step (0: the workload's default batch)")
    ap.add_argument("--oracle-iterations", action="store_true",
                    help="run the oracle to convergence on the CPU-baseline point and print its matvec count")
    ap.add_argument("--matvec-only", type=int, default=0,
                    help="time only the FFT matvec on this many systems of the workload (profiling)")
    ap.add_argument("--serve-requests", type=int, default=12)
    ap.add_argument("--serve-energies", type=int, default=2)
    ap.add_argument("--serve-beams", type=int, default=4)
    ap.add_argument("--serve-concurrency", type=int, default=8)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--solver", default="qmr2", choices=["qmr2", "qmr", "bicgstab"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--inner-max-iter", type=int, default=0,
                    help="FP32 iterations per inner solve before the FP64 restart (0: the library default)")
    ap.add_argument("--device-loop", action="store_true",
                    help="each inner solve as one graph launch with a WHILE node (eels_opts.device_loop)")
    ap.add_argument("--fp64-sample", type=int, default=5,
                    help="energies of the plain FP64 single-system comparison (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="steps of the end-to-end pass (default: one pass over the batches, at most 4)")
    ap.add_argument("--matvec-reps", type=int, default=20)
    args = ap.parse_args()
    if args.workload == "serve":
        run_serve(args)
        return
    if args.matvec_only:
        run_matvec_only(args)
        return
    w = WORKLOADS[args.workload]()
    if args.oracle_iterations:
        run_oracle_iterations(args, w)
        return
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
                                solver={"qmr2": dd.EELS_QMR2, "qmr": dd.EELS_QMR, "bicgstab": dd.EELS_BICGSTAB}[args.solver],
                                device_loop=int(args.device_loop))
    if args.inner_max_iter > 0:
        opts.inner_max_iter = args.inner_max_iter
    dd.eels_set_grid(ctx, g.occ, g.d_nm)

    # one step = one batch of the workload: E consecutive energies (all beams);
    # step k takes batch k mod n_batches
    n_e = len(w.energies_eV)
    E = min(args.step_energies or STEP_ENERGIES.get(args.workload, n_e), n_e)
    batches = [np.arange(i, min(i + E, n_e)) for i in range(0, n_e, E)]
    n_beam = len(w.beams_nm)

    def step(k):
        ie = batches[k % len(batches)]
        return ie, dd.eels_solve(ctx, opts, w.energies_eV[ie], w.eps_p[ie], w.eps_h[ie], w.beams_nm, want_cl=True)

    for k in range(args.warmup):
        _, res = step(k)
        assert res.converged.all(), "warm-up solve did not converge"
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = dd.eels_kernel_launches()
    pts_timed = 0
    results = {}
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for k in range(args.steps):
            ie, res = step(k)
            pts_timed += len(ie) * n_beam
            results[k % len(batches)] = (ie, res)
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = dd.eels_kernel_launches() - l0
    barrier()
    ms_total = ev0.elapsed_time(ev1)
    if dist:
        t = torch.tensor([ms_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms = ms_total / args.steps
    value = pts_timed * world / (ms_total * 1e-3)
    clocks = clk.summary()
    iters = np.concatenate([r.iters.ravel() for _, r in results.values()])
    resid = np.concatenate([r.residual.ravel() for _, r in results.values()])

    # end to end through the host API: lattice upload + host inputs + host outputs
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pts_e2e, h2d, d2h = 0, 0, 0
    e2e_steps = args.e2e_steps if args.e2e_steps > 0 else min(len(batches), 4)
    for k in range(e2e_steps):
        dd.eels_set_grid(ctx, g.occ, g.d_nm)
        ie, r2 = step(k)
        pts_e2e += len(ie) * n_beam
        h2d += g.occ.nbytes + 8 * len(ie) + 16 * w.eps_p[ie].size + 16 * len(ie) + w.beams_nm.nbytes
        d2h += len(ie) * n_beam * (4 * 8 + 24)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())

    # roofline of the FFT matvec (the dominant kernel set) on one batch's systems
    S = len(batches[0]) * n_beam
    tiles = dd.eels_tile_widths(ctx)
    xtuned = dd.eels_tuned_xpass(ctx)
    # every x-pass candidate the autotuner timed (ms of three launches)
    xnames = ["heuristic", "loads", "tensor copies"]
    xtimed = {f"{xnames[m]}, {b} beams/block": round(t, 4) for m, b, t in dd.eels_xpass_timings(ctx)}
    ie0 = batches[0]
    dd.eels_prepare_operator(ctx, np.repeat(w.energies_eV[ie0], n_beam), np.repeat(w.eps_p[ie0], n_beam, axis=0),
                             np.repeat(w.eps_h[ie0], n_beam))
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
    # complex64: per system x, y and two round trips of the half-padded
    # intermediate; D-hat once per energy (shared by its n_beam beams)
    alg_bytes = (S * (6 * M + 6 * n) + len(ie0) * 6 * Mr) * 8
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (mv_ms * 1e-3) / 1e9
    traffic = None
    if (TRAFFIC_BYTES_PER_SYSTEM is not None and args.workload == TRAFFIC_WORKLOAD
            and TRAFFIC_SRC_HASH == kernel_src_hash()):
        traffic = TRAFFIC_BYTES_PER_SYSTEM * S

    # the plain FP64 path, one system per solve, on a sample of the energies
    # (first beam): its points/s, and how far the mixed results are from it
    fp64_cmp = None
    if prec == dd.EELS_MIXED and world == 1 and args.fp64_sample > 0 and results:
        ie_all = np.concatenate([v[0] for v in results.values()])
        pe_all = np.concatenate([v[1].p_eels[:, 0] for v in results.values()])
        pc_all = np.concatenate([v[1].p_cl[:, 0] for v in results.values()])
        pick = np.unique(np.linspace(0, len(ie_all) - 1, args.fp64_sample).round().astype(int))
        idx = ie_all[pick]
        o64 = dd.eels_default_opts(ekin_keV=w.ekin_keV, precision=dd.EELS_FP64, eps_it=1e-8, n_dir=w.n_dir,
                                   max_batch=1)
        dd.eels_set_grid(ctx, g.occ, g.d_nm)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r64 = dd.eels_solve(ctx, o64, w.energies_eV[idx], w.eps_p[idx], w.eps_h[idx], w.beams_nm[:1], want_cl=True)
        torch.cuda.synchronize()
        v64 = len(idx) / (time.perf_counter() - t0)
        rel_e = np.abs(pe_all[pick] - r64.p_eels[:, 0]) / np.abs(r64.p_eels[:, 0])
        rel_c = np.abs(pc_all[pick] - r64.p_cl[:, 0]) / np.abs(r64.p_cl[:, 0])
        fp64_cmp = {"value": v64, "unit": "points/s",
                    "sample": f"energies {idx.tolist()} of {w.name}, beam 0, one system per solve, eps 1e-8",
                    "mixed_over_fp64": value / world / v64, "p_eels_max_rel_diff": float(rel_e.max()),
                    "p_cl_max_rel_diff": float(rel_c.max())}
    dd.eels_destroy(ctx)

    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec == dd.EELS_MIXED else "f64",
        "data": "synthetic (Drude permittivities stand in for tabulated optical data)",
        "config": {"workload": w.name, "points_per_gpu": n_e * n_beam, "points_per_step": E * n_beam,
                   "step": f"{E} energies x {n_beam} beams, batches cycled", "dipoles": n, "fft": [mx, my, mz],
                   "precision": args.precision, "solver": args.solver, "inner_loop": "device" if args.device_loop else "host bursts",
                   "inner_max_iter": opts.inner_max_iter, "x_tile": list(tiles),
                   "x_pass": {"mode": xnames[xtuned[0]], "beams_per_block": xtuned[1], "timed_ms": xtimed},
                   "eps_it": 1e-8,
                   "eps_inner": 1e-5, "n_dir": w.n_dir,
                   "l2": "working set of a step > L2 (several GB of per-system vectors and FFT scratch)",
                   "iters_mean": float(np.mean(iters)), "residual_max": float(np.max(resid))},
        "e2e": {"value": pts_e2e * world / e2e_s, "unit": "points/s", "h2d_bytes_per_step": int(h2d / e2e_steps),
                "d2h_bytes_per_step": int(d2h / e2e_steps), "ms_per_step": e2e_s * 1e3 / e2e_steps},
        "roofline": {"bound": "hbm",
                     "kernel": f"fft_matvec (3 launches: slab forward, x pass, slab inverse; {mx}x{my}x{mz} FFT)",
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
