"""Benchmark of the Nekbone hot path on one GB300 (or N replicas).

A step is one fixed-iteration CG solve (500 iterations, tol <= 0) of the
synthetic Nekbone box problem with E = 4096 elements (16 x 16 x 16) and
n = 10 GLL points per direction (degree 9), FP64-accurate: every iteration
runs the ax_e head (x += alpha p, p = r + beta p, w = ax_e(p), mask,
<w,p>_c, alpha) and the fused dssum + r update (<r,r>_c, beta).  The metric
is Ax throughput in GDOF/s: local points (E n^3) times CG iterations,
divided by the device time.  The solver runs as it does untimed, with CUDA
graphs; per-kernel CUDA events are recorded around one CG iteration in 16
(sampled timing), which gives the roofline's kernel time in the same
region, and `gpu_launches` counts every kernel launched.  The working set (gxyz pairs 197 MB + four
33 MB vectors) is larger than the 129 MB L2, so no flush is needed between
iterations; the standalone ax_e timings below flush L2.

The JSON line adds: `e2e` (the same solve through nb_cg_solve_host with
pinned host buffers, copies timed), `roofline` / `roofline_other` (the CG
head against the FP32-instruction ALU bound and the measured HBM peak, with
the DRAM traffic recorded in profiles/ for the same kernel sources),
`ax_sweep_n10` (ax_e alone and with dssum, L2 flushed, and the CG iteration
time at E = 1024, 2048 and 4096),
`mixed_vs_fp64` (time to relres 1e-10, FP64 vs mixed, n = 8 and 10),
`batched` / `batched_mixed` and `serving` (the engine, FP64 and mixed),
`clocks` (nvidia-smi during the timed region) and `cpu_baseline` (the
oracle on the host cores).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
N > 1 runs under torchrun as independent replicas (weak scaling): each rank
solves its own copy of the problem; the only collectives are the timing
barrier and the max-over-ranks of the elapsed time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2005_13425_gb300 import inputs, metrics  # noqa: E402

METRIC = "Ax GDOF/s, % HBM roofline (N=10); served solves/s + p99, mixed vs FP64"
DIMS = (16, 16, 16)
NGLL = 10
CG_ITERS = 500


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Dist:
    """Barrier and max-over-ranks of host scalars (replicas only)."""

    def __init__(self, world: int, backend: str):
        self.world = world
        self.pg = None
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend=backend)
            self.dist = dist

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def max(self, value: float) -> float:
        if self.world == 1:
            return value
        import torch
        dev = "cuda" if self.dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([value], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.world > 1:
            self.dist.destroy_process_group()


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.th.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def hardware_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ---------------------------------------------------------------- oracle arm
def oracle_problem():
    import oracle
    s = inputs.perturbation_coeffs(inputs.SEED_MESH)
    P = oracle.box_problem(*DIMS, NGLL, inputs.PERTURB_AMP, s)
    fu = inputs.unique_field(*DIMS, NGLL, inputs.SEED_F)
    f = oracle.apply_mask(P["mask"], oracle.scatter_unique(*DIMS, NGLL, fu))
    return oracle, P, f


_ORACLE_CACHE = {}


def time_oracle_cg(iters: int):
    """Wall time of the oracle's CG for `iters` fixed iterations (the
    problem is built once and reused)."""
    if "p" not in _ORACLE_CACHE:
        _ORACLE_CACHE["p"] = oracle_problem()
    oracle, P, f = _ORACLE_CACHE["p"]
    t0 = time.perf_counter()
    _, it, _, _, _ = oracle.cg(*DIMS, NGLL, P["D"], P["gxyz"], P["mask"], f, tol=0.0, maxit=iters)
    dt = time.perf_counter() - t0
    return dt, it


class omp_threads:
    """Run the oracle's OpenMP loops on `k` threads inside the block (the
    oracle library shares the process's OpenMP runtime)."""

    def __init__(self, k: int):
        self.k = k

    def __enter__(self):
        import ctypes
        self.lib = ctypes.CDLL("libgomp.so.1")
        self.old = self.lib.omp_get_max_threads()
        self.lib.omp_set_num_threads(self.k)
        return self

    def __exit__(self, *a):
        self.lib.omp_set_num_threads(self.old)


def config1_oracle():
    """Config 1 (4x4x4 elements, n = 8, 100 fixed CG iterations) with the
    oracle, at all host cores and at one thread (median of 3)."""
    import oracle
    dims, n = (4, 4, 4), 8
    s = inputs.perturbation_coeffs(inputs.SEED_MESH)
    P = oracle.box_problem(*dims, n, inputs.PERTURB_AMP, s)
    f = oracle.apply_mask(P["mask"], oracle.scatter_unique(*dims, n, inputs.unique_field(*dims, n, inputs.SEED_F)))

    def run():
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            oracle.cg(*dims, n, P["D"], P["gxyz"], P["mask"], f, tol=0.0, maxit=100)
            ts.append(time.perf_counter() - t0)
        return statistics.median(ts)
    t_all = run()
    with omp_threads(1):
        t_one = run()
    dofs = 64 * n ** 3
    return {"ms_all_cores": 1e3 * t_all, "ms_one_thread": 1e3 * t_one,
            "gdofs_all_cores": dofs * 100 / t_all / 1e9, "gdofs_one_thread": dofs * 100 / t_one / 1e9}


def cpu_baseline(target_s: float = 15.0):
    """The oracle's CG on the host cores, on a bounded sample of the same
    workload: a 4-iteration probe sizes the sample to ~target_s seconds.
    Also: the same at one thread (a shorter sample) and config 1."""
    dt0, it0 = time_oracle_cg(4)
    iters = int(max(4, min(2000, target_s / max(dt0 / max(it0, 1), 1e-6))))
    dt, it = time_oracle_cg(iters)
    dofs = P_dofs()
    with omp_threads(1):
        dt1, it1 = time_oracle_cg(4)
    return {"value": dofs * it / dt / 1e9, "unit": "GDOF/s", "cores": hardware_threads(),
            "kind": "oracle", "cpu": cpu_model(),
            "sample": f"{it} fixed CG iterations (plus the initial residual) of the same "
                      f"E=4096, n=10 problem, wall {dt:.2f} s",
            "one_thread": {"value": dofs * it1 / dt1 / 1e9, "unit": "GDOF/s", "cores": 1,
                           "sample": f"{it1} CG iterations of the same problem, wall {dt1:.2f} s"},
            "config1_4x4x4_n8_cg100": config1_oracle()}


def P_dofs() -> int:
    return DIMS[0] * DIMS[1] * DIMS[2] * NGLL ** 3


def run_reference(args, rank, world):
    """The oracle, as it stands, on the host cores: the reference arm."""
    if rank != 0:
        return 0
    per_step = 2
    for _ in range(args.warmup):
        time_oracle_cg(per_step)
    times = []
    for _ in range(args.steps):
        dt, it = time_oracle_cg(per_step)
        times.append(dt)
    total = sum(times)
    value = P_dofs() * per_step * args.steps / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GDOF/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "nekbone_box_16x16x16_n10_cg500_fp64", "E": 4096, "n": NGLL,
                   "mesh": "16x16x16", "local_dofs": P_dofs(),
                   "sample": f"each step runs {per_step} of the workload's 500 CG iterations "
                             "(GDOF/s is per iteration, so the sample keeps the metric)",
                   "cg_iterations_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": hardware_threads(),
                         "kind": "oracle", "cpu": cpu_model(),
                         "sample": f"{per_step} CG iterations (+ initial residual) per step, "
                                   f"E=4096, n=10, oracle CG with OpenMP ax_e"},
        "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- mixed vs FP64
def mixed_vs_fp64(nekgb, stream, n, tol=1e-10):
    """Config 3: manufactured solution u* = sin(pi x) sin(pi y) sin(pi z) at
    the nodes (masked), f = A u* with the FP64 operator; time to relative
    residual `tol` with the FP64 solver and with FP32-operator defect
    correction; error of each result against u* (the exact discrete
    solution up to the operator's rounding)."""
    import torch
    E = DIMS[0] * DIMS[1] * DIMS[2]
    s = inputs.perturbation_coeffs(inputs.SEED_MESH)
    out = {"n": n, "E": E, "tol": tol,
           "inputs": "u* at the device-built nodes, f = A u* with the library's FP64 operator "
                     "(parity-checked against the oracle at 1e-12); the oracle-built f and the "
                     "comparison with the oracle's FP64 CG solution at this size are the GPU test "
                     "test_mixed_gpu.py::test_config3_full_size_against_oracle"}
    c64 = nekgb.nb_setup_box(DIMS, n, inputs.PERTURB_AMP, s, nekgb.NB_FP64, stream)
    cmx = nekgb.nb_setup_box(DIMS, n, inputs.PERTURB_AMP, s, nekgb.NB_MIXED, stream)
    try:
        xyz = torch.empty(E, 3, n ** 3, dtype=torch.float64, device="cuda")
        nekgb.nb_box_coords(c64, xyz)
        us = (torch.sin(torch.pi * xyz[:, 0]) * torch.sin(torch.pi * xyz[:, 1])
              * torch.sin(torch.pi * xyz[:, 2])).contiguous()
        nekgb.nb_mask(c64, us)
        f = torch.empty_like(us)
        nekgb.nb_apply(c64, us, f)
        umax = float(us.abs().max())
        def solve(ctx):
            x = torch.zeros_like(us)
            nekgb.nb_cg_solve(ctx, f, x, tol=tol, maxit=20000)          # warm-up
            x.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            stream.synchronize()
            a.record(stream)
            st, it, rr = nekgb.nb_cg_solve(ctx, f, x, tol=tol, maxit=20000)
            b.record(stream)
            b.synchronize()
            iters, outer = nekgb.nb_solve_stats(ctx)
            err = float((x - us).abs().max()) / umax
            return {"ms": a.elapsed_time(b), "iterations": it, "outer": outer,
                    "relres": rr, "max_err_vs_ustar": err}

        out["fp64"] = solve(c64)
        sweep = {}
        for itol in (1e-2, 1e-3, 1e-4, 1e-5):
            nekgb.nb_set_mixed_params(cmx, itol, 50)
            sweep[f"{itol:g}"] = solve(cmx)
        best = min(sweep, key=lambda k: sweep[k]["ms"])
        out["mixed"] = dict(sweep[best], inner_tol=float(best))
        out["mixed_inner_tol_sweep"] = sweep
        out["speedup_mixed"] = out["fp64"]["ms"] / out["mixed"]["ms"]
    finally:
        nekgb.nb_destroy(c64)
        nekgb.nb_destroy(cmx)
    return out


# ---------------------------------------------------------------- serving
def serving(nekgb, stream, count, capacity_gdofs=None):
    """Config 5: Poisson arrivals at 0.5, 0.95 and 2 x the FP64 batched
    capacity (measured here when not given), FP64 and mixed requests."""
    from paper_2005_13425_gb300 import workloads
    if capacity_gdofs is None:
        capacity_gdofs = workloads.batched_run(nekgb, stream, workloads.batch_list(256, seed=4), iters=100,
                                               sequential=False)["gdofs"]
    reqs = workloads.serving_requests(count, seed=5)
    arena = 48 << 30
    its = workloads.measure_iterations(nekgb, stream, reqs, arena)
    out = []
    for u in (0.5, 0.95, 2.0):
        for prec in (nekgb.NB_FP64, nekgb.NB_MIXED):
            srv = workloads.serving_run(nekgb, stream, reqs, u, capacity_gdofs * 1e9, its, arena, prec=prec)
            srv["config"] = (f"{len(reqs)} requests, Poisson arrivals at {u} x the FP64 batched capacity, "
                             "E log-uniform in [64, 32768], n from {6, 8, 10, 12}, tol 1e-8 or 1e-10, "
                             "48 GiB arena")
            out.append(srv)
    return out


# ---------------------------------------------------------------- GPU arm
def run_gpu(args, rank, world, local):
    import torch

    from paper_2005_13425_gb300 import nekgb

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = Dist(world, "nccl")
    nekgb.load()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    if args.serving_study:
        out = {"serving_study": serving(nekgb, stream, args.serve_requests)}
        if rank == 0:
            print(json.dumps(out))
        dist.close()
        return 0
    E = DIMS[0] * DIMS[1] * DIMS[2]
    D = E * NGLL ** 3
    s = inputs.perturbation_coeffs(inputs.SEED_MESH)
    ctx = nekgb.nb_setup_box(DIMS, NGLL, inputs.PERTURB_AMP, s, nekgb.NB_FP64, stream)
    info = nekgb.nb_get_info(ctx)
    fu = torch.from_numpy(inputs.unique_field(*DIMS, NGLL, inputs.SEED_F)).cuda()
    f = torch.empty(E, NGLL ** 3, dtype=torch.float64, device="cuda")
    nekgb.nb_scatter_unique(ctx, fu, f)
    nekgb.nb_mask(ctx, f)
    x = torch.zeros_like(f)

    def step():
        x.zero_()
        nekgb.nb_cg_solve(ctx, f, x, tol=0.0, maxit=CG_ITERS)

    # ---- timed region: the solver's own execution (CUDA graphs), with
    # per-kernel CUDA events on the library's stream around one CG iteration
    # in every 16 (sampled timing, nb_timing_enable(ctx, 2)); the warm-up
    # runs in the same mode, so its graphs exist before the region starts
    nekgb.nb_timing_enable(ctx, 2)
    for _ in range(args.warmup):
        step()
    stream.synchronize()
    nekgb.nb_timing_enable(ctx, 2)        # resets the times and the launch count
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    dist.barrier()
    t_ms = dist.max(ev0.elapsed_time(ev1))
    # per kernel class: the event-timed launches and their average; the CG
    # kernels are timed on one iteration in 16, the once-per-solve kernels on
    # every launch.  est_ms weights each average by the class's launches per
    # solve (1 + CG_ITERS ax_e launches: the initial residual and the heads;
    # CG_ITERS updates; one each of the rest).
    per_step = {"ax_e": CG_ITERS + 1, "update": CG_ITERS}
    kern = {}
    for kid, name in nekgb.KERNEL_NAMES.items():
        ms, cnt = nekgb.nb_timing_read(ctx, kid)
        avg = ms / cnt if cnt else 0.0
        kern[name] = {"ms_timed": ms, "launches_timed": cnt, "ms_avg": avg,
                      "est_ms": avg * per_step.get(name, 1) * args.steps if cnt else 0.0}
    launches = nekgb.nb_launch_count(ctx)
    nekgb.nb_timing_enable(ctx, False)
    value = world * D * CG_ITERS * args.steps / (t_ms * 1e-3) / 1e9

    # ---- the same steps with timing off, for reference
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    t_graph = dist.max(e0.elapsed_time(e1))
    value_graph = world * D * CG_ITERS * args.steps / (t_graph * 1e-3) / 1e9

    # ---- e2e: host buffers through the C ABI, copies inside the timed region
    f_host = torch.empty(E * NGLL ** 3, dtype=torch.float64).pin_memory()
    f_host.copy_(f.reshape(-1).cpu())
    x_host = torch.zeros(E * NGLL ** 3, dtype=torch.float64).pin_memory()
    xh = x_host.numpy()
    fh = f_host.numpy()
    for _ in range(1):
        xh[:] = 0.0
        nekgb.nb_cg_solve_host(ctx, fh, xh, tol=0.0, maxit=CG_ITERS)
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        xh[:] = 0.0
        nekgb.nb_cg_solve_host(ctx, fh, xh, tol=0.0, maxit=CG_ITERS)
    t_e2e = dist.max(time.perf_counter() - t0)
    value_e2e = world * D * CG_ITERS * args.steps / t_e2e / 1e9

    # ---- ax_e alone and ax_e + dssum, L2 flushed between repetitions
    u = torch.from_numpy(inputs.local_field(E, NGLL, inputs.SEED_U)).cuda()
    w = torch.empty_like(u)
    l2 = torch.cuda.get_device_properties(local).L2_cache_size
    scrub = torch.empty(2 * l2 // 4 + 1024, dtype=torch.float32, device="cuda")

    def timed(fn, reps=20):
        out = []
        for _ in range(reps):
            scrub.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
        return statistics.median(out)

    nekgb.nb_ax(ctx, u, w)
    t_ax = timed(lambda: nekgb.nb_ax(ctx, u, w))
    t_axds = timed(lambda: (nekgb.nb_ax(ctx, u, w), nekgb.nb_dssum(ctx, w)))
    variant_default = nekgb.nb_get_info(ctx)["ax_variant"]
    nekgb.nb_set_ax_variant(ctx, 1)       # native FP64 kernel, for comparison
    nekgb.nb_ax(ctx, u, w)
    t_ax_fp64 = timed(lambda: nekgb.nb_ax(ctx, u, w), reps=5)
    nekgb.nb_set_ax_variant(ctx, variant_default)

    # ---- the Ax sweep over E = 1024, 2048, 4096 (n = 10): ax_e alone and
    # ax_e + dssum with L2 flushed (median of 20), and the per-iteration time
    # of a 500-iteration CG solve
    sweep = []
    for dims in ((16, 8, 8), (16, 16, 8), DIMS):
        Es = dims[0] * dims[1] * dims[2]
        Ds = Es * NGLL ** 3
        cs = nekgb.nb_setup_box(dims, NGLL, inputs.PERTURB_AMP, s, nekgb.NB_FP64, stream)
        try:
            us = torch.from_numpy(inputs.local_field(Es, NGLL, inputs.SEED_U)).cuda()
            ws = torch.empty_like(us)
            nekgb.nb_ax(cs, us, ws)
            ta = timed(lambda: nekgb.nb_ax(cs, us, ws))
            tad = timed(lambda: (nekgb.nb_ax(cs, us, ws), nekgb.nb_dssum(cs, ws)))
            fus = torch.from_numpy(inputs.unique_field(*dims, NGLL, inputs.SEED_F)).cuda()
            fs = torch.empty(Es, NGLL ** 3, dtype=torch.float64, device="cuda")
            nekgb.nb_scatter_unique(cs, fus, fs)
            nekgb.nb_mask(cs, fs)
            xs = torch.zeros_like(fs)
            nekgb.nb_cg_solve(cs, fs, xs, tol=0.0, maxit=CG_ITERS)
            xs.zero_()
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            nekgb.nb_cg_solve(cs, fs, xs, tol=0.0, maxit=CG_ITERS)
            c1.record(stream)
            c1.synchronize()
            tcg = c0.elapsed_time(c1) / CG_ITERS
            sweep.append({"E": Es, "mesh": "x".join(map(str, dims)), "ax_ms": ta,
                          "ax_gdofs": Ds / (ta * 1e-3) / 1e9, "ax_dssum_ms": tad,
                          "ax_dssum_gdofs": Ds / (tad * 1e-3) / 1e9,
                          "cg_iteration_ms": tcg, "cg_gdofs": Ds / (tcg * 1e-3) / 1e9})
        finally:
            nekgb.nb_destroy(cs)

    # ---- the partitioned box on one GPU: two slabs of 8 element layers,
    # the host-driven partitioned CG (interface exchanges as device copies)
    from paper_2005_13425_gb300 import partition
    slabs = [partition.GpuSlab(nekgb, DIMS, z0, z1, NGLL, inputs.PERTURB_AMP, s, stream)
             for z0, z1 in partition.slab_bounds(DIMS[2], 2)]
    try:
        pbox = partition.PartitionedBox(slabs, partition.Exchange(2, 0, 2))
        layer = DIMS[0] * DIMS[1]
        fs = [f[z0 * layer:z1 * layer].contiguous() for z0, z1 in partition.slab_bounds(DIMS[2], 2)]
        xs = [sl.new_field() for sl in slabs]
        pbox.cg(fs, xs, tol=0.0, maxit=3)
        for xx in xs:
            xx.zero_()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        pbox.cg(fs, xs, tol=0.0, maxit=20)
        p1.record(stream)
        p1.synchronize()
        pit = p0.elapsed_time(p1) / 20
        partitioned = {"slabs": 2, "ms_per_iteration": pit, "gdofs": D / (pit * 1e-3) / 1e9,
                       "note": "host-driven partitioned CG (two exchanges of 168 KB planes and two "
                               "scalar reductions per iteration, no CUDA graph), both slabs on one GPU"}
    finally:
        for sl in slabs:
            sl.close()

    # ---- config 1: 4x4x4 elements, n = 8, 100 fixed CG iterations (the
    # paper's run length), median of 20 solves
    c1 = nekgb.nb_setup_box((4, 4, 4), 8, inputs.PERTURB_AMP, s, nekgb.NB_FP64, stream)
    try:
        f1u = torch.from_numpy(inputs.unique_field(4, 4, 4, 8, inputs.SEED_F)).cuda()
        f1 = torch.empty(64, 8 ** 3, dtype=torch.float64, device="cuda")
        nekgb.nb_scatter_unique(c1, f1u, f1)
        nekgb.nb_mask(c1, f1)
        x1 = torch.zeros_like(f1)
        t1 = []
        for rep in range(23):
            x1.zero_()
            c0, c1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            nekgb.nb_cg_solve(c1, f1, x1, tol=0.0, maxit=100)
            c1e.record(stream)
            c1e.synchronize()
            if rep >= 3:
                t1.append(c0.elapsed_time(c1e))
        config1 = {"mesh": "4x4x4", "n": 8, "cg_iterations": 100, "ms": statistics.median(t1),
                   "gdofs": 64 * 8 ** 3 * 100 / (statistics.median(t1) * 1e-3) / 1e9,
                   "note": "32,768 local points: launch- and latency-bound (2 kernels per iteration)"}
    finally:
        nekgb.nb_destroy(c1)

    # ---- roofline of the dominant kernel, from the timed region's events
    fp32_peak = nekgb.nb_fp32_rate() / 1e12
    hbm, _, peak_src = metrics.measured_peaks(ROOT)
    ax = kern["ax_e"]
    ax_avg_ms = ax["ms_avg"]
    ax_bytes = metrics.cg_head_bytes_per_point(8) * D
    variant = nekgb.nb_get_info(ctx)["ax_variant"]
    double_float = variant in (0, 2)      # automatic selection picks the double-float kernel at n = 10
    ach_gbs = ax_bytes / (ax_avg_ms * 1e-3) / 1e9
    hbm_frac = ach_gbs / hbm
    total_kernel_ms = sum(v["est_ms"] for v in kern.values())
    traffic = None
    if double_float:
        traffic = metrics.recorded_traffic(
            os.path.join(ROOT, "profiles", "traffic.json"), "cg_head_ax_df_e4096_n10",
            metrics.source_digest(os.path.join(ROOT, "paper_2005_13425_gb300", "csrc")))
    roof_hbm = {"bound": "hbm", "achieved": ach_gbs, "peak": hbm, "unit": "GB/s",
                "frac": hbm_frac, "traffic": traffic,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs, of {peak_src})",
                "kernel": "ax_e (CG head)", "algorithmic_bytes_per_launch": ax_bytes,
                "avg_launch_ms": ax_avg_ms, "launches": ax["launches_timed"]}
    if double_float:
        # the double-float ax_e runs on the FP32 pipe: its ALU bound is the
        # FP32 instruction rate, its work the algorithm's FP32 instructions
        ops = metrics.df_fp32_ops_per_point(NGLL) * D
        ach = ops / (ax_avg_ms * 1e-3) / 1e12
        roof_alu = {"bound": "alu", "achieved": ach, "peak": fp32_peak,
                    "unit": "T FP32 instr/s", "frac": ach / fp32_peak, "traffic": traffic,
                    "peak_source": "measured: nb_fp32_rate (FFMA rate, all SMs, this run); nominal "
                                   f"152 SMs x 128 lanes x 2070 MHz = {metrics.FP32_PEAK_TOPS:.2f}",
                    "kernel": "ax_e (CG head)", "algorithmic_fp32_instr_per_launch": ops,
                    "avg_launch_ms": ax_avg_ms, "launches": ax["launches_timed"]}
    else:
        ach = metrics.ax_flops_per_point(NGLL) * D / (ax_avg_ms * 1e-3) / 1e12
        roof_alu = {"bound": "alu", "achieved": ach, "peak": metrics.NOMINAL_FP64_TFLOPS,
                    "unit": "TFLOP/s", "frac": ach / metrics.NOMINAL_FP64_TFLOPS, "traffic": None,
                    "peak_source": "nominal GB300 FP64 1.25 TFLOP/s",
                    "kernel": "ax_e (CG head)", "avg_launch_ms": ax_avg_ms, "launches": ax["launches_timed"]}
    roofline = roof_hbm if hbm_frac >= roof_alu["frac"] else roof_alu
    other_roofline = roof_alu if roofline is roof_hbm else roof_hbm

    line = {
        "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "nekbone_box_16x16x16_n10_cg500_fp64", "E": E, "n": NGLL,
                   "mesh": "16x16x16", "cg_iterations_per_step": CG_ITERS, "local_dofs": D,
                   "unique_dofs": int(info["nunique"]), "perturbation": inputs.PERTURB_AMP,
                   "l2": "inputs larger than L2 (gxyz 197 MB + 5 vectors of 33 MB > 129 MB)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "ax_variant": variant},
        "roofline": roofline,
        "roofline_other": other_roofline,
        "gpu_launches": launches,
        "kernels_timed_region": kern,
        "kernel_share": {k: v["est_ms"] / total_kernel_ms for k, v in kern.items() if total_kernel_ms},
        "timing": "sampled: per-kernel CUDA events on one CG iteration in 16 (plain launches), the other 15 "
                  "as a CUDA graph; gpu_launches counts every kernel launched in the timed region",
        "value_graph_mode": value_graph,
        "eq1_gflops": value * metrics.cg_flops_per_point(NGLL),
        "eq2_accounting_gbs": value * metrics.cg_bytes_per_point(),
        "eq2_accounting_note": "GDOF/s x the paper's 240 B per point per CG iteration (Eq. 2); the "
                               "fused iteration moves about 120 B per point, so this is not a "
                               "roofline fraction",
        "ax_only": {"ms": t_ax, "gdofs": D / (t_ax * 1e-3) / 1e9,
                    "hbm_frac": metrics.ax_bytes_per_point(8) * D / (t_ax * 1e-3) / 1e9 / hbm,
                    "l2": "flushed between reps"},
        "ax_dssum": {"ms": t_axds, "gdofs": D / (t_axds * 1e-3) / 1e9},
        "ax_sweep_n10": sweep,
        "config1_4x4x4_n8_cg100": config1,
        "partitioned_2slabs_one_gpu": partitioned,
        "ax_only_native_fp64": {"ms": t_ax_fp64, "gdofs": D / (t_ax_fp64 * 1e-3) / 1e9,
                                "fp64_tflops": metrics.ax_flops_per_point(NGLL) * D / (t_ax_fp64 * 1e-3) / 1e12},
        "e2e": {"value": value_e2e, "unit": "GDOF/s",
                "h2d_bytes_per_step": 2 * 8 * D, "d2h_bytes_per_step": 8 * D,
                "api": "nb_cg_solve_host (pinned host f, x)"},
        "clocks": clocks.summary(),
    }
    if not args.no_mixed:
        line["mixed_vs_fp64"] = [mixed_vs_fp64(nekgb, stream, nn) for nn in (8, 10)]
    if not args.no_engine:
        from paper_2005_13425_gb300 import workloads
        batch = workloads.batch_list(256, seed=4)
        line["batched"] = workloads.batched_run(nekgb, stream, batch, iters=100)
        line["batched"]["config"] = ("256 box problems, E log-uniform in [64, 4096] rounded to box dims, "
                                     "n from {6, 8, 10, 12}, FP64-accurate, 100 fixed CG iterations")
        line["batched_mixed"] = workloads.batched_run(nekgb, stream, batch, iters=100, sequential=False,
                                                      prec=nekgb.NB_MIXED)
        line["batched_mixed"]["config"] = ("the same 256 problems, mixed precision (FP32 inner CG, FP64 "
                                           "defect correction), 100 inner iterations")
        line["serving"] = serving(nekgb, stream, args.serve_requests, line["batched"]["gdofs"])
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    nekgb.nb_destroy(ctx)
    if rank == 0:
        print(json.dumps(line))
    dist.close()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-vs-FP64 solves")
    ap.add_argument("--no-engine", action="store_true", help="skip the batched and served solves")
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serving-study", action="store_true",
                    help="run only the served workload (config 5) and print its records")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_gpu(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
