"""Batched and served solve workloads on the engine (nb_engine_*).

The engine (native, in libnekgb) owns admission, arena memory, stepping and
retirement; this module only feeds requests and records times.

batched_run: every problem of a list is admitted, then all advance together
    by a fixed number of CG iterations (the paper's fixed-iteration mode,
    Sec. V); throughput = sum of E n^3 x iterations / device time.  The same
    problems solved one after another through the engine give the
    sequential reference.  Mixed requests are stepped until every one has
    used its inner-iteration budget (an inner solve that ends inside a step
    waits for the next step's outer pass), and throughput counts the inner
    iterations each request completed.
serving_run: requests arrive as a Poisson process; a request is admitted as
    soon as its footprint fits in the free arena (first come, first served),
    all admitted requests advance together in steps of a few iterations, and
    finished ones are retired at once.  Latency = completion - arrival.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs


def _rhs(torch, dims, n, seed):
    return torch.from_numpy(inputs.unique_field(*dims, n, seed=seed)).cuda()


def footprint_total(nekgb, probs, prec=0):
    return sum(nekgb.nb_engine_footprint(p["dims"], p["n"], prec) for p in probs)


def batched_run(nekgb, stream, probs, iters=100, sequential=True, prec=0):
    """Fixed-iteration batched solve of `probs` (dicts with dims, n,
    mesh_seed, f_seed).  Returns throughput numbers.  With prec = NB_MIXED
    the iterations are inner (FP32) iterations of the defect correction, the
    problems run with tol = 0, so they never stop early; the engine is
    stepped in chunks until every request is done and the GDOF/s counts the
    inner iterations each request completed."""
    import torch
    need = footprint_total(nekgb, probs, prec)
    eng = nekgb.nb_engine_create(int(need * 1.1) + (64 << 20), stream)
    out = {"problems": len(probs), "iterations": iters}
    try:
        rhs = [_rhs(torch, p["dims"], p["n"], p["f_seed"]) for p in probs]
        # one warm-up problem per n so the autotuner has run before timing
        for n in sorted({p["n"] for p in probs}):
            q = next(p for p in probs if p["n"] == n)
            _, rid = nekgb.nb_engine_submit_unique(eng, q["dims"], n, inputs.PERTURB_AMP,
                                                   inputs.perturbation_coeffs(q["mesh_seed"]), 0.0, 8,
                                                   rhs[probs.index(q)], prec=prec)
            nekgb.nb_engine_step(eng, 8)
            nekgb.nb_engine_retire(eng, rid)
        t0 = time.perf_counter()
        ids = []
        for p, f in zip(probs, rhs):
            _, rid = nekgb.nb_engine_submit_unique(eng, p["dims"], p["n"], inputs.PERTURB_AMP,
                                                   inputs.perturbation_coeffs(p["mesh_seed"]), 0.0,
                                                   iters, f, prec=prec)
            ids.append(rid)
        out["setup_s"] = time.perf_counter() - t0
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        a.record(stream)
        steps = 0
        if prec == 0:
            nekgb.nb_engine_step(eng, iters)
            steps = 1
        else:
            for steps in range(1, 4 * iters + 1):
                nekgb.nb_engine_step(eng, 8)
                if all(nekgb.nb_engine_poll(eng, rid)[0] for rid in ids):
                    break
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        dofs = sum(p["E"] * p["n"] ** 3 for p in probs)
        polls = [nekgb.nb_engine_poll(eng, rid) for rid in ids]
        done = all(pl[0] for pl in polls)
        done_its = [pl[1] for pl in polls]
        dof_its = sum(p["E"] * p["n"] ** 3 * it for p, it in zip(probs, done_its))
        out.update({"ms": ms, "local_dofs": dofs, "all_done": done, "engine_steps": steps,
                    "iterations_completed_min": min(done_its), "iterations_completed_max": max(done_its),
                    "gdofs": dof_its / (ms * 1e-3) / 1e9})
        if prec != 0:
            out["outer_passes_mean"] = float(np.mean([nekgb.nb_engine_request_info(eng, rid)[1] for rid in ids]))
        for rid in ids:
            nekgb.nb_engine_retire(eng, rid)
        if sequential:
            seq_ms = 0.0
            for p, f in zip(probs, rhs):
                _, rid = nekgb.nb_engine_submit_unique(eng, p["dims"], p["n"], inputs.PERTURB_AMP,
                                                       inputs.perturbation_coeffs(p["mesh_seed"]),
                                                       0.0, iters, f, prec=prec)
                stream.synchronize()
                a.record(stream)
                nekgb.nb_engine_step(eng, iters)
                b.record(stream)
                b.synchronize()
                seq_ms += a.elapsed_time(b)
                nekgb.nb_engine_retire(eng, rid)
            out["sequential_ms"] = seq_ms
            out["sequential_gdofs"] = dofs * iters / (seq_ms * 1e-3) / 1e9
            out["batching_speedup"] = seq_ms / ms
        out["tuning"] = {n: nekgb.nb_engine_tuning(eng, n, prec) for n in sorted({p["n"] for p in probs})}
    finally:
        nekgb.nb_engine_destroy(eng)
    return out


def measure_iterations(nekgb, stream, reqs, arena_bytes, step_iters=32, prec=0):
    """Iterations each request needs (solved together once, not timed)."""
    import torch
    eng = nekgb.nb_engine_create(arena_bytes, stream)
    its = [None] * len(reqs)
    try:
        pending = list(range(len(reqs)))
        active = {}
        while pending or active:
            while pending:
                k = pending[0]
                r = reqs[k]
                st, rid = nekgb.nb_engine_submit_unique(
                    eng, r["dims"], r["n"], inputs.PERTURB_AMP, inputs.perturbation_coeffs(r["mesh_seed"]),
                    r["tol"], r["maxit"], _rhs(torch, r["dims"], r["n"], r["f_seed"]),
                    allow=(nekgb.NB_OK, nekgb.NB_ERR_OOM), prec=prec)
                if st != nekgb.NB_OK:
                    break
                active[rid] = k
                pending.pop(0)
            nekgb.nb_engine_step(eng, step_iters)
            for rid in list(active):
                done, it, rr, st = nekgb.nb_engine_poll(eng, rid)
                if done:
                    its[active.pop(rid)] = it
                    nekgb.nb_engine_retire(eng, rid)
    finally:
        nekgb.nb_engine_destroy(eng)
    return its


def serving_run(nekgb, stream, reqs, utilisation, capacity_dof_its, iterations, arena_bytes,
                step_iters=16, seed=11, prec=0):
    """Poisson arrivals at a rate that offers `utilisation` x the measured
    capacity (DOF-iterations per second).  The arrival times depend only on
    the requests, the utilisation and the seed, so FP64 and mixed runs see
    the same arrivals.  When no request is in the system the clock jumps to
    the next arrival instead of sleeping (an idle gap changes no latency).
    Returns latency statistics with the number of requests behind them."""
    import torch
    work = np.array([r["E"] * r["n"] ** 3 * it for r, it in zip(reqs, iterations)], dtype=float)
    rate = utilisation * capacity_dof_its / work.mean()          # requests per second
    gaps = np.random.default_rng(seed).exponential(1.0 / rate, size=len(reqs))
    arrivals = np.cumsum(gaps) - gaps[0]
    rhs = [_rhs(torch, r["dims"], r["n"], r["f_seed"]) for r in reqs]
    eng = nekgb.nb_engine_create(arena_bytes, stream)
    lat = [None] * len(reqs)
    relres = [None] * len(reqs)
    try:
        # warm the autotuner for every n outside the timed loop
        for n in sorted({r["n"] for r in reqs}):
            r = next(q for q in reqs if q["n"] == n)
            _, rid = nekgb.nb_engine_submit_unique(eng, r["dims"], n, inputs.PERTURB_AMP,
                                                   inputs.perturbation_coeffs(r["mesh_seed"]), 0.0, 1,
                                                   rhs[reqs.index(r)], prec=prec)
            nekgb.nb_engine_step(eng, 8)
            nekgb.nb_engine_retire(eng, rid)
        t0 = time.perf_counter()
        skipped = 0.0
        clock = lambda: time.perf_counter() - t0 + skipped
        nxt = 0
        queue, active = [], {}
        while nxt < len(reqs) or queue or active:
            now = clock()
            while nxt < len(reqs) and arrivals[nxt] <= now:
                queue.append(nxt)
                nxt += 1
            while queue:                                   # FCFS admission by footprint
                k = queue[0]
                r = reqs[k]
                st, rid = nekgb.nb_engine_submit_unique(
                    eng, r["dims"], r["n"], inputs.PERTURB_AMP, inputs.perturbation_coeffs(r["mesh_seed"]),
                    r["tol"], r["maxit"], rhs[k], allow=(nekgb.NB_OK, nekgb.NB_ERR_OOM), prec=prec)
                if st != nekgb.NB_OK:
                    break
                active[rid] = k
                queue.pop(0)
            if active:
                nekgb.nb_engine_step(eng, step_iters)
                now = clock()
                for rid in list(active):
                    done, it, rr, st = nekgb.nb_engine_poll(eng, rid)
                    if done:
                        k = active.pop(rid)
                        nekgb.nb_engine_retire(eng, rid)
                        lat[k] = now - arrivals[k]
                        relres[k] = rr
            elif queue:
                raise RuntimeError("a request does not fit in the empty arena")
            elif nxt < len(reqs):
                skipped += max(0.0, arrivals[nxt] - now)      # idle: jump to the next arrival
        span = clock()
    finally:
        nekgb.nb_engine_destroy(eng)
    lat_ms = np.array(lat) * 1e3
    return {"precision": "mixed" if prec else "fp64",
            "requests": len(reqs), "utilisation_target": utilisation, "rate_per_s": rate,
            "solves_per_s": len(reqs) / span, "p50_ms": float(np.percentile(lat_ms, 50)),
            "p99_ms": float(np.percentile(lat_ms, 99)), "p99_of_requests": len(reqs),
            "idle_skipped_s": skipped, "mean_ms": float(lat_ms.mean()),
            "max_relres_over_tol": float(max(rr / r["tol"] for rr, r in zip(relres, reqs)))}


def serving_requests(count, seed=5, e_lo=64, e_hi=32768, degrees=(6, 8, 10, 12), tols=(1e-8, 1e-10)):
    rng = np.random.default_rng(seed + 1)
    reqs = []
    for p in inputs.batch_problems(count, seed, e_lo, e_hi, degrees):
        dims = p["dims"]
        reqs.append(dict(p, E=dims[0] * dims[1] * dims[2], tol=float(rng.choice(tols)), maxit=20000))
    return reqs


def batch_list(count=256, seed=4):
    out = []
    for p in inputs.batch_problems(count, seed, 64, 4096, (6, 8, 10, 12)):
        dims = p["dims"]
        out.append(dict(p, E=dims[0] * dims[1] * dims[2]))
    return out
