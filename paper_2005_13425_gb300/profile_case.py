"""Run one hot-path operation a few times on a synthetic box problem, for
profilers (ncu) that need a short, self-contained command.

    python -m paper_2005_13425_gb300.profile_case --op ax --dims 16 16 16 --n 10 --reps 3

--op ax     w = ax_e(u)                       (nb_ax)
--op apply  w = mask(dssum(ax_e(u)))          (nb_apply)
--op cg     --reps CG iterations of one solve (nb_cg_solve, fixed iterations)
--op grad   w = D_r u + D_s u + D_t u by nb_probe_grad --method (0: double-float
            line products, 1: tensor cores on a digit split); with --time the
            median kernel time of the launches after the first is printed
"""
from __future__ import annotations

import argparse

import torch

from paper_2005_13425_gb300 import inputs, nekgb


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["ax", "apply", "cg", "grad"], default="ax")
    ap.add_argument("--dims", type=int, nargs=3, default=[16, 16, 16])
    ap.add_argument("--n", type=int, default=10)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--variant", type=int, default=0)
    ap.add_argument("--mixed", action="store_true")
    ap.add_argument("--method", type=int, default=0)
    ap.add_argument("--time", action="store_true")
    args = ap.parse_args(argv)
    dims, n = tuple(args.dims), args.n
    E = dims[0] * dims[1] * dims[2]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    prec = nekgb.NB_MIXED if args.mixed else nekgb.NB_FP64
    ctx = nekgb.nb_setup_box(dims, n, inputs.PERTURB_AMP, inputs.perturbation_coeffs(inputs.SEED_MESH),
                             prec, stream)
    nekgb.nb_set_ax_variant(ctx, args.variant)
    u = torch.from_numpy(inputs.local_field(E, n, inputs.SEED_U)).cuda()
    w = torch.empty_like(u)
    if args.op == "ax":
        for _ in range(args.reps):
            nekgb.nb_ax(ctx, u, w)
    elif args.op == "apply":
        for _ in range(args.reps):
            nekgb.nb_apply(ctx, u, w)
    elif args.op == "grad":
        umax = float(u.abs().max())
        nekgb.nb_probe_grad(ctx, args.method, u, w, umax)          # warm-up, not timed
        times = []
        for _ in range(args.reps):
            nekgb.nb_timing_enable(ctx, args.time)
            nekgb.nb_probe_grad(ctx, args.method, u, w, umax)
            if args.time:
                ms, _cnt = nekgb.nb_timing_read(ctx, nekgb.NB_K_AX, reset=True)
                times.append(ms)
        if args.time:
            times.sort()
            print(f"profile_case grad method={args.method} median_us={1e3 * times[len(times) // 2]:.2f} "
                  f"min_us={1e3 * times[0]:.2f} reps={len(times)}")
    else:
        fu = torch.from_numpy(inputs.unique_field(*dims, n, inputs.SEED_F)).cuda()
        f = torch.empty_like(u)
        nekgb.nb_scatter_unique(ctx, fu, f)
        nekgb.nb_mask(ctx, f)
        x = torch.zeros_like(u)
        nekgb.nb_cg_solve(ctx, f, x, tol=0.0, maxit=args.reps)
    stream.synchronize()
    nekgb.nb_destroy(ctx)
    print(f"profile_case {args.op} dims={dims} n={n} reps={args.reps} ok")


if __name__ == "__main__":
    main()
