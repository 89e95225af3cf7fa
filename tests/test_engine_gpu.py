"""Batched / served solves through the engine (nb_engine_*).

* Each admitted problem converges: its returned x has an FP64 residual, in
  the oracle's operator, within 2x the requested tolerance.
* A problem's result is bit-identical whether it is solved alone or in a
  mix of other problems (per-problem tiles and fixed-order reductions).
* Admission is by arena footprint: too-large requests are refused with
  NB_ERR_OOM until retired requests free space.
* Mixed-precision requests (FP32 inner CG, FP64 defect correction) reach
  the FP64 tolerance in the oracle's operator, alone or next to FP64
  requests, with bit-identical results in any mix.
"""
import numpy as np
import pytest

from paper_2005_13425_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GIB = 1 << 30


@pytest.fixture(scope="module")
def nek(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    os.environ.setdefault("NEKGB_TUNE_CACHE", str(tmp_path_factory.mktemp("tune") / "tune.txt"))
    from paper_2005_13425_gb300 import build as b
    b.build()
    from paper_2005_13425_gb300 import nekgb
    nekgb.load()
    torch.cuda.set_stream(torch.cuda.Stream())
    return nekgb


def problem(oracle, dims, n, pid):
    s = inputs.perturbation_coeffs(100 + pid)
    P = oracle.box_problem(*dims, n, inputs.PERTURB_AMP, s)
    f = oracle.apply_mask(P["mask"], oracle.scatter_unique(*dims, n, inputs.unique_field(*dims, n, seed=200 + pid)))
    return P, s, f


def run_engine(nek, items, arena=4 * GIB, iters_per_step=64, max_steps=400):
    """items: list of (dims, n, s, f, tol, maxit[, prec]).  Returns per-item
    (x, iters, relres, status, outer corrections)."""
    stream = torch.cuda.current_stream()
    eng = nek.nb_engine_create(arena, stream)
    try:
        ids = []
        for dims, n, s, f, tol, maxit, *prec in items:
            st, rid = nek.nb_engine_submit(eng, dims, n, inputs.PERTURB_AMP, s, tol, maxit,
                                           torch.from_numpy(f).cuda(), prec=prec[0] if prec else nek.NB_FP64)
            ids.append(rid)
        out = [None] * len(items)
        for _ in range(max_steps):
            nek.nb_engine_step(eng, iters_per_step)
            for k, rid in enumerate(ids):
                if out[k] is None:
                    done, it, rr, st = nek.nb_engine_poll(eng, rid)
                    if done:
                        _, outer = nek.nb_engine_request_info(eng, rid)
                        x = torch.empty(items[k][3].shape, dtype=torch.float64, device="cuda")
                        nek.nb_engine_retire(eng, rid, x)
                        stream.synchronize()
                        out[k] = (x.cpu().numpy(), it, rr, st, outer)
            if all(o is not None for o in out):
                break
        return out
    finally:
        nek.nb_engine_destroy(eng)


def true_relres(oracle, dims, n, P, f, x):
    r = f - oracle.apply_A(*dims, n, P["D"], P["gxyz"], P["mask"], x)
    return np.sqrt(oracle.dot_c(*dims, n, r, r) / oracle.dot_c(*dims, n, f, f))


def test_engine_batch_converges_against_oracle(nek, oracle):
    specs = [((2, 2, 2), 6), ((4, 2, 2), 8), ((2, 2, 1), 10), ((3, 2, 2), 6), ((2, 2, 2), 12)]
    items, probs = [], []
    for pid, (dims, n) in enumerate(specs):
        P, s, f = problem(oracle, dims, n, pid)
        probs.append((dims, n, P, f))
        items.append((dims, n, s, f, 1e-10, 5000))
    out = run_engine(nek, items)
    for (dims, n, P, f), (x, it, rr, st, _) in zip(probs, out):
        assert st == nek.NB_OK and rr <= 1e-10 and it > 0
        assert true_relres(oracle, dims, n, P, f, x) <= 2e-10


def test_engine_alone_equals_mix(nek, oracle):
    target = ((3, 2, 2), 8)
    P, s, f = problem(oracle, *target, 7)
    item = (target[0], target[1], s, f, 1e-10, 5000)
    alone = run_engine(nek, [item])[0]
    others = []
    for pid, (dims, n) in enumerate([((2, 2, 2), 6), ((4, 4, 2), 8), ((2, 1, 1), 10)]):
        _, s2, f2 = problem(oracle, dims, n, 20 + pid)
        others.append((dims, n, s2, f2, 1e-9, 3000))
    mixed = run_engine(nek, others[:2] + [item] + others[2:])[2]
    assert alone[1] == mixed[1] and alone[2] == mixed[2]
    assert np.array_equal(alone[0], mixed[0])          # bit-identical


def test_engine_fixed_iterations_match_single_solver(nek, oracle):
    dims, n = (3, 3, 2), 6
    P, s, f = problem(oracle, dims, n, 3)
    x_eng, it, rr, st, _ = run_engine(nek, [(dims, n, s, f, 0.0, 24)], iters_per_step=8)[0]
    assert it == 24
    x_ref, it_ref, rr_ref, _, _ = oracle.cg(*dims, n, P["D"], P["gxyz"], P["mask"], f, tol=0.0, maxit=24)
    assert np.abs(x_eng - x_ref).max() <= 1e-8 * np.abs(x_ref).max()
    assert abs(rr - rr_ref) <= 1e-8 * rr_ref


def test_engine_admission_by_footprint(nek, oracle):
    dims, n = (4, 4, 4), 8
    need = nek.nb_engine_footprint(dims, n)
    _, s, f = problem(oracle, dims, n, 5)
    fd = torch.from_numpy(f).cuda()
    eng = nek.nb_engine_create(int(need * 1.5) + (1 << 20), torch.cuda.current_stream())
    try:
        st1, a = nek.nb_engine_submit(eng, dims, n, 0.05, s, 1e-8, 100, fd)
        st2, b = nek.nb_engine_submit(eng, dims, n, 0.05, s, 1e-8, 100, fd, allow=(nek.NB_OK, nek.NB_ERR_OOM))
        assert st1 == nek.NB_OK and st2 == nek.NB_ERR_OOM and b == -1
        used, cap, active = nek.nb_engine_stats(eng)
        assert active == 1 and used >= need
        nek.nb_engine_retire(eng, a)
        st3, c = nek.nb_engine_submit(eng, dims, n, 0.05, s, 1e-8, 100, fd)
        assert st3 == nek.NB_OK
        lpt, te = nek.nb_engine_tuning(eng, n, nek.NB_FP64)
        assert lpt in (1, 2) and te in (4, 8, 16)
        nek.nb_engine_retire(eng, c)
    finally:
        nek.nb_engine_destroy(eng)


def test_engine_mixed_converges_against_oracle(nek, oracle):
    specs = [((2, 2, 2), 6), ((4, 2, 2), 8), ((2, 2, 1), 10), ((3, 3, 2), 12)]
    items, probs = [], []
    for pid, (dims, n) in enumerate(specs):
        P, s, f = problem(oracle, dims, n, 40 + pid)
        probs.append((dims, n, P, f))
        items.append((dims, n, s, f, 1e-10, 20000, nek.NB_MIXED))
    # one FP64 request in the same engine
    P, s, f = problem(oracle, (3, 2, 2), 8, 49)
    probs.append(((3, 2, 2), 8, P, f))
    items.append(((3, 2, 2), 8, s, f, 1e-10, 5000, nek.NB_FP64))
    out = run_engine(nek, items, iters_per_step=32)
    for k, ((dims, n, P, f), (x, it, rr, st, outer)) in enumerate(zip(probs, out)):
        assert st == nek.NB_OK and rr <= 1e-10 and it > 0
        assert true_relres(oracle, dims, n, P, f, x) <= 2e-10
        if k < len(specs):
            assert outer >= 2          # at least one correction after the first inner solve
        else:
            assert outer == 0


def test_engine_mixed_alone_equals_mix(nek, oracle):
    target = ((3, 2, 2), 10)
    P, s, f = problem(oracle, *target, 57)
    item = (target[0], target[1], s, f, 1e-10, 20000, nek.NB_MIXED)
    alone = run_engine(nek, [item], iters_per_step=16)[0]
    others = []
    for pid, (dims, n, prec) in enumerate([((2, 2, 2), 6, nek.NB_MIXED), ((4, 4, 2), 8, nek.NB_FP64),
                                           ((2, 1, 1), 10, nek.NB_MIXED)]):
        _, s2, f2 = problem(oracle, dims, n, 60 + pid)
        others.append((dims, n, s2, f2, 1e-9, 3000, prec))
    mixed = run_engine(nek, others[:2] + [item] + others[2:], iters_per_step=16)[2]
    assert alone[1] == mixed[1] and alone[2] == mixed[2] and alone[4] == mixed[4]
    assert np.array_equal(alone[0], mixed[0])          # bit-identical


def test_engine_mixed_footprint_and_budget(nek, oracle):
    dims, n = (3, 2, 2), 8
    f64 = nek.nb_engine_footprint(dims, n, nek.NB_FP64)
    fmx = nek.nb_engine_footprint(dims, n, nek.NB_MIXED)
    pts = 12 * n ** 3
    assert fmx > f64 and fmx - f64 >= (72 + 40 - 48 - 32) * pts
    # a budget too small to converge ends the request with NB_ERR_NOT_CONVERGED
    P, s, f = problem(oracle, dims, n, 70)
    x, it, rr, st, outer = run_engine(nek, [(dims, n, s, f, 1e-12, 10, nek.NB_MIXED)], iters_per_step=8)[0]
    assert st == nek.NB_ERR_NOT_CONVERGED and 0 < it <= 10 and rr > 1e-12


def test_engine_tunes_per_precision(nek, oracle):
    dims, n = (2, 2, 2), 7
    _, s, f = problem(oracle, dims, n, 80)
    eng = nek.nb_engine_create(1 << 30, torch.cuda.current_stream())
    try:
        assert nek.nb_engine_tuning(eng, n, nek.NB_MIXED) == (0, 0)        # not used yet
        st, rid = nek.nb_engine_submit(eng, dims, n, inputs.PERTURB_AMP, s, 1e-8, 1000,
                                       torch.from_numpy(f).cuda(), prec=nek.NB_MIXED)
        lpt, te = nek.nb_engine_tuning(eng, n, nek.NB_MIXED)
        assert lpt == 1 and te in (4, 8, 16)
        assert nek.nb_engine_tuning(eng, n, nek.NB_FP64) == (0, 0)         # tuned separately
        nek.nb_engine_retire(eng, rid)
    finally:
        nek.nb_engine_destroy(eng)


def test_engine_staged_f32_head_matches_plain(nek, oracle):
    """The bulk-copy staged FP32 head (n = 10) and the plain one give
    bit-identical mixed solves; the staged one crosses tile and problem
    boundaries (several problems of the same n)."""
    import os
    items = []
    for pid, (dims, n) in enumerate([((3, 2, 2), 10), ((2, 2, 3), 10), ((5, 3, 2), 10)]):
        _, s, f = problem(oracle, dims, n, 90 + pid)
        items.append((dims, n, s, f, 1e-10, 20000, nek.NB_MIXED))
    outs = []
    for staged in ("1", "0"):
        old = os.environ.get("NEKGB_F32_STAGED")
        os.environ["NEKGB_F32_STAGED"] = staged
        try:
            outs.append(run_engine(nek, items, iters_per_step=32))
        finally:
            if old is None:
                del os.environ["NEKGB_F32_STAGED"]
            else:
                os.environ["NEKGB_F32_STAGED"] = old
    for a, b in zip(*outs):
        assert a[1] == b[1] and a[2] == b[2] and a[4] == b[4] and a[3] == nek.NB_OK
        assert np.array_equal(a[0], b[0])


def test_engine_batch_at_full_sizes_against_oracle(nek, oracle):
    """The batched engine at the sizes the 256-problem list draws: 16^3
    elements at n = 10 and 8^3 at n = 12 (the largest E and n), with small
    problems of other n in the same batch.  FP64 requests run 30 fixed
    iterations and are compared with the oracle's CG (rho history and x to
    1e-8, CG's reduction-order amplification); mixed requests of the two
    large problems reach relative residual 1e-10 in the oracle's operator."""
    big = [((16, 16, 16), 10), ((8, 8, 8), 12)]
    small = [((2, 2, 2), 6), ((4, 2, 2), 8)]
    items, probs = [], []
    for pid, (dims, n) in enumerate(big + small):
        P, s, f = problem(oracle, dims, n, 120 + pid)
        probs.append((dims, n, P, f))
        items.append((dims, n, s, f, 0.0, 30, nek.NB_FP64))
    for pid, (dims, n) in enumerate(big):
        _, s, f = problem(oracle, dims, n, 120 + pid)
        items.append((dims, n, s, f, 1e-10, 20000, nek.NB_MIXED))
    out = run_engine(nek, items, arena=16 * GIB, iters_per_step=32)
    for (dims, n, P, f), (x, it, rr, st, _) in zip(probs, out[:len(probs)]):
        x_ref, it_ref, rr_ref, _, _ = oracle.cg(*dims, n, P["D"], P["gxyz"], P["mask"], f, tol=0.0, maxit=30)
        assert st == nek.NB_OK and it == 30 == it_ref
        assert np.abs(x - x_ref).max() <= 1e-8 * np.abs(x_ref).max()
        assert abs(rr - rr_ref) <= 1e-8 * rr_ref
    for (dims, n, P, f), (x, it, rr, st, outer) in zip(probs, out[len(probs):]):
        assert st == nek.NB_OK and rr <= 1e-10 and outer >= 2
        assert true_relres(oracle, dims, n, P, f, x) <= 2e-10
