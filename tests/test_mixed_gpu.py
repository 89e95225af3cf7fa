"""Mixed precision (FP32 inner operator inside FP64 defect correction).

* The FP32 operator against the oracle, to an FP32 tolerance: max-norm
  relative 2e-5 (FP32 unit roundoff 6e-8 times n-term sums and the ~25x
  cancellation of the transposed derivative for random data).
* The FP32 dssum against a brute-force FP32 sum in ascending element order
  (bit-exact: same additions in the same order in IEEE single precision).
* The defect-correction solve reaches the FP64 relative residual asked for
  and agrees with the FP64 oracle's solution (manufactured solution).
"""
import numpy as np
import pytest

from paper_2005_13425_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nek():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_13425_gb300 import build as b
    b.build()
    from paper_2005_13425_gb300 import nekgb
    nekgb.load()
    torch.cuda.set_stream(torch.cuda.Stream())
    return nekgb


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.current_stream().synchronize()
    return t.cpu().numpy()


def mixed_ctx(nek, P, dims, n):
    return nek.nb_setup(dims, n, P["D"], P["gxyz"], prec=nek.NB_MIXED, stream=torch.cuda.current_stream())


@pytest.mark.parametrize("dims,n", [((3, 2, 2), 4), ((3, 2, 2), 8), ((2, 2, 2), 10), ((2, 1, 1), 16)])
def test_f32_operator_parity(nek, oracle, dims, n):
    P = oracle.box_problem(*dims, n, 0.05, inputs.perturbation_coeffs(0))
    u = inputs.local_field(P["E"], n, seed=n)
    want = oracle.ax_e(P["D"], P["gxyz"], u)
    h = mixed_ctx(nek, P, dims, n)
    try:
        w = torch.empty(P["E"], n ** 3, dtype=torch.float32, device="cuda")
        nek.nb_ax_f32(h, dev(u.astype(np.float32)), w)
        got = host(w).astype(np.float64)
    finally:
        nek.nb_destroy(h)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err <= 2e-5, err


def test_f32_dssum_exact(nek, oracle):
    dims, n = (3, 2, 2), 4
    E = 12
    rng = np.random.default_rng(3)
    w = rng.uniform(-1, 1, (E, n ** 3)).astype(np.float32)
    gid = oracle.gid(*dims, n)
    want = np.empty_like(w)
    groups = {}
    for e in range(E):
        for q in range(n ** 3):
            groups.setdefault(int(gid[e, q]), []).append((e, q))
    for copies in groups.values():
        s = np.float32(0.0)
        for e, q in sorted(copies):
            s = np.float32(s + w[e, q])
        for e, q in copies:
            want[e, q] = s
    P = oracle.box_problem(*dims, n, 0.0, (0, 0, 0))
    h = mixed_ctx(nek, P, dims, n)
    try:
        wd = dev(w)
        nek.nb_dssum_f32(h, wd)
        got = host(wd)
    finally:
        nek.nb_destroy(h)
    assert np.array_equal(got, want)


def manufactured(oracle, dims, n, seed=1):
    P = oracle.box_problem(*dims, n, 0.05, inputs.perturbation_coeffs(seed))
    xyz = P["xyz"]
    us = np.sin(np.pi * xyz[:, 0]) * np.sin(np.pi * xyz[:, 1]) * np.sin(np.pi * xyz[:, 2])
    us = oracle.apply_mask(P["mask"], us)
    f = oracle.apply_A(*dims, n, P["D"], P["gxyz"], P["mask"], us)
    return P, us, f


@pytest.mark.parametrize("dims,n", [((3, 3, 2), 6), ((4, 4, 4), 8)])
def test_mixed_defect_correction_reaches_fp64_residual(nek, oracle, dims, n):
    P, us, f = manufactured(oracle, dims, n)
    x_ref, it_ref, rr_ref, _, _ = oracle.cg(*dims, n, P["D"], P["gxyz"], P["mask"], f, tol=1e-10, maxit=10000)
    h = mixed_ctx(nek, P, dims, n)
    try:
        x = torch.zeros_like(dev(f))
        st, it, rr = nek.nb_cg_solve(h, dev(f), x, tol=1e-10, maxit=20000)
        iters, outer = nek.nb_solve_stats(h)
        xm = host(x)
    finally:
        nek.nb_destroy(h)
    assert rr <= 1e-10 and outer >= 2 and iters == it
    # FP64 residual of the returned x, recomputed by the oracle
    r = f - oracle.apply_A(*dims, n, P["D"], P["gxyz"], P["mask"], xm)
    true_rel = np.sqrt(oracle.dot_c(*dims, n, r, r) / oracle.dot_c(*dims, n, f, f))
    assert true_rel <= 1.5e-10
    # same discrete solution as the FP64 oracle (both within kappa * 1e-10)
    assert np.abs(xm - x_ref).max() <= 1e-7 * np.abs(x_ref).max()
    assert np.abs(xm - us).max() <= 1e-7


def test_mixed_params_and_errors(nek, oracle):
    dims, n = (2, 2, 2), 5
    P, us, f = manufactured(oracle, dims, n)
    h = mixed_ctx(nek, P, dims, n)
    try:
        with pytest.raises(nek.NekgbError):
            nek.nb_set_mixed_params(h, 0.0, 3)
        nek.nb_set_mixed_params(h, 1e-3, 2)
        x = torch.zeros_like(dev(f))
        st, it, rr = nek.nb_cg_solve(h, dev(f), x, tol=1e-12, maxit=5000,
                                     allow=(nek.NB_ERR_NOT_CONVERGED,))
        _, outer = nek.nb_solve_stats(h)
        assert st == nek.NB_ERR_NOT_CONVERGED and outer == 2 and rr > 1e-12
    finally:
        nek.nb_destroy(h)
    # the FP32 operator needs an NB_MIXED context
    h = nek.nb_setup(dims, n, P["D"], P["gxyz"], stream=torch.cuda.current_stream())
    try:
        w = torch.empty(8, n ** 3, dtype=torch.float32, device="cuda")
        with pytest.raises(nek.NekgbError) as ei:
            nek.nb_ax_f32(h, w.clone(), w)
        assert ei.value.status == nek.NB_ERR_STATE
    finally:
        nek.nb_destroy(h)


def _ctx_with_staging(nek, P, dims, n, staged):
    import os
    old = os.environ.get("NEKGB_F32_STAGED")
    os.environ["NEKGB_F32_STAGED"] = "1" if staged else "0"
    try:
        return mixed_ctx(nek, P, dims, n)
    finally:
        if old is None:
            del os.environ["NEKGB_F32_STAGED"]
        else:
            os.environ["NEKGB_F32_STAGED"] = old


@pytest.mark.parametrize("dims,n", [((7, 7, 7), 10), ((3, 2, 1), 10), ((9, 8, 6), 6), ((8, 8, 6), 8)])
def test_f32_staged_operator_and_solve_match_plain(nek, oracle, dims, n):
    """The bulk-copy staged FP32 kernel (two elements in flight per CTA; the
    meshes have more elements than resident CTAs, so the stage ring turns
    over) computes the same arithmetic as the plain kernel: bit-identical
    operator output and inner CG, and the oracle's operator to FP32
    tolerance."""
    P = oracle.box_problem(*dims, n, 0.05, inputs.perturbation_coeffs(3))
    u = inputs.local_field(P["E"], n, seed=n + 1)
    want = oracle.ax_e(P["D"], P["gxyz"], u)
    fu = inputs.unique_field(*dims, n, seed=4)
    f = oracle.apply_mask(P["mask"], oracle.scatter_unique(*dims, n, fu))
    outs = []
    for staged in (True, False):
        h = _ctx_with_staging(nek, P, dims, n, staged)
        try:
            w = torch.empty(P["E"], n ** 3, dtype=torch.float32, device="cuda")
            nek.nb_ax_f32(h, dev(u.astype(np.float32)), w)
            x = torch.zeros_like(dev(f))
            st, it, rr = nek.nb_cg_solve(h, dev(f), x, tol=1e-10, maxit=20000)
            outs.append((host(w), host(x), it, rr))
        finally:
            nek.nb_destroy(h)
    (w1, x1, it1, rr1), (w0, x0, it0, rr0) = outs
    assert np.array_equal(w1, w0)
    assert it1 == it0 and rr1 == rr0 and np.array_equal(x1, x0)
    err = np.abs(w1.astype(np.float64) - want).max() / np.abs(want).max()
    assert err <= 2e-5, err
    assert rr1 <= 1e-10


@pytest.mark.parametrize("n", [8, 10])
def test_config3_full_size_against_oracle(nek, oracle, n):
    """The mixed configuration at its own size: E = 4096 (16 x 16 x 16),
    n = 8 and 10, manufactured solution u* = sin(pi x) sin(pi y) sin(pi z)
    with f = A u* from the FP64 oracle on the oracle's mesh; defect
    correction to relative residual 1e-10.  Checked: the FP64 relative
    residual of the result recomputed by the oracle, and its error against
    u* and against the oracle's own FP64 CG solution (both within
    kappa * 1e-10 of the exact discrete solution)."""
    dims = (16, 16, 16)
    P, us, f = manufactured(oracle, dims, n, seed=inputs.SEED_MESH)
    x_ref, it_ref, rr_ref, _, st_ref = oracle.cg(*dims, n, P["D"], P["gxyz"], P["mask"], f,
                                                  tol=1e-10, maxit=20000)
    assert st_ref == 0 and rr_ref <= 1e-10
    h = mixed_ctx(nek, P, dims, n)
    try:
        x = torch.zeros_like(dev(f))
        st, it, rr = nek.nb_cg_solve(h, dev(f), x, tol=1e-10, maxit=20000)
        _, outer = nek.nb_solve_stats(h)
        xm = host(x)
    finally:
        nek.nb_destroy(h)
    assert st == nek.NB_OK and rr <= 1e-10 and outer >= 2
    r = f - oracle.apply_A(*dims, n, P["D"], P["gxyz"], P["mask"], xm)
    true_rel = np.sqrt(oracle.dot_c(*dims, n, r, r) / oracle.dot_c(*dims, n, f, f))
    assert true_rel <= 1.5e-10, true_rel
    umax = np.abs(us).max()
    assert np.abs(xm - us).max() <= 1e-7 * umax
    assert np.abs(xm - x_ref).max() <= 1e-7 * umax
