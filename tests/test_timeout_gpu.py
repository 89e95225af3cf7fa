"""Bounded device waits: the staged FP32 CG head gives up on a wait that runs
out, drains its copies in flight and ends the solve with NB_ERR_TIMEOUT.

The failure is made without faulting anything: a context set up with
NEKGB_TEST_UNARMED_WAIT_NS makes each CTA's first wait use a barrier that
nothing arrives on, with that (short) limit.  The copies actually in flight
complete and are waited for with the normal bound, so every CTA returns with
no copy outstanding; the host reads the status.  A fresh context then
solves normally on the same device.
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


def test_staged_head_wait_runs_out_then_fresh_context_solves(nek, oracle, monkeypatch):
    dims, n = (5, 4, 4), 10          # n = 10 takes the bulk-copy staged FP32 head
    P = oracle.box_problem(*dims, n, inputs.PERTURB_AMP, inputs.perturbation_coeffs(0))
    f = oracle.apply_mask(P["mask"], oracle.scatter_unique(*dims, n, inputs.unique_field(*dims, n, seed=3)))
    stream = torch.cuda.current_stream()
    fd = torch.from_numpy(f).cuda()

    monkeypatch.setenv("NEKGB_TEST_UNARMED_WAIT_NS", "2000000")      # 2 ms
    h = nek.nb_setup(dims, n, P["D"], P["gxyz"], prec=nek.NB_MIXED, stream=stream)
    monkeypatch.delenv("NEKGB_TEST_UNARMED_WAIT_NS")
    try:
        x = torch.zeros_like(fd)
        st, it, rr = nek.nb_cg_solve(h, fd, x, tol=1e-10, maxit=2000, allow=(nek.NB_ERR_TIMEOUT,))
        assert st == nek.NB_ERR_TIMEOUT
        assert "wait" in nek.nb_last_error()
        # the context's stream is still usable: the FP64 operator runs on it
        w = torch.empty_like(fd)
        nek.nb_apply(h, fd, w)
        stream.synchronize()
        assert torch.isfinite(w).all()
    finally:
        nek.nb_destroy(h)

    h = nek.nb_setup(dims, n, P["D"], P["gxyz"], prec=nek.NB_MIXED, stream=stream)
    try:
        x = torch.zeros_like(fd)
        st, it, rr = nek.nb_cg_solve(h, fd, x, tol=1e-10, maxit=5000)
        assert st == nek.NB_OK and rr <= 1e-10
        xm = x.cpu().numpy()
    finally:
        nek.nb_destroy(h)
    r = f - oracle.apply_A(*dims, n, P["D"], P["gxyz"], P["mask"], xm)
    assert np.sqrt(oracle.dot_c(*dims, n, r, r) / oracle.dot_c(*dims, n, f, f)) <= 1.5e-10


def test_exact_sum_range_check_stops_the_solve(nek, oracle, monkeypatch):
    """The FP64 CG head adds <w,p>_c exactly as 128-bit fixed-point shares
    whose scale comes from the <p,p>_c recursion.  A share that could
    overflow the sum sets a device-side flag and the solve stops with
    NB_ERR_BREAKDOWN instead of using a wrong alpha.  The test shifts the
    scale far up (NEKGB_TEST_DOT_SHIFT, read at set-up) so the first
    iteration's shares exceed the bound; a context without the shift solves
    normally."""
    dims, n = (4, 3, 3), 8
    P = oracle.box_problem(*dims, n, inputs.PERTURB_AMP, inputs.perturbation_coeffs(2))
    f = oracle.apply_mask(P["mask"], oracle.scatter_unique(*dims, n, inputs.unique_field(*dims, n, seed=5)))
    stream = torch.cuda.current_stream()
    fd = torch.from_numpy(f).cuda()
    monkeypatch.setenv("NEKGB_TEST_DOT_SHIFT", "60")
    h = nek.nb_setup(dims, n, P["D"], P["gxyz"], stream=stream)
    monkeypatch.delenv("NEKGB_TEST_DOT_SHIFT")
    try:
        x = torch.zeros_like(fd)
        st, it, rr = nek.nb_cg_solve(h, fd, x, tol=0.0, maxit=20, allow=(nek.NB_ERR_BREAKDOWN,))
        assert st == nek.NB_ERR_BREAKDOWN and "range" in nek.nb_last_error()
    finally:
        nek.nb_destroy(h)
    h = nek.nb_setup(dims, n, P["D"], P["gxyz"], stream=stream)
    try:
        x = torch.zeros_like(fd)
        st, it, rr = nek.nb_cg_solve(h, fd, x, tol=0.0, maxit=20)
        assert st == nek.NB_OK and it == 20
    finally:
        nek.nb_destroy(h)
    x_ref, *_ = oracle.cg(*dims, n, P["D"], P["gxyz"], P["mask"], f, tol=0.0, maxit=20)
    xg = x.cpu().numpy()
    assert np.abs(xg - x_ref).max() <= 1e-8 * np.abs(x_ref).max()
