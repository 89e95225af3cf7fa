"""The tensor-core measurement probe (nb_probe_grad) against FP64.

w_e = D_r u_e + D_s u_e + D_t u_e (the forward half of ax_e, Listing 1) by
the double-float line products (method 0) and by tcgen05 MMAs on a
base-512 digit split of u and D (methods 1 and 2: the directions one after
another or together), compared element by element
with the same sum formed in FP64 by numpy from the device's own D.  Both
must meet the 1e-12 max-norm relative bound of the FP64 operator; the
digit split is exact in its class sums, so any loss of bits in the tensor
cores' FP32 accumulation would show as errors near 2^-24.
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


def fp64_grad_sum(D, u, n):
    U = u.reshape(-1, n, n, n)                      # [e][k][j][i], i (r) fastest
    ur = np.einsum("il,ekjl->ekji", D, U)
    us = np.einsum("jl,ekli->ekji", D, U)
    ut = np.einsum("kl,elji->ekji", D, U)
    return (ur + us + ut).reshape(u.shape)


@pytest.mark.parametrize("dims,n,scale", [((2, 2, 3), 8, 1.0), ((3, 2, 2), 10, 1.0), ((5, 3, 2), 10, 3.7e5),
                                          ((16, 16, 16), 10, 1.0), ((16, 16, 16), 8, 2.0 ** -30)])
def test_probe_methods_match_fp64(nek, dims, n, scale):
    stream = torch.cuda.current_stream()
    s = inputs.perturbation_coeffs(inputs.SEED_MESH)
    ctx = nek.nb_setup_box(dims, n, inputs.PERTURB_AMP, s, stream=stream)
    try:
        E = dims[0] * dims[1] * dims[2]
        D = nek.nb_get_operator(ctx, n)
        u = inputs.local_field(E, n, seed=11 + n) * scale
        want = fp64_grad_sum(D, u, n)
        ud = torch.from_numpy(u).cuda()
        umax = float(np.abs(u).max())
        for method in (0, 1, 2):
            w = torch.full_like(ud, float("nan"))
            nek.nb_probe_grad(ctx, method, ud, w, umax)
            stream.synchronize()
            got = w.cpu().numpy()
            err = np.abs(got - want).max() / np.abs(want).max()
            assert np.isfinite(got).all()
            assert err <= 1e-12, (method, err)
    finally:
        nek.nb_destroy(ctx)


def test_probe_rejects_other_orders(nek):
    stream = torch.cuda.current_stream()
    ctx = nek.nb_setup_box((2, 2, 2), 6, inputs.PERTURB_AMP, inputs.perturbation_coeffs(inputs.SEED_MESH),
                           stream=stream)
    try:
        u = torch.zeros(8, 216, dtype=torch.float64, device="cuda")
        w = torch.zeros_like(u)
        with pytest.raises(nek.NekgbError) as ei:
            nek.nb_probe_grad(ctx, 1, u, w, 1.0)
        assert ei.value.status == nek.NB_ERR_ARG
    finally:
        nek.nb_destroy(ctx)
