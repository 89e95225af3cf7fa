"""The allocation-free weighted dot product, nb_dot_c_noalloc.

Some callers cannot allocate device memory: code whose device memory is all
owned by another allocator or a fixed pool, and code that must not block (a
device allocation or free can synchronise the device).  nb_dot_c_noalloc
serves them: it needs no context and keeps its scratch in a fixed device
array of the library.  This test calls it through the C ABI twice in a row,
on different inputs, and checks each result against the context-based
nb_dot_c and against the CPU oracle's dot_c on the same fields, with the
relative tolerance the other dot-product tests use.
"""
import numpy as np
import pytest

from paper_2005_13425_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DOT_TOL = 1e-12


@pytest.fixture(scope="module")
def nek():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_13425_gb300 import build as b
    b.build()
    from paper_2005_13425_gb300 import nekgb
    nekgb.load()
    return nekgb


@pytest.mark.parametrize("dims,n", [((4, 3, 3), 8), ((16, 16, 16), 10)])
def test_noalloc_dot_matches_context_dot_twice(nek, oracle, dims, n):
    stream = torch.cuda.Stream()
    E = dims[0] * dims[1] * dims[2]
    ah = inputs.local_field(E, n, seed=11)
    bh = inputs.local_field(E, n, seed=12)
    with torch.cuda.stream(stream):
        a = torch.from_numpy(ah).cuda()
        b = torch.from_numpy(bh).cuda()
        out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        ctx = nek.nb_setup_box(dims, n, 0.05, inputs.perturbation_coeffs(0), stream=stream)
        try:
            for (x, y), (xh, yh) in zip(((a, b), (b, b)), ((ah, bh), (bh, bh))):   # two calls in a row
                nek.nb_dot_c_noalloc(dims, n, x, y, out, stream)
                stream.synchronize()
                got = float(out.cpu()[0])
                want = nek.nb_dot_c(ctx, x, y)
                assert abs(got - want) <= DOT_TOL * abs(want), (got, want)
                ref = oracle.dot_c(*dims, n, xh, yh)
                assert abs(got - ref) <= DOT_TOL * abs(ref), (got, ref)
        finally:
            nek.nb_destroy(ctx)


def test_noalloc_dot_rejects_meshes_beyond_its_scratch(nek):
    big = (33, 33, 33)                                # 35937 elements > 32768
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(nek.NekgbError) as ei:
        nek.nb_dot_c_noalloc(big, 2, x, x, x[:1])
    assert ei.value.status == nek.NB_ERR_ARG
    assert "32768" in str(ei.value)
