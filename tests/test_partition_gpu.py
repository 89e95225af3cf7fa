"""The partitioned box on one GPU: several slab contexts (nb_setup_slab) in
one process, the interface exchanges as device copies between them.

* The assembled operator over the slabs equals the single-box nb_apply bit
  for bit (same device-built geometry per element, the interface sums
  continued in ascending element order), including slabs one element layer
  thick, meshes one element wide, n = 2..12 and 16^3 elements in two slabs.
* CG over the slabs follows the single-box solver and the oracle's CG
  (rho history and x to 1e-8 after fixed iterations).
* Whole-box calls on a slab context are refused.
"""
import numpy as np
import pytest

from paper_2005_13425_gb300 import inputs, partition

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


def host(t):
    torch.cuda.current_stream().synchronize()
    return t.cpu().numpy()


def slab_box(nek, dims, n, parts, s):
    stream = torch.cuda.current_stream()
    slabs = [partition.GpuSlab(nek, dims, z0, z1, n, inputs.PERTURB_AMP, s, stream)
             for z0, z1 in partition.slab_bounds(dims[2], parts)]
    return slabs, partition.PartitionedBox(slabs, partition.Exchange(parts, 0, parts))


def split(a, dims, parts):
    per = dims[0] * dims[1]
    return [torch.from_numpy(np.ascontiguousarray(a[z0 * per:z1 * per])).cuda()
            for z0, z1 in partition.slab_bounds(dims[2], parts)]


@pytest.mark.parametrize("dims,n,parts", [((5, 4, 7), 8, 3), ((3, 2, 4), 5, 4), ((16, 16, 16), 10, 2),
                                          ((1, 1, 3), 4, 3), ((2, 1, 5), 3, 5), ((1, 3, 2), 2, 2),
                                          ((4, 4, 6), 12, 4)])
def test_slab_operator_equals_single_box(nek, oracle, dims, n, parts):
    s = inputs.perturbation_coeffs(inputs.SEED_MESH)
    E = dims[0] * dims[1] * dims[2]
    u = inputs.local_field(E, n, seed=9)
    stream = torch.cuda.current_stream()
    one = nek.nb_setup_box(dims, n, inputs.PERTURB_AMP, s, stream=stream)
    try:
        w = torch.empty(E, n ** 3, dtype=torch.float64, device="cuda")
        nek.nb_apply(one, torch.from_numpy(u).cuda(), w)
        want = host(w)
    finally:
        nek.nb_destroy(one)
    slabs, box = slab_box(nek, dims, n, parts, s)
    try:
        us = split(u, dims, parts)
        ws = [sl.new_field() for sl in slabs]
        box.apply(us, ws)
        got = np.concatenate([host(w) for w in ws])
        with pytest.raises(nek.NekgbError) as ei:
            nek.nb_dot_c(slabs[0].ctx, ws[0], ws[0])
        assert ei.value.status == nek.NB_ERR_STATE
    finally:
        for sl in slabs:
            sl.close()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dims,n,parts,iters", [((5, 4, 7), 8, 3, 30), ((16, 16, 16), 10, 2, 20)])
def test_slab_cg_matches_single_box_and_oracle(nek, oracle, dims, n, parts, iters):
    s = inputs.perturbation_coeffs(inputs.SEED_MESH)
    P = oracle.box_problem(*dims, n, inputs.PERTURB_AMP, s)
    f = oracle.apply_mask(P["mask"], oracle.scatter_unique(*dims, n, inputs.unique_field(*dims, n, inputs.SEED_F)))
    x_ref, it_ref, rr_ref, hist_ref, st = oracle.cg(*dims, n, P["D"], P["gxyz"], P["mask"], f, tol=0.0, maxit=iters)
    stream = torch.cuda.current_stream()
    one = nek.nb_setup_box(dims, n, inputs.PERTURB_AMP, s, stream=stream)
    try:
        x1 = torch.zeros(P["E"], n ** 3, dtype=torch.float64, device="cuda")
        nek.nb_cg_solve(one, torch.from_numpy(f).cuda(), x1, tol=0.0, maxit=iters)
        x1 = host(x1)
        h1 = nek.nb_cg_history(one)
    finally:
        nek.nb_destroy(one)
    slabs, box = slab_box(nek, dims, n, parts, s)
    try:
        fs = split(f, dims, parts)
        xs = [sl.new_field() for sl in slabs]
        it, rr, hist, bad = box.cg(fs, xs, tol=0.0, maxit=iters)
        x = np.concatenate([host(v) for v in xs])
    finally:
        for sl in slabs:
            sl.close()
    hist = np.asarray(hist)
    assert not bad and it == iters == it_ref
    assert np.abs(hist - h1).max() <= 1e-10 * h1.max()
    assert np.abs(x - x1).max() <= 1e-10 * np.abs(x1).max()
    assert np.abs(hist - hist_ref).max() <= 1e-8 * hist_ref.max()
    assert np.abs(x - x_ref).max() <= 1e-8 * np.abs(x_ref).max()
