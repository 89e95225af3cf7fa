"""The box partitioned into slabs of element layers (z), on CPU ranks.

The orchestration in paper_2005_13425_gb300.partition (slab bounds, the
interface protocol of the assembled operator, the scalar all-reduces, the
CG iteration) runs here with a test backend that does each slab's
arithmetic with the oracle (ax_e, the slab-local dssum, the mask, the
weighted products) and the interface-plane steps written out from their
definition.  Checked against the unpartitioned oracle:

* the assembled operator is the oracle's mask(dssum(ax_e)) bit for bit (the
  interface sums continue the lower slab's partial sums in ascending element
  order, exactly as the single-box dssum adds);
* 30 fixed CG iterations follow the oracle's CG (rho history and x to 1e-8:
  only the order of the inner-product sums differs);
* the same with two gloo ranks (world size 2, three slabs: rank 0 holds two
  of them, so local copies and point-to-point exchanges both occur) and with
  three (one slab per rank: the middle rank exchanges with both neighbours).
"""
import json
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

from paper_2005_13425_gb300 import inputs, partition

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DIMS, NGLL, PARTS = (3, 2, 5), 5, 3


def test_slab_bounds_and_ranks():
    assert partition.slab_bounds(5, 3) == [(0, 2), (2, 4), (4, 5)]
    assert partition.slab_bounds(16, 1) == [(0, 16)]
    assert partition.slab_bounds(16, 4) == [(0, 4), (4, 8), (8, 12), (12, 16)]
    with pytest.raises(ValueError):
        partition.slab_bounds(3, 4)
    assert [partition.slabs_of_rank(3, 2, r) for r in range(2)] == [(0, 2), (2, 3)]
    assert [partition.slabs_of_rank(8, 8, r) for r in range(8)] == [(k, k + 1) for k in range(8)]
    assert partition.plane_nodes((16, 16, 16), 10) == 145 * 145


class OracleSlab:
    """One slab with the oracle's arithmetic on torch CPU tensors."""

    def __init__(self, oracle, P, dims, n, z0, z1):
        Ex, Ey, Ez = dims
        e0, e1 = z0 * Ex * Ey, z1 * Ex * Ey
        self.o, self.n, self.sub = oracle, n, (Ex, Ey, z1 - z0)
        self.E = e1 - e0
        self.D = P["D"]
        self.g = np.ascontiguousarray(P["gxyz"][e0:e1])
        self.msk = np.ascontiguousarray(P["mask"][e0:e1])
        self.cw = 1.0 / P["mult"][e0:e1]
        self.has_below, self.has_above = z0 > 0, z1 < Ez
        self.plane = partition.plane_nodes(dims, n)
        self.top = self._plane_copies(z1 - z0 - 1, n - 1)
        self.bottom = self._plane_copies(0, 0)

    def _plane_copies(self, ezl, k):
        """Per plane node (x fastest), its copies (element, point) in
        ascending element order."""
        Ex, Ey, _ = self.sub
        n = self.n
        out = []
        for gy in range(Ey * (n - 1) + 1):
            for gx in range(Ex * (n - 1) + 1):
                cx = [(e, gx - e * (n - 1)) for e in range(Ex) if 0 <= gx - e * (n - 1) <= n - 1]
                cy = [(e, gy - e * (n - 1)) for e in range(Ey) if 0 <= gy - e * (n - 1) <= n - 1]
                out.append([(ex + Ex * (ey + Ey * ezl), i + n * (j + n * k)) for ey, j in cy for ex, i in cx])
        return out

    def new_field(self):
        return torch.zeros(self.E, self.n ** 3, dtype=torch.float64)

    def new_plane(self):
        return torch.zeros(self.plane, dtype=torch.float64)

    def ax(self, u, w):
        w.numpy()[:] = self.o.ax_e(self.D, self.g, u.numpy())

    def dssum(self, w):
        w.numpy()[:] = self.o.dssum(*self.sub, self.n, w.numpy())

    def mask(self, w):
        w.numpy()[:] = self.o.apply_mask(self.msk, w.numpy())

    def top_partial(self, w, buf):
        W, B = w.numpy(), buf.numpy()
        for q, cps in enumerate(self.top):
            s = 0.0
            for e, p in cps:
                s = s + W[e, p]
            B[q] = s

    def add_bottom(self, w, buf):
        W, B = w.numpy(), buf.numpy()
        for q, cps in enumerate(self.bottom):
            e, p = cps[0]
            W[e, p] = B[q] + W[e, p]

    def bottom_value(self, w, buf):
        W, B = w.numpy(), buf.numpy()
        for q, cps in enumerate(self.bottom):
            e, p = cps[0]
            B[q] = W[e, p]

    def set_top(self, w, buf):
        W, B = w.numpy(), buf.numpy()
        for q, cps in enumerate(self.top):
            for e, p in cps:
                W[e, p] = B[q]

    def dot(self, a, b):
        return float(np.sum(a.numpy() * self.cw * b.numpy()))

    def axpby(self, alpha, x, beta, y):
        Y = y.numpy()
        Y[:] = alpha * x.numpy() if beta == 0.0 else alpha * x.numpy() + beta * Y

    def copy(self, dst, src):
        dst.numpy()[:] = src.numpy()


def problem(oracle):
    P = oracle.box_problem(*DIMS, NGLL, inputs.PERTURB_AMP, inputs.perturbation_coeffs(3))
    f = oracle.apply_mask(P["mask"], oracle.scatter_unique(*DIMS, NGLL, inputs.unique_field(*DIMS, NGLL, seed=4)))
    u = inputs.local_field(P["E"], NGLL, seed=5)
    return P, f, u


def run_slabs(oracle, k0, k1, exchange):
    """The partitioned operator on u and 30 CG iterations on f, on slabs
    k0..k1-1; returns their local pieces."""
    P, f, u = problem(oracle)
    bounds = partition.slab_bounds(DIMS[2], PARTS)[k0:k1]
    slabs = [OracleSlab(oracle, P, DIMS, NGLL, z0, z1) for z0, z1 in bounds]
    per = DIMS[0] * DIMS[1]
    cut = lambda a, z0, z1: torch.from_numpy(np.ascontiguousarray(a[z0 * per:z1 * per]))
    box = partition.PartitionedBox(slabs, exchange)
    us = [cut(u, z0, z1) for z0, z1 in bounds]
    ws = [s.new_field() for s in slabs]
    box.apply(us, ws)
    fs = [cut(f, z0, z1) for z0, z1 in bounds]
    xs = [s.new_field() for s in slabs]
    it, rr, hist, bad = box.cg(fs, xs, tol=0.0, maxit=30)
    return np.concatenate([w.numpy() for w in ws]), np.concatenate([x.numpy() for x in xs]), it, hist, bad


def check_against_oracle(oracle, w, x, it, hist, bad):
    P, f, u = problem(oracle)
    want = oracle.apply_A(*DIMS, NGLL, P["D"], P["gxyz"], P["mask"], u)
    assert np.array_equal(w, want)                              # bit for bit
    x_ref, it_ref, rr_ref, hist_ref, st = oracle.cg(*DIMS, NGLL, P["D"], P["gxyz"], P["mask"], f,
                                                   tol=0.0, maxit=30)
    assert not bad and it == it_ref == 30
    hist = np.asarray(hist)
    assert np.abs(hist - hist_ref).max() <= 1e-8 * hist_ref.max()
    assert np.abs(x - x_ref).max() <= 1e-8 * np.abs(x_ref).max()


def test_partitioned_box_single_process(oracle):
    ex = partition.Exchange(PARTS, 0, PARTS)
    check_against_oracle(oracle, *run_slabs(oracle, 0, PARTS, ex))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_worker(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    import oracle as orc
    import test_partition as tp
    from paper_2005_13425_gb300 import partition as part
    orc.build()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        k0, k1 = part.slabs_of_rank(tp.PARTS, world, rank)
        ex = part.Exchange(tp.PARTS, k0, k1, dist=dist, rank=rank, world=world)
        w, x, it, hist, bad = tp.run_slabs(orc, k0, k1, ex)
        np.savez(os.path.join(outdir, f"rank{rank}.npz"), w=w, x=x)
        with open(os.path.join(outdir, f"rank{rank}.json"), "w") as fh:
            json.dump({"it": it, "hist": list(hist), "bad": bad}, fh)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_box_gloo_ranks(oracle, tmp_path, world):
    """world 2: rank 0 holds two of the three slabs (a local copy and a
    point-to-point exchange); world 3: one slab per rank, so the middle rank
    exchanges planes with both neighbours in both directions."""
    ctx = mp.get_context("spawn")
    port = _free_port()
    ps = [ctx.Process(target=_gloo_worker, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=300)
        assert p.exitcode == 0
    parts = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    meta = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert all(m["hist"] == meta[0]["hist"] for m in meta)     # the all-reduced scalars agree
    w = np.concatenate([p["w"] for p in parts])
    x = np.concatenate([p["x"] for p in parts])
    check_against_oracle(oracle, w, x, meta[0]["it"], meta[0]["hist"], meta[0]["bad"])


@pytest.mark.parametrize("dims,n,parts", [((2, 3, 4), 2, 4), ((3, 1, 5), 3, 2), ((1, 1, 3), 4, 3),
                                          ((2, 2, 7), 6, 5), ((4, 3, 2), 5, 2), ((1, 2, 9), 3, 9)])
def test_partitioned_operator_bit_exact_over_layouts(oracle, dims, n, parts):
    """The interface protocol over uneven slab counts, slabs one element
    layer thick, meshes one element wide and n = 2..6: the assembled
    operator equals the single-box mask(dssum(ax_e)) bit for bit."""
    P = oracle.box_problem(*dims, n, inputs.PERTURB_AMP, inputs.perturbation_coeffs(parts))
    u = inputs.local_field(P["E"], n, seed=parts + n)
    bounds = partition.slab_bounds(dims[2], parts)
    slabs = [OracleSlab(oracle, P, dims, n, z0, z1) for z0, z1 in bounds]
    per = dims[0] * dims[1]
    box = partition.PartitionedBox(slabs, partition.Exchange(parts, 0, parts))
    us = [torch.from_numpy(np.ascontiguousarray(u[z0 * per:z1 * per])) for z0, z1 in bounds]
    ws = [s.new_field() for s in slabs]
    box.apply(us, ws)
    got = np.concatenate([w.numpy() for w in ws])
    assert np.array_equal(got, oracle.apply_A(*dims, n, P["D"], P["gxyz"], P["mask"], u))
    # the slab shares of <a,b>_c add up to the whole box's
    a = [torch.from_numpy(np.ascontiguousarray(got[z0 * per:z1 * per])) for z0, z1 in bounds]
    tot = box.dots([(a, us)])[0]
    want = oracle.dot_c(*dims, n, got, u)
    assert abs(tot - want) <= 1e-13 * max(abs(want), 1e-300) * P["E"]
