"""The box solved on several slabs: host-side orchestration of the
partitioned CG (one slab of element layers along z per GPU or rank).

Nekbone distributes its elements over MPI processes (arXiv 2005.13425,
Sec. I-II); within the operator, the second step sums element results into
the shared nodes (Sec. III), which across a partition becomes an exchange
between neighbouring slabs, and every CG inner product becomes a sum over
the slabs.  This module holds only the orchestration:

* which element layers each slab holds (``slab_bounds``);
* the interface protocol of the assembled operator (``PartitionedBox.apply``):
  the top-plane partial sums go up, the upper slab continues the sum from
  them inside its own dssum, and the final values come back down, which
  gives the single-box dssum bit for bit (the library's slab kernels
  document why);
* the scalar all-reduces of CG (<w,p>_c and <r,r>_c per iteration, summed
  over the local slabs in slab order, then over ranks);
* the CG iteration in Nekbone's form (unpreconditioned, local storage, the
  stopping test on sqrt(<r,r>_c / <f,f>_c)).

Every arithmetic step runs in a per-slab backend: on the GPU, ``GpuSlab``
calls the library's kernels (libnekgb, ``nb_setup_slab`` and ``nb_slab_*``).
``Exchange`` moves plane buffers between the slabs a process holds by copy
and to and from other ranks with ``torch.distributed`` point-to-point
operations (NCCL for device buffers, gloo for host buffers); no kernel waits
on another slab.
"""
from __future__ import annotations

import math


def slab_bounds(ez: int, parts: int):
    """Element layers [z0, z1) of each of `parts` slabs of a box `ez` layers
    high: contiguous, the first ez % parts slabs one layer thicker."""
    if parts < 1 or parts > ez:
        raise ValueError(f"cannot cut {ez} element layers into {parts} slabs")
    base, extra = divmod(ez, parts)
    out, z = [], 0
    for k in range(parts):
        h = base + (1 if k < extra else 0)
        out.append((z, z + h))
        z += h
    return out


def slabs_of_rank(parts: int, world: int, rank: int):
    """Contiguous range [k0, k1) of slab indices held by `rank`."""
    if parts < world:
        raise ValueError("need at least one slab per rank")
    base, extra = divmod(parts, world)
    k0 = rank * base + min(rank, extra)
    return k0, k0 + base + (1 if rank < extra else 0)


def plane_nodes(dims, n: int) -> int:
    """Nodes of one interface plane: (Ex (n-1) + 1) (Ey (n-1) + 1)."""
    return (dims[0] * (n - 1) + 1) * (dims[1] * (n - 1) + 1)


class Exchange:
    """Plane buffers between consecutive slabs and sums over all slabs.

    The process holds slabs k0 .. k1-1 of `parts`; rank r holds the range
    ``slabs_of_rank(parts, world, r)``.  Buffers are torch tensors (on the
    device with NCCL, on the host with gloo)."""

    def __init__(self, parts: int, k0: int, k1: int, dist=None, rank: int = 0, world: int = 1,
                 device="cpu"):
        self.parts, self.k0, self.k1 = parts, k0, k1
        self.dist, self.rank, self.world, self.device = dist, rank, world, device
        if dist is not None and world > 1:
            dist.barrier()       # the first batched point-to-point call is then not the group's first

    def _p2p(self, sends, recvs):
        """sends / recvs: lists of (tensor, peer rank)."""
        if not sends and not recvs:
            return
        d = self.dist
        ops = [d.P2POp(d.isend, t, peer) for t, peer in sends] + \
              [d.P2POp(d.irecv, t, peer) for t, peer in recvs]
        for req in d.batch_isend_irecv(ops):
            req.wait()

    def shift_up(self, send, recv):
        """recv[i] (bottom plane of local slab k0+i) := send of slab k0+i-1
        (its top plane).  send[i] / recv[i] are None where the slab has no
        neighbour above / below."""
        for i in range(1, len(send)):
            recv[i].copy_(send[i - 1])
        sends, recvs = [], []
        if self.k1 < self.parts:
            sends.append((send[-1], self.rank + 1))
        if self.k0 > 0:
            recvs.append((recv[0], self.rank - 1))
        self._p2p(sends, recvs)

    def shift_down(self, send, recv):
        """recv[i] (top plane of local slab k0+i) := send of slab k0+i+1
        (its bottom plane)."""
        for i in range(len(send) - 1):
            recv[i].copy_(send[i + 1])
        sends, recvs = [], []
        if self.k0 > 0:
            sends.append((send[0], self.rank - 1))
        if self.k1 < self.parts:
            recvs.append((recv[-1], self.rank + 1))
        self._p2p(sends, recvs)

    def allreduce(self, values):
        """Sum of per-slab scalars: over the local slabs in slab order, then
        over ranks (FP64)."""
        local = [0.0] * len(values[0])
        for v in values:
            for q in range(len(local)):
                local[q] += v[q]
        if self.dist is None or self.world == 1:
            return local
        import torch
        t = torch.tensor(local, dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return [float(x) for x in t.cpu()]


class PartitionedBox:
    """The assembled operator, inner products and CG over the slabs held by
    this process.  `slabs` are backends in slab order (see GpuSlab)."""

    def __init__(self, slabs, exchange: Exchange):
        self.slabs = slabs
        self.ex = exchange
        self._up = [s.new_plane() for s in slabs]
        self._down = [s.new_plane() for s in slabs]
        self._from_below = [s.new_plane() for s in slabs]
        self._from_above = [s.new_plane() for s in slabs]

    def apply(self, us, ws):
        """ws = mask(dssum(ax_e(us))) over the whole box."""
        S = self.slabs
        for s, u, w in zip(S, us, ws):
            s.ax(u, w)
        for s, w, b in zip(S, ws, self._up):
            if s.has_above:
                s.top_partial(w, b)
        self.ex.shift_up(self._up, self._from_below)
        for s, w, b in zip(S, ws, self._from_below):
            if s.has_below:
                s.add_bottom(w, b)
        for s, w in zip(S, ws):
            s.dssum(w)
        for s, w, b in zip(S, ws, self._down):
            if s.has_below:
                s.bottom_value(w, b)
        self.ex.shift_down(self._down, self._from_above)
        for s, w, b in zip(S, ws, self._from_above):
            if s.has_above:
                s.set_top(w, b)
        for s, w in zip(S, ws):
            s.mask(w)

    def dots(self, pairs):
        """Whole-box <a,b>_c for each (as, bs) pair of per-slab field lists."""
        vals = [[s.dot(a[i], b[i]) for (a, b) in pairs] for i, s in enumerate(self.slabs)]
        return self.ex.allreduce(vals)

    def cg(self, fs, xs, tol: float = 0.0, maxit: int = 100):
        """Unpreconditioned CG in Nekbone's form on local storage (x in:
        initial guess, out: solution; f masked).  Returns (iterations,
        relative residual sqrt(<r,r>_c / <f,f>_c), <r,r>_c history,
        breakdown flag)."""
        S = self.slabs
        rs = [s.new_field() for s in S]
        ps = [s.new_field() for s in S]
        ws = [s.new_field() for s in S]
        self.apply(xs, ws)
        for s, r, f, w in zip(S, rs, fs, ws):
            s.copy(r, f)
            s.axpby(-1.0, w, 1.0, r)
        rho, f2 = self.dots([(rs, rs), (fs, fs)])
        fnorm = math.sqrt(f2)
        hist = [rho]
        rho_old = 1.0
        iters = 0
        breakdown = False
        for it in range(1, maxit + 1):
            if rho == 0.0 or (tol > 0.0 and math.sqrt(rho) / fnorm <= tol):
                break
            beta = 0.0 if it == 1 else rho / rho_old
            for s, p, r in zip(S, ps, rs):
                s.axpby(1.0, r, beta, p)
            self.apply(ps, ws)
            pap = self.dots([(ws, ps)])[0]
            if not (pap > 0.0) or not math.isfinite(pap):
                breakdown = True
                break
            alpha = rho / pap
            for s, x, p, r, w in zip(S, xs, ps, rs, ws):
                s.axpby(alpha, p, 1.0, x)
                s.axpby(-alpha, w, 1.0, r)
            rho_old = rho
            rho = self.dots([(rs, rs)])[0]
            iters = it
            hist.append(rho)
        relres = math.sqrt(rho) / fnorm if fnorm > 0.0 else 0.0
        return iters, relres, hist, breakdown


class GpuSlab:
    """One slab on the current CUDA device: every step is a library kernel
    on the context's stream (``nb_setup_slab``, ``nb_ax``, ``nb_dssum``,
    ``nb_mask``, ``nb_slab_*``, ``nb_axpby``)."""

    def __init__(self, nekgb, dims, z0: int, z1: int, n: int, amp: float, s, stream):
        import torch
        self.nek, self.torch = nekgb, torch
        self.ctx = nekgb.nb_setup_slab(dims, z0, z1, n, amp, s, stream)
        self.E = dims[0] * dims[1] * (z1 - z0)
        self.n = n
        self.plane, self.has_below, self.has_above = nekgb.nb_slab_info(self.ctx)

    def close(self):
        if self.ctx is not None:
            self.nek.nb_destroy(self.ctx)
            self.ctx = None

    def new_field(self):
        return self.torch.zeros(self.E, self.n ** 3, dtype=self.torch.float64, device="cuda")

    def new_plane(self):
        return self.torch.zeros(self.plane, dtype=self.torch.float64, device="cuda")

    def ax(self, u, w):
        self.nek.nb_ax(self.ctx, u, w)

    def dssum(self, w):
        self.nek.nb_dssum(self.ctx, w)

    def mask(self, w):
        self.nek.nb_mask(self.ctx, w)

    def top_partial(self, w, buf):
        self.nek.nb_slab_top_partial(self.ctx, w, buf)

    def add_bottom(self, w, buf):
        self.nek.nb_slab_add_bottom(self.ctx, w, buf)

    def bottom_value(self, w, buf):
        self.nek.nb_slab_bottom_value(self.ctx, w, buf)

    def set_top(self, w, buf):
        self.nek.nb_slab_set_top(self.ctx, w, buf)

    def dot(self, a, b) -> float:
        return self.nek.nb_slab_dot(self.ctx, a, b)

    def axpby(self, alpha, x, beta, y):
        self.nek.nb_axpby(self.ctx, alpha, x, beta, y)

    def copy(self, dst, src):
        self.nek.nb_axpby(self.ctx, 1.0, src, 0.0, dst)
