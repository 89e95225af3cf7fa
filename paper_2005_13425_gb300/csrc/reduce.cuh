// Deterministic two-level reductions.
//
// Every CTA reduces its values with a fixed shuffle tree and publishes one
// partial per value into a slot of a partials array; the last CTA to arrive
// (ticket counter) sums all slots of the reduction in a fixed order.  The
// order depends only on the launch configuration, so repeated runs of the
// same problem give bit-identical sums.
#pragma once

#include "internal.cuh"

namespace nekgb {

// Fixed-order CTA sum; the result is valid in thread 0.  `red` holds 32
// doubles of shared memory.  Every thread of the CTA must call it.
__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? red[lane] : 0.0;
    if (wid == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// Publishes NV partials of this CTA at partials[q*stride + slot] and takes a
// ticket.  Returns true in every thread of the CTA that arrives last; that
// CTA's thread 0 then holds in tot[q] the fixed-order sum of slots
// [0, count) of each value q.  `ticket` is reset for the next reduction.
// Slots written by earlier kernels on the same stream are included when
// they fall in [0, count).
template <int NV>
__device__ bool last_block_reduce(const double (&v)[NV], double *partials, int stride, int slot,
                                  int count, int nblocks, unsigned int *ticket, double (&tot)[NV]) {
    __shared__ double red[32];
    __shared__ int s_last;
    double b[NV];
#pragma unroll
    for (int q = 0; q < NV; q++) b[q] = block_sum(v[q], red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; q++) partials[q * stride + slot] = b[q];
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        s_last = (t == (unsigned)nblocks - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
#pragma unroll
    for (int q = 0; q < NV; q++) {
        double acc = 0.0;
        for (int k = threadIdx.x; k < count; k += blockDim.x) acc += __ldcg(partials + q * stride + k);
        tot[q] = block_sum(acc, red);
    }
    if (threadIdx.x == 0) *ticket = 0;
    return true;
}

// The CG step after <w,p>_c is known: alpha = rho/<w,p>_c, or a breakdown
// flag when <w,p>_c <= 0 or is not finite (the owed x update is dropped).
__device__ __forceinline__ void finalize_alpha(CgScalars *sc, double pap) {
    sc->pap = pap;
    // an error status set by another CTA of this kernel (a bounded wait that
    // ran out, the exact sum's range check) ends the solve; read past L1,
    // which may hold the scalar block's line from the kernel's start
    if (__ldcg(&sc->status) != 0) {
        sc->done = 1;
        sc->x_alpha = 0.0;
    } else if (!(pap > 0.0) || !isfinite(pap)) {
        sc->status = (int)NB_ERR_BREAKDOWN;
        sc->done = 1;
        sc->x_alpha = 0.0;
    } else {
        sc->alpha = sc->rho / pap;
        sc->x_alpha = sc->alpha;
    }
}

// Copies of local point (i,j,k) of element (ex,ey,ez) -> 1/multiplicity.
__device__ __forceinline__ double inv_mult(int i, int j, int k, int ex, int ey, int ez, const Mesh &m) {
    const int mu = mult_1d(i, ex, m.ex, m.n) * mult_1d(j, ey, m.ey, m.n) * mult_1d(k, ez, m.ez, m.n);
    return mu == 1 ? 1.0 : (mu == 2 ? 0.5 : (mu == 4 ? 0.25 : 0.125));
}

// log2 of the multiplicity of local point (i,j,k) of element (ex,ey,ez).
__device__ __forceinline__ int log2_mult(int i, int j, int k, int ex, int ey, int ez, const Mesh &m) {
    return (mult_1d(i, ex, m.ex, m.n) >> 1) + (mult_1d(j, ey, m.ey, m.n) >> 1) +
           (mult_1d(k, ez, m.ez, m.n) >> 1);
}

// x * 2^-s for s in 0..3 by exponent arithmetic (no FP64 instruction).
// Values whose exponent field is <= 3 return 0: they only occur where the
// caller squares them (|x|^2 < 2^-2040 underflows to 0 in FP64 as well).
__device__ __forceinline__ double scale_down_pow2(double x, int s) {
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    return ex > 3 ? __longlong_as_double(b - ((long long)s << 52)) : 0.0;
}

// True when local point (i,j,k) of element (ex,ey,ez) lies on a face of the box.
__device__ __forceinline__ bool on_box_face(int i, int j, int k, int ex, int ey, int ez, const Mesh &m) {
    const int n = m.n;
    return (i == 0 && ex == 0) || (i == n - 1 && ex == m.ex - 1) || (j == 0 && ey == 0) ||
           (j == n - 1 && ey == m.ey - 1) || (k == 0 && ez == 0) || (k == n - 1 && ez == m.ez - 1);
}

// Faces of the element that local point q lies on, as bits: i = 0, i = n-1,
// j = 0, j = n-1, k = 0, k = n-1.
template <int N>
__device__ __forceinline__ unsigned point_faces(int q) {
    const int i = q % N, j = (q / N) % N, k = q / (N * N);
    return (unsigned)(i == 0) | ((unsigned)(i == N - 1) << 1) | ((unsigned)(j == 0) << 2) |
           ((unsigned)(j == N - 1) << 3) | ((unsigned)(k == 0) << 4) | ((unsigned)(k == N - 1) << 5);
}

// The point_faces bits of the points q = threadIdx.x + k T (k < PPT) that a
// thread owns in a pointwise pass, six bits per point, five points per
// 32-bit word: one register per five points instead of one per point.
// pf[k] with a compile-time k is a shift and a mask.
template <int N, int T, int PPT>
struct FaceBits {
    static constexpr int W = (PPT + 4) / 5;
    unsigned w[W];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int k = 0; k < W; k++) w[k] = 0u;
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            const int q = (int)threadIdx.x + k * T;
            if (q < N * N * N) w[k / 5] |= point_faces<N>(q) << (6 * (k % 5));
        }
    }
    __device__ __forceinline__ unsigned operator[](int k) const { return (w[k / 5] >> (6 * (k % 5))) & 63u; }
};

// Faces of element (ex,ey,ez) shared with a neighbour, in point_faces' bit
// order: log2 of a point's multiplicity is popc(point_faces & shared_faces).
__device__ __forceinline__ unsigned shared_faces(int ex, int ey, int ez, const Mesh &m) {
    return (unsigned)(ex > 0) | ((unsigned)(ex < m.ex - 1) << 1) | ((unsigned)(ey > 0) << 2) |
           ((unsigned)(ey < m.ey - 1) << 3) | ((unsigned)(ez > 0) << 4) | ((unsigned)(ez < m.ez - 1) << 5);
}

// Faces of element (ex,ey,ez) on the box boundary, in point_faces' bit order.
__device__ __forceinline__ unsigned box_faces(int ex, int ey, int ez, const Mesh &m) {
    return (unsigned)(ex == 0) | ((unsigned)(ex == m.ex - 1) << 1) | ((unsigned)(ey == 0) << 2) |
           ((unsigned)(ey == m.ey - 1) << 3) | ((unsigned)(ez == 0) << 4) | ((unsigned)(ez == m.ez - 1) << 5);
}

// Element id -> (ex, ey, ez): two multiply-high divisions by the mesh's
// exact reciprocals (make_box_mesh).
__device__ __forceinline__ void element_coords(int64_t e, const Mesh &m, int &ex, int &ey, int &ez) {
    const unsigned ei = (unsigned)e;
    const unsigned exy = (unsigned)(m.ex * m.ey);
    const unsigned z = m.inv_exy ? (unsigned)__umul64hi((unsigned long long)ei, m.inv_exy) : ei;
    const unsigned r = ei - z * exy;
    const unsigned y = m.inv_ex ? (unsigned)__umul64hi((unsigned long long)r, m.inv_ex) : r;
    ez = (int)z;
    ey = (int)y;
    ex = (int)(r - y * (unsigned)m.ex);
}

}  // namespace nekgb
