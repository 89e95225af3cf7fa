// FP32 ax_e element operator (Listing 1, arXiv 2005.13425 Sec. III, with
// FP32 u, w and gxyz) shared by the single-problem kernel (ax_f32.cu) and
// the batched engine (engine.cu).
//
// Line-thread layout: 3n^2 line tasks own one 1-D line each; D entries are
// compile-time-indexed kernel parameters (constant-bank operands); a
// pointwise pass contracts with the six geometric factors; the transposed
// derivatives go to three partial arrays that a final pass adds.  The
// element's geometric factors stream into shared memory with cp.async while
// the forward derivatives are computed.
#pragma once

#include "bulk.cuh"
#include "df.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace nekgb {

template <int N>
struct F32Mat {
    float d[N * N];   // d[m*N + l] = D(m, l)
};

__host__ __device__ constexpr int ax_f32_threads(int n) {
    return n <= 12 ? ((3 * n * n + 31) / 32) * 32 : ((3 * n * n + 1) / 2 + 31) / 32 * 32;
}

// Floats of dynamic shared memory f32_element needs: six n^3 work arrays and
// the six n^3 geometric factors (16-byte aligned).
__host__ __device__ constexpr int f32_smem_floats(int n) {
    return ((6 * n * n * n + 3) / 4) * 4 + 6 * n * n * n;
}

template <int N>
__device__ __forceinline__ int f32_line_of(int task, int &stride) {
    constexpr int N2 = N * N;
    const int d = task / N2;
    const int c = task - d * N2;
    const int a0 = c % N, a1 = c / N;
    if (d == 0) { stride = 1; return N * (a0 + N * a1); }
    if (d == 1) { stride = N; return a0 + N2 * a1; }
    stride = N2;
    return a0 + N * a1;
}

// Asynchronous global->shared copies (no register staging): 16-byte chunks
// when the element's slab is 16-byte aligned (n^3 a multiple of 4), 4-byte
// otherwise.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// One line product along a direction of compile-time stride S (1, N or
// N^2): out[m S] = sum_l M(m,l) in[l S], M = D or (TR) D^T, accumulated as
// M(m,0) x_0 followed by FMAs in l order.  A constant stride lets every
// shared-memory access use an immediate offset (no address arithmetic per
// access); along r (S = 1, even N) the line is read and written as float2,
// which also removes the 2-way bank conflicts of 32 consecutive lines that
// are N floats apart.
template <int N, int S, bool TR>
__device__ __forceinline__ void f32_line(const float *in, float *out, const F32Mat<N> &D) {
    constexpr bool PAIRS = S == 1 && N % 2 == 0;
    float x[N];
    if constexpr (PAIRS) {
        const float2 *in2 = reinterpret_cast<const float2 *>(in);
#pragma unroll
        for (int l = 0; l < N / 2; l++) {
            const float2 v = in2[l];
            x[2 * l] = v.x;
            x[2 * l + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int l = 0; l < N; l++) x[l] = in[l * S];
    }
    auto dot_row = [&](int mm) {
        float acc = (TR ? D.d[mm] : D.d[mm * N]) * x[0];
#pragma unroll
        for (int l = 1; l < N; l++) acc = fmaf(TR ? D.d[l * N + mm] : D.d[mm * N + l], x[l], acc);
        return acc;
    };
    if constexpr (PAIRS) {
        float2 *o2 = reinterpret_cast<float2 *>(out);
#pragma unroll
        for (int mm = 0; mm < N / 2; mm++) o2[mm] = make_float2(dot_row(2 * mm), dot_row(2 * mm + 1));
    } else {
#pragma unroll
        for (int mm = 0; mm < N; mm++) out[mm * S] = dot_row(mm);
    }
}

// The same line product with a runtime stride, for warps whose lines run
// in two directions.
template <int N, bool TR>
__device__ __forceinline__ void f32_line_rt(const float *in, float *out, int stride, const F32Mat<N> &D) {
    float x[N];
#pragma unroll
    for (int l = 0; l < N; l++) x[l] = in[l * stride];
#pragma unroll
    for (int mm = 0; mm < N; mm++) {
        float acc = (TR ? D.d[mm] : D.d[mm * N]) * x[0];
#pragma unroll
        for (int l = 1; l < N; l++) acc = fmaf(TR ? D.d[l * N + mm] : D.d[mm * N + l], x[l], acc);
        out[mm * stride] = acc;
    }
}

// The 3 N^2 line products of one pass, thread t taking tasks t, t + T, ...:
// lines along r read i0 and write o0, along s i1 / o1, along t i2 / o2.  A
// warp whose 32 tasks lie in one direction takes that direction's
// constant-stride body; a warp that straddles two directions takes the
// runtime-stride body for all its lanes (no warp runs two bodies serially).
template <int N, int T, bool TR>
__device__ __forceinline__ void f32_line_pass(const float *i0, const float *i1, const float *i2, float *o0,
                                              float *o1, float *o2, const F32Mat<N> &D) {
    constexpr int N2 = N * N;
    static_assert(T % 32 == 0, "warp-aligned task groups");
    for (int task = threadIdx.x; task < 3 * N2; task += T) {
        const int first = task & ~31;
        const int last = first + 31 < 3 * N2 - 1 ? first + 31 : 3 * N2 - 1;
        if (first / N2 != last / N2) {           // warp-uniform
            int stride;
            const int base = f32_line_of<N>(task, stride);
            const float *in = task < N2 ? i0 : (task < 2 * N2 ? i1 : i2);
            float *out = task < N2 ? o0 : (task < 2 * N2 ? o1 : o2);
            f32_line_rt<N, TR>(in + base, out + base, stride, D);
        } else if (task < N2) {
            f32_line<N, 1, TR>(i0 + N * task, o0 + N * task, D);
        } else if (task < 2 * N2) {
            const int c = task - N2;
            const int base = c % N + N2 * (c / N);
            f32_line<N, N, TR>(i1 + base, o1 + base, D);
        } else {
            const int c = task - 2 * N2;
            f32_line<N, N2, TR>(i2 + c, o2 + c, D);
        }
    }
}

// Box-face masks (point_faces) of the points q = threadIdx.x + k T a thread
// owns in the pointwise passes, computed once per kernel.
template <int N, int T>
__host__ __device__ constexpr int f32_points_per_thread() {
    return (N * N * N + T - 1) / T;
}
template <int N, int T>
__device__ __forceinline__ void f32_point_masks(unsigned *pf) {
#pragma unroll
    for (int k = 0; k < f32_points_per_thread<N, T>(); k++) {
        const int q = threadIdx.x + k * T;
        pf[k] = q < N * N * N ? point_faces<N>(q) : 0u;
    }
}

// Per-element arguments of f32_element (pointers offset to the element).
struct F32ElemIO {
    const float *u;   // MODE 0: input
    const float *r;   // MODE 1: residual
    float *p;         // MODE 1: search direction (updated in place)
    float *x;         // MODE 1: iterate (owed update applied when xa != 0)
    float *w;         // output
    const float *g;   // gxyz [6][n^3] of the element
};

// One element, executed by the whole CTA of T threads (contains barriers;
// every thread must call it).  MODE 0: w = ax_e(u).  MODE 1: the inner CG
// head, x += xa p, p = r + beta p, w = ax_e(p) with box-face points zeroed
// and the local products w p added to dot (their sum over all elements is
// <w,p>_c after assembly, because p is continuous).  (ex, ey, ez) is the
// element's position in the box m.
template <int N, int MODE, int T>
__device__ __forceinline__ void f32_element(const F32ElemIO &io, float beta, float xa, int ex, int ey, int ez,
                                            const Mesh &m, const F32Mat<N> &D, float *smf, dfa::Acc32 &dot) {
    constexpr int N2 = N * N, N3 = N * N * N;
    float *U = smf, *W0 = smf + N3, *W1 = smf + 2 * N3, *W2 = smf + 3 * N3;
    float *P1 = smf + 4 * N3, *P2 = smf + 5 * N3;
    float *G = smf + ((6 * N3 + 3) / 4) * 4;
    const int t = threadIdx.x;
    if (MODE == 1) {
        if (xa != 0.f) {
            for (int q = t; q < N3; q += T) {
                const float pold = io.p[q];
                io.x[q] = fmaf(xa, pold, io.x[q]);
                const float v = fmaf(beta, pold, io.r[q]);
                io.p[q] = v;
                U[q] = v;
            }
        } else {
            for (int q = t; q < N3; q += T) {
                const float v = fmaf(beta, io.p[q], io.r[q]);
                io.p[q] = v;
                U[q] = v;
            }
        }
    } else {
        for (int q = t; q < N3; q += T) U[q] = __ldg(io.u + q);
    }
    // prefetch the geometric factors (consumed after the forward phase)
    if ((N3 % 4) == 0) {
        for (int q = t; q < 6 * N3 / 4; q += T) cp_async16(G + 4 * q, io.g + 4 * q);
    } else {
        for (int q = t; q < 6 * N3; q += T) cp_async4(G + q, io.g + q);
    }
    cp_async_commit();
    __syncthreads();
    f32_line_pass<N, T, false>(U, U, U, W0, W1, W2, D);
    cp_async_wait_all();
    __syncthreads();
    for (int q = t; q < N3; q += T) {
        const float wr = W0[q], ws = W1[q], wt = W2[q];
        const float g0 = G[q], g1 = G[N3 + q], g2 = G[2 * N3 + q];
        const float g3 = G[3 * N3 + q], g4 = G[4 * N3 + q], g5 = G[5 * N3 + q];
        W0[q] = fmaf(g0, wr, fmaf(g1, ws, g2 * wt));
        W1[q] = fmaf(g1, wr, fmaf(g3, ws, g4 * wt));
        W2[q] = fmaf(g2, wr, fmaf(g4, ws, g5 * wt));
    }
    __syncthreads();
    f32_line_pass<N, T, true>(W0, W1, W2, U, P1, P2, D);
    __syncthreads();
    const unsigned bf = MODE == 1 ? box_faces(ex, ey, ez, m) : 0u;
    for (int q = t; q < N3; q += T) {
        float wv = U[q] + P1[q] + P2[q];
        if (MODE == 1) {
            if (point_faces<N>(q) & bf)
                wv = 0.f;
            else
                dot.add_prod(wv, io.p[q]);
        }
        io.w[q] = wv;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- staged
// The same element operator with every input of an element staged in
// shared memory by bulk copies (bulk.cuh), two stages deep: while a CTA
// computes one element, the copy engine fetches the next one's geometric
// factors and vectors, so the loads of a whole element are always in
// flight.  Used for even n up to 10 (n^3 a multiple of 4, so every
// per-element slab is 16-byte aligned, and two CTAs of 21 n^3 floats fit
// on an SM).  The batched engine stages only at n = 10: there it measured
// +5.5 % at n = 10 and -7 % at n = 8, where the unstaged kernel's smaller
// shared memory fits nine CTAs per SM instead of five; the single-problem
// solve measured faster staged at n = 8 as well (51.5 vs 54.0 ms).
//
// Shared memory (floats): stage s at s*f32_stage_floats holds the element's
// vectors (MODE 1: r, p, z; MODE 0: u); after both stages, W0..W2 [3n^3]
// (forward derivatives, then their geometric contraction) and the three
// backward partials [3n^3].  The geometric factors do not pass through
// shared memory: each thread loads its own points' six factors into
// registers at the start of the element (streaming loads, coalesced), and
// they arrive while the update and forward passes run.  That keeps a CTA at
// 12 n^3 floats (48 KB at n = 10), four CTAs per SM instead of two.
template <int N, int MODE>
__host__ __device__ constexpr int f32_stage_floats() {
    return (MODE == 1 ? 3 : 1) * N * N * N;
}
template <int N, int MODE>
__host__ __device__ constexpr int f32_staged_smem_floats() {
    return 2 * f32_stage_floats<N, MODE>() + 6 * N * N * N;
}
// CTAs per SM the staged kernels ask the register allocator to allow:
// as many as the shared memory holds (228 KB, 1 KB reserved per CTA), at
// most four.
template <int N>
__host__ __device__ constexpr int f32_staged_min_blocks() {
    constexpr int by_smem = (228 * 1024) / (4 * f32_staged_smem_floats<N, 1>() + 1024);
    return by_smem < 3 ? (by_smem < 1 ? 1 : by_smem) : 3;
}

// Geometric factors of a thread's points, gv[k][c] = g[c n^3 + t + k T]
// (streaming loads; zero past the element's last point).
template <int N, int T>
__device__ __forceinline__ void f32_load_factors(const float *__restrict__ g, float (&gv)[f32_points_per_thread<N, T>()][6]) {
    constexpr int N3 = N * N * N;
    constexpr int PPT = f32_points_per_thread<N, T>();
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int q = threadIdx.x + k * T;
        if (PPT * T == N3 || q < N3) {
#pragma unroll
            for (int c = 0; c < 6; c++) gv[k][c] = __ldcs(g + c * N3 + q);
        } else {
#pragma unroll
            for (int c = 0; c < 6; c++) gv[k][c] = 0.f;
        }
    }
}

template <int N>
__host__ __device__ constexpr bool f32_staged_ok() {
    return (N % 2 == 0) && N <= 10;
}

// Global outputs of one staged element (offset to the element).
struct F32StagedOut {
    float *p;   // MODE 1: p = r + beta p written back
    float *x;   // MODE 1: x += xa p_old written back (when xa != 0)
    float *w;   // ax_e output
};

// Element body on stage `st` (whole CTA).  gv holds this element's
// geometric factors on entry (f32_load_factors); right after the
// contraction consumes them it is refilled from gnext, the next element's
// factors (null: none), so those loads are in flight through the rest of
// this element and the next one's update and forward passes.  pf: the
// thread's point-face masks (f32_point_masks).  Ends with fence + barrier,
// after which the stage may be refilled.
template <int N, int MODE, int T>
__device__ __forceinline__ void f32_element_staged(float *st, float *W, float (&gv)[f32_points_per_thread<N, T>()][6],
                                                   const float *__restrict__ gnext, const F32StagedOut &o,
                                                   float beta, float xa, int ex, int ey, int ez, const Mesh &m,
                                                   const F32Mat<N> &D, dfa::Acc32 &dot, const unsigned *pf) {
    constexpr int N3 = N * N * N;
    constexpr int PPT = f32_points_per_thread<N, T>();
    constexpr bool RAGGED = PPT * T != N3;
    float *U = st;                             // MODE 0: u; MODE 1: r then (below) p
    float *W0 = W, *W1 = W + N3, *W2 = W + 2 * N3;
    float *P0 = W + 3 * N3, *P1 = W + 4 * N3, *P2 = W + 5 * N3;
    const int t = threadIdx.x;
    if (MODE == 1) {
        float *R = st, *P = st + N3, *Z = st + 2 * N3;
        if (xa != 0.f) {
            for (int q = t; q < N3; q += T) {
                const float pold = P[q];
                const float pn = fmaf(beta, pold, R[q]);
                P[q] = pn;
                o.p[q] = pn;
                o.x[q] = fmaf(xa, pold, Z[q]);
            }
        } else {
            for (int q = t; q < N3; q += T) {
                const float pn = fmaf(beta, P[q], R[q]);
                P[q] = pn;
                o.p[q] = pn;
            }
        }
        U = P;
        __syncthreads();
    }
    f32_line_pass<N, T, false>(U, U, U, W0, W1, W2, D);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int q = t + k * T;
        if (RAGGED && q >= N3) break;
        const float wr = W0[q], ws = W1[q], wt = W2[q];
        W0[q] = fmaf(gv[k][0], wr, fmaf(gv[k][1], ws, gv[k][2] * wt));
        W1[q] = fmaf(gv[k][1], wr, fmaf(gv[k][3], ws, gv[k][4] * wt));
        W2[q] = fmaf(gv[k][2], wr, fmaf(gv[k][4], ws, gv[k][5] * wt));
    }
    if (gnext) f32_load_factors<N, T>(gnext, gv);
    __syncthreads();
    f32_line_pass<N, T, true>(W0, W1, W2, P0, P1, P2, D);
    __syncthreads();
    const unsigned bf = MODE == 1 ? box_faces(ex, ey, ez, m) : 0u;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int q = t + k * T;
        if (RAGGED && q >= N3) break;
        float wv = P0[q] + P1[q] + P2[q];
        if (MODE == 1) {
            if (pf[k] & bf)
                wv = 0.f;
            else
                dot.add_prod(wv, U[q]);
        }
        o.w[q] = wv;
    }
    fence_proxy_async();
    __syncthreads();
}

}  // namespace nekgb
