// ax_e in double-float arithmetic on the FP32 pipes: the element-local
// Poisson operator of Listing 1 (arXiv 2005.13425, Sec. III) to FP64
// accuracy on GB300, whose FP64 pipe delivers only ~1 TFLOP/s.
//
// Arithmetic.  u, gxyz and D are split into pairs of floats (48-bit
// significands).  Every contraction -- the forward derivatives wr, ws, wt,
// the 3x3 geometric contraction and the transposed derivatives -- is a
// compensated dot product (TwoProd + TwoSum, Dot2), and the three
// transposed-derivative partial sums are added as pairs.  Inputs are scaled
// by exact powers of two (per element for u, once per context for gxyz) so
// the pairs keep their full relative precision whatever the data's
// magnitude; the output is scaled back exactly.
//
// Thread layout ("line threads").  A CTA owns one element at a time and has
// 3 n^2 working threads: thread (d, a0, a1) owns one line of the element
// along direction d (r: (j,k); s: (i,k); t: (i,j)).  In the forward phase a
// thread loads its n inputs once from shared memory and produces the n
// derivative values of its line; the entries of D are compile-time indexed
// kernel parameters, so they are constant-bank operands and cost no loads.
// A pointwise phase contracts (wr, ws, wt) with the six geometric factors
// (streamed from HBM, coalesced) into (ur, us, ut) in place.  The backward
// phase is the same line pattern with D^T, each direction writing its own
// partial array, and a final pointwise phase adds the three partials and
// writes w.  Six barriers per element (four in the CG head, see
// cg_head_pipelined); shared memory holds six n^3 arrays
// of pairs (48 KB at n = 10).
#include <math.h>

#include "ax_df_core.cuh"

namespace nekgb {

struct AxDfArgs {
    const double *u;      // MODE 0 input
    double *w;            // output (FP64, local storage)
    const double *r;      // MODE 1: residual
    double *p;            // MODE 1: search direction, updated in place
    double *x;            // MODE 1: iterate, receives the owed x += x_alpha p
    const double *minv;   // MODE 1: Jacobi inverse diagonal or null
    CgScalars *sc;        // MODE 1
    double *partials;     // MODE 1 fused: one <w,p> partial per CTA
    int finalize;         // MODE 1 fused: the last CTA reduces <w,p>_c and forms alpha
    int dot_shift0;       // MODE 1 two-kernel CG: scale of the exact <w,p>_c sum (see launch_df_nv)
    int dot_lim;          // MODE 1 two-kernel CG: a share of 2^dot_lim or more (scaled) may overflow the sum
    int fuse;             // MODE 1: zero box-face points, local products w p
    Mesh m;
    const float2 *g;      // gxyz pairs [E][6][n^3], scaled by 2^-(gexp-1023)
    int gexp;             // biased exponent of max|gxyz|
    int64_t E;
};

// ---- exact 128-bit fixed-point sums (the CG head's <w,p>_c)
using u128 = unsigned __int128;

// v 2^S truncated toward zero to an integer, as a two's-complement 128-bit
// value.  The caller's S keeps |v| 2^S below 2^lim (lim = 125 - log2 of the
// number of shares, see the head), so no sum of shares overflows; a share
// that may reach 2^lim sets `out_of_range` (the solve then stops with a
// status instead of using a wrong sum).  The shift is clamped at 73; values
// whose scaled magnitude is below 1 give 0.
__device__ __forceinline__ u128 fixed_of(double v, int S, int lim, bool &out_of_range) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) return 0;
    out_of_range |= ex - 1022 + S > lim;                 // |v| 2^S < 2^(ex - 1022 + S)
    const unsigned long long M = (b & 0xfffffffffffffull) | (1ull << 52);
    int sh = ex - 1075 + S;
    u128 mag;
    if (sh >= 0) {
        sh = sh > 73 ? 73 : sh;
        mag = (u128)M << sh;
    } else {
        mag = sh > -64 ? (u128)(M >> (-sh)) : (u128)0;
    }
    return (b >> 63) ? (u128)0 - mag : mag;
}

__device__ __forceinline__ u128 shfl_down_u128(u128 v, int o) {
    const unsigned long long lo = __shfl_down_sync(0xffffffffu, (unsigned long long)v, o);
    const unsigned long long hi = __shfl_down_sync(0xffffffffu, (unsigned long long)(v >> 64), o);
    return ((u128)hi << 64) | lo;
}

// Sum over the CTA (modulo 2^128, i.e. exact for the signed values the head
// produces); the total is valid in thread 0.  red: 2 * (warps) doubles.
__device__ __forceinline__ u128 block_sum_u128(u128 v, double *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_down_u128(v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        red[2 * wid] = __longlong_as_double((long long)(unsigned long long)(v >> 64));
        red[2 * wid + 1] = __longlong_as_double((long long)(unsigned long long)v);
    }
    __syncthreads();
    u128 t = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); k++)
            t += ((u128)(unsigned long long)__double_as_longlong(red[2 * k]) << 64) |
                 (unsigned long long)__double_as_longlong(red[2 * k + 1]);
    return t;
}

// x 2^k for any k (two exact power-of-two factors).
__device__ __forceinline__ double scale2(double x, int k) {
    const int k1 = k / 2, k2 = k - k1;
    return x * __longlong_as_double((long long)(k1 + 1023) << 52) * __longlong_as_double((long long)(k2 + 1023) << 52);
}

// The unpreconditioned two-kernel CG head with a software-pipelined,
// dynamically scheduled element loop.
//
// Scale.  The pairs of p are scaled by one power of two per iteration, 2^sh
// with sqrt(<p,p>_c) 2^sh in [1, 2) (<p,p>_c from the scalar block; every
// |p| is at most sqrt(8 <p,p>_c), as c >= 1/8), instead of a per-element
// maximum: that removes the exponent reduction and its barrier, and lets p
// be split straight from registers into shared memory.  Tiny entries lose
// low-order bits only below 2^-78 of that scale, far under the operator's
// rounding relative to max|w|.
//
// Pipeline.  The six shared arrays rotate roles between consecutive
// elements (X the input, F the three derivative arrays, P the partials):
//   even step: X = S0, F = (S1, S2, S3), P = (S0, S4, S5)
//   odd step:  X = S1, F = (S0, S2, S3), P = (S1, S4, S5)
// so the next element is staged into its X while the final pass reads the
// current P, which needs no barrier in between: four barriers per element.
//
// Schedule.  After its first element (blockIdx.x) a CTA takes the next one
// from a counter in the scalar block, so SMs that run slower take fewer
// elements (a static assignment left the slowest SM 12 % behind the mean).
// The counter is read at the start of a step and published just before the
// barrier that ends the backward pass, which hides the atomic's latency.
// <w,p>_c stays independent of the schedule because it is summed exactly:
// each thread's share of an element (its points' products, in a fixed
// order, in FP64) is converted to a 128-bit integer at the fixed scale 2^S
// (fixed_of, truncating) and added to the thread's integer sum; integer
// sums do not depend on the order of the additions.  The caller chooses S
// from <p,p>_c and a bound on the operator so that no sum can overflow
// (see launch_df_nv); the result is rounded to FP64 once, at the end.
template <int N, bool EO>
__device__ __forceinline__ u128 cg_head_pipelined(const AxDfArgs &a, double beta, double xa, int S,
                                                  const typename DfConsts<N, EO>::type &D, float2 *sm,
                                                  bool &out_of_range) {
    constexpr int N2 = N * N, N3 = N * N * N;
    constexpr int T = ax_df_threads(N);
    __shared__ long long s_next;
    const int t = threadIdx.x;
    const double pn = a.sc->it == 0 ? a.sc->rr : a.sc->pn2;
    const int ep = (int)((__double_as_longlong(pn) >> 52) & 0x7ff);
    const int sh_in = ep == 0 ? 0 : -((ep - 1023) >> 1);
    const int sh_out = -sh_in + (a.gexp - 1023);
    float2 *S0 = sm, *S1 = sm + N3, *S2 = sm + 2 * N3, *S3 = sm + 3 * N3, *S4 = sm + 4 * N3, *S5 = sm + 5 * N3;
    // x += xa p (the owed update), p = r + beta p, X = pairs of p 2^sh
    auto stage = [&](int64_t e, float2 *X) {
        const int64_t eb = e * N3;
        double *p = a.p + eb;
        const double *r = a.r + eb;
        if (xa != 0.0) {
            double *x = a.x + eb;
            for (int q = t; q < N3; q += T) {
                const double pold = p[q];
                __stcs(x + q, fma(xa, pold, __ldcs(x + q)));
                const double v = fma(beta, pold, r[q]);
                p[q] = v;
                X[q] = dfa::split_scaled<true>(v, sh_in);
            }
        } else {
            for (int q = t; q < N3; q += T) {
                const double v = fma(beta, p[q], r[q]);
                p[q] = v;
                X[q] = dfa::split_scaled<true>(v, sh_in);
            }
        }
    };
    // the box-face bits of this thread's points in the final pass, computed once
    constexpr int PPT = df_points_per_thread<N, T>();
    FaceBits<N, T, PPT> pf;
    pf.init();
    u128 acc = 0;
    int64_t e = blockIdx.x;
    if (e < a.E) stage(e, S0);
    __syncthreads();
    for (int k = 0; e < a.E; k++) {
        const bool odd = k & 1;
        unsigned nxt = 0;
        if (t == 0) nxt = atomicAdd(&a.sc->next_elem, 1u);
        float2 *X = odd ? S1 : S0;
        float2 *F0 = odd ? S0 : S1;
        // forward: wr, ws, wt along this thread's line
        for (int task = t; task < 3 * N2; task += T) {
            int stride;
            const int base = line_of<N>(task, stride);
            float2 *Fd = task < N2 ? F0 : (task < 2 * N2 ? S2 : S3);
            if constexpr (EO)
                line_eo<N>(X, Fd, base, stride, D.fwd);
            else
                line_plain<N, false>(X, Fd, base, stride, D);
        }
        __syncthreads();
        // geometric contraction, pointwise, in place
        const float2 *g = a.g + e * 6 * N3;
        for (int q = t; q < N3; q += T) {
            const float2 wr = F0[q], ws = S2[q], wt = S3[q];
            const float2 g0 = __ldcs(g + q), g1 = __ldcs(g + N3 + q), g2 = __ldcs(g + 2 * N3 + q);
            const float2 g3 = __ldcs(g + 3 * N3 + q), g4 = __ldcs(g + 4 * N3 + q), g5 = __ldcs(g + 5 * N3 + q);
            dfa::Acc ur = dfa::first(g0.x, g0.y, wr.x, wr.y);
            dfa::fma(ur, g1.x, g1.y, ws.x, ws.y);
            dfa::fma(ur, g2.x, g2.y, wt.x, wt.y);
            dfa::Acc us = dfa::first(g1.x, g1.y, wr.x, wr.y);
            dfa::fma(us, g3.x, g3.y, ws.x, ws.y);
            dfa::fma(us, g4.x, g4.y, wt.x, wt.y);
            dfa::Acc ut = dfa::first(g2.x, g2.y, wr.x, wr.y);
            dfa::fma(ut, g4.x, g4.y, ws.x, ws.y);
            dfa::fma(ut, g5.x, g5.y, wt.x, wt.y);
            F0[q] = dfa::raw(ur);
            S2[q] = dfa::raw(us);
            S3[q] = dfa::raw(ut);
        }
        __syncthreads();
        // backward: the three partials of w, into X (consumed), S4, S5
        for (int task = t; task < 3 * N2; task += T) {
            int stride;
            const int base = line_of<N>(task, stride);
            const float2 *Fd = task < N2 ? F0 : (task < 2 * N2 ? S2 : S3);
            float2 *Pd = task < N2 ? X : (task < 2 * N2 ? S4 : S5);
            if constexpr (EO)
                line_eo<N>(Fd, Pd, base, stride, D.bwd);
            else
                line_plain<N, true>(Fd, Pd, base, stride, D);
        }
        if (t == 0) s_next = (long long)gridDim.x + (long long)nxt;
        __syncthreads();
        // w = sum of the partials, box faces zeroed, this thread's share of
        // <w,p>_c into its exact sum; then the next element is staged into
        // the other input array
        {
            int ex, ey, ez;
            element_coords(e, a.m, ex, ey, ez);
            const unsigned bf = box_faces(ex, ey, ez, a.m);
            const int64_t eb = e * N3;
            const double *p = a.p + eb;
            double *w = a.w + eb;
            double de = 0.0;
#pragma unroll
            for (int kk = 0; kk < PPT; kk++) {
                const int q = t + kk * T;
                if (PPT * T != N3 && q >= N3) break;
                const float2 s = dfa::add(dfa::add(X[q], S4[q]), S5[q]);
                double wv = dfa::join_scaled(s, sh_out);
                if (pf[kk] & bf)
                    wv = 0.0;
                else
                    de = fma(wv, p[q], de);
                w[q] = wv;
            }
            acc += fixed_of(de, S, a.dot_lim, out_of_range);
        }
        const int64_t en = s_next;
        if (en < a.E) stage(en, odd ? S0 : S1);
        __syncthreads();
        e = en;
    }
    return acc;
}

// As many CTAs per SM as the shared memory holds (df_min_blocks); the
// register bound keeps them resident.
template <int N, int MODE, bool EO>
__global__ void __launch_bounds__(ax_df_threads(N), df_min_blocks<N, ax_df_threads(N)>())
ax_df_kernel(AxDfArgs a, const __grid_constant__ typename DfConsts<N, EO>::type D) {
    constexpr int N3 = N * N * N;
    extern __shared__ float2 sm[];
    __shared__ int s_emax;
    __shared__ double red[32];
    double beta = 0.0, xa = 0.0, dot = 0.0;
    if (MODE == 1) {
        if (a.sc->done) return;
        beta = a.sc->it == 0 ? 0.0 : a.sc->beta;
        xa = a.sc->x_alpha;
    }
    if (MODE == 1 && a.fuse && a.finalize && !a.minv) {
        // the exact sums: per CTA, then over the CTAs by the last one
        const double pn = a.sc->it == 0 ? a.sc->rr : a.sc->pn2;
        const int S = a.dot_shift0 - ((int)((__double_as_longlong(pn) >> 52) & 0x7ff) - 1023);
        bool out_of_range = false;
        const u128 mine = block_sum_u128(cg_head_pipelined<N, EO>(a, beta, xa, S, D, sm, out_of_range), red);
        const int range_fault = __syncthreads_or(out_of_range);
        __shared__ int s_last;
        if (threadIdx.x == 0) {
            if (range_fault) {           // seen by the last CTA's finalize_alpha, which ends the solve
                a.sc->fault = kFaultExactSumRange;
                a.sc->status = (int)NB_ERR_BREAKDOWN;
            }
            a.partials[2 * blockIdx.x] = __longlong_as_double((long long)(unsigned long long)(mine >> 64));
            a.partials[2 * blockIdx.x + 1] = __longlong_as_double((long long)(unsigned long long)mine);
            __threadfence();
            s_last = atomicAdd(&a.sc->ticket, 1u) == gridDim.x - 1;
        }
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        u128 v = 0;
        for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x)
            v += ((u128)(unsigned long long)__double_as_longlong(__ldcg(a.partials + 2 * q)) << 64) |
                 (unsigned long long)__double_as_longlong(__ldcg(a.partials + 2 * q + 1));
        v = block_sum_u128(v, red);
        if (threadIdx.x == 0) {
            // the signed 128-bit total, rounded to FP64 once, scaled back by 2^-S
            const long long hi = (long long)(unsigned long long)(v >> 64);
            const unsigned long long lo = (unsigned long long)v;
            const double pap = scale2(fma((double)hi, 18446744073709551616.0, (double)lo), -S);
            a.sc->ticket = 0;
            a.sc->next_elem = 0;
            finalize_alpha(a.sc, pap);
        }
        return;
    } else {
    if (threadIdx.x == 0) s_emax = 0;
    __syncthreads();
    for (int64_t e = blockIdx.x; e < a.E; e += gridDim.x) {
        const int64_t eb = e * N3;
        DfElemIO io;
        io.u = MODE == 0 ? a.u + eb : nullptr;
        io.r = MODE == 1 ? a.r + eb : nullptr;
        io.p = MODE == 1 ? a.p + eb : nullptr;
        io.x = MODE == 1 ? a.x + eb : nullptr;
        io.minv = (MODE == 1 && a.minv) ? a.minv + eb : nullptr;
        io.w = a.w + eb;
        io.g = a.g + e * 6 * N3;
        int ex = 0, ey = 0, ez = 0;
        if (MODE == 1) element_coords(e, a.m, ex, ey, ez);
        df_element<N, MODE, EO>(io, beta, xa, a.fuse != 0, a.gexp, a.m, ex, ey, ez, D, sm, &s_emax, dot);
    }
    }
    if (MODE == 1 && a.fuse) {
        if (a.finalize) {
            double v[1] = {dot}, tot[1];
            if (last_block_reduce<1>(v, a.partials, 0, blockIdx.x, gridDim.x, gridDim.x, &a.sc->ticket, tot) &&
                threadIdx.x == 0)
                finalize_alpha(a.sc, tot[0]);
        } else {
            const double b = block_sum(dot, red);
            if (threadIdx.x == 0) a.partials[blockIdx.x] = b;
        }
    }
}

// ---------------------------------------------------------------- set-up
// Largest binary exponent (biased) of |x| over an array.
__global__ void max_exponent_kernel(const double *__restrict__ x, int64_t n, int *out) {
    int emax = 0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int ex = (int)((__double_as_longlong(x[q]) >> 52) & 0x7ff);
        emax = ex > emax ? ex : emax;
    }
    emax = __reduce_max_sync(0xffffffffu, emax);
    if ((threadIdx.x & 31) == 0) atomicMax(out, emax);
}

__global__ void split_scaled_kernel(const double *__restrict__ x, float2 *__restrict__ y, int64_t n,
                                    const int *eptr) {
    int ex = *eptr;
    ex = ex < 1 ? 1 : (ex > 2046 ? 2046 : ex);
    const double sc = __longlong_as_double((long long)(2046 - ex) << 52);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        y[q] = dfa::split(x[q] * sc);
}

nb_status prepare_df(nb_ctx *c) {
    const int64_t ng = (int64_t)6 * c->m.n * c->m.n * c->m.n * c->m.E;
    cudaError_t e = dev_alloc((void **)&c->d_gxyz_df, sizeof(float2) * ng);
    if (e != cudaSuccess) return cuda_fail(e, "alloc gxyz pairs");
    c->device_bytes += sizeof(float2) * ng;
    int *d_ex = nullptr;
    if ((e = dev_alloc((void **)&d_ex, sizeof(int))) != cudaSuccess) return cuda_fail(e, "alloc exponent");
    int gexp = 0;
    e = cudaMemsetAsync(d_ex, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) {
        max_exponent_kernel<<<1024, 256, 0, c->stream>>>(c->d_gxyz, ng, d_ex);
        split_scaled_kernel<<<1024, 256, 0, c->stream>>>(c->d_gxyz, c->d_gxyz_df, ng, d_ex);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&gexp, d_ex, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_ex);
    if (e != cudaSuccess) return cuda_fail(e, "split gxyz");
    gexp = gexp < 1 ? 1 : (gexp > 2046 ? 2046 : gexp);
    c->gxyz_exp = gexp;
    c->d_eo = centro_antisymmetric(c->D_host, c->m.n);
    return NB_OK;
}

bool df_supported(int n) { return n >= 2 && n <= kMaxN; }

// True when D(i,l) = -D(n-1-i, n-1-l) to rounding (GLL derivative matrices).
bool centro_antisymmetric(const double *D, int n) {
    double mx = 0.0, asym = 0.0;
    for (int q = 0; q < n * n; q++) mx = fmax(mx, fabs(D[q]));
    for (int i = 0; i < n; i++)
        for (int l = 0; l < n; l++)
            asym = fmax(asym, fabs(D[i * n + l] + D[(n - 1 - i) * n + (n - 1 - l)]));
    return asym <= 1e-14 * mx;
}

// The fixed-point scale of the CG head's exact <w,p>_c: S = dot_shift0 -
// e(<p,p>_c), e the binary exponent.  Every |w_q| is at most
// A max|p| with A = 9 |D|_1 |D|_inf max|G| (three derivatives, the 3x3
// contraction, three transposed derivatives), and max|p| <= sqrt(8 <p,p>_c),
// so a thread's share of an element (P points) is below 8 P A <p,p>_c.
// sa below takes 72 P A (a further factor 9 of margin) and another 16x for
// the recursion's <p,p>_c, so the share stays below 2^(sa + e).  Summing E T shares (E elements, T threads) then
// stays below 2^(sa + e + S + log2(E T)) <= 2^125: no 128-bit sum overflows.
// The grid of the sum, 2^-S, is 2^-(125 - log2(E T)) of that bound.
template <int N>
static int dot_lim(const nb_ctx *c);

template <int N>
static int dot_shift0(const nb_ctx *c) {
    constexpr int T = ax_df_threads(N);
    constexpr int P = (N * N * N + T - 1) / T;
    double d1 = 0.0, dinf = 0.0;
    for (int i = 0; i < N; i++) {
        double rs = 0.0, cs = 0.0;
        for (int l = 0; l < N; l++) {
            rs += fabs(c->D_host[i * N + l]);
            cs += fabs(c->D_host[l * N + i]);
        }
        dinf = fmax(dinf, rs);
        d1 = fmax(d1, cs);
    }
    // max|G| < 2^(gexp - 1022)
    const int sa = (int)ceil(log2(72.0 * P * 9.0 * d1 * dinf)) + (c->gxyz_exp - 1022) + 1 + 4;
    return dot_lim<N>(c) - sa;
}

// The bound of one scaled share: 2^(125 - log2(E T)), so that E T shares
// sum below 2^125.
template <int N>
static int dot_lim(const nb_ctx *c) {
    constexpr int T = ax_df_threads(N);
    return 125 - (int)ceil(log2((double)c->m.E * T));
}

template <int N, bool EO>
static nb_status launch_df_nv(nb_ctx *c, const double *u, double *w, int mode) {
    constexpr int T = ax_df_threads(N);
    const size_t smem = sizeof(float2) * 6 * N * N * N;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    typename DfConsts<N, EO>::type D;
    df_consts<N, EO>(c->D_host, D);
    AxDfArgs args{};
    args.g = c->d_gxyz_df;
    args.gexp = c->gxyz_exp;
    args.E = c->m.E;
    if (mode == 0) {
        args.u = u;
        args.w = w;
    } else {
        args.r = c->d_r;
        args.p = c->d_p;
        args.x = c->d_x;
        args.minv = c->d_minv;
        args.w = c->d_w;
        args.sc = c->d_sc;
        args.partials = c->d_partials;
        args.fuse = c->fused_cg ? 1 : 0;
        args.finalize = c->two_kernel ? 1 : 0;
        args.dot_shift0 = dot_shift0<N>(c) + c->test_dot_shift;
        args.dot_lim = dot_lim<N>(c);
    }
    args.m = c->m;
    auto kern = mode == 0 ? ax_df_kernel<N, 0, EO> : ax_df_kernel<N, 1, EO>;
    {
        const nb_status s = set_smem(kern, smem);
        if (s != NB_OK) return s;
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, T, smem);
    if (occ < 1) occ = 1;
    const int64_t cap = (int64_t)sms * occ;
    const int grid = (int)(c->m.E < cap ? c->m.E : cap);
    if (mode == 1) c->ax_grid = grid;
    LaunchTimer tm(c, NB_K_AX);
    kern<<<grid, T, smem, c->stream>>>(args, D);
    NB_LAUNCH_CHECK("ax_df_kernel");
    return NB_OK;
}

template <int N>
static nb_status launch_df_n(nb_ctx *c, const double *u, double *w, int mode) {
    return c->d_eo ? launch_df_nv<N, true>(c, u, w, mode) : launch_df_nv<N, false>(c, u, w, mode);
}

nb_status launch_ax_df(nb_ctx *c, const double *u, double *w, int mode) {
    switch (c->m.n) {
#define NB_CASE(NN) case NN: return launch_df_n<NN>(c, u, w, mode);
        NB_CASE(2) NB_CASE(3) NB_CASE(4) NB_CASE(5) NB_CASE(6) NB_CASE(7) NB_CASE(8)
        NB_CASE(9) NB_CASE(10) NB_CASE(11) NB_CASE(12) NB_CASE(13) NB_CASE(14) NB_CASE(15)
        NB_CASE(16)
#undef NB_CASE
    }
    return fail(NB_ERR_ARG, "unsupported n");
}

}  // namespace nekgb
