// Core of the double-float ax_e (Listing 1, arXiv 2005.13425 Sec. III) shared
// by the single-problem kernel (ax_df.cu) and the batched engine
// (engine.cu): derivative-matrix constants, the line products (plain and
// even-odd) and the per-element operator df_element().  See ax_df.cu for
// the arithmetic and thread layout.
#pragma once

#include "df.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace nekgb {

template <int N>
struct DfMat {
    float h[N * N];   // h[m*N + l] + l_[m*N + l] = D(m, l)
    float l[N * N];
};

// Even-odd form of a centro-antisymmetric matrix M (M(N-1-m, N-1-l) =
// -M(m,l), which holds for the GLL derivative matrix and its transpose).
// With H = N/2, xs_l = x_l + x_{N-1-l}, xd_l = x_l - x_{N-1-l} (l < H):
//   y_m       = P_m + Q_m,   y_{N-1-m} = P_m - Q_m   (m < H)
//   P_m = sum_{l<H} a(m,l) xd_l,            a(m,l) = (M(m,l) + M(N-1-m,l))/2
//   Q_m = sum_{l<H} b(m,l) xs_l + b(m,H) x_H, b(m,l) = (M(m,l) - M(N-1-m,l))/2
// and for odd N the middle output y_H = sum_{l<H} M(H,l) xd_l + M(H,H) x_H.
// This halves the products of a line (Solomonoff's even-odd decomposition).
// The outputs are stored as unnormalised pairs (dfa::add_acc_raw).
template <int N>
struct EoMat {
    static constexpr int H = N / 2;
    float ah[H * H], al[H * H];
    float bh[H * (H + 1)], bl[H * (H + 1)];
    float ch[H + 1], cl[H + 1];
};

template <int N>
struct DfEo {
    EoMat<N> fwd;   // M = D
    EoMat<N> bwd;   // M = D^T
};


// One line task per thread up to n = 12; two per thread above, so that the
// n-long line held in registers does not spill at n = 16.
__host__ __device__ constexpr int ax_df_threads(int n) {
    return n <= 12 ? ((3 * n * n + 31) / 32) * 32 : ((3 * n * n + 1) / 2 + 31) / 32 * 32;
}

// Threads of a CTA that gives each thread `lpt` line tasks (lpt >= 1).
__host__ __device__ constexpr int df_threads_lpt(int n, int lpt) {
    return ((3 * n * n + lpt - 1) / lpt + 31) / 32 * 32;
}

// CTAs of T threads per SM that the register bound of a kernel around the
// element operator asks for: as many as the six n^3 pair arrays allow in
// 228 KB of shared memory (1 KB reserved per CTA), but no more than leave R
// registers per thread (a line at n <= 10 needs 48; the batched kernel's
// tile head then spills about 100 bytes at n = 10, which costs less than
// the CTA a 64-register bound loses); 4 at n = 10, 2 at n = 11, 12 for R = 48.
// Above n = 12 a line's registers cannot be bounded without spilling.
template <int N, int T, int R = 48>
__host__ __device__ constexpr int df_min_blocks() {
    constexpr int by_smem = (228 * 1024) / (6 * N * N * N * 8 + 1024);
    constexpr int by_regs = 65536 / (T * R);
    return N > 12 ? 1 : (N > 10 ? by_smem : (by_smem < by_regs ? by_smem : by_regs));
}

// Line task -> (first point, stride) of the line and the direction.
template <int N>
__device__ __forceinline__ int line_of(int task, int &stride) {
    constexpr int N2 = N * N;
    const int d = task / N2;
    const int c = task - d * N2;
    const int a0 = c % N, a1 = c / N;
    if (d == 0) {        // along r: line (j = a0, k = a1)
        stride = 1;
        return N * (a0 + N * a1);
    }
    if (d == 1) {        // along s: line (i = a0, k = a1)
        stride = N;
        return a0 + N2 * a1;
    }
    stride = N2;         // along t: line (i = a0, j = a1)
    return a0 + N * a1;
}

// out(base + m*stride) = sum_l M(m,l) in(base + l*stride), M = D or D^T,
// n compensated dot products of n terms.
template <int N, bool TR>
__device__ __forceinline__ void line_plain(const float2 *in, float2 *out, int base, int stride,
                                           const DfMat<N> &D) {
    float xh[N], xl[N];
#pragma unroll
    for (int l = 0; l < N; l++) {
        const float2 v = in[base + l * stride];
        xh[l] = v.x;
        xl[l] = v.y;
    }
#pragma unroll
    for (int m = 0; m < N; m++) {
        const int i0 = TR ? m : m * N;
        dfa::Acc acc = dfa::first(D.h[i0], D.l[i0], xh[0], xl[0]);
#pragma unroll
        for (int l = 1; l < N; l++) {
            const int il = TR ? l * N + m : m * N + l;
            dfa::fma(acc, D.h[il], D.l[il], xh[l], xl[l]);
        }
        out[base + m * stride] = dfa::norm(acc);
    }
}

// The same line product in even-odd form (see EoMat): pair sums and
// differences, then 2 dot products of N/2 terms per output pair.
template <int N>
__device__ __forceinline__ void line_eo(const float2 *in, float2 *out, int base, int stride,
                                        const EoMat<N> &M) {
    constexpr int H = N / 2;
    float sh[H], sl[H], dh[H], dl[H];
#pragma unroll
    for (int l = 0; l < H; l++) {
        const float2 a = in[base + l * stride], b = in[base + (N - 1 - l) * stride];
        const float2 s = dfa::add(a, b);
        const float2 d = dfa::add(a, make_float2(-b.x, -b.y));
        sh[l] = s.x; sl[l] = s.y;
        dh[l] = d.x; dl[l] = d.y;
    }
    float ch = 0.f, cl = 0.f;
    if (N & 1) {
        const float2 c = in[base + H * stride];
        ch = c.x;
        cl = c.y;
    }
#pragma unroll
    for (int m = 0; m < H; m++) {
        dfa::Acc P = dfa::first(M.ah[m * H], M.al[m * H], dh[0], dl[0]);
#pragma unroll
        for (int l = 1; l < H; l++) dfa::fma(P, M.ah[m * H + l], M.al[m * H + l], dh[l], dl[l]);
        dfa::Acc Q = dfa::first(M.bh[m * (H + 1)], M.bl[m * (H + 1)], sh[0], sl[0]);
#pragma unroll
        for (int l = 1; l < H; l++) dfa::fma(Q, M.bh[m * (H + 1) + l], M.bl[m * (H + 1) + l], sh[l], sl[l]);
        if (N & 1) dfa::fma(Q, M.bh[m * (H + 1) + H], M.bl[m * (H + 1) + H], ch, cl);
        out[base + m * stride] = dfa::add_acc_raw(P, Q, 1.f);
        out[base + (N - 1 - m) * stride] = dfa::add_acc_raw(P, Q, -1.f);
    }
    if (N & 1) {
        dfa::Acc Y = dfa::first(M.ch[0], M.cl[0], dh[0], dl[0]);
#pragma unroll
        for (int l = 1; l < H; l++) dfa::fma(Y, M.ch[l], M.cl[l], dh[l], dl[l]);
        dfa::fma(Y, M.ch[H], M.cl[H], ch, cl);
        out[base + H * stride] = dfa::norm(Y);
    }
}

template <int N, bool EO>
struct DfConsts;
template <int N>
struct DfConsts<N, false> { using type = DfMat<N>; };
template <int N>
struct DfConsts<N, true> { using type = DfEo<N>; };


// Per-element arguments of df_element (pointers already offset to the element).
struct DfElemIO {
    const double *u;    // MODE 0: input
    const double *r;    // MODE 1: residual
    double *p;          // MODE 1: search direction (updated in place)
    double *x;          // MODE 1: iterate (owed update applied when xa != 0)
    const double *minv; // MODE 1: Jacobi inverse diagonal (z = minv r), or null
    double *w;          // output
    const float2 *g;    // gxyz pairs [6][n^3] of the element, scaled by 2^-(gexp-1023)
};

// Points of an element per thread of a T-thread CTA in the pointwise phases.
template <int N, int T>
__host__ __device__ constexpr int df_points_per_thread() {
    return (N * N * N + T - 1) / T;
}

// This thread's point-face masks (point_faces of q = threadIdx.x + k T),
// computed once per kernel for df_element's fused CG head.
template <int N, int T>
__device__ __forceinline__ void df_point_masks(unsigned *pf) {
#pragma unroll
    for (int k = 0; k < df_points_per_thread<N, T>(); k++) {
        const int q = threadIdx.x + k * T;
        pf[k] = q < N * N * N ? point_faces<N>(q) : 0u;
    }
}

// One element of ax_e in double-float arithmetic, executed by the whole CTA
// (every thread must call it; it contains barriers).  sm holds 6 n^3 pairs,
// s_emax is a shared int that must be 0 on entry (left 0 on exit).
// MODE 1 is the CG head: x += xa p, p = r + beta p, w = ax_e(p); with fuse,
// box-face points of w are zeroed and the element's share of <w,p>_c (the
// local products, see the final loop) is added to dot; pf holds the thread's point-face masks (df_point_masks; null:
// computed per point) and (ex, ey, ez) is the element's position in the box m.  The geometric
// factors and x are loaded with the streaming (evict-first) cache policy:
// they are not read again in the iteration, which keeps w and p in L2 for
// the dssum and update kernels that follow.
template <int N, int MODE, bool EO, int T = ax_df_threads(N)>
__device__ __forceinline__ void df_element(const DfElemIO &io, double beta, double xa, bool fuse,
                                           int gexp, const Mesh &m, int ex, int ey, int ez,
                                           const typename DfConsts<N, EO>::type &D, float2 *sm,
                                           int *s_emax, double &dot, const unsigned *pf = nullptr) {
    constexpr int N2 = N * N, N3 = N * N * N;
    float2 *U = sm;            // input pairs; later the r-partial of w
    float2 *W0 = sm + N3;      // wr -> ur
    float2 *W1 = sm + 2 * N3;  // ws -> us
    float2 *W2 = sm + 3 * N3;  // wt -> ut
    float2 *P1 = sm + 4 * N3;  // s-partial of w
    float2 *P2 = sm + 5 * N3;  // t-partial of w
    double *raw = reinterpret_cast<double *>(U);
    const int t = threadIdx.x;
    // ---- stage the element (raw FP64 first, to find its scale)
    int emax = 0;
    // x += alpha p of the previous iteration, then p = z + beta p; the
    // preconditioner and owed-update branches are uniform, so they are taken
    // outside the point loops
    auto stage = [&](double v, int q) {
        raw[q] = v;
        const int exb = (int)((__double_as_longlong(v) >> 52) & 0x7ff);
        emax = exb > emax ? exb : emax;
    };
    if (MODE == 0) {
        for (int q = t; q < N3; q += T) stage(__ldg(io.u + q), q);
    } else if (io.minv) {
        for (int q = t; q < N3; q += T) {
            const double pold = io.p[q];
            if (xa != 0.0) __stcs(io.x + q, fma(xa, pold, __ldcs(io.x + q)));
            const double v = fma(beta, pold, io.r[q] * io.minv[q]);
            io.p[q] = v;
            stage(v, q);
        }
    } else if (xa != 0.0) {
        for (int q = t; q < N3; q += T) {
            const double pold = io.p[q];
            __stcs(io.x + q, fma(xa, pold, __ldcs(io.x + q)));
            const double v = fma(beta, pold, io.r[q]);
            io.p[q] = v;
            stage(v, q);
        }
    } else {
        for (int q = t; q < N3; q += T) {
            const double v = fma(beta, io.p[q], io.r[q]);
            io.p[q] = v;
            stage(v, q);
        }
    }
    emax = __reduce_max_sync(0xffffffffu, emax);
    if ((t & 31) == 0) atomicMax(s_emax, emax);
    __syncthreads();
    int eu = *s_emax;
    eu = eu < 1 ? 1 : (eu > 2046 ? 2046 : eu);
    // u is scaled by 2^(1023-eu) so the element's max is in [1,2); w is
    // scaled back by 2^(eu-1023) and by the gxyz scale 2^(gexp-1023)
    const int sh_in = 1023 - eu;
    const int sh_out = (eu - 1023) + (gexp - 1023);
    for (int q = t; q < N3; q += T) U[q] = dfa::split_scaled(raw[q], sh_in);  // own entries only
    __syncthreads();

    // ---- forward: wr, ws, wt along this thread's line
    for (int task = t; task < 3 * N2; task += T) {
        int stride;
        const int base = line_of<N>(task, stride);
        float2 *Wd = task < N2 ? W0 : (task < 2 * N2 ? W1 : W2);
        if constexpr (EO)
            line_eo<N>(U, Wd, base, stride, D.fwd);
        else
            line_plain<N, false>(U, Wd, base, stride, D);
    }
    __syncthreads();

    // ---- geometric contraction, pointwise, in place
    const float2 *g = io.g;
    for (int q = t; q < N3; q += T) {
        const float2 wr = W0[q], ws = W1[q], wt = W2[q];
        const float2 g0 = __ldcs(g + q), g1 = __ldcs(g + N3 + q), g2 = __ldcs(g + 2 * N3 + q);
        const float2 g3 = __ldcs(g + 3 * N3 + q), g4 = __ldcs(g + 4 * N3 + q), g5 = __ldcs(g + 5 * N3 + q);
        dfa::Acc r = dfa::first(g0.x, g0.y, wr.x, wr.y);
        dfa::fma(r, g1.x, g1.y, ws.x, ws.y);
        dfa::fma(r, g2.x, g2.y, wt.x, wt.y);
        dfa::Acc s = dfa::first(g1.x, g1.y, wr.x, wr.y);
        dfa::fma(s, g3.x, g3.y, ws.x, ws.y);
        dfa::fma(s, g4.x, g4.y, wt.x, wt.y);
        dfa::Acc tt = dfa::first(g2.x, g2.y, wr.x, wr.y);
        dfa::fma(tt, g4.x, g4.y, ws.x, ws.y);
        dfa::fma(tt, g5.x, g5.y, wt.x, wt.y);
        W0[q] = dfa::raw(r);
        W1[q] = dfa::raw(s);
        W2[q] = dfa::raw(tt);
    }
    __syncthreads();

    // ---- backward: w_d(m) = sum_l dxtm1(m,l) u_d(l) = sum_l D(l,m) u_d(l)
    for (int task = t; task < 3 * N2; task += T) {
        int stride;
        const int base = line_of<N>(task, stride);
        const float2 *Ud = task < N2 ? W0 : (task < 2 * N2 ? W1 : W2);
        float2 *Pd = task < N2 ? U : (task < 2 * N2 ? P1 : P2);
        if constexpr (EO)
            line_eo<N>(Ud, Pd, base, stride, D.bwd);
        else
            line_plain<N, true>(Ud, Pd, base, stride, D);
    }
    __syncthreads();

    // ---- w = r-partial + s-partial + t-partial, scaled back, FP64 out
    if (MODE == 1 && fuse) {
        // Dirichlet points are zeroed before dssum (their sum is then +0, as
        // mask-after-dssum gives).  <w,p>_c is summed here over all local
        // points: p is continuous, so sum_g (sum_copies w) p_g equals the
        // sum of the local products before assembly.
        const unsigned bf = box_faces(ex, ey, ez, m);
#pragma unroll
        for (int k = 0; k < df_points_per_thread<N, T>(); k++) {
            const int q = t + k * T;
            if (df_points_per_thread<N, T>() * T != N3 && q >= N3) break;
            const float2 s = dfa::add(dfa::add(U[q], P1[q]), P2[q]);
            double wv = dfa::join_scaled(s, sh_out);
            const unsigned f = pf ? pf[k] : point_faces<N>(q);
            if (f & bf)
                wv = 0.0;
            else
                dot = fma(wv, io.p[q], dot);
            io.w[q] = wv;
        }
    } else {
        for (int q = t; q < N3; q += T) {
            const float2 s = dfa::add(dfa::add(U[q], P1[q]), P2[q]);
            io.w[q] = dfa::join_scaled(s, sh_out);
        }
    }
    if (t == 0) *s_emax = 0;
    __syncthreads();
}

// Even-odd constants of M (M = D, or D^T when tr) from the FP64 matrix.
template <int N>
inline void eo_consts(const double *Dm, bool tr, EoMat<N> &E) {
    constexpr int H = N / 2;
    auto M = [&](int mm, int l) { return tr ? Dm[l * N + mm] : Dm[mm * N + l]; };
    auto put = [](double v, float &h, float &l) {
        h = (float)v;
        l = (float)(v - (double)h);
    };
    for (int mm = 0; mm < H; mm++) {
        for (int l = 0; l < H; l++) put(0.5 * (M(mm, l) + M(N - 1 - mm, l)), E.ah[mm * H + l], E.al[mm * H + l]);
        for (int l = 0; l <= H; l++) {
            const double v = l < H ? 0.5 * (M(mm, l) - M(N - 1 - mm, l)) : ((N & 1) ? M(mm, H) : 0.0);
            put(v, E.bh[mm * (H + 1) + l], E.bl[mm * (H + 1) + l]);
        }
    }
    for (int l = 0; l <= H; l++) put((N & 1) ? M(H, l) : 0.0, E.ch[l], E.cl[l]);
}

// Fill the kernel-parameter constants for D (plain pairs or even-odd form).
template <int N, bool EO>
inline void df_consts(const double *Dh, typename DfConsts<N, EO>::type &D) {
    if constexpr (EO) {
        eo_consts<N>(Dh, false, D.fwd);
        eo_consts<N>(Dh, true, D.bwd);
    } else {
        for (int q = 0; q < N * N; q++) {
            const float h = (float)Dh[q];
            D.h[q] = h;
            D.l[q] = (float)(Dh[q] - (double)h);
        }
    }
}

}  // namespace nekgb
