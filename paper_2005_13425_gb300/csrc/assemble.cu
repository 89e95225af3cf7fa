// The second kernel of the two-kernel CG iteration: direct stiffness
// summation fused with the residual update (arXiv 2005.13425 Sec. III: the
// second step of Ax communicates element results to the neighbours; the CG
// vector update r -= alpha w follows).
//
// With <w,p>_c summed by the head as local products (p is continuous), alpha
// is known before dssum.  The assembled w is then needed only to update r,
// so this kernel never writes w back:
//  * element-interior points have one copy: r -= alpha w there.  The other
//    single-copy points lie on box faces, where the Dirichlet mask keeps w
//    (zeroed by the head) and r at +0.0, so they are left alone;
//  * every shared node gathers its copies of w in ascending element order
//    (the dssum order, so the sum is the one dssum writes), updates r once
//    (r is continuous: every copy holds the same value) and writes the new
//    value to every copy.
// <r,r>_c = sum over unique nodes of r^2 is accumulated on the way: each
// single-copy point once, each shared node once (no multiplicity weights).
// The last CTA forms rho, beta and the convergence decision.  The FP64
// variant squares on the FP32 pipes (dfa::SqAcc32, r scaled by 2^sh from
// the previous <r,r>_c); the FP32 variant uses compensated FP32 sums.
#include <type_traits>

#include "df.cuh"
#include "gs_fast.cuh"
#include "gs_nodes.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace nekgb {

constexpr int kAsmThreads = 256;

template <typename T, int N>
__global__ void __launch_bounds__(kAsmThreads, 5)
assemble_update_kernel(T *__restrict__ r, const T *__restrict__ w, Mesh m, DsCat dd, CgScalars *sc,
                       double *partials, double *hist) {
    if (sc->done) return;
    constexpr bool F32 = std::is_same<T, float>::value;
    constexpr int N3 = N * N * N;
    const T alpha = (T)sc->alpha;
    const int erb = (int)((__double_as_longlong(sc->rr) >> 52) & 0x7ff);
    const int sh = erb == 0 ? 0 : -((erb - 1023) >> 1);
    dfa::SqAcc32 sq;
    dfa::Acc32 acc32;
    auto add_sq = [&](T rn) {
        if constexpr (F32) {
            acc32.add_prod(rn, rn);
        } else {
            const float2 v = dfa::split_scaled<true>(rn, sh);
            sq.add_sq(v.x, v.y, 1.f);
        }
    };
    // element-interior points, element by element
    if constexpr (N > 2) {
        constexpr int NI = N - 2, NI3 = NI * NI * NI;
        constexpr int KI = (NI3 + kAsmThreads - 1) / kAsmThreads;
        int qk[KI];
#pragma unroll
        for (int k = 0; k < KI; k++) {
            const int qi = threadIdx.x + k * kAsmThreads;
            const int a = qi % NI, b = (qi / NI) % NI, c = qi / (NI * NI);
            qk[k] = (1 + a) + N * (1 + b) + N * N * (1 + c);
        }
        for (int64_t e = blockIdx.x; e < m.E; e += gridDim.x) {
            const int64_t base = e * N3;
#pragma unroll
            for (int k = 0; k < KI; k++) {
                if (KI * kAsmThreads != NI3 && threadIdx.x + k * kAsmThreads >= NI3) break;
                const int64_t q = base + qk[k];
                const T rn = fma(-alpha, __ldcs(w + q), r[q]);
                r[q] = rn;
                add_sq(rn);
            }
        }
    }
    // shared nodes
    const int total = dd.o[7];
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        int64_t idx[8];
        const int c = cat_copies<N>(q, dd, idx);
        T s;
        if (c == 2) {
            s = plus_zero(__ldcs(w + idx[0])) + __ldcs(w + idx[1]);
        } else if (c == 4) {
            T a[4];
#pragma unroll
            for (int k = 0; k < 4; k++) a[k] = __ldcs(w + idx[k]);
            s = plus_zero(a[0]);
#pragma unroll
            for (int k = 1; k < 4; k++) s = s + a[k];
        } else {
            T a[8];
#pragma unroll
            for (int k = 0; k < 8; k++) a[k] = __ldcs(w + idx[k]);
            s = plus_zero(a[0]);
#pragma unroll
            for (int k = 1; k < 8; k++) s = s + a[k];
        }
        const T rn = fma(-alpha, s, r[idx[0]]);
        for (int k = 0; k < c; k++) r[idx[k]] = rn;
        add_sq(rn);
    }
    double v[1], tot[1];
    if constexpr (F32) v[0] = acc32.value();
    else v[0] = sq.value() * __longlong_as_double((long long)(1023 - 2 * sh) << 52);
    if (!last_block_reduce<1>(v, partials, 0, blockIdx.x, gridDim.x, gridDim.x, &sc->ticket, tot)) return;
    if (threadIdx.x != 0) return;
    const double rho = tot[0];
    // <p,p>_c of the next search direction p' = r' + beta p: r' is
    // orthogonal to p, so <p',p'>_c = rho' + beta^2 <p,p>_c (p_0 = r_0).
    // Only a scale for the head's pairs is taken from it.
    const double pprev = sc->it == 0 ? sc->rho : sc->pn2;
    sc->rr = rho;
    sc->rho_old = sc->rho;
    sc->rho = rho;
    sc->beta = rho / sc->rho_old;
    sc->pn2 = fma(sc->beta * sc->beta, pprev, rho);
    const int it = sc->it + 1;
    sc->it = it;
    if (hist) hist[it] = rho;
    const bool conv = sc->tol > 0.0 && sqrt(rho) / sqrt(sc->fnorm2) <= sc->tol;
    if (rho == 0.0 || conv || it >= sc->maxit) sc->done = 1;
}

static int asm_grid(const nb_ctx *c) {
    const int64_t cap = (int64_t)device_sms() * 5;
    return (int)(c->m.E < cap ? c->m.E : cap);
}

template <typename T>
static void asm_launch(nb_ctx *c, T *r, const T *w, double *hist) {
    const DsCat dd = make_ds_cat(c->m);
    const int grid = asm_grid(c);
    switch (c->m.n) {
#define NB_CASE(NN)                                                                                   \
    case NN:                                                                                          \
        assemble_update_kernel<T, NN><<<grid, kAsmThreads, 0, c->stream>>>(r, w, c->m, dd, c->d_sc,   \
                                                                           c->d_partials, hist);      \
        break;
        NB_CASE(2) NB_CASE(3) NB_CASE(4) NB_CASE(5) NB_CASE(6) NB_CASE(7) NB_CASE(8)
        NB_CASE(9) NB_CASE(10) NB_CASE(11) NB_CASE(12) NB_CASE(13) NB_CASE(14) NB_CASE(15)
        NB_CASE(16)
#undef NB_CASE
        default: break;
    }
}

// FP64 CG: r -= alpha QQ^T w with <r,r>_c, rho, beta, convergence.
nb_status launch_assemble_update(nb_ctx *c) {
    LaunchTimer tm(c, NB_K_UPDATE);
    asm_launch<double>(c, c->d_r, c->d_w, c->d_hist);
    NB_LAUNCH_CHECK("assemble_update_kernel");
    return NB_OK;
}

// The inner FP32 CG of the mixed-precision solve (no history).
nb_status launch_assemble_update32(nb_ctx *c) {
    LaunchTimer tm(c, NB_K_UPDATE);
    asm_launch<float>(c, c->d_r32, c->d_w32, nullptr);
    NB_LAUNCH_CHECK("assemble_update_kernel<f32>");
    return NB_OK;
}

}  // namespace nekgb
