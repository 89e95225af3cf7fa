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

// The shared nodes q in [a, b) with C copies each that fall to this thread
// (q = tid mod S, the same round-robin over all shared nodes as one loop
// would give), U of them per step: every load of a step is issued before
// the first sum, so each thread keeps up to U (C + 1) loads in flight.  The
// copies are summed in ascending element order (the dssum order), r is
// updated once and written to every copy.
template <int N, int C, int U, typename T, typename Sq>
__device__ __forceinline__ void update_nodes(T *__restrict__ r, const T *__restrict__ w, const DsCat &dd,
                                             int a, int b, int tid, int S, T alpha, Sq &add_sq) {
    const int first = a + ((tid - a % S) % S + S) % S;
    for (int64_t q = first; q < b; q += (int64_t)U * S) {
        int64_t i0[U];
        int kind[U];
        T v[U][C], rv[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int64_t qu = q + u * S;
            kind[u] = 0;
            i0[u] = 0;
            if (qu < b) {
                if constexpr (C == 2) i0[u] = face_first<N>((int)qu, dd, kind[u]);
                else if constexpr (C == 4) i0[u] = edge_first<N>((int)qu, dd, kind[u]);
                else i0[u] = vertex_first<N>((int)qu, dd);
                v[u][0] = __ldcs(w + i0[u]);
#pragma unroll
                for (int k = 1; k < C; k++) v[u][k] = __ldcs(w + i0[u] + copy_offset<N, C>(k, kind[u], dd));
                rv[u] = r[i0[u]];
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (q + u * S < b) {
                T s = plus_zero(v[u][0]);
#pragma unroll
                for (int k = 1; k < C; k++) s = s + v[u][k];
                const T rn = fma(-alpha, s, rv[u]);
                r[i0[u]] = rn;
#pragma unroll
                for (int k = 1; k < C; k++) r[i0[u] + copy_offset<N, C>(k, kind[u], dd)] = rn;
                add_sq(rn);
            }
        }
    }
}

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
    // element-interior points: each step takes UE elements (KI points of
    // each for this thread) and issues the loads of CH points before their
    // updates, so up to 2 CH loads are in flight per thread
    if constexpr (N > 2) {
        constexpr int NI = N - 2, NI3 = NI * NI * NI;
        constexpr int KI = (NI3 + kAsmThreads - 1) / kAsmThreads;
        constexpr int UE = KI >= 4 ? 1 : 4 / KI, NB = UE * KI, CH = F32 ? 6 : 4;
        int qk[KI];
        bool ok[KI];
#pragma unroll
        for (int k = 0; k < KI; k++) {
            const int qi = threadIdx.x + k * kAsmThreads;
            const int a = qi % NI, b = (qi / NI) % NI, c = qi / (NI * NI);
            qk[k] = (1 + a) + N * (1 + b) + N * N * (1 + c);
            ok[k] = KI * kAsmThreads == NI3 || qi < NI3;
        }
        for (int64_t e = blockIdx.x; e < m.E; e += (int64_t)UE * gridDim.x) {
#pragma unroll
            for (int j0 = 0; j0 < NB; j0 += CH) {
                T wv[CH], rv[CH];
                int64_t qa[CH];
                bool go[CH];
#pragma unroll
                for (int jj = 0; jj < CH; jj++) {
                    const int j = j0 + jj, u = j / KI, k = j % KI;
                    const int64_t eu = e + (int64_t)u * gridDim.x;
                    go[jj] = j < NB && ok[k] && eu < m.E;
                    qa[jj] = eu * N3 + qk[k];
                    if (go[jj]) {
                        wv[jj] = __ldcs(w + qa[jj]);
                        rv[jj] = r[qa[jj]];
                    }
                }
#pragma unroll
                for (int jj = 0; jj < CH; jj++) {
                    if (go[jj]) {
                        const T rn = fma(-alpha, wv[jj], rv[jj]);
                        r[qa[jj]] = rn;
                        add_sq(rn);
                    }
                }
            }
        }
    }
    // shared nodes, one copy count at a time
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int S = gridDim.x * blockDim.x;
    update_nodes<N, 2, F32 ? 3 : 2>(r, w, dd, dd.o[0], dd.o[3], tid, S, alpha, add_sq);
    update_nodes<N, 4, F32 ? 2 : 1>(r, w, dd, dd.o[3], dd.o[6], tid, S, alpha, add_sq);
    update_nodes<N, 8, 1>(r, w, dd, dd.o[6], dd.o[7], tid, S, alpha, add_sq);
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
