// Measurement probe: the forward half of ax_e (Listing 1, arXiv 2005.13425
// Sec. III), w = D_r u + D_s u + D_t u per element, computed two ways in
// the same element loop so that their cost can be compared:
//
//  method 0  the CG head's double-float even-odd line products (line_eo) on
//            the FP32 pipes;
//  method 1  the tensor cores (tcgen05, kind::f16, FP32 accumulation in
//            tensor memory) on an error-free digit split in the manner of
//            Ozaki et al. (2012).  Each input value (|u 2^sh| <= 1) is cut
//            into six balanced base-512 digits and each entry of D into six
//            more, so that a product of two digits is an integer below
//            2^16 + and every class sum S_q = sum_{a+d=q} sum_j sigma_a(u_j)
//            delta_d(D_ij) is an integer below 2^24: the MMA adds exactly in
//            FP32.  The contraction of one direction is one chain of n/2
//            MMAs with M = 128 lines (n^2 used), K = 8n (n points x 8 digit
//            slots, six used) and N = 8n (n outputs x 8 classes, seven
//            used); the classes are recombined into a float pair on the CUDA
//            cores.  Remainders below 2^-54 of the scale and classes above 6
//            are dropped.
//
// Both methods stage the element, form the three directions' outputs as
// float pairs in shared memory, and finish with the same pass (the three
// pairs summed, reassembled in FP64 and stored).  Not used by the solvers.
#include <cuda_fp16.h>
#include <math.h>

#include <new>
#include <vector>

#include "ax_df_core.cuh"
#include "bulk.cuh"

namespace nekgb {

constexpr int kProbeThreads = 256;

// ---------------------------------------------------------------- tcgen05
__device__ __forceinline__ void tmem_alloc(unsigned *dst, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
}
// After its one allocation a CTA gives up the right to allocate, so that
// further CTAs can be scheduled onto the SM while it runs.
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D(tmem) (+)= A(smem) B(smem), both operands K-major, f16 in, f32 out.
__device__ __forceinline__ void tc_mma_f16(unsigned d_tmem, uint64_t adesc, uint64_t bdesc, unsigned idesc,
                                           unsigned accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// The barrier completes one phase when this thread's issued MMAs are done.
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}
// 8 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld8(unsigned taddr, unsigned (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// Keeps a value's uses after the preceding volatile asm (the TMEM load wait).
__device__ __forceinline__ unsigned after_wait(unsigned v) {
    asm volatile("" : "+r"(v));
    return v;
}

// Shared-memory matrix descriptor, no swizzle: core matrices of 8 rows x 16
// bytes, `lbo` bytes apart along K and `sbo` bytes apart along M (or N).
__device__ __forceinline__ uint64_t umma_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: f16 A and B, both K-major, f32 D.
__host__ __device__ constexpr unsigned umma_idesc_f16(int M, int N) {
    return (1u << 4) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

// NA = directions staged at once (1: one after another, 3: all together).
template <int N, int NA = 1>
struct TcLayout {
    static constexpr int M = 128;              // MMA rows: the n^2 lines of a direction, padded
    static constexpr int K = 8 * N;            // n points x 8 digit slots
    static constexpr int NOUT = 8 * N;         // n outputs x 8 classes
    static constexpr int LBO_A = 144;          // 128-byte core + 16 bytes: no bank conflicts on the stores
    static constexpr int SBO_A = N * LBO_A;
    static constexpr int A_BYTES = (M / 8) * SBO_A;   // one direction's A
    static constexpr int A_ALL = NA * A_BYTES;
    static constexpr int LBO_B = 128;
    static constexpr int SBO_B = N * LBO_B;
    static constexpr int B_BYTES = N * SBO_B;
    // output pairs: one array that the directions, taken one after another,
    // add into (NA = 1), or one per direction
    static constexpr int F_BYTES = (NA == 1 ? 1 : 3) * N * N * N * 8;
    static constexpr int SMEM = A_ALL + B_BYTES + F_BYTES;
    static constexpr int COLS = NA * NOUT;
    static constexpr unsigned TMEM_COLS = COLS <= 32 ? 32 : (COLS <= 64 ? 64 : (COLS <= 128 ? 128 : 256));
};

// Six balanced base-512 digits of h + l (|h + l| <= 1): h + l = sum_a
// sigma_a 2^(1 - 9(a+1)) + rest, |sigma_a| <= 260, |rest| <= 2^-54.  x holds
// the exact remainder of h; l is folded in at the third digit with its
// rounding error carried one digit further.  Returned as f16 pairs (a in the
// low half of word a/2) with the two unused slots zero.
__device__ __forceinline__ uint4 digits6(float h, float l) {
    const float MAG = 12582912.f;   // 1.5 2^23: (x + MAG) - MAG rounds |x| < 2^22 to an integer
    auto rnd = [&](float x) { return __fsub_rn(__fadd_rn(x, MAG), MAG); };
    float x = __fmul_rn(h, 256.f);
    const float d0 = rnd(x);
    x = __fmul_rn(__fsub_rn(x, d0), 512.f);
    const float d1 = rnd(x);
    x = __fmul_rn(__fsub_rn(x, d1), 512.f);
    float z, ez;
    dfa::two_sum(x, __fmul_rn(l, 67108864.f), z, ez);   // l 2^8 2^18 in the units of digit 2
    const float d2 = rnd(z);
    x = __fmaf_rn(ez, 512.f, __fmul_rn(__fsub_rn(z, d2), 512.f));
    const float d3 = rnd(x);
    x = __fmul_rn(__fsub_rn(x, d3), 512.f);
    const float d4 = rnd(x);
    x = __fmul_rn(__fsub_rn(x, d4), 512.f);
    const float d5 = rnd(x);
    auto pk = [](float lo, float hi) {
        const __half2 v = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<const unsigned *>(&v);
    };
    return make_uint4(pk(d0, d1), pk(d2, d3), pk(d4, d5), 0u);
}

// The pair sc sum_q S_q 2^(-9q) (S_q exact integers in FP32, sc = 2^(1 + ED
// - 18) for inputs <= 1 and |D| <= 2^(ED-1)): the two leading classes by
// TwoSum, classes 3..6 by a plain sum below them; unnormalised.
__device__ __forceinline__ float2 recombine(const unsigned (&r)[8], float sc) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; q++) v[q] = __uint_as_float(after_wait(r[q]));
    float s, e1, e2;
    dfa::two_sum(v[0], __fmul_rn(v[1], 0x1p-9f), s, e1);
    dfa::two_sum(s, __fmul_rn(v[2], 0x1p-18f), s, e2);
    const float tail =
        __fmaf_rn(v[6], 0x1p-54f, __fmaf_rn(v[5], 0x1p-45f, __fmaf_rn(v[4], 0x1p-36f, __fmul_rn(v[3], 0x1p-27f))));
    const float e = __fadd_rn(e1, __fadd_rn(e2, tail));
    // unnormalised (|e| within a few ulps of s), as the line products leave theirs
    return make_float2(__fmul_rn(s, sc), __fmul_rn(e, sc));
}

struct ProbeArgs {
    const double *u;
    double *w;
    const uint4 *bimg;    // method 1: the digit matrix of D in its shared-memory layout
    int64_t E;
    int sh;               // u 2^sh has |.| <= 1
    float rscale;         // method 1: 2^(1 + ED - 18), |D| <= 2^(ED-1)
    int *status;          // set to NB_ERR_TIMEOUT if an MMA does not complete
};

// METHOD 0: line products; 1: tensor cores, one direction at a time; 2:
// tensor cores, the three directions' MMAs issued together.
template <int N, int METHOD>
__global__ void __launch_bounds__(kProbeThreads)
probe_grad_kernel(ProbeArgs a, const __grid_constant__ EoMat<N> Dm) {
    constexpr int NA = METHOD == 2 ? 3 : 1;
    using L = TcLayout<N, NA>;
    constexpr int N2 = N * N, N3 = N * N * N;
    constexpr int T = kProbeThreads;
    constexpr int PPT = (N3 + T - 1) / T;
    extern __shared__ __align__(128) unsigned char psm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ unsigned s_tmem;
    const int t = threadIdx.x;
    // [3][N3] output pairs; method 0 keeps its input pairs X in front of them
    float2 *F = reinterpret_cast<float2 *>(psm + (METHOD >= 1 ? L::A_ALL + L::B_BYTES : N3 * 8));
    float2 *X = reinterpret_cast<float2 *>(psm);
    unsigned tbase = 0;
    if constexpr (METHOD >= 1) {
        if (t == 0) {
            mbar_init(&bar, 1);
            fence_mbar_init();
        }
        if (t < 32) {
            tmem_alloc(&s_tmem, L::TMEM_COLS);
            tmem_relinquish();
        }
        for (int q = t; q < L::B_BYTES / 16; q += T)
            reinterpret_cast<uint4 *>(psm + L::A_ALL)[q] = a.bimg[q];
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        tbase = s_tmem;
    }
    const unsigned a_addr = smem_addr(psm), b_addr = smem_addr(psm + L::A_ALL);
    constexpr unsigned IDESC = umma_idesc_f16(L::M, L::NOUT);
    unsigned phase = 0;
    bool ok = true;
    // A offsets of this thread's points in each direction's layout (row =
    // line, core = position along the line) and the bases of its output
    // points: the same for every element
    int aoff[PPT][3];
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int q = t + k * T;
        const int pi = q % N, pj = (q / N) % N, pk = q / N2;
        const int ln[3] = {pj + N * pk, pi + N * pk, pi + N * pj}, pos[3] = {pi, pj, pk};
#pragma unroll
        for (int d = 0; d < 3; d++) aoff[k][d] = (ln[d] >> 3) * L::SBO_A + pos[d] * L::LBO_A + (ln[d] & 7) * 16;
    }
    const int wq = t >> 5, line = 32 * (wq & 3) + (t & 31);   // this thread's TMEM lane
    const int i0 = (wq >> 2) * (N / 2);                        // its outputs i0 .. i0 + N/2 - 1
    // output point of (line, i) in direction d: obase[d] + i * ostep[d]
    const int obase[3] = {N * line, (line % N) + N2 * (line / N), line};
    constexpr int ostep[3] = {1, N, N2};
    for (int64_t e = blockIdx.x; e < a.E && ok; e += gridDim.x) {
        const double *u = a.u + e * N3;
        if constexpr (METHOD == 0) {
            for (int q = t; q < N3; q += T) X[q] = dfa::split_scaled<true>(__ldcs(u + q), a.sh);
            __syncthreads();
            for (int task = t; task < 3 * N2; task += T) {
                int stride;
                const int base = line_of<N>(task, stride);
                line_eo<N>(X, F + (task / N2) * N3, base, stride, Dm);
            }
            __syncthreads();
        } else {
            uint4 dg[PPT];
#pragma unroll
            for (int k = 0; k < PPT; k++) {
                const int q = t + k * T;
                if (q < N3) {
                    const float2 v = dfa::split_scaled<true>(__ldcs(u + q), a.sh);
                    dg[k] = digits6(v.x, v.y);
                }
            }
            const unsigned lrow = (unsigned)(32 * (wq & 3)) << 16;
#pragma unroll
            for (int d0 = 0; d0 < 3; d0 += NA) {
#pragma unroll
                for (int dd = 0; dd < NA; dd++) {
#pragma unroll
                    for (int k = 0; k < PPT; k++)
                        if (t + k * T < N3)
                            *reinterpret_cast<uint4 *>(psm + dd * L::A_BYTES + aoff[k][d0 + dd]) = dg[k];
                }
                fence_proxy_async();
                tc_fence_before();
                __syncthreads();
                tc_fence_after();
                bool done = true;
                if (t == 0) {
#pragma unroll
                    for (int dd = 0; dd < NA; dd++)
#pragma unroll
                        for (int ks = 0; ks < N / 2; ks++)
                            tc_mma_f16(tbase + dd * L::NOUT,
                                       umma_desc(a_addr + dd * L::A_BYTES + ks * 2 * L::LBO_A, L::LBO_A, L::SBO_A),
                                       umma_desc(b_addr + ks * 2 * L::LBO_B, L::LBO_B, L::SBO_B), IDESC, ks > 0);
                    tc_commit(&bar);
                    // one thread observes completion; the barrier and the
                    // fence after it order the others' TMEM loads behind it
                    done = mbar_wait(&bar, phase);
                }
                tc_fence_before();
                if (!__syncthreads_and(done)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                phase ^= 1u;
#pragma unroll
                for (int dd = 0; dd < NA; dd++) {
                    const int dir = d0 + dd;
                    // this thread's outputs, TB at a time: TMEM loads, one wait, recombination
                    constexpr int TB = 2;
#pragma unroll
                    for (int o0 = 0; o0 < N / 2; o0 += TB) {
                        unsigned r[TB][8];
#pragma unroll
                        for (int o = 0; o < TB; o++)
                            if (o0 + o < N / 2) tc_ld8(tbase + lrow + dd * L::NOUT + 8 * (i0 + o0 + o), r[o]);
                        tc_wait_ld();
                        if (line < N2) {
#pragma unroll
                            for (int o = 0; o < TB; o++) {
                                if (o0 + o >= N / 2) break;
                                const float2 v = recombine(r[o], a.rscale);
                                const int P = obase[dir] + (i0 + o0 + o) * ostep[dir];
                                if (NA == 1)   // directions in turn: add into the one array
                                    F[P] = dir == 0 ? v : dfa::add(F[P], v);
                                else
                                    F[dir * N3 + P] = v;
                            }
                        }
                    }
                }
                tc_fence_before();
            }
            if (!ok) break;
            __syncthreads();
        }
        double *w = a.w + e * N3;
        for (int q = t; q < N3; q += T) {
            const float2 v = METHOD == 1 ? F[q] : dfa::add(dfa::add(F[q], F[N3 + q]), F[2 * N3 + q]);
            __stcs(w + q, dfa::join_scaled(v, -a.sh));
        }
        __syncthreads();
    }
    if constexpr (METHOD >= 1) {
        if (!ok) {   // an MMA did not complete in time: wait once more (bounded), then free TMEM
            if (t == 0) {
                mbar_wait(&bar, phase);
                atomicExch(a.status, (int)NB_ERR_TIMEOUT);
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (t < 32) tmem_dealloc(tbase, L::TMEM_COLS);
    }
}

// ---------------------------------------------------------------- host
// Balanced base-512 digits of v (|v| <= 1/2) in FP64, exact: v = sum_d
// delta_d 2^(-9(d+1)) + rest.
static void digits_host(double v, int (&dg)[6]) {
    double x = v * 512.0;
    for (int d = 0; d < 6; d++) {
        const double r = nearbyint(x);
        dg[d] = (int)r;
        x = (x - r) * 512.0;
    }
}

template <int N>
static std::vector<uint16_t> b_image(const double *Dm, int ED) {
    using L = TcLayout<N>;
    std::vector<uint16_t> img(L::B_BYTES / 2, 0);
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            int dg[6];
            digits_host(ldexp(Dm[i * N + j], -ED), dg);
            for (int q = 0; q < 8; q++)
                for (int aa = 0; aa < 6; aa++) {
                    const int d = q - aa;
                    if (d < 0 || d > 5) continue;
                    const size_t off = (size_t)(i * L::SBO_B + j * L::LBO_B + q * 16) / 2 + aa;
                    img[off] = __half_as_ushort(__float2half_rn((float)dg[d]));
                }
        }
    return img;
}

template <int N, int METHOD>
static nb_status probe_launch(nb_ctx *c, const double *u, double *w, int sh) {
    using L = TcLayout<N, METHOD == 2 ? 3 : 1>;
    const size_t smem = METHOD >= 1 ? (size_t)L::SMEM : (size_t)(N * N * N * 8 * 4);   // method 0: X + 3 arrays
    EoMat<N> Dm;
    eo_consts<N>(c->D_host, false, Dm);
    ProbeArgs a{};
    a.u = u;
    a.w = w;
    a.E = c->m.E;
    a.sh = sh;
    uint4 *d_img = nullptr;
    int *d_status = nullptr;
    NB_CUDA(dev_alloc((void **)&d_status, sizeof(int)));
    nb_status st = NB_OK;
    do {
        if (cudaMemsetAsync(d_status, 0, sizeof(int), c->stream) != cudaSuccess) {
            st = cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
            break;
        }
        a.status = d_status;
        if (METHOD >= 1) {
            double dmax = 0.0;
            for (int q = 0; q < N * N; q++) dmax = fmax(dmax, fabs(c->D_host[q]));
            const int ED = (int)ceil(log2(dmax)) + 1;   // |D| 2^-ED <= 1/2
            a.rscale = ldexpf(1.f, 1 + ED - 18);
            const std::vector<uint16_t> img = b_image<N>(c->D_host, ED);
            if (dev_alloc((void **)&d_img, L::B_BYTES) != cudaSuccess) {
                st = fail(NB_ERR_OOM, "probe image");
                break;
            }
            if (cudaMemcpyAsync(d_img, img.data(), L::B_BYTES, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
                st = cuda_fail(cudaGetLastError(), "cudaMemcpyAsync");
                break;
            }
            a.bimg = d_img;
        }
        auto kern = probe_grad_kernel<N, METHOD>;
        if ((st = set_smem(kern, smem)) != NB_OK) break;
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kProbeThreads, smem);
        if (METHOD >= 1) {
            // the occupancy query answers 1 for this kernel; take the limits
            // of shared memory, registers and tensor memory (512 columns)
            cudaFuncAttributes fa{};
            if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
                st = cuda_fail(cudaGetLastError(), "cudaFuncGetAttributes");
                break;
            }
            const int by_smem = (227 * 1024) / ((int)smem + (int)fa.sharedSizeBytes + 1024);
            const int by_regs = 65536 / (((fa.numRegs + 7) / 8) * 8 * kProbeThreads);
            const int by_tmem = 512 / (int)L::TMEM_COLS;
            occ = by_smem < by_regs ? by_smem : by_regs;
            occ = occ < by_tmem ? occ : by_tmem;
        }
        if (occ < 1) occ = 1;
        const int64_t cap = (int64_t)device_sms() * occ;
        const int grid = (int)(c->m.E < cap ? c->m.E : cap);
        {
            LaunchTimer tm(c, NB_K_AX);
            kern<<<grid, kProbeThreads, smem, c->stream>>>(a, Dm);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            st = cuda_fail(e, "probe_grad_kernel");
            break;
        }
        int h_status = 0;
        if (cudaMemcpyAsync(&h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            st = cuda_fail(cudaGetLastError(), "probe status");
            break;
        }
        if (h_status != 0) st = fail(NB_ERR_TIMEOUT, "a tensor-core MMA of the probe did not complete");
    } while (0);
    if (d_img) cudaFree(d_img);
    cudaFree(d_status);
    if (st == NB_OK) st = harvest_timing(c);
    return st;
}

}  // namespace nekgb

using namespace nekgb;

extern "C" nb_status nb_probe_grad(nb_ctx *c, int method, const double *u, double *w, double umax) {
    try {
        if (!c) return fail(NB_ERR_ARG, "NULL context");
        if (!u || !w || !(umax > 0.0) || !isfinite(umax)) return fail(NB_ERR_ARG, "nb_probe_grad: bad arguments");
        if (method < 0 || method > 2) return fail(NB_ERR_ARG, "nb_probe_grad: method is 0, 1 or 2");
        const int sh = -(int)ceil(log2(umax));   // |u| 2^sh <= 1
        switch (c->m.n) {
            case 8:
                return method == 0 ? probe_launch<8, 0>(c, u, w, sh)
                                   : (method == 1 ? probe_launch<8, 1>(c, u, w, sh) : probe_launch<8, 2>(c, u, w, sh));
            case 10:
                return method == 0 ? probe_launch<10, 0>(c, u, w, sh)
                                   : (method == 1 ? probe_launch<10, 1>(c, u, w, sh)
                                                  : probe_launch<10, 2>(c, u, w, sh));
            default: return fail(NB_ERR_ARG, "nb_probe_grad: n must be 8 or 10");
        }
    } catch (const std::bad_alloc &) {
        return fail(NB_ERR_OOM, "host allocation failed");
    } catch (...) {
        return fail(NB_ERR_STATE, "unexpected C++ exception");
    }
}
