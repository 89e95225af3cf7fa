// Internal declarations shared by the CUDA sources of libnekgb.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/nekgb.h"

namespace nekgb {

constexpr int kMaxN = 16;

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
nb_status fail(nb_status s, const std::string &msg);
nb_status cuda_fail(cudaError_t e, const char *what);

#define NB_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return ::nekgb::cuda_fail(_e, #call);    \
    } while (0)

#define NB_LAUNCH_CHECK(what)                                           \
    do {                                                                \
        cudaError_t _e = cudaGetLastError();                            \
        if (_e != cudaSuccess) return ::nekgb::cuda_fail(_e, what);     \
    } while (0)

// Device allocation with host-side fault injection: NEKGB_FAIL_ALLOC=k
// makes the k-th allocation of the process (1-based) fail, so failure
// paths can be tested without touching the GPU.
cudaError_t dev_alloc(void **p, size_t bytes);

// Allow `bytes` of dynamic shared memory for a kernel on the current device
// (set once per kernel and device; thread-safe).
nb_status smem_attr(const void *kernel, size_t bytes);
// Number of SMs of the current device (queried once per device; thread-safe).
int device_sms();
template <typename K>
inline nb_status set_smem(K *kernel, size_t bytes) {
    return smem_attr(reinterpret_cast<const void *>(kernel), bytes);
}

// ---------------------------------------------------------------- mesh
// Everything a kernel needs to know about the box topology.
struct Mesh {
    int ex, ey, ez, n;
    int64_t E, npts;
    int64_t NX, NY, NZ;
    // exact reciprocals for element id -> (ex, ey, ez): ceil(2^64 / d) for
    // d = ex and d = ex ey (0 when d = 1); see make_box_mesh
    unsigned long long inv_ex, inv_exy;
};

// The box mesh of ex x ey x ez elements with n points per direction.
// floor(q / d) = floor(q ceil(2^64 / d) / 2^64) for every 32-bit q and
// d >= 2 (Granlund and Montgomery, 1994), so element coordinates need one
// multiply-high per division.
inline Mesh make_box_mesh(int ex, int ey, int ez, int n) {
    Mesh m;
    m.ex = ex; m.ey = ey; m.ez = ez; m.n = n;
    m.E = (int64_t)ex * ey * ez;
    m.npts = m.E * n * n * n;
    m.NX = (int64_t)ex * (n - 1) + 1;
    m.NY = (int64_t)ey * (n - 1) + 1;
    m.NZ = (int64_t)ez * (n - 1) + 1;
    auto recip = [](unsigned long long d) { return d <= 1 ? 0ull : (~0ull / d) + 1ull; };
    m.inv_ex = recip((unsigned long long)ex);
    m.inv_exy = recip((unsigned long long)ex * ey);
    return m;
}

// ---------------------------------------------------------------- CG state
// Device-resident scalars of one CG solve.
// CgScalars::fault: a scaled share of the FP64 CG head's exact <w,p>_c sum
// reached the bound that keeps the 128-bit sum from overflowing.
constexpr int kFaultExactSumRange = 1;

struct CgScalars {
    double rho;        // <r,z>_c (z = r without a preconditioner, minv r with Jacobi)
    double rr;         // <r,r>_c (convergence test and history)
    double rho_old;    // previous rho
    double alpha, beta;
    double pap;        // <w,p>_c
    double fnorm2;     // <f,f>_c
    double tol;        // relative tolerance (<= 0: fixed iterations)
    double x_alpha;    // alpha of the x update still owed to x (0: none)
    double pn2;        // <p,p>_c of the next iteration's p (unpreconditioned CG; see assemble.cu)
    int it;            // iterations completed
    int maxit;
    int done;          // 1: no further iteration runs
    int status;        // 0 ok, NB_ERR_BREAKDOWN, NB_ERR_TIMEOUT
    int fault;         // detail of a BREAKDOWN status: 0, or kFaultExactSumRange
    unsigned int ticket;  // last-block-done counter for reductions
    unsigned int next_elem;  // element counter of the CG head's dynamic schedule (reset by its last CTA)
};

struct TimingRec {
    int kid;
    cudaEvent_t a, b;
};

}  // namespace nekgb

struct nb_ctx {
    nekgb::Mesh m;
    nb_precision prec;
    cudaStream_t stream;
    int ax_variant;       // 0 auto, 1 fp64, 2 double-float
    double D_host[nekgb::kMaxN * nekgb::kMaxN];
    // operator data
    double *d_D = nullptr;      // n*n, D[i*n+l]
    double *d_gxyz = nullptr;   // [E][6][n^3]
    uint8_t *d_mask = nullptr;  // [E][n^3] or null (box mask)
    float *d_Df = nullptr;      // D as double-float pairs / fp32 (2*n*n)
    float2 *d_gxyz_df = nullptr;  // [E][6][n^3] (hi,lo) pairs for double-float ax
    float *d_gxyz32 = nullptr;  // [E][6][n^3] fp32 for the mixed inner solve
    int gxyz_exp = 1023;
    bool d_eo = false;          // D is centro-antisymmetric: even-odd line products
    bool is_box = false;        // built by nb_setup_box (coordinates known)
    // slab of a z-partitioned box (nb_setup_slab): element layers
    // slab_z0 .. slab_z0 + m.ez - 1 of a box slab_ez_global layers high
    bool slab = false;
    int slab_z0 = 0, slab_ez_global = 0;
    double box_amp = 0.0, box_s[3] = {0, 0, 0};        // biased exponent of max|gxyz| (pairs are scaled by 2^-(gxyz_exp-1023))
    // CG workspace
    double *d_r = nullptr, *d_p = nullptr, *d_w = nullptr, *d_x = nullptr;
    double *d_partials = nullptr;
    int partial_cap = 0;
    double *d_minv = nullptr;           // Jacobi: 1/diag(A) (0 at Dirichlet points), or null
    nekgb::CgScalars *d_sc = nullptr;
    nekgb::CgScalars *h_sc = nullptr;   // pinned mirror
    double *d_hist = nullptr;
    int hist_cap = 0;
    int last_iters = 0;
    int ax_grid = 0;                    // partial slots written by the fused ax_e
    bool fused_cg = false;              // box mask: fused CG iteration
    bool two_kernel = false;            // fused and no preconditioner: head + assemble_update
    // mixed precision workspace
    float *d_r32 = nullptr, *d_p32 = nullptr, *d_w32 = nullptr, *d_z32 = nullptr;
    // CUDA graphs of chunks of FP64 and FP32 (inner) CG iterations
    cudaGraphExec_t cg_graph = nullptr;
    int cg_graph_chunk = 0;
    bool cg_graph_two = false;          // the iteration form captured in cg_graph
    cudaGraphExec_t cg_graph32 = nullptr;
    int cg_graph32_chunk = 0;
    // mixed-precision parameters and statistics
    bool f32_plain = false;             // FP32 ax_e without bulk staging (NEKGB_F32_STAGED=0)
    unsigned long long test_unarmed_wait_ns = 0;   // NEKGB_TEST_UNARMED_WAIT_NS (tests of the timeout path)
    int test_dot_shift = 0;             // NEKGB_TEST_DOT_SHIFT: added to the exact sum's scale (tests of its range check)
    double mixed_inner_tol = 1e-4;
    int mixed_max_outer = 50;
    int last_outer = 0;
    // timing: 0 off, 1 every launch event-timed (no graphs), 2 sampled (the
    // FP64 CG keeps its graphs and event-times one iteration per chunk)
    int timing = 0;
    bool capturing = false;             // a graph is being captured: launches are counted into capture_count
    int capture_count = 0;
    int cg_graph_kernels = 0;           // kernels in cg_graph
    int cg_graph32_kernels = 0;         // kernels in cg_graph32
    int64_t n_launched = 0;             // kernels launched since timing was last enabled (graph kernels included)
    std::vector<nekgb::TimingRec> pending;
    std::vector<cudaEvent_t> event_pool;
    double t_ms[NB_K_COUNT] = {0};
    int64_t t_launch[NB_K_COUNT] = {0};
    size_t device_bytes = 0;
};

namespace nekgb {

// Event bracketing of one launch when timing is on.
struct LaunchTimer {
    nb_ctx *c;
    int kid;
    cudaEvent_t a = nullptr, b = nullptr;
    LaunchTimer(nb_ctx *ctx, int k);
    ~LaunchTimer();
};
nb_status harvest_timing(nb_ctx *c);

// ---------------------------------------------------------------- kernels
// ax_e (ax_fp64.cu / ax_df.cu)
nb_status launch_ax(nb_ctx *c, const double *u, double *w);
// CG fused: p = r + beta p, w = ax_e(p)   (beta from CgScalars)
nb_status launch_ax_cg(nb_ctx *c);
// gather-scatter (gs.cu)
nb_status launch_dssum(nb_ctx *c, double *w, bool with_mask);
nb_status launch_mask(nb_ctx *c, double *w);
nb_status launch_scatter_unique(nb_ctx *c, const double *g, double *loc);
nb_status launch_tables(nb_ctx *c, int64_t *gid, int32_t *mult, uint8_t *mask);
// FP32 operator for the mixed-precision inner solve (ax_f32.cu, gs.cu)
nb_status launch_ax_f32(nb_ctx *c, const float *u, float *w, int mode);
nb_status launch_dssum32(nb_ctx *c, float *w);
// geometry (geom.cu)
nb_status host_gll(int n, double *xi, double *w);
nb_status host_dmat(int n, const double *xi, double *D);
nb_status launch_box_geometry(nb_ctx *c, double amp, const double *s, int *bad_dev);
nb_status launch_box_coords(nb_ctx *c, double *xyz);
nb_status launch_box_geometry_pairs(const Mesh &m, double amp, const double *s, const double *D,
                                    float2 *out, int *bad_dev, cudaStream_t stream);
// reductions + CG (cg.cu)
nb_status dot_c(nb_ctx *c, const double *a, const double *b, double *out_host);
nb_status dot_c_noalloc(const Mesh &m, const double *a, const double *b, double *out,
                        cudaStream_t stream);
nb_status cg_solve_fp64(nb_ctx *c, const double *f, double *x, double tol, int maxit,
                        int *iters, double *relres);
nb_status cg_solve_mixed(nb_ctx *c, const double *f, double *x, double tol, int maxit,
                         int *iters, double *relres);
nb_status ensure_cg_workspace(nb_ctx *c);
nb_status set_preconditioner(nb_ctx *c, int kind);   // precond.cu
nb_status prepare_df(nb_ctx *c);   // double-float copies of D and gxyz
bool centro_antisymmetric(const double *D, int n);
nb_status prepare_fp32(nb_ctx *c); // fp32 copy of gxyz for the mixed solve

// ---------------------------------------------------------------- device helpers
__host__ __device__ inline int mult_1d(int idx, int e, int ne, int n) {
    // copies of a node along one direction: 2 on an interior element face
    return ((idx == 0 && e > 0) || (idx == n - 1 && e < ne - 1)) ? 2 : 1;
}

__host__ __device__ inline int grid_blocks(int64_t work, int per_block, int cap) {
    int64_t b = (work + per_block - 1) / per_block;
    if (b < 1) b = 1;
    return (int)(b < cap ? b : cap);
}

}  // namespace nekgb
