/*
 * nekgb.h -- C ABI of the GB300-native Nekbone hot path.
 *
 * The library evaluates the spectral-element Poisson operator of Nekbone
 * (Karp et al., "Optimization of Tensor-product Operations in Nekbone on
 * GPUs", arXiv 2005.13425) on one NVIDIA GB300 (sm_103a):
 *
 *   Ax = mask( dssum( ax_e(u) ) )
 *
 * where ax_e is the element-local tensor-product operator of Listing 1
 * (Sec. III), dssum is the direct-stiffness summation that "communicates
 * the local results to the neighbouring elements" (Sec. III, second step of
 * Ax), and the mask applies homogeneous Dirichlet conditions (Sec. VI.B).
 * nb_cg_solve runs the unpreconditioned conjugate-gradient solve of
 * Ax = f (Sec. III; no preconditioner, Sec. VII) with all vector updates
 * and reductions on the device.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Mesh: a structured box of Ex x Ey x Ez hexahedral elements covering the
 *   unit cube, element id e = ex + Ex*(ey + Ey*ez).
 * n: GLL points per direction (n = polynomial degree + 1), 2 <= n <= 16.
 * Local storage ("[E][n^3]"): a field holds one double per local point,
 *   u[e*n^3 + i + n*(j + n*k)], i fastest, exactly Listing 1's u(i,j,k,e).
 *   Points shared by several elements are stored once per element.
 * Global node of (e; i,j,k): (gx,gy,gz) = (ex(n-1)+i, ey(n-1)+j, ez(n-1)+k),
 *   gid = gx + NX*(gy + NY*gz), NX = Ex(n-1)+1, NY = Ey(n-1)+1,
 *   NZ = Ez(n-1)+1.
 * D: row major, D[i*n + l] = dxm1(i,l) = derivative of the l-th Lagrange
 *   basis polynomial at GLL node i (Listing 1's dxm1; dxtm1 = D^T).
 * gxyz: [E][6][n^3], components rr, rs, rt, ss, st, tt, i.e. Listing 1's
 *   gxyz(i,j,k,1..6,e) = w_i w_j w_k |J| (J^-1 J^-T).
 * Device pointers ("_dev") are CUDA device addresses of doubles (8-byte
 *   aligned, contiguous, local storage), owned by the caller; the library
 *   never frees them.  Host pointers ("_host") are plain host memory.
 * Streams: every call is enqueued on the stream given to nb_setup* and is
 *   asynchronous unless stated otherwise.  Inputs and outputs may not alias
 *   unless stated.
 * Errors: every entry point returns an nb_status; nothing is thrown or
 *   aborted across the ABI.  Argument checks happen before any work.  A
 *   thread-local message for the last failure is available from
 *   nb_last_error().  CUDA failures map to NB_ERR_CUDA, failed
 *   allocations to NB_ERR_OOM.
 */
#ifndef NEKGB_H
#define NEKGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nb_ctx nb_ctx; /* opaque; owns all device-side mesh state */

typedef enum {
    NB_OK = 0,
    NB_ERR_ARG = 1,           /* bad argument: size, pointer, alignment */
    NB_ERR_CUDA = 2,          /* a CUDA runtime call or launch failed */
    NB_ERR_OOM = 3,           /* device or pinned-host allocation failed */
    NB_ERR_NOT_CONVERGED = 4, /* tol > 0 and maxit reached first */
    NB_ERR_BREAKDOWN = 5,     /* CG breakdown: <Ap,p>_c <= 0 or not finite */
    NB_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
    NB_ERR_STATE = 7          /* call not valid in the context's state */
} nb_status;

typedef enum {
    NB_FP64 = 0,  /* FP64-accurate everywhere */
    NB_MIXED = 1  /* FP32 inner operator inside FP64 defect correction */
} nb_precision;

typedef struct {
    int ex, ey, ez; /* elements per direction; E = ex*ey*ez */
} nb_box;

typedef struct {
    int ex, ey, ez, n;
    int64_t nelt;      /* E */
    int64_t npts;      /* E * n^3 local points */
    int64_t nunique;   /* NX * NY * NZ unique nodes */
    int precision;     /* nb_precision */
    int ax_variant;    /* kernel used by nb_ax (see nb_set_ax_variant) */
    size_t device_bytes; /* device memory owned by the context */
} nb_info;

/* --------------------------------------------------------------------- */
/* Set-up and tear-down                                                  */
/* --------------------------------------------------------------------- */

/* Environment switches (all optional; the first two and the test switches
 * below are read when a context or an engine is set up):
 *   NEKGB_F32_STAGED=0        FP32 heads without bulk-copy staging.
 *   NEKGB_TUNE_CACHE=<file>   the engine's autotuner cache (see the engine).
 *   NEKGB_FAIL_ALLOC=<k>      tests: the k-th device allocation of the
 *       process fails (host-side fault injection).
 *   NEKGB_TEST_UNARMED_WAIT_NS=<ns>  tests: each CTA's first wait in the
 *       staged FP32 head uses a barrier that nothing arrives on, with this
 *       limit, so the solve ends with NB_ERR_TIMEOUT (bounded-wait path).
 *   NEKGB_TEST_DOT_SHIFT=<k>  tests: shifts the scale of the FP64 head's
 *       exact <w,p>_c sum by 2^k, to exercise its range check
 *       (NB_ERR_BREAKDOWN). */

/* Build a context for the box `mesh` with n GLL points per direction from
 * caller-supplied operator data (the inputs of Listing 1).
 *   D     host, n*n doubles, D[i*n+l] = dxm1(i,l).
 *   gxyz  host, E*6*n^3 doubles, [E][6][n^3] (rr,rs,rt,ss,st,tt).
 *   mask  host, E*n^3 bytes, 1 = keep, 0 = Dirichlet (set to +0.0); NULL
 *         selects homogeneous Dirichlet on all six faces of the box.
 *   prec  NB_FP64 or NB_MIXED.
 *   cuda_stream  cudaStream_t to enqueue all work on (NULL = default).
 * The context copies D, gxyz and mask to the device; the caller keeps
 * ownership of its arrays.  On failure *out is NULL and nothing leaks. */
nb_status nb_setup(nb_ctx **out, nb_box mesh, int n, const double *D,
                   const double *gxyz, const uint8_t *mask, nb_precision prec,
                   void *cuda_stream);

/* Build the synthetic Nekbone box problem on the device: GLL nodes and
 * weights, D, and gxyz for the unit cube perturbed by
 *   x_d = X_d + amp * s[d] * sin(pi X) sin(pi Y) sin(pi Z),  d = 0,1,2
 * (the perturbation vanishes on the boundary, so the box mask applies).
 * s: host, 3 doubles.  Fails with NB_ERR_ARG if the map folds (|J| <= 0). */
nb_status nb_setup_box(nb_ctx **out, nb_box mesh, int n, double amp,
                       const double *s, nb_precision prec, void *cuda_stream);

/* Free every device resource of the context (synchronises its stream).
 * NULL is accepted. */
nb_status nb_destroy(nb_ctx *ctx);

nb_status nb_get_info(const nb_ctx *ctx, nb_info *info);

/* --------------------------------------------------------------------- */
/* Operator pieces (Sec. III: Ax computed in two steps)                   */
/* --------------------------------------------------------------------- */

/* w = ax_e(u) element by element (Listing 1), no dssum, no mask.
 * u_dev, w_dev: device, E*n^3 doubles, must not overlap. */
nb_status nb_ax(nb_ctx *ctx, const double *u_dev, double *w_dev);

/* In place: each global node's value becomes the sum of its local copies,
 * added from +0.0 in ascending element order, written back to every copy
 * (direct stiffness summation, Sec. III).  Bit-for-bit deterministic. */
nb_status nb_dssum(nb_ctx *ctx, double *w_dev);

/* In place: w := +0.0 at Dirichlet points (a select, not a product). */
nb_status nb_mask(nb_ctx *ctx, double *w_dev);

/* w = mask(dssum(ax_e(u))): the assembled operator. */
nb_status nb_apply(nb_ctx *ctx, const double *u_dev, double *w_dev);

/* --------------------------------------------------------------------- */
/* Conjugate gradient (Sec. III; 100 fixed iterations in Sec. V)          */
/* --------------------------------------------------------------------- */

/* Solve A x = f by unpreconditioned CG with the weighted inner product
 * <a,b>_c = sum_local a*b/multiplicity (the unique-node dot product):
 *   r = f - A x0, p = 0, rho = <r,r>_c
 *   repeat: stop if rho == 0 or (tol > 0 and sqrt(rho/<f,f>_c) <= tol)
 *           beta = rho/rho_old (0 first), p = r + beta p, w = A p,
 *           alpha = rho/<w,p>_c, x += alpha p, r -= alpha w
 * f_dev: device, E*n^3, continuous and masked.  x_dev: device, in: initial
 * guess, out: solution.  tol <= 0 runs exactly maxit iterations (the
 * paper's fixed-iteration mode).  iters_out/relres_out (host, optional)
 * receive the iterations done and sqrt(<r,r>_c/<f,f>_c).  Blocks until the
 * solve is finished.  Returns NB_ERR_NOT_CONVERGED if tol > 0 was not
 * reached within maxit, NB_ERR_BREAKDOWN if <w,p>_c <= 0 or not finite
 * (x then holds the last good iterate).  Results are bit-for-bit
 * reproducible: every reduction has a fixed order or is exact (the FP64
 * head's <w,p>_c is an exact fixed-point sum, so its dynamic element
 * schedule does not change it).  For NB_MIXED contexts this runs
 * FP64 defect correction around an FP32 inner CG (nb_set_mixed_params):
 * maxit bounds the total inner iterations, *iters_out receives them, and
 * relres is the FP64 residual sqrt(<r,r>_c/<f,f>_c) of the returned x; the
 * mixed solve needs the box mask (NB_ERR_STATE with a mask array). */
nb_status nb_cg_solve(nb_ctx *ctx, const double *f_dev, double *x_dev,
                      double tol, int maxit, int *iters_out, double *relres_out);

/* The same solve from host buffers: f_host is copied to the device, x_host
 * (initial guess in, solution out) is copied both ways.  Plain or pinned
 * host memory; E*n^3 doubles each. */
nb_status nb_cg_solve_host(nb_ctx *ctx, const double *f_host, double *x_host,
                           double tol, int maxit, int *iters_out,
                           double *relres_out);

/* <r_k,r_k>_c of the last FP64 solve, k = 0..iters (host copy).
 * Writes min(cap, iters+1) values, *count = iters + 1. */
nb_status nb_cg_history(nb_ctx *ctx, double *rho_host, int cap, int *count);

/* --------------------------------------------------------------------- */
/* Helpers used by the solver, exposed for tests and applications        */
/* --------------------------------------------------------------------- */

/* *out_host = <a,b>_c (deterministic; blocks until done). */
nb_status nb_dot_c(nb_ctx *ctx, const double *a_dev, const double *b_dev,
                   double *out_host);

/* Allocation-free weighted dot product (the paper has no counterpart).  It
 * exists for callers that cannot call cudaMalloc: code whose device memory
 * is all owned by another allocator or a fixed pool (a framework's caching
 * allocator, an application that reserves the GPU's memory up front), and
 * code on a latency path that must not block (cudaMalloc and cudaFree can
 * synchronise the device).  *out_dev (device, 1 double) = <a,b>_c on the
 * box `mesh` with n points per direction, as nb_dot_c computes it, without
 * a context and without allocating: its scratch is a fixed device array in
 * the library (one partial per element, at most 32768 elements; larger
 * meshes return NB_ERR_ARG before any work).  Asynchronous on cuda_stream.
 * The first call on a device looks up the array's address
 * (cudaGetSymbolAddress), so make that first call before any stream
 * capture.  All calls share the one array, which keeps the last call's
 * contents (the reduction ticket is cleared on every call): calls that
 * overlap on the GPU (for example on two streams) race and give wrong
 * results. */
nb_status nb_dot_c_noalloc(nb_box mesh, int n, const double *a_dev,
                           const double *b_dev, double *out_dev,
                           void *cuda_stream);

/* local_dev[e][p] = g_dev[gid(e,p)]: copy a field given per unique node
 * (NX*NY*NZ doubles, x fastest) to every local copy. */
nb_status nb_scatter_unique(nb_ctx *ctx, const double *g_dev, double *local_dev);

/* Index work of dssum and mask, for bit-exact checks: any pointer may be
 * NULL.  gid_dev: int64 [E][n^3]; mult_dev: int32 [E][n^3] (copies of the
 * point's node); mask_dev: uint8 [E][n^3] (the mask in force). */
nb_status nb_tables(nb_ctx *ctx, int64_t *gid_dev, int32_t *mult_dev,
                    uint8_t *mask_dev);

/* Copy out the operator data the context holds: D_host (n*n) and/or
 * gxyz_dev (device, [E][6][n^3]).  Either may be NULL. */
nb_status nb_get_operator(nb_ctx *ctx, double *D_host, double *gxyz_dev);

/* Nodal coordinates of an nb_setup_box context: xyz_dev (device,
 * [E][3][n^3] doubles: x, y, z per element) receives the perturbed box map
 * at the GLL nodes.  NB_ERR_STATE for contexts built by nb_setup. */
nb_status nb_box_coords(nb_ctx *ctx, double *xyz_dev);

/* FP32 operator of the mixed-precision inner solve (NB_MIXED contexts):
 * w = ax_e(u) with FP32 u, w and gxyz (Listing 1 in single precision).
 * u_dev, w_dev: device, E*n^3 floats, local storage, must not overlap.
 * NB_ERR_STATE for an NB_FP64 context. */
nb_status nb_ax_f32(nb_ctx *ctx, const float *u_dev, float *w_dev);

/* In-place FP32 dssum (sums in FP32, ascending element order). */
nb_status nb_dssum_f32(nb_ctx *ctx, float *w_dev);

/* Mixed-precision defect correction (NB_MIXED): the inner FP32 CG stops at
 * relative residual inner_tol (default 1e-4, 0 < inner_tol < 1); at most
 * max_outer FP64 corrections (default 50).  The outer residual, every dot
 * product and norm, and the update x += d are FP64. */
nb_status nb_set_mixed_params(nb_ctx *ctx, double inner_tol, int max_outer);

/* Preconditioner of nb_cg_solve for NB_FP64 contexts: 0 = none (the
 * paper's plain CG), 1 = Jacobi, the inverse of the assembled diagonal of A
 * (computed on the device from D and gxyz, 0 at Dirichlet points).  With
 * Jacobi the solve is PCG with z = minv r: rho = <r,z>_c drives beta and
 * alpha, while the stopping test, relres and the history use <r,r>_c.
 * Preconditioned CG is the paper's stated future work (Sec. VII). */
nb_status nb_set_preconditioner(nb_ctx *ctx, int kind);

/* Copy the Jacobi inverse diagonal (device, E*n^3 doubles). */
nb_status nb_jacobi_diagonal(nb_ctx *ctx, double *minv_dev);

/* Iterations of the last solve: for NB_FP64 CG iterations; for NB_MIXED
 * the total inner iterations and the number of outer corrections. */
nb_status nb_solve_stats(const nb_ctx *ctx, int *iters, int *outer);

/* Select the ax_e kernel: 0 = automatic (fastest FP64-accurate kernel),
 * 1 = native FP64 layer kernel, 2 = double-float (FP32-pair) kernel.  All
 * variants meet the same accuracy contract. */
nb_status nb_set_ax_variant(nb_ctx *ctx, int variant);

/* --------------------------------------------------------------------- */
/* Batched and served solves (the paper's small-problem limit, Sec. VI.B  */
/* and VII: many small box problems share the GPU)                        */
/* --------------------------------------------------------------------- */

typedef struct nb_engine nb_engine;  /* opaque; owns a device arena */

/* One solve request: the synthetic box problem of nb_setup_box (mesh, n,
 * perturbation amp * s[d]) with right-hand side f, solved from x0 = 0 to
 * relative residual tol.
 *   prec = NB_FP64: FP64-accurate CG; tol <= 0 runs exactly maxit
 *     iterations.
 *   prec = NB_MIXED: defect correction around an FP32 inner CG (as
 *     nb_cg_solve on an NB_MIXED context): the FP64 residual f - A x decides
 *     convergence; each inner solve runs to relative residual inner_tol
 *     (<= 0: 1e-4); maxit bounds the inner iterations in total; at most 50
 *     outer corrections.
 * Zero-initialise the struct: prec = 0 is NB_FP64. */
typedef struct {
    nb_box mesh;
    int n;
    double amp;
    double s[3];
    double tol;
    int maxit;
    nb_precision prec;
    double inner_tol;
} nb_request;

/* Create an engine with a device arena of arena_bytes (>= 1 MiB) on
 * cuda_stream.  Every admitted request lives in the arena. */
nb_status nb_engine_create(nb_engine **out, size_t arena_bytes, void *cuda_stream);
nb_status nb_engine_destroy(nb_engine *eng);

/* Bytes of arena a request of this mesh, n and precision needs, the
 * admission criterion.  NB_FP64: gxyz pairs (48 B/point), four FP64 CG
 * vectors and reduction partials.  NB_MIXED: gxyz pairs and FP32 gxyz
 * (72 B/point), three FP64 vectors (f, w, x), four FP32 vectors and
 * partials. */
nb_status nb_engine_footprint(nb_box mesh, int n, nb_precision prec, size_t *bytes);

/* Admit a request: builds its geometry in the arena, copies f (device,
 * E*n^3 doubles, local storage; continuous and masked) and starts its solve.
 * *id_out receives the request id.  NB_ERR_OOM when the footprint does not
 * fit in the free arena (or all 1024 request slots are in use): the caller
 * retries after retiring finished requests.  The first request of a given n
 * runs the autotuner (a few ms) unless NEKGB_TUNE_CACHE names a file that
 * already holds the choice.  Blocks until the request is set up. */
nb_status nb_engine_submit(nb_engine *eng, const nb_request *req, const double *f_dev,
                           int *id_out);

/* As nb_engine_submit with the right-hand side given per unique node:
 * fu_dev (device, NX*NY*NZ doubles, x fastest) is copied to every local copy
 * and zeroed on the faces of the box. */
nb_status nb_engine_submit_unique(nb_engine *eng, const nb_request *req, const double *fu_dev,
                                  int *id_out);

/* Advance every active request by `iters` CG iterations (rounded up to a
 * multiple of 8; for NB_MIXED requests, inner iterations): per iteration,
 * one launch per kernel and per distinct (n, precision) covers all active
 * requests of that kind; the iterations are replayed from a captured CUDA
 * graph.  Each group of 8 starts with the outer pass of the NB_MIXED
 * requests whose inner solve ended.  Finished requests are skipped.  Blocks
 * until done. */
nb_status nb_engine_step(nb_engine *eng, int iters);

/* State of a request after the last step: *done = 1 once it converged, hit
 * maxit or broke down; iterations, relative residual sqrt(<r,r>_c/<f,f>_c)
 * and the solve status (NB_OK, NB_ERR_NOT_CONVERGED, NB_ERR_BREAKDOWN). */
nb_status nb_engine_poll(nb_engine *eng, int id, int *done, int *iters, double *relres,
                         int *status);

/* Precision of a request and, for NB_MIXED, the outer corrections so far
 * (the count of FP64 residual passes that started an inner solve). */
nb_status nb_engine_request_info(nb_engine *eng, int id, int *prec, int *outer);

/* Copy the request's solution to x_dev (device, E*n^3 doubles; NULL to
 * drop it) and free its slot and arena space.  Blocks until done. */
nb_status nb_engine_retire(nb_engine *eng, int id, double *x_dev);

/* Arena bytes in use, arena capacity and active requests. */
nb_status nb_engine_stats(const nb_engine *eng, size_t *used, size_t *capacity, int *active);

/* The autotuner's choice for (n, precision): line tasks per thread of the
 * CG head (1 for NB_MIXED, whose FP32 head has one layout) and elements per
 * tile (0 if that (n, precision) has not been used yet). */
nb_status nb_engine_tuning(const nb_engine *eng, int n, nb_precision prec, int *lines_per_thread,
                           int *elems_per_tile);

/* --------------------------------------------------------------------- */
/* Kernel timing (CUDA events recorded on the context's stream)           */
/* --------------------------------------------------------------------- */

typedef enum {
    NB_K_AX = 0,      /* ax_e (alone or fused with the CG p update) */
    NB_K_DSSUM = 1,   /* dssum (+ mask in the solver) */
    NB_K_MASK = 2,
    NB_K_DOT = 3,     /* weighted dot products and their finalisation */
    NB_K_UPDATE = 4,  /* CG r update + <r,r>_c (in the two-kernel iteration
                         fused with dssum) */
    NB_K_OTHER = 5,
    NB_K_COUNT = 6
} nb_kernel_id;

/* on = 1: record an event pair around every kernel launch (CUDA graphs
 * are not used while timing is on).  on = 2 (sampled): the same, except in
 * the FP64 CG solve, which keeps its CUDA graphs and runs the first
 * iteration of every chunk of 16 as event-timed plain launches and the other
 * 15 as a graph, so that timing barely changes the solve's own speed.
 * on = 0: off.  Each call resets the accumulated times and the launch count
 * (nb_launch_count).  NB_ERR_ARG for other values of on. */
nb_status nb_timing_enable(nb_ctx *ctx, int on);

/* Kernels of the library launched on the context's stream since timing was
 * last enabled or disabled (nb_timing_enable), timed or not; a graph launch
 * counts the kernels the graph holds. */
nb_status nb_launch_count(nb_ctx *ctx, int64_t *launched);

/* Accumulated device time (ms) and launch count per kernel class since
 * timing was enabled or last reset (synchronises the stream). */
nb_status nb_timing_read(nb_ctx *ctx, int kernel_id, double *ms_total,
                         int64_t *launches, int reset);

/* --------------------------------------------------------------------- */
/* Partitioned box: slabs of element layers along z                       */
/* --------------------------------------------------------------------- */
/* Nekbone distributes elements over processes (Sec. I-II); the second step
 * of Ax sums element results into the shared nodes (Sec. III), which across
 * a partition is an exchange between neighbouring slabs.  A slab context
 * holds the element layers z0 .. z1-1 of the global box `global` (geometry
 * built on the device at the global coordinates, the Dirichlet mask of the
 * global boundary, FP64-accurate).  nb_ax, nb_dssum (slab-local) and
 * nb_mask work on it; nb_apply, nb_dot_c and the CG solves return
 * NB_ERR_STATE (they need the neighbours' copies).  The assembled operator
 * of the whole box, bit for bit equal to the single-box dssum, is
 *   w = ax(p) on every slab;
 *   nb_slab_top_partial(w, up)         -> send up[] to the slab above;
 *   nb_slab_add_bottom(w, from_below)  (slabs with a slab below);
 *   nb_dssum(w);
 *   nb_slab_bottom_value(w, down)      -> send down[] to the slab below;
 *   nb_slab_set_top(w, from_above)     (slabs with a slab above);
 *   nb_mask(w).
 * Plane buffers are device arrays of plane_nodes = (ex(n-1)+1)(ey(n-1)+1)
 * doubles (x fastest).  All calls are asynchronous on the context's stream
 * except nb_slab_dot.  Errors: NB_ERR_ARG (sizes, NULL or misaligned
 * pointers), NB_ERR_STATE (not a slab context), NB_ERR_CUDA. */
nb_status nb_setup_slab(nb_ctx **out, nb_box global, int z0, int z1, int n,
                        double amp, const double *s, void *cuda_stream);
/* Plane size and whether the slab has neighbours below (z0 > 0) and above. */
nb_status nb_slab_info(nb_ctx *ctx, int64_t *plane_nodes, int *has_below,
                       int *has_above);
/* buf[node] = the slab's copies of each top-plane node summed from +0.0 in
 * ascending element order (w as ax_e left it, before any dssum). */
nb_status nb_slab_top_partial(nb_ctx *ctx, const double *w_dev, double *buf_dev);
/* The first (lowest element) copy of each bottom-plane node += buf[node]:
 * the sum continues from the slab below's partial. */
nb_status nb_slab_add_bottom(nb_ctx *ctx, double *w_dev, const double *buf_dev);
/* buf[node] = the assembled value of each bottom-plane node (after nb_dssum). */
nb_status nb_slab_bottom_value(nb_ctx *ctx, const double *w_dev, double *buf_dev);
/* Every copy of each top-plane node := buf[node] (the value from above). */
nb_status nb_slab_set_top(nb_ctx *ctx, double *w_dev, const double *buf_dev);
/* *out_host = the slab's share of <a,b>_c with the global multiplicities
 * (the shares of all slabs add up to the whole box's <a,b>_c).  Blocks. */
nb_status nb_slab_dot(nb_ctx *ctx, const double *a_dev, const double *b_dev,
                      double *out_host);
/* y = alpha x + beta y over the context's local points (any context);
 * beta = 0 does not read y. */
nb_status nb_axpby(nb_ctx *ctx, double alpha, const double *x_dev, double beta,
                   double *y_dev);

/* Measured FP32 instruction rate of the current device (FFMA per second,
 * all SMs, 16 independent chains per thread, best of 5 timed runs after a
 * warm-up; about 30 ms).  The paper has no counterpart: its roofline is
 * bandwidth-only (Sec. V, Eq. 2).  This is the ceiling of the double-float
 * ax_e, whose work is FP32 instructions.  Allocates and frees a small
 * scratch buffer and a private stream; synchronous. */
nb_status nb_fp32_rate(double *ffma_per_s);

/* Measurement probe (not used by the solvers): the forward half of ax_e
 * (Listing 1, Sec. III), w_e = D_r u_e + D_s u_e + D_t u_e for every
 * element of the context, in FP64-level accuracy, computed by
 *   method 0: the CG head's double-float even-odd line products on the
 *             FP32 pipes;
 *   method 1: the tensor cores (tcgen05 kind::f16, FP32 accumulation in
 *             tensor memory) on an error-free split of u and D into six
 *             balanced base-512 digits each (Ozaki et al. 2012), one chain
 *             of n/2 MMAs (M = 128 lines, N = K = 8n) per direction and
 *             element, the exact class sums recombined into float pairs;
 *             the three directions one after another;
 *   method 2: as method 1 with the three directions' MMAs issued together
 *             (three operand buffers and accumulators per CTA).
 * u_dev, w_dev: [E][n^3] FP64 on the device (r fastest); umax: an upper
 * bound on max|u| (> 0).  n must be 8 or 10 and method 0, 1 or 2 (NB_ERR_ARG
 * otherwise).  The
 * kernel is timed as NB_K_AX when timing is on.  Allocates and frees a
 * 13 KB digit image and a status word; synchronous.  NB_ERR_TIMEOUT if an
 * MMA did not complete within about 1 s (its CTA then frees its tensor
 * memory and stops). */
nb_status nb_probe_grad(nb_ctx *ctx, int method, const double *u_dev, double *w_dev,
                        double umax);

/* --------------------------------------------------------------------- */
/* Status                                                                */
/* --------------------------------------------------------------------- */
const char *nb_status_str(nb_status s);
const char *nb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NEKGB_H */
