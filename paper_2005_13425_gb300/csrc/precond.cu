// Jacobi (diagonal) preconditioner for the CG solve.  Preconditioned CG is
// the paper's stated future work (arXiv 2005.13425, Sec. VII); the diagonal
// of the assembled operator is the cheapest preconditioner, a point the
// paper also makes about preconditioners' low computational intensity.
//
// The diagonal of the element matrix of Listing 1 at (i,j,k) only involves
// the three lines through the point (d/dr of the basis function of p is
// nonzero only on the r-line, and so on):
//   A_e(p,p) = sum_a D(a,i)^2 g_rr(a,j,k) + sum_b D(b,j)^2 g_ss(i,b,k)
//            + sum_c D(c,k)^2 g_tt(i,j,c) + 2 D(i,i) D(j,j) g_rs(p)
//            + 2 D(i,i) D(k,k) g_rt(p) + 2 D(j,j) D(k,k) g_st(p).
// The assembled diagonal is dssum of that; minv = 1/diag at free points and
// 0 at Dirichlet points.
#include "internal.cuh"
#include "reduce.cuh"

namespace nekgb {

nb_status launch_dssum_sc(nb_ctx *c, double *w, const CgScalars *sc);

__global__ void diag_e_kernel(const double *__restrict__ gxyz, const double *__restrict__ Dg, Mesh m,
                              double *__restrict__ diag) {
    const int n = m.n;
    const int64_t n3 = (int64_t)n * n * n;
    __shared__ double sD[kMaxN * kMaxN];
    for (int q = threadIdx.x; q < n * n; q += blockDim.x) sD[q] = Dg[q];
    __syncthreads();
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m.npts;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = q / n3;
        const int p = (int)(q - e * n3);
        const int i = p % n, j = (p / n) % n, k = p / (n * n);
        const double *g = gxyz + e * 6 * n3;
        double d = 0.0;
        for (int a = 0; a < n; a++) {
            const double da = sD[a * n + i], db = sD[a * n + j], dc = sD[a * n + k];
            d = fma(da * da, g[a + n * (j + n * k)], d);
            d = fma(db * db, g[3 * n3 + i + n * (a + n * k)], d);
            d = fma(dc * dc, g[5 * n3 + i + n * (j + n * a)], d);
        }
        const double dii = sD[i * n + i], djj = sD[j * n + j], dkk = sD[k * n + k];
        d = fma(2.0 * dii * djj, g[1 * n3 + p], d);
        d = fma(2.0 * dii * dkk, g[2 * n3 + p], d);
        d = fma(2.0 * djj * dkk, g[4 * n3 + p], d);
        diag[q] = d;
    }
}

__global__ void invert_masked_kernel(double *__restrict__ d, Mesh m, const uint8_t *__restrict__ mask) {
    const int n = m.n;
    const int64_t n3 = (int64_t)n * n * n;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m.npts;
         q += (int64_t)gridDim.x * blockDim.x) {
        bool fixed;
        if (mask) {
            fixed = mask[q] == 0;
        } else {
            const int64_t e = q / n3;
            const int p = (int)(q - e * n3);
            int ex, ey, ez;
            element_coords(e, m, ex, ey, ez);
            fixed = on_box_face(p % n, (p / n) % n, p / (n * n), ex, ey, ez, m);
        }
        d[q] = fixed ? 0.0 : 1.0 / d[q];
    }
}

nb_status set_preconditioner(nb_ctx *c, int kind) {
    if (kind == 0) {
        if (c->d_minv) {
            NB_CUDA(cudaStreamSynchronize(c->stream));
            cudaFree(c->d_minv);
            c->d_minv = nullptr;
            c->device_bytes -= sizeof(double) * c->m.npts;
        }
    } else {
        if (!c->d_minv) {
            cudaError_t e = dev_alloc((void **)&c->d_minv, sizeof(double) * c->m.npts);
            if (e != cudaSuccess) return cuda_fail(e, "alloc Jacobi diagonal");
            c->device_bytes += sizeof(double) * c->m.npts;
        }
        const int grid = grid_blocks(c->m.npts, 256, device_sms() * 8);
        diag_e_kernel<<<grid, 256, 0, c->stream>>>(c->d_gxyz, c->d_D, c->m, c->d_minv);
        NB_LAUNCH_CHECK("diag_e_kernel");
        nb_status s = launch_dssum_sc(c, c->d_minv, nullptr);
        if (s != NB_OK) return s;
        invert_masked_kernel<<<grid, 256, 0, c->stream>>>(c->d_minv, c->m, c->d_mask);
        NB_LAUNCH_CHECK("invert_masked_kernel");
    }
    if (c->cg_graph) {   // the captured iteration embeds the preconditioner pointer
        cudaGraphExecDestroy(c->cg_graph);
        c->cg_graph = nullptr;
    }
    return NB_OK;
}

}  // namespace nekgb
