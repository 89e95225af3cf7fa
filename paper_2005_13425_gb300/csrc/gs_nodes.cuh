// Shared-node enumeration of the structured box used by dssum: which
// global nodes have several local copies, and where those copies live.
// Used by the single-problem kernels (gs.cu) and the batched engine.
#pragma once

#include "internal.cuh"

namespace nekgb {

// Non-plane coordinate q (of NX - (Ex - 1)) -> global coordinate: 0, the
// element-interior indices, and the last node.
__device__ __forceinline__ int nonplane_coord(int q, int ne, int n, int NG) {
    if (q == 0) return 0;
    const int last = ne * (n - 2) + 1;
    if (q == last) return NG - 1;
    const int qq = q - 1;
    return (qq / (n - 2)) * (n - 1) + 1 + qq % (n - 2);
}

// Copies of global coordinate g along one direction: up to two (element,
// local index) pairs, in ascending element order.
__device__ __forceinline__ int copies_1d(int g, int ne, int n, int *el, int *li) {
    const int a = g / (n - 1);
    const int rem = g - a * (n - 1);
    if (rem == 0 && a > 0 && a < ne) {
        el[0] = a - 1; li[0] = n - 1;
        el[1] = a;     li[1] = 0;
        return 2;
    }
    const int ee = a < ne ? a : ne - 1;
    el[0] = ee;
    li[0] = g - ee * (n - 1);
    return 1;
}

// Work item q -> global node (gx, gy, gz) with more than one copy.  The set
// is enumerated as: nodes on interior x-planes; then nodes on interior
// y-planes off the x-planes; then nodes on interior z-planes off both.
__device__ __forceinline__ void shared_node(int q, const Mesh &m, int cx, int cy, int &gx, int &gy,
                                            int &gz) {
    const int n = m.n;
    const int NX = (int)m.NX, NY = (int)m.NY, NZ = (int)m.NZ;
    const int NXp = NX - (m.ex - 1), NYp = NY - (m.ey - 1);
    if (q < cx) {
        int r = q;
        gy = r % NY; r /= NY;
        gz = r % NZ; r /= NZ;
        gx = (r + 1) * (n - 1);
    } else if (q < cx + cy) {
        int r = q - cx;
        gx = nonplane_coord(r % NXp, m.ex, n, NX); r /= NXp;
        gz = r % NZ; r /= NZ;
        gy = (r + 1) * (n - 1);
    } else {
        int r = q - cx - cy;
        gx = nonplane_coord(r % NXp, m.ex, n, NX); r /= NXp;
        gy = nonplane_coord(r % NYp, m.ey, n, NY); r /= NYp;
        gz = (r + 1) * (n - 1);
    }
}

// Local indices of the copies of node (gx,gy,gz), ascending element order.
__device__ __forceinline__ int node_copies(int gx, int gy, int gz, const Mesh &m, int64_t *idx) {
    const int n = m.n;
    const int64_t n3 = (int64_t)n * n * n;
    int elx[2], lix[2], ely[2], liy[2], elz[2], liz[2];
    const int nx = copies_1d(gx, m.ex, n, elx, lix);
    const int ny = copies_1d(gy, m.ey, n, ely, liy);
    const int nz = copies_1d(gz, m.ez, n, elz, liz);
    int c = 0;
    for (int a = 0; a < nz; a++)
        for (int b = 0; b < ny; b++)
            for (int d = 0; d < nx; d++) {
                const int64_t e = elx[d] + (int64_t)m.ex * (ely[b] + (int64_t)m.ey * elz[a]);
                idx[c++] = e * n3 + lix[d] + n * (liy[b] + n * liz[a]);
            }
    return c;
}

// (+0.0) + v, computed with integer operations: -0.0 becomes +0.0.
__device__ __forceinline__ double plus_zero(double v) {
    return (__double_as_longlong(v) << 1) == 0 ? 0.0 : v;
}
__device__ __forceinline__ float plus_zero(float v) { return (__float_as_uint(v) << 1) == 0u ? 0.f : v; }

// dot += s * 2^-lg * ps (the node's w times the sum of its p copies, each
// weighted by 1/multiplicity = 2^-lg); the power-of-two scaling is exact.
__device__ __forceinline__ double node_dot(double dot, double s, int lg, double ps) {
    const double cinv = lg == 1 ? 0.5 : (lg == 2 ? 0.25 : 0.125);
    return fma(s * cinv, ps, dot);
}
__device__ __forceinline__ double node_dot(double dot, float s, int lg, double ps) {
    return node_dot(dot, (double)s, lg, ps);
}


// Shared-node counts: nodes on interior x-planes; on interior y-planes off
// the x-planes; on interior z-planes off both.
__host__ __device__ inline void shared_counts(const Mesh &m, int &cx, int &cy, int &cz) {
    const int64_t NXp = m.NX - (m.ex - 1), NYp = m.NY - (m.ey - 1);
    cx = (int)((int64_t)(m.ex - 1) * m.NY * m.NZ);
    cy = (int)((int64_t)(m.ey - 1) * NXp * m.NZ);
    cz = (int)((int64_t)(m.ez - 1) * NXp * NYp);
}

}  // namespace nekgb
