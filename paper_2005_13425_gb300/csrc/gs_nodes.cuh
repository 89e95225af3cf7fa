// Shared-node helpers of the structured box used by dssum: the count of
// shared nodes and the signed-zero rule of the node sums.  The enumeration
// of the nodes and their copies is in gs_fast.cuh.
#pragma once

#include "internal.cuh"

namespace nekgb {

// (+0.0) + v, computed with integer operations: -0.0 becomes +0.0.
__device__ __forceinline__ double plus_zero(double v) {
    return (__double_as_longlong(v) << 1) == 0 ? 0.0 : v;
}
__device__ __forceinline__ float plus_zero(float v) { return (__float_as_uint(v) << 1) == 0u ? 0.f : v; }

// Shared-node counts: nodes on interior x-planes; on interior y-planes off
// the x-planes; on interior z-planes off both.
__host__ __device__ inline void shared_counts(const Mesh &m, int &cx, int &cy, int &cz) {
    const int64_t NXp = m.NX - (m.ex - 1), NYp = m.NY - (m.ey - 1);
    cx = (int)((int64_t)(m.ex - 1) * m.NY * m.NZ);
    cy = (int)((int64_t)(m.ey - 1) * NXp * m.NZ);
    cz = (int)((int64_t)(m.ez - 1) * NXp * NYp);
}

}  // namespace nekgb
