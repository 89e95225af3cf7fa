// Shared-node enumeration of the structured box with the polynomial order
// known at compile time and the mesh-dependent divisors replaced by exact
// multiply-high reciprocals (Granlund and Montgomery, 1994: for d >= 2,
// m = ceil(2^64 / d) gives floor(q / d) = floor(q m / 2^64) for every
// 32-bit q, because q (m d - 2^64) < 2^64).  Each node's copies are listed
// in ascending element order, the order in which dssum adds them.
#pragma once

#include "gs_nodes.cuh"
#include "internal.cuh"

namespace nekgb {

struct FastDiv {
    unsigned long long m = 0;
    unsigned d = 1;
    static FastDiv make(unsigned d) {
        FastDiv f;
        f.d = d;
        f.m = d <= 1 ? 0ull : (~0ull / d) + 1ull;
        return f;
    }
    __device__ __forceinline__ unsigned div(unsigned q) const {
        return d <= 1 ? q : (unsigned)__umul64hi((unsigned long long)q, m);
    }
};

}  // namespace nekgb

namespace nekgb {

// ---------------------------------------------------------------- by category
// The shared nodes grouped by how many coordinates lie on an interior
// element interface: face nodes (one; 2 copies), edge nodes (two; 4 copies)
// and vertices (three; 8 copies).  Within a category every node has the
// same copy count and the copies sit at fixed offsets from the first, so a
// warp runs one branch-free path.  Non-interface coordinates are counted in
// "non-plane" indices (box-boundary nodes and element-interior nodes).
struct DsCat {
    int ex, ey, ez;
    int NXp, NYp, NZp;              // non-plane coordinate counts per direction
    int o[8];                        // range starts: Fx, Fy, Fz, Exy, Exz, Eyz, V, end
    FastDiv fNXp, fNYp, fNZp, fEx1, fEy1;
};

inline DsCat make_ds_cat(const Mesh &m) {
    DsCat d;
    d.ex = m.ex; d.ey = m.ey; d.ez = m.ez;
    d.NXp = (int)(m.NX - (m.ex - 1));
    d.NYp = (int)(m.NY - (m.ey - 1));
    d.NZp = (int)(m.NZ - (m.ez - 1));
    const int64_t ax = m.ex - 1, ay = m.ey - 1, az = m.ez - 1;
    const int64_t cnt[7] = {ax * d.NYp * d.NZp, ay * d.NXp * d.NZp, az * d.NXp * d.NYp,
                            ax * ay * d.NZp,    ax * az * d.NYp,    ay * az * d.NXp,
                            ax * ay * az};
    d.o[0] = 0;
    for (int k = 0; k < 7; k++) d.o[k + 1] = d.o[k] + (int)cnt[k];
    d.fNXp = FastDiv::make((unsigned)d.NXp);
    d.fNYp = FastDiv::make((unsigned)d.NYp);
    d.fNZp = FastDiv::make((unsigned)d.NZp);
    d.fEx1 = FastDiv::make((unsigned)(ax > 0 ? ax : 1));
    d.fEy1 = FastDiv::make((unsigned)(ay > 0 ? ay : 1));
    return d;
}

// Non-plane index g (of ne (N-2) + 2) -> (element, local index) along one
// direction: 0 -> (0, 0), the last -> (ne - 1, N - 1), others are
// element-interior points.
template <int N>
__device__ __forceinline__ void nonplane_elem(int g, int ne, int &el, int &li) {
    if (g == 0) { el = 0; li = 0; return; }
    if (g == ne * (N - 2) + 1) { el = ne - 1; li = N - 1; return; }
    if constexpr (N > 2) {
        const int qq = g - 1;
        el = qq / (N - 2);
        li = 1 + qq % (N - 2);
    } else {
        el = 0; li = 0;
    }
}

__device__ __forceinline__ void divmod(unsigned q, const FastDiv &f, unsigned &quo, unsigned &rem) {
    quo = f.div(q);
    rem = q - quo * f.d;
}

// Copies of shared node q (a global enumeration over the seven ranges of
// DsCat) in ascending element order; returns the copy count (2, 4 or 8).
template <int N>
__device__ __forceinline__ int cat_copies(int q, const DsCat &d, int64_t *idx) {
    constexpr int N1 = N - 1, N2 = N * N;
    constexpr int64_t N3 = (int64_t)N * N * N;
    const int64_t sy = d.ex, sz = (int64_t)d.ex * d.ey;   // element id strides
    unsigned t, r0, r1;
    int ex, ey, ez, lx, ly, lz;
    if (q < d.o[3]) {                         // face nodes: 2 copies
        if (q < d.o[1]) {                     // x-interface a+1 between elements a and a+1
            divmod((unsigned)q, d.fNYp, t, r0);
            divmod(t, d.fNZp, t, r1);
            nonplane_elem<N>((int)r0, d.ey, ey, ly);
            nonplane_elem<N>((int)r1, d.ez, ez, lz);
            const int64_t e = (int64_t)t + sy * ey + sz * ez;
            idx[0] = e * N3 + N1 + N * ly + N2 * lz;
            idx[1] = idx[0] + N3 - N1;
        } else if (q < d.o[2]) {              // y-interface
            divmod((unsigned)(q - d.o[1]), d.fNXp, t, r0);
            divmod(t, d.fNZp, t, r1);
            nonplane_elem<N>((int)r0, d.ex, ex, lx);
            nonplane_elem<N>((int)r1, d.ez, ez, lz);
            const int64_t e = ex + sy * (int64_t)t + sz * ez;
            idx[0] = e * N3 + lx + N * N1 + N2 * lz;
            idx[1] = idx[0] + sy * N3 - N * N1;
        } else {                              // z-interface
            divmod((unsigned)(q - d.o[2]), d.fNXp, t, r0);
            divmod(t, d.fNYp, t, r1);
            nonplane_elem<N>((int)r0, d.ex, ex, lx);
            nonplane_elem<N>((int)r1, d.ey, ey, ly);
            const int64_t e = ex + sy * ey + sz * (int64_t)t;
            idx[0] = e * N3 + lx + N * ly + N2 * N1;
            idx[1] = idx[0] + sz * N3 - N2 * N1;
        }
        return 2;
    }
    if (q < d.o[6]) {                         // edge nodes: 4 copies
        int64_t e, s1, s2;
        int l0;
        if (q < d.o[4]) {                     // x- and y-interfaces, along z
            divmod((unsigned)(q - d.o[3]), d.fNZp, t, r0);
            divmod(t, d.fEx1, t, r1);         // r1 = a, t = b
            nonplane_elem<N>((int)r0, d.ez, ez, lz);
            e = (int64_t)r1 + sy * (int64_t)t + sz * ez;
            l0 = N1 + N * N1 + N2 * lz;
            s1 = 1; s2 = sy;
            idx[0] = e * N3 + l0;
            idx[1] = (e + s1) * N3 + l0 - N1;
            idx[2] = (e + s2) * N3 + l0 - N * N1;
            idx[3] = (e + s1 + s2) * N3 + l0 - N1 - N * N1;
        } else if (q < d.o[5]) {              // x- and z-interfaces, along y
            divmod((unsigned)(q - d.o[4]), d.fNYp, t, r0);
            divmod(t, d.fEx1, t, r1);         // r1 = a, t = c
            nonplane_elem<N>((int)r0, d.ey, ey, ly);
            e = (int64_t)r1 + sy * ey + sz * (int64_t)t;
            l0 = N1 + N * ly + N2 * N1;
            s1 = 1; s2 = sz;
            idx[0] = e * N3 + l0;
            idx[1] = (e + s1) * N3 + l0 - N1;
            idx[2] = (e + s2) * N3 + l0 - N2 * N1;
            idx[3] = (e + s1 + s2) * N3 + l0 - N1 - N2 * N1;
        } else {                              // y- and z-interfaces, along x
            divmod((unsigned)(q - d.o[5]), d.fNXp, t, r0);
            divmod(t, d.fEy1, t, r1);         // r1 = b, t = c
            nonplane_elem<N>((int)r0, d.ex, ex, lx);
            e = ex + sy * (int64_t)r1 + sz * (int64_t)t;
            l0 = lx + N * N1 + N2 * N1;
            s1 = sy; s2 = sz;
            idx[0] = e * N3 + l0;
            idx[1] = (e + s1) * N3 + l0 - N * N1;
            idx[2] = (e + s2) * N3 + l0 - N2 * N1;
            idx[3] = (e + s1 + s2) * N3 + l0 - N * N1 - N2 * N1;
        }
        return 4;
    }
    // vertices: 8 copies, z outer, y, x inner
    divmod((unsigned)(q - d.o[6]), d.fEx1, t, r0);   // r0 = a
    divmod(t, d.fEy1, t, r1);                          // r1 = b, t = c
    const int64_t e = (int64_t)r0 + sy * (int64_t)r1 + sz * (int64_t)t;
#pragma unroll
    for (int dz = 0; dz < 2; dz++)
#pragma unroll
        for (int dy = 0; dy < 2; dy++)
#pragma unroll
            for (int dx = 0; dx < 2; dx++)
                idx[dz * 4 + dy * 2 + dx] = (e + dx + sy * dy + sz * dz) * N3 + (dx ? 0 : N1) +
                                            N * (dy ? 0 : N1) + N2 * (dz ? 0 : N1);
    return 8;
}


// ------------------------------------------------ first copy + fixed offsets
// The same enumeration as cat_copies, one category at a time, returning only
// the first copy of node q and which of the category's three kinds it is
// (x, y or z face; the edge along z, y or x; vertices have one kind): the
// other copies sit at offsets that depend on the kind and the mesh only
// (copy_offset), so a caller keeps one index per node instead of eight.
template <int N>
__device__ __forceinline__ int64_t face_first(int q, const DsCat &d, int &kind) {
    constexpr int N1 = N - 1, N2 = N * N;
    constexpr int64_t N3 = (int64_t)N * N * N;
    const int64_t sy = d.ex, sz = (int64_t)d.ex * d.ey;
    unsigned t, r0, r1;
    int ex, ey, ez, lx, ly, lz;
    if (q < d.o[1]) {
        kind = 0;
        divmod((unsigned)q, d.fNYp, t, r0);
        divmod(t, d.fNZp, t, r1);
        nonplane_elem<N>((int)r0, d.ey, ey, ly);
        nonplane_elem<N>((int)r1, d.ez, ez, lz);
        return ((int64_t)t + sy * ey + sz * ez) * N3 + N1 + N * ly + N2 * lz;
    }
    if (q < d.o[2]) {
        kind = 1;
        divmod((unsigned)(q - d.o[1]), d.fNXp, t, r0);
        divmod(t, d.fNZp, t, r1);
        nonplane_elem<N>((int)r0, d.ex, ex, lx);
        nonplane_elem<N>((int)r1, d.ez, ez, lz);
        return (ex + sy * (int64_t)t + sz * ez) * N3 + lx + N * N1 + N2 * lz;
    }
    kind = 2;
    divmod((unsigned)(q - d.o[2]), d.fNXp, t, r0);
    divmod(t, d.fNYp, t, r1);
    nonplane_elem<N>((int)r0, d.ex, ex, lx);
    nonplane_elem<N>((int)r1, d.ey, ey, ly);
    return (ex + sy * ey + sz * (int64_t)t) * N3 + lx + N * ly + N2 * N1;
}

template <int N>
__device__ __forceinline__ int64_t edge_first(int q, const DsCat &d, int &kind) {
    constexpr int N1 = N - 1, N2 = N * N;
    constexpr int64_t N3 = (int64_t)N * N * N;
    const int64_t sy = d.ex, sz = (int64_t)d.ex * d.ey;
    unsigned t, r0, r1;
    int ex, ey, ez, lx, ly, lz;
    if (q < d.o[4]) {
        kind = 0;
        divmod((unsigned)(q - d.o[3]), d.fNZp, t, r0);
        divmod(t, d.fEx1, t, r1);
        nonplane_elem<N>((int)r0, d.ez, ez, lz);
        return ((int64_t)r1 + sy * (int64_t)t + sz * ez) * N3 + N1 + N * N1 + N2 * lz;
    }
    if (q < d.o[5]) {
        kind = 1;
        divmod((unsigned)(q - d.o[4]), d.fNYp, t, r0);
        divmod(t, d.fEx1, t, r1);
        nonplane_elem<N>((int)r0, d.ey, ey, ly);
        return ((int64_t)r1 + sy * ey + sz * (int64_t)t) * N3 + N1 + N * ly + N2 * N1;
    }
    kind = 2;
    divmod((unsigned)(q - d.o[5]), d.fNXp, t, r0);
    divmod(t, d.fEy1, t, r1);
    nonplane_elem<N>((int)r0, d.ex, ex, lx);
    return (ex + sy * (int64_t)r1 + sz * (int64_t)t) * N3 + lx + N * N1 + N2 * N1;
}

template <int N>
__device__ __forceinline__ int64_t vertex_first(int q, const DsCat &d) {
    constexpr int N1 = N - 1, N2 = N * N;
    constexpr int64_t N3 = (int64_t)N * N * N;
    const int64_t sy = d.ex, sz = (int64_t)d.ex * d.ey;
    unsigned t, r0, r1;
    divmod((unsigned)(q - d.o[6]), d.fEx1, t, r0);
    divmod(t, d.fEy1, t, r1);
    return ((int64_t)r0 + sy * (int64_t)r1 + sz * (int64_t)t) * N3 + N1 + N * N1 + N2 * N1;
}

// Offset of copy k (ascending element order, k < C) from the first copy of a
// node with C copies (2 face, 4 edge, 8 vertex) of the given kind.  The
// first copy sits at local coordinate N-1 along every interface direction,
// copy k's element is one step further along the directions k selects and
// its local coordinate there is 0.
template <int N, int C>
__device__ __forceinline__ int64_t copy_offset(int k, int kind, const DsCat &d) {
    constexpr int N1 = N - 1, N2 = N * N;
    constexpr int64_t N3 = (int64_t)N * N * N;
    const int64_t sy = d.ex, sz = (int64_t)d.ex * d.ey;
    const int64_t ox = N3 - N1, oy = sy * N3 - N * N1, oz = sz * N3 - N2 * N1;
    if constexpr (C == 2) {
        return kind == 0 ? ox : kind == 1 ? oy : oz;
    } else if constexpr (C == 4) {
        const int64_t o1 = kind == 2 ? oy : ox, o2 = kind == 0 ? oy : oz;
        return ((k & 1) ? o1 : 0) + ((k & 2) ? o2 : 0);
    } else {
        return ((k & 1) ? ox : 0) + ((k & 2) ? oy : 0) + ((k & 4) ? oz : 0);
    }
}

}  // namespace nekgb
