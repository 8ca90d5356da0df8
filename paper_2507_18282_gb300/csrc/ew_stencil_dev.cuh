// ew_stencil_dev.cuh -- device helpers shared by the stencil kernels: the
// order-2 / order-4 Laplacian read from global memory with the Dirichlet
// closure applied on the fly (boundary points 0, ghosts the odd reflection).
#pragma once

#include "ew_internal.h"

namespace ew {

// ---------------------------------------------------------------------------
// global-memory stencil with the Dirichlet closure
// ---------------------------------------------------------------------------
// neighbour at offset `off` along an axis with stride `stride`; `i` is the
// point's coordinate on that axis, `n` the axis length.
template <typename T>
__device__ __forceinline__ T ld_axis(const T* __restrict__ u, int64_t base, int64_t stride, int64_t i,
                                     int64_t n, int off) {
    int64_t p = i + off;
    if (p >= 0 && p < n) return u[base + off * stride];
    if (p == -1 || p == n) return T(0);
    int64_t q = (p < 0) ? (-2 - p) : (2 * n - p);  // odd reflection about -1 / n
    return -u[base + (q - i) * stride];
}

template <typename T, int DIM, int ORDER>
__device__ __forceinline__ T lap_global(const T* __restrict__ u, const Stencil<T>& s, int64_t base,
                                        int64_t i, int64_t j, int64_t k, int64_t nx, int64_t ny,
                                        int64_t nz) {
    T r = s.c0 * u[base];
    r += s.c1[0] * (ld_axis(u, base, 1, i, nx, -1) + ld_axis(u, base, 1, i, nx, 1));
    r += s.c1[1] * (ld_axis(u, base, nx, j, ny, -1) + ld_axis(u, base, nx, j, ny, 1));
    if (DIM == 3)
        r += s.c1[2] * (ld_axis(u, base, nx * ny, k, nz, -1) + ld_axis(u, base, nx * ny, k, nz, 1));
    if (ORDER == 4) {
        r += s.c2[0] * (ld_axis(u, base, 1, i, nx, -2) + ld_axis(u, base, 1, i, nx, 2));
        r += s.c2[1] * (ld_axis(u, base, nx, j, ny, -2) + ld_axis(u, base, nx, j, ny, 2));
        if (DIM == 3)
            r += s.c2[2] * (ld_axis(u, base, nx * ny, k, nz, -2) + ld_axis(u, base, nx * ny, k, nz, 2));
    }
    return r;
}

}  // namespace ew
