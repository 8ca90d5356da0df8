// ew_stencil_dev.cuh -- device helpers shared by the stencil kernels: the
// order-2 / order-4 Laplacian read from global memory with the box closure
// applied on the fly (Dirichlet walls 0, beyond a wall the odd or even
// reflection, ew_bc_dev.cuh).
#pragma once

#include "ew_bc_dev.cuh"
#include "ew_internal.h"

namespace ew {

// ---------------------------------------------------------------------------
// global-memory stencil with the box closure
// ---------------------------------------------------------------------------
// neighbour at offset `off` along an axis with stride `stride`; `i` is the
// point's coordinate on that axis, `n` the axis length, `code` its face code.
template <typename T>
__device__ __forceinline__ T ld_axis(const T* __restrict__ u, int64_t base, int64_t stride, int64_t i,
                                     int64_t n, int off, int code) {
    const int64_t p = i + off;
    if (p >= 0 && p < n) return u[base + off * stride];
    int sg = 1;
    const int64_t q = ext_axis<int64_t>(p, n, code, sg);
    if (q < 0) return T(0);
    const T v = u[base + (q - i) * stride];
    return sg < 0 ? -v : v;
}

template <typename T, int DIM, int ORDER>
__device__ __forceinline__ T lap_global(const T* __restrict__ u, const Stencil<T>& s, int64_t base,
                                        int64_t i, int64_t j, int64_t k, int64_t nx, int64_t ny,
                                        int64_t nz) {
    const int bx = axis_bc(s.bc, 0), by = axis_bc(s.bc, 1), bz = axis_bc(s.bc, 2);
    T r = s.c0 * u[base];
    r += s.c1[0] * (ld_axis(u, base, 1, i, nx, -1, bx) + ld_axis(u, base, 1, i, nx, 1, bx));
    r += s.c1[1] * (ld_axis(u, base, nx, j, ny, -1, by) + ld_axis(u, base, nx, j, ny, 1, by));
    if (DIM == 3)
        r += s.c1[2] * (ld_axis(u, base, nx * ny, k, nz, -1, bz) + ld_axis(u, base, nx * ny, k, nz, 1, bz));
    if (ORDER == 4) {
        r += s.c2[0] * (ld_axis(u, base, 1, i, nx, -2, bx) + ld_axis(u, base, 1, i, nx, 2, bx));
        r += s.c2[1] * (ld_axis(u, base, nx, j, ny, -2, by) + ld_axis(u, base, nx, j, ny, 2, by));
        if (DIM == 3)
            r += s.c2[2] * (ld_axis(u, base, nx * ny, k, nz, -2, bz) + ld_axis(u, base, nx * ny, k, nz, 2, bz));
    }
    return r;
}

}  // namespace ew
