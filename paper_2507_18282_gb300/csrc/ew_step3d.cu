// ew_step3d.cu -- one fused leapfrog + filter step on 3D grids, streamed
// along z (eqs. explicitScheme, filterQuadrature).
//
//   D^{n+1} = D^n + dt^2 L_h W^n (in place),  W^{n+1} = W^n + D^{n+1},  acc += c W^{n+1}
//   (D^n = W^n - W^{n-1}: the summed form of the leapfrog recurrence)
//
// A thread owns one (x, y) column of a z-chunk and marches up z, keeping the
// column's z-neighbours of W^n in a register queue (one new load per point);
// the x- and y-neighbours come through L1 from the neighbouring threads' rows.
// The box closure is folded into per-thread constants: since x and y are
// fixed for the whole march, each x/y neighbour is "offset o with sign s"
// (s = 1 inside or for an even-reflected Neumann ghost, 0 on a Dirichlet wall,
// -1 for an odd-reflected ghost), so the step has no branch.  Per point and step the
// kernel moves W^n, D^n and the filter sum in and D^{n+1}, W^{n+1} and the sum
// out: 24 B (FP32), the unblocked algorithmic traffic.
#include <algorithm>

#include "ew_bc_dev.cuh"
#include "ew_internal.h"

namespace ew {

constexpr int kS3X = 32, kS3Y = 8, kS3Z = 32;  // CTA = 32 x 8 columns, 32 planes per chunk

// neighbour of coordinate i at offset d along an axis of length n with face
// code `code`: the in-range coordinate holding its value and the sign (0: a
// Dirichlet wall, ew_bc_dev.cuh)
__device__ __forceinline__ void nb(int i, int d, int n, int code, int& j, int& s) {
    const int p = i + d;
    if (p >= 0 && p < n) {
        j = p;
        s = 1;
        return;
    }
    int sg = 1;
    const int q = ext_axis<int>(p, n, code, sg);
    j = q < 0 ? i : q;
    s = q < 0 ? 0 : sg;
}

template <typename T, int R>
__global__ void __launch_bounds__(kS3X* kS3Y)
    k_step3d(int nx, int ny, int nz, const T* __restrict__ W, T* __restrict__ D, T* __restrict__ Wout,
             T* __restrict__ acc, Stencil<T> st, T c) {
    const int x = blockIdx.x * kS3X + threadIdx.x;
    const int y = blockIdx.y * kS3Y + threadIdx.y;
    const int z0 = blockIdx.z * kS3Z;
    if (x >= nx || y >= ny || z0 >= nz) return;
    const int64_t plane = (int64_t)nx * ny;
    // x / y neighbour offsets (in elements, within a plane) and signs
    const int bx = axis_bc(st.bc, 0), by = axis_bc(st.bc, 1), bz = axis_bc(st.bc, 2);
    int jx, sx_m1, sx_p1, sx_m2 = 0, sx_p2 = 0, sy_m1, sy_p1, sy_m2 = 0, sy_p2 = 0;
    int ox_m1, ox_p1, ox_m2 = 0, ox_p2 = 0, oy_m1, oy_p1, oy_m2 = 0, oy_p2 = 0;
    nb(x, -1, nx, bx, jx, sx_m1); ox_m1 = jx - x;
    nb(x, 1, nx, bx, jx, sx_p1); ox_p1 = jx - x;
    nb(y, -1, ny, by, jx, sy_m1); oy_m1 = (jx - y) * nx;
    nb(y, 1, ny, by, jx, sy_p1); oy_p1 = (jx - y) * nx;
    if (R == 2) {
        nb(x, -2, nx, bx, jx, sx_m2); ox_m2 = jx - x;
        nb(x, 2, nx, bx, jx, sx_p2); ox_p2 = jx - x;
        nb(y, -2, ny, by, jx, sy_m2); oy_m2 = (jx - y) * nx;
        nb(y, 2, ny, by, jx, sy_p2); oy_p2 = (jx - y) * nx;
    }
    const T fx_m1 = (T)sx_m1, fx_p1 = (T)sx_p1, fy_m1 = (T)sy_m1, fy_p1 = (T)sy_p1;
    const T fx_m2 = (T)sx_m2, fx_p2 = (T)sx_p2, fy_m2 = (T)sy_m2, fy_p2 = (T)sy_p2;
    const int64_t col = (int64_t)y * nx + x;
    // z queue: q[0..2R] = W at z-R .. z+R (the closure's extension in z)
    auto zval = [&](int z) -> T {
        if (z >= 0 && z < nz) return W[(int64_t)z * plane + col];
        int sg = 1;
        const int m = ext_axis<int>(z, nz, bz, sg);
        if (m < 0) return T(0);
        const T v = W[(int64_t)m * plane + col];
        return sg < 0 ? -v : v;
    };
    T q[2 * R + 1];
#pragma unroll
    for (int k = 0; k < 2 * R + 1; ++k) q[k] = zval(z0 - R + k);
    const int z1 = min(nz, z0 + kS3Z);
    for (int z = z0; z < z1; ++z) {
        const int64_t p = (int64_t)z * plane + col;
        const T u = q[R];
        T lap = st.c0 * u + st.c1[0] * (fx_m1 * W[p + ox_m1] + fx_p1 * W[p + ox_p1]) +
                st.c1[1] * (fy_m1 * W[p + oy_m1] + fy_p1 * W[p + oy_p1]) + st.c1[2] * (q[R - 1] + q[R + 1]);
        if (R == 2)
            lap += st.c2[0] * (fx_m2 * W[p + ox_m2] + fx_p2 * W[p + ox_p2]) +
                   st.c2[1] * (fy_m2 * W[p + oy_m2] + fy_p2 * W[p + oy_p2]) + st.c2[2] * (q[0] + q[4]);
        const T d = D[p] + lap;
        const T wn = u + d;
        D[p] = d;
        Wout[p] = wn;
        acc[p] += c * wn;
#pragma unroll
        for (int k = 0; k < 2 * R; ++k) q[k] = q[k + 1];
        q[2 * R] = zval(z + R + 1);
    }
}

template <typename T>
ew_status step3d(const GridGeom& g, const T* W, T* D, T* Wout, T* acc, T c, const Stencil<T>& s, int nvec,
                 int64_t fstride, cudaStream_t st) {
    dim3 grid((unsigned)((g.n[0] + kS3X - 1) / kS3X), (unsigned)((g.n[1] + kS3Y - 1) / kS3Y),
              (unsigned)((g.n[2] + kS3Z - 1) / kS3Z));
    for (int v = 0; v < nvec; ++v) {
        cudaEvent_t ev = fused_begin(st);
        if (g.order == 2)
            k_step3d<T, 1><<<grid, dim3(kS3X, kS3Y), 0, st>>>((int)g.n[0], (int)g.n[1], (int)g.n[2], W + v * fstride,
                                                              D + v * fstride, Wout + v * fstride, acc + v * g.N, s,
                                                              c);
        else
            k_step3d<T, 2><<<grid, dim3(kS3X, kS3Y), 0, st>>>((int)g.n[0], (int)g.n[1], (int)g.n[2], W + v * fstride,
                                                              D + v * fstride, Wout + v * fstride, acc + v * g.N, s,
                                                              c);
        EW_CUDA_TRY(cudaGetLastError());
        fused_end(ev, st, g.N, g.N);
    }
    return EW_OK;
}
template ew_status step3d<float>(const GridGeom&, const float*, float*, float*, float*, float, const Stencil<float>&,
                                 int, int64_t, cudaStream_t);
template ew_status step3d<double>(const GridGeom&, const double*, double*, double*, double*, double,
                                  const Stencil<double>&, int, int64_t, cudaStream_t);

}  // namespace ew
