// ew_reduce.cu -- reductions over active-point vectors (inner products of the
// power iteration, the Rayleigh quotient and the multigrid residual test,
// max-norm residuals).  Two passes with a fixed block count, so every result
// is deterministic: pass 1 reduces a grid-stride slice per block (warp
// shuffles, then shared memory), pass 2 sums the per-block partials in block
// order.  A thread's own slice accumulates in FP64 for FP64 vectors and, for
// FP32 vectors, in a pair of FP32 numbers (each product split exactly into
// two FP32 numbers, the running sum's rounding errors gathered in the second:
// about 48 significant bits, on the FP32 units, where FP64 accumulation of
// FP32 data is bound by this part's FP64 rate); the partials are summed in
// FP64.
#include "ew_bc_dev.cuh"
#include "ew_dd.cuh"
#include "ew_internal.h"

namespace ew {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <bool MAX>
__device__ __forceinline__ double block_reduce(double v, double* sh) {
    v = MAX ? warp_max(v) : warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : (MAX ? 0.0 : 0.0);
    if (wid == 0) v = MAX ? warp_max(v) : warp_sum(v);
    __syncthreads();
    return v;
}

// part[j * gridDim.x + b] = partial sum of x_j . y_j
template <typename T>
__global__ void __launch_bounds__(256) k_dots(const T* __restrict__ x, const T* __restrict__ y, int64_t N,
                                             double* __restrict__ part) {
    __shared__ double sh[32];
    const int64_t j = blockIdx.y;
    x += j * N;
    y += j * N;
    double s = 0.0;
    if constexpr (sizeof(T) == 4) {
        float hi = 0.f, lo = 0.f;
        for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
            float p, pe, t, te;
            two_prod(x[q], y[q], p, pe);  // x y = p + pe exactly
            two_sum(hi, p, t, te);        // hi + p = t + te exactly
            hi = t;
            lo = EW_DD_ADD(lo, EW_DD_ADD(te, pe));
        }
        s = (double)hi + (double)lo;
    } else {
        for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x)
            s += (double)x[q] * (double)y[q];
    }
    s = block_reduce<false>(s, sh);
    if (threadIdx.x == 0) part[j * gridDim.x + blockIdx.x] = s;
}

__global__ void k_finish_sum(const double* __restrict__ part, int nb, double* __restrict__ out) {
    __shared__ double sh[32];
    const int j = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[j * nb + b];
    s = block_reduce<false>(s, sh);
    if (threadIdx.x == 0) out[j] = s;
}

__global__ void k_finish_max(const double* __restrict__ part, int nb, double* __restrict__ out) {
    __shared__ double sh[32];
    const int j = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s = fmax(s, part[j * nb + b]);
    s = block_reduce<true>(s, sh);
    if (threadIdx.x == 0) out[j] = s;
}

template <typename T>
ew_status launch_dots(const T* x, const T* y, int64_t N, int nvec, double* part, double* out,
                      cudaStream_t st) {
    k_dots<T><<<dim3(kReduceBlocks, nvec), 256, 0, st>>>(x, y, N, part);
    k_finish_sum<<<nvec, 256, 0, st>>>(part, kReduceBlocks, out);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch(2);
    return EW_OK;
}
template ew_status launch_dots<float>(const float*, const float*, int64_t, int, double*, double*, cudaStream_t);
template ew_status launch_dots<double>(const double*, const double*, int64_t, int, double*, double*,
                                       cudaStream_t);

// residual max-norm: max |Lx + lam2 x| and max |x|; lam2 from the device
template <typename T>
__global__ void __launch_bounds__(256) k_resid_inf(const T* __restrict__ Lx, const T* __restrict__ x, int64_t N,
                                                  const double* __restrict__ lam2, double* __restrict__ part) {
    __shared__ double sh[32];
    const int64_t j = blockIdx.y;
    Lx += j * N;
    x += j * N;
    const double l2 = lam2[j];
    double r = 0.0, m = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
        double xv = (double)x[q];
        r = fmax(r, fabs((double)Lx[q] + l2 * xv));
        m = fmax(m, fabs(xv));
    }
    r = block_reduce<true>(r, sh);
    m = block_reduce<true>(m, sh);
    if (threadIdx.x == 0) {
        part[(2 * j) * gridDim.x + blockIdx.x] = r;
        part[(2 * j + 1) * gridDim.x + blockIdx.x] = m;
    }
}

template <typename T>
ew_status launch_resid_inf(const T* Lx, const T* x, int64_t N, int nvec, const double* lam2, double* part,
                           double* out_res, double* out_xinf, cudaStream_t st) {
    k_resid_inf<T><<<dim3(kReduceBlocks, nvec), 256, 0, st>>>(Lx, x, N, lam2, part);
    // part rows alternate (res, xinf); finish into a 2*nvec array then split
    k_finish_max<<<2 * nvec, 256, 0, st>>>(part, kReduceBlocks, out_res);
    (void)out_xinf;
    EW_CUDA_TRY(cudaGetLastError());
    count_launch(2);
    return EW_OK;
}
template ew_status launch_resid_inf<float>(const float*, const float*, int64_t, int, const double*, double*,
                                           double*, double*, cudaStream_t);
template ew_status launch_resid_inf<double>(const double*, const double*, int64_t, int, const double*, double*,
                                            double*, double*, cudaStream_t);

template <typename T>
__global__ void k_scale(T* __restrict__ x, int64_t N, const double* __restrict__ s) {
    const int64_t j = blockIdx.y;
    x += j * N;
    const T f = (T)s[j];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x)
        x[q] *= f;
}

template <typename T>
ew_status launch_scale(T* x, int64_t N, int nvec, const double* s, cudaStream_t st) {
    k_scale<T><<<dim3(kReduceBlocks, nvec), 256, 0, st>>>(x, N, s);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch();
    return EW_OK;
}
template ew_status launch_scale<float>(float*, int64_t, int, const double*, cudaStream_t);
template ew_status launch_scale<double>(double*, int64_t, int, const double*, cudaStream_t);

__global__ void k_axpy_f(int64_t n, float alpha, const float* __restrict__ x, float* __restrict__ y) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        y[q] += alpha * x[q];
}

ew_status axpy_f(int64_t n, float alpha, const float* x, float* y, cudaStream_t st) {
    k_axpy_f<<<kReduceBlocks * 4, 256, 0, st>>>(n, alpha, x, y);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch();
    return EW_OK;
}

// ||xnew - sign(beta) xold||_2^2 (one vector)
template <typename T>
__global__ void __launch_bounds__(256) k_diff_sign(const T* __restrict__ a, const T* __restrict__ b, int64_t N,
                                                  const double* __restrict__ beta, double* __restrict__ part) {
    __shared__ double sh[32];
    const double sg = beta[0] < 0.0 ? -1.0 : 1.0;
    double s = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
        double d = (double)a[q] - sg * (double)b[q];
        s += d * d;
    }
    s = block_reduce<false>(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <typename T>
ew_status launch_diffnorm_sign(const T* xnew, const T* xold, int64_t N, const double* beta, double* part,
                               double* out, cudaStream_t st) {
    k_diff_sign<T><<<kReduceBlocks, 256, 0, st>>>(xnew, xold, N, beta, part);
    k_finish_sum<<<1, 256, 0, st>>>(part, kReduceBlocks, out);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch(2);
    return EW_OK;
}
template ew_status launch_diffnorm_sign<float>(const float*, const float*, int64_t, const double*, double*,
                                               double*, cudaStream_t);
template ew_status launch_diffnorm_sign<double>(const double*, const double*, int64_t, const double*, double*,
                                                double*, cudaStream_t);

// out = W^{e/2} in (e = +1 or -1) for nvec vectors of N active points: W the
// trapezoid weights of the box, 1/2 for each Neumann wall coordinate of a
// point (so 1/4 on a 2D corner of two Neumann faces), 1 elsewhere.  On a grid
// with Neumann faces L_h is symmetric in the W-weighted sums (the discrete
// L_2 inner product), and W^{1/2} L_h W^{-1/2} in the plain ones.
template <typename T>
__global__ void k_wsqrt(const T* __restrict__ in, T* __restrict__ out, int64_t nx, int64_t ny, int64_t N,
                        int64_t total, int bc, T f) {
    const int bx = axis_bc(bc, 0), by = axis_bc(bc, 1), bz = axis_bc(bc, 2);
    const int64_t nz = N / (nx * ny);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q % N, i = r % nx, j = (r / nx) % ny, k = r / (nx * ny);
        T s = T(1);
        if (((bx & 1) && i == 0) || ((bx & 2) && i == nx - 1)) s *= f;
        if (((by & 1) && j == 0) || ((by & 2) && j == ny - 1)) s *= f;
        if (((bz & 1) && k == 0) || ((bz & 2) && k == nz - 1)) s *= f;
        out[q] = s * in[q];
    }
}

template <typename T>
ew_status launch_wsqrt(const GridGeom& g, const T* in, T* out, int nvec, int e, cudaStream_t st) {
    if (g.map) return mapped_wsqrt<T>(g, in, out, nvec, e, st);
    const T f = e > 0 ? T(0.70710678118654752440) : T(1.41421356237309504880);
    k_wsqrt<T><<<kReduceBlocks * 4, 256, 0, st>>>(in, out, g.n[0], g.n[1], g.N, g.N * (int64_t)nvec, g.bc, f);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch();
    return EW_OK;
}
template ew_status launch_wsqrt<float>(const GridGeom&, const float*, float*, int, int, cudaStream_t);
template ew_status launch_wsqrt<double>(const GridGeom&, const double*, double*, int, int, cudaStream_t);

}  // namespace ew
