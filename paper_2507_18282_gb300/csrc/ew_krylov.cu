// ew_krylov.cu -- FP64 tall-skinny kernels of the Krylov eigen-solver (Arnoldi
// section): block Gram products C = A^T B with warp-shuffle reductions (the
// classical Gram-Schmidt coefficients, applied twice), block updates
// B <- beta B + alpha A M (the Gram-Schmidt subtraction, the thick-restart
// basis rotation V Y and the Cholesky-QR scaling), and precision conversions
// between the FP64 basis and the filter's FP32 fields.
//
// Layout: a block of vectors is column-major with leading dimension ld (each
// vector contiguous, vector j at offset j * ld).  The Gram product is
// deterministic: fixed block count, per-block partials summed in order.
#include <algorithm>

#include "ew_internal.h"

namespace ew {

constexpr int kGramTile = 4;    // 4 x 4 output entries per thread
constexpr int kGramThreads = 256;

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// part[(chunk * ma + i) * mb + j] = sum over the chunk's rows of A[r,i] B[r,j]
__global__ void __launch_bounds__(kGramThreads)
    k_gram(int64_t N, const double* __restrict__ A, int64_t lda, int ma, const double* __restrict__ B,
           int64_t ldb, int mb, double* __restrict__ part) {
    __shared__ double sh[kGramThreads / 32][kGramTile * kGramTile];
    const int i0 = blockIdx.y * kGramTile, j0 = blockIdx.z * kGramTile;
    double acc[kGramTile][kGramTile];
#pragma unroll
    for (int a = 0; a < kGramTile; ++a)
#pragma unroll
        for (int c = 0; c < kGramTile; ++c) acc[a][c] = 0.0;
    const int64_t chunk = (N + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = blockIdx.x * chunk;
    const int64_t r1 = min(N, r0 + chunk);
    for (int64_t r = r0 + threadIdx.x; r < r1; r += kGramThreads) {
        double av[kGramTile], bv[kGramTile];
#pragma unroll
        for (int a = 0; a < kGramTile; ++a) av[a] = (i0 + a < ma) ? A[(int64_t)(i0 + a) * lda + r] : 0.0;
#pragma unroll
        for (int c = 0; c < kGramTile; ++c) bv[c] = (j0 + c < mb) ? B[(int64_t)(j0 + c) * ldb + r] : 0.0;
#pragma unroll
        for (int a = 0; a < kGramTile; ++a)
#pragma unroll
            for (int c = 0; c < kGramTile; ++c) acc[a][c] = fma(av[a], bv[c], acc[a][c]);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < kGramTile; ++a)
#pragma unroll
        for (int c = 0; c < kGramTile; ++c) {
            double v = wsum(acc[a][c]);
            if (lane == 0) sh[wid][a * kGramTile + c] = v;
        }
    __syncthreads();
    if (threadIdx.x < kGramTile * kGramTile) {
        const int a = threadIdx.x / kGramTile, c = threadIdx.x % kGramTile;
        double v = 0.0;
        for (int w = 0; w < kGramThreads / 32; ++w) v += sh[w][threadIdx.x];
        if (i0 + a < ma && j0 + c < mb) part[((int64_t)blockIdx.x * ma + i0 + a) * mb + j0 + c] = v;
    }
}

// C[i * mb + j] = sum over chunks of part (fixed order)
__global__ void k_gram_finish(const double* __restrict__ part, int nchunks, int ma, int mb, double* __restrict__ C) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ma * mb) return;
    double s = 0.0;
    for (int q = 0; q < nchunks; ++q) s += part[(int64_t)q * ma * mb + e];
    C[e] = s;
}

constexpr int kGramChunks = 304;

ew_status gram(int64_t N, const double* A, int64_t lda, int ma, const double* B, int64_t ldb, int mb,
               double* part, double* C, cudaStream_t st) {
    dim3 grid(kGramChunks, (ma + kGramTile - 1) / kGramTile, (mb + kGramTile - 1) / kGramTile);
    k_gram<<<grid, kGramThreads, 0, st>>>(N, A, lda, ma, B, ldb, mb, part);
    k_gram_finish<<<(ma * mb + 127) / 128, 128, 0, st>>>(part, kGramChunks, ma, mb, C);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch(2);
    return EW_OK;
}
size_t gram_part_doubles(int ma, int mb) { return (size_t)kGramChunks * ma * mb; }

// Out[:, j] = beta * Bin[:, j] + alpha * sum_i A[:, i] M[i * mb + j], j < mb.
// Rows are staged in shared memory first, so Out may alias A or Bin (the
// in-place basis rotation V[:, :k] = V[:, :m] Y).
constexpr int kUpdRows = 32;
constexpr int kUpdThreads = 256;

__global__ void __launch_bounds__(kUpdThreads)
    k_update(int64_t N, const double* A, int64_t lda, int ma, const double* Bin, int64_t ldb, int mb,
             const double* __restrict__ M, double alpha, double beta, double* Out, int64_t ldo) {
    extern __shared__ double sm[];
    double* sA = sm;                    // kUpdRows x ma
    double* sB = sA + kUpdRows * ma;    // kUpdRows x mb
    double* sM = sB + kUpdRows * mb;    // ma x mb
    const int64_t r0 = (int64_t)blockIdx.x * kUpdRows;
    const int nr = (int)min((int64_t)kUpdRows, N - r0);
    for (int e = threadIdx.x; e < ma * mb; e += kUpdThreads) sM[e] = M[e];
    for (int e = threadIdx.x; e < kUpdRows * ma; e += kUpdThreads) {
        int i = e / kUpdRows, r = e % kUpdRows;
        sA[r * ma + i] = (r < nr) ? A[(int64_t)i * lda + r0 + r] : 0.0;
    }
    if (beta != 0.0)
        for (int e = threadIdx.x; e < kUpdRows * mb; e += kUpdThreads) {
            int j = e / kUpdRows, r = e % kUpdRows;
            sB[r * mb + j] = (r < nr) ? Bin[(int64_t)j * ldb + r0 + r] : 0.0;
        }
    __syncthreads();
    for (int e = threadIdx.x; e < kUpdRows * mb; e += kUpdThreads) {
        int j = e / kUpdRows, r = e % kUpdRows;
        if (r >= nr) continue;
        double s = 0.0;
        for (int i = 0; i < ma; ++i) s = fma(sA[r * ma + i], sM[i * mb + j], s);
        double o = alpha * s;
        if (beta != 0.0) o = fma(beta, sB[r * mb + j], o);
        Out[(int64_t)j * ldo + r0 + r] = o;
    }
}

ew_status update(int64_t N, const double* A, int64_t lda, int ma, const double* Bin, int64_t ldb, int mb,
                 const double* M, double alpha, double beta, double* Out, int64_t ldo, cudaStream_t st) {
    size_t smem = sizeof(double) * ((size_t)kUpdRows * (ma + mb) + (size_t)ma * mb);
    if (smem > 200 * 1024) return set_error(EW_EINVAL, "basis too wide for the update kernel");
    static bool attr = false;
    if (!attr) {
        EW_CUDA_TRY(cudaFuncSetAttribute(k_update, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr = true;
    }
    unsigned blocks = (unsigned)((N + kUpdRows - 1) / kUpdRows);
    k_update<<<blocks, kUpdThreads, smem, st>>>(N, A, lda, ma, Bin, ldb, mb, M, alpha, beta, Out, ldo);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch();
    return EW_OK;
}

template <typename S, typename D>
__global__ void k_convert(int64_t n, const S* __restrict__ x, D* __restrict__ y) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        y[q] = (D)x[q];
}

template <typename S, typename D>
ew_status convert(int64_t n, const S* x, D* y, cudaStream_t st) {
    int64_t b = (n + 255) / 256;
    k_convert<S, D><<<(unsigned)std::min<int64_t>(b, 152 * 32), 256, 0, st>>>(n, x, y);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch();
    return EW_OK;
}
template ew_status convert<double, float>(int64_t, const double*, float*, cudaStream_t);
template ew_status convert<float, double>(int64_t, const float*, double*, cudaStream_t);

// SplitMix64 (Steele, Lea, Flood 2014): draw i of stream `seed` mapped to
// uniform [-1, 1): 2 (z >> 11) 2^-53 - 1, z = mix(seed + (i + 1) * golden).
__global__ void k_splitmix_uniform(int64_t n, uint64_t seed, double* __restrict__ out) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (uint64_t)(q + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z = z ^ (z >> 31);
        out[q] = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
    }
}

ew_status splitmix_uniform(int64_t n, uint64_t seed, double* out, cudaStream_t st) {
    int64_t b = (n + 255) / 256;
    k_splitmix_uniform<<<(unsigned)std::min<int64_t>(b, 152 * 32), 256, 0, st>>>(n, seed, out);
    EW_CUDA_TRY(cudaGetLastError());
    count_launch();
    return EW_OK;
}

}  // namespace ew
