// k_gemm.cu -- CUDA-core GEMM (FP64 / FP32) for the plain forms of the factored contraction.
// C[M x N] = alpha op(A) op(B) + beta C, row-major.  64x64 output tile per 256-thread block,
// each thread a 4x4 register micro-tile, K staged through shared memory in steps of 16.
#include "lrtei_internal.h"

namespace lrtei {

template <typename T, bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm(int64_t M, int64_t N, int64_t K, T alpha, const T* __restrict__ A,
                                              int64_t lda, const T* __restrict__ B, int64_t ldb, T beta,
                                              T* __restrict__ C, int64_t ldc) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int64_t k0 = 0; k0 < K; k0 += BK) {
    // A tile: BM x BK  (op(A)(i, k))
    for (int t = threadIdx.x; t < BM * BK; t += 256) {
      int i, k;
      if (TA) { i = t % BM; k = t / BM; } else { k = t % BK; i = t / BK; }
      const int64_t gi = m0 + i, gk = k0 + k;
      T v = T(0);
      if (gi < M && gk < K) v = TA ? A[gk * lda + gi] : A[gi * lda + gk];
      As[k][i] = v;
    }
    // B tile: BK x BN  (op(B)(k, j))
    for (int t = threadIdx.x; t < BK * BN; t += 256) {
      int j, k;
      if (TB) { k = t % BK; j = t / BK; } else { j = t % BN; k = t / BN; }
      const int64_t gj = n0 + j, gk = k0 + k;
      T v = T(0);
      if (gj < N && gk < K) v = TB ? B[gj * ldb + gk] : B[gk * ldb + gj];
      Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gi = m0 + ty * 4 + i;
    if (gi >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gj = n0 + tx * 4 + j;
      if (gj >= N) continue;
      T v = alpha * acc[i][j];
      if (beta != T(0)) v += beta * C[gi * ldc + gj];
      C[gi * ldc + gj] = v;
    }
  }
}

template <typename T>
void gemm_cuda_core(bool transA, bool transB, int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t lda,
                    const T* B, int64_t ldb, T beta, T* C, int64_t ldc, cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  // grid.y is limited to 65535 tiles: split M if needed
  const int64_t maxM = 65535LL * 64;
  for (int64_t mo = 0; mo < M; mo += maxM) {
    const int64_t Mc = (M - mo) < maxM ? (M - mo) : maxM;
    dim3 grid((unsigned)((N + 63) / 64), (unsigned)((Mc + 63) / 64));
    const T* Ao = transA ? A + mo : A + mo * lda;
    T* Co = C + mo * ldc;
    count_launch();
    if (!transA && !transB) k_gemm<T, false, false><<<grid, 256, 0, st>>>(Mc, N, K, alpha, Ao, lda, B, ldb, beta, Co, ldc);
    else if (transA && !transB) k_gemm<T, true, false><<<grid, 256, 0, st>>>(Mc, N, K, alpha, Ao, lda, B, ldb, beta, Co, ldc);
    else if (!transA && transB) k_gemm<T, false, true><<<grid, 256, 0, st>>>(Mc, N, K, alpha, Ao, lda, B, ldb, beta, Co, ldc);
    else k_gemm<T, true, true><<<grid, 256, 0, st>>>(Mc, N, K, alpha, Ao, lda, B, ldb, beta, Co, ldc);
  }
}
template void gemm_cuda_core<double>(bool, bool, int64_t, int64_t, int64_t, double, const double*, int64_t,
                                     const double*, int64_t, double, double*, int64_t, cudaStream_t);
template void gemm_cuda_core<float>(bool, bool, int64_t, int64_t, int64_t, float, const float*, int64_t, const float*,
                                    int64_t, float, float*, int64_t, cudaStream_t);

__global__ void k_f64_to_f32(const double* in, float* out, int64_t count) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = (float)in[t];
}
__global__ void k_f32_to_f64(const float* in, double* out, int64_t count) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = (double)in[t];
}
void convert_f64_to_f32(const double* in, float* out, int64_t count, cudaStream_t st) {
  int64_t b = (count + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (count > 0) count_launch();
  if (count > 0) k_f64_to_f32<<<(unsigned)b, 256, 0, st>>>(in, out, count);
}
void convert_f32_to_f64(const float* in, double* out, int64_t count, cudaStream_t st) {
  int64_t b = (count + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (count > 0) count_launch();
  if (count > 0) k_f32_to_f64<<<(unsigned)b, 256, 0, st>>>(in, out, count);
}

}  // namespace lrtei
