// peaks.cu -- measured FMA rate of the CUDA cores (FP64 or FP32), the denominator of the
// rooflines of the FP64/FP32 CUDA-core kernels.  The paper has no counterpart: this is
// measurement infrastructure.  Every thread runs kChains independent FMA chains, so the rate is
// throughput-bound; the chains' sum is stored so that the work is kept.
#include "lrtei_internal.h"

namespace lrtei {

namespace {
constexpr int kChains = 16;
constexpr int kUnroll = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_rate(int iters, T seed, T* __restrict__ out) {
  T a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + (T)(threadIdx.x + c);
  const T m = (T)0.9999999, add = (T)1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, add);
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

template <typename T>
lrtei_status fma_rate(double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  LRTEI_CUDA(cudaGetDevice(&dev));
  LRTEI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  const int iters = sizeof(T) == 8 ? 2048 : 32768;
  T* out = nullptr;
  LRTEI_CUDA(scratch_alloc((void**)&out, sizeof(T) * (size_t)blocks * threads, st));
  cudaEvent_t e0, e1;
  LRTEI_CUDA(cudaEventCreate(&e0));
  LRTEI_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, st);
    count_launch();
    k_fma_rate<T><<<blocks, threads, 0, st>>>(iters, (T)1, out);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return cuda_fail(e, "fma rate");
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;  // the first launch carries one-time costs
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  LRTEI_CUDA(cudaFreeAsync(out, st));
  const double flops = 2.0 * kChains * kUnroll * (double)iters * blocks * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return LRTEI_OK;
}
}  // namespace

}  // namespace lrtei

extern "C" lrtei_status lrtei_measure_fma_peak(int fp64, double* tflops, void* stream) {
  using namespace lrtei;
  if (!tflops) {
    set_error("tflops is NULL");
    return LRTEI_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  return fp64 ? fma_rate<double>(tflops, st) : fma_rate<float>(tflops, st);
}
