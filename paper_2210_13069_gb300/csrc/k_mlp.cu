// k_mlp.cu -- the learned (n, P) selector: a 3-layer FP32 MLP (6 -> H -> H -> 2, ReLU) with
// hand-written forward, backward (mean squared error) and Adam kernels.
//
// Parameters are packed W1 (H x 6), b1 (H), W2 (H x H), b2 (H), W3 (2 x H), b3 (2), row-major,
// and live on the device.  One thread evaluates one sample; the weights are staged in shared
// memory; gradients are reduced per block in shared memory and added to the global gradient
// with one atomic per parameter per block.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "lrtei_internal.h"

namespace lrtei {
namespace mlp {

constexpr int kIn = 6, kOut = 2, kMaxH = 64, kThreads = 128;

__host__ __device__ inline int64_t nparams(int H) { return (int64_t)H * kIn + H + (int64_t)H * H + H + kOut * H + kOut; }

struct Off {
  int w1, b1, w2, b2, w3, b3;
};
__host__ __device__ inline Off offsets(int H) {
  Off o;
  o.w1 = 0;
  o.b1 = o.w1 + H * kIn;
  o.w2 = o.b1 + H;
  o.b2 = o.w2 + H * H;
  o.w3 = o.b2 + H;
  o.b3 = o.w3 + kOut * H;
  return o;
}

__device__ inline void forward_one(const float* __restrict__ w, const Off& o, int H, const float* x, float* h1,
                                   float* h2, float* y) {
  for (int j = 0; j < H; ++j) {
    float a = w[o.b1 + j];
    for (int i = 0; i < kIn; ++i) a += w[o.w1 + j * kIn + i] * x[i];
    h1[j] = a > 0.f ? a : 0.f;
  }
  for (int j = 0; j < H; ++j) {
    float a = w[o.b2 + j];
    for (int k = 0; k < H; ++k) a += w[o.w2 + j * H + k] * h1[k];
    h2[j] = a > 0.f ? a : 0.f;
  }
  for (int q = 0; q < kOut; ++q) {
    float a = w[o.b3 + q];
    for (int k = 0; k < H; ++k) a += w[o.w3 + q * H + k] * h2[k];
    y[q] = a;
  }
}

__global__ void k_forward(const float* __restrict__ params, int H, const float* __restrict__ X, int N,
                          float* __restrict__ Y) {
  extern __shared__ float sw[];
  const int64_t np = nparams(H);
  for (int64_t t = threadIdx.x; t < np; t += blockDim.x) sw[t] = params[t];
  __syncthreads();
  const Off o = offsets(H);
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  float x[kIn], h1[kMaxH], h2[kMaxH], y[kOut];
  for (int i = 0; i < kIn; ++i) x[i] = X[(int64_t)s * kIn + i];
  forward_one(sw, o, H, x, h1, h2, y);
  for (int q = 0; q < kOut; ++q) Y[(int64_t)s * kOut + q] = y[q];
}

// Gradient of L = (1 / (N kOut)) sum_s sum_q (y_sq - t_sq)^2 over the rows idx[0..n) (or 0..n).
__global__ void k_backward(const float* __restrict__ params, int H, const float* __restrict__ X,
                           const float* __restrict__ T, const int* __restrict__ idx, int n, float inv_count,
                           float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ float sm[];
  const int64_t np = nparams(H);
  float* sw = sm;
  float* sg = sm + np;
  for (int64_t t = threadIdx.x; t < np; t += blockDim.x) {
    sw[t] = params[t];
    sg[t] = 0.f;
  }
  __syncthreads();
  const Off o = offsets(H);
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (b < n) {
    const int64_t s = idx ? idx[b] : b;
    float x[kIn], h1[kMaxH], h2[kMaxH], y[kOut], dy[kOut];
    for (int i = 0; i < kIn; ++i) x[i] = X[s * kIn + i];
    forward_one(sw, o, H, x, h1, h2, y);
    for (int q = 0; q < kOut; ++q) {
      const float d = y[q] - T[s * kOut + q];
      l += d * d;
      dy[q] = 2.f * d * inv_count;
      atomicAdd(&sg[o.b3 + q], dy[q]);
      for (int k = 0; k < H; ++k) atomicAdd(&sg[o.w3 + q * H + k], dy[q] * h2[k]);
    }
    // dh2 (reuse h2 storage after its use above): dh2_k = sum_q W3[q][k] dy_q, masked by ReLU
    for (int k = 0; k < H; ++k) {
      float a = 0.f;
      for (int q = 0; q < kOut; ++q) a += sw[o.w3 + q * H + k] * dy[q];
      h2[k] = h2[k] > 0.f ? a : 0.f;
    }
    for (int j = 0; j < H; ++j) {
      atomicAdd(&sg[o.b2 + j], h2[j]);
      for (int k = 0; k < H; ++k) atomicAdd(&sg[o.w2 + j * H + k], h2[j] * h1[k]);
    }
    // dh1_k = sum_j W2[j][k] dh2_j, masked by ReLU
    float dh1[kMaxH];
    for (int k = 0; k < H; ++k) {
      float a = 0.f;
      for (int j = 0; j < H; ++j) a += sw[o.w2 + j * H + k] * h2[j];
      dh1[k] = h1[k] > 0.f ? a : 0.f;
    }
    for (int j = 0; j < H; ++j) {
      atomicAdd(&sg[o.b1 + j], dh1[j]);
      for (int i = 0; i < kIn; ++i) atomicAdd(&sg[o.w1 + j * kIn + i], dh1[j] * x[i]);
    }
  }
  // block loss
  for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
  if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, l * inv_count);
  __syncthreads();
  for (int64_t t = threadIdx.x; t < np; t += blockDim.x)
    if (sg[t] != 0.f) atomicAdd(&grad[t], sg[t]);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t np, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace mlp
}  // namespace lrtei

struct lrtei_selector {
  int hidden = 64;
  int64_t np = 0;
  float* d_params = nullptr;
  float* d_m = nullptr;
  float* d_v = nullptr;
  float* d_grad = nullptr;
  float* d_loss = nullptr;
  float* d_io = nullptr;  // one feature row and its two outputs (lrtei_select_np)
  int* d_idx = nullptr;
  int idx_cap = 0;
  int64_t step = 0;
  uint64_t rng = 0;
};

namespace {
uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
double uniform01(uint64_t& s) { return (splitmix64(s) >> 11) * (1.0 / 9007199254740992.0); }

size_t smem_fwd(int H) { return sizeof(float) * lrtei::mlp::nparams(H); }
size_t smem_bwd(int H) { return 2 * sizeof(float) * lrtei::mlp::nparams(H); }
}  // namespace

extern "C" {

lrtei_status lrtei_selector_create(int hidden, uint64_t seed, lrtei_selector** out) {
  using namespace lrtei;
  if (!out) { set_error("out is NULL"); return LRTEI_ERR_ARG; }
  *out = nullptr;
  if (hidden < 1 || hidden > mlp::kMaxH) { set_error("hidden width must be in 1..%d", mlp::kMaxH); return LRTEI_ERR_ARG; }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    set_error("no CUDA device available");
    return LRTEI_ERR_CUDA;
  }
  lrtei_selector* s = new lrtei_selector();
  s->hidden = hidden;
  s->np = mlp::nparams(hidden);
  s->rng = seed;
  // He-uniform initialisation from a counter-based generator (splitmix64)
  std::vector<float> h(s->np, 0.f);
  const mlp::Off o = mlp::offsets(hidden);
  auto fill = [&](int off, int count, int fan_in) {
    const double a = sqrt(6.0 / fan_in);
    for (int i = 0; i < count; ++i) h[off + i] = (float)((2.0 * uniform01(s->rng) - 1.0) * a);
  };
  fill(o.w1, hidden * mlp::kIn, mlp::kIn);
  fill(o.w2, hidden * hidden, hidden);
  fill(o.w3, mlp::kOut * hidden, hidden);
  cudaError_t e;
  for (int k = 0; k < 5; ++k) count_alloc();
  if ((e = cudaMalloc(&s->d_params, sizeof(float) * s->np)) != cudaSuccess ||
      (e = cudaMalloc(&s->d_m, sizeof(float) * s->np)) != cudaSuccess ||
      (e = cudaMalloc(&s->d_v, sizeof(float) * s->np)) != cudaSuccess ||
      (e = cudaMalloc(&s->d_grad, sizeof(float) * s->np)) != cudaSuccess ||
      (e = cudaMalloc(&s->d_loss, sizeof(float))) != cudaSuccess) {
    lrtei_selector_destroy(s);
    return cuda_fail(e, "selector allocation");
  }
  cudaMemcpy(s->d_params, h.data(), sizeof(float) * s->np, cudaMemcpyHostToDevice);
  cudaMemset(s->d_m, 0, sizeof(float) * s->np);
  cudaMemset(s->d_v, 0, sizeof(float) * s->np);
  if ((e = cudaGetLastError()) != cudaSuccess) {
    lrtei_selector_destroy(s);
    return cuda_fail(e, "selector init");
  }
  *out = s;
  return LRTEI_OK;
}

void lrtei_selector_destroy(lrtei_selector* s) {
  if (!s) return;
  cudaFree(s->d_params);
  cudaFree(s->d_m);
  cudaFree(s->d_v);
  cudaFree(s->d_grad);
  cudaFree(s->d_loss);
  cudaFree(s->d_io);
  cudaFree(s->d_idx);
  delete s;
}

int64_t lrtei_selector_nparams(const lrtei_selector* s) { return s ? s->np : 0; }

lrtei_status lrtei_selector_forward(lrtei_selector* s, const float* d_X, float* d_Yhat, int N, void* stream) {
  using namespace lrtei;
  if (!s || N < 0 || (N > 0 && (!d_X || !d_Yhat))) { set_error("invalid selector forward arguments"); return LRTEI_ERR_ARG; }
  if (N == 0) return LRTEI_OK;
  count_launch();
  mlp::k_forward<<<(N + mlp::kThreads - 1) / mlp::kThreads, mlp::kThreads, smem_fwd(s->hidden), (cudaStream_t)stream>>>(
      s->d_params, s->hidden, d_X, N, d_Yhat);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LRTEI_OK : cuda_fail(e, "selector forward");
}

lrtei_status lrtei_selector_grad(lrtei_selector* s, const float* d_X, const float* d_Y, int N, float* d_grad, float* loss,
                                 void* stream) {
  using namespace lrtei;
  if (!s || N <= 0 || !d_X || !d_Y || !d_grad) { set_error("invalid selector grad arguments"); return LRTEI_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  LRTEI_CUDA(cudaMemsetAsync(d_grad, 0, sizeof(float) * s->np, st));
  LRTEI_CUDA(cudaMemsetAsync(s->d_loss, 0, sizeof(float), st));
  count_launch();
  mlp::k_backward<<<(N + mlp::kThreads - 1) / mlp::kThreads, mlp::kThreads, smem_bwd(s->hidden), st>>>(
      s->d_params, s->hidden, d_X, d_Y, nullptr, N, 1.f / (float)(N * mlp::kOut), d_grad, s->d_loss);
  LRTEI_CUDA(cudaGetLastError());
  if (loss) {
    LRTEI_CUDA(cudaMemcpyAsync(loss, s->d_loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    LRTEI_CUDA(cudaStreamSynchronize(st));
  }
  return LRTEI_OK;
}

lrtei_status lrtei_selector_train_epoch(lrtei_selector* s, const float* d_X, const float* d_Y, int N, int batch, float lr,
                                        float* loss, void* stream) {
  using namespace lrtei;
  if (!s || N <= 0 || batch <= 0 || !d_X || !d_Y || !(lr > 0.f)) { set_error("invalid selector train arguments"); return LRTEI_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  if (s->idx_cap < N) {
    cudaFree(s->d_idx);
    s->d_idx = nullptr;
    count_alloc();
    LRTEI_CUDA(cudaMalloc(&s->d_idx, sizeof(int) * N));
    s->idx_cap = N;
  }
  // a fresh permutation of the rows for this epoch (Fisher-Yates on the host, splitmix64)
  std::vector<int> perm(N);
  for (int i = 0; i < N; ++i) perm[i] = i;
  for (int i = N - 1; i > 0; --i) {
    const int j = (int)(splitmix64(s->rng) % (uint64_t)(i + 1));
    std::swap(perm[i], perm[j]);
  }
  LRTEI_CUDA(cudaMemcpyAsync(s->d_idx, perm.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st));
  LRTEI_CUDA(cudaMemsetAsync(s->d_loss, 0, sizeof(float), st));
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  int nb = 0;
  for (int off = 0; off < N; off += batch, ++nb) {
    const int n = std::min(batch, N - off);
    LRTEI_CUDA(cudaMemsetAsync(s->d_grad, 0, sizeof(float) * s->np, st));
    count_launch();
    mlp::k_backward<<<(n + mlp::kThreads - 1) / mlp::kThreads, mlp::kThreads, smem_bwd(s->hidden), st>>>(
        s->d_params, s->hidden, d_X, d_Y, s->d_idx + off, n, 1.f / (float)(n * mlp::kOut), s->d_grad, s->d_loss);
    ++s->step;
    const float c1 = 1.f - powf(b1, (float)s->step), c2 = 1.f - powf(b2, (float)s->step);
    count_launch();
    mlp::k_adam<<<(int)((s->np + 255) / 256), 256, 0, st>>>(s->d_params, s->d_grad, s->d_m, s->d_v, s->np, lr, b1, b2,
                                                            eps, c1, c2);
  }
  LRTEI_CUDA(cudaGetLastError());
  if (loss) {
    float l = 0.f;
    LRTEI_CUDA(cudaMemcpyAsync(&l, s->d_loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    LRTEI_CUDA(cudaStreamSynchronize(st));
    *loss = l / (float)nb;  // mean over the epoch's mini-batches
  }
  return LRTEI_OK;
}

lrtei_status lrtei_selector_get_params(const lrtei_selector* s, float* h_params) {
  using namespace lrtei;
  if (!s || !h_params) { set_error("NULL argument"); return LRTEI_ERR_ARG; }
  LRTEI_CUDA(cudaMemcpy(h_params, s->d_params, sizeof(float) * s->np, cudaMemcpyDeviceToHost));
  return LRTEI_OK;
}

lrtei_status lrtei_selector_set_params(lrtei_selector* s, const float* h_params) {
  using namespace lrtei;
  if (!s || !h_params) { set_error("NULL argument"); return LRTEI_ERR_ARG; }
  LRTEI_CUDA(cudaMemcpy(s->d_params, h_params, sizeof(float) * s->np, cudaMemcpyHostToDevice));
  return LRTEI_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ selection policy
// The network maps normalised features of an instance to the normalised cheapest (n, P) that met
// a target in the error sweeps; the policy around it (feature normalisation, training ranges,
// fallback, margins and the grids) lives here so that a caller selects (n, P) through the C ABI
// alone.
namespace lrtei {
namespace selpol {
constexpr int kNGrid[] = {8, 12, 16, 20, 24, 28, 32, 40, 48, 56, 64};      // last: N_MAX
constexpr int kPGrid[] = {8, 12, 16, 20, 24, 28, 32, 40, 48, 64, 80, 96, 128};  // last: P_MAX
constexpr int kFallbackN = 32, kFallbackP = 48, kMarginN = 4, kMarginP = 8;
// training ranges of (omega, box half-width, log10 alpha_min, log10 alpha_max, max l, log10 target)
constexpr double kLo[6] = {0.2, 3.0, -1.4, -0.4, 0.0, -9.0};
constexpr double kHi[6] = {1.0, 34.0, 0.1, 3.4, 2.0, -3.0};

bool valid_raw(const double* raw) {
  for (int i = 0; i < 6; ++i)
    if (!isfinite(raw[i])) return false;
  return raw[0] > 0.0 && raw[1] > 0.0 && raw[2] > 0.0 && raw[3] > 0.0 && raw[4] >= 0.0 && raw[5] > 0.0;
}
void features(const double* raw, float* out) {
  out[0] = (float)raw[0];
  out[1] = (float)(raw[1] / 30.0);
  out[2] = (float)log10(raw[2]);
  out[3] = (float)(log10(raw[3]) / 4.0);
  out[4] = (float)(raw[4] / 2.0);
  out[5] = (float)(-log10(raw[5]) / 10.0);
}
bool in_range(const double* raw) {
  const double v[6] = {raw[0], raw[1], log10(raw[2]), log10(raw[3]), raw[4], log10(raw[5])};
  for (int i = 0; i < 6; ++i)
    if (v[i] < kLo[i] - 1e-9 || v[i] > kHi[i] + 1e-9) return false;
  return true;
}
template <size_t K>
int round_up(const int (&grid)[K], double x) {
  for (size_t i = 0; i < K; ++i)
    if (grid[i] >= x) return grid[i];
  return grid[K - 1];
}

// FNV-1a, 64 bit, over the checkpoint's bytes.
uint64_t fnv1a(const unsigned char* p, size_t n, uint64_t h = 1469598103934665603ULL) {
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ULL;
  }
  return h;
}
constexpr char kMagic[8] = {'L', 'R', 'T', 'E', 'I', 'S', 'E', 'L'};
constexpr uint32_t kVersion = 2;
}  // namespace selpol
}  // namespace lrtei

extern "C" {

lrtei_status lrtei_selector_features(const double* raw, float* out) {
  using namespace lrtei;
  if (!raw || !out) { set_error("NULL argument"); return LRTEI_ERR_ARG; }
  if (!selpol::valid_raw(raw)) {
    set_error("selector features: omega, box half-width, exponents and target must be positive and finite");
    return LRTEI_ERR_ARG;
  }
  selpol::features(raw, out);
  return LRTEI_OK;
}

lrtei_status lrtei_selector_encode(int n, int P, float* out) {
  using namespace lrtei;
  if (!out || n < 1 || P < 1) { set_error("invalid selector encode arguments"); return LRTEI_ERR_ARG; }
  out[0] = (float)((n - 8.0) / 56.0);
  out[1] = (float)((P - 8.0) / 120.0);
  return LRTEI_OK;
}

lrtei_status lrtei_select_np(lrtei_selector* sel, const double* raw, int* n, int* P, int* used_fallback) {
  using namespace lrtei;
  if (!sel || !raw || !n || !P) { set_error("NULL argument"); return LRTEI_ERR_ARG; }
  if (!selpol::valid_raw(raw)) {
    set_error("select_np: omega, box half-width, exponents and target must be positive and finite");
    return LRTEI_ERR_ARG;
  }
  if (!selpol::in_range(raw)) {  // outside the trained ranges: the conservative fixed orders
    *n = selpol::kFallbackN;
    *P = selpol::kFallbackP;
    if (used_fallback) *used_fallback = 1;
    return LRTEI_OK;
  }
  float h[8];
  selpol::features(raw, h);
  if (!sel->d_io) {
    count_alloc();
    LRTEI_CUDA(cudaMalloc(&sel->d_io, sizeof(float) * 8));
  }
  LRTEI_CUDA(cudaMemcpy(sel->d_io, h, sizeof(float) * mlp::kIn, cudaMemcpyHostToDevice));
  count_launch();
  mlp::k_forward<<<1, mlp::kThreads, smem_fwd(sel->hidden)>>>(sel->d_params, sel->hidden, sel->d_io, 1,
                                                              sel->d_io + mlp::kIn);
  LRTEI_CUDA(cudaGetLastError());
  LRTEI_CUDA(cudaMemcpy(h + mlp::kIn, sel->d_io + mlp::kIn, sizeof(float) * mlp::kOut, cudaMemcpyDeviceToHost));
  const double nf = 8.0 + 56.0 * h[mlp::kIn], pf = 8.0 + 120.0 * h[mlp::kIn + 1];
  if (!isfinite(nf) || !isfinite(pf)) { set_error("selector network output is not finite"); return LRTEI_ERR_NUMERIC; }
  *n = selpol::round_up(selpol::kNGrid, nf + selpol::kMarginN);
  *P = selpol::round_up(selpol::kPGrid, pf + selpol::kMarginP);
  if (used_fallback) *used_fallback = 0;
  return LRTEI_OK;
}

lrtei_status lrtei_selector_train(lrtei_selector* sel, const float* d_X, const float* d_Y, int N, int epochs,
                                  int batch, float lr, float* h_loss, void* stream) {
  using namespace lrtei;
  if (!sel || epochs <= 0) { set_error("invalid selector train arguments"); return LRTEI_ERR_ARG; }
  for (int ep = 0; ep < epochs; ++ep) {
    const float cur = ep < epochs * 2 / 3 ? lr : 0.1f * lr;  // step decay for the last third
    float l = 0.f;
    const lrtei_status s = lrtei_selector_train_epoch(sel, d_X, d_Y, N, batch, cur, h_loss ? &l : nullptr, stream);
    if (s != LRTEI_OK) return s;
    if (h_loss) h_loss[ep] = l;
  }
  return LRTEI_OK;
}

lrtei_status lrtei_selector_save(const lrtei_selector* sel, const char* path, const char* meta) {
  using namespace lrtei;
  if (!sel || !path) { set_error("NULL argument"); return LRTEI_ERR_ARG; }
  std::vector<float> params((size_t)sel->np);
  LRTEI_CUDA(cudaMemcpy(params.data(), sel->d_params, sizeof(float) * sel->np, cudaMemcpyDeviceToHost));
  const uint32_t mlen = meta ? (uint32_t)strlen(meta) : 0u;
  std::vector<unsigned char> buf;
  auto put = [&](const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    buf.insert(buf.end(), c, c + n);
  };
  const uint32_t ver = selpol::kVersion, hid = (uint32_t)sel->hidden;
  const uint64_t np = (uint64_t)sel->np;
  put(selpol::kMagic, 8);
  put(&ver, 4);
  put(&hid, 4);
  put(&np, 8);
  put(&mlen, 4);
  if (mlen) put(meta, mlen);
  put(params.data(), sizeof(float) * params.size());
  const uint64_t sum = selpol::fnv1a(buf.data(), buf.size());
  put(&sum, 8);
  FILE* f = fopen(path, "wb");
  if (!f) { set_error("cannot open %s for writing", path); return LRTEI_ERR_ARG; }
  const size_t w = fwrite(buf.data(), 1, buf.size(), f);
  const int c = fclose(f);
  if (w != buf.size() || c != 0) { set_error("writing %s failed", path); return LRTEI_ERR_ARG; }
  return LRTEI_OK;
}

lrtei_status lrtei_selector_load(const char* path, lrtei_selector** out, char* meta, size_t meta_cap) {
  using namespace lrtei;
  if (!path || !out) { set_error("NULL argument"); return LRTEI_ERR_ARG; }
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) { set_error("cannot open %s", path); return LRTEI_ERR_ARG; }
  std::vector<unsigned char> buf;
  unsigned char tmp[65536];
  size_t r;
  while ((r = fread(tmp, 1, sizeof(tmp), f)) > 0) buf.insert(buf.end(), tmp, tmp + r);
  fclose(f);
  const size_t head = 8 + 4 + 4 + 8 + 4;
  if (buf.size() < head + 8 || memcmp(buf.data(), selpol::kMagic, 8) != 0) {
    set_error("%s is not a selector checkpoint", path);
    return LRTEI_ERR_ARG;
  }
  uint32_t ver, hid, mlen;
  uint64_t np, sum;
  memcpy(&ver, buf.data() + 8, 4);
  memcpy(&hid, buf.data() + 12, 4);
  memcpy(&np, buf.data() + 16, 8);
  memcpy(&mlen, buf.data() + 24, 4);
  if (ver != selpol::kVersion) { set_error("selector checkpoint version %u, this library reads %u", ver, selpol::kVersion); return LRTEI_ERR_ARG; }
  if (hid < 1 || hid > (uint32_t)mlp::kMaxH || np != (uint64_t)mlp::nparams((int)hid) ||
      buf.size() != head + mlen + np * sizeof(float) + 8) {
    set_error("selector checkpoint %s: inconsistent sizes", path);
    return LRTEI_ERR_ARG;
  }
  memcpy(&sum, buf.data() + buf.size() - 8, 8);
  if (selpol::fnv1a(buf.data(), buf.size() - 8) != sum) { set_error("selector checkpoint %s: checksum mismatch", path); return LRTEI_ERR_ARG; }
  if (meta && meta_cap > 0) {
    const size_t k = std::min((size_t)mlen, meta_cap - 1);
    memcpy(meta, buf.data() + head, k);
    meta[k] = 0;
  }
  lrtei_selector* s = nullptr;
  lrtei_status st = lrtei_selector_create((int)hid, 0, &s);
  if (st != LRTEI_OK) return st;
  std::vector<float> params((size_t)np);
  memcpy(params.data(), buf.data() + head + mlen, sizeof(float) * np);
  st = lrtei_selector_set_params(s, params.data());
  if (st != LRTEI_OK) { lrtei_selector_destroy(s); return st; }
  *out = s;
  return LRTEI_OK;
}

}  // extern "C"
