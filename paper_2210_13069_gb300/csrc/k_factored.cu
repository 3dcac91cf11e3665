// k_factored.cu -- kernels of the Khatri-Rao factored form (eq. tensors) and its application:
//   M(mu nu, (m1 n + m2) n + m3) = sum_{j in mu nu} c_j S_x(j, m1) S_y(j, m2) S_z(j, m3)
//   B = (w/sqrt(pi)) M K M^T,  K = sum_p w_p A_x^(p) (x) A_y^(p) (x) A_z^(p)
// K is applied either densely (tensor-core path) or by three mode products per node (eq. ig1).
// Also the symmetric expansion of the unique-pair matrix B_u into the full N_b^2 x N_b^2 B and
// the density packing of the J-build (Section 5).
#include <algorithm>

#include "lrtei_internal.h"
#include "tc_common.h"

namespace lrtei {

__device__ __forceinline__ int64_t pair_idx(int nbf, int a, int b) {
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  return (int64_t)lo * nbf - (int64_t)lo * (lo - 1) / 2 + (hi - lo);
}

// One block (x) per pair r in [r0, r1); threads over the n^3 columns.
template <typename T>
__global__ void k_build_F(int n, int64_t nrows, const int64_t* __restrict__ pair_row, const double* __restrict__ row_c,
                          const double* __restrict__ S, int64_t r0, T* __restrict__ F, int64_t ldF) {
  const int64_t r = r0 + blockIdx.x;
  const int64_t j0 = pair_row[r], j1 = pair_row[r + 1];
  const int n3 = n * n * n;
  const double* Sx = S;
  const double* Sy = S + (size_t)nrows * n;
  const double* Sz = S + 2 * (size_t)nrows * n;
  T* out = F + (size_t)blockIdx.x * ldF;
  for (int m = threadIdx.x; m < n3; m += blockDim.x) {
    const int m1 = m / (n * n), m2 = (m / n) % n, m3 = m % n;
    double acc = 0.0;
    for (int64_t j = j0; j < j1; ++j)
      acc += row_c[j] * Sx[(size_t)j * n + m1] * Sy[(size_t)j * n + m2] * Sz[(size_t)j * n + m3];
    out[m] = (T)acc;
  }
}

// The same F_u with the pair's rows staged: X_j = c_j S_x(j, .) in shared memory (zero padded to a
// multiple of 8 columns), and each thread owning a column q = m2 n + m3 and eight consecutive m1,
// so that a row j costs one multiply (S_y S_z) and eight FMAs for eight outputs instead of three
// FP64 operations per output.  The sum over j runs in the same order as above.
template <typename T>
__global__ void __launch_bounds__(256) k_build_F_staged(int n, int64_t nrows, const int64_t* __restrict__ pair_row,
                                                        const double* __restrict__ row_c, const double* __restrict__ S,
                                                        int64_t r0, T* __restrict__ F, int64_t ldF) {
  extern __shared__ double X[];  // [rows of the pair][n8]
  const int64_t r = r0 + blockIdx.x;
  const int64_t j0 = pair_row[r];
  const int I = (int)(pair_row[r + 1] - j0);
  const int n8 = (n + 7) / 8 * 8, nn = n * n;
  const double* Sx = S;
  const double* Sy = S + (size_t)nrows * n;
  const double* Sz = S + 2 * (size_t)nrows * n;
  for (int e = threadIdx.x; e < I * n8; e += blockDim.x) {
    const int j = e / n8, m1 = e % n8;
    X[e] = m1 < n ? row_c[j0 + j] * Sx[(size_t)(j0 + j) * n + m1] : 0.0;
  }
  __syncthreads();
  T* out = F + (size_t)blockIdx.x * ldF;
  const int items = nn * (n8 / 8);
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int q = it % nn, g = it / nn;
    const int m2 = q / n, m3 = q % n;
    double acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0.0;
    for (int j = 0; j < I; ++j) {
      const double y = Sy[(size_t)(j0 + j) * n + m2] * Sz[(size_t)(j0 + j) * n + m3];
      const double2* xr = reinterpret_cast<const double2*>(X + j * n8 + g * 8);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const double2 x2 = xr[i];
        acc[2 * i] = fma(x2.x, y, acc[2 * i]);
        acc[2 * i + 1] = fma(x2.y, y, acc[2 * i + 1]);
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (g * 8 + i < n) out[(size_t)(g * 8 + i) * nn + q] = (T)acc[i];
  }
}

template <typename T>
void launch_build_F(const PairTable& t, int n, const double* d_S, int64_t r0, int64_t r1, T* d_F, int64_t ldF,
                    cudaStream_t st) {
  const size_t smem = sizeof(double) * (size_t)t.maxI * ((n + 7) / 8 * 8);
  const bool staged = t.maxI > 0 && smem <= 48 * 1024;
  int64_t nr = r1 - r0;
  while (nr > 0) {
    int64_t chunk = nr > (1LL << 30) ? (1LL << 30) : nr;
    count_launch();
    if (staged)
      k_build_F_staged<T><<<(unsigned)chunk, 256, smem, st>>>(n, t.nrows, t.pair_row, t.row_c, d_S, r0, d_F, ldF);
    else
      k_build_F<T><<<(unsigned)chunk, 256, 0, st>>>(n, t.nrows, t.pair_row, t.row_c, d_S, r0, d_F, ldF);
    r0 += chunk;
    d_F += chunk * ldF;
    nr -= chunk;
  }
}
template void launch_build_F<double>(const PairTable&, int, const double*, int64_t, int64_t, double*, int64_t,
                                     cudaStream_t);
template void launch_build_F<float>(const PairTable&, int, const double*, int64_t, int64_t, float*, int64_t,
                                    cudaStream_t);

// The same K with the node sum in pairs of FP32 numbers (this part's FP32 rate is ~70 times its
// FP64 rate; K only feeds 30-bit slices).  Each value is the unevaluated sum hi + lo of two floats
// (Dekker 1971); a term r_p z_p is formed exactly in its leading part by an FMA (TwoProd) plus
// the cross products, and summed by the compensated dot product Dot2 of Ogita, Rump and Oishi
// ("Accurate sum and dot product", 2005): the running sum by Knuth's TwoSum, the errors in a
// second float.  The result, hi + lo in FP64, is accurate to ~2^-44 of the row maximum.
//
// Block (g tile, (a1, b1)): r_p(g) = scale w_p A_x^p(a1, b1) A_y^p(a2, b2) for kKG consecutive
// g = (a2, b2) in shared memory (FP64, then split); thread t owns e = (a3, b3) in {t, t + blockDim}
// (+ 2 blockDim ...) and the kKG outputs (g, e), reading z_p(e) = A_z^p(a3, b3) from a pair table
// zp[p][e].  Sixteen independent sums per thread keep the FP32 pipes busy at modest occupancy;
// consecutive threads write consecutive columns b3.
constexpr int kKG = 8;  // g per pass (two passes of the block's 16-g tile)

struct Pair32 {
  float hi, lo;
};

__device__ __forceinline__ Pair32 to_pair(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

__global__ void k_K_zpairs(int nn, int P, const double* __restrict__ C, Pair32* __restrict__ zp) {
  const int64_t total = (int64_t)nn * P;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    zp[i] = to_pair(C[(size_t)2 * P * nn + i]);  // zp[p][e] = A_z^p(e)
}

// One term of the compensated dot product (the _rn intrinsics are never contracted into FMAs,
// which would break the exact steps).
__device__ __forceinline__ void dot2_step(Pair32 x, Pair32 z, float& sum, float& err) {
  const float ph = __fmul_rn(x.hi, z.hi);
  float pe = fmaf(x.hi, z.hi, -ph);              // TwoProd: ph + pe = x.hi z.hi exactly
  pe = fmaf(x.hi, z.lo, fmaf(x.lo, z.hi, pe));  // cross products (x.lo z.lo ~ 2^-48 dropped)
  const float t = __fadd_rn(sum, ph);           // TwoSum: t + d = sum + ph exactly
  const float bp = __fsub_rn(t, sum);
  const float d = __fadd_rn(__fsub_rn(sum, __fsub_rn(t, bp)), __fsub_rn(ph, bp));
  sum = t;
  err = __fadd_rn(err, __fadd_rn(d, pe));
}

// F_u for the tensor-core precisions, whose F_u only feeds 30-bit slices: the same staged walk
// with every product and the sum over the pair's rows j in pairs of FP32 numbers (the moments
// converted to pairs once, y = S_y S_z by TwoProd, the sum over j by the compensated dot product
// below), stored as FP64 from the pair by integer arithmetic: ~2^-44 of each term's size, against
// FP64's 2^-53, at this part's FP32 rate instead of its FP64 rate.
__global__ void k_S_pairs(int64_t count, const double* __restrict__ S, float2* __restrict__ Sp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const Pair32 q = to_pair(S[i]);
    Sp[i] = make_float2(q.hi, q.lo);
  }
}

__global__ void __launch_bounds__(256) k_build_F_pairs(int n, int64_t nrows, const int64_t* __restrict__ pair_row,
                                                       const double* __restrict__ row_c, const double* __restrict__ S,
                                                       const float2* __restrict__ Sp, int64_t r0,
                                                       double* __restrict__ F, int64_t ldF) {
  extern __shared__ float2 Xp[];  // [rows of the pair][n8]: c_j S_x(j, m1) as pairs
  const int64_t r = r0 + blockIdx.x;
  const int64_t j0 = pair_row[r];
  const int I = (int)(pair_row[r + 1] - j0);
  const int n8 = (n + 7) / 8 * 8, nn = n * n;
  const float2* Sy = Sp + (size_t)nrows * n;
  const float2* Sz = Sp + 2 * (size_t)nrows * n;
  for (int e = threadIdx.x; e < I * n8; e += blockDim.x) {
    const int j = e / n8, m1 = e % n8;
    const Pair32 q = to_pair(m1 < n ? row_c[j0 + j] * S[(size_t)(j0 + j) * n + m1] : 0.0);
    Xp[e] = make_float2(q.hi, q.lo);
  }
  __syncthreads();
  double* out = F + (size_t)blockIdx.x * ldF;
  const int items = nn * (n8 / 8);
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int q = it % nn, g = it / nn;
    const int m2 = q / n, m3 = q % n;
    float sum[8], err[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) sum[i] = err[i] = 0.f;
    for (int j = 0; j < I; ++j) {
      const float2 a = Sy[(size_t)(j0 + j) * n + m2], b = Sz[(size_t)(j0 + j) * n + m3];
      const float yh = __fmul_rn(a.x, b.x);
      float yl = fmaf(a.x, b.x, -yh);  // TwoProd
      yl = fmaf(a.x, b.y, fmaf(a.y, b.x, yl));
      const Pair32 y{yh, yl};
      const float2* xr = Xp + j * n8 + g * 8;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float2 x = xr[i];
        dot2_step(Pair32{x.x, x.y}, y, sum[i], err[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (g * 8 + i < n) out[(size_t)(g * 8 + i) * nn + q] = tc::fpair_ldexp(sum[i], err[i], 0);
  }
}

void launch_build_F_pairs(const PairTable& t, int n, const double* d_S, int64_t r0, int64_t r1, double* d_F,
                          int64_t ldF, cudaStream_t st) {
  const size_t smem = sizeof(float2) * (size_t)t.maxI * ((n + 7) / 8 * 8);
  if (t.maxI <= 0 || smem > 48 * 1024) {  // very long pair blocks: the FP64 build
    launch_build_F<double>(t, n, d_S, r0, r1, d_F, ldF, st);
    return;
  }
  const int64_t count = 3 * t.nrows * n;
  float2* Sp = nullptr;
  if (scratch_alloc((void**)&Sp, sizeof(float2) * (size_t)std::max<int64_t>(count, 1), st) != cudaSuccess) {
    cudaGetLastError();
    launch_build_F<double>(t, n, d_S, r0, r1, d_F, ldF, st);  // no scratch: the FP64 build
    return;
  }
  count_launch();
  k_S_pairs<<<(unsigned)std::min<int64_t>((count + 255) / 256, 152 * 32), 256, 0, st>>>(count, d_S, Sp);
  int64_t nr = r1 - r0;
  while (nr > 0) {
    const int64_t chunk = nr > (1LL << 30) ? (1LL << 30) : nr;
    count_launch();
    k_build_F_pairs<<<(unsigned)chunk, 256, smem, st>>>(n, t.nrows, t.pair_row, t.row_c, d_S, Sp, r0, d_F, ldF);
    r0 += chunk;
    d_F += chunk * ldF;
    nr -= chunk;
  }
  cudaFreeAsync(Sp, st);
}

__global__ void __launch_bounds__(512, 1) k_build_K_tiled(int n, int P, const double* __restrict__ C,
                                                       const double* __restrict__ w, const Pair32* __restrict__ zp,
                                                       double scale, double* __restrict__ K) {
  __shared__ Pair32 r[2 * kKG * kMaxP];
  const int nn = n * n;
  const int64_t n3 = (int64_t)nn * n;
  const int g0 = blockIdx.x * 2 * kKG;
  const int ab = blockIdx.y, a1 = ab / n, b1 = ab % n;
  for (int i = threadIdx.x; i < 2 * kKG * P; i += blockDim.x) {
    const int g = g0 + i / P, p = i % P;
    r[i] = to_pair(g < nn ? scale * w[p] * C[(size_t)p * nn + ab] * C[((size_t)P + p) * nn + g] : 0.0);
  }
  __syncthreads();
  for (int half = 0; half < 2; ++half) {
    const Pair32* rh = r + half * kKG * P;
    const int gb = g0 + half * kKG;
    if (gb >= nn) break;
    for (int eb = 0; eb < nn; eb += 2 * blockDim.x) {
      const int e0 = eb + threadIdx.x, e1 = e0 + blockDim.x;
      const bool l0 = e0 < nn, l1 = e1 < nn;
      if (!l0) break;
      float sum[2][kKG], err[2][kKG];
#pragma unroll
      for (int j = 0; j < kKG; ++j) sum[0][j] = err[0][j] = sum[1][j] = err[1][j] = 0.f;
      for (int p = 0; p < P; ++p) {
        const Pair32 z0 = zp[(size_t)p * nn + e0];
        const Pair32 z1 = l1 ? zp[(size_t)p * nn + e1] : Pair32{0.f, 0.f};
#pragma unroll
        for (int j = 0; j < kKG; ++j) {
          const Pair32 x = rh[j * P + p];
          dot2_step(x, z0, sum[0][j], err[0][j]);
          dot2_step(x, z1, sum[1][j], err[1][j]);
        }
      }
#pragma unroll
      for (int j = 0; j < kKG; ++j) {
        const int g = gb + j;
        if (g >= nn) break;
        const int a2 = g / n, b2 = g % n;
        const int64_t row0 = (int64_t)(a1 * n + a2) * n, col0 = (int64_t)(b1 * n + b2) * n;
        K[(row0 + e0 / n) * n3 + col0 + e0 % n] = (double)sum[0][j] + (double)err[0][j];
        if (l1) K[(row0 + e1 / n) * n3 + col0 + e1 % n] = (double)sum[1][j] + (double)err[1][j];
      }
    }
  }
}

cudaError_t launch_build_K(int n, int P, const double* d_C, const double* d_w, double scale, double* d_K,
                           cudaStream_t st) {
  const int nn = n * n;
  Pair32* zp = nullptr;
  cudaError_t e = scratch_alloc((void**)&zp, sizeof(Pair32) * (size_t)nn * P, st);
  if (e != cudaSuccess) return e;
  count_launch();
  k_K_zpairs<<<(unsigned)std::min<int64_t>(((int64_t)nn * P + 255) / 256, 152 * 8), 256, 0, st>>>(nn, P, d_C, zp);
  // two e per thread; at most 512 threads
  const int threads = std::min(512, ((nn + 1) / 2 + 31) / 32 * 32);
  count_launch();
  k_build_K_tiled<<<dim3((unsigned)((nn + 2 * kKG - 1) / (2 * kKG)), (unsigned)nn), threads, 0, st>>>(n, P, d_C, d_w, zp,
                                                                                                     scale, d_K);
  e = cudaGetLastError();
  cudaFreeAsync(zp, st);
  return e;
}

// Mode product on a tensor viewed as (I, n, Kd): out[i][a][k] = sum_m C[a][m] in[i][m][k].
// If acc_w != 0, out = (first ? 0 : out) + acc_w * result.
__global__ void k_mode(int64_t I, int n, int64_t Kd, const double* __restrict__ Cm, const double* __restrict__ in,
                       double* __restrict__ out, double acc_w, int accumulate, int first) {
  const int64_t total = I * n * Kd;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t % Kd;
    const int a = (int)((t / Kd) % n);
    const int64_t i = t / Kd / n;
    const double* src = in + (size_t)i * n * Kd + k;
    const double* c = Cm + (size_t)a * n;
    double acc = 0.0;
    for (int m = 0; m < n; ++m) acc += c[m] * src[(size_t)m * Kd];
    if (accumulate)
      out[t] = (first ? 0.0 : out[t]) + acc_w * acc;
    else
      out[t] = acc;
  }
}

__global__ void k_axpy_w(int64_t count, const double* __restrict__ w, int p, const double* __restrict__ x,
                         double* __restrict__ y, int first) {
  const double wp = w[p];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    y[t] = (first ? 0.0 : y[t]) + wp * x[t];
}

static void launch_axpy_w(int64_t count, const double* w, int p, const double* x, double* y, int first, cudaStream_t st) {
  int64_t blocks = (count + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  count_launch();
  k_axpy_w<<<(unsigned)blocks, 256, 0, st>>>(count, w, p, x, y, first);
}

void launch_kron_apply(int n, int P, const double* d_C, const double* d_w, const double* d_X, double* d_Y,
                       int64_t ncol, double* d_t1, double* d_t2, cudaStream_t st) {
  // X, Y: ncol rows of length n^3 (cube index (m1, m2, m3), m3 fastest).
  const int64_t n3 = (int64_t)n * n * n;
  const int64_t total = ncol * n3;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  const size_t nn = (size_t)n * n;
  for (int p = 0; p < P; ++p) {
    const double* cx = d_C + ((size_t)0 * P + p) * nn;
    const double* cy = d_C + ((size_t)1 * P + p) * nn;
    const double* cz = d_C + ((size_t)2 * P + p) * nn;
    count_launch();
    k_mode<<<(unsigned)blocks, 256, 0, st>>>(ncol, n, (int64_t)n * n, cx, d_X, d_t1, 0.0, 0, 0);
    count_launch();
    k_mode<<<(unsigned)blocks, 256, 0, st>>>(ncol * n, n, n, cy, d_t1, d_t2, 0.0, 0, 0);
    // mode 3, then Y += w_p * result (the weight is read on the device)
    count_launch();
    k_mode<<<(unsigned)blocks, 256, 0, st>>>(ncol * nn, n, 1, cz, d_t2, d_t1, 0.0, 0, 0);
    launch_axpy_w(total, d_w, p, d_t1, d_Y, p == 0, st);
  }
}

// One block per unique pair r = (mu, nu); writes full rows mu*N_b+nu and nu*N_b+mu.
// The column walk of one B row: col = t, t + step, ... with (ka, la) = (col / N_b, col % N_b)
// advanced by additions (no 64-bit division per element), the non-finite test on the bit pattern
// and the scale applied only when it is not 1 (this device's FP64 rate would otherwise make the
// expansion ALU-bound rather than bound by its 12 GB of traffic).
struct ColWalk {
  int ka, la, dka, dla, nbf;
  __device__ ColWalk(int nbf_, int t, int step) : nbf(nbf_) {
    ka = t / nbf;
    la = t % nbf;
    dka = step / nbf;
    dla = step % nbf;
  }
  __device__ void next() {
    ka += dka;
    la += dla;
    if (la >= nbf) {
      la -= nbf;
      ++ka;
    }
  }
};

__device__ __forceinline__ bool nonfinite_bits(double v) {
  return ((__double_as_longlong(v) >> 52) & 0x7FF) == 0x7FF;
}

__global__ void k_expand_B(int nbf, const double* __restrict__ Bu, int64_t ldu, double scale, double* __restrict__ B,
                           int64_t ldB, const int* __restrict__ pair_mu, const int* __restrict__ pair_nu, int* status) {
  const int64_t r = blockIdx.x;
  const int mu = pair_mu[r], nu = pair_nu[r];
  const double* src = Bu + (size_t)r * ldu;
  double* row1 = B + ((size_t)mu * nbf + nu) * ldB;
  double* row2 = B + ((size_t)nu * nbf + mu) * ldB;
  const int nc = nbf * nbf;
  const bool scaled = scale != 1.0;
  bool bad = false;
  ColWalk w(nbf, threadIdx.x, blockDim.x);
  for (int col = threadIdx.x; col < nc; col += blockDim.x, w.next()) {
    double v = src[pair_idx(nbf, w.ka, w.la)];
    if (scaled) v *= scale;
    bad |= nonfinite_bits(v);
    row1[col] = v;
    if (mu != nu) row2[col] = v;
  }
  latch_nonfinite_warp(status, bad);
}

void launch_expand_B(const PairTable& t, int nbf, const double* d_Bu, int64_t ldu, double scale, double* d_B,
                     int64_t ldB, int* d_status, cudaStream_t st) {
  count_launch();
  k_expand_B<<<(unsigned)t.npair, 256, 0, st>>>(nbf, d_Bu, ldu, scale, d_B, ldB, t.pair_mu, t.pair_nu, d_status);
}

// One block per row R = a N_b + b of B: out row R - R0 = B_u row pair(a, b) over the columns (ka, la).
__global__ void k_expand_B_rows(int nbf, const double* __restrict__ Bu, int64_t ldu, int64_t R0, double* __restrict__ out,
                                int64_t ldo, int* status) {
  const int64_t R = R0 + blockIdx.x;
  const int a = (int)(R / nbf), b = (int)(R % nbf);
  const double* src = Bu + (size_t)pair_idx(nbf, a, b) * ldu;
  double* dst = out + (size_t)blockIdx.x * ldo;
  const int nc = nbf * nbf;
  bool bad = false;
  ColWalk w(nbf, threadIdx.x, blockDim.x);
  for (int col = threadIdx.x; col < nc; col += blockDim.x, w.next()) {
    const double v = src[pair_idx(nbf, w.ka, w.la)];
    bad |= nonfinite_bits(v);
    dst[col] = v;
  }
  latch_nonfinite_warp(status, bad);
}

void launch_expand_B_rows(int nbf, const double* d_Bu, int64_t ldu, int64_t R0, int64_t R1, double* d_out, int64_t ldo,
                          int* d_status, cudaStream_t st) {
  if (R1 <= R0) return;
  count_launch();
  k_expand_B_rows<<<(unsigned)(R1 - R0), 256, 0, st>>>(nbf, d_Bu, ldu, R0, d_out, ldo, d_status);
}

// d_u[r][q] = D_q(mu, nu) * (mu == nu ? 1 : 2); D stored R x N_b x N_b.
__global__ void k_pack_density(int nbf, int R, int64_t npair, const double* __restrict__ D, double* __restrict__ u) {
  const int64_t total = npair * R;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(t % R);
    const int64_t r = t / R;
    // invert r -> (mu, nu): mu is the largest a with a*nbf - a(a-1)/2 <= r
    int lo = 0, hi = nbf - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) / 2;
      if ((int64_t)mid * nbf - (int64_t)mid * (mid - 1) / 2 <= r) lo = mid; else hi = mid - 1;
    }
    const int mu = lo;
    const int nu = (int)(r - ((int64_t)mu * nbf - (int64_t)mu * (mu - 1) / 2)) + mu;
    const double v = D[(size_t)q * nbf * nbf + (size_t)mu * nbf + nu];
    u[t] = (mu == nu) ? v : 2.0 * v;
  }
}

void launch_pack_density(int nbf, int R, const double* d_D, double* d_u, cudaStream_t st) {
  const int64_t npair = (int64_t)nbf * (nbf + 1) / 2;
  int64_t blocks = (npair * R + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  count_launch();
  k_pack_density<<<(unsigned)blocks, 256, 0, st>>>(nbf, R, npair, d_D, d_u);
}

// J_q(mu, nu) = J_q(nu, mu) = scale * Ju[r - r0][q] for the unique pairs r in [r0, r1); J is
// zeroed first by the caller.  One thread per (r, q).
__global__ void k_unpack_J_range(int nbf, int R, int64_t r0, int64_t r1, const int* __restrict__ pair_mu,
                                 const int* __restrict__ pair_nu, const double* __restrict__ Ju, double scale,
                                 double* __restrict__ J, int* status) {
  const int64_t total = (r1 - r0) * R;
  bool bad = false;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = r0 + t / R;
    const int q = (int)(t % R);
    const int mu = pair_mu[r], nu = pair_nu[r];
    const double v = scale * Ju[t];
    bad |= !isfinite(v);
    J[(size_t)q * nbf * nbf + (size_t)mu * nbf + nu] = v;
    J[(size_t)q * nbf * nbf + (size_t)nu * nbf + mu] = v;
  }
  latch_nonfinite_warp(status, bad);
}

void launch_unpack_J_range(const PairTable& t, int nbf, int R, int64_t r0, int64_t r1, const double* d_Ju, double scale,
                           double* d_J, int* d_status, cudaStream_t st) {
  if (r1 <= r0) return;
  const int64_t total = (r1 - r0) * R;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  count_launch();
  k_unpack_J_range<<<(unsigned)blocks, 256, 0, st>>>(nbf, R, r0, r1, t.pair_mu, t.pair_nu, d_Ju, scale, d_J, d_status);
}

// J_q(mu, nu) = J_q(nu, mu) = scale * Ju[r][q].
__global__ void k_unpack_J(int nbf, int R, const double* __restrict__ Ju, double scale, double* __restrict__ J,
                           int* status) {
  const int64_t total = (int64_t)R * nbf * nbf;
  bool bad = false;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(t / ((int64_t)nbf * nbf));
    const int mu = (int)((t / nbf) % nbf), nu = (int)(t % nbf);
    const double v = scale * Ju[pair_idx(nbf, mu, nu) * R + q];
    bad |= !isfinite(v);
    J[t] = v;
  }
  latch_nonfinite_warp(status, bad);
}

void launch_unpack_J(int nbf, int R, const double* d_Ju, double scale, double* d_J, int* d_status, cudaStream_t st) {
  const int64_t total = (int64_t)R * nbf * nbf;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  count_launch();
  k_unpack_J<<<(unsigned)blocks, 256, 0, st>>>(nbf, R, d_Ju, scale, d_J, d_status);
}

}  // namespace lrtei
