// k_hadamard.cu -- FP64 CUDA-core form of Theorem 1 / Algorithm 1 (entry-wise Hadamard form):
//   B_u(r, c) = (w/sqrt(pi)) sum_p w_p sum_{j in r} sum_{j' in c} c_j c_j' prod_d (T_{d,p}(j,:) . S_d(j',:))
// with T_{d,p} = S_d A_d^(p) computed once per plan.  The sum over the quadrature nodes is
// Neumaier-compensated in FP64.  This is the FP64 CUDA-core form of the contraction; on the tensor
// cores the same B comes from the Khatri-Rao factored form (k_tcgen05.cu) or, for bases with one
// primitive pair per unique pair, from the tensor-core Hadamard form (k_tc_hadamard.cu).
#include "lrtei_internal.h"

namespace lrtei {

// T[d][p][row][b] = sum_a S[d][row][a] C[d][p][a][b]; one thread per (d, p, row, b).
__global__ void k_tmat(int64_t nrows, int n, int P, const double* __restrict__ S, const double* __restrict__ C,
                       double* __restrict__ T) {
  const int64_t total = 3LL * P * nrows * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(t % n);
    const int64_t row = (t / n) % nrows;
    const int p = (int)((t / n / nrows) % P);
    const int d = (int)(t / n / nrows / P);
    const double* s = S + ((size_t)d * nrows + row) * n;
    const double* c = C + ((size_t)d * P + p) * n * n;
    double acc = 0.0;
    for (int a = 0; a < n; ++a) acc += s[a] * c[a * n + b];
    T[t] = acc;
  }
}

void launch_tmat(int64_t nrows, int n, int P, const double* d_S, const double* d_C, double* d_T, cudaStream_t st) {
  const int64_t total = 3LL * P * nrows * n;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  count_launch();
  k_tmat<<<blocks, 256, 0, st>>>(nrows, n, P, d_S, d_C, d_T);
}

__device__ double hadamard_entry(int64_t r, int64_t c, int n, int P, int64_t nrows, const int64_t* __restrict__ pair_row,
                                 const double* __restrict__ row_c, const double* __restrict__ S,
                                 const double* __restrict__ T, const double* __restrict__ w) {
  const int64_t j0 = pair_row[r], j1 = pair_row[r + 1];
  const int64_t k0 = pair_row[c], k1 = pair_row[c + 1];
  double s = 0.0, comp = 0.0;
  for (int p = 0; p < P; ++p) {
    double acc = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
      const double cj = row_c[j];
      for (int64_t k = k0; k < k1; ++k) {
        double prod = cj * row_c[k];
        for (int d = 0; d < 3; ++d) {
          const double* tj = T + (((size_t)d * P + p) * nrows + j) * n;
          const double* sk = S + ((size_t)d * nrows + k) * n;
          double g = 0.0;
          for (int b = 0; b < n; ++b) g += tj[b] * sk[b];
          prod *= g;
        }
        acc += prod;
      }
    }
    const double term = w[p] * acc;
    const double tsum = s + term;
    comp += (fabs(s) >= fabs(term)) ? (s - tsum) + term : (term - tsum) + s;
    s = tsum;
  }
  return s + comp;
}

__global__ void k_hadamard_pairs(int n, int P, int64_t nrows, const int64_t* pair_row, const double* row_c,
                                 const double* S, const double* T, const double* w, double pref, const int64_t* rr,
                                 const int64_t* cc, int64_t count, double* out, int* status) {
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // every thread of the block runs the same number of iterations, so the warp vote is convergent
  const int64_t iters = (count + stride - 1) / stride;
  for (int64_t it = 0; it < iters; ++it) {
    const int64_t e = it * stride + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < count) {
      const int64_t r = rr[e], c = cc[e];
      if (r < 0 || c < 0) {
        out[e] = __longlong_as_double(0x7FF8000000000000LL);  // an index outside the basis
      } else {
        const double v = pref * hadamard_entry(r, c, n, P, nrows, pair_row, row_c, S, T, w);
        bad |= !isfinite(v);
        out[e] = v;
      }
    }
  }
  latch_nonfinite_warp(status, bad);
}

// Few entries: one warp per entry, the lanes share the quadrature nodes (p = lane, lane + 32, ...)
// and their partial node sums are added by a warp reduction.
__global__ void k_hadamard_pairs_warp(int n, int P, int64_t nrows, const int64_t* __restrict__ pair_row,
                                      const double* __restrict__ row_c, const double* __restrict__ S,
                                      const double* __restrict__ T, const double* __restrict__ w, double pref,
                                      const int64_t* rr, const int64_t* cc, int64_t count, double* out,
                                      int* status) {
  const int lane = threadIdx.x & 31;
  const int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (e >= count) return;  // whole warps: e is uniform across the warp
  const int64_t r = rr[e], c = cc[e];
  if (r < 0 || c < 0) {  // an index outside the basis
    if (lane == 0) out[e] = __longlong_as_double(0x7FF8000000000000LL);
    return;
  }
  const int64_t j0 = pair_row[r], j1 = pair_row[r + 1], k0 = pair_row[c], k1 = pair_row[c + 1];
  double s = 0.0;
  for (int p = lane; p < P; p += 32) {
    double acc = 0.0;
    for (int64_t j = j0; j < j1; ++j)
      for (int64_t k = k0; k < k1; ++k) {
        double prod = row_c[j] * row_c[k];
        for (int d = 0; d < 3; ++d) {
          const double* tj = T + (((size_t)d * P + p) * nrows + j) * n;
          const double* sk = S + ((size_t)d * nrows + k) * n;
          double g = 0.0;
          for (int b = 0; b < n; ++b) g += tj[b] * sk[b];
          prod *= g;
        }
        acc += prod;
      }
    s += w[p] * acc;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    out[e] = pref * s;
    if (!isfinite(pref * s)) latch_status(status, (int)kDevNonFinite);
  }
}

void launch_hadamard_pairs(const PairTable& t, int n, int P, const double* d_S, const double* d_T,
                           const double* d_w, double pref, const int64_t* d_r, const int64_t* d_c, int64_t count,
                           double* d_out, int* d_status, cudaStream_t st) {
  if (count <= 0) return;
  count_launch();
  if (count < 152 * 128) {  // too few entries to fill the GPU one thread each
    const int64_t threads = count * 32;
    k_hadamard_pairs_warp<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(n, P, t.nrows, t.pair_row, t.row_c, d_S,
                                                                            d_T, d_w, pref, d_r, d_c, count, d_out, d_status);
    return;
  }
  int blocks = (int)((count + 127) / 128);
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_hadamard_pairs<<<blocks, 128, 0, st>>>(n, P, t.nrows, t.pair_row, t.row_c, d_S, d_T, d_w, pref, d_r, d_c, count,
                                          d_out, d_status);
}

// Rows [r0, r1) of B_u, all npair columns; blockIdx.y = row, threads over columns.
__global__ void k_hadamard_rows(int n, int P, int64_t nrows, int64_t npair, const int64_t* pair_row,
                                const double* row_c, const double* S, const double* T, const double* w, double pref,
                                int64_t r0, double* Bu, int64_t ld) {
  const int64_t r = r0 + blockIdx.y;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < npair; c += (int64_t)gridDim.x * blockDim.x)
    Bu[(size_t)(r - r0) * ld + c] = pref * hadamard_entry(r, c, n, P, nrows, pair_row, row_c, S, T, w);
}

void launch_hadamard_rows(const PairTable& t, int n, int P, const double* d_S, const double* d_T, const double* d_w,
                          double pref, int64_t r0, int64_t r1, double* d_Bu, int64_t ld, cudaStream_t st) {
  if (r1 <= r0) return;
  int64_t nr = r1 - r0;
  while (nr > 0) {
    int64_t chunk = nr > 65535 ? 65535 : nr;
    dim3 grid((unsigned)((t.npair + 127) / 128), (unsigned)chunk);
    count_launch();
    k_hadamard_rows<<<grid, 128, 0, st>>>(n, P, t.nrows, t.npair, t.pair_row, t.row_c, d_S, d_T, d_w, pref, r0, d_Bu,
                                         ld);
    r0 += chunk;
    d_Bu += chunk * ld;
    nr -= chunk;
  }
}

// The caller's indices are checked here, on the device: an index outside [0, nbf) gives the pair
// -1 (the entry kernels then write NaN and read nothing) and latches kDevBadIndex.
__global__ void k_idx4_to_pairs(int nbf, const int32_t* idx4, int64_t count, int64_t* r, int64_t* c, int* status) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pr = checked_pair_index(nbf, idx4[4 * e], idx4[4 * e + 1]);
    const int64_t pc = checked_pair_index(nbf, idx4[4 * e + 2], idx4[4 * e + 3]);
    if (pr < 0 || pc < 0) latch_status(status, (int)kDevBadIndex);
    r[e] = pr < 0 || pc < 0 ? -1 : pr;
    c[e] = pr < 0 || pc < 0 ? -1 : pc;
  }
}

void launch_idx4_to_pairs(int nbf, const int32_t* d_idx4, int64_t count, int64_t* d_r, int64_t* d_c, int* d_status,
                          cudaStream_t st) {
  if (count <= 0) return;
  int blocks = (int)((count + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  count_launch();
  k_idx4_to_pairs<<<blocks, 256, 0, st>>>(nbf, d_idx4, count, d_r, d_c, d_status);
}

}  // namespace lrtei
