// k_adaptive.cu -- the adaptive choice of the integration domain (Section 6, "Adaptive approach
// for the choice of the integration domain"): every unique basis pair belongs to one partition s,
// whose cube [c - b_s, c + b_s]^3 holds the numerical support of all its primitive pairs; its
// moment matrices are integrated over that cube, and the kernel between partitions s and t is
// interpolated on the two cubes' Chebyshev grids (coefficient blocks A^(p)_{st}, A_{ts} = A_{st}^T).
//   B(mu nu, ka la) = (w/sqrt(pi)) sum_p w_p sum_{j, j'} c_j c_j' prod_d (S_d(j) A^(p)_{st,d} S_d(j')^T)
// The factored form of a partition block is B_{st} = F_s K_{st} F_t^T; the host code gathers each
// partition's rows of F_u, runs the block products, and scatters the blocks into B_u.
#include <algorithm>

#include "lrtei_internal.h"

namespace lrtei {

__global__ void k_gather_rows(const double* __restrict__ in, const int64_t* __restrict__ idx, int64_t count, int64_t len,
                              double* __restrict__ out) {
  for (int64_t i = blockIdx.x; i < count; i += gridDim.x) {
    const double* src = in + idx[i] * len;
    double* dst = out + i * len;
    for (int64_t k = threadIdx.x; k < len; k += blockDim.x) dst[k] = src[k];
  }
}

void launch_gather_rows(const double* d_in, const int64_t* d_idx, int64_t count, int64_t len, double* d_out,
                        cudaStream_t st) {
  if (count <= 0) return;
  count_launch();
  k_gather_rows<<<(unsigned)std::min<int64_t>(count, 152 * 16), 256, 0, st>>>(d_in, d_idx, count, len, d_out);
}

// Block (i, j) of the partition pair into B_u; the mirror writes B_u[cols[j]][rows[i]], one block
// row of threads along j for the direct write, along i (consecutive rows of blk) for the mirror.
__global__ void k_scatter_block(const double* __restrict__ blk, int64_t ldb, const int64_t* __restrict__ rows,
                                int64_t nr, const int64_t* __restrict__ cols, int64_t nc, double* __restrict__ Bu,
                                int64_t ldu, int mirror) {
  const int64_t total = nr * nc;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / nc, j = t % nc;
    Bu[rows[i] * ldu + cols[j]] = blk[i * ldb + j];
  }
  if (!mirror) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / nr, i = t % nr;
    Bu[cols[j] * ldu + rows[i]] = blk[i * ldb + j];
  }
}

void launch_scatter_block(const double* d_blk, int64_t ldb, const int64_t* d_rows, int64_t nr, const int64_t* d_cols,
                          int64_t nc, double* d_Bu, int64_t ldu, bool mirror, cudaStream_t st) {
  if (nr <= 0 || nc <= 0) return;
  count_launch();
  const int64_t b = std::min<int64_t>((nr * nc + 255) / 256, 152 * 32);
  k_scatter_block<<<(unsigned)b, 256, 0, st>>>(d_blk, ldb, d_rows, nr, d_cols, nc, d_Bu, ldu, mirror ? 1 : 0);
}

__global__ void k_scatter_rows(const double* __restrict__ blk, const int64_t* __restrict__ rows, int64_t nr, int64_t R,
                               double* __restrict__ Ju) {
  const int64_t total = nr * R;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    Ju[rows[t / R] * R + t % R] = blk[t];
}

void launch_scatter_rows(const double* d_blk, const int64_t* d_rows, int64_t nr, int64_t R, double* d_Ju,
                         cudaStream_t st) {
  if (nr <= 0 || R <= 0) return;
  count_launch();
  const int64_t b = std::min<int64_t>((nr * R + 255) / 256, 152 * 32);
  k_scatter_rows<<<(unsigned)b, 256, 0, st>>>(d_blk, d_rows, nr, R, d_Ju);
}

// Algorithm 1 per entry with the partition blocks of the Chebyshev coefficients; Neumaier node sum.
__global__ void k_adaptive_entries(int n, int P, int npart, int64_t nrows, const int64_t* __restrict__ pair_row,
                                   const double* __restrict__ row_c, const int* __restrict__ pair_part,
                                   const double* __restrict__ S, const double* __restrict__ Cpp,
                                   const double* __restrict__ w, double pref, const int64_t* __restrict__ rr,
                                   const int64_t* __restrict__ cc, int64_t count, double* __restrict__ out,
                                   int* status) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = rr[e], c = cc[e];
    if (r < 0 || c < 0) {  // an index outside the basis
      out[e] = __longlong_as_double(0x7FF8000000000000LL);
      continue;
    }
    const double* C = Cpp + (size_t)(pair_part[r] * npart + pair_part[c]) * 3 * P * n * n;
    const int64_t j0 = pair_row[r], j1 = pair_row[r + 1], k0 = pair_row[c], k1 = pair_row[c + 1];
    double s = 0.0, comp = 0.0;
    for (int p = 0; p < P; ++p) {
      double acc = 0.0;
      for (int64_t j = j0; j < j1; ++j)
        for (int64_t k = k0; k < k1; ++k) {
          double prod = row_c[j] * row_c[k];
          for (int d = 0; d < 3; ++d) {
            const double* sj = S + ((size_t)d * nrows + j) * n;
            const double* sk = S + ((size_t)d * nrows + k) * n;
            const double* A = C + ((size_t)d * P + p) * n * n;
            double g = 0.0;
            for (int a = 0; a < n; ++a) {
              double t = 0.0;
              for (int b = 0; b < n; ++b) t += A[a * n + b] * sk[b];
              g += sj[a] * t;
            }
            prod *= g;
          }
          acc += prod;
        }
      const double term = w[p] * acc;
      const double tsum = s + term;
      comp += (fabs(s) >= fabs(term)) ? (s - tsum) + term : (term - tsum) + s;
      s = tsum;
    }
    out[e] = pref * (s + comp);
    if (!isfinite(out[e])) latch_status(status, (int)kDevNonFinite);
  }
}

void launch_adaptive_entries(const PairTable& t, int n, int P, int npart, const int* d_pair_part, const double* d_S,
                             const double* d_Cpp, const double* d_w, double pref, const int64_t* d_r,
                             const int64_t* d_c, int64_t count, double* d_out, int* d_status, cudaStream_t st) {
  if (count <= 0) return;
  count_launch();
  const int64_t b = std::min<int64_t>((count + 127) / 128, 152 * 32);
  k_adaptive_entries<<<(unsigned)b, 128, 0, st>>>(n, P, npart, t.nrows, t.pair_row, t.row_c, d_pair_part, d_S, d_Cpp,
                                                  d_w, pref, d_r, d_c, count, d_out, d_status);
}

}  // namespace lrtei
