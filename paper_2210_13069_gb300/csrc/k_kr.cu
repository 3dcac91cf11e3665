// k_kr.cu -- Khatri-Rao low-rank compression of the factored form (Section 6, "Compression by
// using low-rank methods": eq. SVD, then eq. approxepsilon), FP64 on the device.
//
// With one Chebyshev order n for every node, the moment matrix W~_d = S_d (rows of all primitive
// pairs, n columns) is shared by all nodes.  Its truncated SVD S_d ~ U_d V_d^T (V_d: n x R right
// singular vectors, U_d = S_d V_d) and the mixed-product property of the Khatri-Rao and Kronecker
// products give B ~ (w/sqrt(pi)) U~ [sum_p w_p (x)_d V_d^T A_d^(p) V_d] U~^T: the same factored
// form with S_d replaced by S_d V_d and A_d^(p) by V_d^T A_d^(p) V_d.
//
// The SVD is computed in two passes of one-block Jacobi eigen-solves on n x n Gram matrices:
//   pass 1: G = S^T S (FP64, fixed-order partial sums) -> G = Q0 diag Q0^T
//   pass 2: G1 = (S Q0)^T (S Q0), nearly diagonal and graded, -> Q1; V = Q0 Q1.
// Pass 1 alone resolves the small singular values only to eps * sigma_1^2 (absolute); Jacobi on
// the graded G1 of pass 2 resolves them to high relative accuracy (Demmel and Veselic, "Jacobi's
// method is more accurate than QR", SIAM J. Matrix Anal. Appl. 1992), so that the kept subspace
// is the one a direct SVD of S keeps.
#include <algorithm>

#include "lrtei_internal.h"

namespace lrtei {

constexpr int kGramRows = 64;     // rows of S staged per chunk
constexpr int kGramThreads = 256;

// Partial Gram matrices of X = S_d (or S_d Q_d): block b of dimension d = blockIdx.y sums the rows
// of chunks b, b + gridDim.x, ... into part[d][b][a][c] (all n x n entries, fixed order).
__global__ void __launch_bounds__(kGramThreads) k_gram_partial(int64_t nrows, int n, const double* __restrict__ S,
                                                             const double* __restrict__ Q, double* __restrict__ part) {
  extern __shared__ double sm[];
  double* Xs = sm;                        // [kGramRows][n] staged (rotated) rows
  double* Qs = sm + kGramRows * n;        // [n][n] (pass 2)
  double* Ss = Qs + (Q ? n * n : 0);      // [kGramRows][n] raw rows (pass 2)
  const int d = blockIdx.y;
  const double* Sd = S + (size_t)d * nrows * n;
  if (Q)
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) Qs[i] = Q[(size_t)d * n * n + i];
  const int nn = n * n;
  constexpr int kMaxPer = (kMaxN * kMaxN + kGramThreads - 1) / kGramThreads;
  double acc[kMaxPer];
#pragma unroll
  for (int k = 0; k < kMaxPer; ++k) acc[k] = 0.0;
  const int64_t nchunks = (nrows + kGramRows - 1) / kGramRows;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int64_t r0 = ch * kGramRows;
    const int rows = (int)(nrows - r0 < kGramRows ? nrows - r0 : kGramRows);
    __syncthreads();  // the previous chunk's products are done
    double* dst = Q ? Ss : Xs;
    for (int i = threadIdx.x; i < kGramRows * n; i += blockDim.x)
      dst[i] = (i / n) < rows ? Sd[(size_t)r0 * n + i] : 0.0;
    __syncthreads();
    if (Q) {  // X = S Q for the staged rows
      for (int i = threadIdx.x; i < kGramRows * n; i += blockDim.x) {
        const int r = i / n, c = i % n;
        double x = 0.0;
        for (int a = 0; a < n; ++a) x += Ss[r * n + a] * Qs[a * n + c];
        Xs[i] = x;
      }
      __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kMaxPer; ++k) {
      const int e = threadIdx.x + k * kGramThreads;
      if (e < nn) {
        const int a = e / n, c = e % n;
        double s = acc[k];
        for (int r = 0; r < kGramRows; ++r) s += Xs[r * n + a] * Xs[r * n + c];
        acc[k] = s;
      }
    }
  }
  double* out = part + ((size_t)d * gridDim.x + blockIdx.x) * nn;
#pragma unroll
  for (int k = 0; k < kMaxPer; ++k) {
    const int e = threadIdx.x + k * kGramThreads;
    if (e < nn) out[e] = acc[k];
  }
}

// G[d] = sum over the nblk partials, in block order.
__global__ void k_gram_reduce(int n, int nblk, const double* __restrict__ part, double* __restrict__ G) {
  const int d = blockIdx.y, nn = n * n;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[((size_t)d * nblk + b) * nn + e];
    G[(size_t)d * nn + e] = s;
  }
}

// Symmetric eigen-solve of G[d] (n x n) by parallel cyclic Jacobi, one block per dimension:
// every round rotates n/2 disjoint index pairs (round-robin ordering), rows first, then columns
// and the accumulated V.  V starts from V0 (or the identity) so that pass 2 returns Q0 Q1.
// relative != 0: a pair is rotated while |a_pq| > tol sqrt(|a_pp a_qq|) (graded matrices);
// otherwise while |a_pq| > tol max_i |a_ii|.  Output: eigenvalues descending (lam[d][i]) and the
// matching columns of V (Vout[d][a][i]).
__global__ void k_jacobi(int n, const double* __restrict__ G, const double* __restrict__ V0, int relative,
                         double tol, int max_sweeps, double* __restrict__ lam, double* __restrict__ Vout,
                         int* __restrict__ sweeps_out) {
  extern __shared__ double sm[];
  const int d = blockIdx.x;
  const int m = n + (n & 1);  // padded to even: index n (if any) is a dummy that is never rotated
  double* A = sm;             // [n][n]
  double* V = A + n * n;      // [n][n]
  double* cs = V + n * n;     // [m/2][2]
  int* pr = reinterpret_cast<int*>(cs + m);  // [m/2][2] pairs of the round
  int* order = pr + m;                       // [m] round-robin arrangement
  __shared__ double offmax;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    A[i] = G[(size_t)d * n * n + i];
    V[i] = V0 ? V0[(size_t)d * n * n + i] : ((i / n) == (i % n) ? 1.0 : 0.0);
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) order[i] = i;
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) {
      double mx = 0.0, dmax = 0.0;
      for (int i = 0; i < n; ++i) dmax = fmax(dmax, fabs(A[i * n + i]));
      for (int p = 0; p < n; ++p)
        for (int q = p + 1; q < n; ++q) {
          const double a = fabs(A[p * n + q]);
          const double ref = relative ? fmax(sqrt(fabs(A[p * n + p] * A[q * n + q])), 1e-30 * dmax) : dmax;
          mx = fmax(mx, ref > 0.0 ? a / ref : (a > 0.0 ? 1.0 : 0.0));
        }
      offmax = mx;
    }
    __syncthreads();
    if (offmax <= tol) break;
    for (int round = 0; round < m - 1; ++round) {
      if (threadIdx.x < m / 2) {
        const int t = threadIdx.x;
        int p = order[t], q = order[m - 1 - t];
        if (p > q) { const int x = p; p = q; q = x; }
        double c = 1.0, s = 0.0;
        if (q < n) {
          const double app = A[p * n + p], aqq = A[q * n + q], apq = A[p * n + q];
          const double ref = relative ? sqrt(fabs(app * aqq)) : 0.0;  // skip only negligible pairs
          if (apq != 0.0 && fabs(apq) > (relative ? tol * 1e-2 * ref : 0.0)) {
            const double theta = (aqq - app) / (2.0 * apq);
            double tt;
            if (fabs(theta) > 1e150)
              tt = 0.5 / theta;
            else
              tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(tt * tt + 1.0);
            s = tt * c;
          }
        }
        pr[2 * t] = p;
        pr[2 * t + 1] = q;
        cs[2 * t] = c;
        cs[2 * t + 1] = s;
      }
      __syncthreads();
      // rows: A <- J^T A for every pair (disjoint pairs commute)
      for (int i = threadIdx.x; i < (m / 2) * n; i += blockDim.x) {
        const int t = i / n, k = i % n;
        const int p = pr[2 * t], q = pr[2 * t + 1];
        if (q >= n) continue;
        const double c = cs[2 * t], s = cs[2 * t + 1];
        const double ap = A[p * n + k], aq = A[q * n + k];
        A[p * n + k] = c * ap - s * aq;
        A[q * n + k] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int i = threadIdx.x; i < (m / 2) * n; i += blockDim.x) {
        const int t = i / n, k = i % n;
        const int p = pr[2 * t], q = pr[2 * t + 1];
        if (q >= n) continue;
        const double c = cs[2 * t], s = cs[2 * t + 1];
        const double ap = A[k * n + p], aq = A[k * n + q];
        A[k * n + p] = c * ap - s * aq;
        A[k * n + q] = s * ap + c * aq;
        const double vp = V[k * n + p], vq = V[k * n + q];
        V[k * n + p] = c * vp - s * vq;
        V[k * n + q] = s * vp + c * vq;
      }
      __syncthreads();
      // next round-robin arrangement: order[0] stays, the rest rotate by one
      if (threadIdx.x == 0) {
        const int last = order[m - 1];
        for (int i = m - 1; i > 1; --i) order[i] = order[i - 1];
        order[1] = last;
      }
      __syncthreads();
    }
  }
  // eigenvalues descending, with their columns of V (selection order by one thread)
  if (threadIdx.x == 0) {
    for (int i = 0; i < n; ++i) order[i] = i;
    for (int i = 0; i < n; ++i) {
      int best = i;
      for (int j = i + 1; j < n; ++j)
        if (A[order[j] * n + order[j]] > A[order[best] * n + order[best]]) best = j;
      const int x = order[i];
      order[i] = order[best];
      order[best] = x;
    }
    if (sweeps_out) sweeps_out[d] = sweep;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) lam[(size_t)d * n + i] = A[order[i] * n + order[i]];
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int a = i / n, k = i % n;
    Vout[(size_t)d * n * n + i] = V[a * n + order[k]];
  }
}

// S_new[d][row][k] = sum_a S[d][row][a] V[d][a][k], k < R.
__global__ void k_project_S(int64_t nrows, int n, int R, const double* __restrict__ S, const double* __restrict__ V,
                            double* __restrict__ Snew) {
  const int64_t total = 3 * nrows * R;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(t % R);
    const int64_t dr = t / R;  // d nrows + row
    const int d = (int)(dr / nrows);
    const double* s = S + (size_t)dr * n;
    const double* v = V + (size_t)d * n * n;
    double x = 0.0;
    for (int a = 0; a < n; ++a) x += s[a] * v[a * n + k];
    Snew[t] = x;
  }
}

// C_new[d][p] = V_d^T C[d][p] V_d (R x R); one block per (p, d).
__global__ void k_project_C(int n, int P, int R, const double* __restrict__ C, const double* __restrict__ V,
                            double* __restrict__ Cnew) {
  extern __shared__ double T[];  // [n][R] = C V
  const int p = blockIdx.x, d = blockIdx.y;
  const double* c = C + ((size_t)d * P + p) * n * n;
  const double* v = V + (size_t)d * n * n;
  for (int i = threadIdx.x; i < n * R; i += blockDim.x) {
    const int a = i / R, k = i % R;
    double x = 0.0;
    for (int b = 0; b < n; ++b) x += c[a * n + b] * v[b * n + k];
    T[i] = x;
  }
  __syncthreads();
  double* out = Cnew + ((size_t)d * P + p) * R * R;
  for (int i = threadIdx.x; i < R * R; i += blockDim.x) {
    const int k = i / R, l = i % R;
    double x = 0.0;
    for (int a = 0; a < n; ++a) x += v[a * n + k] * T[a * R + l];
    out[i] = x;
  }
}

// Right singular vectors and squared singular values of the three n-column moment matrices.
// d_part: scratch of kr_gram_blocks() * 3 * n * n doubles; d_G, d_V1: 3 n n; d_lam: 3 n
// (descending); d_V: 3 n n (columns = right singular vectors, descending).
int kr_gram_blocks(int64_t nrows) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(152 * 2, (nrows + kGramRows - 1) / kGramRows));
}

cudaError_t launch_kr_svd(int64_t nrows, int n, const double* d_S, double* d_part, double* d_G, double* d_V1,
                          double* d_lam, double* d_V, int* d_sweeps, cudaStream_t st) {
  const int nblk = kr_gram_blocks(nrows);
  const size_t sm1 = sizeof(double) * (size_t)kGramRows * n;
  const size_t sm2 = sizeof(double) * ((size_t)2 * kGramRows * n + (size_t)n * n);
  cudaError_t e = cudaFuncSetAttribute(k_gram_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
  if (e != cudaSuccess) return e;
  const int m = n + (n & 1);
  const size_t smj = sizeof(double) * ((size_t)2 * n * n + m) + sizeof(int) * (size_t)2 * m;
  e = cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smj);
  if (e != cudaSuccess) return e;
  const dim3 gg((unsigned)nblk, 3);
  const dim3 gr((unsigned)((n * n + 255) / 256), 3);
  // pass 1: absolute criterion
  count_launch();
  k_gram_partial<<<gg, kGramThreads, sm1, st>>>(nrows, n, d_S, nullptr, d_part);
  count_launch();
  k_gram_reduce<<<gr, 256, 0, st>>>(n, nblk, d_part, d_G);
  count_launch();
  k_jacobi<<<3, 256, smj, st>>>(n, d_G, nullptr, 0, 1e-15, 60, d_lam, d_V1, d_sweeps);
  // pass 2: the Gram matrix of S Q0, relative criterion, V accumulated onto Q0
  count_launch();
  k_gram_partial<<<gg, kGramThreads, sm2, st>>>(nrows, n, d_S, d_V1, d_part);
  count_launch();
  k_gram_reduce<<<gr, 256, 0, st>>>(n, nblk, d_part, d_G);
  count_launch();
  k_jacobi<<<3, 256, smj, st>>>(n, d_G, d_V1, 1, 1e-15, 60, d_lam, d_V, d_sweeps ? d_sweeps + 3 : nullptr);
  return cudaGetLastError();
}

cudaError_t launch_kr_project(int64_t nrows, int n, int P, int R, const double* d_S, const double* d_C,
                              const double* d_V, double* d_Snew, double* d_Cnew, cudaStream_t st) {
  const int64_t total = 3 * nrows * R;
  if (total > 0) {
    count_launch();
    k_project_S<<<(unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32), 256, 0, st>>>(nrows, n, R, d_S, d_V,
                                                                                            d_Snew);
  }
  count_launch();
  k_project_C<<<dim3((unsigned)P, 3), 256, sizeof(double) * (size_t)n * R, st>>>(n, P, R, d_C, d_V, d_Cnew);
  return cudaGetLastError();
}

}  // namespace lrtei
