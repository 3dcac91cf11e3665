// k_setup.cu -- FP64 set-up kernels of a plan: Gauss-Legendre nodes (eq. TEI2, Proposition 3),
// Chebyshev coefficient matrices (Definition 1, eq. chebcheb), basis normalisation, the
// primitive-pair table (Proposition 1) and the 1D moment matrices S_d (eq. defV).
//
// All of this is FP64 on the device.  The moment integrals are computed by an 8-panel (16 above
// n = 32), 16-point Gauss-Legendre rule over the window |x - P| <= 9/sqrt(p) of each primitive-pair
// Gaussian, clipped to the box: one warp per (row, dimension), two panels per step (one per
// half-warp), one lane per quadrature point.
#include <math.h>

#include <algorithm>

#include "lrtei_internal.h"

namespace lrtei {

// ------------------------------------------------------------------ Gauss-Legendre ----
// One thread per root.  Initial guess from Tricomi's asymptotic formula, Newton steps on the
// Legendre polynomial with its derivative carried along the three-term recurrence
// (P'_k = k P_{k-1} + x P'_{k-1}), weight 2 / ((1 - x)(1 + x) P'_N(x)^2).  The recurrence is taken
// as P_k = x P_{k-1} + q_k (x P_{k-1} - P_{k-2}) with q_k = (k - 1) / k tabulated per block, so that
// no FP64 division runs inside the loop.  (The equivalent form
// 2 (1 - x^2) / (N P_{N-1}(x))^2 loses digits at the outermost nodes for large N: 8e-12 relative at
// N = 96, 4e-11 at N = 128, against 1e-13 for the derivative recurrence.)
constexpr int kMaxGL = 256;  // largest rule k_gauss_legendre tabulates q_k for

__global__ void k_gauss_legendre(int N, double* z, double* w) {
  __shared__ double q[kMaxGL + 1];
  for (int k = threadIdx.x; k <= N && k <= kMaxGL; k += blockDim.x) q[k] = k >= 1 ? (double)(k - 1) / k : 0.0;
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double pi = 3.141592653589793238;
  double th = pi * (4.0 * (i + 1) - 1.0) / (4.0 * N + 2.0);
  double x = (1.0 - 1.0 / (8.0 * N * N) + 1.0 / (8.0 * N * N * N)) * cos(th);
  double dp = 1.0;
  // Newton converges quadratically: once a step is below 1e-11 the next one leaves an error far
  // below rounding, so one more step ends the iteration (the 100-step cap only bounds the loop)
  bool last = false;
  for (int it = 0; it < 100; ++it) {
    double a = 1.0, b = x, db = 1.0;  // P_0, P_1, P_1'
    for (int k = 2; k <= N; ++k) {
      const double xb = x * b;
      const double c = fma(q[k], xb - a, xb);
      const double dc = k * b + x * db;
      a = b;
      b = c;
      db = dc;
    }
    const double pn = (N == 0) ? 1.0 : b;
    dp = (N == 0) ? 0.0 : db;
    const double dx = pn / dp;
    x -= dx;
    if (last || dx == 0.0) break;
    last = fabs(dx) <= 1e-11;
  }
  {
    double a = 1.0, b = x, db = 1.0;
    for (int k = 2; k <= N; ++k) {
      const double xb = x * b;
      const double c = fma(q[k], xb - a, xb);
      const double dc = k * b + x * db;
      a = b;
      b = c;
      db = dc;
    }
    dp = db;
  }
  // roots come out in descending order of x; store ascending
  z[N - 1 - i] = x;
  w[N - 1 - i] = 2.0 / ((1.0 - x) * (1.0 + x) * dp * dp);
}

void launch_gauss_legendre(int N, double* d_z, double* d_w, cudaStream_t st) {
  if (N < 1 || N > kMaxGL) return;  // callers keep N <= kMaxP (128) and the 32-point panel rule
  count_launch();
  k_gauss_legendre<<<(N + 63) / 64, 64, 0, st>>>(N, d_z, d_w);
}

__global__ void k_nodes_map(int P, double omega, const double* z, double* s) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P) s[i] = 0.5 * omega * (1.0 + z[i]);
}

void launch_nodes_map(int P, double omega, const double* d_z, double* d_s, cudaStream_t st) {
  count_launch();
  k_nodes_map<<<(P + 127) / 128, 128, 0, st>>>(P, omega, d_z, d_s);
}

// ---------------------------------------------------------------- Chebyshev coefficients ----
// One block per (d, p).  With Tm(a, k) = T_a(u_k) = cos(a (2k+1) pi / (2n)) and
// F(k, k') = exp(-(s_p b_d)^2 (u_k - u_k')^2), alpha = (c_ab / n^2) (Tm F Tm^T)(a, b).
// Two intervals (the adaptive boxes of Section 6): x = c + hx_d u on one side, y = c + hy_d v on
// the other, F(k, k') = exp(-s_p^2 (hx_d u_k - hy_d u_k')^2); hy3 == NULL means hy3 = hx3.
//
// The first-kind grid is mirror-symmetric: node kb = n - 1 - k has u_kb = -u_k, so
// T_a(u_kb) = (-1)^a T_a(u_k) and F(kb, kb') = F(k, k'), F(kb, k') = F(k, kb') (both intervals flip
// together).  Folding the double sum over the mirror pairs k < h = floor(n/2) (plus the middle node
// km = (n-1)/2, u = 0, when n is odd):
//   Y_b(k) = sum_k' F(k, k') T_b(u_k') = sum_{k' < h} T_b(u_k') (F(k, k') + (-1)^b F(k, kb'))
//            [+ T_b(0) F(k, km)],
//   Y_b(kb) = (-1)^b Y_b(k), so alpha_ab = 0 when a + b is odd, and otherwise
//   alpha_ab = (c_ab / n^2) (2 sum_{k < h} T_a(u_k) Y_b(k) [+ T_a(0) Y_b(km)]).
// The same terms as the full double sum, regrouped: a quarter of its multiply-adds, half its exps.
__global__ void k_cheb_coeff(int n, int P, const double* s, const double* half3, const double* hy3, double* C) {
  extern __shared__ double sm[];
  const int h = n / 2, hh = (n + 1) / 2;  // mirror pairs; rows with the middle node
  const bool odd = (n & 1) != 0;
  double* Tm = sm;             // n x hh : T_a(u_k), k < hh
  double* Fp = Tm + n * hh;    // hh x hh : F(k, k') + F(k, kb') (k' < h); F(k, km) in column km
  double* Fm = Fp + hh * hh;   // hh x hh : F(k, k') - F(k, kb') (k' < h)
  double* Y = Fm + hh * hh;    // hh x n : Y_b(k)
  const int d = blockIdx.x / P, p = blockIdx.x % P;
  const double pi = 3.141592653589793238;
  const double sb = s[p] * half3[d];
  const bool cross = hy3 != nullptr && hy3[d] != half3[d];
  const double hx = half3[d], hy = cross ? hy3[d] : hx;
  for (int t = threadIdx.x; t < n * hh; t += blockDim.x) {
    const int a = t / hh, k = t % hh;
    Tm[t] = cos(a * (2.0 * k + 1.0) * pi / (2.0 * n));
  }
  for (int t = threadIdx.x; t < hh * hh; t += blockDim.x) {
    const int k = t / hh, kk = t % hh;
    const double uk = cos((2.0 * k + 1.0) * pi / (2.0 * n));
    const double vk = cos((2.0 * kk + 1.0) * pi / (2.0 * n));
    const double df = cross ? s[p] * (hx * uk - hy * vk) : sb * (uk - vk);
    const double f = exp(-df * df);
    if (kk < h) {
      const double vb = cos((2.0 * (n - 1 - kk) + 1.0) * pi / (2.0 * n));
      const double dg = cross ? s[p] * (hx * uk - hy * vb) : sb * (uk - vb);
      const double g = exp(-dg * dg);
      Fp[t] = f + g;
      Fm[t] = f - g;
    } else {  // the middle node's column (n odd)
      Fp[t] = f;
      Fm[t] = 0.0;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < hh * n; t += blockDim.x) {
    const int k = t / n, b = t % n;
    const double* F = (b & 1) ? Fm : Fp;
    const int kend = (b & 1) ? h : hh;
    double acc = 0.0;
    for (int kk = 0; kk < kend; ++kk) acc += F[k * hh + kk] * Tm[b * hh + kk];
    Y[t] = acc;
  }
  __syncthreads();
  double* out = C + (size_t)blockIdx.x * n * n;
  const double inv = 1.0 / ((double)n * n);
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int a = t / n, b = t % n;
    double v = 0.0;
    if (((a + b) & 1) == 0) {
      double acc = 0.0;
      for (int k = 0; k < h; ++k) acc += Tm[a * hh + k] * Y[k * n + b];
      acc *= 2.0;
      if (odd) acc += Tm[a * hh + h] * Y[h * n + b];
      const double cab = (a == 0 ? 1.0 : 2.0) * (b == 0 ? 1.0 : 2.0);
      v = cab * inv * acc;
    }
    out[t] = v;
  }
}

static size_t cheb_smem(int n) {
  const size_t hh = (n + 1) / 2;
  return sizeof(double) * (2 * n * hh + 2 * hh * hh);
}

void launch_cheb_coeff(int n, int P, const double* d_s, const double* d_half3, double* d_C, cudaStream_t st) {
  size_t smem = cheb_smem(n);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_cheb_coeff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  count_launch();
  k_cheb_coeff<<<3 * P, 256, smem, st>>>(n, P, d_s, d_half3, nullptr, d_C);
}

void launch_cheb_coeff_cross(int n, int P, const double* d_s, const double* d_hx3, const double* d_hy3, double* d_C,
                             cudaStream_t st) {
  size_t smem = cheb_smem(n);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_cheb_coeff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  count_launch();
  k_cheb_coeff<<<3 * P, 256, smem, st>>>(n, P, d_s, d_hx3, d_hy3, d_C);
}

// ------------------------------------------------------------------ normalisation ----
__device__ __forceinline__ double dfact_d(int k) {
  double r = 1.0;
  for (int i = k; i > 1; i -= 2) r *= i;
  return r;
}

// One thread per basis function: primitive normalisation (2a/pi)^{3/4} (4a)^{L/2} / sqrt(prod
// (2l_d - 1)!!) and contraction normalisation so that the contracted component has unit norm:
// the overlap of two normalised primitives of one component is (2 sqrt(ab)/(a+b))^{L + 3/2}.
__global__ void k_normalise(int nbf, const int* bf_shell, const int* bf_pow, const int* shell_nprim,
                            const int* shell_poff, const double* exps, const double* coefs, const int* bf_coff,
                            double* ncoef) {
  int mu = blockIdx.x * blockDim.x + threadIdx.x;
  if (mu >= nbf) return;
  const int sh = bf_shell[mu];
  const int K = shell_nprim[sh], off = shell_poff[sh];
  const int lx = bf_pow[3 * mu], ly = bf_pow[3 * mu + 1], lz = bf_pow[3 * mu + 2];
  const int L = lx + ly + lz;
  const double pi = 3.141592653589793238;
  double denom = sqrt(dfact_d(2 * lx - 1) * dfact_d(2 * ly - 1) * dfact_d(2 * lz - 1));
  double* out = ncoef + bf_coff[mu];
  for (int k = 0; k < K; ++k) {
    double a = exps[off + k];
    out[k] = coefs[off + k] * pow(2.0 * a / pi, 0.75) * pow(4.0 * a, 0.5 * L) / denom;
  }
  double S = 0.0;
  for (int k = 0; k < K; ++k)
    for (int q = 0; q < K; ++q) {
      double a = exps[off + k], b = exps[off + q];
      double r = 2.0 * sqrt(a * b) / (a + b);
      S += coefs[off + k] * coefs[off + q] * pow(r, L + 1.5);
    }
  // S is the self-overlap in units of normalised primitives; scale all coefficients.
  double inv = 1.0 / sqrt(S);
  for (int k = 0; k < K; ++k) out[k] *= inv;
}

void launch_normalise(int nbf, const int* d_bf_shell, const int* d_bf_pow, const int* d_shell_nprim,
                      const int* d_shell_poff, const double* d_exps, const double* d_coefs, const int* d_bf_coff,
                      double* d_ncoef, cudaStream_t st) {
  count_launch();
  k_normalise<<<(nbf + 127) / 128, 128, 0, st>>>(nbf, d_bf_shell, d_bf_pow, d_shell_nprim, d_shell_poff, d_exps,
                                                 d_coefs, d_bf_coff, d_ncoef);
}

// ------------------------------------------------------------------ pair table ----
// One block per unique pair (mu <= nu); threads over its I_mu I_nu primitive pairs.
// Gaussian product rule (Proposition 1): exp(-a(x-A)^2) exp(-b(x-B)^2) = K_AB exp(-p (x-P)^2).
__global__ void k_pair_rows(int64_t npair, const int* pair_mu, const int* pair_nu, const int64_t* pair_row,
                            const int* pair_I, const uint8_t* row_prim,
                            const int* bf_shell, const int* bf_pow, const int* shell_nprim, const int* shell_poff,
                            const double* shell_center, const double* exps, const int* bf_coff,
                            const double* ncoef, int64_t nrows, int* row_pair, double* row_c, double* row_p,
                            double* row_P, double* row_K, double* row_A, double* row_B, int8_t* row_pa,
                            int8_t* row_pb) {
  const int64_t r = blockIdx.x;
  if (r >= npair) return;
  const int mu = pair_mu[r], nu = pair_nu[r];
  const int sm = bf_shell[mu], sn = bf_shell[nu];
  const int64_t base = pair_row[r];
  for (int j = threadIdx.x; j < pair_I[r]; j += blockDim.x) {  // the pair's kept primitive pairs
    const int64_t row = base + j;
    const int j1 = row_prim[row] >> 4, j2 = row_prim[row] & 15;
    const double a = exps[shell_poff[sm] + j1], b = exps[shell_poff[sn] + j2];
    const double p = a + b;
    row_pair[row] = (int)r;
    row_c[row] = ncoef[bf_coff[mu] + j1] * ncoef[bf_coff[nu] + j2];
    row_p[row] = p;
    for (int d = 0; d < 3; ++d) {
      const double A = shell_center[3 * sm + d], B = shell_center[3 * sn + d];
      row_P[d * nrows + row] = A + b / p * (B - A);  // exactly A for one centre
      row_K[d * nrows + row] = exp(-a * b / p * (A - B) * (A - B));
      row_A[d * nrows + row] = A;
      row_B[d * nrows + row] = B;
      row_pa[d * nrows + row] = (int8_t)bf_pow[3 * mu + d];
      row_pb[d * nrows + row] = (int8_t)bf_pow[3 * nu + d];
    }
  }
}

void launch_pair_rows(const PairTable& t, const int* d_bf_shell, const int* d_bf_pow, const int* d_shell_nprim,
                      const int* d_shell_poff, const double* d_shell_center, const double* d_exps,
                      const int* d_bf_coff, const double* d_ncoef, cudaStream_t st) {
  count_launch();
  k_pair_rows<<<(unsigned)t.npair, 64, 0, st>>>(t.npair, t.pair_mu, t.pair_nu, t.pair_row, t.pair_I, t.row_prim,
                                                d_bf_shell, d_bf_pow,
                                                d_shell_nprim, d_shell_poff, d_shell_center, d_exps, d_bf_coff,
                                                d_ncoef, t.nrows, t.row_pair, t.row_c, t.row_p, t.row_P, t.row_K,
                                                t.row_A, t.row_B, t.row_pa, t.row_pb);
}

// ------------------------------------------------------------------ moments ----
// S_d(row, m) = int_{lo_d}^{hi_d} (x-A)^i (x-B)^k K_AB exp(-p (x-P)^2) T_m((x - c_d)/h_d) dx.
// One warp per (row, d); lane q holds quadrature point q % 16 of every other panel and
// accumulates f(x_q) w_q T_m(u_q) for all m in registers; a shared-memory transpose then sums
// over lanes.
// Items are (d, row) = dr / nrows, dr % nrows with dr = rep[item] (or dr = item without rep;
// rep[item] < 0 marks an unused item); item's moments go to S[item * n + m].
template <int NM>
__global__ void __launch_bounds__(128) k_moments(int64_t nrows, int n, const double* row_p, const double* row_P,
                                                 const double* row_K, const double* row_A, const double* row_B,
                                                 const int8_t* row_pa, const int8_t* row_pb, const double* lo3,
                                                 const double* hi3, const uint8_t* row_box, const double* gz,
                                                 const double* gw, const int64_t* rep, int64_t nitems, double* S) {
  __shared__ double red[4][32][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t item = (int64_t)blockIdx.x * 4 + warp;
  int64_t dr = item < nitems ? (rep ? rep[item] : item) : -1;
  const bool active = dr >= 0;  // keys that no row holds have rep = -1
  if (!active) dr = 0;
  const int d = (int)(dr / nrows);
  const int64_t row = dr % nrows;
  double acc[NM];
#pragma unroll
  for (int m = 0; m < NM; ++m) acc[m] = 0.0;
  if (active) {
    const double p = row_p[row];
    const double Pc = row_P[d * nrows + row], K = row_K[d * nrows + row];
    const double A = row_A[d * nrows + row], B = row_B[d * nrows + row];
    const int ia = row_pa[d * nrows + row], ib = row_pb[d * nrows + row];
    const int box = row_box ? (int)row_box[row] : 0;  // adaptive boxes: the row's partition
    const double lo = lo3[3 * box + d], hi = hi3[3 * box + d];
    const double cen = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
    const double reach = 9.0 / sqrt(p);
    const double wl = fmax(lo, Pc - reach), wh = fmin(hi, Pc + reach);
    if (wh > wl) {
      // T_{n-1} oscillates across the box: above n = 32 the window takes twice the panels.  The
      // 16-point rule (exact to degree 31 on a panel) resolves each panel's share of the
      // Gaussian times the polynomial factor times T_m to rounding: half-warps take alternate
      // panels, lane & 15 the point.
      const int npan = n <= 32 ? kMomentPanels : 2 * kMomentPanels;
      const double hp = (wh - wl) / npan;
      const double zq = gz[lane & 15], wq = gw[lane & 15];
      for (int pan = lane >> 4; pan < npan; pan += 2) {
        const double mid = wl + (pan + 0.5) * hp;
        const double x = mid + 0.5 * hp * zq;
        const double dx = x - Pc;
        double f = K * exp(-p * dx * dx) * (0.5 * hp * wq);
        const double xa = x - A, xb = x - B;
        for (int e = 0; e < ia; ++e) f *= xa;
        for (int e = 0; e < ib; ++e) f *= xb;
        const double u = (x - cen) / half;
        double t0 = 1.0, t1 = u;
        acc[0] += f;
        if (NM > 1) acc[1] += f * u;
#pragma unroll
        for (int m = 2; m < NM; ++m) {
          double t2 = 2.0 * u * t1 - t0;
          acc[m] += f * t2;
          t0 = t1;
          t1 = t2;
        }
      }
    }
  }
  // sum over lanes: 32 moments at a time through shared memory
#pragma unroll
  for (int m0 = 0; m0 < NM; m0 += 32) {
#pragma unroll
    for (int m = 0; m < 32; ++m)
      if (m0 + m < NM) red[warp][lane][m] = acc[m0 + m];
    __syncwarp();
    double s = 0.0;
    for (int l = 0; l < 32; ++l) s += red[warp][l][lane];
    if (active && m0 + lane < n) S[(size_t)item * n + m0 + lane] = s;
    __syncwarp();
  }
}

// Moment key of every (d, row): S_d of a row depends only on its shell pair (s_mu <= s_nu), its
// primitive pair (j1, j2), d and the powers (i, k) of mu and nu in d, so rows that agree in these
// have identical moments.  key = off(s_mu, s_nu) + ((j1 K_nu + j2) 3 + d) (l_mu + 1)(l_nu + 1)
// + i (l_nu + 1) + k; rep[key] receives one (d, row) = d nrows + row holding it (any of them: their
// inputs are identical, so a racing store of another one is harmless).
__global__ void k_moment_keys(const PairTable t, const int* __restrict__ bf_shell, const int* __restrict__ bf_pow,
                              const int* __restrict__ shell_nprim, const int* __restrict__ shell_l,
                              const int64_t* __restrict__ sp_off, int nshells, int* __restrict__ key,
                              int64_t* __restrict__ rep) {
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < t.nrows;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int r = t.row_pair[row];
    const int mu = t.pair_mu[r], nu = t.pair_nu[r];
    const int s1 = bf_shell[mu], s2 = bf_shell[nu];
    const int Kn = shell_nprim[s2];
    const int j1 = t.row_prim[row] >> 4, j2 = t.row_prim[row] & 15;
    const int lb = shell_l[s2] + 1, cmb = (shell_l[s1] + 1) * lb;
    const int64_t tri = (int64_t)s1 * nshells - (int64_t)s1 * (s1 - 1) / 2 + (s2 - s1);
    const int64_t base = sp_off[tri] + (int64_t)(j1 * Kn + j2) * 3 * cmb;
    for (int d = 0; d < 3; ++d) {
      const int64_t u = base + d * cmb + bf_pow[3 * mu + d] * lb + bf_pow[3 * nu + d];
      key[d * t.nrows + row] = (int)u;
      rep[u] = d * t.nrows + row;
    }
  }
}

// S[dr][m] = Su[key[dr]][m] for dr < 3 nrows.
__global__ void k_gather_moments(int64_t count, int n, const int* __restrict__ key, const double* __restrict__ Su,
                                 double* __restrict__ S) {
  const int64_t total = count * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t dr = e / n;
    S[e] = Su[(int64_t)key[dr] * n + (e - dr * n)];
  }
}

void launch_moment_keys(const PairTable& t, const int* d_bf_shell, const int* d_bf_pow, const int* d_shell_nprim,
                        const int* d_shell_l, const int64_t* d_sp_off, int nshells, int* d_key, int64_t* d_rep,
                        cudaStream_t st) {
  if (t.nrows <= 0) return;
  count_launch();
  const int64_t blocks = std::min<int64_t>((t.nrows + 255) / 256, 152 * 16);
  k_moment_keys<<<(unsigned)blocks, 256, 0, st>>>(t, d_bf_shell, d_bf_pow, d_shell_nprim, d_shell_l, d_sp_off, nshells,
                                                  d_key, d_rep);
}

void launch_gather_moments(int64_t count, int n, const int* d_key, const double* d_Su, double* d_S, cudaStream_t st) {
  if (count <= 0) return;
  count_launch();
  const int64_t blocks = std::min<int64_t>((count * n + 255) / 256, 152 * 16);
  k_gather_moments<<<(unsigned)blocks, 256, 0, st>>>(count, n, d_key, d_Su, d_S);
}

void launch_moments(const PairTable& t, int n, const double* d_lo3, const double* d_hi3, const uint8_t* d_row_box,
                    const double* d_gz, const double* d_gw, const int64_t* d_rep, int64_t nitems, double* d_S,
                    cudaStream_t st) {
  if (nitems <= 0) return;
  const int64_t items = nitems;
  const unsigned blocks = (unsigned)((items + 3) / 4);
  count_launch();
  // accumulators for n rounded up to a multiple of 8 (the recurrence costs two FMAs per term)
#define LRTEI_MOMENTS(NM)                                                                                       \
  k_moments<NM><<<blocks, 128, 0, st>>>(t.nrows, n, t.row_p, t.row_P, t.row_K, t.row_A, t.row_B, t.row_pa, t.row_pb, \
                                        d_lo3, d_hi3, d_row_box, d_gz, d_gw, d_rep, nitems, d_S)
  switch ((n + 7) / 8) {
    case 1: LRTEI_MOMENTS(8); break;
    case 2: LRTEI_MOMENTS(16); break;
    case 3: LRTEI_MOMENTS(24); break;
    case 4: LRTEI_MOMENTS(32); break;
    case 5: LRTEI_MOMENTS(40); break;
    case 6: LRTEI_MOMENTS(48); break;
    case 7: LRTEI_MOMENTS(56); break;
    default: LRTEI_MOMENTS(64); break;
  }
#undef LRTEI_MOMENTS
}

}  // namespace lrtei
