// lrtei_internal.h -- internal declarations shared by the CUDA translation units of liblrtei.
// Not part of the C ABI (include/lrtei.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lrtei.h"

namespace lrtei {

constexpr int kMaxN = 64;        // Chebyshev nodes per dimension
constexpr int kMaxP = 128;       // Gauss-Legendre nodes over [0, omega]
constexpr int kMomentPanels = 8; // panels of the device moment quadrature (n <= 32; 16 above)
constexpr int kMomentPts = 16;   // Gauss-Legendre points per panel (two panels per warp step)

// Device-side status word (latched by kernels, read by lrtei_plan_status).
enum DevStatus : int { kDevOk = 0, kDevTimeout = 1, kDevNonFinite = 2, kDevBadIndex = 3 };

// Latch a device status code unless one is latched already (the first failure is reported).
__device__ __forceinline__ void latch_status(int* status, int code) {
  if (status) atomicCAS(status, (int)kDevOk, code);
}
// Warp-wide non-finite flag: every lane of a full warp calls it once with its own flag; one lane
// latches kDevNonFinite if any lane saw a NaN or an infinity.
__device__ __forceinline__ void latch_nonfinite_warp(int* status, bool bad) {
  const unsigned any = __ballot_sync(0xffffffffu, bad);
  if (any && (threadIdx.x & 31) == 0) latch_status(status, (int)kDevNonFinite);
}
// Unique-pair index of (a, b) in the row-major upper triangle of nbf basis functions, or -1 when
// a or b lies outside [0, nbf) (the caller's index lists are checked on the device).
__host__ __device__ __forceinline__ int64_t checked_pair_index(int nbf, int a, int b) {
  if (a < 0 || b < 0 || a >= nbf || b >= nbf) return -1;
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  return (int64_t)lo * nbf - (int64_t)lo * (lo - 1) / 2 + (hi - lo);
}

void set_error(const char* fmt, ...);
lrtei_status cuda_fail(cudaError_t e, const char* what);

#define LRTEI_CUDA(call)                                  \
  do {                                                    \
    cudaError_t e__ = (call);                             \
    if (e__ != cudaSuccess) return cuda_fail(e__, #call); \
  } while (0)

// Counts kernel launches made by the library (reported by lrtei_profile_get("*")).
void count_launch();
void count_launches(long long n);
long long launch_count();
void set_launch_count(long long n);
// Stream-ordered scratch from the library's memory pool of the current device (keeps up to 2 GiB
// reserved across synchronisations, so that small calls do not map their scratch anew each time);
// released with cudaFreeAsync.  Counts as one allocation request.
cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t st);

// Counts device allocation requests (cudaMalloc / cudaMallocAsync) made by the library
// (reported by lrtei_profile_get("alloc"); never reset).
void count_alloc();

// Kernel timing: events recorded on the launching stream when profiling is enabled.
struct ProfScope {
  const char* name;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(const char* n, cudaStream_t s);
  ~ProfScope();
};

// Pair / row table on the device (structure of arrays; rows are primitive pairs of unique
// basis pairs mu <= nu, grouped by pair).
struct PairTable {
  int64_t npair = 0, nrows = 0;
  int maxI = 0;                // largest number of rows of one pair (host copy)
  int* pair_mu = nullptr;      // [npair]
  int* pair_nu = nullptr;      // [npair]
  int64_t* pair_row = nullptr; // [npair + 1] first row of each pair
  int* pair_I = nullptr;       // [npair] rows of each pair (I_mu I_nu, fewer when screened)
  uint8_t* row_prim = nullptr; // [nrows] (j1 << 4) | j2: the primitives of mu and nu of each row
  // per row
  int* row_pair = nullptr;     // [nrows]
  double* row_c = nullptr;     // [nrows] c_j = c_{j1} c_{j2} (normalised)
  double* row_p = nullptr;     // [nrows] a + b
  double* row_P = nullptr;     // [3 * nrows] product centre (d-major)
  double* row_K = nullptr;     // [3 * nrows] exp(-ab/p (A_d - B_d)^2)
  double* row_A = nullptr;     // [3 * nrows] centre of mu
  double* row_B = nullptr;     // [3 * nrows] centre of nu
  int8_t* row_pa = nullptr;    // [3 * nrows] power of mu in d
  int8_t* row_pb = nullptr;    // [3 * nrows] power of nu in d
};

// ---------------------------------------------------------------- setup kernels
// Gauss-Legendre nodes/weights on [-1, 1] for N points (device, one thread per root).
void launch_gauss_legendre(int N, double* d_z, double* d_w, cudaStream_t st);
// s_p = omega (1 + z_p) / 2.
void launch_nodes_map(int P, double omega, const double* d_z, double* d_s, cudaStream_t st);
// C[d][p] = Chebyshev coefficients of exp(-s_p^2 half_d^2 (u - v)^2), n x n.
void launch_cheb_coeff(int n, int P, const double* d_s, const double* d_half3, double* d_C, cudaStream_t st);
// The same between two intervals of half-widths hx3[d] (first index) and hy3[d] (second index),
// both centred at the same point (the adaptive boxes of Section 6).
void launch_cheb_coeff_cross(int n, int P, const double* d_s, const double* d_hx3, const double* d_hy3, double* d_C,
                             cudaStream_t st);
// Normalised coefficients per (basis function, primitive).
void launch_normalise(int nbf, const int* d_bf_shell, const int* d_bf_pow, const int* d_shell_nprim,
                      const int* d_shell_poff, const double* d_exps, const double* d_coefs, const int* d_bf_coff,
                      double* d_ncoef, cudaStream_t st);
// Fill the per-row part of the pair table.
void launch_pair_rows(const PairTable& t, const int* d_bf_shell, const int* d_bf_pow, const int* d_shell_nprim,
                      const int* d_shell_poff, const double* d_shell_center, const double* d_exps,
                      const int* d_bf_coff, const double* d_ncoef, cudaStream_t st);
// S[d][row][m] for m < n, FP64.  d_gz/d_gw: kMomentPts Gauss-Legendre rule on [-1,1].
// Items (d, row) = rep[i] (d nrows + row; i < nitems; rep NULL: i itself, nitems = 3 nrows; rep[i] < 0:
// skipped) -> d_S[i][m].  The box of a row is [lo3[3 b + d], hi3[3 b + d]] with b = row_box[row]
// (row_box NULL: b = 0).
void launch_moments(const PairTable& t, int n, const double* d_lo3, const double* d_hi3, const uint8_t* d_row_box,
                    const double* d_gz, const double* d_gw, const int64_t* d_rep, int64_t nitems, double* d_S,
                    cudaStream_t st);
// Moment keys: rows that share shell pair, primitive pair, d and the powers in d share S_d.
// key[d nrows + row] in [0, nkeys) with nkeys = sum over shell pairs s1 <= s2 of
// K_s1 K_s2 3 (l_s1 + 1)(l_s2 + 1) (offsets sp_off, triangular in the shell pair); rep[key] = one
// d nrows + row holding it (rep preset to -1).
void launch_moment_keys(const PairTable& t, const int* d_bf_shell, const int* d_bf_pow, const int* d_shell_nprim,
                        const int* d_shell_l, const int64_t* d_sp_off, int nshells, int* d_key, int64_t* d_rep,
                        cudaStream_t st);
// S[dr][m] = Su[key[dr]][m] for dr < count.
void launch_gather_moments(int64_t count, int n, const int* d_key, const double* d_Su, double* d_S, cudaStream_t st);

// ---------------------------------------------------------------- Hadamard form (FP64)
// T[d][p][row][b] = sum_a S[d][row][a] C[d][p][a][b]
void launch_tmat(int64_t nrows, int n, int P, const double* d_S, const double* d_C, double* d_T, cudaStream_t st);

// Operands of the tensor-core Hadamard form (k_tc_hadamard.cu), for plans whose unique pairs hold
// one primitive pair each: slices of T_{d,p} = S'_d A_d^(p) (A operand, rows [d][p][row]) and of
// S'_d (B operand, rows [d][row]), S'_x carrying the rows' contraction coefficients; per-row
// exponents; node factors f[row][p] = (w/sqrt(pi)) w_p 2^(Ea_p - Ra) as FP32 pairs, Ra and Eb.
struct HadOperands {
  int64_t nrows = 0;
  int n = 0, kpad = 0, P = 0;
  uint16_t *t0 = nullptr, *t1 = nullptr, *t2 = nullptr;                 // [3 P nrows][kpad]
  uint16_t *s0 = nullptr, *s1 = nullptr, *s1h = nullptr, *s2 = nullptr;  // [3 nrows][kpad]
  int *te = nullptr, *se = nullptr;                                      // [3 P nrows], [3 nrows]
  float2* f = nullptr;                                                   // [nrows][P]
  int *ra = nullptr, *eb = nullptr;                                      // [nrows]
};
// Fill h from the plan's moments (S, [3][nrows][n]), coefficients and weights; d_Ss (3 nrows n)
// and d_T (3 P nrows n) are FP64 scratch.
void launch_had_prepare(const HadOperands& h, const double* d_S, const double* d_C, const double* d_w, double pref,
                        const double* d_row_c, double* d_Ss, double* d_T, cudaStream_t st);
// Rows [r0, r1) of B_u by the tensor-core Hadamard form: the whole upper triangle with mirrors
// into out (ld) when [r0, r1) is every row, else rows r0.. of a band at out + (r - r0) ld.
lrtei_status had_tc_rows(const HadOperands& h, int64_t r0, int64_t r1, double* d_out, int64_t ld, int* d_status,
                         cudaStream_t st);
// Entries by Algorithm 1 on unique pairs: out[e] = B_u(r_e, c_e), prefactor included.
// Entries whose r or c is negative (an index outside the basis) come out as NaN; a non-finite
// result of a valid entry latches kDevNonFinite into *d_status.
void launch_hadamard_pairs(const PairTable& t, int n, int P, const double* d_S, const double* d_T,
                           const double* d_w, double pref, const int64_t* d_r, const int64_t* d_c, int64_t count,
                           double* d_out, int* d_status, cudaStream_t st);
// Block of B_u rows [r0, r1) x all columns, Hadamard form.
void launch_hadamard_rows(const PairTable& t, int n, int P, const double* d_S, const double* d_T, const double* d_w,
                          double pref, int64_t r0, int64_t r1, double* d_Bu, int64_t ld, cudaStream_t st);
// (mu,nu,ka,la) quadruples -> unique pair indices; an index outside [0, nbf) gives -1 and latches
// kDevBadIndex into *d_status.
void launch_idx4_to_pairs(int nbf, const int32_t* d_idx4, int64_t count, int64_t* d_r, int64_t* d_c, int* d_status,
                          cudaStream_t st);

// ---------------------------------------------------------------- factored form
// F_u[r][m] = sum_{j in r} c_j S_x(j,m1) S_y(j,m2) S_z(j,m3), m = (m1 n + m2) n + m3, for r in [r0, r1).
template <typename T>
void launch_build_F(const PairTable& t, int n, const double* d_S, int64_t r0, int64_t r1, T* d_F, int64_t ldF,
                    cudaStream_t st);
// The same F_u in pairs of FP32 numbers, stored as FP64 (~2^-44 relative per term): for the
// tensor-core precisions, whose F_u only feeds 30-bit slices.
void launch_build_F_pairs(const PairTable& t, int n, const double* d_S, int64_t r0, int64_t r1, double* d_F,
                          int64_t ldF, cudaStream_t st);
// Dense K = sum_p w_p C_x^p (x) C_y^p (x) C_z^p  (n^3 x n^3), FP64.
cudaError_t launch_build_K(int n, int P, const double* d_C, const double* d_w, double scale, double* d_K,
                           cudaStream_t st);
// Y = sum_p w_p (C_x^p (x) C_y^p (x) C_z^p) X, X/Y: n^3 x ncol (column index fastest).
void launch_kron_apply(int n, int P, const double* d_C, const double* d_w, const double* d_X, double* d_Y,
                       int64_t ncol, double* d_t1, double* d_t2, cudaStream_t st);
// Expand the unique-pair square B_u (npair x npair, ld) into full B (N_b^2 x N_b^2, ldB), times scale.
// The expansion and unpacking kernels latch kDevNonFinite into *d_status if they store a NaN or an
// infinity (a warp vote per store loop; no extra memory traffic).
void launch_expand_B(const PairTable& t, int nbf, const double* d_Bu, int64_t ldu, double scale, double* d_B,
                     int64_t ldB, int* d_status, cudaStream_t st);
// Rows [R0, R1) of full B (R = a N_b + b) from complete rows of B_u: out row R - R0 (ldo) is
// row pair(min(a, b), max(a, b)) of B_u gathered over the columns (ka, la).
void launch_expand_B_rows(int nbf, const double* d_Bu, int64_t ldu, int64_t R0, int64_t R1, double* d_out, int64_t ldo,
                          int* d_status, cudaStream_t st);
// Densities -> unique-pair vectors: d_u[r][q] = D_q(mu,nu) * (mu == nu ? 1 : 2).
void launch_pack_density(int nbf, int R, const double* d_D, double* d_u, cudaStream_t st);
// Unique-pair results -> full symmetric J: J_q(mu,nu) = J_q(nu,mu) = scale * Ju[r][q].
void launch_unpack_J(int nbf, int R, const double* d_Ju, double scale, double* d_J, int* d_status, cudaStream_t st);
// The unique pairs [r0, r1) only (Ju holds their rows); other entries of J are left as they are.
void launch_unpack_J_range(const PairTable& t, int nbf, int R, int64_t r0, int64_t r1, const double* d_Ju, double scale,
                           double* d_J, int* d_status, cudaStream_t st);

// ---------------------------------------------------------------- Khatri-Rao compression
// Scratch blocks of the Gram partial sums (d_part holds kr_gram_blocks * 3 * n * n doubles).
int kr_gram_blocks(int64_t nrows);
// Right singular vectors d_V (3 x n x n, columns descending) and squared singular values d_lam
// (3 x n, descending) of the three moment matrices S_d (nrows x n), by two Jacobi passes on Gram
// matrices; d_G, d_V1: 3 n n scratch; d_sweeps (6 ints, may be NULL): sweeps of each solve.
cudaError_t launch_kr_svd(int64_t nrows, int n, const double* d_S, double* d_part, double* d_G, double* d_V1,
                          double* d_lam, double* d_V, int* d_sweeps, cudaStream_t st);
// S_new = S_d V_d[:, :R] (3 x nrows x R) and C_new = V_d^T A_d^(p) V_d (3 x P x R x R).
cudaError_t launch_kr_project(int64_t nrows, int n, int P, int R, const double* d_S, const double* d_C,
                              const double* d_V, double* d_Snew, double* d_Cnew, cudaStream_t st);

// ---------------------------------------------------------------- adaptive boxes (Section 6)
// out[i][:] = in[idx[i]][:] (rows of length len, both with leading dimension len).
void launch_gather_rows(const double* d_in, const int64_t* d_idx, int64_t count, int64_t len, double* d_out,
                        cudaStream_t st);
// Bu[rows[i]][cols[j]] = blk[i][j] (ldb), and Bu[cols[j]][rows[i]] too when mirror.
void launch_scatter_block(const double* d_blk, int64_t ldb, const int64_t* d_rows, int64_t nr, const int64_t* d_cols,
                          int64_t nc, double* d_Bu, int64_t ldu, bool mirror, cudaStream_t st);
// Ju[rows[i]][:] = blk[i][:] (R columns).
void launch_scatter_rows(const double* d_blk, const int64_t* d_rows, int64_t nr, int64_t R, double* d_Ju,
                         cudaStream_t st);
// Algorithm 1 entries with per-pair partitions: C block (part[r], part[c]) of Cpp (npart^2 x 3 x P x n x n).
void launch_adaptive_entries(const PairTable& t, int n, int P, int npart, const int* d_pair_part, const double* d_S,
                             const double* d_Cpp, const double* d_w, double pref, const int64_t* d_r,
                             const int64_t* d_c, int64_t count, double* d_out, int* d_status, cudaStream_t st);

// ---------------------------------------------------------------- long-range exchange
// MT[(mu n3 + m) nbf + la] = F[pair(mu, la) ldF + m]  (nbf n3 rows of nbf).
void launch_gather_MT(int nbf, int64_t n3, const double* d_F, int64_t ldF, double* d_MT, cudaStream_t st);
// Zp[mu][j n3 + m] = Z[(j nbf + mu) n3 + m] for j < nj.
void launch_perm_orbital_rows(int nbf, int64_t n3, int nj, const double* d_Z, double* d_Zp, cudaStream_t st);

// ---------------------------------------------------------------- CUDA-core GEMM
// C[M x N] = alpha * op(A) op(B) + beta * C, row-major; transA: A is K x M; transB: B is N x K.
template <typename T>
void gemm_cuda_core(bool transA, bool transB, int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t lda,
                    const T* B, int64_t ldb, T beta, T* C, int64_t ldc, cudaStream_t st);
void convert_f64_to_f32(const double* in, float* out, int64_t count, cudaStream_t st);
void convert_f32_to_f64(const float* in, double* out, int64_t count, cudaStream_t st);

// ---------------------------------------------------------------- tensor cores (tcgen05)
struct SplitMatrix {  // row-major rows x kpad, three FP16 integer slices + per-row scale exponent
  int64_t rows = 0, kpad = 0;
  uint16_t* s0 = nullptr;
  uint16_t* s1 = nullptr;
  uint16_t* s2 = nullptr;  // third slice t2, pre-scaled by 2^-11 (FP16 bits)
  uint16_t* s1h = nullptr; // second slice t1 pre-scaled by 2^-11 (B operand only)
  int* expo = nullptr;     // [rows]
  bool plain = false;      // plain BF16 operands in s0 only (no slices)
  bool eight = false;      // eight-product scheme: every operand carries s1h (A: t1 t2 products)
};
// Slice an FP64 row-major matrix (rows x k, ld) into a SplitMatrix (zero padded to kpad).
void launch_split_rows(const double* d_src, int64_t rows, int64_t k, int64_t ld, SplitMatrix& m, bool with_s1h,
                       int nslices, cudaStream_t st);
// nslices == 1 keeps only the leading slice (s1 = s2 = 0): plain BF16 operands.
// C = scale * A B^T through tcgen05 (see k_tcgen05.cu).  A: M rows with slices s0, s1, s2;
// B: N rows with s0, s1, s1h, s2; shared kpad (multiple of 256).  transpose_out writes C^T;
// symmetric_upper computes the upper-triangular 128x128 blocks of a square C and mirrors them.
// splits > 1 splits K (at most 32768 per split) into d_part (splits * M * N doubles), reduced
// into C afterwards.
lrtei_status tc_gemm(const SplitMatrix& A, const SplitMatrix& B, int64_t M, int64_t N, double scale, double* d_C,
                     int64_t ldc, bool transpose_out, bool symmetric_upper, int splits, double* d_part,
                     int* d_status, cudaStream_t st);
// Block rows [row0, row1) of the symmetric product C = A B^T (N x N): the upper-triangular
// 128 x 128 blocks of those rows, computed and mirrored.  A holds rows [row0, row1) only; row0 is a
// multiple of 128, as is row1 unless it is N.  Rows of C at or above row0 are complete once every
// band up to this one has run.
lrtei_status tc_gemm_sym_band(const SplitMatrix& A, const SplitMatrix& B, int64_t row0, int64_t row1, int64_t N,
                              double* d_C, int64_t ldc, int* d_status, cudaStream_t st);
void launch_transpose(const double* in, int64_t rows, int64_t cols, int64_t ldi, double* out, int64_t ldo,
                      cudaStream_t st);
// out[i][j] = sum_q part[q * stride + i * ld + j] for i < rows, j < cols.
void launch_reduce_splits(const double* part, int splits, int64_t stride, int64_t rows, int64_t cols, int64_t ld,
                          double* out, int64_t ldo, cudaStream_t st);
inline int64_t kpad256(int64_t k) { return (k + 255) / 256 * 256; }

// Read-only view of a plan's resident device tables (for entry points defined outside
// lrtei_api.cu).
struct PlanView {
  int nbf, n, P;
  double omega;
  const PairTable* t;
  const double* S;  // 3 x nrows x n moments
  const double* C;  // 3 x P x n x n Chebyshev coefficients
  const double* w;  // P quadrature weights
  int* status;      // the plan's device status word
  const double* half3;  // box half-widths per dimension (device)
  int kr_rank;      // 0, or the rank of a Khatri-Rao compressed plan
  int npart;        // 0, or the number of adaptive-box partitions
};
lrtei_status plan_view(const lrtei_plan* plan, PlanView* v);

}  // namespace lrtei
