/* lrtei.h -- C ABI of the GB300 (sm_103a) library for the tensorized approximation (TA) of the
 * long-range two-electron integrals tensor B^lr (Badreddine, Chollet, Grigori, arXiv 2210.13069).
 *
 * What the library computes (paper references are to that article):
 *   B^lr(mu,nu,ka,la) = int int g_mu(x) g_nu(x) erf(w|x-y|)/|x-y| g_ka(y) g_la(y) dx dy over a box
 *   (Section 1, eq. "long-range" and eq. "compact"), approximated by
 *     K(x,y) ~ (w/sqrt(pi)) sum_p w_p prod_d sum_{a,b} A_d^(p)(a,b) T_a(u_d) T_b(v_d)
 *   (Section 3.1, eq. TEI2, eq. chebcheb, eq. Approx_kernel), which gives Theorem 1:
 *     B(mu nu, ka la) = (w/sqrt(pi)) sum_p w_p sum_{j,j'} c_j c_j' prod_d (S_d A_d^(p) S_d^T)(j, j')
 *   with S_d the 1D moment matrices of eq. defV, and its Khatri-Rao factored form (eq. tensors)
 *     B = (w/sqrt(pi)) sum_p w_p M (A_x^(p) (x) A_y^(p) (x) A_z^(p)) M^T,
 *   which applies B to densities (J-builds, Section 5, eq. coulapprox) without forming it.
 *
 * Conventions shared by every call:
 *   - Basis: contracted Cartesian Gaussians (eq. "basis", "primi").  A shell of angular momentum
 *     l expands into its (l+1)(l+2)/2 components in the order lx = l..0, ly = l-lx..0,
 *     lz = l-lx-ly.  Each component is normalised on R^3; each contraction to unit norm.
 *   - Box: per dimension [lo_d, hi_d]; NULL selects the default cube centred on the atoms'
 *     extent with half-width (half extent + sqrt(ln(1e16) / (2 alpha_min))).
 *   - Chebyshev nodes of the first kind, n per dimension, degrees 0..n-1 (Definition 1).
 *   - Gauss-Legendre nodes z_p, weights w_p on [-1,1]; s_p = w (1 + z_p)/2 (eq. TEI2).
 *   - B is the mode-(1,2) unfolding: row mu*N_b + nu, column ka*N_b + la, row-major, 0-based.
 *   - Every compute call is asynchronous on the CUDA stream it is given (NULL = legacy default
 *     stream).  Device pointers (d_*) are owned by the caller; the library owns plans and their
 *     workspaces.  Inputs are validated on the host before anything is launched; a failed
 *     call returns a status and leaves a message for lrtei_last_error().  Device-side failures
 *     are latched in the plan's status word (the first one wins) and reported by
 *     lrtei_plan_status(), which synchronises the device: a bounded wait of the tensor-core
 *     GEMM that gave up (LRTEI_ERR_TIMEOUT), a NaN or infinity stored into B, J or an entries
 *     output (LRTEI_ERR_NUMERIC; checked by a warp vote in the kernels that write them), and a
 *     basis-function index outside [0, N_b) in a device index list (LRTEI_ERR_ARG).
 *   - No call falls back to the CPU: without a usable CUDA device every call that computes
 *     returns LRTEI_ERR_CUDA.
 */
#ifndef LRTEI_H
#define LRTEI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LRTEI_OK = 0,
  LRTEI_ERR_ARG = 1,         /* invalid argument (checked on the host before any launch) */
  LRTEI_ERR_ALLOC = 2,       /* device or host allocation failed */
  LRTEI_ERR_CUDA = 3,        /* a CUDA runtime call failed (no device, launch failure ...) */
  LRTEI_ERR_TIMEOUT = 4,     /* a device-side bounded wait gave up */
  LRTEI_ERR_NUMERIC = 5,     /* a non-finite value was detected on the device */
  LRTEI_ERR_UNSUPPORTED = 6  /* valid but not supported by this build (e.g. size limits) */
} lrtei_status;

/* Arithmetic of the contractions (moments, nodes, Chebyshev coefficients and the node sum
 * are FP64 in every mode). */
typedef enum {
  LRTEI_FP64 = 0,        /* FP64 CUDA-core contractions */
  LRTEI_FP32 = 1,        /* FP32 CUDA-core contractions */
  LRTEI_SPLIT_F16 = 2,  /* tcgen05 tensor cores, split operands: per row a power-of-two scale and
                            three integer slices (8 + 12 + 12 bits) held exactly in 16-bit floats;
                            the leading products accumulate exactly in FP32 within each 128-deep K
                            chunk, chunks are summed in int32 / FP32 registers (about 32 bits);
                            1e-8 to 5e-8 measured */
  LRTEI_BF16 = 3,        /* tcgen05 tensor cores, plain BF16 operands (one rounding per element),
                            FP32 accumulation */
  LRTEI_SPLIT_F16_8 = 4  /* as LRTEI_SPLIT_F16, plus the two next-order slice products (t1 t2 and
                            t2 t1), with the small terms in a third accumulator: 8 tensor-core
                            products per K step instead of 6 and 128 x 64 tiles, an error several
                            times smaller (1e-9 to 1.5e-8 measured) */
} lrtei_precision;

/* Which of the two equivalent forms of Theorem 1 assembles B.  On the FP64 and FP32 paths both
 * run on the CUDA cores.  With LRTEI_SPLIT_F16 the factored form runs on the tensor cores, and so
 * does the Hadamard form when every unique pair holds one primitive pair (an uncontracted basis,
 * n <= 64, no compression or adaptive boxes): per node and dimension the tile products
 * T_{d,p} S_d^T (depth n) on the tensor cores, the product over dimensions and the node sum in
 * pairs of FP32 numbers; elsewhere the tensor-core precisions take the factored form whatever
 * `form` asks.  lrtei_plan_info_get reports the form the last assembly used (last_form). */
typedef enum {
  LRTEI_FORM_AUTO = 0,      /* cost model: Hadamard when P Ibar^2 (6n + 3) <= 2 n^3, else factored */
  LRTEI_FORM_HADAMARD = 1,  /* entry-wise Hadamard form (Theorem 1 / Algorithm 1) */
  LRTEI_FORM_FACTORED = 2   /* Khatri-Rao factored form (eq. tensors) */
} lrtei_form;

typedef struct lrtei_basis lrtei_basis;
typedef struct lrtei_plan lrtei_plan;

typedef struct {
  int nbf;          /* N_b */
  int64_t npair;    /* unique basis pairs mu <= nu: N_b (N_b + 1) / 2 */
  int64_t nrows;    /* primitive-pair rows over unique pairs: sum_{mu<=nu} I_mu I_nu */
  int n, P;
  double omega;
  double box_lo[3], box_hi[3];
  int precision;    /* lrtei_precision */
  int last_form;    /* lrtei_form used by the last lrtei_assemble_B call */
  size_t workspace_bytes; /* device bytes the plan currently holds */
  double tau_screening;   /* primitive-pair screening threshold of the plan (0: none) */
  int cheb_n;       /* Chebyshev nodes per dimension the plan was created with */
  int kr_rank;      /* 0, or the rank R after lrtei_plan_compress (then n == R) */
  int npartitions;  /* 0, or the number of adaptive-box partitions (lrtei_plan_create_adaptive) */
  double partition_b[8]; /* their cubes' half-widths b_s, ascending (the box above is the largest) */
} lrtei_plan_info;

/* ---- basis (Section 1, eq. "basis"/"primi") ------------------------------------------
 * Host arrays, copied: centers[3*nshells] (bohr), l[nshells] in 0..4, nprim[nshells] in 1..16,
 * exps/coefs concatenated in shell order (sum(nprim) each, exps > 0).  Returns LRTEI_ERR_ARG
 * on invalid input. */
lrtei_status lrtei_basis_create(int nshells, const double* centers, const int* l, const int* nprim,
                                const double* exps, const double* coefs, lrtei_basis** out);
void lrtei_basis_destroy(lrtei_basis* basis);
int lrtei_basis_nbf(const lrtei_basis* basis);

/* ---- plan (Section 3.1: w, box, n = N^(1/3), P = N_q1) --------------------------------
 * Uploads the basis and computes, on the device and on `stream`: Gauss-Legendre nodes and
 * weights (eq. TEI2), the Chebyshev coefficient matrices A_d^(p) (Definition 1, eq. chebcheb),
 * the primitive-pair table (Proposition 1) and the moment matrices S_d (eq. defV).
 * omega > 0; 1 <= n <= 64; 1 <= P <= 128; box_lo/box_hi: 3 doubles each or both NULL. */
lrtei_status lrtei_plan_create(const lrtei_basis* basis, double omega, int n, int P, const double* box_lo,
                               const double* box_hi, lrtei_precision precision, void* stream, lrtei_plan** out);
/* The same with primitive-pair screening (Section 6, "Compression by using Screening"): the
 * primitive pair (j1, j2) of a basis pair (mu, nu) is discarded when
 * exp(-a_j1 b_j2 / (a_j1 + b_j2) |A - B|^2) <= tau_screening (exponents a, b, centres A, B),
 * decided on the host in FP64; its row leaves the pair table, so the moments, F_u and every
 * sum over j skip it.  tau_screening in [0, 1]; 0 keeps every pair (lrtei_plan_create).
 * lrtei_factors then returns the kept rows only, in the same order. */
lrtei_status lrtei_plan_create_ex(const lrtei_basis* basis, double omega, int n, int P, const double* box_lo,
                                  const double* box_hi, lrtei_precision precision, double tau_screening,
                                  void* stream, lrtei_plan** out);
/* Adaptive choice of the integration domain (Section 6, "Adaptive approach for the choice of the
 * integration domain"; paper's tau_adaptive = 1e-20).  The numerical support of a primitive pair
 * j in dimension l is |x_l - P_{j,l}| < sqrt(ln(1/tau_adaptive) / p_j) (where its Gaussian factor
 * exceeds tau_adaptive); a unique basis pair's support is the smallest cube about the centre c of
 * the atoms' extent holding those of all its primitive pairs.  The pairs, sorted by that half-width
 * (stable), are cut into npartitions groups of about equal count (a cut never splits pairs of equal
 * support, so the Cartesian components of one shell pair stay together; empty groups are dropped);
 * partition s is the cube [c - b_s, c + b_s]^3, b_s the largest support of its group.  A pair's
 * moments are integrated over its partition's cube (eq. defV on that cube), and between partitions
 * s and t the kernel is interpolated on the two cubes' first-kind Chebyshev grids:
 *   A^(p)_{st}(a, b) = c_a c_b / n^2 sum_{k,k'} exp(-s_p^2 (b_s u_k - b_t u_k')^2) T_a(u_k) T_b(u_k'),
 * B(mu nu, ka la) = (w/sqrt(pi)) sum_p w_p sum_{j,j'} c_j c_j' prod_d (S_d(j) A^(p)_{st,d} S_d(j')^T).
 * One n serves every partition.  Supported on the plan: lrtei_assemble_B (partition blocks
 * B_st = F_s K_st F_t^T: tensor cores for the split precisions, FP64 mode products otherwise; into
 * device memory or mapped pinned memory), lrtei_entries, lrtei_jbuild (FP64 for every precision),
 * lrtei_factors (d_C then holds npartitions^2 blocks, index (s npartitions + t), each 3 x P x n x n).
 * Other calls return LRTEI_ERR_UNSUPPORTED.  tau_adaptive in (0, 1), npartitions in 1..8. */
lrtei_status lrtei_plan_create_adaptive(const lrtei_basis* basis, double omega, int n, int P, double tau_adaptive,
                                        int npartitions, lrtei_precision precision, void* stream, lrtei_plan** out);
void lrtei_plan_destroy(lrtei_plan* plan);
lrtei_status lrtei_plan_info_get(const lrtei_plan* plan, lrtei_plan_info* info);
/* Synchronises the plan's stream and returns the latched device-side status (then clears it). */
lrtei_status lrtei_plan_status(lrtei_plan* plan);

/* ---- full tensor (Theorem 1; eq. tensors) ----------------------------------------------
 * Writes all N_b^2 x N_b^2 entries of B, FP64, row-major with leading dimension ld >= N_b^2,
 * into the caller's buffer d_B: device memory, or page-locked host memory (cudaHostAlloc /
 * cudaHostRegister).  Pageable host memory returns LRTEI_ERR_ARG.  `form` selects the Hadamard
 * or the factored form.  Into host memory, the tensor-core precisions compute B_u in bands of
 * 128-row blocks of its upper triangle and move each band's completed rows of B to the host
 * with copy-engine transfers on a second stream while the next band runs (the call returns with
 * that work queued on `stream`; ~1 GiB of device staging; LRTEI_HOST_BANDS (default 16) and
 * LRTEI_HOST_CHUNK_ROWS override the band count and the rows per transfer); the FP64 and FP32
 * paths write host memory from their expansion kernel directly across the host link. */
lrtei_status lrtei_assemble_B(lrtei_plan* plan, lrtei_form form, double* d_B, int64_t ld, void* stream);

/* Rows [row_begin, row_end) of the unique-pair matrix B_u (rows and columns are unique pairs
 * mu <= nu in the order (0,0),(0,1)..(0,N_b-1),(1,1)..), FP64, leading dimension ld >= npair.
 * B(mu nu, ka la) = B_u(pair(min,max), pair(min,max)). */
lrtei_status lrtei_assemble_Bu_rows(lrtei_plan* plan, lrtei_form form, int64_t row_begin, int64_t row_end,
                                    double* d_Bu, int64_t ld, void* stream);

/* ---- entries (Algorithm 1) ---------------------------------------------------------------
 * d_idx4: device int32[4*count] of (mu, nu, ka, la); d_out: device double[count].  The indices
 * are checked on the device: an entry with an index outside [0, N_b) reads nothing, comes out
 * as NaN, and lrtei_plan_status then returns LRTEI_ERR_ARG. */
lrtei_status lrtei_entries(lrtei_plan* plan, const int32_t* d_idx4, int64_t count, double* d_out, void* stream);

/* ---- entries without device allocation ---------------------------------------------------
 * The paper has no counterpart to this call; it exists for callers that cannot allocate device
 * memory where they need integrals (memory held by their own pool, paths where the device-wide
 * synchronisation of cudaMalloc/cudaFree is not acceptable).  Same arguments and results as
 * lrtei_entries, computed from the plan's resident moments and Chebyshev coefficients; it calls
 * no allocator.  Its scratch is one fixed device array per device, 4 MiB, held while the
 * library is loaded: at most 262144 entries per call (more returns LRTEI_ERR_UNSUPPORTED).  All
 * calls on a device share the array, so calls whose kernels overlap on the GPU race.  The
 * first call on a device performs a one-time lookup of the array's address with that device
 * current; make that first call before any stream capture begins.  That address is cached for
 * the life of the process: calls after a device reset (cudaDeviceReset, or a primary context
 * released and created again) are not supported.  Out-of-range indices are handled as in
 * lrtei_entries. */
lrtei_status lrtei_entries_noalloc(lrtei_plan* plan, const int32_t* d_idx4, int64_t count, double* d_out,
                                   void* stream);

/* ---- entries at other orders (error sweeps of the plain method) ---------------------------
 * Algorithm 1 entries of the plan's basis, box and omega at ncombo other orders (n_c, P_c) =
 * (h_n[c], h_P[c]), 1 <= n_c <= the plan's n, 1 <= P_c <= 128 (host arrays): the moment integrals
 * of eq. defV do not depend on n, so the plan's moments serve every n_c <= n through their first
 * n_c columns; the Gauss-Legendre nodes (eq. TEI2) and Chebyshev coefficients (Definition 1) are
 * computed for each order.  d_idx4 as for lrtei_entries; d_out: device double[ncombo * count],
 * order-major (d_out[c * count + e]).  These sweeps are the selector's training data.  Plans
 * compressed by lrtei_plan_compress return LRTEI_ERR_UNSUPPORTED. */
lrtei_status lrtei_entries_orders(lrtei_plan* plan, int ncombo, const int* h_n, const int* h_P, const int32_t* d_idx4,
                                  int64_t count, double* d_out, void* stream);

/* ---- factors (Theorem 1: w_p, s_p, A^(p), W~ = S_d) ---------------------------------------
 * Any pointer may be NULL.  d_s, d_w: P doubles; d_C: 3*P*n*n (d, p, a, b); d_S: 3*nrows*n
 * (d, row, m), rows ordered by unique pair then j = j1*I_nu + j2; d_c: nrows coefficients c_j. */
lrtei_status lrtei_factors(lrtei_plan* plan, double* d_S, double* d_C, double* d_s, double* d_w, double* d_c,
                           void* stream);

/* ---- Khatri-Rao low-rank compression (Section 6, eq. SVD and eq. approxepsilon) ----------
 * Computes, on the device in FP64, the SVD of the three moment matrices W~_d = S_d (all
 * primitive-pair rows x n) by two Jacobi passes on n x n Gram matrices, keeps in dimension d the
 * R_d leading right singular vectors V_d (R_d = number of singular values >= eps * sigma_1; eps = 0
 * keeps all n), and replaces the plan's factors by S_d V_d (rows x R) and V_d^T A_d^(p) V_d
 * (R x R), with R = max_d R_d (capped at max_rank when max_rank > 0).  Every later call of the plan
 * (B, entries, factors, K, J-builds) then computes eq. approxepsilon,
 *   B ~ (w/sqrt(pi)) U~ [sum_p w_p (x)_d V_d^T A_d^(p) V_d] U~^T,
 * whose difference from the uncompressed B is set by the dropped singular values.  The plan's n
 * becomes R (lrtei_plan_info: n = kr_rank = R, cheb_n = the original n); tables built from the
 * uncompressed factors are dropped.  A plan is compressed at most once (LRTEI_ERR_UNSUPPORTED).
 * Host outputs, may be NULL: h_sigma[3 * n] the singular values of each S_d (descending, the
 * original n), h_ranks[3] the R_d.  Synchronises `stream`.  eps in [0, 1), max_rank in [0, n]. */
lrtei_status lrtei_plan_compress(lrtei_plan* plan, double eps, int max_rank, double* h_sigma, int* h_ranks,
                                 void* stream);

/* ---- node sum of the factored form (Theorem 1, factored form; eq. approx33) ---------------
 * d_K: n^3 x n^3 FP64, row-major, K((a1 n + a2) n + a3, (b1 n + b2) n + b3) =
 * (omega / sqrt(pi)) sum_p w_p A_x^p(a1, b1) A_y^p(a2, b2) A_z^p(a3, b3), so that
 * B_u = F_u K F_u^T.  The node sum runs in pairs of FP32 numbers (TwoProd and a compensated dot
 * product), accurate to ~1e-13 of each row's largest entry; the tensor-core precisions slice this
 * K.  Caller-owned output; LRTEI_ERR_ARG for NULL arguments. */
lrtei_status lrtei_dense_K(lrtei_plan* plan, double* d_K, void* stream);

/* ---- J-build (Section 5, eq. coulapprox in the density form J = mat(B vec(D))) ----------
 * d_D: R symmetric N_b x N_b densities (FP64, row-major, consecutive); d_J: same shape.
 * J_r(mu, nu) = sum_{ka, la} B(mu nu, ka la) D_r(ka, la), through the factored form, never
 * forming B.  Uses the plan's precision for the two M-contractions.  When the resident operands
 * (F_u, F_u^T and the dense n^3 x n^3 K, with their slices) would take more than half of the free
 * device memory, F_u is instead built in blocks of unique pairs, twice per call, and the node sum
 * runs as FP64 mode products (eq. ig1); LRTEI_JBUILD_BLOCK=<pairs> in the environment forces this
 * streamed form with that block size.  A call repeating an earlier one-pass call's plan, d_D, d_J
 * and R replays a CUDA graph of its kernels, captured after that call ran (the densities are read
 * at replay time; up to 32 graphs are kept, least recently used dropped first, each holding its
 * scratch memory; a plan's graphs are dropped when its operands are rebuilt or it is destroyed).
 * Streamed calls, calls on a stream the caller is capturing, and LRTEI_JBUILD_GRAPH=0 launch
 * kernel by kernel.  The environment switches are read when a call is made; a replayed graph
 * keeps the choices of the call it was captured from. */
lrtei_status lrtei_jbuild(lrtei_plan* plan, const double* d_D, int R, double* d_J, void* stream);

/* ---- a J-build split over ranks by unique pairs -----------------------------------------
 * The two halves of eq. coulapprox for one range [pair_begin, pair_end) of unique pairs (rows of
 * F_u, pair order as in lrtei_assemble_Bu_rows), for callers that shard a molecule's J-builds over
 * processes or GPUs:
 *   lrtei_jbuild_partial_x: d_X (device, R x n^3, FP64) = sum over the range of u_r F_u(r, :), where
 *     u_r = D(mu, nu) (mu == nu) or 2 D(mu, nu) are the densities d_D (as lrtei_jbuild) on pair r;
 *     the sum of the ranks' d_X over a partition of [0, npair) is X = F_u^T vec(D) (an all-reduce).
 *   lrtei_jbuild_apply_x: from the summed d_X, Y = sum_p w_p (A_x^p (x) A_y^p (x) A_z^p) X by mode
 *     products (eq. ig1, FP64), then J(mu, nu) = J(nu, mu) = (w/sqrt(pi)) F_u(r, :) Y for the pairs
 *     r of the range; every other entry of d_J (R x N_b x N_b) is set to 0, so the sum of the
 *     ranks' d_J is lrtei_jbuild's J (a second all-reduce).
 * Rows of F_u are built for the range on each call (FP64); split precisions contract them on the
 * tensor cores.  LRTEI_ERR_ARG for a range outside [0, npair); adaptive-box plans return
 * LRTEI_ERR_UNSUPPORTED. */
lrtei_status lrtei_jbuild_partial_x(lrtei_plan* plan, const double* d_D, int R, int64_t pair_begin, int64_t pair_end,
                                    double* d_X, void* stream);
lrtei_status lrtei_jbuild_apply_x(lrtei_plan* plan, const double* d_X, int R, int64_t pair_begin, int64_t pair_end,
                                  double* d_J, void* stream);

/* ---- long-range exchange (appendix "The Hartree-Fock exchange", eq. exchange) -------------
 * K^lr(mu, nu) = 2 sum_j sum_{la, ka} q_{j la} q_{j ka} B(mu la, ka nu) for the orbital
 * coefficients d_Q (device, norb x N_b, row-major) into d_K (device, N_b x N_b, row-major),
 * without forming B: through the factored form, K^lr = 2 sum_j X_j K X_j^T with
 * X_j(mu, :) = sum_la q_{j la} M(mu la, :) (M of eq. tensors, K = (w/sqrt(pi)) sum_p w_p
 * (x)_d A_d^(p)).  Orbitals are processed in blocks (X of a block within ~1 GiB;
 * LRTEI_EXCHANGE_BLOCK=<orbitals> in the environment sets the block).  Tensor-core
 * precisions run the three products on tcgen05 with split operands; FP64 / FP32 plans run FP64
 * CUDA-core GEMMs and apply K by mode products (eq. ig1).  A compressed plan gives eq.
 * approxepsilon's exchange.  Device scratch ~6 x min(norb, block) N_b n^3 doubles plus N_b^2 n^3
 * (and their slices).  LRTEI_ERR_ARG for NULL pointers or norb <= 0. */
lrtei_status lrtei_exchange(lrtei_plan* plan, const double* d_Q, int norb, double* d_K, void* stream);

/* ---- batched J-builds (many molecules of uneven size in one graph-captured launch) -------
 * plans[nmol]: plans (each with its own omega, n, P); d_D[m], d_J[m], R[m]: per-molecule
 * densities and outputs.  All plans must share the precision.  On the first call for a set of
 * plans the library captures the whole batch into one CUDA graph; later calls with the same
 * plans and pointers replay it. */
lrtei_status lrtei_jbuild_batched(lrtei_plan* const* plans, int nmol, const double* const* d_D, const int* R,
                                  double* const* d_J, void* stream);

/* ---- the (n, P) selector (a 3-layer MLP, FP32, trained on the GPU) ----------------------
 * The paper picks the number of Chebyshev nodes with chebfun2 and studies how the error trades
 * n against P (Section 3.1, Section 6.1); here a network (6 -> H -> H -> 2, ReLU) predicts the
 * cheapest (n, P) that reaches a requested relative error, trained on error sweeps of the plain
 * method.  Raw features (6, host doubles): omega, box half-width (bohr), alpha_min, alpha_max,
 * max angular momentum l, target relative error.  Normalised features: omega, half / 30,
 * log10 alpha_min, log10 alpha_max / 4, l / 2, -log10 target / 10; normalised outputs:
 * (n - 8) / 56, (P - 8) / 120.  Weights live on the device. */
typedef struct lrtei_selector lrtei_selector;
lrtei_status lrtei_selector_create(int hidden, uint64_t seed, lrtei_selector** out);
void lrtei_selector_destroy(lrtei_selector* sel);
/* One epoch of mini-batch Adam on (d_X[N*6], d_Y[N*2]) (device, FP32, normalised targets).
 * Returns the mean loss of the epoch in *loss (synchronises). */
lrtei_status lrtei_selector_train_epoch(lrtei_selector* sel, const float* d_X, const float* d_Y, int N, int batch,
                                        float lr, float* loss, void* stream);
/* Forward pass for N rows: d_X[N*6] -> d_Yhat[N*2] (device). */
lrtei_status lrtei_selector_forward(lrtei_selector* sel, const float* d_X, float* d_Yhat, int N, void* stream);
/* Forward + backward of the mean squared error for N rows; gradients to d_grad (device,
 * lrtei_selector_nparams floats, packed W1,b1,W2,b2,W3,b3). */
lrtei_status lrtei_selector_grad(lrtei_selector* sel, const float* d_X, const float* d_Y, int N, float* d_grad,
                                 float* loss, void* stream);
int64_t lrtei_selector_nparams(const lrtei_selector* sel);
/* Parameters to / from host memory (packed as above), for checkpointing. */
lrtei_status lrtei_selector_get_params(const lrtei_selector* sel, float* h_params);
lrtei_status lrtei_selector_set_params(lrtei_selector* sel, const float* h_params);
/* Normalised features of raw[6] into out[6] (host); LRTEI_ERR_ARG unless omega, the half-width,
 * both exponents and the target are positive and finite and l >= 0. */
lrtei_status lrtei_selector_features(const double* raw, float* out);
/* Normalised training target of (n, P) into out[2] (host). */
lrtei_status lrtei_selector_encode(int n, int P, float* out);
/* The selection (host in, host out; runs the network on the device and synchronises): if raw
 * lies inside the training ranges (omega in [0.2, 1], half-width in [3, 34] bohr, log10 alpha_min
 * in [-1.4, 0.1], log10 alpha_max in [-0.4, 3.4], l in [0, 2], log10 target in [-9, -3]) the
 * network's (n, P) plus a margin of (4, 8), each rounded up to the grids
 * n in {8, 12, 16, 20, 24, 28, 32, 40, 48, 56, 64}, P in {8, 12, ..., 96, 128}; otherwise the
 * conservative fixed (32, 48).  *used_fallback (may be NULL) tells which. */
lrtei_status lrtei_select_np(lrtei_selector* sel, const double* raw, int* n, int* P, int* used_fallback);
/* Training: `epochs` epochs of lrtei_selector_train_epoch on (d_X, d_Y), at rate lr for the first
 * two thirds and lr / 10 after; h_loss[epochs] (may be NULL) receives each epoch's mean loss. */
lrtei_status lrtei_selector_train(lrtei_selector* sel, const float* d_X, const float* d_Y, int N, int epochs,
                                  int batch, float lr, float* h_loss, void* stream);
/* Checkpoints: a versioned little-endian file ("LRTEISEL", version 2, hidden width, parameter
 * count, an optional caller text `meta`, the FP32 parameters, an FNV-1a 64-bit checksum of all
 * preceding bytes).  Load rejects another version, inconsistent sizes or a checksum mismatch
 * (LRTEI_ERR_ARG) and creates a selector with those parameters (Adam state zero); meta (may be
 * NULL) receives the text, truncated to meta_cap - 1 bytes. */
lrtei_status lrtei_selector_save(const lrtei_selector* sel, const char* path, const char* meta);
lrtei_status lrtei_selector_load(const char* path, lrtei_selector** out, char* meta, size_t meta_cap);

/* ---- kernel timing (tracing) ----------------------------------------------------------
 * When enabled, the library records a pair of CUDA events on the launching stream around each
 * launch of its main kernels ("tc_gemm", "gemm_fp64", "gemm_fp32", "hadamard", "kron",
 * "expand_B", "moments", "build_F", "build_K", "split", "jbuild", "batched" for a replayed
 * J-build graph).  lrtei_profile_get synchronises those
 * events and returns the summed device time and the launch count of one kernel name.  Two
 * names are counters rather than kernels: "*" gives the number of kernels the library launched
 * since the last reset (time 0), and "alloc" the number of device allocations (cudaMalloc and
 * stream-ordered cudaMallocAsync) it has requested since it was loaded (time 0; never reset).
 * Off by default; process-wide; not thread-safe against concurrent enable/reset. */
lrtei_status lrtei_profile_enable(int on);
lrtei_status lrtei_profile_get(const char* kernel, double* total_ms, int64_t* launches);
void lrtei_profile_reset(void);

/* ---- CUDA-core FMA peak (measurement infrastructure; no counterpart in the paper) -------
 * Runs a throughput-bound FMA kernel (FP64 if fp64 != 0, else FP32) on all SMs of the current
 * device on `stream`, synchronises it, and writes the best of two timed launches in TFLOP/s
 * (2 flops per FMA) to *tflops (host).  Used as the roofline denominator of the FP64/FP32
 * CUDA-core kernels.  Allocates a small output buffer stream-ordered; LRTEI_ERR_CUDA on a
 * device error, LRTEI_ERR_ARG if tflops is NULL. */
lrtei_status lrtei_measure_fma_peak(int fp64, double* tflops, void* stream);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char* lrtei_last_error(void);
/* Library version string. */
const char* lrtei_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LRTEI_H */
