/* lrtei_oracle.h -- plain FP64 CPU oracle of the tensorized approximation (TA) of the
 * long-range two-electron integrals, Badreddine, Chollet & Grigori, arXiv 2210.13069.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load this library.  It shares no code, header, table or constant
 * with the CUDA library; it is the reference its results are checked against.
 *
 * Conventions (the readings of the paper this oracle implements):
 *   - basis functions: contracted Cartesian Gaussians (eq. "basis"/"primi", Section 1);
 *     within a shell of angular momentum l the components are ordered lx = l..0,
 *     ly = l-lx..0, lz = l-lx-ly; every Cartesian component is normalised on R^3
 *     individually and the contraction is normalised to unit self-overlap.
 *   - box [lo_d, hi_d] per dimension (eq. "compact"); centre c_d, half-width b_d.
 *     Default: c_d = midpoint of the atom extent, b_d = half extent + sqrt(ln(1e16)/p_min)
 *     with p_min = 2 * (smallest exponent); a cube (b_d = max_d b_d).
 *   - Chebyshev nodes of the first kind, n per dimension, degrees 0..n-1 (Definition 1).
 *   - Gauss-Legendre nodes z_p, weights w_p on [-1,1]; s_p = omega (1 + z_p) / 2 (eq. TEI2).
 *   - B row index = mu*N_b + nu, column index = kappa*N_b + lambda (mode-(1,2) unfolding).
 */
#ifndef LRTEI_ORACLE_H
#define LRTEI_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_ctx orc_ctx;

/* Shells: centers[ns*3], l[ns], nprim[ns], exps/coefs concatenated in shell order.
 * box_lo/box_hi: NULL for the default box rule.  Returns NULL on invalid input. */
orc_ctx* orc_create(int nshells, const double* centers, const int* l, const int* nprim,
                    const double* exps, const double* coefs, double omega, int n, int P,
                    const double* box_lo, const double* box_hi);
void orc_destroy(orc_ctx* c);
/* Primitive-pair screening (Section 6, "Compression by using Screening"): from now on the
   primitive pair (j1, j2) of (mu, nu) with exp(-a b / (a + b) |A - B|^2) <= tau is discarded (its
   c_j is taken as 0 in every sum over j).  tau = 0 (the default) keeps every pair. */
void orc_set_screening(orc_ctx* c, double tau);

int orc_nbf(const orc_ctx* c);
void orc_box(const orc_ctx* c, double* lo3, double* hi3);
/* per basis function: center[3], powers[3], nprim, and normalised primitive coefficients */
void orc_basis_function(const orc_ctx* c, int mu, double* center3, int* pow3, int* nprim,
                        double* exps, double* coefs);

/* Gauss-Legendre rule on [-1, 1] (Proposition 3), Newton on P_N. */
void orc_gauss_legendre(int N, double* z, double* w);
/* quadrature nodes of eq. TEI2: s_p and the [-1,1] weights w_p */
void orc_nodes(const orc_ctx* c, double* s, double* w);
/* Chebyshev coefficient matrix A^{(p)} for dimension d (Definition 1 / eq. chebcheb), n*n */
void orc_cheb_coeff(const orc_ctx* c, int d, int p, double* A);
/* Moment matrix W~^{(d)}_{mu nu} (eq. defV): (I_mu*I_nu) x n, row j = j1*I_nu + j2 */
void orc_moments(const orc_ctx* c, int mu, int nu, int d, double* W);

/* Algorithm 1: one entry B(mu, nu, kappa, lambda) */
double orc_entry(orc_ctx* c, int mu, int nu, int ka, int la);
/* many entries; idx4 holds (mu, nu, kappa, lambda) quadruples; uses nthreads OpenMP threads */
void orc_entries(orc_ctx* c, const int32_t* idx4, int64_t count, double* out, int nthreads);
/* full B (N_b^2 x N_b^2, row-major) by Algorithm 1 per entry */
void orc_assemble_B(orc_ctx* c, double* B, int nthreads);
/* rows of B: rows[nrows] are row indices mu*N_b+nu; out is nrows x N_b^2 */
void orc_B_rows(orc_ctx* c, const int64_t* rows, int64_t nrows, double* out, int nthreads);

/* Factored form (eq. tensors) with the fast Kronecker product (eq. ig1):
 * J_r = omega/sqrt(pi) * M (sum_p w_p (A_x^p (x) A_y^p (x) A_z^p)) M^T vec(D_r).
 * D: R x N_b x N_b, J: R x N_b x N_b. */
void orc_jbuild_factored(orc_ctx* c, const double* D, int R, double* J, int nthreads);
/* The Khatri-Rao factor M (eq. tensors): N_b^2 x n^3, row mu*N_b+nu, col (m1*n+m2)*n+m3 */
void orc_factor_M(orc_ctx* c, double* M, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
