/* lrtei_oracle.c -- plain, slow FP64 CPU oracle of the tensorized approximation (TA) of the
 * long-range two-electron-integrals tensor B^lr (Badreddine, Chollet, Grigori, arXiv 2210.13069).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU-baseline leg of
 * the benchmark.  It shares no code with the CUDA library.  Every function follows the
 * paper's definitions in the paper's order, in double precision, with no blocking or fusion
 * beyond what a definition states.  Where a value is a pure function of its arguments
 * (the moment matrices of a basis-function pair) it is computed once and kept.
 *
 * Paper sections followed:
 *   Section 1, eq. "basis"/"primi"     contracted Cartesian Gaussian basis
 *   Section 1, eq. "compact"           restriction to a box
 *   Proposition 3 / eq. TEI2           Gauss-Legendre quadrature of the kernel integral over s
 *   Definition 1 / eq. chebcheb        2D Chebyshev interpolation, coefficient formula
 *   eq. approx4 / eq. defV             1D moment integrals W~ of primitive-pair products
 *   Theorem 1 / Algorithm 1            entry-wise evaluation (Hadamard form)
 *   eq. tensors / eq. ig1              Khatri-Rao factor M and mode products of (x)A
 *   eq. coulapprox                     Coulomb (J) application in the factored form
 */
#include "lrtei_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORC_QPTS 24      /* Gauss-Legendre points per panel of the moment quadrature */
#define ORC_WINDOW 10.0  /* integrate |x-P| <= 10/sqrt(p): the rest is below e^-100 */

typedef struct {
  double center[3];
  int pw[3];
  int nprim;
  const double* exps;  /* points into ctx->exps */
  double* coefs;       /* normalised coefficients, owned by ctx->ncoefs */
} orc_bf;

struct orc_ctx {
  int nbf;
  orc_bf* bf;
  double* exps;
  double* ncoefs;
  double omega;
  int n, P;
  double lo[3], hi[3], cen[3], half[3];
  double* s;   /* P */
  double* w;   /* P */
  double* A;   /* 3 * P * n * n */
  double qz[ORC_QPTS], qw[ORC_QPTS];
  double** mom;         /* nbf*nbf*3 slots, each (I_mu I_nu) x n, lazily filled */
  double tau_screening; /* primitive-pair screening threshold (0: keep every pair) */
};

/* ---------------------------------------------------------------- small helpers ---- */

static double dfact(int k) { /* double factorial, (-1)!! = 1 */
  double r = 1.0;
  for (int i = k; i > 1; i -= 2) r *= (double)i;
  return r;
}

/* --------------------------------------------- Gauss-Legendre (Proposition 3) ---- */

void orc_gauss_legendre(int N, double* z, double* w) {
  /* Roots of the Legendre polynomial P_N by Newton's method.  P_k from the three-term
   * recurrence k P_k = (2k-1) x P_{k-1} - (k-1) P_{k-2}; the derivative from
   * P'_k = k P_{k-1} + x P'_{k-1}; weights 2 / ((1 - x)(1 + x) P_N'(x)^2). */
  for (int i = 0; i < N; ++i) {
    double x = cos(M_PI * (i + 0.75) / (N + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 200; ++it) {
      double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
      for (int k = 2; k <= N; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / (double)k;
        double d2 = k * p1 + x * d1;
        p0 = p1; p1 = p2; d0 = d1; d1 = d2;
      }
      (void)d0;
      dp = d1;
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-17) break;
    }
    {
      double p0 = 1.0, p1 = x, d1 = 1.0;
      for (int k = 2; k <= N; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / (double)k;
        double d2 = k * p1 + x * d1;
        p0 = p1; p1 = p2; d1 = d2;
      }
      dp = d1;
    }
    /* store ascending */
    z[N - 1 - i] = x;
    w[N - 1 - i] = 2.0 / ((1.0 - x) * (1.0 + x) * dp * dp);
  }
}

/* -------------------------------------------------------------- context set-up ---- */

orc_ctx* orc_create(int nshells, const double* centers, const int* l, const int* nprim,
                    const double* exps, const double* coefs, double omega, int n, int P,
                    const double* box_lo, const double* box_hi) {
  if (nshells <= 0 || n < 1 || n > 128 || P < 1 || P > 256 || !(omega > 0.0)) return NULL;
  int nb = 0, np = 0;
  for (int s = 0; s < nshells; ++s) {
    if (l[s] < 0 || l[s] > 4 || nprim[s] < 1 || nprim[s] > 16) return NULL;
    nb += (l[s] + 1) * (l[s] + 2) / 2;
    np += nprim[s];
  }
  orc_ctx* c = (orc_ctx*)calloc(1, sizeof(orc_ctx));
  c->nbf = nb;
  c->omega = omega;
  c->n = n;
  c->P = P;
  c->bf = (orc_bf*)calloc((size_t)nb, sizeof(orc_bf));
  c->exps = (double*)malloc(sizeof(double) * (size_t)np);
  memcpy(c->exps, exps, sizeof(double) * (size_t)np);
  /* each basis function gets its own normalised coefficient array */
  int ncoef_total = 0;
  for (int s = 0; s < nshells; ++s) ncoef_total += nprim[s] * (l[s] + 1) * (l[s] + 2) / 2;
  c->ncoefs = (double*)malloc(sizeof(double) * (size_t)ncoef_total);

  int mu = 0, poff = 0, coff = 0;
  double amin = 1e300;
  for (int s = 0; s < nshells; ++s) {
    const int L = l[s], K = nprim[s];
    for (int k = 0; k < K; ++k) amin = fmin(amin, exps[poff + k]);
    for (int lx = L; lx >= 0; --lx) {
      for (int ly = L - lx; ly >= 0; --ly) {
        const int lz = L - lx - ly;
        orc_bf* f = &c->bf[mu];
        for (int d = 0; d < 3; ++d) f->center[d] = centers[3 * s + d];
        f->pw[0] = lx; f->pw[1] = ly; f->pw[2] = lz;
        f->nprim = K;
        f->exps = c->exps + poff;
        f->coefs = c->ncoefs + coff;
        /* primitive normalisation on R^3: int x^{2l} e^{-2 a x^2} dx = (2l-1)!!/(4a)^l sqrt(pi/(2a)) */
        double dfs = dfact(2 * lx - 1) * dfact(2 * ly - 1) * dfact(2 * lz - 1);
        for (int k = 0; k < K; ++k) {
          double a = exps[poff + k];
          double Nk = pow(2.0 * a / M_PI, 0.75) * pow(4.0 * a, 0.5 * L) / sqrt(dfs);
          f->coefs[k] = coefs[poff + k] * Nk;
        }
        /* contraction normalisation: self-overlap of the contracted function on R^3 */
        double S = 0.0;
        for (int k = 0; k < K; ++k)
          for (int q = 0; q < K; ++q) {
            double pq = exps[poff + k] + exps[poff + q];
            double ov = 1.0;
            for (int d = 0; d < 3; ++d)
              ov *= dfact(2 * f->pw[d] - 1) / pow(2.0 * pq, f->pw[d]) * sqrt(M_PI / pq);
            S += f->coefs[k] * f->coefs[q] * ov;
          }
        for (int k = 0; k < K; ++k) f->coefs[k] /= sqrt(S);
        ++mu;
        coff += K;
      }
    }
    poff += K;
  }

  /* box (eq. compact) */
  if (box_lo && box_hi) {
    for (int d = 0; d < 3; ++d) {
      if (!(box_hi[d] > box_lo[d])) { orc_destroy(c); return NULL; }
      c->lo[d] = box_lo[d];
      c->hi[d] = box_hi[d];
    }
  } else {
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int s = 0; s < nshells; ++s)
      for (int d = 0; d < 3; ++d) {
        mn[d] = fmin(mn[d], centers[3 * s + d]);
        mx[d] = fmax(mx[d], centers[3 * s + d]);
      }
    double margin = sqrt(log(1e16) / (2.0 * amin));
    double b = 0.0;
    for (int d = 0; d < 3; ++d) b = fmax(b, 0.5 * (mx[d] - mn[d]) + margin);
    for (int d = 0; d < 3; ++d) {
      double cd = 0.5 * (mx[d] + mn[d]);
      c->lo[d] = cd - b;
      c->hi[d] = cd + b;
    }
  }
  for (int d = 0; d < 3; ++d) {
    c->cen[d] = 0.5 * (c->lo[d] + c->hi[d]);
    c->half[d] = 0.5 * (c->hi[d] - c->lo[d]);
  }

  /* quadrature nodes on [0, omega] (eq. TEI2) */
  c->s = (double*)malloc(sizeof(double) * (size_t)P);
  c->w = (double*)malloc(sizeof(double) * (size_t)P);
  {
    double* z = (double*)malloc(sizeof(double) * (size_t)P);
    orc_gauss_legendre(P, z, c->w);
    for (int p = 0; p < P; ++p) c->s[p] = 0.5 * omega * (1.0 + z[p]);
    free(z);
  }
  /* Chebyshev coefficient matrices (Definition 1, eq. chebcheb) */
  c->A = (double*)malloc(sizeof(double) * 3 * (size_t)P * n * n);
  #pragma omp parallel for schedule(dynamic)
  for (int dp = 0; dp < 3 * P; ++dp) orc_cheb_coeff(c, dp / P, dp % P, c->A + (size_t)dp * n * n);

  orc_gauss_legendre(ORC_QPTS, c->qz, c->qw);
  c->mom = (double**)calloc((size_t)nb * nb * 3, sizeof(double*));
  return c;
}

void orc_destroy(orc_ctx* c) {
  if (!c) return;
  if (c->mom) {
    for (size_t i = 0; i < (size_t)c->nbf * c->nbf * 3; ++i) free(c->mom[i]);
    free(c->mom);
  }
  free(c->bf); free(c->exps); free(c->ncoefs); free(c->s); free(c->w); free(c->A);
  free(c);
}

void orc_set_screening(orc_ctx* c, double tau) { c->tau_screening = tau; }

int orc_nbf(const orc_ctx* c) { return c->nbf; }

void orc_box(const orc_ctx* c, double* lo3, double* hi3) {
  for (int d = 0; d < 3; ++d) { lo3[d] = c->lo[d]; hi3[d] = c->hi[d]; }
}

void orc_basis_function(const orc_ctx* c, int mu, double* center3, int* pow3, int* nprim,
                        double* exps, double* coefs) {
  const orc_bf* f = &c->bf[mu];
  for (int d = 0; d < 3; ++d) { center3[d] = f->center[d]; pow3[d] = f->pw[d]; }
  *nprim = f->nprim;
  for (int k = 0; k < f->nprim; ++k) {
    if (exps) exps[k] = f->exps[k];
    if (coefs) coefs[k] = f->coefs[k];
  }
}

void orc_nodes(const orc_ctx* c, double* s, double* w) {
  for (int p = 0; p < c->P; ++p) { s[p] = c->s[p]; w[p] = c->w[p]; }
}

/* ------------------------------------------------- Chebyshev coefficients ---- */

void orc_cheb_coeff(const orc_ctx* c, int d, int p, double* A) {
  /* alpha_{ab} = c_ab / n^2 * sum_{k,k'} f(u_k, u_k') T_a(u_k) T_b(u_k'),
   * u_k = cos((2k-1) pi / (2n)), c_ab = 1, 2, 4 as a, b are zero or not;
   * f(u, v) = exp(-s_p^2 (x - y)^2) with x = c_d + b_d u, y = c_d + b_d v. */
  const int n = c->n;
  const double sb = c->s[p] * c->half[d];
  /* The kernel values f(u_k, u_k') and the cosines T_a(u_k) = cos(a th_k) are tabulated once
   * (the same expressions as in the double sum, so every term and the summation order are those
   * of the literal sum). */
  double* F = (double*)malloc(sizeof(double) * (size_t)n * n);
  double* Tc = (double*)malloc(sizeof(double) * (size_t)n * n);
  for (int k = 1; k <= n; ++k) {
    double th = (2.0 * k - 1.0) * M_PI / (2.0 * n);
    double uk = cos(th);
    for (int kk = 1; kk <= n; ++kk) {
      double th2 = (2.0 * kk - 1.0) * M_PI / (2.0 * n);
      double vk = cos(th2);
      double diff = uk - vk;
      F[(k - 1) * n + (kk - 1)] = exp(-sb * sb * diff * diff);
    }
    for (int a = 0; a < n; ++a) Tc[a * n + (k - 1)] = cos(a * th);
  }
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      double sum = 0.0;
      for (int k = 1; k <= n; ++k)
        for (int kk = 1; kk <= n; ++kk)
          sum += F[(k - 1) * n + (kk - 1)] * Tc[a * n + (k - 1)] * Tc[b * n + (kk - 1)];
      double cab = (a == 0 && b == 0) ? 1.0 : ((a == 0 || b == 0) ? 2.0 : 4.0);
      A[a * n + b] = cab / ((double)n * n) * sum;
    }
  free(F);
  free(Tc);
}

/* ------------------------------------------------------------ 1D moments ---- */

/* int_{lo_d}^{hi_d} (x-A)^i (x-B)^k exp(-a (x-A)^2 - b (x-B)^2) T_m((x - c_d)/b_d) dx, m < n.
 * Composite Gauss-Legendre; the integrand is integrated over |x - P| <= 10/sqrt(p) inside
 * the box (p = a + b, P = (a A + b B)/p), outside of which it is below e^-100 times the
 * polynomial factor.  Panel width min(0.5/sqrt(p), b_d/8), 24 points per panel. */
static void moment_row(const orc_ctx* c, int d, double a, double Ad, int i, double b, double Bd,
                       int k, double* out) {
  const int n = c->n;
  for (int m = 0; m < n; ++m) out[m] = 0.0;
  const double p = a + b, Pc = (a * Ad + b * Bd) / p;
  double wl = fmax(c->lo[d], Pc - ORC_WINDOW / sqrt(p));
  double wh = fmin(c->hi[d], Pc + ORC_WINDOW / sqrt(p));
  if (!(wh > wl)) return;
  double h = fmin(0.5 / sqrt(p), c->half[d] / 8.0);
  int npan = (int)ceil((wh - wl) / h);
  if (npan < 1) npan = 1;
  double hp = (wh - wl) / npan;
  double T[130];
  for (int q = 0; q < npan; ++q) {
    double x0 = wl + q * hp, mid = x0 + 0.5 * hp, hh = 0.5 * hp;
    for (int t = 0; t < ORC_QPTS; ++t) {
      double x = mid + hh * c->qz[t];
      double wt = hh * c->qw[t];
      double f = pow(x - Ad, i) * pow(x - Bd, k) * exp(-a * (x - Ad) * (x - Ad) - b * (x - Bd) * (x - Bd));
      double u = (x - c->cen[d]) / c->half[d];
      T[0] = 1.0;
      if (n > 1) T[1] = u;
      for (int m = 2; m < n; ++m) T[m] = 2.0 * u * T[m - 1] - T[m - 2];
      for (int m = 0; m < n; ++m) out[m] += wt * f * T[m];
    }
  }
}

void orc_moments(const orc_ctx* c, int mu, int nu, int d, double* W) {
  const orc_bf* f = &c->bf[mu];
  const orc_bf* g = &c->bf[nu];
  for (int j1 = 0; j1 < f->nprim; ++j1)
    for (int j2 = 0; j2 < g->nprim; ++j2) {
      int j = j1 * g->nprim + j2;
      moment_row(c, d, f->exps[j1], f->center[d], f->pw[d], g->exps[j2], g->center[d], g->pw[d],
                 W + (size_t)j * c->n);
    }
}

static const double* moments_cached(const orc_ctx* c, int mu, int nu, int d) {
  return c->mom[((size_t)mu * c->nbf + nu) * 3 + d];
}

/* fill the cache for a list of (mu, nu) pairs, in parallel over pairs */
static void ensure_moments(orc_ctx* c, const int64_t* pairs, int64_t npairs, int nthreads) {
  const int nb = c->nbf;
  int64_t* todo = (int64_t*)malloc(sizeof(int64_t) * (size_t)(npairs > 0 ? npairs : 1));
  char* mark = (char*)calloc((size_t)nb * nb, 1);
  int64_t nt = 0;
  for (int64_t q = 0; q < npairs; ++q) {
    int64_t pr = pairs[q];
    if (c->mom[pr * 3] == NULL && !mark[pr]) { mark[pr] = 1; todo[nt++] = pr; }
  }
  free(mark);
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(dynamic, 4)
#endif
  for (int64_t q = 0; q < nt; ++q) {
    int64_t pr = todo[q];
    int mu = (int)(pr / nb), nu = (int)(pr % nb);
    int I = c->bf[mu].nprim * c->bf[nu].nprim;
    for (int d = 0; d < 3; ++d) {
      double* W = (double*)malloc(sizeof(double) * (size_t)I * c->n);
      orc_moments(c, mu, nu, d, W);
      c->mom[pr * 3 + d] = W;
    }
  }
  (void)nthreads;
  free(todo);
}

/* --------------------------------------------------------------- Algorithm 1 ---- */

/* c_j = c_{j1} c_{j2} of the primitive pair (j1, j2) of (mu, nu) (eq. approx4), or 0 when the pair
   is discarded by screening (Section 6, "Compression by using Screening"):
   exp(-a b / (a + b) |A - B|^2) <= tau_screening with a, b the two exponents and A, B the two
   centres.  A discarded pair contributes nothing to any sum over j. */
static double pair_coef(const orc_ctx* c, const orc_bf* f1, const orc_bf* f2, int j1, int j2) {
  if (c->tau_screening > 0.0) {
    const double a = f1->exps[j1], b = f2->exps[j2];
    double d2 = 0.0;
    for (int l = 0; l < 3; ++l) d2 += (f1->center[l] - f2->center[l]) * (f1->center[l] - f2->center[l]);
    if (exp(-(a * b / (a + b)) * d2) <= c->tau_screening) return 0.0;
  }
  return f1->coefs[j1] * f2->coefs[j2];
}

static double entry_cached(const orc_ctx* c, int mu, int nu, int ka, int la) {
  const int n = c->n, P = c->P;
  const orc_bf *f1 = &c->bf[mu], *f2 = &c->bf[nu], *g1 = &c->bf[ka], *g2 = &c->bf[la];
  const int I1 = f1->nprim * f2->nprim, I2 = g1->nprim * g2->nprim;
  double* cj = (double*)malloc(sizeof(double) * (size_t)(I1 + I2 + I1 * n + 2 * I1 * I2));
  double* cjp = cj + I1;
  double* T = cjp + I2;
  double* G = T + (size_t)I1 * n;
  double* F = G + (size_t)I1 * I2;
  /* c_j = c_{j1} c_{j2} (eq. approx4) */
  for (int j1 = 0; j1 < f1->nprim; ++j1)
    for (int j2 = 0; j2 < f2->nprim; ++j2) cj[j1 * f2->nprim + j2] = pair_coef(c, f1, f2, j1, j2);
  for (int j1 = 0; j1 < g1->nprim; ++j1)
    for (int j2 = 0; j2 < g2->nprim; ++j2) cjp[j1 * g2->nprim + j2] = pair_coef(c, g1, g2, j1, j2);

  double s = 0.0, comp = 0.0; /* Neumaier-compensated sum over the nodes */
  for (int p = 0; p < P; ++p) {
    /* F^{(p)} = Hadamard over d of W~_{mu nu}^{(d)} A^{(p)}_d W~_{ka la}^{(d) T} (Theorem 1) */
    for (int t = 0; t < I1 * I2; ++t) F[t] = 1.0;
    for (int d = 0; d < 3; ++d) {
      const double* Wmn = moments_cached(c, mu, nu, d);
      const double* Wkl = moments_cached(c, ka, la, d);
      const double* A = c->A + ((size_t)d * P + p) * n * n;
      for (int j = 0; j < I1; ++j)
        for (int b = 0; b < n; ++b) {
          double t = 0.0;
          for (int a = 0; a < n; ++a) t += Wmn[(size_t)j * n + a] * A[a * n + b];
          T[(size_t)j * n + b] = t;
        }
      for (int j = 0; j < I1; ++j)
        for (int jp = 0; jp < I2; ++jp) {
          double g = 0.0;
          for (int b = 0; b < n; ++b) g += T[(size_t)j * n + b] * Wkl[(size_t)jp * n + b];
          G[j * I2 + jp] = g;
        }
      for (int t = 0; t < I1 * I2; ++t) F[t] *= G[t];
    }
    /* s = s + w_p sum_{j, j'} c_j c_j' F^{(p)}(j, j') */
    double acc = 0.0;
    for (int j = 0; j < I1; ++j)
      for (int jp = 0; jp < I2; ++jp) acc += cj[j] * cjp[jp] * F[j * I2 + jp];
    double term = c->w[p] * acc;
    double tsum = s + term;
    if (fabs(s) >= fabs(term)) comp += (s - tsum) + term;
    else comp += (term - tsum) + s;
    s = tsum;
  }
  free(cj);
  return c->omega / sqrt(M_PI) * (s + comp);
}

double orc_entry(orc_ctx* c, int mu, int nu, int ka, int la) {
  int64_t pr[2] = {(int64_t)mu * c->nbf + nu, (int64_t)ka * c->nbf + la};
  ensure_moments(c, pr, 2, 1);
  return entry_cached(c, mu, nu, ka, la);
}

void orc_entries(orc_ctx* c, const int32_t* idx4, int64_t count, double* out, int nthreads) {
  const int nb = c->nbf;
  int64_t* pr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * count + 1));
  for (int64_t e = 0; e < count; ++e) {
    pr[2 * e] = (int64_t)idx4[4 * e] * nb + idx4[4 * e + 1];
    pr[2 * e + 1] = (int64_t)idx4[4 * e + 2] * nb + idx4[4 * e + 3];
  }
  ensure_moments(c, pr, 2 * count, nthreads);
  free(pr);
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(dynamic, 16)
#endif
  for (int64_t e = 0; e < count; ++e)
    out[e] = entry_cached(c, idx4[4 * e], idx4[4 * e + 1], idx4[4 * e + 2], idx4[4 * e + 3]);
}

static void ensure_all_moments(orc_ctx* c, int nthreads) {
  const int64_t np = (int64_t)c->nbf * c->nbf;
  int64_t* pr = (int64_t*)malloc(sizeof(int64_t) * (size_t)np);
  for (int64_t q = 0; q < np; ++q) pr[q] = q;
  ensure_moments(c, pr, np, nthreads);
  free(pr);
}

void orc_B_rows(orc_ctx* c, const int64_t* rows, int64_t nrows, double* out, int nthreads) {
  const int nb = c->nbf;
  const int64_t nc = (int64_t)nb * nb;
  ensure_all_moments(c, nthreads);
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(dynamic, 8) collapse(2)
#endif
  for (int64_t r = 0; r < nrows; ++r)
    for (int64_t col = 0; col < nc; ++col) {
      int mu = (int)(rows[r] / nb), nu = (int)(rows[r] % nb);
      int ka = (int)(col / nb), la = (int)(col % nb);
      out[r * nc + col] = entry_cached(c, mu, nu, ka, la);
    }
}

void orc_assemble_B(orc_ctx* c, double* B, int nthreads) {
  const int64_t nr = (int64_t)c->nbf * c->nbf;
  int64_t* rows = (int64_t*)malloc(sizeof(int64_t) * (size_t)nr);
  for (int64_t r = 0; r < nr; ++r) rows[r] = r;
  orc_B_rows(c, rows, nr, B, nthreads);
  free(rows);
}

/* ----------------------------------------------------- factored form (eq. tensors) ---- */

/* row mu*N_b+nu of M: M(mu nu, (m1 n + m2) n + m3) = sum_j c_j W~x(j,m1) W~y(j,m2) W~z(j,m3) */
static void factor_row(const orc_ctx* c, int mu, int nu, double* row) {
  const int n = c->n;
  const orc_bf *f1 = &c->bf[mu], *f2 = &c->bf[nu];
  const double* Wx = moments_cached(c, mu, nu, 0);
  const double* Wy = moments_cached(c, mu, nu, 1);
  const double* Wz = moments_cached(c, mu, nu, 2);
  const size_t n3 = (size_t)n * n * n;
  for (size_t t = 0; t < n3; ++t) row[t] = 0.0;
  for (int j1 = 0; j1 < f1->nprim; ++j1)
    for (int j2 = 0; j2 < f2->nprim; ++j2) {
      int j = j1 * f2->nprim + j2;
      double cj = pair_coef(c, f1, f2, j1, j2);
      for (int m1 = 0; m1 < n; ++m1)
        for (int m2 = 0; m2 < n; ++m2)
          for (int m3 = 0; m3 < n; ++m3)
            row[((size_t)m1 * n + m2) * n + m3] += cj * Wx[(size_t)j * n + m1] * Wy[(size_t)j * n + m2] *
                                                   Wz[(size_t)j * n + m3];
    }
}

void orc_factor_M(orc_ctx* c, double* M, int nthreads) {
  const int nb = c->nbf;
  const size_t n3 = (size_t)c->n * c->n * c->n;
  ensure_all_moments(c, nthreads);
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(dynamic, 4)
#endif
  for (int64_t r = 0; r < (int64_t)nb * nb; ++r) factor_row(c, (int)(r / nb), (int)(r % nb), M + r * n3);
}

/* y = (A_x (x) A_y (x) A_z) x by three mode products (eq. ig1); x, y indexed (m1 n + m2) n + m3 */
static void kron3_apply(int n, const double* Ax, const double* Ay, const double* Az, const double* x,
                        double* y, double* t1, double* t2) {
  for (int a1 = 0; a1 < n; ++a1)
    for (int m2 = 0; m2 < n; ++m2)
      for (int m3 = 0; m3 < n; ++m3) {
        double s = 0.0;
        for (int m1 = 0; m1 < n; ++m1) s += Ax[a1 * n + m1] * x[((size_t)m1 * n + m2) * n + m3];
        t1[((size_t)a1 * n + m2) * n + m3] = s;
      }
  for (int a1 = 0; a1 < n; ++a1)
    for (int a2 = 0; a2 < n; ++a2)
      for (int m3 = 0; m3 < n; ++m3) {
        double s = 0.0;
        for (int m2 = 0; m2 < n; ++m2) s += Ay[a2 * n + m2] * t1[((size_t)a1 * n + m2) * n + m3];
        t2[((size_t)a1 * n + a2) * n + m3] = s;
      }
  for (int a1 = 0; a1 < n; ++a1)
    for (int a2 = 0; a2 < n; ++a2)
      for (int a3 = 0; a3 < n; ++a3) {
        double s = 0.0;
        for (int m3 = 0; m3 < n; ++m3) s += Az[a3 * n + m3] * t2[((size_t)a1 * n + a2) * n + m3];
        y[((size_t)a1 * n + a2) * n + a3] = s;
      }
}

void orc_jbuild_factored(orc_ctx* c, const double* D, int R, double* J, int nthreads) {
  const int nb = c->nbf, n = c->n, P = c->P;
  const int64_t npair = (int64_t)nb * nb;
  const size_t n3 = (size_t)n * n * n;
  ensure_all_moments(c, nthreads);
  double* X = (double*)calloc((size_t)R * n3, sizeof(double)); /* x_r = M^T vec(D_r) */
  double* Y = (double*)calloc((size_t)R * n3, sizeof(double));
  int nth = nthreads > 0 ? nthreads : 1;
  /* pass 1: x_r = M^T vec(D_r), rows of M produced one at a time, per-thread partial sums */
  double* Xp = (double*)calloc((size_t)nth * R * n3, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel num_threads(nth)
#endif
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double* row = (double*)malloc(sizeof(double) * n3);
    double* Xt = Xp + (size_t)tid * R * n3;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 8)
#endif
    for (int64_t r = 0; r < npair; ++r) {
      factor_row(c, (int)(r / nb), (int)(r % nb), row);
      for (int q = 0; q < R; ++q) {
        double dv = D[(size_t)q * npair + r];
        if (dv == 0.0) continue;
        for (size_t t = 0; t < n3; ++t) Xt[(size_t)q * n3 + t] += row[t] * dv;
      }
    }
    free(row);
  }
  for (int t = 0; t < nth; ++t)
    for (size_t e = 0; e < (size_t)R * n3; ++e) X[e] += Xp[(size_t)t * R * n3 + e];
  free(Xp);
  /* y_r = sum_p w_p (A_x^p (x) A_y^p (x) A_z^p) x_r */
#ifdef _OPENMP
#pragma omp parallel for num_threads(nth) schedule(static)
#endif
  for (int q = 0; q < R; ++q) {
    double* t1 = (double*)malloc(sizeof(double) * n3 * 3);
    double* t2 = t1 + n3;
    double* yp = t2 + n3;
    for (int p = 0; p < P; ++p) {
      const double* Ax = c->A + ((size_t)0 * P + p) * n * n;
      const double* Ay = c->A + ((size_t)1 * P + p) * n * n;
      const double* Az = c->A + ((size_t)2 * P + p) * n * n;
      kron3_apply(n, Ax, Ay, Az, X + (size_t)q * n3, yp, t1, t2);
      for (size_t t = 0; t < n3; ++t) Y[(size_t)q * n3 + t] += c->w[p] * yp[t];
    }
    free(t1);
  }
  /* pass 2: vec(J_r) = omega/sqrt(pi) * M y_r */
  const double pref = c->omega / sqrt(M_PI);
#ifdef _OPENMP
#pragma omp parallel num_threads(nth)
#endif
  {
    double* row = (double*)malloc(sizeof(double) * n3);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 8)
#endif
    for (int64_t r = 0; r < npair; ++r) {
      factor_row(c, (int)(r / nb), (int)(r % nb), row);
      for (int q = 0; q < R; ++q) {
        double s = 0.0;
        for (size_t t = 0; t < n3; ++t) s += row[t] * Y[(size_t)q * n3 + t];
        J[(size_t)q * npair + r] = pref * s;
      }
    }
    free(row);
  }
  free(X);
  free(Y);
}
