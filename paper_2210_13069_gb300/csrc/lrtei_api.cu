// lrtei_api.cu -- the C ABI of include/lrtei.h: basis and plan objects, host-side validation,
// workspace management and the orchestration of the device kernels.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "lrtei_internal.h"

namespace lrtei {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

lrtei_status cuda_fail(cudaError_t e, const char* what) {
  set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
  return LRTEI_ERR_CUDA;
}

namespace {
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;
}  // namespace

cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t st) {
  count_alloc();
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it == g_pools.end()) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&pool, &props);
      if (e != cudaSuccess) return e;
      uint64_t keep = 2ULL << 30;
      e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      if (e != cudaSuccess) return e;
      g_pools[dev] = pool;
    } else {
      pool = it->second;
    }
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

lrtei_status finish_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what);
  return LRTEI_OK;
}

}  // namespace lrtei

using namespace lrtei;

struct lrtei_basis {
  int nshells = 0, nbf = 0;
  std::vector<double> centers, exps, coefs;
  std::vector<int> l, nprim, poff;
  std::vector<int> bf_shell, bf_pow, bf_coff;
  int ncoef = 0;
  double amin = 0.0;
};

struct lrtei_plan {
  lrtei_basis basis;
  double omega = 0.0;
  int n = 0, P = 0;
  double lo[3], hi[3];
  lrtei_precision prec = LRTEI_FP64;
  double tau = 0.0;  // primitive-pair screening threshold
  int last_form = 0;
  // adaptive boxes (Section 6): 0 partitions = one box for every pair
  int npart = 0;
  double tau_adapt = 0.0;
  std::vector<int> h_pair_part;        // partition of each unique pair
  std::vector<double> part_b;          // half-width of each partition's cube
  double adapt_c[3] = {0.0, 0.0, 0.0}; // the cubes' common centre
  int* d_pair_part = nullptr;
  uint8_t* d_row_box = nullptr;        // partition of each primitive-pair row (moments' box)
  int cheb_n = 0;         // Chebyshev nodes per dimension (n before a Khatri-Rao compression)
  int kr_rank = 0;        // 0, or the common rank R of the compressed moment matrices (n == R then)
  int kr_ranks[3] = {0, 0, 0};
  PairTable t;
  // device data
  int *d_bf_shell = nullptr, *d_bf_pow = nullptr, *d_shell_nprim = nullptr, *d_shell_poff = nullptr,
      *d_bf_coff = nullptr;
  double *d_shell_center = nullptr, *d_exps = nullptr, *d_coefs = nullptr, *d_ncoef = nullptr;
  double *d_z = nullptr, *d_s = nullptr, *d_w = nullptr, *d_gz = nullptr, *d_gw = nullptr;
  double *d_lo3 = nullptr, *d_hi3 = nullptr, *d_half3 = nullptr;
  double *d_C = nullptr, *d_S = nullptr;
  int* d_status = nullptr;
  // lazily built
  double* d_T = nullptr;      // Hadamard: 3 * P * nrows * n
  double* d_F = nullptr;      // factored: npair * n^3 (FP64)
  float* d_F32 = nullptr;     // factored: npair * n^3 (FP32)
  SplitMatrix Fsp, Ksp, FTsp; // tensor-core operands: F_u, K, F_u^T as BF16 slices
  bool have_Fsp = false, have_Ksp = false, have_FTsp = false;
  HadOperands had;            // tensor-core Hadamard form (one primitive pair per unique pair)
  bool have_had = false;
  std::vector<void*> allocs;
  size_t bytes = 0;

  template <typename T>
  lrtei_status alloc(T** p, size_t count) {
    void* q = nullptr;
    size_t b = count * sizeof(T);
    if (b == 0) b = 16;
    count_alloc();
    cudaError_t e = cudaMalloc(&q, b);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("device allocation of %zu bytes failed: %s", b, cudaGetErrorString(e));
      return LRTEI_ERR_ALLOC;
    }
    allocs.push_back(q);
    bytes += b;
    *p = (T*)q;
    return LRTEI_OK;
  }
  void release(void* q, size_t b) {
    if (!q) return;
    auto it = std::find(allocs.begin(), allocs.end(), q);
    if (it != allocs.end()) {
      allocs.erase(it);
      cudaFree(q);
      bytes -= b;
    }
  }
  ~lrtei_plan() {
    for (void* q : allocs) cudaFree(q);
  }
};

static void forget_plan_graphs(const lrtei_plan* pl);
static lrtei_status jbuild_direct(lrtei_plan* plan, const double* d_D, int R, double* d_J, cudaStream_t st);

#define LRTEI_TRY(expr)                    \
  do {                                     \
    lrtei_status s__ = (expr);             \
    if (s__ != LRTEI_OK) return s__;       \
  } while (0)

static inline int64_t npair_of(int nbf) { return (int64_t)nbf * (nbf + 1) / 2; }

extern "C" {

const char* lrtei_last_error(void) { return g_err.c_str(); }
const char* lrtei_version(void) { return "lrtei 0.1 (sm_103a)"; }

lrtei_status lrtei_basis_create(int nshells, const double* centers, const int* l, const int* nprim,
                                const double* exps, const double* coefs, lrtei_basis** out) {
  if (!out) { set_error("out is NULL"); return LRTEI_ERR_ARG; }
  *out = nullptr;
  if (nshells <= 0 || !centers || !l || !nprim || !exps || !coefs) {
    set_error("invalid basis arguments (nshells=%d)", nshells);
    return LRTEI_ERR_ARG;
  }
  lrtei_basis* b = new lrtei_basis();
  b->nshells = nshells;
  int np = 0;
  for (int s = 0; s < nshells; ++s) {
    if (l[s] < 0 || l[s] > 4 || nprim[s] < 1 || nprim[s] > 16) {
      set_error("shell %d: l=%d nprim=%d out of range (l in 0..4, nprim in 1..16)", s, l[s], nprim[s]);
      delete b;
      return LRTEI_ERR_ARG;
    }
    for (int d = 0; d < 3; ++d)
      if (!isfinite(centers[3 * s + d])) { set_error("shell %d: non-finite centre", s); delete b; return LRTEI_ERR_ARG; }
    b->poff.push_back(np);
    np += nprim[s];
  }
  b->amin = 1e300;
  for (int k = 0; k < np; ++k) {
    if (!(exps[k] > 0.0) || !isfinite(exps[k]) || !isfinite(coefs[k])) {
      set_error("primitive %d: exponent must be > 0 and finite, coefficient finite", k);
      delete b;
      return LRTEI_ERR_ARG;
    }
    b->amin = std::min(b->amin, exps[k]);
  }
  b->centers.assign(centers, centers + 3 * nshells);
  b->l.assign(l, l + nshells);
  b->nprim.assign(nprim, nprim + nshells);
  b->exps.assign(exps, exps + np);
  b->coefs.assign(coefs, coefs + np);
  // Cartesian expansion: lx = l..0, ly = l-lx..0, lz = l-lx-ly
  for (int s = 0; s < nshells; ++s)
    for (int lx = l[s]; lx >= 0; --lx)
      for (int ly = l[s] - lx; ly >= 0; --ly) {
        b->bf_shell.push_back(s);
        b->bf_pow.push_back(lx);
        b->bf_pow.push_back(ly);
        b->bf_pow.push_back(l[s] - lx - ly);
        b->bf_coff.push_back(b->ncoef);
        b->ncoef += nprim[s];
      }
  b->nbf = (int)b->bf_shell.size();
  *out = b;
  return LRTEI_OK;
}

void lrtei_basis_destroy(lrtei_basis* basis) { delete basis; }
int lrtei_basis_nbf(const lrtei_basis* basis) { return basis ? basis->nbf : 0; }

lrtei_status lrtei_plan_create(const lrtei_basis* basis, double omega, int n, int P, const double* box_lo,
                               const double* box_hi, lrtei_precision precision, void* stream, lrtei_plan** out) {
  return lrtei_plan_create_ex(basis, omega, n, P, box_lo, box_hi, precision, 0.0, stream, out);
}

static lrtei_status plan_create_impl(const lrtei_basis* basis, double omega, int n, int P, const double* box_lo,
                                     const double* box_hi, lrtei_precision precision, double tau_screening,
                                     double tau_adapt, int npart, void* stream, lrtei_plan** out);

lrtei_status lrtei_plan_create_ex(const lrtei_basis* basis, double omega, int n, int P, const double* box_lo,
                                  const double* box_hi, lrtei_precision precision, double tau_screening,
                                  void* stream, lrtei_plan** out) {
  return plan_create_impl(basis, omega, n, P, box_lo, box_hi, precision, tau_screening, 0.0, 0, stream, out);
}

lrtei_status lrtei_plan_create_adaptive(const lrtei_basis* basis, double omega, int n, int P, double tau_adaptive,
                                        int npartitions, lrtei_precision precision, void* stream, lrtei_plan** out) {
  if (!out) { set_error("out is NULL"); return LRTEI_ERR_ARG; }
  if (!(tau_adaptive > 0.0 && tau_adaptive < 1.0)) {
    set_error("tau_adaptive must be in (0, 1) (got %g)", tau_adaptive);
    return LRTEI_ERR_ARG;
  }
  if (npartitions < 1 || npartitions > 8) { set_error("npartitions must be in 1..8 (got %d)", npartitions); return LRTEI_ERR_ARG; }
  return plan_create_impl(basis, omega, n, P, nullptr, nullptr, precision, 0.0, tau_adaptive, npartitions, stream, out);
}

}  // extern "C"

static lrtei_status plan_create_impl(const lrtei_basis* basis, double omega, int n, int P, const double* box_lo,
                                     const double* box_hi, lrtei_precision precision, double tau_screening,
                                     double tau_adapt, int npart, void* stream, lrtei_plan** out) {
  if (!out) { set_error("out is NULL"); return LRTEI_ERR_ARG; }
  if (!(tau_screening >= 0.0 && tau_screening <= 1.0)) {
    set_error("tau_screening must be in [0, 1] (got %g)", tau_screening);
    return LRTEI_ERR_ARG;
  }
  *out = nullptr;
  if (!basis) { set_error("basis is NULL"); return LRTEI_ERR_ARG; }
  if (!(omega > 0.0) || !isfinite(omega)) { set_error("omega must be > 0 (got %g)", omega); return LRTEI_ERR_ARG; }
  if (n < 1 || n > kMaxN) { set_error("n must be in 1..%d (got %d)", kMaxN, n); return LRTEI_ERR_ARG; }
  if (P < 1 || P > kMaxP) { set_error("P must be in 1..%d (got %d)", kMaxP, P); return LRTEI_ERR_ARG; }
  if ((box_lo == nullptr) != (box_hi == nullptr)) { set_error("box_lo and box_hi must both be given or both NULL"); return LRTEI_ERR_ARG; }
  if (precision < LRTEI_FP64 || precision > LRTEI_SPLIT_F16_8) { set_error("unknown precision %d", (int)precision); return LRTEI_ERR_ARG; }
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    set_error("no CUDA device available (%s)", cudaGetErrorString(ce));
    return LRTEI_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  lrtei_plan* pl = new lrtei_plan();
  pl->basis = *basis;
  pl->omega = omega;
  pl->n = n;
  pl->P = P;
  pl->prec = precision;
  pl->tau = tau_screening;
  pl->cheb_n = n;
  const lrtei_basis& b = pl->basis;
  // box (eq. compact)
  if (box_lo) {
    for (int d = 0; d < 3; ++d) {
      if (!(box_hi[d] > box_lo[d]) || !isfinite(box_lo[d]) || !isfinite(box_hi[d])) {
        set_error("box: hi[%d] must exceed lo[%d]", d, d);
        delete pl;
        return LRTEI_ERR_ARG;
      }
      pl->lo[d] = box_lo[d];
      pl->hi[d] = box_hi[d];
    }
  } else {
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int s = 0; s < b.nshells; ++s)
      for (int d = 0; d < 3; ++d) {
        mn[d] = std::min(mn[d], b.centers[3 * s + d]);
        mx[d] = std::max(mx[d], b.centers[3 * s + d]);
      }
    const double margin = sqrt(log(1e16) / (2.0 * b.amin));
    double half = 0.0;
    for (int d = 0; d < 3; ++d) half = std::max(half, 0.5 * (mx[d] - mn[d]) + margin);
    for (int d = 0; d < 3; ++d) {
      const double c = 0.5 * (mn[d] + mx[d]);
      pl->lo[d] = c - half;
      pl->hi[d] = c + half;
    }
  }
  // pair table structure (host integer bookkeeping)
  const int nbf = b.nbf;
  PairTable& t = pl->t;
  t.npair = npair_of(nbf);
  if (npart > 0) {
    // Adaptive boxes (Section 6): the support of a unique pair is the smallest cube about the
    // centre c of the atoms' extent holding |x_l - P_{j,l}| < sqrt(ln(1/tau) / p_j) for all its
    // primitive pairs j and dimensions l; the pairs sorted by it (stable) are cut into npart groups
    // of about equal count, each cut moved past a run of equal supports, empty groups dropped.
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300}, c[3];
    for (int s2 = 0; s2 < b.nshells; ++s2)
      for (int d = 0; d < 3; ++d) {
        mn[d] = std::min(mn[d], b.centers[3 * s2 + d]);
        mx[d] = std::max(mx[d], b.centers[3 * s2 + d]);
      }
    for (int d = 0; d < 3; ++d) c[d] = 0.5 * (mn[d] + mx[d]);
    const double lr = log(1.0 / tau_adapt);
    std::vector<double> bsup((size_t)t.npair);
    int64_t r = 0;
    for (int mu = 0; mu < nbf; ++mu)
      for (int nu = mu; nu < nbf; ++nu, ++r) {
        const int s1 = b.bf_shell[mu], s2 = b.bf_shell[nu];
        double bb = 0.0;
        for (int j1 = 0; j1 < b.nprim[s1]; ++j1)
          for (int j2 = 0; j2 < b.nprim[s2]; ++j2) {
            const double a = b.exps[b.poff[s1] + j1], e = b.exps[b.poff[s2] + j2], p = a + e;
            double m = 0.0;
            for (int d = 0; d < 3; ++d)
              m = std::max(m, fabs((a * b.centers[3 * s1 + d] + e * b.centers[3 * s2 + d]) / p - c[d]));
            bb = std::max(bb, m + sqrt(lr / p));
          }
        bsup[r] = bb;
      }
    std::vector<int64_t> order((size_t)t.npair);
    for (int64_t i = 0; i < t.npair; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return bsup[x] < bsup[y]; });
    std::vector<int64_t> cuts{0};
    for (int k = 1; k < npart; ++k) {
      int64_t ct = std::max(cuts.back(), (int64_t)k * t.npair / npart);
      while (ct > 0 && ct < t.npair && bsup[order[ct]] == bsup[order[ct - 1]]) ++ct;
      cuts.push_back(ct);
    }
    cuts.push_back(t.npair);
    pl->h_pair_part.assign((size_t)t.npair, 0);
    for (int k = 0; k < npart; ++k) {
      if (cuts[k + 1] <= cuts[k]) continue;
      double bmax = 0.0;
      for (int64_t i = cuts[k]; i < cuts[k + 1]; ++i) {
        pl->h_pair_part[order[i]] = (int)pl->part_b.size();
        bmax = std::max(bmax, bsup[order[i]]);
      }
      pl->part_b.push_back(bmax);
    }
    pl->npart = (int)pl->part_b.size();
    pl->tau_adapt = tau_adapt;
    for (int d = 0; d < 3; ++d) pl->adapt_c[d] = c[d];
    for (int d = 0; d < 3; ++d) {  // the reported box is the largest partition's
      pl->lo[d] = c[d] - pl->part_b.back();
      pl->hi[d] = c[d] + pl->part_b.back();
    }
  }
  const int nbox = std::max(1, pl->npart);
  // Rows are the primitive pairs (j1, j2) of each unique pair, j1 of mu's shell major; with
  // screening (Section 6) a primitive pair with exp(-a b / (a + b) |A - B|^2) <= tau is left out.
  std::vector<int> pmu(t.npair), pnu(t.npair), pI(t.npair);
  std::vector<int64_t> prow(t.npair + 1);
  std::vector<uint8_t> rprim;
  int64_t r = 0, rows = 0;
  for (int mu = 0; mu < nbf; ++mu)
    for (int nu = mu; nu < nbf; ++nu) {
      const int s1 = b.bf_shell[mu], s2 = b.bf_shell[nu];
      double d2 = 0.0;
      for (int l = 0; l < 3; ++l) d2 += (b.centers[3 * s1 + l] - b.centers[3 * s2 + l]) * (b.centers[3 * s1 + l] - b.centers[3 * s2 + l]);
      int kept = 0;
      for (int j1 = 0; j1 < b.nprim[s1]; ++j1)
        for (int j2 = 0; j2 < b.nprim[s2]; ++j2) {
          const double a = b.exps[b.poff[s1] + j1], e = b.exps[b.poff[s2] + j2];
          if (tau_screening > 0.0 && exp(-(a * e / (a + e)) * d2) <= tau_screening) continue;
          rprim.push_back((uint8_t)((j1 << 4) | j2));
          ++kept;
        }
      pmu[r] = mu;
      pnu[r] = nu;
      pI[r] = kept;
      t.maxI = std::max(t.maxI, pI[r]);
      prow[r] = rows;
      rows += pI[r];
      ++r;
    }
  prow[t.npair] = rows;
  t.nrows = rows;

  lrtei_status s;
#define PA(ptr, cnt)                           \
  if ((s = pl->alloc(&(ptr), (cnt))) != LRTEI_OK) { delete pl; return s; }
  PA(pl->d_bf_shell, nbf);
  PA(pl->d_bf_pow, 3 * nbf);
  PA(pl->d_bf_coff, nbf);
  PA(pl->d_shell_nprim, b.nshells);
  PA(pl->d_shell_poff, b.nshells);
  PA(pl->d_shell_center, 3 * b.nshells);
  PA(pl->d_exps, b.exps.size());
  PA(pl->d_coefs, b.coefs.size());
  PA(pl->d_ncoef, b.ncoef);
  PA(pl->d_z, P);
  PA(pl->d_s, P);
  PA(pl->d_w, P);
  PA(pl->d_gz, kMomentPts);
  PA(pl->d_gw, kMomentPts);
  PA(pl->d_lo3, 3 * nbox);
  PA(pl->d_hi3, 3 * nbox);
  PA(pl->d_half3, 3 * nbox);
  PA(pl->d_C, (size_t)nbox * nbox * 3 * P * n * n);
  if (pl->npart > 0) {
    PA(pl->d_pair_part, t.npair);
    PA(pl->d_row_box, t.nrows);
  }
  PA(pl->d_S, (size_t)3 * t.nrows * n);
  PA(pl->d_status, 1);
  PA(t.pair_mu, t.npair);
  PA(t.pair_nu, t.npair);
  PA(t.pair_row, t.npair + 1);
  PA(t.pair_I, t.npair);
  PA(t.row_pair, t.nrows);
  PA(t.row_c, t.nrows);
  PA(t.row_p, t.nrows);
  PA(t.row_P, 3 * t.nrows);
  PA(t.row_K, 3 * t.nrows);
  PA(t.row_A, 3 * t.nrows);
  PA(t.row_B, 3 * t.nrows);
  PA(t.row_pa, 3 * t.nrows);
  PA(t.row_pb, 3 * t.nrows);
  PA(t.row_prim, t.nrows);
#undef PA
  std::vector<double> lo3(3 * (size_t)nbox), hi3(3 * (size_t)nbox), half3(3 * (size_t)nbox);
  for (int k = 0; k < nbox; ++k)
    for (int d = 0; d < 3; ++d) {
      lo3[3 * k + d] = pl->npart > 0 ? pl->adapt_c[d] - pl->part_b[k] : pl->lo[d];
      hi3[3 * k + d] = pl->npart > 0 ? pl->adapt_c[d] + pl->part_b[k] : pl->hi[d];
      half3[3 * k + d] = 0.5 * (hi3[3 * k + d] - lo3[3 * k + d]);
    }
  std::vector<uint8_t> row_box;
  if (pl->npart > 0) {
    row_box.resize((size_t)t.nrows);
    for (int64_t r2 = 0; r2 < t.npair; ++r2)
      for (int64_t j = prow[r2]; j < prow[r2 + 1]; ++j) row_box[j] = (uint8_t)pl->h_pair_part[r2];
  }
#define UP(dst, src, cnt)                                                                                 \
  if ((ce = cudaMemcpyAsync((dst), (src), sizeof(*(src)) * (cnt), cudaMemcpyHostToDevice, st)) != cudaSuccess) { \
    delete pl;                                                                                            \
    return cuda_fail(ce, "upload " #dst);                                                                 \
  }
  UP(pl->d_bf_shell, b.bf_shell.data(), nbf);
  UP(pl->d_bf_pow, b.bf_pow.data(), 3 * nbf);
  UP(pl->d_bf_coff, b.bf_coff.data(), nbf);
  UP(pl->d_shell_nprim, b.nprim.data(), b.nshells);
  UP(pl->d_shell_poff, b.poff.data(), b.nshells);
  UP(pl->d_shell_center, b.centers.data(), 3 * b.nshells);
  UP(pl->d_exps, b.exps.data(), b.exps.size());
  UP(pl->d_coefs, b.coefs.data(), b.coefs.size());
  UP(pl->d_lo3, lo3.data(), 3 * nbox);
  UP(pl->d_hi3, hi3.data(), 3 * nbox);
  UP(pl->d_half3, half3.data(), 3 * nbox);
  if (pl->npart > 0) {
    UP(pl->d_pair_part, pl->h_pair_part.data(), t.npair);
    if (t.nrows > 0) UP(pl->d_row_box, row_box.data(), t.nrows);
  }
  UP(t.pair_mu, pmu.data(), t.npair);
  UP(t.pair_nu, pnu.data(), t.npair);
  UP(t.pair_row, prow.data(), t.npair + 1);
  UP(t.pair_I, pI.data(), t.npair);
  if (t.nrows > 0) UP(t.row_prim, rprim.data(), t.nrows);
#undef UP
  // The uploads above are from pageable memory: they complete (staged) before returning.
  ce = cudaMemsetAsync(pl->d_status, 0, sizeof(int), st);
  if (ce != cudaSuccess) { delete pl; return cuda_fail(ce, "status reset"); }
  launch_normalise(nbf, pl->d_bf_shell, pl->d_bf_pow, pl->d_shell_nprim, pl->d_shell_poff, pl->d_exps, pl->d_coefs,
                   pl->d_bf_coff, pl->d_ncoef, st);
  launch_pair_rows(t, pl->d_bf_shell, pl->d_bf_pow, pl->d_shell_nprim, pl->d_shell_poff, pl->d_shell_center,
                   pl->d_exps, pl->d_bf_coff, pl->d_ncoef, st);
  launch_gauss_legendre(P, pl->d_z, pl->d_w, st);
  launch_nodes_map(P, omega, pl->d_z, pl->d_s, st);
  launch_gauss_legendre(kMomentPts, pl->d_gz, pl->d_gw, st);
  if (pl->npart == 0) {
    launch_cheb_coeff(n, P, pl->d_s, pl->d_half3, pl->d_C, st);
  } else {  // one coefficient block per ordered partition pair (s, t): x in box s, y in box t
    for (int s1 = 0; s1 < nbox; ++s1)
      for (int s2 = 0; s2 < nbox; ++s2)
        launch_cheb_coeff_cross(n, P, pl->d_s, pl->d_half3 + 3 * s1, pl->d_half3 + 3 * s2,
                                pl->d_C + (size_t)(s1 * nbox + s2) * 3 * P * n * n, st);
  }
  // Moments of the distinct keys (shell pair, primitive pair, d, powers in d) only, gathered into
  // the rows afterwards: rows that share a key have identical inputs, so S is the same as computed
  // row by row (about half the work for an s/p/d basis).
  {
    const int ns = b.nshells;
    std::vector<int64_t> sp_off((size_t)ns * (ns + 1) / 2);
    int64_t nkeys = 0;
    for (int s1 = 0, k = 0; s1 < ns; ++s1)
      for (int s2 = s1; s2 < ns; ++s2, ++k) {
        sp_off[k] = nkeys;
        nkeys += (int64_t)b.nprim[s1] * b.nprim[s2] * 3 * (b.l[s1] + 1) * (b.l[s2] + 1);
      }
    if (nkeys >= (int64_t)INT32_MAX) {  // keys are 32-bit: compute every row's moments directly
      ProfScope ps("moments", st);
      launch_moments(t, n, pl->d_lo3, pl->d_hi3, pl->d_row_box, pl->d_gz, pl->d_gw, nullptr, 3 * t.nrows, pl->d_S, st);
    } else {
      int* d_key = nullptr;
      int* d_l = nullptr;
      int64_t *d_rep = nullptr, *d_off = nullptr;
      double* d_Su = nullptr;
      auto fin = [&](cudaError_t e, const char* what) {
        for (void* q : {(void*)d_key, (void*)d_l, (void*)d_rep, (void*)d_off, (void*)d_Su})
          if (q) cudaFreeAsync(q, st);
        if (e != cudaSuccess) { delete pl; return cuda_fail(e, what); }
        return LRTEI_OK;
      };
      if ((ce = scratch_alloc((void**)&d_key, sizeof(int) * 3 * (size_t)t.nrows, st)) != cudaSuccess ||
          (ce = scratch_alloc((void**)&d_l, sizeof(int) * (size_t)ns, st)) != cudaSuccess ||
          (ce = scratch_alloc((void**)&d_rep, sizeof(int64_t) * (size_t)nkeys, st)) != cudaSuccess ||
          (ce = scratch_alloc((void**)&d_off, sizeof(int64_t) * sp_off.size(), st)) != cudaSuccess ||
          (ce = scratch_alloc((void**)&d_Su, sizeof(double) * (size_t)nkeys * n, st)) != cudaSuccess)
        return fin(ce, "moment key scratch");
      if ((ce = cudaMemcpyAsync(d_l, b.l.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
          (ce = cudaMemcpyAsync(d_off, sp_off.data(), sizeof(int64_t) * sp_off.size(), cudaMemcpyHostToDevice, st)) !=
              cudaSuccess ||
          (ce = cudaMemsetAsync(d_rep, 0xFF, sizeof(int64_t) * (size_t)nkeys, st)) != cudaSuccess)
        return fin(ce, "moment key upload");
      launch_moment_keys(t, pl->d_bf_shell, pl->d_bf_pow, pl->d_shell_nprim, d_l, d_off, ns, d_key, d_rep, st);
      {
        ProfScope ps("moments", st);
        launch_moments(t, n, pl->d_lo3, pl->d_hi3, pl->d_row_box, pl->d_gz, pl->d_gw, d_rep, nkeys, d_Su, st);
      }
      launch_gather_moments(3 * t.nrows, n, d_key, d_Su, pl->d_S, st);
      if ((s = fin(cudaGetLastError(), "moment kernels")) != LRTEI_OK) return s;
    }
  }
  if ((s = finish_launch("plan set-up kernels")) != LRTEI_OK) { delete pl; return s; }
  *out = pl;
  return LRTEI_OK;
}

extern "C" {

void lrtei_plan_destroy(lrtei_plan* plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  forget_plan_graphs(plan);
  delete plan;
}

lrtei_status lrtei_plan_info_get(const lrtei_plan* plan, lrtei_plan_info* info) {
  if (!plan || !info) { set_error("NULL argument"); return LRTEI_ERR_ARG; }
  info->nbf = plan->basis.nbf;
  info->npair = plan->t.npair;
  info->nrows = plan->t.nrows;
  info->n = plan->n;
  info->P = plan->P;
  info->omega = plan->omega;
  for (int d = 0; d < 3; ++d) { info->box_lo[d] = plan->lo[d]; info->box_hi[d] = plan->hi[d]; }
  info->precision = plan->prec;
  info->last_form = plan->last_form;
  info->workspace_bytes = plan->bytes;
  info->tau_screening = plan->tau;
  info->cheb_n = plan->cheb_n;
  info->kr_rank = plan->kr_rank;
  info->npartitions = plan->npart;
  for (int k = 0; k < 8; ++k) info->partition_b[k] = k < plan->npart ? plan->part_b[k] : 0.0;
  return LRTEI_OK;
}

lrtei_status lrtei_plan_status(lrtei_plan* plan) {
  if (!plan) { set_error("plan is NULL"); return LRTEI_ERR_ARG; }
  LRTEI_CUDA(cudaDeviceSynchronize());
  int h = 0;
  LRTEI_CUDA(cudaMemcpy(&h, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  LRTEI_CUDA(cudaMemset(plan->d_status, 0, sizeof(int)));
  if (h == kDevTimeout) { set_error("a device-side bounded wait gave up"); return LRTEI_ERR_TIMEOUT; }
  if (h == kDevNonFinite) { set_error("non-finite value detected on the device"); return LRTEI_ERR_NUMERIC; }
  if (h == kDevBadIndex) { set_error("an index list held a basis-function index outside [0, N_b)"); return LRTEI_ERR_ARG; }
  return LRTEI_OK;
}

}  // extern "C"

namespace lrtei {
__global__ void k_scale_copy_rows(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t rows, int64_t cols,
                                  double scale) {
  const int64_t total = rows * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / cols, j = t % cols;
    dst[i * ldd + j] = scale * src[i * lds + j];
  }
}
}  // namespace lrtei

static void scale_copy_rows(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t rows, int64_t cols,
                     double scale, cudaStream_t st) {
  int64_t b = (rows * cols + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (rows * cols > 0) count_launch();
  if (rows * cols > 0) lrtei::k_scale_copy_rows<<<(unsigned)b, 256, 0, st>>>(src, lds, dst, ldd, rows, cols, scale);
}

// ------------------------------------------------------------------ internals of the forms
namespace {

const double kPi = 3.14159265358979323846;

lrtei_status ensure_T(lrtei_plan* pl, cudaStream_t st) {
  if (pl->d_T) return LRTEI_OK;
  LRTEI_TRY(pl->alloc(&pl->d_T, (size_t)3 * pl->P * pl->t.nrows * pl->n));
  launch_tmat(pl->t.nrows, pl->n, pl->P, pl->d_S, pl->d_C, pl->d_T, st);
  return finish_launch("tmat");
}

bool is_split(const lrtei_plan* pl);

lrtei_status ensure_F64(lrtei_plan* pl, cudaStream_t st) {
  if (pl->d_F) return LRTEI_OK;
  const int64_t n3 = (int64_t)pl->n * pl->n * pl->n;
  LRTEI_TRY(pl->alloc(&pl->d_F, (size_t)pl->t.npair * n3));
  {
    ProfScope ps("build_F", st);
    // the tensor-core precisions read F_u through 30-bit slices: FP32 pairs (~2^-44) suffice
    if (is_split(pl)) launch_build_F_pairs(pl->t, pl->n, pl->d_S, 0, pl->t.npair, pl->d_F, n3, st);
    else launch_build_F<double>(pl->t, pl->n, pl->d_S, 0, pl->t.npair, pl->d_F, n3, st);
  }
  return finish_launch("build_F");
}

lrtei_status ensure_F32(lrtei_plan* pl, cudaStream_t st) {
  if (pl->d_F32) return LRTEI_OK;
  const int64_t n3 = (int64_t)pl->n * pl->n * pl->n;
  LRTEI_TRY(pl->alloc(&pl->d_F32, (size_t)pl->t.npair * n3));
  launch_build_F<float>(pl->t, pl->n, pl->d_S, 0, pl->t.npair, pl->d_F32, n3, st);
  return finish_launch("build_F32");
}

bool is_split(const lrtei_plan* pl) {
  return pl->prec == LRTEI_SPLIT_F16 || pl->prec == LRTEI_SPLIT_F16_8 || pl->prec == LRTEI_BF16;
}
bool eight_products(const lrtei_plan* pl) { return pl->prec == LRTEI_SPLIT_F16_8; }
int nslices(const lrtei_plan* pl) { return pl->prec == LRTEI_BF16 ? 1 : 3; }

lrtei_status alloc_split(lrtei_plan* pl, SplitMatrix& m, int64_t rows, int64_t k, bool with_s1h) {
  m.rows = rows;
  m.kpad = kpad256(k);
  m.plain = pl->prec == LRTEI_BF16;
  m.eight = eight_products(pl);
  const size_t cnt = (size_t)rows * m.kpad;
  LRTEI_TRY(pl->alloc(&m.s0, cnt));
  if (!m.plain) {
    LRTEI_TRY(pl->alloc(&m.s1, cnt));
    LRTEI_TRY(pl->alloc(&m.s2, cnt));
    if (with_s1h || m.eight) LRTEI_TRY(pl->alloc(&m.s1h, cnt));
  }
  LRTEI_TRY(pl->alloc(&m.expo, rows));
  return LRTEI_OK;
}

// Captured J-build graphs hold the plan's operand pointers: they are dropped before any of the
// plan's buffers is freed (an operand rebuilt with another layout would otherwise be read
// through its freed address by the next replay).
void release_split(lrtei_plan* pl, SplitMatrix& m) {
  forget_plan_graphs(pl);
  const size_t b = (size_t)m.rows * m.kpad * sizeof(uint16_t);
  pl->release(m.s0, b);
  pl->release(m.s1, b);
  pl->release(m.s2, b);
  pl->release(m.s1h, b);
  pl->release(m.expo, (size_t)m.rows * sizeof(int));
  m = SplitMatrix();
}

// F_u slices.  The fourth plane (t1 / 2^12) is only needed when F_u is the B operand (the
// assembly B_u = G F_u^T); J-builds use F_u as the A operand only.
lrtei_status ensure_Fsp(lrtei_plan* pl, cudaStream_t st, bool need_s1h) {
  if (pl->have_Fsp && (!need_s1h || pl->Fsp.plain || pl->Fsp.s1h)) return LRTEI_OK;
  if (pl->have_Fsp) {
    release_split(pl, pl->Fsp);
    pl->have_Fsp = false;
  }
  const int64_t n3 = (int64_t)pl->n * pl->n * pl->n;
  LRTEI_TRY(ensure_F64(pl, st));
  LRTEI_TRY(alloc_split(pl, pl->Fsp, pl->t.npair, n3, need_s1h));
  {
    ProfScope ps("split", st);
    launch_split_rows(pl->d_F, pl->t.npair, n3, n3, pl->Fsp, need_s1h, nslices(pl), st);
  }
  pl->have_Fsp = true;
  return finish_launch("split F");
}

// A split-precision plan keeps no FP64 copy of F_u once both slice layouts exist.
void drop_F64_if_sliced(lrtei_plan* pl, cudaStream_t st) {
  if (!is_split(pl) || !pl->d_F || !pl->have_Fsp || !pl->have_FTsp) return;
  cudaStreamSynchronize(st);  // the slicing kernels read d_F
  const int64_t n3 = (int64_t)pl->n * pl->n * pl->n;
  forget_plan_graphs(pl);
  pl->release(pl->d_F, sizeof(double) * (size_t)pl->t.npair * n3);
  pl->d_F = nullptr;
}

// Scratch buffer owned by the call (freed at the end of the call, stream-ordered).
struct Scratch {
  std::vector<void*> ptrs;
  cudaStream_t st;
  explicit Scratch(cudaStream_t s) : st(s) {}
  template <typename T>
  lrtei_status get(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = scratch_alloc(&q, std::max<size_t>(16, count * sizeof(T)), st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("scratch allocation of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
      return LRTEI_ERR_ALLOC;
    }
    ptrs.push_back(q);
    *p = (T*)q;
    return LRTEI_OK;
  }
  ~Scratch() {
    for (void* q : ptrs) cudaFreeAsync(q, st);
  }
};

// Dense K = (omega / sqrt(pi)) sum_p w_p A_x^p (x) A_y^p (x) A_z^p as slices: the prefactor of
// eq. approx33 is carried by K, so that every tensor-core GEMM runs with scale 1 and its
// epilogue needs no FP64 multiply.  The fourth plane only when K is the B operand (G = F_u K);
// the J-build uses K as the A operand.
lrtei_status ensure_Ksp(lrtei_plan* pl, cudaStream_t st, bool need_s1h) {
  if (pl->have_Ksp && (!need_s1h || pl->Ksp.plain || pl->Ksp.s1h)) return LRTEI_OK;
  if (pl->have_Ksp) {
    release_split(pl, pl->Ksp);
    pl->have_Ksp = false;
  }
  const int64_t n3 = (int64_t)pl->n * pl->n * pl->n;
  Scratch sc(st);
  double* K;
  LRTEI_TRY(sc.get(&K, (size_t)n3 * n3));
  {
    ProfScope ps("build_K", st);
    LRTEI_CUDA(launch_build_K(pl->n, pl->P, pl->d_C, pl->d_w, pl->omega / sqrt(kPi), K, st));
  }
  LRTEI_TRY(alloc_split(pl, pl->Ksp, n3, n3, need_s1h));
  {
    ProfScope ps("split", st);
    launch_split_rows(K, n3, n3, n3, pl->Ksp, need_s1h, nslices(pl), st);
  }
  pl->have_Ksp = true;
  return finish_launch("split K");
}

lrtei_status ensure_FTsp(lrtei_plan* pl, cudaStream_t st) {
  if (pl->have_FTsp) return LRTEI_OK;
  const int64_t n3 = (int64_t)pl->n * pl->n * pl->n, npair = pl->t.npair;
  LRTEI_TRY(ensure_F64(pl, st));
  Scratch sc(st);
  double* FT;
  LRTEI_TRY(sc.get(&FT, (size_t)n3 * npair));
  launch_transpose(pl->d_F, npair, n3, n3, FT, npair, st);
  LRTEI_TRY(alloc_split(pl, pl->FTsp, n3, npair, false));
  {
    ProfScope ps("split", st);
    launch_split_rows(FT, n3, npair, npair, pl->FTsp, false, nslices(pl), st);
  }
  pl->have_FTsp = true;
  return finish_launch("split F^T");
}

// Operands of the tensor-core J-build: F_u^T and F_u (A operands) and K (A operand).
lrtei_status ensure_jbuild_operands(lrtei_plan* pl, cudaStream_t st) {
  LRTEI_TRY(ensure_FTsp(pl, st));
  LRTEI_TRY(ensure_Fsp(pl, st, false));
  LRTEI_TRY(ensure_Ksp(pl, st, false));
  drop_F64_if_sliced(pl, st);
  return LRTEI_OK;
}

// A scratch split operand (planes owned by the call).
lrtei_status scratch_split(Scratch& sc, SplitMatrix& m, int64_t rows, int64_t k, bool with_s1h, const lrtei_plan* pl) {
  m.rows = rows;
  m.kpad = kpad256(k);
  m.plain = pl->prec == LRTEI_BF16;
  m.eight = eight_products(pl);
  const size_t cnt = (size_t)rows * m.kpad;
  LRTEI_TRY(sc.get(&m.s0, cnt));
  if (!m.plain) {
    LRTEI_TRY(sc.get(&m.s1, cnt));
    LRTEI_TRY(sc.get(&m.s2, cnt));
    if (with_s1h || m.eight) LRTEI_TRY(sc.get(&m.s1h, cnt));
  }
  LRTEI_TRY(sc.get(&m.expo, rows));
  return LRTEI_OK;
}

// Positive integer from the environment (0 when unset): the host-output pipeline's band count
// and copy chunk, for tests that need many bands on a small molecule.
static int64_t env_count(const char* name) {
  const char* v = getenv(name);
  return (v && *v) ? std::max<long long>(0, atoll(v)) : 0;
}

// Split-K count of a skinny tensor-core product (M rows, K deep); LRTEI_SPLITK overrides it.
int splits_for(int64_t M, int64_t K) {
  const int64_t tiles = (M + 127) / 128;
  int64_t s = (kpad256(K) + 32767) / 32768;
  const int64_t forced = env_count("LRTEI_SPLITK");
  if (forced > 0) return (int)std::max(s, std::min<int64_t>(forced, kpad256(K) / 256));
  while (tiles * s < 2 * 152 && s * 256 * 2 <= kpad256(K)) s *= 2;
  return (int)s;
}

// Rows [r0, r1) of B_u through the tensor-core GEMMs (split precision); the prefactor is in K.
lrtei_status bu_rows_tc(lrtei_plan* pl, int64_t r0, int64_t r1, double* out, int64_t ld, cudaStream_t st) {
  const int64_t n3 = (int64_t)pl->n * pl->n * pl->n, npair = pl->t.npair, nr = r1 - r0;
  LRTEI_TRY(ensure_Fsp(pl, st, true));
  LRTEI_TRY(ensure_Ksp(pl, st, true));
  Scratch sc(st);
  double* G;
  LRTEI_TRY(sc.get(&G, (size_t)nr * n3));
  SplitMatrix Fr = pl->Fsp;  // row view [r0, r1)
  Fr.rows = nr;
  Fr.s0 += r0 * Fr.kpad;
  if (Fr.s1h) Fr.s1h += r0 * Fr.kpad;
  if (Fr.s1) Fr.s1 += r0 * Fr.kpad;
  if (Fr.s2) Fr.s2 += r0 * Fr.kpad;
  Fr.expo += r0;
  LRTEI_TRY(tc_gemm(Fr, pl->Ksp, nr, n3, 1.0, G, n3, false, false, 1, nullptr, pl->d_status, st));
  SplitMatrix Gs;
  LRTEI_TRY(scratch_split(sc, Gs, nr, n3, false, pl));
  {
    ProfScope ps("split", st);
    launch_split_rows(G, nr, n3, n3, Gs, false, nslices(pl), st);
  }
  const bool sym = (r0 == 0 && r1 == npair && ld == npair);
  return tc_gemm(Gs, pl->Fsp, nr, npair, 1.0, out, ld, false, sym, 1, nullptr, pl->d_status, st);
}

// B into page-locked host memory through the tensor-core path.  B_u is computed in bands of
// 128-row blocks of its upper triangle (G_b = F_u,b K, then the band's blocks of G_b F_u^T, each
// written with its mirror), so that after band b every B_u row below the band's end is complete.
// The rows a N_b + b of B whose pairs are all complete (every a with pair(a, N_b - 1) done) are
// expanded into one of two device staging slots and copied to the host by a copy engine on a
// second stream, while the next band runs on the tensor cores.  Bands have equal GEMM work: block
// row i costs ~ n^3 (its rows of G) + npair - 128 i (its part of the triangle).
static lrtei_status assemble_B_host_banded(lrtei_plan* pl, double* hB, int64_t ld, cudaStream_t st) {
  const int nbf = pl->basis.nbf;
  const int64_t nb2 = (int64_t)nbf * nbf, npair = pl->t.npair, n3 = (int64_t)pl->n * pl->n * pl->n;
  LRTEI_TRY(ensure_Fsp(pl, st, true));
  LRTEI_TRY(ensure_Ksp(pl, st, true));
  const int64_t nblk = (npair + 127) / 128;
  int64_t nbands = env_count("LRTEI_HOST_BANDS");
  if (nbands <= 0) nbands = 16;
  nbands = std::min(nbands, nblk);
  std::vector<int64_t> edge{0};  // band edges in 128-row blocks
  {
    double total = 0.0, acc = 0.0;
    for (int64_t i = 0; i < nblk; ++i) total += (double)(n3 + npair - 128 * i);
    for (int64_t i = 0; i < nblk; ++i) {
      acc += (double)(n3 + npair - 128 * i);
      if (acc >= total * (double)edge.size() / (double)nbands && i + 1 < nblk) edge.push_back(i + 1);
    }
    edge.push_back(nblk);
  }
  int64_t maxrows = 0;
  for (size_t k = 0; k + 1 < edge.size(); ++k)
    maxrows = std::max(maxrows, std::min(npair, 128 * edge[k + 1]) - 128 * edge[k]);
  int64_t chunk = env_count("LRTEI_HOST_CHUNK_ROWS");
  if (chunk <= 0) chunk = std::max<int64_t>(1, (int64_t)((512ULL << 20) / (sizeof(double) * (size_t)nb2)));
  chunk = std::min(chunk, nb2);
  Scratch sc(st);
  double *Bu, *G, *stage[2];
  LRTEI_TRY(sc.get(&Bu, (size_t)npair * npair));
  LRTEI_TRY(sc.get(&G, (size_t)maxrows * n3));
  LRTEI_TRY(sc.get(&stage[0], (size_t)chunk * nb2));
  LRTEI_TRY(sc.get(&stage[1], (size_t)chunk * nb2));
  SplitMatrix Gs;
  LRTEI_TRY(scratch_split(sc, Gs, maxrows, n3, false, pl));
  cudaStream_t cs = nullptr;
  cudaEvent_t ready[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr}, fin = nullptr;
  lrtei_status status = LRTEI_OK;
  auto fail = [&](cudaError_t e, const char* what) { if (status == LRTEI_OK) status = cuda_fail(e, what); };
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "copy stream");
  for (int i = 0; i < 2 && status == LRTEI_OK; ++i) {
    if ((e = cudaEventCreateWithFlags(&ready[i], cudaEventDisableTiming)) != cudaSuccess) fail(e, "event");
    else if ((e = cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming)) != cudaSuccess) fail(e, "event");
  }
  if (status == LRTEI_OK && (e = cudaEventCreateWithFlags(&fin, cudaEventDisableTiming)) != cudaSuccess) fail(e, "event");
  int64_t a_done = 0, nchunk = 0;
  for (size_t k = 0; k + 1 < edge.size() && status == LRTEI_OK; ++k) {
    const int64_t r0 = 128 * edge[k], r1 = std::min(npair, 128 * edge[k + 1]), nr = r1 - r0;
    SplitMatrix Fr = pl->Fsp;  // row view [r0, r1)
    Fr.rows = nr;
    Fr.s0 += r0 * Fr.kpad;
    if (Fr.s1h) Fr.s1h += r0 * Fr.kpad;
    if (Fr.s1) Fr.s1 += r0 * Fr.kpad;
    if (Fr.s2) Fr.s2 += r0 * Fr.kpad;
    Fr.expo += r0;
    if ((status = tc_gemm(Fr, pl->Ksp, nr, n3, 1.0, G, n3, false, false, 1, nullptr, pl->d_status, st)) != LRTEI_OK) break;
    Gs.rows = nr;
    {
      ProfScope ps("split", st);
      launch_split_rows(G, nr, n3, n3, Gs, false, nslices(pl), st);
    }
    if ((status = tc_gemm_sym_band(Gs, pl->Fsp, r0, r1, npair, Bu, npair, pl->d_status, st)) != LRTEI_OK) break;
    // basis functions a whose pairs (a, b >= a) all lie below r1: rows [a_done N_b, a_end N_b) of B
    int64_t a_end = a_done;
    while (a_end < nbf && a_end * nbf - a_end * (a_end - 1) / 2 + (nbf - 1 - a_end) < r1) ++a_end;
    for (int64_t R = a_done * nbf; R < a_end * nbf && status == LRTEI_OK; R += chunk, ++nchunk) {
      const int64_t Rn = std::min(a_end * nbf, R + chunk);
      const int slot = (int)(nchunk & 1);
      if (nchunk >= 2 && (e = cudaStreamWaitEvent(st, copied[slot], 0)) != cudaSuccess) { fail(e, "wait copy"); break; }
      {
        ProfScope ps("expand_B", st);
        launch_expand_B_rows(nbf, Bu, npair, R, Rn, stage[slot], nb2, pl->d_status, st);
      }
      if ((status = finish_launch("expand_B_rows")) != LRTEI_OK) break;
      if ((e = cudaEventRecord(ready[slot], st)) != cudaSuccess) { fail(e, "record"); break; }
      if ((e = cudaStreamWaitEvent(cs, ready[slot], 0)) != cudaSuccess) { fail(e, "wait expand"); break; }
      if (ld == nb2)
        e = cudaMemcpyAsync(hB + R * ld, stage[slot], sizeof(double) * (size_t)(Rn - R) * nb2, cudaMemcpyDeviceToHost, cs);
      else
        e = cudaMemcpy2DAsync(hB + R * ld, sizeof(double) * ld, stage[slot], sizeof(double) * nb2, sizeof(double) * nb2,
                              (size_t)(Rn - R), cudaMemcpyDeviceToHost, cs);
      if (e != cudaSuccess) { fail(e, "copy B rows to host"); break; }
      if ((e = cudaEventRecord(copied[slot], cs)) != cudaSuccess) { fail(e, "record"); break; }
    }
    a_done = a_end;
  }
  // the caller's stream (and the scratch frees queued on it) wait for the last copy
  if (fin && cudaEventRecord(fin, cs) == cudaSuccess) cudaStreamWaitEvent(st, fin, 0);
  else cudaStreamSynchronize(cs);
  for (int i = 0; i < 2; ++i) {
    if (ready[i]) cudaEventDestroy(ready[i]);
    if (copied[i]) cudaEventDestroy(copied[i]);
  }
  if (fin) cudaEventDestroy(fin);
  cudaStreamDestroy(cs);
  return status;  // the last band ends at npair, so every row of B has been written
}

// ---- adaptive boxes (Section 6): partition blocks of the factored form -----------------------
// Rows of F_u regrouped by partition (partition s occupies rows [off[s], off[s+1]) of Fp) and the
// matching unique-pair indices (d_idx, same order).
struct AdaptiveRows {
  std::vector<int64_t> off;
  int64_t* d_idx = nullptr;
  double* Fp = nullptr;
};

lrtei_status adaptive_rows(lrtei_plan* pl, Scratch& sc, AdaptiveRows& ar, bool with_F, cudaStream_t st) {
  const int np = pl->npart;
  const int64_t npair = pl->t.npair, n3 = (int64_t)pl->n * pl->n * pl->n;
  std::vector<int64_t> idx;
  ar.off.assign(1, 0);
  for (int s = 0; s < np; ++s) {
    for (int64_t r = 0; r < npair; ++r)
      if (pl->h_pair_part[r] == s) idx.push_back(r);
    ar.off.push_back((int64_t)idx.size());
  }
  LRTEI_TRY(sc.get(&ar.d_idx, (size_t)npair));
  LRTEI_CUDA(cudaMemcpyAsync(ar.d_idx, idx.data(), sizeof(int64_t) * npair, cudaMemcpyHostToDevice, st));
  if (with_F) {
    LRTEI_TRY(ensure_F64(pl, st));
    LRTEI_TRY(sc.get(&ar.Fp, (size_t)npair * n3));
    launch_gather_rows(pl->d_F, ar.d_idx, npair, n3, ar.Fp, st);
  }
  // the host index list is read by the copy above before this function returns
  LRTEI_CUDA(cudaStreamSynchronize(st));
  return LRTEI_OK;
}

// B_u of an adaptive plan: B_{st} = F_s K_{st} F_t^T for s <= t, scattered (and mirrored) into Bu.
// K_{st} is applied as G = F_s K_{st} (rows of G = K_{ts} applied to rows of F_s): by three mode
// products per node with A_{ts} (FP64 / FP32 plans), or densely on the tensor cores.
lrtei_status bu_adaptive(lrtei_plan* pl, double* Bu, cudaStream_t st) {
  const int np = pl->npart, n = pl->n, P = pl->P;
  const int64_t npair = pl->t.npair, n3 = (int64_t)n * n * n;
  const size_t cblk = (size_t)3 * P * n * n;
  const double pref = pl->omega / sqrt(kPi);
  Scratch sc(st);
  AdaptiveRows ar;
  LRTEI_TRY(adaptive_rows(pl, sc, ar, true, st));
  int64_t maxr = 0;
  for (int s = 0; s < np; ++s) maxr = std::max(maxr, ar.off[s + 1] - ar.off[s]);
  double *G, *blk;
  LRTEI_TRY(sc.get(&G, (size_t)maxr * n3));
  LRTEI_TRY(sc.get(&blk, (size_t)maxr * maxr));
  if (is_split(pl)) {
    SplitMatrix Fsp, Ksp, Gsp;
    LRTEI_TRY(scratch_split(sc, Fsp, npair, n3, true, pl));
    LRTEI_TRY(scratch_split(sc, Ksp, n3, n3, true, pl));
    LRTEI_TRY(scratch_split(sc, Gsp, maxr, n3, false, pl));
    double* K;
    LRTEI_TRY(sc.get(&K, (size_t)n3 * n3));
    {
      ProfScope ps("split", st);
      launch_split_rows(ar.Fp, npair, n3, n3, Fsp, true, nslices(pl), st);
    }
    auto rows_of = [&](int s) {  // row view of partition s
      SplitMatrix v = Fsp;
      const int64_t r0 = ar.off[s];
      v.rows = ar.off[s + 1] - r0;
      v.s0 += r0 * v.kpad;
      if (v.s1) v.s1 += r0 * v.kpad;
      if (v.s2) v.s2 += r0 * v.kpad;
      if (v.s1h) v.s1h += r0 * v.kpad;
      v.expo += r0;
      return v;
    };
    for (int t = 0; t < np; ++t) {
      const int64_t nt = ar.off[t + 1] - ar.off[t];
      for (int s = 0; s <= t; ++s) {
        const int64_t ns = ar.off[s + 1] - ar.off[s];
        if (ns == 0 || nt == 0) continue;
        {  // K_{ts} = (w/sqrt(pi)) sum_p w_p (x)_d A^(p)_{ts,d}, so that G = F_s K_{ts}^T = F_s K_{st}
          ProfScope ps("build_K", st);
          LRTEI_CUDA(launch_build_K(n, P, pl->d_C + (size_t)(t * np + s) * cblk, pl->d_w, pref, K, st));
        }
        {
          ProfScope ps("split", st);
          launch_split_rows(K, n3, n3, n3, Ksp, true, nslices(pl), st);
        }
        SplitMatrix Fs = rows_of(s), Ft = rows_of(t);
        LRTEI_TRY(tc_gemm(Fs, Ksp, ns, n3, 1.0, G, n3, false, false, 1, nullptr, pl->d_status, st));
        Gsp.rows = ns;
        {
          ProfScope ps("split", st);
          launch_split_rows(G, ns, n3, n3, Gsp, false, nslices(pl), st);
        }
        LRTEI_TRY(tc_gemm(Gsp, Ft, ns, nt, 1.0, blk, nt, false, false, 1, nullptr, pl->d_status, st));
        launch_scatter_block(blk, nt, ar.d_idx + ar.off[s], ns, ar.d_idx + ar.off[t], nt, Bu, npair, s != t, st);
      }
    }
    return finish_launch("adaptive B (tensor cores)");
  }
  double *t1, *t2;
  LRTEI_TRY(sc.get(&t1, (size_t)maxr * n3));
  LRTEI_TRY(sc.get(&t2, (size_t)maxr * n3));
  for (int t = 0; t < np; ++t) {
    const int64_t nt = ar.off[t + 1] - ar.off[t];
    for (int s = 0; s <= t; ++s) {
      const int64_t ns = ar.off[s + 1] - ar.off[s];
      if (ns == 0 || nt == 0) continue;
      {  // rows of G = F_s K_{st}: K_{ts} applied to each row of F_s by mode products
        ProfScope ps("kron", st);
        launch_kron_apply(n, P, pl->d_C + (size_t)(t * np + s) * cblk, pl->d_w, ar.Fp + ar.off[s] * n3, G, ns, t1, t2,
                          st);
      }
      {
        ProfScope ps("gemm_fp64", st);
        gemm_cuda_core<double>(false, true, ns, nt, n3, pref, G, n3, ar.Fp + ar.off[t] * n3, n3, 0.0, blk, nt, st);
      }
      launch_scatter_block(blk, nt, ar.d_idx + ar.off[s], ns, ar.d_idx + ar.off[t], nt, Bu, npair, s != t, st);
    }
  }
  return finish_launch("adaptive B");
}

// J-build of an adaptive plan (FP64, every precision): X_t = F_t^T D_t per partition,
// Y_s = sum_t K_{st} X_t (mode products with A_{st}), J_s = F_s Y_s.
lrtei_status jbuild_adaptive(lrtei_plan* pl, const double* d_D, int R, double* d_J, cudaStream_t st) {
  const int np = pl->npart, n = pl->n, P = pl->P, nbf = pl->basis.nbf;
  const int64_t npair = pl->t.npair, n3 = (int64_t)n * n * n;
  const size_t cblk = (size_t)3 * P * n * n;
  const double pref = pl->omega / sqrt(kPi);
  Scratch sc(st);
  AdaptiveRows ar;
  LRTEI_TRY(adaptive_rows(pl, sc, ar, true, st));
  double *Du, *Dp, *X, *Yp, *Y, *t1, *t2, *Jp, *Ju;
  LRTEI_TRY(sc.get(&Du, (size_t)npair * R));
  LRTEI_TRY(sc.get(&Dp, (size_t)npair * R));
  LRTEI_TRY(sc.get(&X, (size_t)np * R * n3));
  LRTEI_TRY(sc.get(&Yp, (size_t)np * R * n3));
  LRTEI_TRY(sc.get(&Y, (size_t)R * n3));
  LRTEI_TRY(sc.get(&t1, (size_t)R * n3));
  LRTEI_TRY(sc.get(&t2, (size_t)R * n3));
  LRTEI_TRY(sc.get(&Jp, (size_t)npair * R));
  LRTEI_TRY(sc.get(&Ju, (size_t)npair * R));
  launch_pack_density(nbf, R, d_D, Du, st);
  launch_gather_rows(Du, ar.d_idx, npair, R, Dp, st);
  for (int t = 0; t < np; ++t) {  // X_t^T (R x n^3) = D_t^T F_t
    const int64_t nt = ar.off[t + 1] - ar.off[t];
    ProfScope ps("gemm_fp64", st);
    gemm_cuda_core<double>(true, false, R, n3, nt, 1.0, Dp + ar.off[t] * R, R, ar.Fp + ar.off[t] * n3, n3, 0.0,
                           X + (size_t)t * R * n3, n3, st);
  }
  for (int s = 0; s < np; ++s) {
    const int64_t ns = ar.off[s + 1] - ar.off[s];
    for (int t = 0; t < np; ++t) {  // K_{st} X_t, rows of X_t^T: A_{st} by mode products
      ProfScope ps("kron", st);
      launch_kron_apply(n, P, pl->d_C + (size_t)(s * np + t) * cblk, pl->d_w, X + (size_t)t * R * n3,
                        Yp + (size_t)t * R * n3, R, t1, t2, st);
    }
    launch_reduce_splits(Yp, np, (int64_t)R * n3, R, n3, n3, Y, n3, st);
    {
      ProfScope ps("gemm_fp64", st);
      gemm_cuda_core<double>(false, true, ns, R, n3, pref, ar.Fp + ar.off[s] * n3, n3, Y, n3, 0.0, Jp + ar.off[s] * R,
                             R, st);
    }
  }
  launch_scatter_rows(Jp, ar.d_idx, npair, R, Ju, st);
  launch_unpack_J(nbf, R, Ju, 1.0, d_J, pl->d_status, st);
  return finish_launch("adaptive J-build");
}

// The tensor-core Hadamard form covers six-product split plans whose unique pairs each hold one
// primitive pair (uncontracted bases), n <= 64, with the plain moments of one box.
bool hadamard_tc_ok(const lrtei_plan* pl) {
  return pl->prec == LRTEI_SPLIT_F16 && pl->t.nrows == pl->t.npair && pl->t.maxI == 1 && pl->n <= 64 &&
         pl->kr_rank == 0 && pl->npart == 0 && 3LL * pl->P * pl->t.nrows < (1LL << 31);
}

int choose_form(const lrtei_plan* pl, lrtei_form form) {
  // Per element of B_u: Hadamard ~ P Ibar^2 (6n + 3); factored ~ 2 n^3 (+ 6 P n^4 per row).
  const double Ibar2 = (double)pl->t.nrows / std::max<int64_t>(1, pl->t.npair);
  const double had = (double)pl->P * Ibar2 * Ibar2 * (6.0 * pl->n + 3.0);
  const double fac = (double)pl->n * pl->n * pl->n * 2.0;
  if (is_split(pl)) {  // tensor cores: the factored form, or the Hadamard form where it applies
    if (!hadamard_tc_ok(pl) || form == LRTEI_FORM_FACTORED) return LRTEI_FORM_FACTORED;
    return (form == LRTEI_FORM_HADAMARD || had <= fac) ? LRTEI_FORM_HADAMARD : LRTEI_FORM_FACTORED;
  }
  if (form == LRTEI_FORM_HADAMARD || form == LRTEI_FORM_FACTORED) return form;
  return had <= fac ? LRTEI_FORM_HADAMARD : LRTEI_FORM_FACTORED;
}

// Slices of T_{d,p} and S'_d and the node tables of the tensor-core Hadamard form (once per plan).
lrtei_status ensure_had(lrtei_plan* pl, cudaStream_t st) {
  if (pl->have_had) return LRTEI_OK;
  HadOperands& h = pl->had;
  h.nrows = pl->t.nrows;
  h.n = pl->n;
  h.P = pl->P;
  h.kpad = pl->n <= 32 ? 32 : 64;
  const size_t tcnt = 3ULL * h.P * h.nrows * h.kpad, scnt = 3ULL * h.nrows * h.kpad;
  LRTEI_TRY(pl->alloc(&h.t0, tcnt));
  LRTEI_TRY(pl->alloc(&h.t1, tcnt));
  LRTEI_TRY(pl->alloc(&h.t2, tcnt));
  LRTEI_TRY(pl->alloc(&h.s0, scnt));
  LRTEI_TRY(pl->alloc(&h.s1, scnt));
  LRTEI_TRY(pl->alloc(&h.s1h, scnt));
  LRTEI_TRY(pl->alloc(&h.s2, scnt));
  LRTEI_TRY(pl->alloc(&h.te, 3ULL * h.P * h.nrows));
  LRTEI_TRY(pl->alloc(&h.se, 3ULL * h.nrows));
  LRTEI_TRY(pl->alloc(&h.f, (size_t)h.nrows * h.P));
  LRTEI_TRY(pl->alloc(&h.ra, (size_t)h.nrows));
  LRTEI_TRY(pl->alloc(&h.eb, (size_t)h.nrows));
  Scratch sc(st);
  double *Ss, *T;
  LRTEI_TRY(sc.get(&Ss, 3ULL * h.nrows * h.n));
  LRTEI_TRY(sc.get(&T, 3ULL * h.P * h.nrows * h.n));
  {
    ProfScope ps("hadamard_prep", st);
    launch_had_prepare(h, pl->d_S, pl->d_C, pl->d_w, pl->omega / sqrt(kPi), pl->t.row_c, Ss, T, st);
  }
  pl->have_had = true;
  return finish_launch("tensor-core Hadamard operands");
}

// Rows [r0, r1) of B_u (full width npair) into out (ld), prefactor included.
lrtei_status bu_rows(lrtei_plan* pl, int form, int64_t r0, int64_t r1, double* out, int64_t ld, cudaStream_t st) {
  const double pref = pl->omega / sqrt(kPi);
  const int n = pl->n, P = pl->P;
  const int64_t npair = pl->t.npair, n3 = (int64_t)n * n * n, nr = r1 - r0;
  if (nr <= 0) return LRTEI_OK;
  if (is_split(pl)) {
    if (form == LRTEI_FORM_HADAMARD) {
      LRTEI_TRY(ensure_had(pl, st));
      LRTEI_TRY(had_tc_rows(pl->had, r0, r1, out, ld, pl->d_status, st));
      return finish_launch("tensor-core Hadamard form");
    }
    return bu_rows_tc(pl, r0, r1, out, ld, st);
  }
  if (form == LRTEI_FORM_HADAMARD) {
    LRTEI_TRY(ensure_T(pl, st));
    {
      ProfScope ps("hadamard", st);
      launch_hadamard_rows(pl->t, n, P, pl->d_S, pl->d_T, pl->d_w, pref, r0, r1, out, ld, st);
    }
    return finish_launch("hadamard_rows");
  }
  // factored: G = kron(F rows), B_u rows = pref * G F^T
  LRTEI_TRY(ensure_F64(pl, st));
  Scratch sc(st);
  double *G, *t1, *t2;
  LRTEI_TRY(sc.get(&G, (size_t)nr * n3));
  LRTEI_TRY(sc.get(&t1, (size_t)nr * n3));
  LRTEI_TRY(sc.get(&t2, (size_t)nr * n3));
  {
    ProfScope ps("kron", st);
    launch_kron_apply(n, P, pl->d_C, pl->d_w, pl->d_F + r0 * n3, G, nr, t1, t2, st);
  }
  if (pl->prec == LRTEI_FP32) {
    LRTEI_TRY(ensure_F32(pl, st));
    float *G32, *B32;
    LRTEI_TRY(sc.get(&G32, (size_t)nr * n3));
    LRTEI_TRY(sc.get(&B32, (size_t)nr * npair));
    convert_f64_to_f32(G, G32, nr * n3, st);
    {
      ProfScope ps("gemm_fp32", st);
      gemm_cuda_core<float>(false, true, nr, npair, n3, 1.0f, G32, n3, pl->d_F32, n3, 0.0f, B32, npair, st);
    }
    double* tmp;
    LRTEI_TRY(sc.get(&tmp, (size_t)nr * npair));
    convert_f32_to_f64(B32, tmp, nr * npair, st);
    scale_copy_rows(tmp, npair, out, ld, nr, npair, pref, st);
    return finish_launch("fp32 B rows");
  }
  {
    ProfScope ps("gemm_fp64", st);
    gemm_cuda_core<double>(false, true, nr, npair, n3, pref, G, n3, pl->d_F, n3, 0.0, out, ld, st);
  }
  return finish_launch("factored B rows");
}

}  // namespace

namespace {
// Captured batches: one CUDA graph per (plans, densities, outputs, R) set.  Molecules are spread
// over kSideStreams capture streams so that the kernels of small molecules run concurrently.
constexpr int kSideStreams = 4;
struct BatchGraph {
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;
  unsigned long long used = 0;  // last use (least recently used graphs are evicted)
};
std::mutex g_batch_mu;
std::map<std::vector<uintptr_t>, BatchGraph> g_batch;
unsigned long long g_batch_tick = 0;
constexpr size_t kMaxGraphs = 32;  // each graph keeps its scratch memory reserved

lrtei_status capture_batch(lrtei_plan* const* plans, int nmol, const double* const* d_D, const int* R,
                           double* const* d_J, cudaStream_t st, BatchGraph* out) {
  (void)st;  // the graph is captured on a stream of its own and launched later on the caller's
  cudaStream_t origin, side[kSideStreams];
  cudaEvent_t fork, join[kSideStreams];
  LRTEI_CUDA(cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking));
  for (int i = 0; i < kSideStreams; ++i) LRTEI_CUDA(cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking));
  LRTEI_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  for (int i = 0; i < kSideStreams; ++i) LRTEI_CUDA(cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming));
  const long long count0 = launch_count();
  lrtei_status status = LRTEI_OK;
  cudaGraph_t graph = nullptr;
  LRTEI_CUDA(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
  cudaEventRecord(fork, origin);
  for (int i = 0; i < kSideStreams; ++i) cudaStreamWaitEvent(side[i], fork, 0);
  for (int m = 0; m < nmol && status == LRTEI_OK; ++m)
    status = jbuild_direct(plans[m], d_D[m], R[m], d_J[m], side[m % kSideStreams]);
  for (int i = 0; i < kSideStreams; ++i) {
    cudaEventRecord(join[i], side[i]);
    cudaStreamWaitEvent(origin, join[i], 0);
  }
  cudaError_t e = cudaStreamEndCapture(origin, &graph);
  set_launch_count(count0);
  if (status == LRTEI_OK && e != cudaSuccess) status = cuda_fail(e, "batched J-build capture");
  if (status == LRTEI_OK) {
    e = cudaGraphInstantiate(&out->exec, graph, 0);
    if (e != cudaSuccess) status = cuda_fail(e, "batched J-build instantiate");
  }
  if (status == LRTEI_OK) {
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(graph, nodes.data(), &nn);
    for (auto nd : nodes) {
      cudaGraphNodeType ty;
      if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++out->kernels;
    }
  }
  if (graph) cudaGraphDestroy(graph);
  cudaEventDestroy(fork);
  for (int i = 0; i < kSideStreams; ++i) {
    cudaEventDestroy(join[i]);
    cudaStreamDestroy(side[i]);
  }
  cudaStreamDestroy(origin);
  cudaGetLastError();
  return status;
}

lrtei_status batched_graph_run(lrtei_plan* const* plans, int nmol, const double* const* d_D, const int* R,
                               double* const* d_J, cudaStream_t st) {
  // operands of every molecule exist before capture (their set-up allocates and synchronises)
  for (int m = 0; m < nmol; ++m) {
    if (is_split(plans[m])) LRTEI_TRY(ensure_jbuild_operands(plans[m], st));
    else LRTEI_TRY(ensure_F64(plans[m], st));
  }
  std::vector<uintptr_t> key;
  key.push_back((uintptr_t)nmol);
  for (int m = 0; m < nmol; ++m) {
    key.push_back((uintptr_t)plans[m]);
    key.push_back((uintptr_t)d_D[m]);
    key.push_back((uintptr_t)d_J[m]);
    key.push_back((uintptr_t)R[m]);
  }
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    auto it = g_batch.find(key);
    if (it != g_batch.end()) {
      it->second.used = ++g_batch_tick;
      ProfScope ps("batched", st);
      LRTEI_CUDA(cudaGraphLaunch(it->second.exec, st));
      count_launches(it->second.kernels);
      return LRTEI_OK;
    }
  }
  // First call for this set: run it directly (this also settles the GEMM tuning choices for
  // every shape), then capture the same work into a graph for the calls that follow.
  for (int m = 0; m < nmol; ++m) LRTEI_TRY(jbuild_direct(plans[m], d_D[m], R[m], d_J[m], st));
  BatchGraph g;
  LRTEI_TRY(capture_batch(plans, nmol, d_D, R, d_J, st, &g));
  std::lock_guard<std::mutex> lk(g_batch_mu);
  if (g_batch.size() >= kMaxGraphs) {
    auto old = g_batch.begin();
    for (auto it = g_batch.begin(); it != g_batch.end(); ++it)
      if (it->second.used < old->second.used) old = it;
    cudaGraphExecDestroy(old->second.exec);
    g_batch.erase(old);
  }
  g.used = ++g_batch_tick;
  g_batch[key] = g;
  return LRTEI_OK;
}
}  // namespace

// Captured batches that involve a plan are dropped when the plan is destroyed.
static void forget_plan_graphs(const lrtei_plan* pl) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (auto it = g_batch.begin(); it != g_batch.end();) {
    bool uses = false;
    for (size_t i = 1; i < it->first.size(); i += 4) uses |= (it->first[i] == (uintptr_t)pl);
    if (uses) {
      cudaGraphExecDestroy(it->second.exec);
      it = g_batch.erase(it);
    } else {
      ++it;
    }
  }
}

extern "C" {

lrtei_status lrtei_assemble_Bu_rows(lrtei_plan* plan, lrtei_form form, int64_t row_begin, int64_t row_end,
                                    double* d_Bu, int64_t ld, void* stream) {
  if (!plan || !d_Bu) { set_error("NULL argument"); return LRTEI_ERR_ARG; }
  if (row_begin < 0 || row_end > plan->t.npair || row_begin > row_end) {
    set_error("row range [%lld, %lld) outside [0, %lld)", (long long)row_begin, (long long)row_end,
              (long long)plan->t.npair);
    return LRTEI_ERR_ARG;
  }
  if (ld < plan->t.npair) { set_error("ld %lld < npair %lld", (long long)ld, (long long)plan->t.npair); return LRTEI_ERR_ARG; }
  if (plan->npart > 0) { set_error("row ranges of B_u are not available for adaptive-box plans"); return LRTEI_ERR_UNSUPPORTED; }
  const int f = choose_form(plan, form);
  plan->last_form = f;
  return bu_rows(plan, f, row_begin, row_end, d_Bu, ld, (cudaStream_t)stream);
}

lrtei_status lrtei_assemble_B(lrtei_plan* plan, lrtei_form form, double* d_B, int64_t ld, void* stream) {
  if (!plan || !d_B) { set_error("NULL argument"); return LRTEI_ERR_ARG; }
  const int nbf = plan->basis.nbf;
  const int64_t nb2 = (int64_t)nbf * nbf, npair = plan->t.npair;
  if (ld < nb2) { set_error("ld %lld < N_b^2 = %lld", (long long)ld, (long long)nb2); return LRTEI_ERR_ARG; }
  // The output may be device memory or page-locked host memory; in the latter case the
  // expansion kernel stores B through the buffer's device alias, so the device-to-host
  // transfer is the kernel's own write stream (no staging copy of B in device memory).
  double* hB = nullptr;
  {
    cudaPointerAttributes pa{};
    cudaError_t e = cudaPointerGetAttributes(&pa, d_B);
    if (e != cudaSuccess) return cuda_fail(e, "cudaPointerGetAttributes(B)");
    if (pa.type == cudaMemoryTypeHost) {
      // copy engines move B on the tensor-core factored path; the other paths' expansion stores
      // through the buffer's device alias
      if (!pa.devicePointer && !(is_split(plan) && choose_form(plan, form) == LRTEI_FORM_FACTORED)) {
        set_error("pinned host B is not mapped into the device address space");
        return LRTEI_ERR_ARG;
      }
      hB = d_B;
      d_B = static_cast<double*>(pa.devicePointer);
    } else if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) {
      set_error("B must be device memory or page-locked (pinned) host memory");
      return LRTEI_ERR_ARG;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int f = choose_form(plan, form);
  plan->last_form = f;
  if (plan->npart > 0) {  // adaptive boxes: partition blocks of the factored form
    plan->last_form = LRTEI_FORM_FACTORED;
    if (hB && d_B == nullptr) {
      set_error("adaptive plans write B through the device alias of pinned host memory (map it)");
      return LRTEI_ERR_ARG;
    }
    Scratch sc(st);
    double* Bu;
    LRTEI_TRY(sc.get(&Bu, (size_t)npair * npair));
    LRTEI_TRY(bu_adaptive(plan, Bu, st));
    {
      ProfScope ps("expand_B", st);
      launch_expand_B(plan->t, nbf, Bu, npair, 1.0, d_B, ld, plan->d_status, st);
    }
    return finish_launch("expand_B");
  }
  if (hB && is_split(plan) && f == LRTEI_FORM_FACTORED) return assemble_B_host_banded(plan, hB, ld, st);
  // process B_u in row blocks of at most ~1 GiB
  int64_t rb = std::max<int64_t>(1, (int64_t)((1ULL << 30) / (sizeof(double) * (size_t)npair)));
  if (f == LRTEI_FORM_FACTORED) {
    const int64_t n3 = (int64_t)plan->n * plan->n * plan->n;
    rb = std::max<int64_t>(1, std::min<int64_t>(rb, (int64_t)((1ULL << 30) / (sizeof(double) * 3 * (size_t)n3))));
  }
  rb = std::min(rb, npair);
  if (is_split(plan)) rb = npair;  // one symmetric tensor-core pass over the whole B_u
  Scratch sc(st);
  double* blk;
  LRTEI_TRY(sc.get(&blk, (size_t)rb * npair));
  for (int64_t r0 = 0; r0 < npair; r0 += rb) {
    const int64_t r1 = std::min(npair, r0 + rb);
    LRTEI_TRY(bu_rows(plan, f, r0, r1, blk, npair, st));
    PairTable sub = plan->t;
    sub.pair_mu += r0;
    sub.pair_nu += r0;
    sub.npair = r1 - r0;
    {
      ProfScope ps("expand_B", st);
      launch_expand_B(sub, nbf, blk, npair, 1.0, d_B, ld, plan->d_status, st);
    }
    LRTEI_TRY(finish_launch("expand_B"));
  }
  return LRTEI_OK;
}

lrtei_status lrtei_entries(lrtei_plan* plan, const int32_t* d_idx4, int64_t count, double* d_out, void* stream) {
  if (!plan) { set_error("plan is NULL"); return LRTEI_ERR_ARG; }
  if (count < 0 || (count > 0 && (!d_idx4 || !d_out))) { set_error("invalid entries arguments"); return LRTEI_ERR_ARG; }
  if (count == 0) return LRTEI_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->npart == 0) LRTEI_TRY(ensure_T(plan, st));
  Scratch sc(st);
  int64_t *r, *c;
  LRTEI_TRY(sc.get(&r, count));
  LRTEI_TRY(sc.get(&c, count));
  launch_idx4_to_pairs(plan->basis.nbf, d_idx4, count, r, c, plan->d_status, st);
  if (plan->npart > 0) {
    launch_adaptive_entries(plan->t, plan->n, plan->P, plan->npart, plan->d_pair_part, plan->d_S, plan->d_C,
                            plan->d_w, plan->omega / sqrt(kPi), r, c, count, d_out, plan->d_status, st);
    return finish_launch("entries (adaptive)");
  }
  launch_hadamard_pairs(plan->t, plan->n, plan->P, plan->d_S, plan->d_T, plan->d_w, plan->omega / sqrt(kPi), r, c,
                        count, d_out, plan->d_status, st);
  return finish_launch("entries");
}

lrtei_status lrtei_factors(lrtei_plan* plan, double* d_S, double* d_C, double* d_s, double* d_w, double* d_c,
                           void* stream) {
  if (!plan) { set_error("plan is NULL"); return LRTEI_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = plan->n, P = plan->P, nrows = plan->t.nrows;
  if (d_S) LRTEI_CUDA(cudaMemcpyAsync(d_S, plan->d_S, sizeof(double) * 3 * nrows * n, cudaMemcpyDeviceToDevice, st));
  const size_t nb2c = (size_t)std::max(1, plan->npart) * std::max(1, plan->npart);  // coefficient blocks
  if (d_C) LRTEI_CUDA(cudaMemcpyAsync(d_C, plan->d_C, sizeof(double) * nb2c * 3 * P * n * n, cudaMemcpyDeviceToDevice, st));
  if (d_s) LRTEI_CUDA(cudaMemcpyAsync(d_s, plan->d_s, sizeof(double) * P, cudaMemcpyDeviceToDevice, st));
  if (d_w) LRTEI_CUDA(cudaMemcpyAsync(d_w, plan->d_w, sizeof(double) * P, cudaMemcpyDeviceToDevice, st));
  if (d_c) LRTEI_CUDA(cudaMemcpyAsync(d_c, plan->t.row_c, sizeof(double) * nrows, cudaMemcpyDeviceToDevice, st));
  return LRTEI_OK;
}

lrtei_status lrtei_dense_K(lrtei_plan* plan, double* d_K, void* stream) {
  if (!plan || !d_K) { set_error("NULL argument"); return LRTEI_ERR_ARG; }
  if (plan->npart > 0) { set_error("adaptive-box plans have one K per partition pair"); return LRTEI_ERR_UNSUPPORTED; }
  {
    ProfScope ps("build_K", (cudaStream_t)stream);
    LRTEI_CUDA(launch_build_K(plan->n, plan->P, plan->d_C, plan->d_w, plan->omega / sqrt(kPi), d_K,
                              (cudaStream_t)stream));
  }
  return finish_launch("dense K");
}

// Long-range exchange (appendix, eq. exchange) through the factored form, in blocks of orbitals:
// X = Q_b MT^T (N_b n^3 columns per orbital), Y = X K, K^lr += 2 Yp Xp^T with the orbital index
// moved into the contraction (Xp[mu][(j, m)]).  Tensor-core precisions run the three products on
// tcgen05 (split operands); FP64 / FP32 plans run them on the CUDA cores in FP64, with K applied by
// mode products (eq. ig1).
lrtei_status lrtei_exchange(lrtei_plan* plan, const double* d_Q, int norb, double* d_K, void* stream) {
  if (!plan || !d_Q || !d_K) { set_error("NULL argument"); return LRTEI_ERR_ARG; }
  if (norb <= 0) { set_error("norb must be positive (got %d)", norb); return LRTEI_ERR_ARG; }
  if (plan->npart > 0) { set_error("the exchange of adaptive-box plans is not supported"); return LRTEI_ERR_UNSUPPORTED; }
  cudaStream_t st = (cudaStream_t)stream;
  const int nbf = plan->basis.nbf, n = plan->n, P = plan->P;
  const int64_t n3 = (int64_t)n * n * n, rowlen = (int64_t)nbf * n3;
  const double pref = plan->omega / sqrt(kPi);
  const bool tc = is_split(plan);
  ProfScope ps_all("exchange", st);
  LRTEI_TRY(ensure_F64(plan, st));
  // orbital block: the block's X (ob N_b x n^3, FP64) within ~1 GiB
  int ob = (int)std::max<int64_t>(1, std::min<int64_t>(norb, (int64_t)((1ULL << 30) / (sizeof(double) * rowlen))));
  if (env_count("LRTEI_EXCHANGE_BLOCK") > 0) ob = (int)std::min<int64_t>(norb, env_count("LRTEI_EXCHANGE_BLOCK"));
  const int nblk = (norb + ob - 1) / ob;
  Scratch sc(st);
  double *MT, *X, *Y, *Xp, *Yp, *Kb;
  LRTEI_TRY(sc.get(&MT, (size_t)rowlen * nbf));
  LRTEI_TRY(sc.get(&X, (size_t)ob * rowlen));
  LRTEI_TRY(sc.get(&Y, (size_t)ob * rowlen));
  LRTEI_TRY(sc.get(&Xp, (size_t)ob * rowlen));
  LRTEI_TRY(sc.get(&Yp, (size_t)ob * rowlen));
  LRTEI_TRY(sc.get(&Kb, (size_t)nblk * nbf * nbf));
  launch_gather_MT(nbf, n3, plan->d_F, n3, MT, st);
  if (tc) {
    LRTEI_TRY(ensure_Ksp(plan, st, true));  // K as the B operand of Y = X K^T (K symmetric)
    SplitMatrix Qsp, MTsp, Xsp, Ypsp, Xpsp;
    LRTEI_TRY(scratch_split(sc, Qsp, norb, nbf, false, plan));
    LRTEI_TRY(scratch_split(sc, MTsp, rowlen, nbf, true, plan));
    LRTEI_TRY(scratch_split(sc, Xsp, (int64_t)ob * nbf, n3, false, plan));
    LRTEI_TRY(scratch_split(sc, Ypsp, nbf, (int64_t)ob * n3, false, plan));
    LRTEI_TRY(scratch_split(sc, Xpsp, nbf, (int64_t)ob * n3, true, plan));
    // split-K partials of the last product: the largest split count of any block (a shorter last
    // block can take more splits than a full one)
    const int nlast = norb - (nblk - 1) * ob;
    const int sK = std::max(splits_for(nbf, (int64_t)ob * n3), splits_for(nbf, (int64_t)nlast * n3));
    double* part;
    LRTEI_TRY(sc.get(&part, (size_t)sK * nbf * nbf));
    {
      ProfScope ps("split", st);
      launch_split_rows(d_Q, norb, nbf, nbf, Qsp, false, nslices(plan), st);
      launch_split_rows(MT, rowlen, nbf, nbf, MTsp, true, nslices(plan), st);
    }
    for (int b = 0; b < nblk; ++b) {
      const int j0 = b * ob, nj = std::min(ob, norb - j0);
      SplitMatrix Qb = Qsp;  // rows [j0, j0 + nj)
      Qb.rows = nj;
      Qb.s0 += (int64_t)j0 * Qb.kpad;
      if (Qb.s1) Qb.s1 += (int64_t)j0 * Qb.kpad;
      if (Qb.s2) Qb.s2 += (int64_t)j0 * Qb.kpad;
      if (Qb.s1h) Qb.s1h += (int64_t)j0 * Qb.kpad;
      Qb.expo += j0;
      LRTEI_TRY(tc_gemm(Qb, MTsp, nj, rowlen, 1.0, X, rowlen, false, false, 1, nullptr, plan->d_status, st));
      SplitMatrix Xb = Xsp;
      Xb.rows = (int64_t)nj * nbf;
      {
        ProfScope ps("split", st);
        launch_split_rows(X, Xb.rows, n3, n3, Xb, false, nslices(plan), st);
      }
      LRTEI_TRY(tc_gemm(Xb, plan->Ksp, Xb.rows, n3, 1.0, Y, n3, false, false, 1, nullptr, plan->d_status, st));
      launch_perm_orbital_rows(nbf, n3, nj, X, Xp, st);
      launch_perm_orbital_rows(nbf, n3, nj, Y, Yp, st);
      SplitMatrix Ya = Ypsp, Xa = Xpsp;
      Ya.kpad = Xa.kpad = kpad256((int64_t)nj * n3);
      {
        ProfScope ps("split", st);
        launch_split_rows(Yp, nbf, (int64_t)nj * n3, (int64_t)nj * n3, Ya, false, nslices(plan), st);
        launch_split_rows(Xp, nbf, (int64_t)nj * n3, (int64_t)nj * n3, Xa, true, nslices(plan), st);
      }
      const int sb = splits_for(nbf, (int64_t)nj * n3);
      if (sb > sK) { set_error("exchange: split count %d beyond the partial buffer's %d", sb, sK); return LRTEI_ERR_CUDA; }
      LRTEI_TRY(tc_gemm(Ya, Xa, nbf, nbf, 2.0, Kb + (size_t)b * nbf * nbf, nbf, false, false, sb, part,
                        plan->d_status, st));
    }
  } else {
    double *t1, *t2;
    LRTEI_TRY(sc.get(&t1, (size_t)ob * rowlen));
    LRTEI_TRY(sc.get(&t2, (size_t)ob * rowlen));
    const int64_t kc = 32768;  // split-K chunk of the last product (an N_b x N_b output)
    const int64_t maxk = (int64_t)ob * n3, nchunk = (maxk + kc - 1) / kc;
    double* part;
    LRTEI_TRY(sc.get(&part, (size_t)nchunk * nbf * nbf));
    for (int b = 0; b < nblk; ++b) {
      const int j0 = b * ob, nj = std::min(ob, norb - j0);
      {
        ProfScope ps("gemm_fp64", st);
        gemm_cuda_core<double>(false, true, nj, rowlen, nbf, 1.0, d_Q + (size_t)j0 * nbf, nbf, MT, nbf, 0.0, X, rowlen, st);
      }
      {
        ProfScope ps("kron", st);
        launch_kron_apply(n, P, plan->d_C, plan->d_w, X, Y, (int64_t)nj * nbf, t1, t2, st);
      }
      launch_perm_orbital_rows(nbf, n3, nj, X, Xp, st);
      launch_perm_orbital_rows(nbf, n3, nj, Y, Yp, st);
      const int64_t K = (int64_t)nj * n3, nc = (K + kc - 1) / kc;
      for (int64_t q = 0; q < nc; ++q) {
        const int64_t k0 = q * kc, kk = std::min(kc, K - k0);
        ProfScope ps("gemm_fp64", st);
        gemm_cuda_core<double>(false, true, nbf, nbf, kk, 2.0 * pref, Yp + k0, K, Xp + k0, K, 0.0,
                               part + (size_t)q * nbf * nbf, nbf, st);
      }
      launch_reduce_splits(part, (int)nc, (int64_t)nbf * nbf, nbf, nbf, nbf, Kb + (size_t)b * nbf * nbf, nbf, st);
    }
  }
  launch_reduce_splits(Kb, nblk, (int64_t)nbf * nbf, nbf, nbf, nbf, d_K, nbf, st);
  return finish_launch("exchange");
}

// Khatri-Rao low-rank compression (Section 6, eq. SVD and eq. approxepsilon): S_d -> S_d V_d and
// A_d^(p) -> V_d^T A_d^(p) V_d with V_d the leading right singular vectors of S_d; every later call
// runs on the compressed factors (the plan's n becomes the rank R).
lrtei_status lrtei_plan_compress(lrtei_plan* plan, double eps, int max_rank, double* h_sigma, int* h_ranks,
                                 void* stream) {
  if (!plan) { set_error("plan is NULL"); return LRTEI_ERR_ARG; }
  if (!(eps >= 0.0 && eps < 1.0)) { set_error("eps must be in [0, 1) (got %g)", eps); return LRTEI_ERR_ARG; }
  if (max_rank < 0 || max_rank > plan->n) {
    set_error("max_rank must be in [0, n = %d] (got %d)", plan->n, max_rank);
    return LRTEI_ERR_ARG;
  }
  if (plan->kr_rank > 0) { set_error("the plan is already compressed (rank %d)", plan->kr_rank); return LRTEI_ERR_UNSUPPORTED; }
  if (plan->npart > 0) { set_error("compression of adaptive-box plans is not supported"); return LRTEI_ERR_UNSUPPORTED; }
  cudaStream_t st = (cudaStream_t)stream;
  const int n = plan->n, P = plan->P;
  const int64_t nrows = plan->t.nrows;
  if (nrows == 0) { set_error("the plan has no primitive-pair rows"); return LRTEI_ERR_ARG; }
  std::vector<double> lam(3 * (size_t)n);
  double *part, *G, *V1, *V, *dlam;
  {
    Scratch sc(st);
    LRTEI_TRY(sc.get(&part, (size_t)kr_gram_blocks(nrows) * 3 * n * n));
    LRTEI_TRY(sc.get(&G, 3 * (size_t)n * n));
    LRTEI_TRY(sc.get(&V1, 3 * (size_t)n * n));
    LRTEI_TRY(sc.get(&dlam, 3 * (size_t)n));
    double* Vk;
    LRTEI_TRY(plan->alloc(&Vk, 3 * (size_t)n * n));  // kept until the projection below has run
    V = Vk;
    {
      ProfScope ps("kr_svd", st);
      LRTEI_CUDA(launch_kr_svd(nrows, n, plan->d_S, part, G, V1, dlam, V, nullptr, st));
    }
    LRTEI_CUDA(cudaMemcpyAsync(lam.data(), dlam, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
    LRTEI_CUDA(cudaStreamSynchronize(st));
  }
  int R = 0, Rd[3];
  for (int d = 0; d < 3; ++d) {
    const double s0 = sqrt(std::max(lam[(size_t)d * n], 0.0));
    int r = n;
    if (eps > 0.0) {
      r = 0;
      while (r < n && sqrt(std::max(lam[(size_t)d * n + r], 0.0)) >= eps * s0 && s0 > 0.0) ++r;
      r = std::max(r, 1);
    }
    Rd[d] = r;
    R = std::max(R, r);
    if (h_sigma)
      for (int i = 0; i < n; ++i) h_sigma[(size_t)d * n + i] = sqrt(std::max(lam[(size_t)d * n + i], 0.0));
  }
  if (max_rank > 0) R = std::min(R, max_rank);
  if (h_ranks) for (int d = 0; d < 3; ++d) h_ranks[d] = Rd[d];
  double *Snew, *Cnew;
  LRTEI_TRY(plan->alloc(&Snew, 3 * (size_t)nrows * R));
  LRTEI_TRY(plan->alloc(&Cnew, 3 * (size_t)P * R * R));
  {
    ProfScope ps("kr_project", st);
    LRTEI_CUDA(launch_kr_project(nrows, n, P, R, plan->d_S, plan->d_C, V, Snew, Cnew, st));
  }
  LRTEI_CUDA(cudaStreamSynchronize(st));
  // the tables built from the uncompressed factors are stale now
  forget_plan_graphs(plan);
  const int64_t n3 = (int64_t)n * n * n;
  plan->release(plan->d_T, sizeof(double) * 3 * (size_t)P * nrows * n);
  plan->d_T = nullptr;
  plan->release(plan->d_F, sizeof(double) * (size_t)plan->t.npair * n3);
  plan->d_F = nullptr;
  plan->release(plan->d_F32, sizeof(float) * (size_t)plan->t.npair * n3);
  plan->d_F32 = nullptr;
  if (plan->have_Fsp) { release_split(plan, plan->Fsp); plan->have_Fsp = false; }
  if (plan->have_Ksp) { release_split(plan, plan->Ksp); plan->have_Ksp = false; }
  if (plan->have_FTsp) { release_split(plan, plan->FTsp); plan->have_FTsp = false; }
  plan->release(plan->d_S, sizeof(double) * 3 * (size_t)nrows * n);
  plan->release(plan->d_C, sizeof(double) * 3 * (size_t)P * n * n);
  plan->release(V, sizeof(double) * 3 * (size_t)n * n);
  plan->d_S = Snew;
  plan->d_C = Cnew;
  plan->n = R;
  plan->kr_rank = R;
  for (int d = 0; d < 3; ++d) plan->kr_ranks[d] = Rd[d];
  return finish_launch("Khatri-Rao compression");
}

static lrtei_status jbuild_tc(lrtei_plan* plan, const double* d_D, int R, double* d_J, cudaStream_t st) {
  const int nbf = plan->basis.nbf, n = plan->n;
  const int64_t npair = plan->t.npair, n3 = (int64_t)n * n * n;
  LRTEI_TRY(ensure_jbuild_operands(plan, st));  // K carries the prefactor omega / sqrt(pi)
  Scratch sc(st);
  double *Du, *DuT, *XT, *YT, *Ju, *part;
  LRTEI_TRY(sc.get(&Du, (size_t)npair * R));
  LRTEI_TRY(sc.get(&DuT, (size_t)npair * R));
  LRTEI_TRY(sc.get(&XT, (size_t)R * n3));
  LRTEI_TRY(sc.get(&YT, (size_t)R * n3));
  LRTEI_TRY(sc.get(&Ju, (size_t)npair * R));
  const int s1 = splits_for(n3, npair), s2 = splits_for(n3, n3), s3 = splits_for(npair, n3);
  const int smax = std::max(s1, std::max(s2, s3));
  LRTEI_TRY(sc.get(&part, (size_t)smax * std::max(n3, npair) * R));
  SplitMatrix Dsp, Xsp, Ysp;
  LRTEI_TRY(scratch_split(sc, Dsp, R, npair, true, plan));
  LRTEI_TRY(scratch_split(sc, Xsp, R, n3, true, plan));
  LRTEI_TRY(scratch_split(sc, Ysp, R, n3, true, plan));
  launch_pack_density(nbf, R, d_D, Du, st);
  launch_transpose(Du, npair, R, R, DuT, npair, st);
  {
    ProfScope ps("split", st);
    launch_split_rows(DuT, R, npair, npair, Dsp, true, nslices(plan), st);
  }
  // X^T = (F^T D_u)^T : R x n^3
  LRTEI_TRY(tc_gemm(plan->FTsp, Dsp, n3, R, 1.0, XT, n3, true, false, s1, part, plan->d_status, st));
  {
    ProfScope ps("split", st);
    launch_split_rows(XT, R, n3, n3, Xsp, true, nslices(plan), st);
  }
  // Y^T = (K X)^T : R x n^3  (K symmetric)
  LRTEI_TRY(tc_gemm(plan->Ksp, Xsp, n3, R, 1.0, YT, n3, true, false, s2, part, plan->d_status, st));
  {
    ProfScope ps("split", st);
    launch_split_rows(YT, R, n3, n3, Ysp, true, nslices(plan), st);
  }
  // J_u = F Y : npair x R
  LRTEI_TRY(tc_gemm(plan->Fsp, Ysp, npair, R, 1.0, Ju, R, false, false, s3, part, plan->d_status, st));
  launch_unpack_J(nbf, R, Ju, 1.0, d_J, plan->d_status, st);
  return finish_launch("jbuild (tensor cores)");
}

// J-builds for plans whose F_u (npair x n^3) or dense K (n^3 x n^3) would not fit in device
// memory: F_u is built in blocks of rb unique pairs, twice (once for X = F_u^T D_u, once for
// J_u = F_u Y), and the node sum Y = sum_p w_p (A_x^p (x) A_y^p (x) A_z^p) X runs as FP64 mode
// products (eq. ig1) instead of the dense K.  Split plans run both F_u contractions of each block
// on the tensor cores; the block partials of X are summed in FP64.
static lrtei_status jbuild_streamed(lrtei_plan* plan, const double* d_D, int R, double* d_J, int64_t rb,
                                    cudaStream_t st) {
  const int nbf = plan->basis.nbf, n = plan->n, P = plan->P;
  const int64_t npair = plan->t.npair, n3 = (int64_t)n * n * n;
  const double pref = plan->omega / sqrt(kPi);
  const bool tc = is_split(plan);
  rb = std::max<int64_t>(1, std::min(rb, npair));
  const int64_t nblk = (npair + rb - 1) / rb;
  Scratch sc(st);
  double *Du, *Xt, *Yt, *t1, *t2, *Ju, *Fb;
  LRTEI_TRY(sc.get(&Du, (size_t)npair * R));
  LRTEI_TRY(sc.get(&Xt, (size_t)R * n3));
  LRTEI_TRY(sc.get(&Yt, (size_t)R * n3));
  LRTEI_TRY(sc.get(&t1, (size_t)R * n3));
  LRTEI_TRY(sc.get(&t2, (size_t)R * n3));
  LRTEI_TRY(sc.get(&Ju, (size_t)npair * R));
  LRTEI_TRY(sc.get(&Fb, (size_t)rb * n3));
  launch_pack_density(nbf, R, d_D, Du, st);
  if (!tc) {
    for (int64_t r0 = 0; r0 < npair; r0 += rb) {  // X = sum over blocks of D_b^T F_b
      const int64_t nr = std::min(npair, r0 + rb) - r0;
      launch_build_F<double>(plan->t, n, plan->d_S, r0, r0 + nr, Fb, n3, st);
      ProfScope ps("gemm_fp64", st);
      gemm_cuda_core<double>(true, false, R, n3, nr, 1.0, Du + r0 * R, R, Fb, n3, r0 == 0 ? 0.0 : 1.0, Xt, n3, st);
    }
    {
      ProfScope ps("kron", st);
      launch_kron_apply(n, P, plan->d_C, plan->d_w, Xt, Yt, R, t1, t2, st);
    }
    for (int64_t r0 = 0; r0 < npair; r0 += rb) {  // J_b = F_b Y
      const int64_t nr = std::min(npair, r0 + rb) - r0;
      launch_build_F<double>(plan->t, n, plan->d_S, r0, r0 + nr, Fb, n3, st);
      ProfScope ps("gemm_fp64", st);
      gemm_cuda_core<double>(false, true, nr, R, n3, 1.0, Fb, n3, Yt, n3, 0.0, Ju + r0 * R, R, st);
    }
    launch_unpack_J(nbf, R, Ju, pref, d_J, plan->d_status, st);
    return finish_launch("jbuild (streamed)");
  }
  // tensor cores: X^T blocks (R x n^3) into per-block partials, summed once
  double *FbT, *DbT, *Xparts, *part;
  LRTEI_TRY(sc.get(&FbT, (size_t)rb * n3));
  LRTEI_TRY(sc.get(&DbT, (size_t)R * rb));
  LRTEI_TRY(sc.get(&Xparts, (size_t)nblk * R * n3));
  // split-K partials of the largest GEMM of any block (full blocks and the last, shorter one)
  const int64_t nlast = npair - (nblk - 1) * rb;
  const int64_t part_n = std::max({(int64_t)splits_for(n3, rb) * n3, (int64_t)splits_for(n3, nlast) * n3,
                                   (int64_t)splits_for(rb, n3) * rb, (int64_t)splits_for(nlast, n3) * nlast});
  LRTEI_TRY(sc.get(&part, (size_t)part_n * R));
  SplitMatrix FbTsp, Dbsp, Fbsp, Ysp;
  LRTEI_TRY(scratch_split(sc, FbTsp, n3, rb, false, plan));
  LRTEI_TRY(scratch_split(sc, Dbsp, R, rb, true, plan));
  LRTEI_TRY(scratch_split(sc, Fbsp, rb, n3, false, plan));
  LRTEI_TRY(scratch_split(sc, Ysp, R, n3, true, plan));
  for (int64_t b = 0; b < nblk; ++b) {
    const int64_t r0 = b * rb, nr = std::min(npair, r0 + rb) - r0;
    launch_build_F<double>(plan->t, n, plan->d_S, r0, r0 + nr, Fb, n3, st);
    launch_transpose(Fb, nr, n3, n3, FbT, nr, st);
    launch_transpose(Du + r0 * R, nr, R, R, DbT, nr, st);
    SplitMatrix A = FbTsp, Bm = Dbsp;  // K = nr for this block
    A.kpad = Bm.kpad = kpad256(nr);
    {
      ProfScope ps("split", st);
      launch_split_rows(FbT, n3, nr, nr, A, false, nslices(plan), st);
      launch_split_rows(DbT, R, nr, nr, Bm, true, nslices(plan), st);
    }
    const int sb = splits_for(n3, nr);
    LRTEI_TRY(tc_gemm(A, Bm, n3, R, 1.0, Xparts + b * R * n3, n3, true, false, sb, part, plan->d_status, st));
  }
  launch_reduce_splits(Xparts, (int)nblk, R * n3, R, n3, n3, Xt, n3, st);
  {
    ProfScope ps("kron", st);
    launch_kron_apply(n, P, plan->d_C, plan->d_w, Xt, Yt, R, t1, t2, st);
  }
  {
    ProfScope ps("split", st);
    launch_split_rows(Yt, R, n3, n3, Ysp, true, nslices(plan), st);
  }
  for (int64_t b = 0; b < nblk; ++b) {
    const int64_t r0 = b * rb, nr = std::min(npair, r0 + rb) - r0;
    launch_build_F<double>(plan->t, n, plan->d_S, r0, r0 + nr, Fb, n3, st);
    SplitMatrix A = Fbsp;
    A.rows = nr;
    {
      ProfScope ps("split", st);
      launch_split_rows(Fb, nr, n3, n3, A, false, nslices(plan), st);
    }
    LRTEI_TRY(tc_gemm(A, Ysp, nr, R, 1.0, Ju + r0 * R, R, false, false, splits_for(nr, n3), part, plan->d_status, st));
  }
  launch_unpack_J(nbf, R, Ju, pref, d_J, plan->d_status, st);
  return finish_launch("jbuild (streamed, tensor cores)");
}

// ---- a J-build split over ranks by unique pairs (the two halves of eq. coulapprox) -------------
// X^T (R x n^3) = sum over the pairs r in [r0, r1) of u_r F_u(r, :), u the packed densities; the
// ranks' X are summed (an all-reduce) and each rank then forms its rows of J_u = F_u Y from the
// node sum Y = K X.  F_u rows of the range are built here (FP64) and contracted on the tensor cores
// (split plans) or the CUDA cores.
static lrtei_status check_range(const lrtei_plan* plan, int64_t r0, int64_t r1) {
  if (r0 < 0 || r1 > plan->t.npair || r0 > r1) {
    set_error("pair range [%lld, %lld) outside [0, %lld)", (long long)r0, (long long)r1, (long long)plan->t.npair);
    return LRTEI_ERR_ARG;
  }
  if (plan->npart > 0) { set_error("pair ranges of adaptive-box plans are not supported"); return LRTEI_ERR_UNSUPPORTED; }
  return LRTEI_OK;
}

lrtei_status lrtei_jbuild_partial_x(lrtei_plan* plan, const double* d_D, int R, int64_t pair_begin, int64_t pair_end,
                                    double* d_X, void* stream) {
  if (!plan || !d_D || !d_X || R <= 0) { set_error("invalid partial J-build arguments"); return LRTEI_ERR_ARG; }
  LRTEI_TRY(check_range(plan, pair_begin, pair_end));
  cudaStream_t st = (cudaStream_t)stream;
  const int nbf = plan->basis.nbf, n = plan->n;
  const int64_t npair = plan->t.npair, n3 = (int64_t)n * n * n, nr = pair_end - pair_begin;
  if (nr == 0) {
    LRTEI_CUDA(cudaMemsetAsync(d_X, 0, sizeof(double) * (size_t)R * n3, st));
    return LRTEI_OK;
  }
  ProfScope ps_all("jbuild", st);
  Scratch sc(st);
  double *Du, *Fb;
  LRTEI_TRY(sc.get(&Du, (size_t)npair * R));
  LRTEI_TRY(sc.get(&Fb, (size_t)nr * n3));
  launch_pack_density(nbf, R, d_D, Du, st);
  launch_build_F<double>(plan->t, n, plan->d_S, pair_begin, pair_end, Fb, n3, st);
  if (!is_split(plan)) {
    ProfScope ps("gemm_fp64", st);
    gemm_cuda_core<double>(true, false, R, n3, nr, 1.0, Du + pair_begin * R, R, Fb, n3, 0.0, d_X, n3, st);
    return finish_launch("partial X");
  }
  double *FbT, *DbT, *part;
  LRTEI_TRY(sc.get(&FbT, (size_t)nr * n3));
  LRTEI_TRY(sc.get(&DbT, (size_t)R * nr));
  const int sb = splits_for(n3, nr);
  LRTEI_TRY(sc.get(&part, (size_t)sb * n3 * R));
  SplitMatrix A, Bm;
  LRTEI_TRY(scratch_split(sc, A, n3, nr, false, plan));
  LRTEI_TRY(scratch_split(sc, Bm, R, nr, true, plan));
  launch_transpose(Fb, nr, n3, n3, FbT, nr, st);
  launch_transpose(Du + pair_begin * R, nr, R, R, DbT, nr, st);
  {
    ProfScope ps("split", st);
    launch_split_rows(FbT, n3, nr, nr, A, false, nslices(plan), st);
    launch_split_rows(DbT, R, nr, nr, Bm, true, nslices(plan), st);
  }
  LRTEI_TRY(tc_gemm(A, Bm, n3, R, 1.0, d_X, n3, true, false, sb, part, plan->d_status, st));
  return finish_launch("partial X (tensor cores)");
}

lrtei_status lrtei_jbuild_apply_x(lrtei_plan* plan, const double* d_X, int R, int64_t pair_begin, int64_t pair_end,
                                  double* d_J, void* stream) {
  if (!plan || !d_X || !d_J || R <= 0) { set_error("invalid partial J-build arguments"); return LRTEI_ERR_ARG; }
  LRTEI_TRY(check_range(plan, pair_begin, pair_end));
  cudaStream_t st = (cudaStream_t)stream;
  const int nbf = plan->basis.nbf, n = plan->n, P = plan->P;
  const int64_t n3 = (int64_t)n * n * n, nr = pair_end - pair_begin;
  const double pref = plan->omega / sqrt(kPi);
  LRTEI_CUDA(cudaMemsetAsync(d_J, 0, sizeof(double) * (size_t)R * nbf * nbf, st));
  if (nr == 0) return LRTEI_OK;
  ProfScope ps_all("jbuild", st);
  Scratch sc(st);
  double *Y, *t1, *t2, *Fb, *Ju;
  LRTEI_TRY(sc.get(&Y, (size_t)R * n3));
  LRTEI_TRY(sc.get(&t1, (size_t)R * n3));
  LRTEI_TRY(sc.get(&t2, (size_t)R * n3));
  LRTEI_TRY(sc.get(&Fb, (size_t)nr * n3));
  LRTEI_TRY(sc.get(&Ju, (size_t)nr * R));
  {
    ProfScope ps("kron", st);
    launch_kron_apply(n, P, plan->d_C, plan->d_w, d_X, Y, R, t1, t2, st);
  }
  launch_build_F<double>(plan->t, n, plan->d_S, pair_begin, pair_end, Fb, n3, st);
  if (!is_split(plan)) {
    ProfScope ps("gemm_fp64", st);
    gemm_cuda_core<double>(false, true, nr, R, n3, 1.0, Fb, n3, Y, n3, 0.0, Ju, R, st);
  } else {
    double* part;
    const int s3 = splits_for(nr, n3);
    LRTEI_TRY(sc.get(&part, (size_t)s3 * nr * R));
    SplitMatrix A, Ysp;
    LRTEI_TRY(scratch_split(sc, A, nr, n3, false, plan));
    LRTEI_TRY(scratch_split(sc, Ysp, R, n3, true, plan));
    {
      ProfScope ps("split", st);
      launch_split_rows(Fb, nr, n3, n3, A, false, nslices(plan), st);
      launch_split_rows(Y, R, n3, n3, Ysp, true, nslices(plan), st);
    }
    LRTEI_TRY(tc_gemm(A, Ysp, nr, R, 1.0, Ju, R, false, false, s3, part, plan->d_status, st));
  }
  launch_unpack_J_range(plan->t, nbf, R, pair_begin, pair_end, Ju, pref, d_J, plan->d_status, st);
  return finish_launch("apply X");
}

// Streamed J-builds: forced by LRTEI_JBUILD_BLOCK=<pairs per block>, else chosen when the
// resident operands of the one-pass J-build would take more than half of the free device memory.
static int64_t jbuild_stream_block(const lrtei_plan* plan) {
  const char* env = getenv("LRTEI_JBUILD_BLOCK");
  if (env && *env) return std::max<int64_t>(1, atoll(env));
  // operands already resident: the one-pass J-build needs nothing more
  if (is_split(plan) ? (plan->have_FTsp && plan->have_Fsp && plan->have_Ksp) : plan->d_F != nullptr) return 0;
  const int64_t npair = plan->t.npair, n3 = (int64_t)plan->n * plan->n * plan->n;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const double f = (double)npair * n3, k = (double)n3 * n3;
  // split: F (FP64) + F^T (FP64, transient) + F^T and F slices + K (FP64) and its slices;
  // FP64: F.  Already-built operands are counted as if they had to be built.
  const double need = is_split(plan) ? f * (8 + 8 + 6 + 8) + k * (8 + 6) : f * 8;
  if (need <= 0.5 * (double)free_b) return 0;
  const double per_row = (double)n3 * (is_split(plan) ? 8 + 8 + 8 + 8 : 8);
  int64_t rb = (int64_t)(0.15 * (double)free_b / per_row);
  rb = std::max<int64_t>(128, rb / 128 * 128);
  return std::min(rb, npair);
}

}  // extern "C"

// One J-build launched kernel by kernel (also what a captured graph replays).
static lrtei_status jbuild_direct(lrtei_plan* plan, const double* d_D, int R, double* d_J, cudaStream_t st) {
  ProfScope ps_all("jbuild", st);
  if (plan->npart > 0) return jbuild_adaptive(plan, d_D, R, d_J, st);
  const int64_t rb = jbuild_stream_block(plan);
  if (rb > 0) return jbuild_streamed(plan, d_D, R, d_J, rb, st);
  if (is_split(plan)) return jbuild_tc(plan, d_D, R, d_J, st);
  const int nbf = plan->basis.nbf, n = plan->n, P = plan->P;
  const int64_t npair = plan->t.npair, n3 = (int64_t)n * n * n;
  const double pref = plan->omega / sqrt(kPi);
  Scratch sc(st);
  double *Du, *Xt, *Yt, *t1, *t2, *Ju;
  LRTEI_TRY(sc.get(&Du, (size_t)npair * R));
  LRTEI_TRY(sc.get(&Xt, (size_t)R * n3));
  LRTEI_TRY(sc.get(&Yt, (size_t)R * n3));
  LRTEI_TRY(sc.get(&t1, (size_t)R * n3));
  LRTEI_TRY(sc.get(&t2, (size_t)R * n3));
  LRTEI_TRY(sc.get(&Ju, (size_t)npair * R));
  launch_pack_density(nbf, R, d_D, Du, st);
  LRTEI_TRY(ensure_F64(plan, st));
  // Xt = Du^T F  (R x n^3); Yt = kron(Xt); Ju = F Yt^T (npair x R)
  {
    ProfScope ps("gemm_fp64", st);
    gemm_cuda_core<double>(true, false, R, n3, npair, 1.0, Du, R, plan->d_F, n3, 0.0, Xt, n3, st);
  }
  {
    ProfScope ps("kron", st);
    launch_kron_apply(n, P, plan->d_C, plan->d_w, Xt, Yt, R, t1, t2, st);
  }
  {
    ProfScope ps("gemm_fp64", st);
    gemm_cuda_core<double>(false, true, npair, R, n3, 1.0, plan->d_F, n3, Yt, n3, 0.0, Ju, R, st);
  }
  launch_unpack_J(nbf, R, Ju, pref, d_J, plan->d_status, st);
  return finish_launch("jbuild");
}

extern "C" {

// Repeated J-builds with the same plan, densities, output and R replay a CUDA graph of the
// kernel sequence (captured after the first such call has run directly); streamed J-builds, calls
// on a stream the caller is capturing, and LRTEI_JBUILD_GRAPH=0 launch kernel by kernel.
lrtei_status lrtei_jbuild(lrtei_plan* plan, const double* d_D, int R, double* d_J, void* stream) {
  if (!plan || !d_D || !d_J) { set_error("NULL argument"); return LRTEI_ERR_ARG; }
  if (R <= 0) { set_error("R must be positive (got %d)", R); return LRTEI_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->npart > 0) return jbuild_direct(plan, d_D, R, d_J, st);
  const char* g = getenv("LRTEI_JBUILD_GRAPH");
  const bool graphs = !(g && g[0] == '0');
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (!graphs || jbuild_stream_block(plan) > 0 || cudaStreamIsCapturing(st, &cap) != cudaSuccess ||
      cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return jbuild_direct(plan, d_D, R, d_J, st);
  }
  return batched_graph_run(&plan, 1, &d_D, &R, &d_J, st);
}

lrtei_status lrtei_jbuild_batched(lrtei_plan* const* plans, int nmol, const double* const* d_D, const int* R,
                                  double* const* d_J, void* stream) {
  if (!plans || nmol <= 0 || !d_D || !R || !d_J) { set_error("invalid batched arguments"); return LRTEI_ERR_ARG; }
  for (int m = 0; m < nmol; ++m) {
    if (!plans[m] || !d_D[m] || !d_J[m] || R[m] <= 0) {
      set_error("batched J-build: molecule %d has a NULL plan/pointer or R <= 0", m);
      return LRTEI_ERR_ARG;
    }
    if (plans[m]->npart > 0) {
      set_error("batched J-build: molecule %d has an adaptive-box plan (use lrtei_jbuild)", m);
      return LRTEI_ERR_UNSUPPORTED;
    }
    if (is_split(plans[m]) != is_split(plans[0])) {
      set_error("batched J-build: all plans must use tensor-core or all CUDA-core precision");
      return LRTEI_ERR_ARG;
    }
  }
  return batched_graph_run(plans, nmol, d_D, R, d_J, (cudaStream_t)stream);
}

}  // extern "C"

namespace lrtei {
lrtei_status plan_view(const lrtei_plan* plan, PlanView* v) {
  if (!plan || !v) {
    set_error("NULL argument");
    return LRTEI_ERR_ARG;
  }
  v->nbf = plan->basis.nbf;
  v->n = plan->n;
  v->P = plan->P;
  v->omega = plan->omega;
  v->t = &plan->t;
  v->S = plan->d_S;
  v->C = plan->d_C;
  v->w = plan->d_w;
  v->status = plan->d_status;
  v->half3 = plan->d_half3;
  v->kr_rank = plan->kr_rank;
  v->npart = plan->npart;
  return LRTEI_OK;
}
}  // namespace lrtei
