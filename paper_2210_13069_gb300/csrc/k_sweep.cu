// k_sweep.cu -- error sweeps of the plain method: Algorithm 1 entries of one plan's basis, box and
// omega at several other orders (n_c, P_c), the training data of the (n, P) selector.
//
// The moment integrals S_d(j, m) of eq. defV do not depend on n (only on the box and on m), so
// the plan's moments serve every n_c <= n through their first n_c columns.  The Gauss-Legendre
// nodes of eq. TEI2 and the Chebyshev coefficients of Definition 1 are computed for each
// (n_c, P_c) by the plan set-up kernels.  One block per (entry, order): thread p forms
// w_p sum_{j, j'} c_j c_j' prod_d (S_d(j) A_d^(p) S_d(j')^T), and the node sum is
// Neumaier-compensated in node order, as in the entries kernels.
#include <algorithm>
#include <vector>

#include "lrtei_internal.h"

namespace lrtei {

// Ct holds each order's coefficients node-fastest, Ct[off + ((d n_c + a) n_c + b) P_c + p], so that
// the threads of a warp (consecutive nodes p) read consecutive words.  For every dimension and
// column primitive pair k a thread forms t = A_d^(p) S_d(k)^T once and reuses it for every row
// primitive pair j (products over d accumulated per (j, k) when the pair block is small).
constexpr int kOrdersMaxJK = 64;

__global__ void __launch_bounds__(128) k_entries_orders(int n, int64_t nrows, const int64_t* __restrict__ pair_row,
                                                        const double* __restrict__ row_c, const double* __restrict__ S,
                                                        const int* __restrict__ cn, const int* __restrict__ cP,
                                                        const int64_t* __restrict__ coff, const double* __restrict__ Ct,
                                                        const double* __restrict__ wall, double pref,
                                                        const int64_t* __restrict__ rr, const int64_t* __restrict__ cc,
                                                        int64_t count, double* __restrict__ out, int* status) {
  __shared__ double term[kMaxP];
  const int64_t e = blockIdx.x;
  const int combo = blockIdx.y;
  const int nc = cn[combo], Pc = cP[combo];
  const int64_t r = rr[e], c = cc[e];
  if (r < 0 || c < 0) {  // an index outside the basis (latched by the index kernel)
    if (threadIdx.x == 0) out[(size_t)combo * count + e] = __longlong_as_double(0x7FF8000000000000LL);
    return;  // uniform across the block
  }
  const double* C = Ct + coff[combo];  // [3][nc][nc][Pc]
  const double* w = wall + (size_t)combo * kMaxP;
  const int64_t j0 = pair_row[r], j1 = pair_row[r + 1], k0 = pair_row[c], k1 = pair_row[c + 1];
  const int Ir = (int)(j1 - j0), Ic = (int)(k1 - k0);
  for (int p = threadIdx.x; p < Pc; p += blockDim.x) {
    double acc = 0.0;
    if (Ir * Ic <= kOrdersMaxJK) {
      double prod[kOrdersMaxJK];
      for (int jk = 0; jk < Ir * Ic; ++jk) prod[jk] = row_c[j0 + jk / Ic] * row_c[k0 + jk % Ic];
      for (int d = 0; d < 3; ++d) {
        const double* A = C + (size_t)d * nc * nc * Pc + p;
        for (int k = 0; k < Ic; ++k) {
          const double* sk = S + ((size_t)d * nrows + k0 + k) * n;
          double t[kMaxN];
          for (int a = 0; a < nc; ++a) {
            double x = 0.0;
            for (int b = 0; b < nc; ++b) x += A[((size_t)a * nc + b) * Pc] * sk[b];
            t[a] = x;
          }
          for (int j = 0; j < Ir; ++j) {
            const double* sj = S + ((size_t)d * nrows + j0 + j) * n;
            double g = 0.0;
            for (int a = 0; a < nc; ++a) g += sj[a] * t[a];
            prod[j * Ic + k] *= g;
          }
        }
      }
      for (int jk = 0; jk < Ir * Ic; ++jk) acc += prod[jk];
    } else {  // large pair blocks: one triple product per (j, k, d)
      for (int64_t j = j0; j < j1; ++j)
        for (int64_t k = k0; k < k1; ++k) {
          double prod = row_c[j] * row_c[k];
          for (int d = 0; d < 3; ++d) {
            const double* sj = S + ((size_t)d * nrows + j) * n;
            const double* sk = S + ((size_t)d * nrows + k) * n;
            const double* A = C + (size_t)d * nc * nc * Pc + p;
            double g = 0.0;
            for (int a = 0; a < nc; ++a) {
              double x = 0.0;
              for (int b = 0; b < nc; ++b) x += A[((size_t)a * nc + b) * Pc] * sk[b];
              g += sj[a] * x;
            }
            prod *= g;
          }
          acc += prod;
        }
    }
    term[p] = w[p] * acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0, comp = 0.0;
    for (int p = 0; p < Pc; ++p) {
      const double t = term[p], tsum = s + t;
      comp += (fabs(s) >= fabs(t)) ? (s - tsum) + t : (t - tsum) + s;
      s = tsum;
    }
    const double v = pref * (s + comp);
    out[(size_t)combo * count + e] = v;
    if (!isfinite(v)) latch_status(status, (int)kDevNonFinite);
  }
}

}  // namespace lrtei

extern "C" lrtei_status lrtei_entries_orders(lrtei_plan* plan, int ncombo, const int* h_n, const int* h_P,
                                             const int32_t* d_idx4, int64_t count, double* d_out, void* stream) {
  using namespace lrtei;
  PlanView v;
  lrtei_status s = plan_view(plan, &v);
  if (s != LRTEI_OK) return s;
  if (v.npart > 0) {
    set_error("lrtei_entries_orders: adaptive-box plans are not supported");
    return LRTEI_ERR_UNSUPPORTED;
  }
  if (v.kr_rank > 0) {
    set_error("lrtei_entries_orders: the plan's moments are compressed; sweeps need the uncompressed ones");
    return LRTEI_ERR_UNSUPPORTED;
  }
  if (ncombo <= 0 || !h_n || !h_P || count < 0 || (count > 0 && (!d_idx4 || !d_out))) {
    set_error("invalid entries_orders arguments");
    return LRTEI_ERR_ARG;
  }
  for (int i = 0; i < ncombo; ++i)
    if (h_n[i] < 1 || h_n[i] > v.n || h_P[i] < 1 || h_P[i] > kMaxP) {
      set_error("order %d: n = %d must be in 1..%d (the plan's n), P = %d in 1..%d", i, h_n[i], v.n, h_P[i], kMaxP);
      return LRTEI_ERR_ARG;
    }
  if (count == 0) return LRTEI_OK;
  if (count > 2147483647LL) { set_error("too many entries"); return LRTEI_ERR_UNSUPPORTED; }
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int64_t> off(ncombo);
  int64_t tot = 0;
  for (int i = 0; i < ncombo; ++i) {
    off[i] = tot;
    tot += 3LL * h_P[i] * h_n[i] * h_n[i];
  }
  // scratch (stream-ordered, freed when the call returns its work to the stream)
  std::vector<void*> mem;
  auto get = [&](void** p, size_t bytes) {
    cudaError_t e = scratch_alloc(p, std::max<size_t>(bytes, 16), st);
    if (e == cudaSuccess) mem.push_back(*p);
    return e;
  };
  auto done = [&](lrtei_status rs) {
    for (void* q : mem) cudaFreeAsync(q, st);
    return rs;
  };
  double *z, *w, *sn, *Call, *Ct;
  int *dn, *dP;
  int64_t *doff, *rr, *cc;
  cudaError_t e;
  if ((e = get((void**)&z, sizeof(double) * (size_t)ncombo * kMaxP)) != cudaSuccess ||
      (e = get((void**)&w, sizeof(double) * (size_t)ncombo * kMaxP)) != cudaSuccess ||
      (e = get((void**)&sn, sizeof(double) * kMaxP)) != cudaSuccess ||
      (e = get((void**)&Call, sizeof(double) * (size_t)tot)) != cudaSuccess ||
      (e = get((void**)&Ct, sizeof(double) * (size_t)tot)) != cudaSuccess ||
      (e = get((void**)&dn, sizeof(int) * ncombo)) != cudaSuccess ||
      (e = get((void**)&dP, sizeof(int) * ncombo)) != cudaSuccess ||
      (e = get((void**)&doff, sizeof(int64_t) * ncombo)) != cudaSuccess ||
      (e = get((void**)&rr, sizeof(int64_t) * count)) != cudaSuccess ||
      (e = get((void**)&cc, sizeof(int64_t) * count)) != cudaSuccess) {
    cudaGetLastError();
    set_error("entries_orders scratch allocation failed: %s", cudaGetErrorString(e));
    return done(LRTEI_ERR_ALLOC);
  }
  if ((e = cudaMemcpyAsync(dn, h_n, sizeof(int) * ncombo, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dP, h_P, sizeof(int) * ncombo, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(doff, off.data(), sizeof(int64_t) * ncombo, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return done(cuda_fail(e, "entries_orders upload"));
  std::vector<int> first(kMaxP + 1, -1);  // first order with each P: its rule serves the others
  for (int i = 0; i < ncombo; ++i) {  // nodes, weights and Chebyshev coefficients of each order
    double* zi = z + (size_t)i * kMaxP;
    double* wi = w + (size_t)i * kMaxP;
    const int f = first[h_P[i]];
    if (f < 0) {
      first[h_P[i]] = i;
      launch_gauss_legendre(h_P[i], zi, wi, st);
    } else {
      zi = z + (size_t)f * kMaxP;
      if ((e = cudaMemcpyAsync(wi, w + (size_t)f * kMaxP, sizeof(double) * h_P[i], cudaMemcpyDeviceToDevice, st)) !=
          cudaSuccess)
        return done(cuda_fail(e, "entries_orders weights"));
    }
    launch_nodes_map(h_P[i], v.omega, zi, sn, st);
    launch_cheb_coeff(h_n[i], h_P[i], sn, v.half3, Call + off[i], st);
    const int64_t nn = (int64_t)h_n[i] * h_n[i];
    for (int d = 0; d < 3; ++d)  // [p][a b] -> [a b][p] for each dimension
      launch_transpose(Call + off[i] + (size_t)d * h_P[i] * nn, h_P[i], nn, nn, Ct + off[i] + (size_t)d * h_P[i] * nn,
                       h_P[i], st);
  }
  launch_idx4_to_pairs(v.nbf, d_idx4, count, rr, cc, v.status, st);
  count_launch();
  k_entries_orders<<<dim3((unsigned)count, (unsigned)ncombo), 128, 0, st>>>(
      v.n, v.t->nrows, v.t->pair_row, v.t->row_c, v.S, dn, dP, doff, Ct, w, v.omega / sqrt(3.14159265358979323846),
      rr, cc, count, d_out, v.status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return done(cuda_fail(e, "entries_orders launch"));
  return done(LRTEI_OK);
}
