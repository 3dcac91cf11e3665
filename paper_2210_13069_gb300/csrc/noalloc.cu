// noalloc.cu -- lrtei_entries_noalloc: Algorithm 1 entries without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need integrals: code that
// runs while another component holds the whole device memory in its own pool, code on a path
// where the implicit device synchronisation of cudaMalloc/cudaFree would stall other streams, or
// code that must not fail half-way for lack of memory.  This entry point takes only the plan
// (built beforehand), the caller's index list and the caller's output buffer; its scratch (the
// unique-pair indices of the requested entries) is a fixed array in device memory that the
// library declares at file scope.
//
// Properties a caller has to know:
//  - At most kNoAllocMaxEntries entries per call (262144, i.e. 4 MiB of scratch); larger
//    requests are rejected with LRTEI_ERR_UNSUPPORTED before anything is launched.
//  - The scratch array exists once per device for as long as the library is loaded (every GPU
//    that loads the library holds its 4 MiB until the process exits).
//  - All calls on a device share that array, and a call leaves its contents behind.  Two calls
//    whose kernels overlap on the GPU (different streams without ordering) race on it.
//  - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
//    once, with that device current; make that first call before any stream capture begins.
//  - It reads only the plan's moments, Chebyshev coefficients and weights, which the plan
//    computes when it is created, so it never triggers the plan's lazily built tables.
//  - The array's address is cached per device for the life of the process.  A device reset
//    (cudaDeviceReset, or a primary context released and created again) reloads the module and
//    invalidates that address: calls after such a reset are not supported.
//  - Indices outside [0, N_b) are caught on the device: the entry comes out as NaN, nothing is
//    read for it, and lrtei_plan_status then returns LRTEI_ERR_ARG.
#include <mutex>

#include "lrtei_internal.h"

namespace lrtei {

constexpr int64_t kNoAllocMaxEntries = 1 << 18;

// [0, max): row pair of entry e; [max, 2 max): column pair.  Every slot a call reads is written
// by that same call first, so nothing has to be cleared between calls.
static __device__ __align__(256) int64_t g_noalloc_pairs[2 * kNoAllocMaxEntries];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
int64_t* g_addr[kMaxDevices] = {nullptr};

lrtei_status scratch_address(int64_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d beyond %d", dev, kMaxDevices);
    return LRTEI_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_pairs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_addr[dev] = static_cast<int64_t*>(p);
  }
  *out = g_addr[dev];
  return LRTEI_OK;
}

// An index outside [0, nbf) gives the pair -1 and latches kDevBadIndex.
__global__ void k_noalloc_pairs(int nbf, const int32_t* __restrict__ idx4, int64_t count, int64_t* __restrict__ rc,
                                int64_t maxe, int* status) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pr = checked_pair_index(nbf, idx4[4 * e], idx4[4 * e + 1]);
    const int64_t pc = checked_pair_index(nbf, idx4[4 * e + 2], idx4[4 * e + 3]);
    if (pr < 0 || pc < 0) latch_status(status, (int)kDevBadIndex);
    rc[e] = pr < 0 || pc < 0 ? -1 : pr;
    rc[maxe + e] = pr < 0 || pc < 0 ? -1 : pc;
  }
}

// Algorithm 1 per entry, straight from S and A^(p): (S_d(j) A S_d(j')^T) for every node,
// dimension and primitive pair; Neumaier-compensated sum over the nodes.
__global__ void k_noalloc_entries(int n, int P, int64_t nrows, const int64_t* __restrict__ pair_row,
                                  const double* __restrict__ row_c, const double* __restrict__ S,
                                  const double* __restrict__ C, const double* __restrict__ w, double pref,
                                  const int64_t* __restrict__ rc, int64_t maxe, int64_t count,
                                  double* __restrict__ out, int* status) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = rc[e], c = rc[maxe + e];
    if (r < 0 || c < 0) {  // an index outside the basis: nothing is read for this entry
      out[e] = __longlong_as_double(0x7FF8000000000000LL);
      continue;
    }
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
}  // namespace
}  // namespace lrtei

extern "C" lrtei_status lrtei_entries_noalloc(lrtei_plan* plan, const int32_t* d_idx4, int64_t count,
                                              double* d_out, void* stream) {
  using namespace lrtei;
  PlanView v;
  lrtei_status s = plan_view(plan, &v);
  if (s != LRTEI_OK) return s;
  if (count < 0 || (count > 0 && (!d_idx4 || !d_out))) {
    set_error("invalid entries arguments");
    return LRTEI_ERR_ARG;
  }
  if (v.npart > 0) {  // one coefficient block per partition pair: lrtei_entries handles these plans
    set_error("lrtei_entries_noalloc: adaptive-box plans are not supported");
    return LRTEI_ERR_UNSUPPORTED;
  }
  if (count > kNoAllocMaxEntries) {
    set_error("lrtei_entries_noalloc: %lld entries requested, at most %lld per call (fixed scratch of %lld bytes)",
              (long long)count, (long long)kNoAllocMaxEntries, (long long)(2 * kNoAllocMaxEntries * sizeof(int64_t)));
    return LRTEI_ERR_UNSUPPORTED;
  }
  if (count == 0) return LRTEI_OK;
  int64_t* rc = nullptr;
  s = scratch_address(&rc);
  if (s != LRTEI_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  int blocks = (int)((count + 127) / 128);
  if (blocks > 152 * 32) blocks = 152 * 32;
  count_launch();
  k_noalloc_pairs<<<blocks, 128, 0, st>>>(v.nbf, d_idx4, count, rc, kNoAllocMaxEntries, v.status);
  count_launch();
  k_noalloc_entries<<<blocks, 128, 0, st>>>(v.n, v.P, v.t->nrows, v.t->pair_row, v.t->row_c, v.S, v.C, v.w,
                                            v.omega / sqrt(3.14159265358979323846), rc, kNoAllocMaxEntries, count,
                                            d_out, v.status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "lrtei_entries_noalloc launch");
  return LRTEI_OK;
}
