// k_exchange.cu -- data movement of the long-range exchange (appendix "The Hartree-Fock exchange",
// eq. exchange) through the factored form:
//   K^lr(mu, nu) = 2 sum_j sum_{la, ka} q_{j la} q_{j ka} B(mu la, ka nu)
//                = 2 sum_j X_j K X_j^T,   X_j(mu, m) = sum_la q_{j la} M(mu la, m),
// with M the Khatri-Rao factor of eq. tensors (symmetric in its pair, so the ka-side factor is
// X_j(nu, :) again) and K the node sum of the factored form (omega / sqrt(pi) included).
// The contractions run as GEMMs (lrtei_api.cu); these kernels lay out their operands:
//   MT[(mu, m)][la] = M(mu la, m) = F_u(pair(mu, la), m)       (X = Q MT^T: one GEMM, K = N_b)
//   Zp[mu][(j, m)] = Z[(j, mu)][m]                              (K^lr = 2 Yp Xp^T: K = N_orb n^3)
#include "lrtei_internal.h"

namespace lrtei {

__device__ __forceinline__ int64_t ex_pair(int nbf, int a, int b) {
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  return (int64_t)lo * nbf - (int64_t)lo * (lo - 1) / 2 + (hi - lo);
}

// 32 x 32 tiles of (m, la) for one mu: rows of F_u read along m, MT written along la.
__global__ void k_gather_MT(int nbf, int64_t n3, const double* __restrict__ F, int64_t ldF, double* __restrict__ MT) {
  __shared__ double t[32][33];
  const int mu = blockIdx.z;
  const int64_t m0 = (int64_t)blockIdx.x * 32;
  const int la0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {  // r: la offset, threadIdx.x: m offset
    const int la = la0 + r;
    const int64_t m = m0 + threadIdx.x;
    t[r][threadIdx.x] = (la < nbf && m < n3) ? F[ex_pair(nbf, mu, la) * ldF + m] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {  // r: m offset, threadIdx.x: la offset
    const int64_t m = m0 + r;
    const int la = la0 + threadIdx.x;
    if (la < nbf && m < n3) MT[((int64_t)mu * n3 + m) * nbf + la] = t[threadIdx.x][r];
  }
}

void launch_gather_MT(int nbf, int64_t n3, const double* d_F, int64_t ldF, double* d_MT, cudaStream_t st) {
  dim3 grid((unsigned)((n3 + 31) / 32), (unsigned)((nbf + 31) / 32), (unsigned)nbf), block(32, 8);
  count_launch();
  k_gather_MT<<<grid, block, 0, st>>>(nbf, n3, d_F, ldF, d_MT);
}

// Zp[mu][j n3 + m] = Z[(j nbf + mu) n3 + m]; one block per (j, mu) row.
__global__ void k_perm_orbital_rows(int nbf, int64_t n3, int nj, const double* __restrict__ Z, double* __restrict__ Zp) {
  const int64_t row = blockIdx.x;  // j nbf + mu
  const int j = (int)(row / nbf), mu = (int)(row % nbf);
  const double* src = Z + row * n3;
  double* dst = Zp + (int64_t)mu * nj * n3 + (int64_t)j * n3;
  for (int64_t m = threadIdx.x; m < n3; m += blockDim.x) dst[m] = src[m];
}

void launch_perm_orbital_rows(int nbf, int64_t n3, int nj, const double* d_Z, double* d_Zp, cudaStream_t st) {
  count_launch();
  k_perm_orbital_rows<<<(unsigned)((int64_t)nj * nbf), 256, 0, st>>>(nbf, n3, nj, d_Z, d_Zp);
}

}  // namespace lrtei
