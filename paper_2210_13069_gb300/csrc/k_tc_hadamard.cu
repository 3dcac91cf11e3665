// k_tc_hadamard.cu -- the Hadamard form of Theorem 1 / Algorithm 1 on the tensor cores, for bases
// whose unique pairs each hold one primitive pair (uncontracted bases):
//   B_u(r, c) = (w/sqrt(pi)) sum_p w_p c_r c_c prod_d G_{d,p}(r, c),
//   G_{d,p} = T_{d,p} S_d^T,  T_{d,p} = S_d A_d^(p)  (moments of eq. defV, coefficients of
//   Definition 1, nodes and weights of eq. TEI2).
// Each G_{d,p} tile is a product of depth K = n (padded to 32 or 64) in the split-precision
// format of the GEMM (k_tcgen05.cu): three FP16 integer slices of T_{d,p}, four of S_d, six MMAs per
// 16-deep step into two FP32 TMEM accumulators, L0 (exact) and L12 (the lower-order products).
// The epilogue warps form g_d = L0 + L12 / 2^12 per dimension as a pair of FP32 numbers, the
// product over d and the weighted sum over the nodes in FP32 pairs (Dekker-style products with
// fmaf, Knuth's two-sum), and store each tile of B_u once in FP64, with its mirror.
//
// Scales: row r of T_{d,p} carries 2^ea_{d,p}(r), row c of S_d 2^eb_d(c) (one exponent per slice
// row), so G_{d,p}(r, c) = 2^(ea_{d,p}(r) + eb_d(c) - 16) g_d.  With Ea_p(r) = sum_d ea_{d,p}(r),
// Ra(r) = max_p Ea_p(r) and Eb(c) = sum_d eb_d(c):
//   B_u(r, c) = 2^(Ra(r) + Eb(c) - 48) sum_p f_p(r) prod_d g_d,   f_p(r) = (w/sqrt(pi)) w_p 2^(Ea_p(r) - Ra(r)),
// f_p(r) an FP32 pair per (row, node); the contraction coefficients c_r c_c ride in S_x's rows.
//
// Kernel organisation (persistent, one CTA per SM, 18 warps; tiles of 128 rows x 64 columns of B_u,
// the upper triangle with mirrors, or every column of a band of rows):
//   warp 0      TMA producer: the tile's S_d column rows (4 planes x 3 dimensions, resident for
//               the tile), then T_{d,p} row slices for every (p, d) through a ring of stages
//   warp 1      TMEM allocation (512 columns: four accumulator buffers of L0 and L12) and the
//               MMA-issuing thread: 2 x 6 MMAs (M = 128, N = 64, K = 16) per (p, d) and 32-deep step
//   warps 2-17  epilogue: per (p, d) tcgen05.ld of the finished buffer, product over d, node sum;
//               FP64 stores of the tile and its mirror at the end
// Every mbarrier wait is bounded, as in the GEMM: on expiry the CTA raises the device status word,
// stops issuing work, waits (bounded) for what it issued, frees TMEM and exits.
#include <stdlib.h>

#include <algorithm>

#include "lrtei_internal.h"
#include "tc_common.h"

namespace lrtei {
namespace tch {

using namespace tc;

constexpr int BM = 128;          // rows of B_u per tile (MMA M)
constexpr int BN = 64;           // columns of B_u per tile (MMA N)
constexpr int BK = 32;           // K per TMA step (64-byte rows, 64-byte swizzle)
constexpr int NBUF = 4;          // TMEM accumulator buffers (L0 and L12, 64 columns each)
constexpr int EPI = 16;          // epilogue warps, four per TMEM lane quadrant
constexpr int THREADS = 64 + 32 * EPI;
constexpr int QC = BN / (EPI / 4);  // columns per epilogue thread (16)
constexpr uint32_t A_PLANE = BM * BK * 2;            // one T slice plane of a 32-deep step
constexpr uint32_t A_STAGE = 3 * A_PLANE;            // 24 KB
constexpr uint32_t B_PLANE = BN * BK * 2;            // one S slice plane of a 32-deep step
constexpr int kZeroRowExpo = -30000;  // exponent of an all-zero slice row: its products vanish

template <int KS>
struct Cfg {
  static constexpr int STAGES = 4;
  static constexpr uint32_t B_BYTES = 3u * KS * 4u * B_PLANE;  // 48 KB (KS = 1) or 96 KB (KS = 2)
  static constexpr uint32_t RING = STAGES * A_STAGE;
  static constexpr size_t SMEM = (size_t)RING + B_BYTES + 1024 + 256;
};

struct Params {
  int64_t nrows;      // rows of B_u (unique pairs, one primitive pair each)
  int P;
  int64_t r0, r1;     // rows of B_u this launch computes
  int symmetric;      // upper-triangle walk with mirrors (r0 = 0, r1 = nrows)
  int64_t tm0;        // first 128-row block
  int64_t tiles_m;    // 128-row blocks walked
  int64_t tiles_n;    // 64-column blocks of B_u
  int64_t ntiles;
  const float2* f;    // [nrows][P]
  const int* ra;      // [nrows]
  const int* eb;      // [nrows]
  double* out;
  int64_t ld;
  int* status;
  long long test_stall;  // > 0 (tests only): the MMA thread first waits this many cycles on a barrier
                         // that nothing completes, so that the bounded-wait failure path runs
};

// Item -> (row block, column block).  Symmetric: row block I walks column blocks J >= 2 I (the
// blocks that meet the upper triangle), row by row, so that the CTAs running at once share one
// row block's T slices in L2.  Band: every column block of each row block.
__device__ __forceinline__ void tile_of(const Params& p, int64_t item, int64_t& I, int64_t& J) {
  if (p.symmetric) {
    int64_t t = item;
    for (I = 0; I < p.tiles_m; ++I) {
      const int64_t here = p.tiles_n - 2 * I;
      if (t < here) break;
      t -= here;
    }
    J = 2 * I + t;
  } else {
    I = p.tm0 + item / p.tiles_n;
    J = item % p.tiles_n;
  }
}

// (ah + al)(bh + bl) as an unevaluated FP32 pair; every partial product kept (|al|, |bl| may be
// 2^-9 of |ah|, |bh| here), the leading one split exactly with fmaf.
__device__ __forceinline__ void pmul(float ah, float al, float bh, float bl, float& ph, float& pl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  e = fmaf(al, bl, e);
  ph = p;
  pl = e;
}

// (ah, al) += (bh, bl): two-sum of the leading parts, the rest summed into the trailing part.
__device__ __forceinline__ void padd(float& ah, float& al, float bh, float bl) {
  const float s = ah + bh;
  const float v = s - ah;
  const float err = (ah - (s - v)) + (bh - v);
  ah = s;
  al = al + (bl + err);
}

// ------------------------------------------------------------------ the kernel
template <int KS>
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_hadamard(const __grid_constant__ CUtensorMap ta0, const __grid_constant__ CUtensorMap ta1,
                  const __grid_constant__ CUtensorMap ta2, const __grid_constant__ CUtensorMap tb0,
                  const __grid_constant__ CUtensorMap tb1, const __grid_constant__ CUtensorMap tb1h,
                  const __grid_constant__ CUtensorMap tb2, const Params p) {
  using C = Cfg<KS>;
  constexpr int STAGES = C::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;              // ring of T stages
  uint8_t* sB = smem + C::RING;    // the tile's S_d column rows: [d][ks][plane]
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + C::B_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* bfull = empty + STAGES;  // S block of the tile landed
  uint64_t* bempty = bfull + 1;      // S block free (the tile's MMAs retired)
  uint64_t* accf = bempty + 1;       // [NBUF] accumulator buffer ready
  uint64_t* acce = accf + NBUF;      // [NBUF] accumulator buffer drained
  uint64_t* done = acce + NBUF;
  uint64_t* never = done + 1;        // completed by nobody (the test stall waits on it)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* epi_flag = abort_flag + 1;  // [2] the poller's result for the epilogue warps

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int steps_per_tile = p.P * 3;  // (p, d) products per tile

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(bfull, 1);
    mbar_init(bempty, 1);
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], EPI);
    }
    mbar_init(done, 1);
    mbar_init(never, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      uint32_t it = 0, tl = 0;  // T stages issued, tiles started
      bool stop = false;
      for (int64_t item = blockIdx.x; item < p.ntiles && !stop; item += gridDim.x, ++tl) {
        int64_t I, J;
        tile_of(p, item, I, J);
        if (!mbar_wait(bempty, (tl & 1u) ^ 1u, abort_flag, p.status, 64)) break;
        mbar_arrive_expect_tx(bfull, C::B_BYTES);
        for (int d = 0; d < 3; ++d)
          for (int ks = 0; ks < KS; ++ks) {
            uint8_t* b = sB + (size_t)((d * KS + ks) * 4) * B_PLANE;
            const int y = (int)(d * p.nrows + J * BN);
            tma_load_2d(&tb0, b + 0 * B_PLANE, bfull, ks * BK, y);
            tma_load_2d(&tb1, b + 1 * B_PLANE, bfull, ks * BK, y);
            tma_load_2d(&tb1h, b + 2 * B_PLANE, bfull, ks * BK, y);
            tma_load_2d(&tb2, b + 3 * B_PLANE, bfull, ks * BK, y);
          }
        for (int q = 0; q < steps_per_tile && !stop; ++q) {
          const int pp = q / 3, d = q % 3;
          const int y = (int)(((int64_t)d * p.P + pp) * p.nrows + I * BM);
          for (int ks = 0; ks < KS; ++ks, ++it) {
            const int s = (int)(it % STAGES);
            if (!mbar_wait(&empty[s], ((it / STAGES) & 1u) ^ 1u, abort_flag, p.status, 256)) { stop = true; break; }
            mbar_arrive_expect_tx(&full[s], A_STAGE);
            uint8_t* a = sA + (size_t)s * A_STAGE;
            tma_load_2d(&ta0, a + 0 * A_PLANE, &full[s], ks * BK, y);
            tma_load_2d(&ta1, a + 1 * A_PLANE, &full[s], ks * BK, y);
            tma_load_2d(&ta2, a + 2 * A_PLANE, &full[s], ks * BK, y);
          }
        }
      }
      // On abort, wait (bounded) for the loads still in flight before the CTA can exit.
      if (*abort_flag) {
        for (uint32_t j = (it > (uint32_t)STAGES ? it - STAGES : 0u); j < it; ++j) {
          const int s = (int)(j % STAGES);
          long long t0 = clock64();
          while (!mbar_try_wait(&full[s], (j / STAGES) & 1u) && clock64() - t0 < kWaitCycles) {
          }
        }
        if (tl > 0) {
          long long t0 = clock64();
          while (!mbar_try_wait(bfull, (tl - 1) & 1u) && clock64() - t0 < kWaitCycles) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      // kind::f16, FP32 accumulators, FP16 operands, both K-major, M = 128, N = 64
      const uint32_t idesc = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
      uint32_t it = 0, cg = 0, tl = 0;
      bool ok = true;
      // test hook: a wait that runs out (nothing arrives on `never`), then the abort path
      if (p.test_stall > 0) ok = mbar_wait(never, 0u, abort_flag, p.status, 0, p.test_stall);
      for (int64_t item = blockIdx.x; item < p.ntiles && ok; item += gridDim.x, ++tl) {
        if (!mbar_wait(bfull, tl & 1u, abort_flag, p.status)) break;
        tc_fence_after();
        for (int q = 0; q < steps_per_tile && ok; ++q, ++cg) {
          const int d = q % 3;
          const int buf = (int)(cg % NBUF);
          // the epilogue is the slower side: poll its drained buffers at a relaxed pace
          if (!mbar_wait(&acce[buf], ((cg / NBUF) & 1u) ^ 1u, abort_flag, p.status, 128)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d0 = tmem_base + (uint32_t)(buf * 2 * BN);
          const uint32_t d1 = d0 + BN;
          for (int ks = 0; ks < KS; ++ks, ++it) {
            const int s = (int)(it % STAGES);
            if (!mbar_wait(&full[s], (it / STAGES) & 1u, abort_flag, p.status)) { ok = false; break; }
            tc_fence_after();
            const uint32_t abase = smem_u32(sA + (size_t)s * A_STAGE);
            const uint32_t bbase = smem_u32(sB + (size_t)((d * KS + ks) * 4) * B_PLANE);
            const uint64_t a0 = smem_desc<BK>(abase), a1 = smem_desc<BK>(abase + A_PLANE),
                           a2 = smem_desc<BK>(abase + 2 * A_PLANE);
            const uint64_t b0 = smem_desc<BK>(bbase), b1 = smem_desc<BK>(bbase + B_PLANE),
                           b1h = smem_desc<BK>(bbase + 2 * B_PLANE), b2 = smem_desc<BK>(bbase + 3 * B_PLANE);
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
              const uint64_t o = (uint64_t)((k * 32) >> 4);  // +32 bytes along K inside the swizzle atom
              const uint32_t first = (ks == 0 && k == 0) ? 0u : 1u;
              mma_bf16_a<ACol::fill>(d0, a0 + o, b0 + o, idesc, first);
              mma_bf16_a<ACol::use>(d1, a0 + o, b1 + o, idesc, first);
              mma_bf16_a<ACol::lastuse>(d1, a0 + o, b2 + o, idesc, 1u);
              mma_bf16_a<ACol::fill>(d1, a1 + o, b0 + o, idesc, 1u);
              mma_bf16_a<ACol::lastuse>(d1, a1 + o, b1h + o, idesc, 1u);
              mma_bf16(d1, a2 + o, b0 + o, idesc, 1u);
            }
            mma_commit(&empty[s]);  // the T stage may be refilled once these MMAs retire
          }
          if (!ok) break;
          mma_commit(&accf[buf]);
        }
        if (!ok) break;
        mma_commit(bempty);  // the S block may be replaced once the tile's MMAs retire
      }
      mma_commit(done);
      long long t0 = clock64();
      while (!mbar_try_wait(done, 0u) && clock64() - t0 < kWaitCycles) {
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue warps
    const int ew = warp - 2;
    const int quad = warp & 3;        // TMEM lane quadrant this warp may access
    const int col0 = (ew >> 2) * QC;  // first column of this thread inside the tile
    uint32_t cg = 0;
    bool ok = true;
    for (int64_t item = blockIdx.x; item < p.ntiles && ok; item += gridDim.x) {
      int64_t I, J;
      tile_of(p, item, I, J);
      const int64_t r = I * BM + quad * 32 + lane;  // this thread's row of B_u
      const bool rlive = r < p.nrows;
      // node sum as an FP32 pair (as, al): two-sum of the leading parts, the rest in the trailing one
      float as[QC], al[QC];
#pragma unroll
      for (int j = 0; j < QC; ++j) as[j] = al[j] = 0.f;
      float2 fnext = rlive ? p.f[r * p.P] : make_float2(0.f, 0.f);
      for (int pp = 0; pp < p.P && ok; ++pp) {
        const float2 f = fnext;  // this node's factor; the next one is fetched while it is used
        if (pp + 1 < p.P && rlive) fnext = p.f[r * p.P + pp + 1];
        float ph[QC], pl[QC];
#pragma unroll
        for (int d = 0; d < 3; ++d, ++cg) {
          const int buf = (int)(cg % NBUF);
          // one thread polls the buffer's barrier; the epilogue warps meet on a named barrier
          if (ew == 0 && lane == 0)
            epi_flag[cg & 1u] = mbar_wait(&accf[buf], (cg / NBUF) & 1u, abort_flag, p.status) ? 1 : 0;
          asm volatile("bar.sync 1, %0;" ::"r"(32 * EPI) : "memory");
          if (!epi_flag[cg & 1u]) { ok = false; break; }
          tc_fence_after();
          const uint32_t tb = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * 2 * BN + col0);
#pragma unroll
          for (int j0 = 0; j0 < QC; j0 += 8) {
            uint32_t l0[8], l12[8];
            tmem_ld8(tb + j0, l0);
            tmem_ld8(tb + BN + j0, l12);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const float gh = __uint_as_float(l0[j]);                      // exact integer sum
              const float gl = __uint_as_float(l12[j]) * (1.0f / 4096.0f);  // exact scaling
              if (d == 0) {
                // f g: f is a normalised pair, so its trailing part times gl (below 2^-33) is dropped
                const float t = f.x * gh;
                float e = fmaf(f.x, gh, -t);
                e = fmaf(f.x, gl, e);
                e = fmaf(f.y, gh, e);
                ph[j0 + j] = t;
                pl[j0 + j] = e;
              } else {
                pmul(ph[j0 + j], pl[j0 + j], gh, gl, ph[j0 + j], pl[j0 + j]);
              }
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acce[buf]);
        }
        if (!ok) break;
#pragma unroll
        for (int j = 0; j < QC; ++j) padd(as[j], al[j], ph[j], pl[j]);
      }
      // every epilogue warp takes the same exits (the poller's flag), as the named barrier needs
      if (!ok) break;
      // store: B_u(r, c) = 2^(Ra(r) + Eb(c) - 48) (as + al); the mirror B_u(c, r) too
      if (rlive && r >= p.r0 && r < p.r1) {
        const int rk = p.ra[r] - 48;
        const int64_t c0 = J * BN + col0;
        if (p.symmetric) {
#pragma unroll
          for (int j = 0; j < QC; ++j) {
            const int64_t c = c0 + j;
            if (c >= p.nrows || c < r) continue;
            const double v = fpair_ldexp(as[j], al[j], rk + p.eb[c]);
            p.out[r * p.ld + c] = v;
            if (c != r) p.out[c * p.ld + r] = v;
          }
        } else {
          double* orow = p.out + (r - p.r0) * p.ld;
#pragma unroll
          for (int j = 0; j < QC; ++j) {
            const int64_t c = c0 + j;
            if (c < p.nrows) orow[c] = fpair_ldexp(as[j], al[j], rk + p.eb[c]);
          }
        }
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512) : "memory");
  }
}

// ------------------------------------------------------------------ operand preparation
// S'_d rows: S_x rows times the row's contraction coefficient c_j, S_y and S_z unchanged.
__global__ void k_scale_rows(const double* __restrict__ S, const double* __restrict__ row_c, int64_t nrows, int n,
                             double* __restrict__ out) {
  const int64_t total = 3 * nrows * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = t / n;  // over [3][nrows]
    out[t] = row < nrows ? S[t] * row_c[row] : S[t];
  }
}

// One warp per row of n <= 64 FP64 values: the row exponent (max|x| 256/255 < 2^e, as the GEMM's
// slicing) and the three slices, zero padded to kpad; t1 / 2^12 too when s1h is given.  An all-zero
// row gets kZeroRowExpo.
__global__ void k_slice_short_rows(const double* __restrict__ src, int64_t rows, int n, int kpad,
                                   uint16_t* __restrict__ s0, uint16_t* __restrict__ s1, uint16_t* __restrict__ s2,
                                   uint16_t* __restrict__ s1h, int* __restrict__ expo) {
  const int lane = threadIdx.x & 31;
  const int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= rows) return;
  const double* x = src + row * n;
  const double x0 = lane < n ? x[lane] : 0.0, x1 = lane + 32 < n ? x[lane + 32] : 0.0;
  uint64_t mx = (uint64_t)__double_as_longlong(x0) & 0x7FFFFFFFFFFFFFFFULL;
  const uint64_t m1 = (uint64_t)__double_as_longlong(x1) & 0x7FFFFFFFFFFFFFFFULL;
  mx = m1 > mx ? m1 : mx;
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t other = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = other > mx ? other : mx;
  }
  const double m = __longlong_as_double((long long)mx);
  int e = 0;
  if (m > 0.0) frexp(m * (256.0 / 255.0), &e);
  const bool nz = m > 0.0 && e >= -1000;
  if (lane == 0) expo[row] = nz ? e : kZeroRowExpo;
  if (lane < kpad) slice_store(x0, e, nz && lane < n, 3, row * kpad + lane, s0, s1, s2, s1h);
  if (lane + 32 < kpad) slice_store(x1, e, nz && lane + 32 < n, 3, row * kpad + lane + 32, s0, s1, s2, s1h);
}

// Per row j: Ea_p(j) = sum_d te[d][p][j], Ra(j) = max_p Ea_p(j), the node factors
// f_p(j) = pref w_p 2^(Ea_p(j) - Ra(j)) as FP32 pairs, and Eb(j) = sum_d se[d][j].
__global__ void k_had_tables(int64_t nrows, int P, const int* __restrict__ te, const int* __restrict__ se,
                             const double* __restrict__ w, double pref, float2* __restrict__ f, int* __restrict__ ra,
                             int* __restrict__ eb) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nrows) return;
  int R = kZeroRowExpo;
  for (int p = 0; p < P; ++p) {
    const int Ea = te[(0 * (int64_t)P + p) * nrows + j] + te[(1 * (int64_t)P + p) * nrows + j] +
                   te[(2 * (int64_t)P + p) * nrows + j];
    R = max(R, Ea);
  }
  const bool live = R > kZeroRowExpo / 2;  // some node has all three factors non-zero
  for (int p = 0; p < P; ++p) {
    const int Ea = te[(0 * (int64_t)P + p) * nrows + j] + te[(1 * (int64_t)P + p) * nrows + j] +
                   te[(2 * (int64_t)P + p) * nrows + j];
    const int sh = Ea - R;
    float2 v = make_float2(0.f, 0.f);
    if (live && sh > -300) {
      const double x = pref * w[p];
      const float hi = (float)x;
      const float lo = (float)(x - (double)hi);
      v = make_float2(ldexpf(hi, sh), ldexpf(lo, sh));
    }
    f[j * P + p] = v;
  }
  ra[j] = live ? R : 0;
  eb[j] = se[j] + se[nrows + j] + se[2 * nrows + j];
}

}  // namespace tch

void launch_had_prepare(const HadOperands& h, const double* d_S, const double* d_C, const double* d_w, double pref,
                        const double* d_row_c, double* d_Ss, double* d_T, cudaStream_t st) {
  const int64_t nrows = h.nrows;
  const int n = h.n, P = h.P;
  count_launch();
  tch::k_scale_rows<<<(unsigned)std::min<int64_t>((3 * nrows * n + 255) / 256, 152 * 32), 256, 0, st>>>(
      d_S, d_row_c, nrows, n, d_Ss);
  launch_tmat(nrows, n, P, d_Ss, d_C, d_T, st);  // T[d][p][row][:] = S'_d(row, :) A_d^(p)
  const int64_t trows = 3LL * P * nrows, srows = 3LL * nrows;
  count_launch();
  tch::k_slice_short_rows<<<(unsigned)((trows + 7) / 8), 256, 0, st>>>(d_T, trows, n, h.kpad, h.t0, h.t1, h.t2,
                                                                       nullptr, h.te);
  count_launch();
  tch::k_slice_short_rows<<<(unsigned)((srows + 7) / 8), 256, 0, st>>>(d_Ss, srows, n, h.kpad, h.s0, h.s1, h.s2,
                                                                       h.s1h, h.se);
  count_launch();
  tch::k_had_tables<<<(unsigned)((nrows + 127) / 128), 128, 0, st>>>(nrows, P, h.te, h.se, d_w, pref, h.f, h.ra,
                                                                      h.eb);
}

template <int KS>
static lrtei_status launch_had_kernel(const HadOperands& h, const tch::Params& p, cudaStream_t st) {
  using namespace tch;
  CUtensorMap m[7];
  const int64_t trows = 3LL * h.P * h.nrows, srows = 3LL * h.nrows;
  const bool ok = tc::encode_plane(&m[0], h.t0, trows, h.kpad, BM, false, BK) &&
                  tc::encode_plane(&m[1], h.t1, trows, h.kpad, BM, false, BK) &&
                  tc::encode_plane(&m[2], h.t2, trows, h.kpad, BM, false, BK) &&
                  tc::encode_plane(&m[3], h.s0, srows, h.kpad, BN, false, BK) &&
                  tc::encode_plane(&m[4], h.s1, srows, h.kpad, BN, false, BK) &&
                  tc::encode_plane(&m[5], h.s1h, srows, h.kpad, BN, false, BK) &&
                  tc::encode_plane(&m[6], h.s2, srows, h.kpad, BN, false, BK);
  if (!ok) {
    set_error("cuTensorMapEncodeTiled failed for the Hadamard operands");
    return LRTEI_ERR_CUDA;
  }
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_hadamard<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Cfg<KS>::SMEM);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core Hadamard smem attribute");
    attr_set = true;
  }
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(p.ntiles, nsm));
  count_launch();
  k_tc_hadamard<KS><<<(unsigned)grid, THREADS, Cfg<KS>::SMEM, st>>>(m[0], m[1], m[2], m[3], m[4], m[5], m[6], p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core Hadamard launch");
  return LRTEI_OK;
}

lrtei_status had_tc_rows(const HadOperands& h, int64_t r0, int64_t r1, double* d_out, int64_t ld, int* d_status,
                         cudaStream_t st) {
  using namespace tch;
  if (r0 < 0 || r1 > h.nrows || r0 >= r1) return LRTEI_OK;
  if (3LL * h.P * h.nrows >= (1LL << 31) || (h.kpad != 32 && h.kpad != 64)) {
    set_error("tensor-core Hadamard form: 3 P nrows must stay below 2^31 and n at most 64");
    return LRTEI_ERR_UNSUPPORTED;
  }
  Params p{};
  p.nrows = h.nrows;
  p.P = h.P;
  p.r0 = r0;
  p.r1 = r1;
  p.symmetric = (r0 == 0 && r1 == h.nrows) ? 1 : 0;
  p.tiles_n = (h.nrows + BN - 1) / BN;
  if (p.symmetric) {
    p.tm0 = 0;
    p.tiles_m = (h.nrows + BM - 1) / BM;
    p.ntiles = 0;
    for (int64_t I = 0; I < p.tiles_m; ++I) p.ntiles += p.tiles_n - 2 * I;
  } else {
    p.tm0 = r0 / BM;
    p.tiles_m = (r1 + BM - 1) / BM - p.tm0;
    p.ntiles = p.tiles_m * p.tiles_n;
  }
  p.f = h.f;
  p.ra = h.ra;
  p.eb = h.eb;
  p.out = d_out;
  p.ld = ld;
  p.status = d_status;
  {
    // LRTEI_TEST_STALL_CYCLES (tests only), as for the GEMM: every CTA's MMA thread first waits that
    // many cycles on a barrier nothing completes, raises LRTEI_ERR_TIMEOUT and drains
    const char* v = getenv("LRTEI_TEST_STALL_CYCLES");
    p.test_stall = (v && *v) ? std::max(0LL, atoll(v)) : 0;
  }
  ProfScope ps("tc_hadamard", st);
  return h.kpad == 32 ? launch_had_kernel<1>(h, p, st) : launch_had_kernel<2>(h, p, st);
}

}  // namespace lrtei
