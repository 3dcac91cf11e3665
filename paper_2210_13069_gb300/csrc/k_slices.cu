// k_slices.cu -- FP64 rows to the operand planes of the tensor-core GEMM (three integer slices
// held exactly in FP16 and one exponent per row, or one BF16 plane), plus the transpose and
// split-K reduction kernels around the skinny GEMMs of the J-build.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lrtei_internal.h"
#include "tc_common.h"

namespace cg = cooperative_groups;

namespace lrtei {
namespace tc {

// Largest |x| of the row from the bit patterns (finite inputs order like their magnitudes),
// then e with max|x| * 256/255 < 2^e (0 for an all-zero row).
__device__ __forceinline__ int row_exponent(uint64_t mxbits, uint64_t* red, bool& nonzero) {
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t other = __shfl_xor_sync(0xffffffffu, mxbits, o);
    mxbits = other > mxbits ? other : mxbits;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mxbits;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint64_t v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0ULL;
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t other = __shfl_xor_sync(0xffffffffu, v, o);
      v = other > v ? other : v;
    }
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const double mx = __longlong_as_double((long long)red[0]);
  int e = 0;
  if (mx > 0.0) frexp(mx * (256.0 / 255.0), &e);
  nonzero = mx > 0.0 && e >= -1000;  // rows below ~1e-301 are treated as zero
  return e;
}

// One block per row; rows of up to 1024 * EPT elements are read once and kept in registers.
template <int EPT>
__global__ void __launch_bounds__(1024) k_split_rows_reg(const double* __restrict__ src, int64_t rows, int64_t k, int64_t ld,
                                                        int64_t kpad, uint16_t* __restrict__ s0, uint16_t* __restrict__ s1,
                                                        uint16_t* __restrict__ s2, uint16_t* __restrict__ s1h,
                                                        int* __restrict__ expo, int nslices) {
  __shared__ uint64_t red[32];
  const int64_t r = blockIdx.x;
  const double* x = src + r * ld;
  double v[EPT];
  uint64_t mx = 0;
#pragma unroll
  for (int j = 0; j < EPT; ++j) {
    const int64_t i = threadIdx.x + (int64_t)j * blockDim.x;
    v[j] = i < k ? x[i] : 0.0;
    const uint64_t a = (uint64_t)__double_as_longlong(v[j]) & 0x7FFFFFFFFFFFFFFFULL;
    mx = a > mx ? a : mx;
  }
  bool nz;
  const int e = row_exponent(mx, red, nz);
  if (threadIdx.x == 0) expo[r] = e;
#pragma unroll
  for (int j = 0; j < EPT; ++j) {
    const int64_t i = threadIdx.x + (int64_t)j * blockDim.x;
    if (i < kpad) slice_store(v[j], e, i < k && nz, nslices, r * kpad + i, s0, s1, s2, s1h);
  }
  for (int64_t i = threadIdx.x + (int64_t)EPT * blockDim.x; i < kpad; i += blockDim.x)
    slice_store(0.0, e, false, nslices, r * kpad + i, s0, s1, s2, s1h);
}

// Short rows (padded length at most 256): one warp per row, eight consecutive elements per lane
// (16-byte loads where the rows allow them, one 16-byte store per plane); the exponent and the
// slices are those of the one-block-per-row kernels.
__global__ void __launch_bounds__(256) k_split_rows_warp(const double* __restrict__ src, int64_t rows, int64_t k,
                                                         int64_t ld, int64_t kpad, uint16_t* __restrict__ s0,
                                                         uint16_t* __restrict__ s1, uint16_t* __restrict__ s2,
                                                         uint16_t* __restrict__ s1h, int* __restrict__ expo,
                                                         int nslices) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= rows) return;  // the whole warp: r is the same on its lanes
  const double* x = src + r * ld;
  const bool vec = (ld & 1) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0;
  constexpr uint64_t kMag = 0x7FFFFFFFFFFFFFFFULL;
  const int64_t i0 = 8 * (int64_t)lane;
  double v[8];
  if (vec && i0 + 7 < k) {
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      const double2 a = *reinterpret_cast<const double2*>(x + i0 + j);
      v[j] = a.x;
      v[j + 1] = a.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = i0 + j < k ? x[i0 + j] : 0.0;
  }
  uint64_t mx = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint64_t a = (uint64_t)__double_as_longlong(v[j]) & kMag;
    mx = a > mx ? a : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t other = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = other > mx ? other : mx;
  }
  const double mxd = __longlong_as_double((long long)mx);
  int e = 0;
  if (mxd > 0.0) frexp(mxd * (256.0 / 255.0), &e);
  const bool nz = mxd > 0.0 && e >= -1000;  // rows below ~1e-301 are treated as zero
  if (lane == 0) expo[r] = e;
  if (i0 >= kpad) return;
  SliceBits q[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) q[j] = slice_bits(v[j], e, i0 + j < k && nz, nslices);
  const int64_t o = r * kpad + i0;
  *reinterpret_cast<uint4*>(s0 + o) =
      make_uint4(q[0].s0 | (uint32_t)q[1].s0 << 16, q[2].s0 | (uint32_t)q[3].s0 << 16,
                 q[4].s0 | (uint32_t)q[5].s0 << 16, q[6].s0 | (uint32_t)q[7].s0 << 16);
  *reinterpret_cast<uint4*>(s1 + o) =
      make_uint4(q[0].s1 | (uint32_t)q[1].s1 << 16, q[2].s1 | (uint32_t)q[3].s1 << 16,
                 q[4].s1 | (uint32_t)q[5].s1 << 16, q[6].s1 | (uint32_t)q[7].s1 << 16);
  *reinterpret_cast<uint4*>(s2 + o) =
      make_uint4(q[0].s2 | (uint32_t)q[1].s2 << 16, q[2].s2 | (uint32_t)q[3].s2 << 16,
                 q[4].s2 | (uint32_t)q[5].s2 << 16, q[6].s2 | (uint32_t)q[7].s2 << 16);
  if (s1h)
    *reinterpret_cast<uint4*>(s1h + o) =
        make_uint4(q[0].s1h | (uint32_t)q[1].s1h << 16, q[2].s1h | (uint32_t)q[3].s1h << 16,
                   q[4].s1h | (uint32_t)q[5].s1h << 16, q[6].s1h | (uint32_t)q[7].s1h << 16);
}

// Long rows: two passes over the row (maximum, then slices), four consecutive elements per thread
// and step: 16-byte loads where the rows allow them (even ld, 16-byte aligned source) and one
// 8-byte store per plane (kpad is a multiple of 4).
__global__ void __launch_bounds__(256) k_split_rows4(const double* __restrict__ src, int64_t rows, int64_t k,
                                                     int64_t ld, int64_t kpad, uint16_t* __restrict__ s0,
                                                     uint16_t* __restrict__ s1, uint16_t* __restrict__ s2,
                                                     uint16_t* __restrict__ s1h, int* __restrict__ expo, int nslices) {
  __shared__ uint64_t red[32];
  const int64_t r = blockIdx.x;
  const double* x = src + r * ld;
  const bool vec = (ld & 1) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0;
  constexpr uint64_t kMag = 0x7FFFFFFFFFFFFFFFULL;
  uint64_t mx = 0;
  for (int64_t i = 4 * (int64_t)threadIdx.x; i < k; i += 4 * (int64_t)blockDim.x) {
    if (vec && i + 3 < k) {
      const double2 a = *reinterpret_cast<const double2*>(x + i);
      const double2 b = *reinterpret_cast<const double2*>(x + i + 2);
      const uint64_t m0 = (uint64_t)__double_as_longlong(a.x) & kMag, m1 = (uint64_t)__double_as_longlong(a.y) & kMag;
      const uint64_t m2 = (uint64_t)__double_as_longlong(b.x) & kMag, m3 = (uint64_t)__double_as_longlong(b.y) & kMag;
      const uint64_t u = m0 > m1 ? m0 : m1, w = m2 > m3 ? m2 : m3;
      const uint64_t t = u > w ? u : w;
      mx = t > mx ? t : mx;
    } else {
      for (int j = 0; j < 4 && i + j < k; ++j) {
        const uint64_t a = (uint64_t)__double_as_longlong(x[i + j]) & kMag;
        mx = a > mx ? a : mx;
      }
    }
  }
  bool nz;
  const int e = row_exponent(mx, red, nz);
  if (threadIdx.x == 0) expo[r] = e;
  for (int64_t i = 4 * (int64_t)threadIdx.x; i < kpad; i += 4 * (int64_t)blockDim.x) {
    double v[4];
    if (vec && i + 3 < k) {
      const double2 a = *reinterpret_cast<const double2*>(x + i);
      const double2 b = *reinterpret_cast<const double2*>(x + i + 2);
      v[0] = a.x;
      v[1] = a.y;
      v[2] = b.x;
      v[3] = b.y;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = i + j < k ? x[i + j] : 0.0;
    }
    SliceBits q[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) q[j] = slice_bits(v[j], e, i + j < k && nz, nslices);
    const int64_t o = r * kpad + i;
    *reinterpret_cast<ushort4*>(s0 + o) = make_ushort4(q[0].s0, q[1].s0, q[2].s0, q[3].s0);
    *reinterpret_cast<ushort4*>(s1 + o) = make_ushort4(q[0].s1, q[1].s1, q[2].s1, q[3].s1);
    *reinterpret_cast<ushort4*>(s2 + o) = make_ushort4(q[0].s2, q[1].s2, q[2].s2, q[3].s2);
    if (s1h) *reinterpret_cast<ushort4*>(s1h + o) = make_ushort4(q[0].s1h, q[1].s1h, q[2].s1h, q[3].s1h);
  }
}

// Few long rows (fewer rows than SMs, e.g. the R density rows of a J-build): a cluster of
// kSplitCluster CTAs per row, each taking an eighth of the padded row.  Every CTA reduces the
// magnitude bits over its share, the cluster combines the eight maxima through distributed shared
// memory, and each CTA slices its share with the row's exponent: the exponent and the slices are
// those of the one-block-per-row kernels.
constexpr int kSplitCluster = 8;
__global__ void __cluster_dims__(kSplitCluster, 1, 1) __launch_bounds__(256)
    k_split_rows_cluster(const double* __restrict__ src, int64_t k, int64_t ld, int64_t kpad,
                         uint16_t* __restrict__ s0, uint16_t* __restrict__ s1, uint16_t* __restrict__ s2,
                         uint16_t* __restrict__ s1h, int* __restrict__ expo, int nslices) {
  __shared__ uint64_t red[8];
  __shared__ uint64_t share;
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned rank = cluster.block_rank();
  const int64_t r = blockIdx.y;
  const double* x = src + r * ld;
  const int64_t per = (kpad + kSplitCluster - 1) / kSplitCluster;
  const int64_t c0 = (int64_t)rank * per, c1 = min(kpad, c0 + per), ck = min(c1, k);
  uint64_t mx = 0;
  for (int64_t i = c0 + threadIdx.x; i < ck; i += blockDim.x) {
    const uint64_t a = (uint64_t)__double_as_longlong(x[i]) & 0x7FFFFFFFFFFFFFFFULL;
    mx = a > mx ? a : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t other = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = other > mx ? other : mx;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t v = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = red[w] > v ? red[w] : v;
    share = v;
  }
  cluster.sync();  // every CTA's share is written
  uint64_t v = 0;
  for (int q = 0; q < kSplitCluster; ++q) {
    const uint64_t o = *cluster.map_shared_rank(&share, q);
    v = o > v ? o : v;
  }
  cluster.sync();  // every CTA has read the shares before any of them exits
  const double mxd = __longlong_as_double((long long)v);
  int e = 0;
  if (mxd > 0.0) frexp(mxd * (256.0 / 255.0), &e);
  const bool nz = mxd > 0.0 && e >= -1000;
  if (rank == 0 && threadIdx.x == 0) expo[r] = e;
  for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x)
    slice_store(i < k ? x[i] : 0.0, e, i < k && nz, nslices, r * kpad + i, s0, s1, s2, s1h);
}

// Plain BF16 operands: one rounded copy per element, exponent 8 so that the epilogue scale
// 2^(ea + eb - 16) is 1.
__global__ void k_plain_rows(const double* __restrict__ src, int64_t rows, int64_t k, int64_t ld, int64_t kpad,
                             uint16_t* __restrict__ s0, int* __restrict__ expo) {
  const int64_t r = blockIdx.x;
  if (threadIdx.x == 0) expo[r] = 8;
  for (int64_t i = threadIdx.x; i < kpad; i += blockDim.x) {
    const float v = i < k ? (float)src[r * ld + i] : 0.f;
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    s0[r * kpad + i] = *reinterpret_cast<uint16_t*>(&h);
  }
}

// 32 x 32 tiled transpose of an FP64 matrix: out (cols x rows) = in (rows x cols)^T.
__global__ void k_transpose(const double* __restrict__ in, int64_t rows, int64_t cols, int64_t ldi,
                            double* __restrict__ out, int64_t ldo) {
  __shared__ double t[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[i][threadIdx.x] = in[r * ldi + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[c * ldo + r] = t[threadIdx.x][i];
  }
}

// Sum of split-K partials: out[i] = sum_s part[s * stride + i] (row-major rows x cols, ld).
__global__ void k_reduce_splits(const double* __restrict__ part, int splits, int64_t stride, int64_t rows,
                                int64_t cols, int64_t ld, double* __restrict__ out, int64_t ldo) {
  const int64_t total = rows * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / cols, j = t % cols;
    double s = 0.0;
    for (int q = 0; q < splits; ++q) s += part[q * stride + i * ld + j];
    out[i * ldo + j] = s;
  }
}

}  // namespace tc

void launch_split_rows(const double* d_src, int64_t rows, int64_t k, int64_t ld, SplitMatrix& m, bool with_s1h,
                       int nslices, cudaStream_t st) {
  if (rows <= 0) return;
  count_launch();
  if (m.plain) {
    tc::k_plain_rows<<<(unsigned)rows, 256, 0, st>>>(d_src, rows, k, ld, m.kpad, m.s0, m.expo);
    return;
  }
  uint16_t* s1h = (with_s1h || m.eight) ? m.s1h : nullptr;
  if (m.kpad <= 256) {  // short rows (e.g. the N_b-long rows of the exchange's MT): a warp per row
    tc::k_split_rows_warp<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(d_src, rows, k, ld, m.kpad, m.s0, m.s1, m.s2,
                                                                      s1h, m.expo, nslices);
    return;
  }
  // few long rows (fewer than four per SM, e.g. the R density rows of a J-build or the N_b rows of
  // the exchange's last product): eight CTAs per row
  if ((rows < 4 * 152 && k >= 8192) || (rows < 152 && k >= 2048)) {
    tc::k_split_rows_cluster<<<dim3(tc::kSplitCluster, (unsigned)rows), 256, 0, st>>>(d_src, k, ld, m.kpad, m.s0, m.s1,
                                                                                     m.s2, s1h, m.expo, nslices);
    return;
  }
  // Rows of up to 4096 elements stay in registers (one read); longer rows take two passes with
  // 256 threads, more rows in flight per SM (the second pass reads the row from L2).  The padded
  // length is a multiple of 256 here (kpad256).
  if (k <= 4096)
    tc::k_split_rows_reg<4><<<(unsigned)rows, 1024, 0, st>>>(d_src, rows, k, ld, m.kpad, m.s0, m.s1, m.s2, s1h,
                                                            m.expo, nslices);
  else
    tc::k_split_rows4<<<(unsigned)rows, 256, 0, st>>>(d_src, rows, k, ld, m.kpad, m.s0, m.s1, m.s2, s1h, m.expo,
                                                      nslices);
}

void launch_transpose(const double* in, int64_t rows, int64_t cols, int64_t ldi, double* out, int64_t ldo,
                      cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return;
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32)), block(32, 8);
  count_launch();
  tc::k_transpose<<<grid, block, 0, st>>>(in, rows, cols, ldi, out, ldo);
}

void launch_reduce_splits(const double* part, int splits, int64_t stride, int64_t rows, int64_t cols, int64_t ld,
                          double* out, int64_t ldo, cudaStream_t st) {
  const int64_t total = rows * cols;
  if (total <= 0) return;
  int64_t b = (total + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  count_launch();
  tc::k_reduce_splits<<<(unsigned)b, 256, 0, st>>>(part, splits, stride, rows, cols, ld, out, ldo);
}

}  // namespace lrtei
