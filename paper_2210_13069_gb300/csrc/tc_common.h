// tc_common.h -- pieces shared by the tensor-core kernels (k_tcgen05.cu, k_tc_hadamard.cu,
// k_slices.cu): inline PTX for mbarriers, TMA, tcgen05 MMAs and TMEM loads, the shared-memory
// operand descriptor, the tensor-map encoder, and the integer slicing of an FP64 element into the
// three FP16 slices of the split-precision operands.
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include "lrtei_internal.h"

namespace lrtei {
namespace tc {

constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz: every mbarrier wait gives up after this

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false if the CTA is aborting or the wait gave up (which raises the abort).
// sleep_ns > 0 parks the waiting warp between polls, leaving issue slots to the MMA thread.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* status,
                                          unsigned sleep_ns = 0, long long limit = kWaitCycles) {
  long long t0 = clock64();
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (sleep_ns) __nanosleep(sleep_ns);
    if ((++spins & 255u) == 0) {
      if (*abort_flag) return false;
      if (clock64() - t0 > limit) {
        *abort_flag = 1;
        atomicExch(status, (int)kDevTimeout);
        return false;
      }
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, void* dst, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand tile with BK*2-byte rows and the matching swizzle: 8-row atoms of 8*BK*2
// bytes stacked along M/N (128-byte swizzle for BK = 64, 64-byte swizzle for BK = 32).
template <int BK>
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  static_assert(BK == 64 || BK == 32, "BK");
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);          // start address
  d |= (uint64_t)1 << 16;                           // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)((8 * BK * 2) >> 4) << 32;         // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;                           // descriptor version
  d |= (uint64_t)(BK == 64 ? 2 : 4) << 61;          // 128-byte or 64-byte swizzle
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// The same with a collector-buffer hint for A: fill (read A and keep it), use (A from the
// buffer), lastuse (from the buffer, then release it).  Consecutive MMAs on one A slice read
// it from shared memory once.
enum class ACol { fill, use, lastuse };
template <ACol C>
__device__ __forceinline__ void mma_bf16_a(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
  if constexpr (C == ACol::fill)
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  else if constexpr (C == ACol::use)
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16.collector::a::use [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ------------------------------------------------------------------ operand slices
__device__ __forceinline__ uint16_t f16_bits(float f) {
  __half h = __float2half_rn(f);
  return *reinterpret_cast<uint16_t*>(&h);
}

// round(x 2^(32 - e)) as an integer, from the bit pattern of x (no FP64 arithmetic: this
// device's FP64 rate would make the slicing ALU-bound).  For |x| < 2^e 255/256 the result is
// below 255 * 2^24 in magnitude; zeros and subnormals give 0.
__device__ __forceinline__ int64_t fixed32(double x, int e) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0) return 0;
  const uint64_t m = (b & ((1ULL << 52) - 1)) | (1ULL << 52);  // x = +-m 2^(E-1075)
  const int sh = E - 1075 + 32 - e;
  int64_t q;
  if (sh >= 0)
    q = (int64_t)(m << (sh > 9 ? 9 : sh));  // not reached for |x| < 2^e (then sh < -20)
  else if (sh < -62)
    q = 0;
  else
    q = (int64_t)((m + (1ULL << (-sh - 1))) >> (-sh));  // round half up
  return (b >> 63) ? -q : q;
}

// Slices of one element: q = round(x 2^(32-e)), s0 = round(q / 2^24), r = q - s0 2^24,
// t1 = round(r / 2^12), t2 = r - t1 2^12; x ~ 2^e (s0 2^-8 + t1 2^-20 + t2 2^-32), |s0| <= 255,
// |t1|, |t2| <= 2048.  As FP16 bit patterns: s0, t1, t2 / 2^12 and t1 / 2^12 -- all exact
// (integers up to 2^11 in magnitude, and those times 2^-12).
struct SliceBits {
  uint16_t s0, s1, s2, s1h;
};
__device__ __forceinline__ SliceBits slice_bits(double x, int e, bool live, int nslices) {
  float a = 0.f, b = 0.f, c = 0.f;
  if (live) {
    const int64_t q = fixed32(x, e);
    const int64_t q0 = (q + (1LL << 23)) >> 24;
    const int64_t r = q - (q0 << 24);
    const int64_t q1 = (r + (1LL << 11)) >> 12;
    const int64_t q2 = r - (q1 << 12);
    a = (float)q0;
    b = nslices > 1 ? (float)q1 : 0.f;
    c = nslices > 2 ? (float)q2 : 0.f;
  }
  return {f16_bits(a), f16_bits(b), f16_bits(c * (1.0f / 4096.0f)), f16_bits(b * (1.0f / 4096.0f))};
}

__device__ __forceinline__ void slice_store(double x, int e, bool live, int nslices, int64_t o, uint16_t* s0,
                                            uint16_t* s1, uint16_t* s2, uint16_t* s1h) {
  const SliceBits q = slice_bits(x, e, live, nslices);
  s0[o] = q.s0;
  s1[o] = q.s1;
  s2[o] = q.s2;
  if (s1h) s1h[o] = q.s1h;
}

// ------------------------------------------------------------------ FP32 pairs to FP64
// An FP32 number as m 2^e, |m| < 2^24.
__device__ __forceinline__ int64_t f32_int(float f, int& e) {
  const uint32_t b = __float_as_uint(f);
  const int E = (int)((b >> 23) & 0xFFu);
  int64_t m = (int64_t)(b & 0x7FFFFFu);
  if (E) m |= 0x800000;
  e = (E ? E : 1) - 150;
  return (b >> 31) ? -m : m;
}

// (hi + lo) 2^k in FP64 from integer arithmetic (this device's FP64 rate would make FP64
// conversions a visible share of the kernels that store pairs): hi + lo = X 2^q with |X| < 2^63,
// exact when the two exponents lie within 38 bits, else the smaller part rounded at 2^-62 of the
// larger; then X 2^(q+k) rounded to 53 bits (half up on the magnitude).  Results below the normal
// range flush to 0.
__device__ __forceinline__ double fpair_ldexp(float hi, float lo, int k) {
  int eb, es;
  int64_t mb = f32_int(hi, eb), ms = f32_int(lo, es);
  if (mb == 0 || (ms != 0 && es > eb)) {  // (mb, eb): the part with the larger exponent
    const int64_t tm = mb;
    mb = ms;
    ms = tm;
    const int te = eb;
    eb = es;
    es = te;
  }
  if (mb == 0) return 0.0;
  int64_t X;
  int q;
  if (ms == 0) {
    X = mb;
    q = eb;
  } else if (eb - es <= 38) {
    X = (mb << (eb - es)) + ms;
    q = es;
  } else {
    const int sh = eb - es - 38;
    X = mb << 38;
    if (sh < 62) {
      const int64_t half = 1LL << (sh - 1);
      X += ms >= 0 ? ((ms + half) >> sh) : -((-ms + half) >> sh);
    }
    q = es + sh;
  }
  if (X == 0) return 0.0;
  const uint64_t a = (uint64_t)(X < 0 ? -X : X);
  const int top = 63 - __clzll((long long)a);  // leading bit
  uint64_t mant;
  int E = top + q + k + 1023;
  if (top > 52) {
    const int sh = top - 52;
    mant = (a + (1ULL << (sh - 1))) >> sh;
    if (mant >> 53) {
      mant >>= 1;
      ++E;
    }
  } else {
    mant = a << (52 - top);
  }
  if (E <= 0) return 0.0;
  if (E > 2046) E = 2046;
  const uint64_t bits = ((uint64_t)(X < 0) << 63) | ((uint64_t)E << 52) | (mant & ((1ULL << 52) - 1));
  return __longlong_as_double((long long)bits);
}

// ------------------------------------------------------------------ host: tensor maps
inline PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    else
      cudaGetLastError();
  }
  return fn;
}

// 2D tensor map of one 16-bit operand plane (rows x kpad, K contiguous): boxes of bk x box_rows,
// 128-byte swizzle for bk = 64, 64-byte swizzle for bk = 32.
inline bool encode_plane(CUtensorMap* m, const uint16_t* base, int64_t rows, int64_t kpad, int box_rows, bool bf16,
                         int bk) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(kpad * 2)};
  cuuint32_t box[2] = {(cuuint32_t)bk, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (void*)base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace tc
}  // namespace lrtei
