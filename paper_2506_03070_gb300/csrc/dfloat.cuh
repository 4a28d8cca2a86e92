// dfloat.cuh -- FP64-accurate arithmetic on the FP32/INT pipes ("double-float").
//
// GB300's FP64 pipe issues about 1.65 DFMA per clock per SM (about 1 TFLOP/s),
// which caps a native-FP64 pass over A at ~1.9 TB/s.  The LSQR pass instead
// represents every FP64 element a exactly enough as two floats and does its
// sums as unevaluated float pairs (hi + lo), using only FP32 and integer
// instructions:
//
//  - split2(a): a = hi + mid + (6 lowest mantissa bits, dropped), by bit
//    manipulation: hi carries the top 24 significant bits (truncated), mid the
//    next 23 (47 significant bits).  Relative representation error < 2^-46.  Exact zero and
//    |a| < 2^-103 map to (0, 0); finite |a| must be < 2^128.
//  - split2s(a, s): the same split of a * 2^-s for any FP64 exponent shift s,
//    folded into the exponent re-bias (no rounding).  The passes over A take s
//    from the largest exponent of A's entries (found while A is first read),
//    so that max |A 2^-s| lies in [1, 2): nothing overflows the FP32 range, and
//    only entries below 2^-103 max|A| are flushed to zero (a relative
//    perturbation of A below 2^-103 sqrt(mn) in the Frobenius norm).
//  - two_sum (Knuth): s + e = a + b exactly, branch free.
//  - products: p + e = a*b exactly via one FMA.
//  - df_add / df_mul: pair arithmetic with relative error ~2^-46.
//
// Every operation uses the explicitly rounded intrinsics (__fadd_rn, ...), so
// the compiler cannot contract or reassociate them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lsq {

struct df {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// s + e = a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df df_add(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  df r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

// Pair sum without the final renormalisation (chains of these are followed
// by one df_renorm).
__device__ __forceinline__ df df_add_unnorm(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return df{s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  df r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// acc += a * w with a = (hi, mid) and w = (w1, w2); acc.lo collects every
// rounding error (TwoSum of the running high sum) plus the small products.
__device__ __forceinline__ void df_fma_acc(df& acc, float hi, float mid, float w1, float w2) {
  const float p = __fmul_rn(hi, w1);
  float e = __fmaf_rn(hi, w1, -p);
  e = __fmaf_rn(hi, w2, e);
  e = __fmaf_rn(mid, w1, e);
  float s, err;
  two_sum(acc.hi, p, s, err);
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
}

__device__ __forceinline__ df df_renorm(df a) {
  df r;
  fast_two_sum(a.hi, a.lo, r.hi, r.lo);
  return r;
}

// ---------------------------------------------------------------------------
// The same pair arithmetic on two independent lanes at once with the packed
// FP32x2 instructions (sm_100 and later): every operation is the one of the
// scalar form on each half, in the same order with the same rounding, so the
// results are bit for bit those of the scalar functions; each packed
// instruction does two of them.  (hi, lo) accumulators are float2 pairs:
// hi = (hi_0, hi_1), lo = (lo_0, lo_1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// acc += a * w for two entries: a = (hi, mid), w = (w1, w2), as df_fma_acc.
__device__ __forceinline__ void df2_fma_acc(float2& acc_hi, float2& acc_lo, float2 hi, float2 mid, float2 w1,
                                            float2 w2) {
  const float2 p = __fmul2_rn(hi, w1);
  float2 e = __ffma2_rn(hi, w1, neg2(p));
  e = __ffma2_rn(hi, w2, e);
  e = __ffma2_rn(mid, w1, e);
  // two_sum(acc_hi, p)
  const float2 s = __fadd2_rn(acc_hi, p);
  const float2 bp = __fadd2_rn(s, neg2(acc_hi));
  const float2 ap = __fadd2_rn(s, neg2(bp));
  const float2 err = __fadd2_rn(__fadd2_rn(acc_hi, neg2(ap)), __fadd2_rn(p, neg2(bp)));
  acc_hi = s;
  acc_lo = __fadd2_rn(acc_lo, __fadd2_rn(err, e));
}

// df_renorm on two pairs.
__device__ __forceinline__ void df2_renorm(float2& hi, float2& lo) {
  const float2 s = __fadd2_rn(hi, lo);
  lo = __fadd2_rn(lo, neg2(__fadd2_rn(s, neg2(hi))));
  hi = s;
}

// Exact integer split of an FP64 value into (hi, mid) floats; see above.
__device__ __forceinline__ void split2(double a, float& hi, float& mid) {
  const uint32_t hw = (uint32_t)__double2hiint(a), lw = (uint32_t)__double2loint(a);
  // (hw << 3 | lw >> 29): low 9 exponent bits + top 23 mantissa bits; re-bias
  // the exponent from 1023 to 127 (mod 512 suffices inside the valid range)
  const uint32_t t = __funnelshift_l(lw, hw, 3) - 0xC0000000u;
  const bool ok = (hw & 0x7FF00000u) >= 0x39800000u;  // |a| >= 2^-103
  uint32_t hb = (t & 0x7FFFFFFFu) | (hw & 0x80000000u);
  hb = ok ? hb : 0u;
  // mid = (P + next 23 mantissa bits as fraction) - P, P = +-ulp(hi)
  const uint32_t pb = (hb & 0xFF800000u) - 0x0B800000u;
  uint32_t fb = pb | ((lw >> 6) & 0x7FFFFFu);
  fb = ok ? fb : pb;
  hi = __uint_as_float(hb);
  mid = __fsub_rn(__uint_as_float(fb), __uint_as_float(pb));
}

// Exponent shift of split2s: entries are split as a * 2^-s.  thr: the high
// word's exponent field must reach it (|a| 2^-s >= 2^-103, a nonzero);
// rebias: subtracted from the shifted word (exponent 1023 + s -> 127).
struct SplitShift {
  uint32_t thr, rebias;
};
__host__ __device__ __forceinline__ SplitShift split_shift(int s) {
  int t = 920 + s;  // biased FP64 exponent of 2^(s - 103)
  if (t < 1) t = 1;  // zeros and FP64 subnormals always flush
  SplitShift r;
  r.thr = (uint32_t)t << 20;
  r.rebias = ((uint32_t)(384 + s) & 511u) << 23;
  return r;
}

// split2 of a * 2^-s (see above); the caller keeps max |a 2^-s| < 2^128.
__device__ __forceinline__ void split2s(double a, float& hi, float& mid, SplitShift sh) {
  const uint32_t hw = (uint32_t)__double2hiint(a), lw = (uint32_t)__double2loint(a);
  const uint32_t t = __funnelshift_l(lw, hw, 3) - sh.rebias;
  const bool ok = (hw & 0x7FF00000u) >= sh.thr;
  uint32_t hb = (t & 0x7FFFFFFFu) | (hw & 0x80000000u);
  hb = ok ? hb : 0u;
  const uint32_t pb = (hb & 0xFF800000u) - 0x0B800000u;
  uint32_t fb = pb | ((lw >> 6) & 0x7FFFFFu);
  fb = ok ? fb : pb;
  hi = __uint_as_float(hb);
  mid = __fsub_rn(__uint_as_float(fb), __uint_as_float(pb));
}

__device__ __forceinline__ df df_from_double(double a) {
  df r;
  split2(a, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ df df_from_double_s(double a, SplitShift sh) {
  df r;
  split2s(a, r.hi, r.lo, sh);
  return r;
}

// FP64 value of a pair (one conversion pair + DADD: use sparingly).
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df shfl_xor_df(df a, int o) {
  return df{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ df shfl_df(df a, int src) {
  return df{__shfl_sync(0xffffffffu, a.hi, src), __shfl_sync(0xffffffffu, a.lo, src)};
}

// ---------------------------------------------------------------------------
// Bulk async copies (global -> shared) completing on an mbarrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
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
// bytes: multiple of 16; src and dst 16-byte aligned.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// Wait for the phase with the given parity to complete, giving up after
// limit_ns of %globaltimer time.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  uint32_t it = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++it & 255u) == 0) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > limit_ns) return false;
    }
  }
  return true;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace lsq
