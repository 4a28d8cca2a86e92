// tc_gemm.cu -- the blocked Householder QR's trailing updates on the
// 5th-generation tensor cores: tcgen05.mma with TMEM accumulators, operands
// staged in shared memory by TMA (cp.async.bulk.tensor), one elected thread
// issuing, four warps reading the accumulators back with tcgen05.ld.
//
// The QR works in FP64 (plain form) or FP32 (mixed form); the tensor cores
// multiply bf16.  Both are reached exactly by splitting every operand row
// into S bf16 slices of 8 significant bits (error-free splitting in the manner
// of Ozaki et al.'s scheme): a row x with |x_k| < 2^e is written
//   x = 2^e sum_{q<S} s_q 2^(-7-8q),  s_q integers in [-128, 128]
// (the remainder is below 2^(e-8S)).  A product of two slices is an integer
// of magnitude <= 2^14, so the products of slice pairs (q, t) with q + t = p,
// summed over a K chunk of 128, stay below 7 * 128 * 2^14 < 2^24: the FP32
// accumulation in TMEM is exact whatever its order.  Group p of a chunk is
// read back (tcgen05.ld) and added, as the integer it is, into two 64-bit
// integer sums per output (the last min(S, 4) groups into one, the others into
// the second, each group shifted to its weight 2^(-8p)): the whole K
// accumulates exactly, and FP64 arithmetic is needed only once per output at
// the end, where the sums are scaled and the row and column exponents
// 2^(e_a + e_b) applied.  Pairs
// with q + t >= S are dropped: for S = 7 (FP64 data, 56 bits per row) the
// result carries an error of about K 2^-53 max|a_row| max|b_row|, that of an
// FP64 GEMM's normwise bound; S = 4 (FP32 data) gives FP32's for entries down
// to 2^-8 of their row's largest.
//
// D (M x N) = A B^T with A's rows and B's rows both K-major bf16 slices in
// global memory ([S][rows][Kpad]); tiles of 128 x 64 outputs, K staged 32 at a
// time (one 64-byte swizzle row) through a two-slot ring.  Epilogues:
//   mode 0: out[a_row * ldo + b_row] += D (FP64 atomics; split K over grid.z)
//   mode 1: out[b_row * ldo + a_row] -= D (FP64 or FP32, column-major C)
#include <cuda.h>  // CUtensorMap and its enums; the encoder is fetched through the runtime
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "dfloat.cuh"
#include "kernels.h"

namespace lsq {
namespace {

constexpr int kTM = 128;   // output rows per tile = TMEM lanes
constexpr int kTN = 64;    // output columns per tile
constexpr int kKS = 32;    // K per pipeline stage: one 64-byte swizzle row of bf16
constexpr int kKC = 128;   // K per exact FP32 accumulation chunk
constexpr int kStages = 2;
constexpr int kThreadsG = 256;  // 8 warps: warps w and w + 4 read TMEM lanes 32 (w % 4) .. +31, halves of the columns

template <int S>
__host__ __device__ constexpr int stage_bytes() {
  return S * (kTM + kTN) * kKS * 2;
}
template <int S>
__host__ __device__ constexpr int gemm_smem_bytes() {
  return 1024 + kStages * stage_bytes<S>() > 80 * 1024 ? 1024 + kStages * stage_bytes<S>() : 80 * 1024;
}
template <int S>
__host__ __device__ constexpr uint32_t tmem_cols() {
  return S * kTN <= 256 ? 256u : 512u;
}

// ---------------------------------------------------------------------------
// tcgen05 / TMA primitives (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, bf16 inputs, FP32 accumulation.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on an mbarrier once every tcgen05 operation this thread issued so far has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 16 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
// 3-D tiled TMA load (x = K, y = row, z = slice) completing on an mbarrier.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor of a K-major bf16 tile written by TMA with
// 64-byte swizzling: rows of 64 bytes, 8-row atoms of 512 bytes (stride
// dimension byte offset), layout type SWIZZLE_64B, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc_sw64(const void* tile) {
  const uint32_t a = smem_u32(tile);
  uint64_t d = (uint64_t)((a & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;              // leading dimension byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;     // stride dimension byte offset: 8 rows x 64 B
  d |= (uint64_t)1 << 46;              // descriptor version
  d |= (uint64_t)4 << 61;              // SWIZZLE_64B
  return d;
}
// Instruction descriptor: kind::f16 with bf16 A and B, FP32 D, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// The integer value of an FP32 accumulator that holds an exact integer of
// magnitude below 2^24 (a group sum of one chunk), from its IEEE fields:
// mantissa with the hidden bit, shifted right by 150 - exponent (zero gives
// exponent 0 and a shift of 31, hence 0).
__device__ __forceinline__ int32_t exact_int(float g) {
  const uint32_t b = __float_as_uint(g);
  const uint32_t e = (b >> 23) & 0xFFu;
  const uint32_t mant = (b & 0x7FFFFFu) | 0x800000u;
  const uint32_t sh = min(150u - e, 31u);
  const int32_t mag = (int32_t)(mant >> sh);
  return (b >> 31) ? -mag : mag;
}

struct OzParams {
  int M, N, K;        // A rows, B rows, shared dimension
  int k_split;        // K per CTA (multiple of kKC); grid.z = ceil(K / k_split)
  const int* ea;      // [M] row exponents of A
  const int* eb;      // [N] row exponents of B
  int mode;           // 0: out[a * ldo + b] += D (FP64 atomics); 1: out[b * ldo + a] -= D
  int out_f32;        // mode 1: out is float
  void* out;
  int64_t ldo;
  uint32_t* status;
  const GridBarrier* bar;  // wait limit
};

template <int S>
__global__ void __launch_bounds__(kThreadsG, 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap tma_a, const __grid_constant__ CUtensorMap tma_b, OzParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bar_full[kStages];
  __shared__ __align__(8) uint64_t bar_mma[kStages];
  __shared__ __align__(8) uint64_t bar_fin;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  __shared__ int s_lst;
  __shared__ uint32_t s_lpar;
  const int warp = threadIdx.x >> 5;
  const int m0 = blockIdx.x * kTM, n0 = blockIdx.y * kTN;
  const int k_begin = blockIdx.z * p.k_split;
  const int k_end = min(p.K, k_begin + p.k_split);
  const int nk = k_end > k_begin ? (k_end - k_begin + kKS - 1) / kKS : 0;
  constexpr uint32_t kCols = tmem_cols<S>();
  constexpr uint32_t kIdesc = idesc_bf16(kTM, kTN);
  constexpr int kABytes = kTM * kKS * 2, kBBytes = kTN * kKS * 2;
  constexpr uint32_t kTx = (uint32_t)S * (kABytes + kBBytes);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&bar_full[s], 1u);
      mbar_init(&bar_mma[s], 1u);
    }
    mbar_init(&bar_fin, 1u);
    fence_proxy_async_smem();
    s_fail = 0;
    s_lst = 0;
    s_lpar = 0;
  }
  if (warp == 0) {
    tmem_alloc(&s_tmem, kCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const unsigned long long lim = wait_limit_ns(p.bar);

  auto a_tile = [&](int st, int q) { return smem + st * stage_bytes<S>() + q * kABytes; };
  auto b_tile = [&](int st, int t) { return smem + st * stage_bytes<S>() + S * kABytes + t * kBBytes; };
  auto issue_tma = [&](int kb) {
    const int st = kb % kStages;
    const int k = k_begin + kb * kKS;
    mbar_arrive_expect_tx(&bar_full[st], kTx);
#pragma unroll
    for (int q = 0; q < S; ++q) tma_load_3d(a_tile(st, q), &tma_a, k, m0, q, &bar_full[st]);
#pragma unroll
    for (int t = 0; t < S; ++t) tma_load_3d(b_tile(st, t), &tma_b, k, n0, t, &bar_full[st]);
  };

  // exact integer sums of the groups (see the file header), this thread's
  // row and column half: lo over the last L groups, hi over the first S - L
  constexpr int L = S < 4 ? S : 4, H = S - L, kHalf = kTN / 2;
  int64_t acc_lo[kHalf], acc_hi[H > 0 ? kHalf : 1];
#pragma unroll
  for (int c = 0; c < kHalf; ++c) acc_lo[c] = 0;
#pragma unroll
  for (int c = 0; c < (H > 0 ? kHalf : 1); ++c) acc_hi[c] = 0;
  const int col_half = (warp >> 2) * kHalf;

  // thread 0's pipeline state: stages issued to TMA, stages whose data it
  // has waited for, and the barrier phase of the chunk's last commit
  int issued = 0, consumed = 0;
  if (threadIdx.x == 0)
    for (; issued < nk && issued < kStages; ++issued) issue_tma(issued);

  for (int kc = 0; kc < nk; kc += kKC / kKS) {
    const int kc_end = min(nk, kc + kKC / kKS);
    if (threadIdx.x == 0) {
      for (int kb = kc; kb < kc_end && !s_fail; ++kb) {
        const int st = kb % kStages;
        const uint32_t par = (uint32_t)(kb / kStages) & 1u;
        if (!mbar_wait_bounded(&bar_full[st], par, lim)) {
          s_fail = 1;
          break;
        }
        consumed = kb + 1;
        tc_fence_after();
#pragma unroll
        for (int kk = 0; kk < kKS / 16; ++kk) {
#pragma unroll
          for (int pg = 0; pg < S; ++pg) {
#pragma unroll
            for (int q = 0; q <= pg; ++q) {
              const int t = pg - q;
              // K advance inside the swizzle row: 16 bf16 = 32 bytes = 2 descriptor units
              const uint64_t ad = smem_desc_sw64(a_tile(st, q)) + (uint64_t)(kk * 2);
              const uint64_t bd = smem_desc_sw64(b_tile(st, t)) + (uint64_t)(kk * 2);
              const uint32_t accum = (kb == kc && kk == 0 && q == 0) ? 0u : 1u;
              mma_bf16(tmem + (uint32_t)(pg * kTN), ad, bd, kIdesc, accum);
            }
          }
        }
        mma_commit(&bar_mma[st]);
        s_lst = st;
        s_lpar = par;
        if (issued < nk) {
          // the slot is refilled once the MMAs reading it are done
          if (!mbar_wait_bounded(&bar_mma[st], par, lim)) {
            s_fail = 1;
            break;
          }
          issue_tma(issued++);
        }
      }
    }
    __syncthreads();
    if (s_fail) break;
    // every MMA of the chunk has completed once its last commit arrived
    if (!mbar_wait_bounded(&bar_mma[s_lst], s_lpar, lim)) atomicOr(&s_fail, 1);
    tc_fence_after();
    __syncthreads();
    if (s_fail) break;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
#pragma unroll
    for (int pg = 0; pg < S; ++pg) {
#pragma unroll
      for (int c16 = 0; c16 < kHalf / 16; ++c16) {
        float v[16];
        tmem_ld16(tmem + lane_base + (uint32_t)(pg * kTN + col_half + c16 * 16), v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int64_t g = (int64_t)exact_int(v[j]);
          if (pg < H)
            acc_hi[c16 * 16 + j] += g * ((int64_t)1 << (8 * (H - 1 - pg)));
          else
            acc_lo[c16 * 16 + j] += g * ((int64_t)1 << (8 * (S - 1 - pg)));
        }
      }
    }
    tc_fence_before();
    __syncthreads();  // the accumulators are free for the next chunk
  }

  if (s_fail) {
    if (threadIdx.x == 0) atomicOr(p.status, DS_TIMEOUT);
  } else if (nk > 0) {
    const int row = m0 + 32 * (warp & 3) + (threadIdx.x & 31);
    // value = acc_hi 2^(-14 - 8 (H - 1)) + acc_lo 2^(-14 - 8 (S - 1)); the
    // conversions round only past 2^53 (acc_lo over many chunks)
    const double s_hi = ldexp(1.0, -14 - 8 * (H - 1)), s_lo = ldexp(1.0, -14 - 8 * (S - 1));
    double acc[kHalf];
#pragma unroll
    for (int c = 0; c < kHalf; ++c)
      acc[c] = H > 0 ? fma((double)acc_hi[H > 0 ? c : 0], s_hi, (double)acc_lo[c] * s_lo) : (double)acc_lo[c] * s_lo;
    if (row < p.M) {
      const int ea = p.ea[row];
      if (p.mode == 0) {
        double* out = static_cast<double*>(p.out) + (int64_t)row * p.ldo;
#pragma unroll
        for (int c = 0; c < kHalf; ++c) {
          const int col = n0 + col_half + c;
          if (col < p.N) atomicAdd(out + col, ldexp(acc[c], ea + p.eb[col]));
        }
      } else if (p.out_f32) {
        float* out = static_cast<float*>(p.out);
#pragma unroll
        for (int c = 0; c < kHalf; ++c) {
          const int col = n0 + col_half + c;
          if (col < p.N) {
            float* o = out + (int64_t)col * p.ldo + row;
            *o = (float)((double)*o - ldexp(acc[c], ea + p.eb[col]));
          }
        }
      } else {
        double* out = static_cast<double*>(p.out);
#pragma unroll
        for (int c = 0; c < kHalf; ++c) {
          const int col = n0 + col_half + c;
          if (col < p.N) {
            double* o = out + (int64_t)col * p.ldo + row;
            *o -= ldexp(acc[c], ea + p.eb[col]);
          }
        }
      }
    }
  }
  // after a failed wait: the TMA loads still in flight land and the MMAs
  // issued finish before the shared memory and the TMEM are released
  if (threadIdx.x == 0 && s_fail) {
    for (int kb = consumed; kb < issued; ++kb)
      mbar_wait_bounded(&bar_full[kb % kStages], (uint32_t)(kb / kStages) & 1u, lim);
    mma_commit(&bar_fin);
    mbar_wait_bounded(&bar_fin, 0u, lim);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kCols);
  }
}

// Exact bf16 slices of R rows of length K (row r at X + r * ldx): ex[r] = e
// with max_k |x_rk| < 2^e, and out[q][r][k] = s_q (k < Kpad; zero past K).
// One warp per row.  With T (b x b, column-major, upper) given, the row is
// V_r = sum_l X[l * ldx + r] T[k + l b]  (row r of U T^T, U column-major).
//
// The digits come from integer operations on the IEEE fields (the FP64 pipe
// would bound the pass): F = round(x 2^(7 - e + 8 (S - 1))) as a 64-bit
// integer, |F| < 2^(7 + 8 (S - 1)), split into balanced base-256 digits
// (least significant first: d = F mod 256 in [-128, 127], carry into F), the
// leading digit in [-128, 128]; F = sum_q s_q 2^(8 (S - 1 - q)).  Each digit is
// an integer of magnitude <= 128, exact in bf16 (a table in shared memory).
__device__ __forceinline__ int64_t fixed_point(double x, int shift_base) {
  // x 2^(shift_base), rounded to nearest (ties away), as a 64-bit integer
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  if (ex == 0) return 0;  // zero (and FP64 subnormals, far below every row's scale)
  const long long mant = (long long)((bits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  const int sh = ex - 1075 + shift_base;  // x = mant 2^(ex - 1075)
  long long F;
  if (sh >= 0)
    F = mant << sh;
  else if (sh > -54)
    F = ((mant >> (-sh - 1)) + 1) >> 1;
  else
    F = 0;
  return (bits >> 63) ? -F : F;
}

template <typename TX>
__global__ void __launch_bounds__(256) k_slice(const TX* __restrict__ X, int R, int K, int64_t ldx,
                                               const double* __restrict__ T, int S, __nv_bfloat16* __restrict__ out,
                                               int Kpad, int* __restrict__ ex, int Rpad) {
  __shared__ __nv_bfloat16 s_bf[257];  // s_bf[d + 128] = bf16(d), d in [-128, 128]
  for (int i = threadIdx.x; i < 257; i += blockDim.x) s_bf[i] = __float2bfloat16_rn((float)(i - 128));
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  constexpr int kMaxKT = 64;  // the U T^T form has K = b <= 64: two values per lane
  for (int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < Rpad; r += nwarps) {
    if (r >= R) {  // padding rows of the slice arrays are zero
      for (int q = 0; q < S; ++q)
        for (int k = lane; k < Kpad; k += 32) out[((int64_t)q * Rpad + r) * Kpad + k] = s_bf[128];
      if (lane == 0) ex[r] = 0;
      continue;
    }
    double tv[2] = {0.0, 0.0};
    double mx = 0.0;
    if (T) {
      for (int h = 0; h < 2; ++h) {
        const int k = lane + 32 * h;
        double sum = 0.0;
        if (k < K && k < kMaxKT)
          for (int l = k; l < K; ++l) sum = fma((double)X[(int64_t)l * ldx + r], T[k + (int64_t)l * K], sum);
        tv[h] = sum;
        mx = fmax(mx, fabs(sum));
      }
    } else {
      const TX* x = X + (int64_t)r * ldx;
      for (int k = lane; k < K; k += 32) mx = fmax(mx, fabs((double)x[k]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    if (lane == 0) ex[r] = e;
    const int shift_base = 7 - e + 8 * (S - 1);
    for (int k = lane; k < Kpad; k += 32) {
      long long F = 0;
      if (k < K) F = fixed_point(T ? tv[k >> 5] : (double)X[(int64_t)r * ldx + k], shift_base);
      for (int q = S - 1; q > 0; --q) {
        int dg = (int)(F & 0xFF);
        F >>= 8;  // arithmetic: F = floor(F / 256)
        if (dg >= 128) {
          dg -= 256;
          F += 1;
        }
        out[((int64_t)q * Rpad + r) * Kpad + k] = s_bf[dg + 128];
      }
      out[(int64_t)r * Kpad + k] = s_bf[(int)F + 128];  // leading digit, |F| <= 128
    }
  }
}

// The same slices for the plain form (no T) with one block per row: the row's
// largest magnitude by a block reduction, then its entries sliced by all 256
// threads (rows of C and U are thousands of entries long; a warp per row left
// the pass bound by the latency of its ~250 dependent steps).
template <typename TX>
__global__ void __launch_bounds__(256) k_slice_rows(const TX* __restrict__ X, int R, int K, int64_t ldx, int S,
                                                    __nv_bfloat16* __restrict__ out, int Kpad, int* __restrict__ ex,
                                                    int Rpad) {
  __shared__ __nv_bfloat16 s_bf[257];  // s_bf[d + 128] = bf16(d), d in [-128, 128]
  __shared__ double s_red[8];
  __shared__ int s_e;
  for (int i = threadIdx.x; i < 257; i += blockDim.x) s_bf[i] = __float2bfloat16_rn((float)(i - 128));
  __syncthreads();
  for (int r = blockIdx.x; r < Rpad; r += gridDim.x) {
    if (r >= R) {  // padding rows of the slice arrays are zero
      for (int q = 0; q < S; ++q)
        for (int k = threadIdx.x; k < Kpad; k += blockDim.x) out[((int64_t)q * Rpad + r) * Kpad + k] = s_bf[128];
      if (threadIdx.x == 0) ex[r] = 0;
      continue;
    }
    const TX* x = X + (int64_t)r * ldx;
    double mx = 0.0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) mx = fmax(mx, fabs((double)x[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, s_red[w]);
      int e = 0;
      if (m > 0.0) frexp(m, &e);
      s_e = e;
      ex[r] = e;
    }
    __syncthreads();
    const int shift_base = 7 - s_e + 8 * (S - 1);
    for (int k = threadIdx.x; k < Kpad; k += blockDim.x) {
      long long F = 0;
      if (k < K) F = fixed_point((double)x[k], shift_base);
      for (int q = S - 1; q > 0; --q) {
        int dg = (int)(F & 0xFF);
        F >>= 8;  // arithmetic: F = floor(F / 256)
        if (dg >= 128) {
          dg -= 256;
          F += 1;
        }
        out[((int64_t)q * Rpad + r) * Kpad + k] = s_bf[dg + 128];
      }
      out[(int64_t)r * Kpad + k] = s_bf[(int)F + 128];  // leading digit, |F| <= 128
    }
    __syncthreads();  // s_e and s_red are rewritten for the next row
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point query (the
// library links no driver library).
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(f);
  });
  return fn;
}

// Tensor map of S slices [S][rows][Kpad] bf16 with boxes of 32 (K) x box_rows x 1.
cudaError_t slice_map(CUtensorMap* map, const __nv_bfloat16* base, int S, int rows, int Kpad, int box_rows) {
  EncodeTiled enc = encoder();
  if (!enc) return cudaErrorNotSupported;
  cuuint64_t dims[3] = {(cuuint64_t)Kpad, (cuuint64_t)rows, (cuuint64_t)S};
  cuuint64_t strides[2] = {(cuuint64_t)Kpad * 2, (cuuint64_t)Kpad * 2 * (cuuint64_t)rows};
  cuuint32_t box[3] = {(cuuint32_t)kKS, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(base), dims, strides,
                         box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int S>
cudaError_t launch_oz(const OzGemm& g, cudaStream_t st) {
  CUtensorMap ma, mb;
  cudaError_t e;
  if (g.a_rows < g.M || g.b_rows < g.N || g.a_rows < kTM || g.b_rows < kTN || g.Kpad % kKS) return cudaErrorInvalidValue;
  if ((e = slice_map(&ma, static_cast<const __nv_bfloat16*>(g.a), S, g.a_rows, g.Kpad, kTM)) != cudaSuccess) return e;
  if ((e = slice_map(&mb, static_cast<const __nv_bfloat16*>(g.b), S, g.b_rows, g.Kpad, kTN)) != cudaSuccess) return e;
  OzParams p;
  p.M = g.M;
  p.N = g.N;
  p.K = g.K;
  p.k_split = g.mode == 0 ? g.k_split : ((g.K + kKC - 1) / kKC) * kKC;
  p.ea = g.ea;
  p.eb = g.eb;
  p.mode = g.mode;
  p.out_f32 = g.out_f32;
  p.out = g.out;
  p.ldo = g.ldo;
  p.status = g.status;
  p.bar = g.bar;
  const int smem = gemm_smem_bytes<S>();
  if ((e = cudaFuncSetAttribute(k_oz_gemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
    return e;
  dim3 grid((unsigned)((g.M + kTM - 1) / kTM), (unsigned)((g.N + kTN - 1) / kTN),
            (unsigned)((g.K + p.k_split - 1) / p.k_split));
  if (grid.x == 0 || grid.y == 0 || grid.z == 0) return cudaSuccess;
  k_oz_gemm<S><<<grid, kThreadsG, smem, st>>>(ma, mb, p);
  return cudaGetLastError();
}

}  // namespace

int oz_kpad(int K) { return (K + kKS - 1) / kKS * kKS; }

template <typename TX>
cudaError_t oz_slice(const TX* X, int R, int K, int64_t ldx, const double* T, int S, void* out, int Kpad, int* ex,
                     int Rpad, int sms, cudaStream_t st) {
  if (R <= 0 || Rpad < R) return R <= 0 ? cudaSuccess : cudaErrorInvalidValue;
  if (T && K > 64) return cudaErrorInvalidValue;  // the U T^T form holds two values per lane
  if (!T && K > 256) {
    const int blocks = (int)std::min<int64_t>((int64_t)Rpad, (int64_t)sms * 8);
    k_slice_rows<TX><<<blocks, 256, 0, st>>>(X, R, K, ldx, S, static_cast<__nv_bfloat16*>(out), Kpad, ex, Rpad);
    return cudaGetLastError();
  }
  const int blocks = (int)std::min<int64_t>(((int64_t)Rpad + 7) / 8, (int64_t)sms * 8);
  k_slice<TX><<<blocks, 256, 0, st>>>(X, R, K, ldx, T, S, static_cast<__nv_bfloat16*>(out), Kpad, ex, Rpad);
  return cudaGetLastError();
}
template cudaError_t oz_slice<double>(const double*, int, int, int64_t, const double*, int, void*, int, int*, int, int,
                                      cudaStream_t);
template cudaError_t oz_slice<float>(const float*, int, int, int64_t, const double*, int, void*, int, int*, int, int,
                                     cudaStream_t);

cudaError_t oz_gemm(const OzGemm& g, cudaStream_t st) {
  if (g.S == 7) return launch_oz<7>(g, st);
  if (g.S == 4) return launch_oz<4>(g, st);
  if (g.S == 3) return launch_oz<3>(g, st);
  return cudaErrorInvalidValue;
}

}  // namespace lsq
