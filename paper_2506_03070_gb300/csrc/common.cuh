// common.cuh -- device helpers shared by the library's kernels: the Philox
// counter-based generator, bounded grid barriers, warp reductions and the
// status word every kernel reports into.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lsq.h"

namespace lsq {

// Device status bits (OR-ed into a device word, mapped to lsq_status on the host).
enum : uint32_t {
  DS_SKETCH = 1u,     // rejection sampling exceeded its round cap
  DS_NONFINITE = 2u,  // NaN/Inf seen in A or b
  DS_TIMEOUT = 4u,    // a grid barrier wait gave up
  DS_RANK = 8u,       // zero/negligible diagonal of R
  DS_NOCONV = 16u,    // LSQR reached maxit
  DS_CSR = 32u,       // malformed CSR structure (row offsets or column indices)
  DS_ACCURACY = 64u,  // the accuracy pass's backward-error bound exceeded the gate
};

constexpr int kMaxZeta = 64;
constexpr int kMaxRounds = 10000;
// A device wait (grid barrier, bulk-copy mbarrier) gives up after this many
// nanoseconds unless the barrier word carries its own limit (limit_us).
constexpr unsigned long long kBarrierTimeoutNs = 20ull * 1000ull * 1000ull * 1000ull;

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 64x64->128 multiplies with key advance by the two Weyl constants.
// ---------------------------------------------------------------------------
struct U64x4 {
  uint64_t w[4];
};

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                                               uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  U64x4 o;
  o.w[0] = c0;
  o.w[1] = c1;
  o.w[2] = c2;
  o.w[3] = c3;
  return o;
}

// floor(word * d / 2^64): maps a uniform 64-bit word to [0, d).
__device__ __forceinline__ int32_t word_to_index(uint64_t word, uint64_t d) { return (int32_t)__umul64hi(word, d); }

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// Grid barrier for cooperative (co-resident) launches: a ticket barrier on
// one counter.  Thread 0 of each block arrives with one release atomic
// (count += 1) and polls the same word with acquire loads until the round's
// nblocks arrivals are in: target = (arrival / nblocks + 1) * nblocks.  The
// host zeroes `count` before a launch and it advances by nblocks per barrier,
// so it stays a multiple of nblocks between barriers (a launch with a
// different block count needs it zeroed again).  Abort is the top bit of the
// same word, seen by every arrival and poll without an extra load.  Every wait
// is bounded: by limit_us microseconds when the host set it (a run-time
// setting that outlives the zeroing of `count`), else by kBarrierTimeoutNs.
// On timeout the block raises DS_TIMEOUT and the abort bit, and every block
// leaves at its next barrier.  Returns false when the caller must exit.
// ---------------------------------------------------------------------------
struct GridBarrier {
  unsigned int count;     // arrivals (low 31 bits) | kBarrierAbort
  unsigned int limit_us;  // wait limit of every wait tied to this barrier; 0 = kBarrierTimeoutNs
  unsigned int pad[2];
};
constexpr unsigned int kBarrierAbort = 0x80000000u;

// Wait limit (ns) of the waits tied to `bar` (bulk-copy waits of a pass read
// it once per pass).
__device__ __forceinline__ unsigned long long wait_limit_ns(const GridBarrier* bar) {
  const unsigned int us = bar ? *(volatile const unsigned int*)&bar->limit_us : 0u;
  return us ? (unsigned long long)us * 1000ull : kBarrierTimeoutNs;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned int atom_add_release_u32(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Raise the abort bit: every block of the barrier leaves at its next barrier.
__device__ __forceinline__ void barrier_abort(GridBarrier* bar) { atomicOr(&bar->count, kBarrierAbort); }

__device__ __forceinline__ bool grid_sync(GridBarrier* bar, uint32_t* status, unsigned int nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int a = atom_add_release_u32(&bar->count, 1u);
    if (a & kBarrierAbort) {
      ok = 0;
    } else {
      const unsigned int target = (a / nblocks + 1u) * nblocks;
      unsigned int v = ld_acquire_u32(&bar->count);
      if (!(v & kBarrierAbort) && (int)(v - target) < 0) {
        const unsigned long long t0 = globaltimer_ns(), limit = wait_limit_ns(bar);
        unsigned int spins = 0;
        for (;;) {
          __nanosleep(20);
          v = ld_acquire_u32(&bar->count);
          if ((v & kBarrierAbort) || (int)(v - target) >= 0) break;
          if ((++spins & 63u) == 0 && globaltimer_ns() - t0 > limit) {
            atomicOr(status, DS_TIMEOUT);
            barrier_abort(bar);
            v = kBarrierAbort;
            break;
          }
        }
      }
      if (v & kBarrierAbort) ok = 0;
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ bool grid_sync(GridBarrier* bar, uint32_t* status) {
  return grid_sync(bar, status, gridDim.x);
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_allreduce_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_allreduce_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The 32-double scratch of block_sum, one per block for all callers: every
// block_sum starts with a barrier before it writes the scratch, so calls in
// sequence may share it.
__device__ __forceinline__ double* block_scratch() {
  __shared__ double s_scratch[32];
  return s_scratch;
}

// Block-wide sum in a fixed order (deterministic for a fixed block size).
// `scratch` holds at least 32 doubles.  Result valid in every thread.  One
// thread adds the per-warp sums and shares the total: GB300's FP64 pipe
// retires ~1.6 lanes per clock per SM, so every thread adding them would cost
// each warp its own pass through the pipe.  Every thread reads the total
// before it can reach the next call's first barrier, and the total is only
// rewritten after that call's second one.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
  __shared__ double s_total;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_allreduce_sum(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += scratch[i];
    s_total = s;
  }
  __syncthreads();
  return s_total;
}

}  // namespace lsq
