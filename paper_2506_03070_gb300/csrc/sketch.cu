// sketch.cu -- the sparse sign sketch generated and applied in one pass over
// [A | b] (Algorithm 1 "Form Y = SA" with the Sec. 2.1 sketch, columns drawn
// by the Sec. 3.1.2 rejection sampler).  S is never stored: each warp draws
// the columns of S for 32 consecutive rows of A in registers, then streams
// those rows with coalesced loads and scatters s_ik * [A_i, b_i] into Y.
#include <algorithm>

#include "dfloat.cuh"
#include "kernels.h"
#include "sketch.cuh"

namespace lsq {

namespace {

// One thread per column of S: export indices and signs.
template <int N>
__global__ void __launch_bounds__(256) k_sketch_indices(uint64_t seed, int64_t row0, int64_t rows, uint64_t d,
                                                        int zeta, int32_t* __restrict__ idx, int8_t* __restrict__ sgn,
                                                        int32_t* __restrict__ rounds, uint32_t* status,
                                                        int32_t* max_rounds) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rows; t += (int64_t)gridDim.x * blockDim.x) {
    int32_t c[N];
    uint64_t signs;
    const int r = sketch_column<N>(seed, (uint64_t)(row0 + t), d, zeta, c, signs);
    if (r < 0) atomicOr(status, DS_SKETCH);
    if (r > 0) atomicMax(max_rounds, r);
    if (rounds) rounds[t] = r;
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (k < zeta) {
        idx[t * zeta + k] = c[k];
        sgn[t * zeta + k] = ((signs >> k) & 1ull) ? (int8_t)1 : (int8_t)-1;
      }
  }
}

// Exponent field of a finite FP64 value into the running maximum (non-finite
// values are reported separately).
__device__ __forceinline__ void track_exp(double a, uint32_t& emax) {
  const uint32_t e = (uint32_t)__double2hiint(a) & 0x7FF00000u;
  if (e != 0x7FF00000u) emax = max(emax, e);
}
// Warp sum of A_ij^2 into *fro.
__device__ __forceinline__ void flush_fro(double fa, double* fro) {
  if (!fro) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fa += __shfl_xor_sync(0xffffffffu, fa, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(fro, fa);
}

// Warp maxima of the A and b exponent fields into range[0], range[1].
__device__ __forceinline__ void flush_range(uint32_t ea, uint32_t eb, uint32_t* range) {
  if (!range) return;
  ea = __reduce_max_sync(0xffffffffu, ea);
  eb = __reduce_max_sync(0xffffffffu, eb);
  if ((threadIdx.x & 31) == 0) {
    if (ea) atomicMax(range, ea);
    if (eb) atomicMax(range + 1, eb);
  }
}

__device__ __forceinline__ void red_add(double* p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void red_add(float* p, double v) { atomicAdd(p, (float)v); }

__device__ __forceinline__ double flip_sign(double v, bool neg) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)neg << 63));
}

// Warps own 32 consecutive rows at a time.  Lane l draws column (row0+base+l)
// of S into shared memory; then the warp walks the 32 rows, lanes spread over
// the n (+1 for b) entries of each row, and adds +-A_ij/sqrt(zeta) into the
// zeta target rows of Y with global reductions (Y is L2-resident).
template <int N, typename TY>
__global__ void __launch_bounds__(256) k_sketch_apply(const double* __restrict__ A, int64_t m, int n, int64_t lda,
                                                      const double* __restrict__ b, uint64_t d, int zeta,
                                                      uint64_t seed, int64_t row0, TY* __restrict__ Y, int64_t ldy,
                                                      double scale, uint32_t* status, int32_t* max_rounds,
                                                      uint32_t* range, double* fro) {
  extern __shared__ int32_t s_idx[];  // [8 warps][32 rows][N]
  __shared__ uint64_t s_sgn[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* my_idx = s_idx + wib * 32 * N;
  const int ncol = n + (b ? 1 : 0);
  bool bad = false;
  uint32_t ea = 0, eb = 0;
  double fa = 0.0;
  for (int64_t base = ((int64_t)blockIdx.x * 8 + wib) * 32; base < m; base += (int64_t)gridDim.x * 8 * 32) {
    const int64_t row = base + lane;
    if (row < m) {
      int32_t c[N];
      uint64_t signs;
      const int r = sketch_column<N>(seed, (uint64_t)(row0 + row), d, zeta, c, signs);
      if (r < 0) atomicOr(status, DS_SKETCH);
      if (r > 0) atomicMax(max_rounds, r);
#pragma unroll
      for (int k = 0; k < N; ++k) my_idx[lane * N + k] = c[k];
      s_sgn[wib][lane] = signs;
    }
    __syncwarp();
    const int nrows = (int)min((int64_t)32, m - base);
    for (int rr = 0; rr < nrows; ++rr) {
      const int64_t i = base + rr;
      const double* Ai = A + i * lda;
      const uint64_t sg = s_sgn[wib][rr];
      const int32_t* ci = my_idx + rr * N;
      for (int j = lane; j < ncol; j += 32) {
        const double a = j < n ? __ldcs(Ai + j) : b[i];
        bad |= !isfinite(a);
        track_exp(a, j < n ? ea : eb);
        if (j < n) fa = fma(a, a, fa);
        const double sa = a * scale;
        for (int k = 0; k < zeta; ++k) {
          const double v = flip_sign(sa, ((sg >> k) & 1ull) == 0ull);
          red_add(Y + (int64_t)ci[k] * ldy + j, v);
        }
      }
    }
    __syncwarp();
  }
  if (bad) atomicOr(status, DS_NONFINITE);
  flush_range(ea, eb, range);
  flush_fro(fa, fro);
}

__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

__device__ __forceinline__ float flip_sign_f(float v, bool neg) { return __uint_as_float(__float_as_uint(v) ^ ((uint32_t)neg << 31)); }

// Vector atomic add that returns the four old values.
__device__ __forceinline__ float4 atom_add_v4(float* p, float a, float b, float c, float d) {
  float4 o;
  asm volatile("atom.global.add.v4.f32 {%0, %1, %2, %3}, [%4], {%5, %6, %7, %8};"
               : "=f"(o.x), "=f"(o.y), "=f"(o.z), "=f"(o.w)
               : "l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
  return o;
}

// (old + v) - fl(old + v) exactly (Knuth's TwoSum): the rounding error of the
// atomic add that turned `old` into fl(old + v), recomputed from its inputs.
__device__ __forceinline__ float add_err(float old, float v) {
  const float s = __fadd_rn(old, v);
  const float bp = __fsub_rn(s, old);
  const float ap = __fsub_rn(s, bp);
  return __fadd_rn(__fsub_rn(old, ap), __fsub_rn(v, bp));
}

// FP64 entry -> nearest float using integer ops only (the FP64->FP32
// conversion instruction runs at about one per clock per SM on this GPU).
__device__ __forceinline__ float to_float_int(double a) {
  float hi, mid;
  split2(a, hi, mid);
  return __fadd_rn(hi, mid);
}

// FP32 accumulation (mixed form) with 4-wide vector reductions: lane l owns
// column groups 4(l + 32t) .. +3; entries past n are b_i (column n) or 0.
// Requires ldy % 4 == 0 and Y (and Ylo) 16-byte aligned.
//
// COMP (compensated): every add into Y is a vector atomic that returns the
// old values; the exact rounding error of each add (TwoSum of old and the
// term) goes into Ylo with a vector reduction.  Y + Ylo then equals the exact
// sum up to Ylo's own FP32 rounding, errors of size u^2 sqrt(N) relative for N
// terms per entry, instead of u sqrt(N) for plain FP32 accumulation (with
// about 5000 terms per entry at 5e6 rows and d = 8000, 1e-6 relative against
// the 2.5e-8 of rounding an FP64 sketch once).  Atomics are issued eight
// targets at a time so their round trips overlap.
template <int N, bool COMP>
__global__ void __launch_bounds__(256) k_sketch_apply_f32v(const double* __restrict__ A, int64_t m, int n, int64_t lda,
                                                           const double* __restrict__ b, uint64_t d, int zeta,
                                                           uint64_t seed, int64_t row0, float* __restrict__ Y,
                                                           float* __restrict__ Ylo, int64_t ldy, float scale,
                                                           uint32_t* status, int32_t* max_rounds, uint32_t* range,
                                                           double* fro) {
  extern __shared__ int32_t s_idx[];  // [8 warps][32 rows][N]
  __shared__ uint64_t s_sgn[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* my_idx = s_idx + wib * 32 * N;
  const int ncol = n + (b ? 1 : 0);
  const int ngroups = (ncol + 3) / 4;
  bool bad = false;
  uint32_t ea = 0, eb = 0;
  double fa = 0.0;
  for (int64_t base = ((int64_t)blockIdx.x * 8 + wib) * 32; base < m; base += (int64_t)gridDim.x * 8 * 32) {
    const int64_t row = base + lane;
    if (row < m) {
      int32_t c[N];
      uint64_t signs;
      const int r = sketch_column<N>(seed, (uint64_t)(row0 + row), d, zeta, c, signs);
      if (r < 0) atomicOr(status, DS_SKETCH);
      if (r > 0) atomicMax(max_rounds, r);
#pragma unroll
      for (int k = 0; k < N; ++k) my_idx[lane * N + k] = c[k];
      s_sgn[wib][lane] = signs;
    }
    __syncwarp();
    const int nrows = (int)min((int64_t)32, m - base);
    for (int rr = 0; rr < nrows; ++rr) {
      const int64_t i = base + rr;
      const double* Ai = A + i * lda;
      const uint64_t sg = s_sgn[wib][rr];
      const int32_t* ci = my_idx + rr * N;
      for (int g = lane; g < ngroups; g += 32) {
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 4 * g + q;
          const double a = j < n ? __ldcs(Ai + j) : (j == n && b ? b[i] : 0.0);
          bad |= !isfinite(a);
          track_exp(a, j < n ? ea : eb);
          if (j < n) fa = fma(a, a, fa);
          v[q] = __fmul_rn(to_float_int(a), scale);
        }
        if (COMP) {
          for (int k0 = 0; k0 < zeta; k0 += 8) {
            float4 o[8];
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
              const int k = k0 + kk;
              if (k < zeta) {
                const bool neg = ((sg >> k) & 1ull) == 0ull;
                o[kk] = atom_add_v4(Y + (int64_t)ci[k] * ldy + 4 * g, flip_sign_f(v[0], neg), flip_sign_f(v[1], neg),
                                    flip_sign_f(v[2], neg), flip_sign_f(v[3], neg));
              }
            }
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
              const int k = k0 + kk;
              if (k < zeta) {
                const bool neg = ((sg >> k) & 1ull) == 0ull;
                red_add_v4(Ylo + (int64_t)ci[k] * ldy + 4 * g, add_err(o[kk].x, flip_sign_f(v[0], neg)),
                           add_err(o[kk].y, flip_sign_f(v[1], neg)), add_err(o[kk].z, flip_sign_f(v[2], neg)),
                           add_err(o[kk].w, flip_sign_f(v[3], neg)));
              }
            }
          }
        } else {
          for (int k = 0; k < zeta; ++k) {
            const bool neg = ((sg >> k) & 1ull) == 0ull;
            red_add_v4(Y + (int64_t)ci[k] * ldy + 4 * g, flip_sign_f(v[0], neg), flip_sign_f(v[1], neg),
                       flip_sign_f(v[2], neg), flip_sign_f(v[3], neg));
          }
        }
      }
    }
    __syncwarp();
  }
  if (bad) atomicOr(status, DS_NONFINITE);
  flush_range(ea, eb, range);
  flush_fro(fa, fro);
}

// range_scan: one warp per row (grid-stride), lanes over the columns and b_i.
__global__ void __launch_bounds__(256) k_range_scan(const double* __restrict__ A, int64_t m, int n, int64_t lda,
                                                    const double* __restrict__ b, uint32_t* range, uint32_t* status) {
  const int lane = threadIdx.x & 31;
  uint32_t ea = 0, eb = 0;
  bool bad = false;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < m; i += nwarps) {
    const double* Ai = A + i * lda;
    for (int j = lane; j < n; j += 32) {
      const double a = __ldcs(Ai + j);
      bad |= !isfinite(a);
      track_exp(a, ea);
    }
    if (lane == 0 && b) {
      bad |= !isfinite(b[i]);
      track_exp(b[i], eb);
    }
  }
  if (bad) atomicOr(status, DS_NONFINITE);
  flush_range(ea, eb, range);
}

template <int N>
cudaError_t launch_apply_f32v(const double* A, int64_t m, int n, int64_t lda, const double* b, int64_t d, int zeta,
                              uint64_t seed, int64_t row0, float* Y, float* Ylo, int64_t ldy, uint32_t* status,
                              int32_t* max_rounds, uint32_t* range, double* fro, int sms, cudaStream_t st) {
  const size_t smem = (size_t)8 * 32 * N * sizeof(int32_t);
  const void* fn = Ylo ? (const void*)k_sketch_apply_f32v<N, true> : (const void*)k_sketch_apply_f32v<N, false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t groups = (m + 255) / 256;
  const int64_t blocks = std::min<int64_t>(groups, (int64_t)sms * 8);
  const float scale = (float)(1.0 / sqrt((double)zeta));
  if (blocks > 0) {
    if (Ylo)
      k_sketch_apply_f32v<N, true><<<(unsigned)blocks, 256, smem, st>>>(A, m, n, lda, b, (uint64_t)d, zeta, seed,
                                                                        row0, Y, Ylo, ldy, scale, status, max_rounds,
                                                                        range, fro);
    else
      k_sketch_apply_f32v<N, false><<<(unsigned)blocks, 256, smem, st>>>(A, m, n, lda, b, (uint64_t)d, zeta, seed,
                                                                         row0, Y, nullptr, ldy, scale, status,
                                                                         max_rounds, range, fro);
  }
  return cudaGetLastError();
}

__global__ void k_add_lo(float* __restrict__ Y, const float* __restrict__ Ylo, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    Y[e] = __fadd_rn(Y[e], Ylo[e]);
}

template <int N>
cudaError_t launch_indices(uint64_t seed, int64_t row0, int64_t rows, int64_t d, int zeta, int32_t* idx, int8_t* sgn,
                           int32_t* rounds, uint32_t* status, int32_t* max_rounds, int sms, cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>((rows + 255) / 256, (int64_t)sms * 16);
  if (blocks > 0)
    k_sketch_indices<N><<<(unsigned)blocks, 256, 0, st>>>(seed, row0, rows, (uint64_t)d, zeta, idx, sgn, rounds,
                                                          status, max_rounds);
  return cudaGetLastError();
}

template <int N, typename TY>
cudaError_t launch_apply(const double* A, int64_t m, int n, int64_t lda, const double* b, int64_t d, int zeta,
                         uint64_t seed, int64_t row0, TY* Y, int64_t ldy, uint32_t* status, int32_t* max_rounds,
                         uint32_t* range, double* fro, int sms, cudaStream_t st) {
  const size_t smem = (size_t)8 * 32 * N * sizeof(int32_t);
  cudaError_t e = cudaFuncSetAttribute(k_sketch_apply<N, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t groups = (m + 255) / 256;
  const int64_t blocks = std::min<int64_t>(groups, (int64_t)sms * 8);
  if (blocks > 0)
    k_sketch_apply<N, TY><<<(unsigned)blocks, 256, smem, st>>>(A, m, n, lda, b, (uint64_t)d, zeta, seed, row0, Y, ldy,
                                                               1.0 / sqrt((double)zeta), status, max_rounds, range,
                                                               fro);
  return cudaGetLastError();
}

}  // namespace

cudaError_t sketch_indices(uint64_t seed, int64_t row0, int64_t rows, int64_t d, int zeta, int32_t* idx, int8_t* sgn,
                           int32_t* rounds, uint32_t* status, int32_t* max_rounds, int sms, cudaStream_t st) {
  if (zeta <= 8) return launch_indices<8>(seed, row0, rows, d, zeta, idx, sgn, rounds, status, max_rounds, sms, st);
  if (zeta <= 16) return launch_indices<16>(seed, row0, rows, d, zeta, idx, sgn, rounds, status, max_rounds, sms, st);
  if (zeta <= 32) return launch_indices<32>(seed, row0, rows, d, zeta, idx, sgn, rounds, status, max_rounds, sms, st);
  return launch_indices<64>(seed, row0, rows, d, zeta, idx, sgn, rounds, status, max_rounds, sms, st);
}

template <typename TY>
cudaError_t sketch_apply(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, int64_t d, int zeta,
                         uint64_t seed, int64_t row0, TY* Y, int64_t ldy, uint32_t* status, int32_t* max_rounds,
                         uint32_t* range, double* fro, int sms, cudaStream_t st) {
  const int ni = (int)n;
  if (sizeof(TY) == 4 && ldy % 4 == 0 && (uintptr_t)Y % 16 == 0)
    return sketch_apply_f32c(A, m, n, lda, b, d, zeta, seed, row0, reinterpret_cast<float*>(Y), nullptr, ldy, status,
                             max_rounds, range, fro, sms, st);
  if (zeta <= 8)
    return launch_apply<8, TY>(A, m, ni, lda, b, d, zeta, seed, row0, Y, ldy, status, max_rounds, range, fro, sms,
                               st);
  if (zeta <= 16)
    return launch_apply<16, TY>(A, m, ni, lda, b, d, zeta, seed, row0, Y, ldy, status, max_rounds, range, fro, sms,
                               st);
  if (zeta <= 32)
    return launch_apply<32, TY>(A, m, ni, lda, b, d, zeta, seed, row0, Y, ldy, status, max_rounds, range, fro, sms,
                               st);
  return launch_apply<64, TY>(A, m, ni, lda, b, d, zeta, seed, row0, Y, ldy, status, max_rounds, range, fro, sms,
                               st);
}

cudaError_t sketch_apply_f32c(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, int64_t d,
                              int zeta, uint64_t seed, int64_t row0, float* Y, float* Ylo, int64_t ldy,
                              uint32_t* status, int32_t* max_rounds, uint32_t* range, double* fro, int sms,
                              cudaStream_t st) {
  const int ni = (int)n;
  if (ldy % 4 != 0 || (uintptr_t)Y % 16 != 0 || (uintptr_t)Ylo % 16 != 0) return cudaErrorInvalidValue;
  if (zeta <= 8)
    return launch_apply_f32v<8>(A, m, ni, lda, b, d, zeta, seed, row0, Y, Ylo, ldy, status, max_rounds, range, fro, sms, st);
  if (zeta <= 16)
    return launch_apply_f32v<16>(A, m, ni, lda, b, d, zeta, seed, row0, Y, Ylo, ldy, status, max_rounds, range, fro, sms,
                                 st);
  if (zeta <= 32)
    return launch_apply_f32v<32>(A, m, ni, lda, b, d, zeta, seed, row0, Y, Ylo, ldy, status, max_rounds, range, fro, sms,
                                 st);
  return launch_apply_f32v<64>(A, m, ni, lda, b, d, zeta, seed, row0, Y, Ylo, ldy, status, max_rounds, range, fro, sms, st);
}

cudaError_t add_lo(float* Y, const float* Ylo, int64_t count, int sms, cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>((count + 255) / 256, (int64_t)sms * 8);
  if (blocks > 0) k_add_lo<<<(unsigned)blocks, 256, 0, st>>>(Y, Ylo, count);
  return cudaGetLastError();
}

cudaError_t range_scan(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, uint32_t* range,
                       uint32_t* status, int sms, cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>((m + 7) / 8, (int64_t)sms * 8);
  if (blocks > 0) k_range_scan<<<(unsigned)blocks, 256, 0, st>>>(A, m, (int)n, lda, b, range, status);
  return cudaGetLastError();
}

template cudaError_t sketch_apply<double>(const double*, int64_t, int64_t, int64_t, const double*, int64_t, int,
                                          uint64_t, int64_t, double*, int64_t, uint32_t*, int32_t*, uint32_t*, double*,
                                          int, cudaStream_t);
template cudaError_t sketch_apply<float>(const double*, int64_t, int64_t, int64_t, const double*, int64_t, int,
                                         uint64_t, int64_t, float*, int64_t, uint32_t*, int32_t*, uint32_t*, double*,
                                         int, cudaStream_t);

}  // namespace lsq
