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
                                                      double scale, uint32_t* status, int32_t* max_rounds) {
  extern __shared__ int32_t s_idx[];  // [8 warps][32 rows][N]
  __shared__ uint64_t s_sgn[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* my_idx = s_idx + wib * 32 * N;
  const int ncol = n + (b ? 1 : 0);
  bool bad = false;
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
}

__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

__device__ __forceinline__ float flip_sign_f(float v, bool neg) { return __uint_as_float(__float_as_uint(v) ^ ((uint32_t)neg << 31)); }

// FP64 entry -> nearest float using integer ops only (the FP64->FP32
// conversion instruction runs at about one per clock per SM on this GPU).
__device__ __forceinline__ float to_float_int(double a) {
  float hi, mid;
  split2(a, hi, mid);
  return __fadd_rn(hi, mid);
}

// FP32 accumulation (mixed form) with 4-wide vector reductions: lane l owns
// column groups 4(l + 32t) .. +3; entries past n are b_i (column n) or 0.
// Requires ldy % 4 == 0 and Y 16-byte aligned.
template <int N>
__global__ void __launch_bounds__(256) k_sketch_apply_f32v(const double* __restrict__ A, int64_t m, int n, int64_t lda,
                                                           const double* __restrict__ b, uint64_t d, int zeta,
                                                           uint64_t seed, int64_t row0, float* __restrict__ Y,
                                                           int64_t ldy, float scale, uint32_t* status,
                                                           int32_t* max_rounds) {
  extern __shared__ int32_t s_idx[];  // [8 warps][32 rows][N]
  __shared__ uint64_t s_sgn[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* my_idx = s_idx + wib * 32 * N;
  const int ncol = n + (b ? 1 : 0);
  const int ngroups = (ncol + 3) / 4;
  bool bad = false;
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
          v[q] = __fmul_rn(to_float_int(a), scale);
        }
        for (int k = 0; k < zeta; ++k) {
          const bool neg = ((sg >> k) & 1ull) == 0ull;
          red_add_v4(Y + (int64_t)ci[k] * ldy + 4 * g, flip_sign_f(v[0], neg), flip_sign_f(v[1], neg),
                     flip_sign_f(v[2], neg), flip_sign_f(v[3], neg));
        }
      }
    }
    __syncwarp();
  }
  if (bad) atomicOr(status, DS_NONFINITE);
}

template <int N>
cudaError_t launch_apply_f32v(const double* A, int64_t m, int n, int64_t lda, const double* b, int64_t d, int zeta,
                              uint64_t seed, int64_t row0, float* Y, int64_t ldy, uint32_t* status,
                              int32_t* max_rounds, int sms, cudaStream_t st) {
  const size_t smem = (size_t)8 * 32 * N * sizeof(int32_t);
  cudaError_t e =
      cudaFuncSetAttribute(k_sketch_apply_f32v<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t groups = (m + 255) / 256;
  const int64_t blocks = std::min<int64_t>(groups, (int64_t)sms * 8);
  if (blocks > 0)
    k_sketch_apply_f32v<N><<<(unsigned)blocks, 256, smem, st>>>(A, m, n, lda, b, (uint64_t)d, zeta, seed, row0, Y,
                                                                ldy, (float)(1.0 / sqrt((double)zeta)), status,
                                                                max_rounds);
  return cudaGetLastError();
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
                         int sms, cudaStream_t st) {
  const size_t smem = (size_t)8 * 32 * N * sizeof(int32_t);
  cudaError_t e = cudaFuncSetAttribute(k_sketch_apply<N, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t groups = (m + 255) / 256;
  const int64_t blocks = std::min<int64_t>(groups, (int64_t)sms * 8);
  if (blocks > 0)
    k_sketch_apply<N, TY><<<(unsigned)blocks, 256, smem, st>>>(A, m, n, lda, b, (uint64_t)d, zeta, seed, row0, Y, ldy,
                                                               1.0 / sqrt((double)zeta), status, max_rounds);
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
                         int sms, cudaStream_t st) {
  const int ni = (int)n;
  if (sizeof(TY) == 4 && ldy % 4 == 0 && (uintptr_t)Y % 16 == 0) {
    float* Yf = reinterpret_cast<float*>(Y);
    if (zeta <= 8) return launch_apply_f32v<8>(A, m, ni, lda, b, d, zeta, seed, row0, Yf, ldy, status, max_rounds, sms, st);
    if (zeta <= 16)
      return launch_apply_f32v<16>(A, m, ni, lda, b, d, zeta, seed, row0, Yf, ldy, status, max_rounds, sms, st);
    if (zeta <= 32)
      return launch_apply_f32v<32>(A, m, ni, lda, b, d, zeta, seed, row0, Yf, ldy, status, max_rounds, sms, st);
    return launch_apply_f32v<64>(A, m, ni, lda, b, d, zeta, seed, row0, Yf, ldy, status, max_rounds, sms, st);
  }
  if (zeta <= 8) return launch_apply<8, TY>(A, m, ni, lda, b, d, zeta, seed, row0, Y, ldy, status, max_rounds, sms, st);
  if (zeta <= 16)
    return launch_apply<16, TY>(A, m, ni, lda, b, d, zeta, seed, row0, Y, ldy, status, max_rounds, sms, st);
  if (zeta <= 32)
    return launch_apply<32, TY>(A, m, ni, lda, b, d, zeta, seed, row0, Y, ldy, status, max_rounds, sms, st);
  return launch_apply<64, TY>(A, m, ni, lda, b, d, zeta, seed, row0, Y, ldy, status, max_rounds, sms, st);
}

template cudaError_t sketch_apply<double>(const double*, int64_t, int64_t, int64_t, const double*, int64_t, int,
                                          uint64_t, int64_t, double*, int64_t, uint32_t*, int32_t*, int, cudaStream_t);
template cudaError_t sketch_apply<float>(const double*, int64_t, int64_t, int64_t, const double*, int64_t, int,
                                         uint64_t, int64_t, float*, int64_t, uint32_t*, int32_t*, int, cudaStream_t);

}  // namespace lsq
