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

// Terms per FP32 partial sum of the blocked mixed-form sketch (k_sketch_fold).
constexpr int kFoldTerms = 16;

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

__device__ __forceinline__ double flip_sign(double v, bool neg) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)neg << 63));
}

// Warps own 32 consecutive rows at a time.  Lane l draws column (row0+base+l)
// of S into shared memory; then the warp walks the 32 rows, lanes spread over
// the entries c0 .. c1-1 of each row (column n is b_i), and adds
// +-A_ij/sqrt(zeta) into the zeta target rows of Y with global reductions
// (the launch's column slab of Y is L2-resident).
//
// TEE: A and b live in host memory that the device reads in place (pinned or
// registered); every entry read is also stored to the device copy (Aout with
// row stride ldo, bout), so one pass over the host link both sketches and
// moves the problem.  The lane loads its next four entries before it stores
// or reduces any of them, which keeps enough reads in flight to cover the
// link's latency.
template <int N, typename TY, bool TEE = false>
__global__ void __launch_bounds__(256) k_sketch_apply(const double* __restrict__ A, int64_t m, int n, int64_t lda,
                                                      const double* __restrict__ b, uint64_t d, int zeta,
                                                      uint64_t seed, int64_t row0, TY* __restrict__ Y, int64_t ldy,
                                                      double scale, uint32_t* status, int32_t* max_rounds,
                                                      uint32_t* range, double* fro, int c0, int c1,
                                                      double* __restrict__ Aout = nullptr, int64_t ldo = 0,
                                                      double* __restrict__ bout = nullptr) {
  extern __shared__ int32_t s_idx[];  // [8 warps][32 rows][N]
  __shared__ uint64_t s_sgn[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* my_idx = s_idx + wib * 32 * N;
  const int ncol = min(n + (b ? 1 : 0), c1);
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
      if constexpr (TEE) {
        double* Ao = Aout + i * ldo;
        for (int j0 = c0 + lane; j0 < ncol; j0 += 128) {
          double av[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = j0 + 32 * u;
            av[u] = j < n ? Ai[j] : (j == n ? b[i] : 0.0);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = j0 + 32 * u;
            if (j < ncol) {
              const double a = av[u];
              if (j < n)
                __stcs(Ao + j, a);
              else
                __stcs(bout + i, a);
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
        }
      } else {
        for (int j = c0 + lane; j < ncol; j += 32) {
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

// FP64 entry -> nearest float using integer ops only (the FP64->FP32
// conversion instruction runs at about one per clock per SM on this GPU).
__device__ __forceinline__ float to_float_int(double a) {
  float hi, mid;
  split2(a, hi, mid);
  return __fadd_rn(hi, mid);
}

// Mixed-form sketch with blocked FP32 accumulation: every term is added in
// FP32 (4-wide vector reductions into Yc; lane l owns column groups
// 4(l + 32t) .. +3, entries past n are b_i (column n) or 0), but only
// for one chunk of rows at a time; after each chunk the grid meets at a
// barrier, adds the chunk's sums into the running sketch Yp and clears them.
// Yc holds two chunk buffers (chunk k uses buffer k mod 2): a block folds
// chunk k while the others already reduce chunk k+1 into the other buffer,
// and the barrier after chunk k+1 (which every block reaches only after its
// share of chunk k's fold) orders that fold before chunk k+2 reuses the
// buffer -- one grid barrier per chunk.  A chunk is R rows
// per warp of the grid, sized so that each entry of Yc receives about
// kFoldTerms terms (R = kFoldTerms d / (zeta warps), clamped to [1, 32]):
// FP32 rounding then grows with sqrt(kFoldTerms) instead of sqrt(zeta m / d)
// (about 5000 terms at 5e6 rows, d = 8000).  The chunk sums are combined as
// unevaluated float pairs (hi, lo) by TwoSum, ~48 significant bits, on the
// FP32 pipe (an FP64 add per entry per chunk would tie up GB300's FP64 pipe);
// pairs_to_double / round_to_float turn Yp into the sketch.  ||A||_F^2 is
// summed the same way from the FP32 values of the entries (relative error
// about 2^-22).  Yc (2 d x ldc floats, ldc % 4 == 0, 16-byte aligned) and Yp
// must be zero on entry; Yc is zero again on exit.  Cooperative launch (grid
// barriers).
template <int N>
__global__ void __launch_bounds__(256) k_sketch_fold(const double* __restrict__ A, int64_t m, int n, int64_t lda,
                                                     const double* __restrict__ b, uint64_t d, int zeta,
                                                     uint64_t seed, int R, float* __restrict__ Yc, int64_t ldc,
                                                     float2* __restrict__ Yp, int64_t ldy, float scale,
                                                     uint32_t* status, int32_t* max_rounds, uint32_t* range,
                                                     double* fro, GridBarrier* bar) {
  extern __shared__ int32_t s_idx[];  // [8 warps][32 rows][N]
  __shared__ uint64_t s_sgn[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* my_idx = s_idx + wib * 32 * N;
  const int ncol = n + (b ? 1 : 0);
  const int ngroups = (ncol + 3) / 4;
  const int64_t nw = (int64_t)gridDim.x * 8, gw = (int64_t)blockIdx.x * 8 + wib;
  const int64_t chunk = nw * R;
  bool bad = false;
  uint32_t ea = 0, eb = 0;
  float fh = 0.f, fl = 0.f;  // sum of A_ij^2 as a float pair
  for (int64_t c0 = 0, kc = 0; c0 < m; c0 += chunk, ++kc) {
    float* yck = Yc + (kc & 1) * (int64_t)d * ldc;  // this chunk's buffer
    const int64_t base = c0 + gw * R;
    const int nrows = (int)max((int64_t)0, min((int64_t)R, m - base));
    if (lane < nrows) {
      int32_t c[N];
      uint64_t signs;
      const int r = sketch_column<N>(seed, (uint64_t)(base + lane), d, zeta, c, signs);
      if (r < 0) atomicOr(status, DS_SKETCH);
      if (r > 0) atomicMax(max_rounds, r);
#pragma unroll
      for (int k = 0; k < N; ++k) my_idx[lane * N + k] = c[k];
      s_sgn[wib][lane] = signs;
    }
    __syncwarp();
    for (int rr = 0; rr < nrows; ++rr) {
      const int64_t i = base + rr;
      const double* Ai = A + i * lda;
      const uint64_t sg = s_sgn[wib][rr];
      const int32_t* ci = my_idx + rr * N;
      for (int g = lane; g < ngroups; g += 32) {
        float v[4], sq = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 4 * g + q;
          const double a = j < n ? __ldcs(Ai + j) : (j == n && b ? b[i] : 0.0);
          bad |= !isfinite(a);
          track_exp(a, j < n ? ea : eb);
          const float a32 = to_float_int(a);
          if (j < n) sq = __fmaf_rn(a32, a32, sq);
          v[q] = __fmul_rn(a32, scale);
        }
        {
          float t, e;
          two_sum(fh, sq, t, e);
          fh = t;
          fl = __fadd_rn(fl, e);
        }
        for (int k = 0; k < zeta; ++k) {
          const bool neg = ((sg >> k) & 1ull) == 0ull;
          red_add_v4(yck + (int64_t)ci[k] * ldc + 4 * g, flip_sign_f(v[0], neg), flip_sign_f(v[1], neg),
                     flip_sign_f(v[2], neg), flip_sign_f(v[3], neg));
        }
      }
    }
    __syncwarp();
    // every reduction of this chunk has landed, every block's fold of the
    // previous chunk is done
    if (!grid_sync(bar, status, gridDim.x)) break;
    // the chunk's FP32 sums into the running pairs; its buffer cleared for chunk k+2
    for (int64_t r = blockIdx.x; r < (int64_t)d; r += gridDim.x) {
      float* yc = yck + r * ldc;
      float2* y = Yp + r * ldy;
      for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
        const float2 p = __ldcg(y + c);
        float t, e;
        two_sum(p.x, __ldcg(yc + c), t, e);
        __stcg(y + c, make_float2(t, __fadd_rn(p.y, e)));
        __stcg(yc + c, 0.f);
      }
    }
  }
  if (bad) atomicOr(status, DS_NONFINITE);
  flush_range(ea, eb, range);
  flush_fro((double)fh + (double)fl, fro);
}

// In place: the float pair (hi, lo) of each entry becomes the double hi + lo.
__global__ void k_pairs_to_double(float2* __restrict__ Yp, int64_t count) {
  double* Y = reinterpret_cast<double*>(Yp);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const float2 p = Yp[e];
    Y[e] = (double)p.x + (double)p.y;
  }
}

// FP64 sketch in column slabs: the reductions of one slab of Y (d x w FP64
// entries, at most kSketchSlabBytes) stay in L2 while all of A's rows pass
// over it; A is read once in all (each slab reads its columns of every row).
// At 5e6 x 2000, d = 8000 (Y 128 MB) the sketch took 148.6 ms in one piece,
// 127.4 / 125.5 / 131.2 ms in slabs of 96 / 48 / 24 MB.  (The FP32 chunk-sum
// form keeps one piece: its per-chunk barriers repeat per slab, 89.9 ms
// whole against 91.5 ms in 48 MB slabs.)
constexpr double kSketchSlabBytes = 48e6;

// Columns per slab: a multiple of 32 (whole warps of columns), all when Y fits.
int slab_cols(int64_t d, int ncol, size_t elem) {
  int64_t w = (int64_t)(kSketchSlabBytes / ((double)d * (double)elem)) / 32 * 32;
  if (w < 32) w = 32;
  return w >= ncol ? ncol : (int)w;
}

template <int N>
cudaError_t launch_fold(const double* A, int64_t m, int n, int64_t lda, const double* b, int64_t d, int zeta,
                        uint64_t seed, float* Yc, int64_t ldc, float2* Y, int64_t ldy, uint32_t* status,
                        int32_t* max_rounds, uint32_t* range, double* fro, GridBarrier* bar, int sms,
                        cudaStream_t st) {
  const size_t smem = (size_t)8 * 32 * N * sizeof(int32_t);
  cudaError_t e = cudaFuncSetAttribute(k_sketch_fold<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sketch_fold<N>, 256, smem)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = per_sm * sms;
  const int64_t nw = (int64_t)grid * 8;
  const double rr = (double)kFoldTerms * (double)d / ((double)zeta * (double)nw);
  int R = (int)(rr + 0.5);
  R = R < 1 ? 1 : (R > 32 ? 32 : R);
  float scale = (float)(1.0 / sqrt((double)zeta));
  if ((e = cudaMemsetAsync(&bar->count, 0, sizeof(unsigned int), st)) != cudaSuccess) return e;
  uint64_t dd = (uint64_t)d;
  int64_t mm = m, la = lda, lc = ldc, ly = ldy;
  int nn = n, z = zeta;
  void* args[] = {&A, &mm, &nn, &la, &b, &dd, &z, &seed, &R, &Yc, &lc, &Y, &ly, &scale, &status, &max_rounds,
                  &range, &fro, &bar};
  return cudaLaunchCooperativeKernel((const void*)k_sketch_fold<N>, grid, 256, args, smem, st);
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

// The pairs Yp (row stride ldy) rounded to FP32 into out (row stride ldo):
// fl32(hi + lo), one rounding of the pair's exact sum.
__global__ void k_round_to_float(const float2* __restrict__ Yp, int64_t ldy, float* __restrict__ out, int64_t ldo,
                                 int64_t d, int ncol) {
  for (int64_t r = blockIdx.x; r < d; r += gridDim.x)
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
      const float2 p = Yp[r * ldy + c];
      out[r * ldo + c] = __fadd_rn(p.x, p.y);
    }
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
  const int ncol = n + (b ? 1 : 0);
  const int w = slab_cols(d, ncol, sizeof(TY));
  for (int c0 = 0; blocks > 0 && c0 < ncol; c0 += w) {
    k_sketch_apply<N, TY><<<(unsigned)blocks, 256, smem, st>>>(A, m, n, lda, b, (uint64_t)d, zeta, seed, row0, Y, ldy,
                                                               1.0 / sqrt((double)zeta), status, max_rounds, range,
                                                               fro, c0, std::min(ncol, c0 + w));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_apply_tee(const double* A, int64_t m, int n, int64_t lda, const double* b, int64_t d, int zeta,
                             uint64_t seed, double* Y, int64_t ldy, double* Aout, int64_t ldo, double* bout,
                             uint32_t* status, int32_t* max_rounds, uint32_t* range, double* fro, int sms,
                             cudaStream_t st) {
  const size_t smem = (size_t)8 * 32 * N * sizeof(int32_t);
  cudaError_t e = cudaFuncSetAttribute(k_sketch_apply<N, double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t groups = (m + 255) / 256;
  const int64_t blocks = std::min<int64_t>(groups, (int64_t)sms * 8);
  if (blocks > 0)
    k_sketch_apply<N, double, true><<<(unsigned)blocks, 256, smem, st>>>(
        A, m, n, lda, b, (uint64_t)d, zeta, seed, 0, Y, ldy, 1.0 / sqrt((double)zeta), status, max_rounds, range, fro,
        0, n + 1, Aout, ldo, bout);
  return cudaGetLastError();
}

}  // namespace

cudaError_t sketch_apply_tee(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, int64_t d,
                             int zeta, uint64_t seed, double* Y, int64_t ldy, double* Aout, int64_t ldo, double* bout,
                             uint32_t* status, int32_t* max_rounds, uint32_t* range, double* fro, int sms,
                             cudaStream_t st) {
  const int ni = (int)n;
  if (!b || !bout) return cudaErrorInvalidValue;
  if (zeta <= 8)
    return launch_apply_tee<8>(A, m, ni, lda, b, d, zeta, seed, Y, ldy, Aout, ldo, bout, status, max_rounds, range,
                               fro, sms, st);
  if (zeta <= 16)
    return launch_apply_tee<16>(A, m, ni, lda, b, d, zeta, seed, Y, ldy, Aout, ldo, bout, status, max_rounds, range,
                                fro, sms, st);
  if (zeta <= 32)
    return launch_apply_tee<32>(A, m, ni, lda, b, d, zeta, seed, Y, ldy, Aout, ldo, bout, status, max_rounds, range,
                                fro, sms, st);
  return launch_apply_tee<64>(A, m, ni, lda, b, d, zeta, seed, Y, ldy, Aout, ldo, bout, status, max_rounds, range,
                              fro, sms, st);
}

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

cudaError_t sketch_apply_fold(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, int64_t d,
                              int zeta, uint64_t seed, float* Yc, int64_t ldc, float2* Y, int64_t ldy,
                              uint32_t* status, int32_t* max_rounds, uint32_t* range, double* fro, GridBarrier* bar,
                              int sms, cudaStream_t st) {
  const int ni = (int)n;
  if (ldc % 4 != 0 || (uintptr_t)Yc % 16 != 0) return cudaErrorInvalidValue;
  if (zeta <= 8)
    return launch_fold<8>(A, m, ni, lda, b, d, zeta, seed, Yc, ldc, Y, ldy, status, max_rounds, range, fro, bar, sms,
                          st);
  if (zeta <= 16)
    return launch_fold<16>(A, m, ni, lda, b, d, zeta, seed, Yc, ldc, Y, ldy, status, max_rounds, range, fro, bar,
                           sms, st);
  if (zeta <= 32)
    return launch_fold<32>(A, m, ni, lda, b, d, zeta, seed, Yc, ldc, Y, ldy, status, max_rounds, range, fro, bar,
                           sms, st);
  return launch_fold<64>(A, m, ni, lda, b, d, zeta, seed, Yc, ldc, Y, ldy, status, max_rounds, range, fro, bar, sms,
                         st);
}

cudaError_t round_to_float(const float2* Y, int64_t ldy, float* out, int64_t ldo, int64_t d, int64_t ncol, int sms,
                           cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>(d, (int64_t)sms * 8);
  if (blocks > 0) k_round_to_float<<<(unsigned)blocks, 256, 0, st>>>(Y, ldy, out, ldo, d, (int)ncol);
  return cudaGetLastError();
}

cudaError_t pairs_to_double(float2* Y, int64_t count, int sms, cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>((count + 255) / 256, (int64_t)sms * 8);
  if (blocks > 0) k_pairs_to_double<<<(unsigned)blocks, 256, 0, st>>>(Y, count);
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


}  // namespace lsq
