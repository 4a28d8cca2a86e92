// problem_device.cuh -- Algorithm 1 for one problem, run by a "group" of G
// blocks that share it (G = 1: one block, block barriers; G > 1: blocks of a
// persistent launch that claimed the same problem, group barriers over
// exactly those G blocks).  Used by the batched kernel (G = 1) and the
// serving kernel (any G).
//
//   sketch_group     Y += S [A | b] (Sec. 2.1, Sec. 3.1.2), rows split over
//                    the group, scattered with L2 reductions
//   householder_group  Householder QR of the column-major copy of Y
//                    (Algorithm 1 "QR(Y)"), one group barrier per column
//   precond_group    R, the rank test, M = R^{-1} (Sec. 3.2) and x0 = M z
//   lsqr_shape<S>    LSQR (Algorithm 2) with a lanes-per-row pass shape
#pragma once
#include "lsqr_device.cuh"
#include "sketch.cuh"

namespace lsq {
namespace {

// Sketch columns are drawn into 8 registers: problems here take zeta <= 8.
constexpr int kGroupZeta = 8;

struct Group {
  int gidx, gcount;
  GridBarrier* bar;
  uint32_t* status;
  uint32_t* range;  // [2] exponent maxima of A and b (zeroed by the host), or null
};

__device__ __forceinline__ bool gsync(const Group& g) {
  if (g.gcount == 1) {
    __syncthreads();
    return true;
  }
  return grid_sync(g.bar, g.status, (unsigned int)g.gcount);
}

__device__ __forceinline__ int64_t default_maxit_dev(int n, int d, double tol) {
  const double rate = sqrt((double)n / (double)d);
  if (!(tol > 0.0) || !(rate < 1.0)) return 1000;
  return (int64_t)(10.0 * ceil(log(tol) / log(rate)));
}

// ---------------------------------------------------------------------------
// LSQR pass shapes for small n: (lanes per row L, column pairs per lane P).
// A warp takes 32/L rows per step; L*P*2 >= n.
// ---------------------------------------------------------------------------
constexpr int kShapes = 6;
__host__ __device__ constexpr int shape_L(int s) { return s <= 1 ? 8 : s <= 3 ? 16 : 32; }
__host__ __device__ constexpr int shape_P(int s) { return (s & 1) ? 4 : 2; }
__host__ __device__ constexpr int shape_maxn(int s) { return 2 * shape_L(s) * shape_P(s); }

// Doubles per ring buffer of the chunked pass: chunks of about 4 KB.
constexpr int kChunkDoubles = 512;

// Zero the group's share of `count` doubles.
__device__ __forceinline__ void zero_group(double* p, int64_t count, const Group& g) {
  for (int64_t e = (int64_t)g.gidx * kThreads + threadIdx.x; e < count; e += (int64_t)g.gcount * kThreads) p[e] = 0.0;
}

// Y (d x ldy row-major, zeroed) += S [A | b] for this group's rows.  Warps
// take blocks of 32 rows (block q -> warp q mod (G * kWarps) of the group);
// lane l draws the sketch column of row base+l into shared memory, then the
// warp adds +-A_ij/sqrt(zeta) into the zeta rows of Y (L2 reductions).  The
// largest exponent fields of A's and b's finite entries go to g.range (the
// shifts of the double-float LSQR passes).
__device__ void sketch_group(const double* __restrict__ A, const double* __restrict__ b, int64_t m, int n,
                             int64_t lda, int d, int zeta, uint64_t seed, double* Y, int ldy, int32_t* s_idx,
                             uint64_t* s_sgn, const Group& g) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* my_idx = s_idx + wib * 32 * kGroupZeta;
  const int ncol = n + 1;
  const double scale = 1.0 / sqrt((double)zeta);
  bool bad = false;
  uint32_t ea = 0, eb = 0;
  const int64_t wstep = (int64_t)g.gcount * kWarps * 32;
  for (int64_t base = ((int64_t)g.gidx * kWarps + wib) * 32; base < m; base += wstep) {
    const int64_t row = base + lane;
    if (row < m) {
      int32_t c[kGroupZeta];
      uint64_t signs;
      const int r = sketch_column<kGroupZeta>(seed, (uint64_t)row, (uint64_t)d, zeta, c, signs);
      if (r < 0) atomicOr(g.status, DS_SKETCH);
#pragma unroll
      for (int k = 0; k < kGroupZeta; ++k) my_idx[lane * kGroupZeta + k] = c[k];
      s_sgn[wib * 32 + lane] = signs;
    }
    __syncwarp();
    const int nrows = (int)min((int64_t)32, m - base);
    for (int rr = 0; rr < nrows; ++rr) {
      const int64_t i = base + rr;
      const double* Ai = A + i * lda;
      const uint64_t sg = s_sgn[wib * 32 + rr];
      const int32_t* ci = my_idx + rr * kGroupZeta;
      for (int j = lane; j < ncol; j += 32) {
        const double a = j < n ? __ldcs(Ai + j) : b[i];
        bad |= !isfinite(a);
        const uint32_t e = (uint32_t)__double2hiint(a) & 0x7FF00000u;
        if (e != 0x7FF00000u) {
          if (j < n)
            ea = max(ea, e);
          else
            eb = max(eb, e);
        }
        const double sa = a * scale;
        for (int k = 0; k < zeta; ++k) {
          const double v =
              __longlong_as_double(__double_as_longlong(sa) ^ ((long long)(((sg >> k) & 1ull) == 0ull) << 63));
          atomicAdd(Y + (int64_t)ci[k] * ldy + j, v);
        }
      }
    }
    __syncwarp();
  }
  if (bad) atomicOr(g.status, DS_NONFINITE);
  if (g.range) {
    ea = __reduce_max_sync(0xffffffffu, ea);
    eb = __reduce_max_sync(0xffffffffu, eb);
    if (lane == 0) {
      if (ea) atomicMax(g.range, ea);
      if (eb) atomicMax(g.range + 1, eb);
    }
  }
}

// Householder QR of the d x ncol column-major W.  Step k: every block of the
// group forms ||W[k+1:, k]|| in the same fixed order (same value everywhere)
// and the reflector scalars; the group's warps update columns j > k, one warp
// per column.  Column k is never written in step k, so one group barrier per
// column suffices.  rdiag gets R's diagonal; R[k][j] stays in W[j][k].
// Loads go through L2 (other blocks of the group wrote the columns).
__device__ bool householder_group(double* W, int d, int n, int ncol, double* rdiag, double* scratch,
                                  const Group& g) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = g.gidx * kWarps + wib, nw = g.gcount * kWarps;
  const int kmax = n < d ? n : d;
  for (int k = 0; k < kmax; ++k) {
    if (!gsync(g)) return false;
    const double* wk = W + (int64_t)k * d;
    double part = 0.0;
    for (int i = k + 1 + threadIdx.x; i < d; i += kThreads) part = fma(__ldcg(wk + i), __ldcg(wk + i), part);
    const double sigma = block_sum(part, scratch);
    const double alpha = __ldcg(wk + k);
    double beta = alpha, tau = 0.0, inv_v0 = 0.0;
    if (sigma != 0.0) {
      const double nrm = sqrt(fma(alpha, alpha, sigma));
      beta = alpha >= 0.0 ? -nrm : nrm;
      tau = (beta - alpha) / beta;
      inv_v0 = 1.0 / (alpha - beta);
    }
    if (g.gidx == 0 && threadIdx.x == 0) rdiag[k] = beta;
    if (tau == 0.0) continue;
    for (int j = k + 1 + gw; j < ncol; j += nw) {
      double* wj = W + (int64_t)j * d;
      // 8 loads in flight per lane and 8 partial sums (load-latency bound)
      double s8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      int i = k + 1 + lane;
      for (; i + 7 * 32 < d; i += 8 * 32) {
#pragma unroll
        for (int u = 0; u < 8; ++u) s8[u] = fma(__ldcg(wk + i + 32 * u), __ldcg(wj + i + 32 * u), s8[u]);
      }
      for (; i < d; i += 32) s8[0] = fma(__ldcg(wk + i), __ldcg(wj + i), s8[0]);
      const double s =
          warp_allreduce_sum(((s8[0] + s8[1]) + (s8[2] + s8[3])) + ((s8[4] + s8[5]) + (s8[6] + s8[7])));
      const double f = tau * fma(inv_v0, s, __ldcg(wj + k));
      const double fv = f * inv_v0;
      if (lane == 0) wj[k] = __ldcg(wj + k) - f;
      int i2 = k + 1 + lane;
      for (; i2 + 7 * 32 < d; i2 += 8 * 32) {
        double a[8], w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          a[u] = __ldcg(wk + i2 + 32 * u);
          w[u] = __ldcg(wj + i2 + 32 * u);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) wj[i2 + 32 * u] = fma(-fv, a[u], w[u]);
      }
      for (; i2 < d; i2 += 32) wj[i2] = fma(-fv, __ldcg(wk + i2), __ldcg(wj + i2));
    }
  }
  return gsync(g);
}

// From the factored W: R (n x n row-major), the rank test |R_ii| <= n eps
// max|R_jj| (raises DS_RANK), M = R^{-1} by column-wise back substitution
// (written as rows of Mt, then transposed into M) and x0 = M z with z the
// first n entries of the reflected b column W[n].  Returns false if a group
// barrier gave up.
__device__ bool precond_group(const double* W, int d, int n, const double* rdiag, double* R, double* M, double* Mt,
                              double* x0, double* scratch, const Group& g) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = g.gidx * kWarps + wib, nw = g.gcount * kWarps;
  const int64_t tid = (int64_t)g.gidx * kThreads + threadIdx.x, tstride = (int64_t)g.gcount * kThreads;
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += kThreads) mx = fmax(mx, fabs(__ldcg(rdiag + i)));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) scratch[wib] = mx;
  __syncthreads();
  mx = 0.0;
  for (int w = 0; w < kWarps; ++w) mx = fmax(mx, scratch[w]);
  __syncthreads();
  const double thr = (double)n * 2.220446049250313e-16 * mx;
  for (int64_t e = tid; e < (int64_t)n * n; e += tstride) {
    const int i = (int)(e / n), j = (int)(e % n);
    const double rd = __ldcg(rdiag + i);
    R[e] = j < i ? 0.0 : (j == i ? rd : __ldcg(W + (int64_t)j * d + i));
    if (i == j && !(fabs(rd) > thr)) atomicOr(g.status, DS_RANK);
  }
  if (!gsync(g)) return false;
  for (int c = gw; c < n; c += nw) {  // column c of M as row c of Mt
    double* mc = Mt + (int64_t)c * n;
    for (int i = c + 1 + lane; i < n; i += 32) mc[i] = 0.0;
    if (lane == 0) mc[c] = 1.0 / __ldcg(R + (int64_t)c * n + c);
    __syncwarp();
    for (int i = c - 1; i >= 0; --i) {
      const double* Ri = R + (int64_t)i * n;
      double s = 0.0;
      for (int k = i + 1 + lane; k <= c; k += 32) s = fma(__ldcg(Ri + k), mc[k], s);
      s = warp_allreduce_sum(s);
      if (lane == 0) mc[i] = -s / __ldcg(Ri + i);
      __syncwarp();
    }
  }
  if (!gsync(g)) return false;
  for (int64_t e = tid; e < (int64_t)n * n; e += tstride) {
    const int i = (int)(e / n), k = (int)(e % n);
    M[e] = __ldcg(Mt + (int64_t)k * n + i);
  }
  if (!gsync(g)) return false;
  const double* z = W + (int64_t)n * d;
  for (int i = gw; i < n; i += nw) {
    double s = 0.0;
    for (int k = i + lane; k < n; k += 32) s = fma(__ldcg(M + (int64_t)i * n + k), __ldcg(z + k), s);
    s = warp_allreduce_sum(s);
    if (lane == 0) x0[i] = s;
  }
  return gsync(g);
}

// LSQR with chunked pass shape S: K = ring_k steps of 32/L rows per ring buffer.
template <int S>
__device__ __noinline__ void lsqr_shape(LsqrParams& p, double* ring, uint64_t* bars, double* s_scal, uint32_t& seq,
                           float2* s_w) {
  constexpr int R = 32 / shape_L(S);
  const int kk = kChunkDoubles / (R * (int)p.ldi);
  p.ring_k = kk > 1 ? kk : 1;
  DfPass<shape_L(S), shape_P(S), true> pass{ring, bars, s_scal, seq, s_w};
  lsqr_body(p, pass, s_scal);
  seq = pass.seq;
}

}  // namespace
}  // namespace lsq
