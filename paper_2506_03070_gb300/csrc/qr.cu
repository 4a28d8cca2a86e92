// qr.cu -- preconditioner from the sketch: Householder QR of Y (Algorithm 1
// "Factor Q, R = QR(Y)"), explicit M = R^{-1} (Sec. 3.2) and the
// sketch-and-solve start x0 = M z, z = (Q^T S b)[:n] (Algorithm 1).
//
// Two factorisations of the column-major copy W of Y, same reflectors and
// same storage (R's diagonal in a separate array, R[k][j] left in W[j][k]):
//
// Unblocked (sketches whose working copy is below kBlockedMinBytes): one cooperative kernel, one
// block per SM.  Step k: every block recomputes ||Y[k+1:,k]|| (same order, same
// result in all blocks), builds the reflector scalars, and updates its share
// of the trailing columns j > k, two or three at a time.  Column k itself is never
// written, so one grid barrier per column suffices.
//
// Blocked (compact WY, as LAPACK's geqrf/larft/larfb): panels of 64 columns.
// A panel kernel factors the panel with the reflectors of the unblocked
// kernel, touching only the panel's columns (two barriers per column over its
// G blocks, ~256 panel rows each); T of
// Q = H_0 ... H_{b-1} = I - U T U^T comes from the Gram U^T U (larft); the
// trailing columns (and the sketched b column) then take Q^T as
// C <- C - V Z with Z = U^T C and V = U T^T.  The Gram and both large
// products run on the tensor cores (tc_gemm.cu: tcgen05 with TMEM
// accumulators, exact bf16 slicing, FP32 accumulation in TMEM, FP64
// combination): 7 slices per row keep FP64 accuracy in the plain form, 4 keep
// FP32 accuracy in the mixed form.
#include <algorithm>

#include "kernels.h"

namespace lsq {

namespace {

template <typename TY>
__global__ void k_to_colmajor(const TY* __restrict__ Y, int64_t d, int ncol, int64_t ldy, TY* __restrict__ W) {
  // 32x32 tiles through shared memory: read rows of Y, write columns of W.
  __shared__ TY tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = i0 + r;
    const int j = j0 + threadIdx.x;
    TY v = (TY)0;
    if (i < d && j < ncol) v = Y[i * ldy + j];
    tile[r][threadIdx.x] = v;
  }
  __syncthreads();
  for (int c = threadIdx.y; c < 32; c += blockDim.y) {
    const int j = j0 + c;
    const int64_t i = i0 + threadIdx.x;
    if (j < ncol && i < d) W[(int64_t)j * d + i] = tile[threadIdx.x][c];
  }
}

// Fixed-order block sum for float or double (thread 0 adds the per-warp sums
// and shares the total, as block_sum does).
template <typename T>
__device__ __forceinline__ T block_sum_t(T v, T* scratch) {
  __shared__ T s_total;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    T s = 0;
    for (int i = 0; i < nw; ++i) s += scratch[i];
    s_total = s;
  }
  __syncthreads();
  return s_total;
}

// V fixed-order block sums at once, each in block_sum_t's order: lanes v < V
// of warp 0 add the per-warp sums of value v; the totals land in
// scratch[32 V + v] (scratch holds 33 V values) and in a[] of every thread.
template <typename T, int V>
__device__ __forceinline__ void block_sum_multi(T (&a)[V], T* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a[v] += __shfl_xor_sync(0xffffffffu, a[v], o);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int v = 0; v < V; ++v) scratch[v * 32 + wid] = a[v];
  __syncthreads();
  if (threadIdx.x < V) {
    T s = 0;
    for (int i = 0; i < nw; ++i) s += scratch[threadIdx.x * 32 + i];
    scratch[V * 32 + threadIdx.x] = s;
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < V; ++v) a[v] = scratch[V * 32 + v];
}

// TW = double (plain form) or float (mixed form: FP32 factorisation).
// One block per SM; block g owns the trailing columns j = k+1+g, k+1+g+G, ...
// of step k and takes them CB at a time: one loop over the rows loads
// x = W[k+1:, k] and the group's columns and forms ||x||^2 (first group only:
// every block computes it, in the same order, so every block derives the same
// reflector) and the dot products, one block sum reduces them all, thread 0
// forms the reflector and the column scalars and shares them, and a second
// loop applies the reflector.  A step is bound by dependent round trips and
// by the FP64 pipe of the SM that owns the most columns (GB300 retires ~1.6
// FP64 lanes per clock per SM), so the work that is not per row -- the sums
// over warps, sqrt and the divisions -- runs on one lane, not on every
// thread.  Column k is only read in step k: one grid barrier per column.
template <typename TW, int CB>
__global__ void __launch_bounds__(256) k_householder(TW* __restrict__ W, int64_t d, int n, int ncol,
                                                     double* __restrict__ rdiag, GridBarrier* bar, uint32_t* status) {
  __shared__ TW scratch[(CB + 1) * 33];
  __shared__ TW s_sc[CB + 1];  // fv of the group's columns, then tau
  const int kmax = n < d ? n : (int)d;
  const int t = threadIdx.x, G = gridDim.x;
  for (int k = 0; k < kmax; ++k) {
    if (!grid_sync(bar, status)) return;
    const TW* wk = W + (int64_t)k * d;
    const int j0 = k + 1 + blockIdx.x;
    const int nc = j0 < ncol ? (ncol - j0 + G - 1) / G : 0;
    TW tau = 0, inv_v0 = 0;  // thread 0's copy (from the first group) is the one used
    // block 0 writes R's diagonal even when it owns no column
    for (int c0 = 0; c0 < nc || (c0 == 0 && blockIdx.x == 0); c0 += CB) {
      const bool first = c0 == 0;
      const int cn = nc - c0 < CB ? nc - c0 : CB;
      TW acc[CB + 1], wjk[CB];
      TW* wc[CB];
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        acc[c] = 0;
        wc[c] = W + (int64_t)(j0 + G * (c0 + c)) * d;  // dereferenced only for c < cn
        wjk[c] = (c < cn && t == 0) ? wc[c][k] : (TW)0;  // thread 0 rewrites it after the block sum
      }
      acc[CB] = 0;
      for (int64_t i = k + 1 + t; i < d; i += blockDim.x) {
        const TW x = wk[i];
        if (first) acc[CB] = fma(x, x, acc[CB]);
#pragma unroll
        for (int c = 0; c < CB; ++c)
          if (c < cn) acc[c] = fma(x, wc[c][i], acc[c]);
      }
      block_sum_multi<TW, CB + 1>(acc, scratch);
      if (t == 0) {
        if (first) {
          const TW alpha = wk[k];
          const TW sigma = acc[CB];
          TW beta = alpha;
          if (sigma != (TW)0) {
            const TW nrm = sqrt(fma(alpha, alpha, sigma));
            beta = alpha >= (TW)0 ? -nrm : nrm;
            tau = (beta - alpha) / beta;
            inv_v0 = (TW)1 / (alpha - beta);
          }
          if (blockIdx.x == 0) rdiag[k] = (double)beta;
        }
        s_sc[CB] = tau;
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          TW fv = 0;
          if (c < cn && tau != (TW)0) {
            const TW f = tau * fma(inv_v0, acc[c], wjk[c]);
            fv = f * inv_v0;
            wc[c][k] = wjk[c] - f;
          }
          s_sc[c] = fv;
        }
      }
      __syncthreads();
      const TW tau_b = s_sc[CB];
      TW fv[CB];
#pragma unroll
      for (int c = 0; c < CB; ++c) fv[c] = s_sc[c];
      __syncthreads();  // s_sc is rewritten by the next group
      if (tau_b == (TW)0) break;  // H = I: the same in every block
      for (int64_t i = k + 1 + t; i < d; i += blockDim.x) {
        const TW x = wk[i];
#pragma unroll
        for (int c = 0; c < CB; ++c)
          if (c < cn) wc[c][i] = fma(-fv[c], x, wc[c][i]);
      }
    }
  }
  grid_sync(bar, status);
}

// ---------------------------------------------------------------------------
// Blocked Householder QR.
// ---------------------------------------------------------------------------
constexpr int kPanelMax = 64;

template <typename TW>
__device__ __forceinline__ TW warp_sum_t(TW v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Factor the panel P = W[k0:d, k0:k0+b] (L = d - k0 rows, ld = d): for each
// column j, the reflector of the unblocked kernel, applied to the panel's later
// columns only.  Block g of G owns panel rows [L g / G, L (g+1) / G).  Per
// column: (a) partial ||x_{j+1:}||^2 of my rows and partial dots of x_{j+1:}
// with the later columns (both on the columns as the previous reflector left
// them) -> part, the owner of row j publishes row j of the panel -> rowv;
// barrier (the only one of the column); (b) every block sums the partials in
// block order (same scalars everywhere), writes column j of U (unit lower
// trapezoid: 0 above row j, 1 at j, x_i / (alpha - beta) below); (c) every
// block updates its rows of the later columns.  part and rowv alternate by
// column parity: a block reads column j's partials only between barrier j and
// its arrival at barrier j+1, and they are rewritten (column j+2) only after
// barrier j+1.
template <typename TW>
__global__ void __launch_bounds__(256) k_panel(TW* __restrict__ W, int64_t ld, int64_t k0, int64_t L, int b,
                                               TW* __restrict__ U, double* __restrict__ rdiag, TW* __restrict__ tau,
                                               TW* __restrict__ part, TW* __restrict__ rowv, GridBarrier* bar,
                                               uint32_t* status) {
  __shared__ TW scratch[32];
  const int G = gridDim.x, g = blockIdx.x;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int64_t r0 = L * g / G, r1 = L * (g + 1) / G;
  TW* P = W + k0 * ld + k0;
  const int PS = kPanelMax + 2;
  auto sync = [&]() -> bool {
    if (G == 1) {
      __syncthreads();
      return true;
    }
    return grid_sync(bar, status, (unsigned int)G);
  };
  for (int j = 0; j < b; ++j) {
    // the previous step's updates of this block's rows (other warps) come first
    __syncthreads();
    const int par = j & 1;
    const TW* pj = P + (int64_t)j * ld;
    TW* prt = part + (int64_t)par * G * PS;
    TW* rv = rowv + par * kPanelMax;
    const int64_t i0 = r0 > j + 1 ? r0 : (int64_t)j + 1;
    TW s = 0;
    for (int64_t i = i0 + threadIdx.x; i < r1; i += blockDim.x) {
      const TW x = __ldcg(pj + i);
      s = fma(x, x, s);
    }
    s = block_sum_t<TW>(s, scratch);
    if (threadIdx.x == 0) prt[(int64_t)g * PS] = s;
    // dots with the later columns as they are now: same barrier as the norm
    for (int jj = j + 1 + wib; jj < b; jj += nwarps) {
      const TW* pjj = P + (int64_t)jj * ld;
      TW acc = 0;
      for (int64_t i = i0 + lane; i < r1; i += 32) acc = fma(__ldcg(pj + i), __ldcg(pjj + i), acc);
      acc = warp_sum_t<TW>(acc);
      if (lane == 0) prt[(int64_t)g * PS + 1 + jj] = acc;
    }
    if (j >= r0 && j < r1)
      for (int jj = j + threadIdx.x; jj < b; jj += blockDim.x) rv[jj] = __ldcg(P + (int64_t)jj * ld + j);
    if (!sync()) return;
    TW sigma = 0;
    for (int q = 0; q < G; ++q) sigma += __ldcg(prt + (int64_t)q * PS);
    const TW alpha = __ldcg(rv + j);
    TW beta = alpha, t = 0, inv_v0 = 0;
    if (sigma != (TW)0) {
      const TW nrm = sqrt(fma(alpha, alpha, sigma));
      beta = alpha >= (TW)0 ? -nrm : nrm;
      t = (beta - alpha) / beta;
      inv_v0 = (TW)1 / (alpha - beta);
    }
    if (g == 0 && threadIdx.x == 0) {
      rdiag[k0 + j] = (double)beta;
      tau[j] = t;
    }
    TW* uj = U + (int64_t)j * ld;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x)
      uj[i] = i < j ? (TW)0 : (i == j ? (TW)1 : __ldcg(pj + i) * inv_v0);
    if (t == (TW)0) continue;  // same in every block: same barrier count
    for (int jj = j + 1 + wib; jj < b; jj += nwarps) {
      TW S = 0;
      for (int q = 0; q < G; ++q) S += __ldcg(prt + (int64_t)q * PS + 1 + jj);
      const TW wj = __ldcg(rv + jj);
      const TW f = t * fma(inv_v0, S, wj);
      const TW fv = f * inv_v0;
      TW* pjj = P + (int64_t)jj * ld;
      for (int64_t i = i0 + lane; i < r1; i += 32) pjj[i] = fma(-fv, __ldcg(pj + i), __ldcg(pjj + i));
      if (lane == 0 && j >= r0 && j < r1) pjj[j] = wj - f;
    }
  }
}

// The same factorisation with the block's rows of the panel held in shared
// memory (column-major, nr rows per column) for the whole panel: the data
// never leaves the SM between the barriers of the columns, only the
// partial sums (norms, dots) and the published row j go through L2.  Block g
// of G owns panel rows [L g / G, L (g+1) / G) (at most kPanelSmemRows); the
// arithmetic is k_panel's, in the same order.  Writes U (column-major, ld)
// and, at the end, the block's rows of the panel back to W.
constexpr int kPanelSmemRows = 224;  // 224 rows x 64 columns x 8 bytes = 112 KB (FP64)

template <typename TW>
__global__ void __launch_bounds__(256) k_panel_smem(TW* __restrict__ W, int64_t ld, int64_t k0, int64_t L, int b,
                                                    TW* __restrict__ U, double* __restrict__ rdiag,
                                                    TW* __restrict__ tau, TW* __restrict__ part,
                                                    TW* __restrict__ rowv, GridBarrier* bar, uint32_t* status) {
  extern __shared__ __align__(16) unsigned char s_panel_raw[];
  TW* Ps = reinterpret_cast<TW*>(s_panel_raw);  // [b][nrp]
  __shared__ TW scratch[32];
  __shared__ TW s_sc[kPanelMax + 4];  // per-column f * inv_v0, then (tau, inv_v0, beta) of the step
  const int G = gridDim.x, g = blockIdx.x;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int64_t r0 = L * g / G, r1 = L * (g + 1) / G;
  const int nr = (int)(r1 - r0), nrp = nr | 1;  // odd stride: no bank conflicts along a row
  TW* P = W + k0 * ld + k0;
  const int PS = kPanelMax + 2;
  auto sync = [&]() -> bool {
    if (G == 1) {
      __syncthreads();
      return true;
    }
    return grid_sync(bar, status, (unsigned int)G);
  };
  for (int c = 0; c < b; ++c)
    for (int i = threadIdx.x; i < nr; i += blockDim.x) Ps[c * nrp + i] = __ldcg(P + (int64_t)c * ld + r0 + i);
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    const int par = j & 1;
    const TW* pj = Ps + j * nrp;
    TW* prt = part + (int64_t)par * G * PS;
    TW* rv = rowv + par * kPanelMax;
    // own rows strictly below panel row j
    const int i0 = (int)(r0 > j + 1 ? 0 : (int64_t)j + 1 - r0);
    TW sq = 0;
    for (int i = i0 + threadIdx.x; i < nr; i += blockDim.x) sq = fma(pj[i], pj[i], sq);
    sq = block_sum_t<TW>(sq, scratch);
    if (threadIdx.x == 0) prt[(int64_t)g * PS] = sq;
    // the dots of x with the later columns need only the columns as they are
    // now (before this column's reflector), so they go through the same
    // barrier as the norm: one grid barrier per column
    for (int jj = j + 1 + wib; jj < b; jj += nwarps) {
      const TW* pjj = Ps + jj * nrp;
      TW acc = 0;
      for (int i = i0 + lane; i < nr; i += 32) acc = fma(pj[i], pjj[i], acc);
      acc = warp_sum_t<TW>(acc);
      if (lane == 0) prt[(int64_t)g * PS + 1 + jj] = acc;
    }
    if (j >= r0 && j < r1)
      for (int jj = j + threadIdx.x; jj < b; jj += blockDim.x) rv[jj] = Ps[jj * nrp + (j - r0)];
    if (!sync()) return;
    if (threadIdx.x == 0) {
      TW sigma = 0;
      for (int q = 0; q < G; ++q) sigma += __ldcg(prt + (int64_t)q * PS);
      const TW alpha = __ldcg(rv + j);
      TW beta = alpha, t = 0, inv_v0 = 0;
      if (sigma != (TW)0) {
        const TW nrm = sqrt(fma(alpha, alpha, sigma));
        beta = alpha >= (TW)0 ? -nrm : nrm;
        t = (beta - alpha) / beta;
        inv_v0 = (TW)1 / (alpha - beta);
      }
      if (g == 0) {
        rdiag[k0 + j] = (double)beta;
        tau[j] = t;
      }
      s_sc[kPanelMax] = t;
      s_sc[kPanelMax + 1] = inv_v0;
    }
    __syncthreads();
    const TW t = s_sc[kPanelMax], inv_v0 = s_sc[kPanelMax + 1];
    TW* uj = U + (int64_t)j * ld + r0;
    for (int i = threadIdx.x; i < nr; i += blockDim.x) {
      const int64_t gi = r0 + i;
      uj[i] = gi < j ? (TW)0 : (gi == j ? (TW)1 : pj[i] * inv_v0);
    }
    if (t == (TW)0) {
      __syncthreads();
      continue;  // same in every block: same barrier count
    }
    // column scalars, one thread per later column (sums in block order)
    for (int jj = j + 1 + threadIdx.x; jj < b; jj += blockDim.x) {
      TW S = 0;
      for (int q = 0; q < G; ++q) S += __ldcg(prt + (int64_t)q * PS + 1 + jj);
      const TW wj = __ldcg(rv + jj);
      const TW f = t * fma(inv_v0, S, wj);
      s_sc[jj] = f * inv_v0;
      if (j >= r0 && j < r1) Ps[jj * nrp + (j - r0)] = wj - f;
    }
    __syncthreads();
    for (int jj = j + 1 + wib; jj < b; jj += nwarps) {
      const TW fv = s_sc[jj];
      TW* pjj = Ps + jj * nrp;
      for (int i = i0 + lane; i < nr; i += 32) pjj[i] = fma(-fv, pj[i], pjj[i]);
    }
    __syncthreads();
  }
  for (int c = 0; c < b; ++c)
    for (int i = threadIdx.x; i < nr; i += blockDim.x) P[(int64_t)c * ld + r0 + i] = Ps[c * nrp + i];
}

// T (b x b, column-major, upper) of Q = I - U T U^T from the Gram U^T U and
// tau (LAPACK larft, forward, columnwise): T[j][j] = tau_j,
// T[0:j, j] = -tau_j T[0:j, 0:j] (U[:, 0:j]^T u_j).  One block, FP64: row i of
// each column's product is split over four consecutive threads (every fourth
// l from i + q), combined by two shuffles, so its dependent FP64 chain is a
// quarter as long (b <= 64: 256 threads).
template <typename TW>
__global__ void __launch_bounds__(256) k_tform(const double* __restrict__ gram, const TW* __restrict__ tau, int b,
                                               double* __restrict__ T) {
  __shared__ double sT[kPanelMax * kPanelMax];
  __shared__ double w[kPanelMax];
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) sT[e] = 0;
  __syncthreads();
  const int i = threadIdx.x >> 2, q = threadIdx.x & 3;
  for (int j = 0; j < b; ++j) {
    const double tj = (double)tau[j];
    if (threadIdx.x < j) w[threadIdx.x] = gram[threadIdx.x + (int64_t)j * b];
    __syncthreads();
    double s = 0;
    if (i < j)
      for (int l = i + q; l < j; l += 4) s = fma(sT[i + l * b], w[l], s);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (i < j && q == 0) sT[i + j * b] = -tj * s;
    if (threadIdx.x == 0) sT[j + j * b] = tj;
    __syncthreads();
  }
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) T[e] = sT[e];
}

constexpr int kPanelBlocksMax = 64;    // blocks of the global-memory panel kernel
constexpr int kPanelBlocksCap = 320;   // partial-sum slots (the shared-memory kernel may use more blocks)
// Rows per block of the shared-memory panel kernel.  Measured on the 8000 x 2001
// sketch (precond phase): 64 rows per block 88.9 ms, 96 rows 78.6 ms, 192 rows
// 71.4 ms -- more blocks make each grid barrier and the per-column sums over
// the blocks' partials slower than the smaller per-block share saves; fewer,
// larger blocks are slower too (later build: 192 rows 63.4 ms, 256 / 320 / 400
// rows 65.7 / 64.4 / 65.6 ms).
constexpr int kPanelRowsTarget = 192;
constexpr int kSlicesMax = 7;  // bf16 slices per row for FP64 data (3 for FP32)

// bf16 slices per row: 7 (56 bits) for FP64 data; 4 (32 bits) for FP32 data,
// so that entries down to 2^-8 of their row's largest keep FP32's 24 bits
template <typename TW>
constexpr int oz_slices() {
  return sizeof(TW) == 4 ? 4 : 7;
}

// Scratch of the blocked QR for a d x (n+1) sketch (sized for 7 slices).
struct BlockedScratch {
  size_t oU, oGram, oT, oZt, oTau, oPart, oRow, oUs, oCs, oVs, oZs, oEu, oEc, oEv, oEz, bytes;
};
int rows_a(int r) { return r > 128 ? r : 128; }  // slice rows of an A operand (tiles of 128)
int rows_b(int r) { return r > 64 ? r : 64; }    // of a B operand (tiles of 64)
BlockedScratch blocked_layout(int64_t d, int64_t n) {
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  BlockedScratch s;
  size_t o = 0;
  const size_t ncol = (size_t)n + 1;
  const size_t kpd = (size_t)oz_kpad((int)d), kpb = (size_t)oz_kpad(kPanelMax);
  const size_t dr = (size_t)rows_a((int)d), cr = (size_t)rows_a((int)ncol);
  s.oU = o; o += al((size_t)d * kPanelMax * 8);
  s.oGram = o; o += al((size_t)kPanelMax * kPanelMax * 8);
  s.oT = o; o += al((size_t)kPanelMax * kPanelMax * 8);
  s.oZt = o; o += al((size_t)kPanelMax * ncol * 8);
  s.oTau = o; o += al((size_t)kPanelMax * 8);
  s.oPart = o; o += al((size_t)2 * kPanelBlocksCap * (kPanelMax + 2) * 8);
  s.oRow = o; o += al((size_t)2 * kPanelMax * 8);
  s.oUs = o; o += al((size_t)kSlicesMax * 128 * kpd * 2);
  s.oCs = o; o += al((size_t)kSlicesMax * cr * kpd * 2);
  s.oVs = o; o += al((size_t)kSlicesMax * dr * kpb * 2);
  s.oZs = o; o += al((size_t)kSlicesMax * cr * kpb * 2);
  s.oEu = o; o += al((size_t)128 * 4);
  s.oEc = o; o += al(cr * 4);
  s.oEv = o; o += al(dr * 4);
  s.oEz = o; o += al(cr * 4);
  s.bytes = o;
  return s;
}

// K per CTA of a mode-0 GEMM: about two CTAs per SM over the output tiles,
// a multiple of the 128-deep exact accumulation chunk.
int k_split_for(int M, int N, int K, int sms) {
  const int tiles = ((M + 127) / 128) * ((N + 63) / 64);
  int splits = (2 * sms + tiles - 1) / tiles;
  if (splits < 1) splits = 1;
  int ks = (K + splits - 1) / splits;
  ks = (ks + 127) / 128 * 128;
  return ks < 128 ? 128 : ks;
}

// The blocked factorisation of the d x ncol column-major W (first kmax = n
// columns reflected, the rest -- the sketched b column -- transformed).
template <typename TW>
cudaError_t householder_blocked(TW* W, int64_t d, int n, int ncol, double* rdiag, const PrecondBuffers& buf, int sms,
                                cudaStream_t st) {
  const BlockedScratch L0 = blocked_layout(d, n);
  char* s = static_cast<char*>(buf.blk);
  TW* U = reinterpret_cast<TW*>(s + L0.oU);
  double* gram = reinterpret_cast<double*>(s + L0.oGram);
  double* T = reinterpret_cast<double*>(s + L0.oT);
  double* Zt = reinterpret_cast<double*>(s + L0.oZt);
  TW* tau = reinterpret_cast<TW*>(s + L0.oTau);
  TW* part = reinterpret_cast<TW*>(s + L0.oPart);
  TW* rowv = reinterpret_cast<TW*>(s + L0.oRow);
  void* Us = s + L0.oUs;
  void* Cs = s + L0.oCs;
  void* Vs = s + L0.oVs;
  void* Zs = s + L0.oZs;
  int* eU = reinterpret_cast<int*>(s + L0.oEu);
  int* eC = reinterpret_cast<int*>(s + L0.oEc);
  int* eV = reinterpret_cast<int*>(s + L0.oEv);
  int* eZ = reinterpret_cast<int*>(s + L0.oEz);
  constexpr int nb = kPanelMax;
  constexpr int S = oz_slices<TW>();
  const int kmax = n < d ? n : (int)d;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_panel<TW>, 256, 0);
  if (e != cudaSuccess) return e;
  // the shared-memory panel kernel: one block per SM at most, rows <= kPanelSmemRows each
  const int smem_panel = (kPanelSmemRows | 1) * kPanelMax * (int)sizeof(TW);
  int per_sm_s = 0;
  if ((e = cudaFuncSetAttribute(k_panel_smem<TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_panel)) !=
          cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_s, k_panel_smem<TW>, 256, smem_panel)) !=
          cudaSuccess)
    return e;
  for (int k0 = 0; k0 < kmax; k0 += nb) {
    const int b = kmax - k0 < nb ? kmax - k0 : nb;
    const int64_t L = d - k0;
    // the panel's rows spread over blocks (~256 rows each): one block would
    // stream the whole panel from L2 for every column
    int G = (int)std::min<int64_t>((L + 255) / 256, kPanelBlocksMax);
    G = std::min(G, std::max(1, per_sm * sms));
    if (G < 1) G = 1;
    // rows held in shared memory when every block's share fits; about
    // kPanelRowsTarget rows per block (one block per SM at most)
    int Gs = (int)std::max<int64_t>((L + kPanelRowsTarget - 1) / kPanelRowsTarget, 1);
    Gs = std::min(Gs, std::min(std::max(1, per_sm_s * sms), kPanelBlocksCap));
    const bool smem_ok = per_sm_s >= 1 && Gs <= per_sm_s * sms && Gs <= kPanelBlocksCap &&
                         (L + Gs - 1) / Gs <= kPanelSmemRows;
    TW* Wp = W;
    int64_t ld64 = d, k064 = k0, L64 = L;
    int bb = b;
    double* rd = rdiag;
    GridBarrier* bar = buf.bar;
    uint32_t* status = buf.status;
    void* args[] = {&Wp, &ld64, &k064, &L64, &bb, &U, &rd, &tau, &part, &rowv, &bar, &status};
    // the ticket barrier's counter restarts for each launch (G changes with L)
    const int GL = smem_ok ? Gs : G;
    if (GL > 1 && (e = cudaMemsetAsync(&buf.bar->count, 0, sizeof(unsigned int), st)) != cudaSuccess) return e;
    if (smem_ok)
      e = GL == 1 ? cudaLaunchKernel((const void*)k_panel_smem<TW>, 1, 256, args, smem_panel, st)
                  : cudaLaunchCooperativeKernel((const void*)k_panel_smem<TW>, GL, 256, args, smem_panel, st);
    else if (G == 1)
      e = cudaLaunchKernel((const void*)k_panel<TW>, 1, 256, args, 0, st);
    else
      e = cudaLaunchCooperativeKernel((const void*)k_panel<TW>, G, 256, args, 0, st);
    if (e != cudaSuccess) return e;
    const int c = ncol - k0 - b;
    if (c <= 0) continue;
    const int Li = (int)L;
    const int kpl = oz_kpad(Li), kpb = oz_kpad(b);
    // slices of U's b columns (rows of U^T, length L): B operand of Z^T = C^T U
    // and both operands of the Gram U^T U
    if ((e = oz_slice<TW>(U, b, Li, d, nullptr, S, Us, kpl, eU, 128, sms, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(gram, 0, sizeof(double) * b * b, st)) != cudaSuccess) return e;
    OzGemm g;
    g.S = S;
    g.status = buf.status;
    g.bar = buf.bar;
    g.a = Us;
    g.b = Us;
    g.M = b;
    g.N = b;
    g.K = Li;
    g.Kpad = kpl;
    g.a_rows = 128;
    g.b_rows = 128;
    g.ea = eU;
    g.eb = eU;
    g.mode = 0;
    g.out_f32 = 0;
    g.out = gram;
    g.ldo = b;
    g.k_split = k_split_for(b, b, Li, sms);
    if ((e = oz_gemm(g, st)) != cudaSuccess) return e;
    k_tform<TW><<<1, 256, 0, st>>>(gram, tau, b, T);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // Z^T = C^T U (c x b): A operand = C's columns (length L)
    TW* C = W + (int64_t)(k0 + b) * d + k0;
    const int cr = rows_a(c);
    if ((e = oz_slice<TW>(C, c, Li, d, nullptr, S, Cs, kpl, eC, cr, sms, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(Zt, 0, sizeof(double) * (size_t)c * b, st)) != cudaSuccess) return e;
    g.a = Cs;
    g.b = Us;
    g.M = c;
    g.N = b;
    g.a_rows = cr;
    g.b_rows = 128;
    g.ea = eC;
    g.eb = eU;
    g.out = Zt;
    g.ldo = b;
    g.k_split = k_split_for(c, b, Li, sms);
    if ((e = oz_gemm(g, st)) != cudaSuccess) return e;
    // C <- C - V Z, V = U T^T (L x b), Z = (Z^T)^T: A operand = rows of V, B = rows of Z^T
    const int lr = rows_a(Li), zr = rows_b(c);
    if ((e = oz_slice<TW>(U, Li, b, d, T, S, Vs, kpb, eV, lr, sms, st)) != cudaSuccess) return e;
    if ((e = oz_slice<double>(Zt, c, b, b, nullptr, S, Zs, kpb, eZ, zr, sms, st)) != cudaSuccess) return e;
    g.a = Vs;
    g.b = Zs;
    g.M = Li;
    g.N = c;
    g.K = b;
    g.Kpad = kpb;
    g.a_rows = lr;
    g.b_rows = zr;
    g.ea = eV;
    g.eb = eZ;
    g.mode = 1;
    g.out_f32 = sizeof(TW) == 4;
    g.out = C;
    g.ldo = d;
    if ((e = oz_gemm(g, st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Automatic choice: the blocked path once the working copy W reaches 32 MiB
// (in its own precision), the unblocked kernel's single barrier per column
// below.  Measured precond times, unblocked vs blocked (ms, FP64 / FP32):
// 800 x 201 1.7 vs 4.1 / 1.1 vs 3.0; 2000 x 501 6.6 vs 11.0 / 4.2 vs 8.2;
// 4000 x 1001 26.2 vs 26.5 / 17.4 vs 19.8; 9450 x 501 21.9 vs 17.3 / 12.0 vs 13.4;
// 6000 x 1501 74 vs 52 / 49 vs 38; 8000 x 2001 191 vs 83 / 102 vs 62;
// 16000 x 2001 477 vs 129 / 331 vs 95.
constexpr size_t kBlockedMinBytes = (size_t)32 << 20;

// R (row-major n x n, upper), z = W[n][0:n] (x0 slot), and the rank test
// |R_kk| <= n * eps * max_i |R_ii|.
template <typename TW>
__global__ void k_extract_r(const TW* __restrict__ W, int64_t d, int n, const double* __restrict__ rdiag,
                            double* __restrict__ R, double* __restrict__ z, int has_b, uint32_t* status) {
  __shared__ double scratch[32];
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, fabs(rdiag[i]));
  // block max via the sum helper's layout
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncthreads();
    if (lane == 0) scratch[wid] = mx;
    __syncthreads();
    mx = 0.0;
    for (int i = 0; i < nw; ++i) mx = fmax(mx, scratch[i]);
    (void)lane;
  }
  const double thr = (double)n * 2.220446049250313e-16 * mx;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (!(fabs(rdiag[i]) > thr)) atomicOr(status, DS_RANK);
  if (R) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)n * n;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int i = (int)(e / n), j = (int)(e % n);
      R[e] = j < i ? 0.0 : (j == i ? rdiag[i] : (double)W[(int64_t)j * d + i]);
    }
  }
  if (has_b && z && blockIdx.x == 0)
    for (int i = threadIdx.x; i < n; i += blockDim.x) z[i] = (double)W[(int64_t)n * d + i];
}

// Column c of M = R^{-1}, written as row c of Mt (contiguous), by
// column-oriented back substitution in one block: m_c = 1 / R_cc; then for
// k = c, c-1, ..., 1 every row i < k takes p_i += R_ik m_k (column k of R,
// contiguous in Rt = R^T) and the thread that owns row k-1 finishes
// m_{k-1} = -p_{k-1} / R_{k-1,k-1}, published for the next step through a
// two-slot shared word (one block barrier per step).  The partial sums p stay
// in shared memory, so R is read once per column of M and no step waits on a
// reduction across threads.  Blocks take the longest columns first.
__global__ void __launch_bounds__(256) k_tri_inverse(const double* __restrict__ Rt, int n,
                                                     double* __restrict__ Mt) {
  extern __shared__ double s_p[];  // [n]
  __shared__ double s_m[2];
  const int c = n - 1 - (int)blockIdx.x;
  double* mc = Mt + (int64_t)c * n;
  for (int i = threadIdx.x; i < c; i += blockDim.x) s_p[i] = 0.0;
  for (int i = c + 1 + threadIdx.x; i < n; i += blockDim.x) mc[i] = 0.0;
  if (threadIdx.x == 0) {
    const double m = 1.0 / Rt[(int64_t)c * n + c];
    s_m[c & 1] = m;
    mc[c] = m;
  }
  __syncthreads();
  for (int k = c; k > 0; --k) {
    const double mk = s_m[k & 1];
    const double* col = Rt + (int64_t)k * n;
    for (int i = threadIdx.x; i < k; i += blockDim.x) s_p[i] = fma(col[i], mk, s_p[i]);
    if (threadIdx.x == (k - 1) % (int)blockDim.x) {  // owner of row k-1: its update is done
      const double m = -s_p[k - 1] / Rt[(int64_t)(k - 1) * n + (k - 1)];
      s_m[(k - 1) & 1] = m;
      mc[k - 1] = m;
    }
    __syncthreads();
  }
}

__global__ void k_transpose(const double* __restrict__ Mt, int n, double* __restrict__ M) {
  __shared__ double tile[32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, j = j0 + threadIdx.x;
    tile[r][threadIdx.x] = (i < n && j < n) ? Mt[(int64_t)i * n + j] : 0.0;
  }
  __syncthreads();
  for (int c = threadIdx.y; c < 32; c += blockDim.y) {
    const int j = j0 + c, i = i0 + threadIdx.x;
    if (i < n && j < n) M[(int64_t)j * n + i] = tile[threadIdx.x][c];
  }
}

// x0 = M z, one warp per row.
template <typename TZ>
__global__ void k_matvec_upper(const double* __restrict__ M, int n, const TZ* __restrict__ z,
                               double* __restrict__ x) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  double s = 0.0;
  for (int k = i + lane; k < n; k += 32) s = fma(M[(int64_t)i * n + k], (double)z[k], s);
  s = warp_allreduce_sum(s);
  if (lane == 0) x[i] = s;
}

}  // namespace

size_t precond_blocked_bytes(int64_t d, int64_t n) { return blocked_layout(d, n).bytes; }

cudaError_t transpose_square(const double* src, int n, double* dst, cudaStream_t st) {
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32)), block(32, 8);
  k_transpose<<<grid, block, 0, st>>>(src, n, dst);
  return cudaGetLastError();
}

template <typename TY>
cudaError_t precond(const TY* Y, int64_t d, int64_t n64, int64_t ldy, int has_b, double* R, double* M, double* x0,
                    const PrecondBuffers& buf, int sms, cudaStream_t st) {
  const int n = (int)n64;
  const int ncol = n + (has_b ? 1 : 0);
  TY* W = reinterpret_cast<TY*>(buf.W);
  cudaError_t e;
  {
    dim3 grid((unsigned)((d + 31) / 32), (unsigned)((ncol + 31) / 32)), block(32, 8);
    k_to_colmajor<TY><<<grid, block, 0, st>>>(Y, d, ncol, ldy, W);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = cudaMemsetAsync(&buf.bar->count, 0, sizeof(unsigned int), st)) != cudaSuccess) return e;
  const bool big = (size_t)d * ncol * sizeof(TY) >= kBlockedMinBytes;
  const bool blocked = buf.mode == 2 || (buf.mode == 0 && big);
  if (buf.blk && blocked && (size_t)kPanelMax * ncol <= ((size_t)1 << 31)) {
    if ((e = householder_blocked<TY>(W, d, n, ncol, buf.rdiag, buf, sms, st)) != cudaSuccess) return e;
  } else {
    // one block per SM (at most one per trailing column); three columns per
    // group once a block owns more than two (measured: 2000 x 501 5.3 vs 5.7
    // ms, 4000 x 1001 21 vs 23 ms; 800 x 201 1.35 ms with two)
    int blocks = ncol - 1 < sms ? ncol - 1 : sms;
    if (blocks < 1) blocks = 1;
    const void* fn = ncol - 1 > 2 * blocks ? (const void*)k_householder<TY, 3> : (const void*)k_householder<TY, 2>;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    int64_t dd = d;
    int nn = n, nc = ncol;
    double* rd = buf.rdiag;
    GridBarrier* bar = buf.bar;
    uint32_t* status = buf.status;
    void* args[] = {&W, &dd, &nn, &nc, &rd, &bar, &status};
    if ((e = cudaLaunchCooperativeKernel(fn, blocks, 256, args, 0, st)) != cudaSuccess) return e;
  }
  double* Rw = R ? R : buf.R;
  k_extract_r<TY><<<(unsigned)std::min<int64_t>(((int64_t)n * n + 255) / 256, 1024), 256, 0, st>>>(
      W, d, n, buf.rdiag, Rw, nullptr, 0, buf.status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    // R^T into M's memory (the inverse reads columns of R), then Mt = rows of
    // M = columns of R^{-1}, then M = Mt^T over R^T
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32)), block(32, 8);
    k_transpose<<<grid, block, 0, st>>>(Rw, n, M);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem = (size_t)n * sizeof(double);
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k_tri_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
      return e;
    k_tri_inverse<<<(unsigned)n, 256, smem, st>>>(M, n, buf.Mt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_transpose<<<grid, block, 0, st>>>(buf.Mt, n, M);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (has_b && x0) {
    // z = W[n][0:n] (the last column after all reflections) is read in place; x0 = M z
    k_matvec_upper<TY><<<(unsigned)((n + 7) / 8), 256, 0, st>>>(M, n, W + (int64_t)n * d, x0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template cudaError_t precond<double>(const double*, int64_t, int64_t, int64_t, int, double*, double*, double*,
                                     const PrecondBuffers&, int, cudaStream_t);
template cudaError_t precond<float>(const float*, int64_t, int64_t, int64_t, int, double*, double*, double*,
                                    const PrecondBuffers&, int, cudaStream_t);

}  // namespace lsq
