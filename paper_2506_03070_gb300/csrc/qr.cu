// qr.cu -- preconditioner from the sketch: Householder QR of Y (Algorithm 1
// "Factor Q, R = QR(Y)"), explicit M = R^{-1} (Sec. 3.2) and the
// sketch-and-solve start x0 = M z, z = (Q^T S b)[:n] (Algorithm 1).
//
// The QR runs as one cooperative kernel over a column-major FP64 copy of Y.
// Step k: every block recomputes ||Y[k+1:,k]|| (same order, same result in
// all blocks), builds the reflector scalars, and the grid's warps update the
// trailing columns j > k, one warp per column.  Column k itself is never
// written, so one grid barrier per column suffices; R's diagonal goes to a
// separate array and R[k][j] is left in W[j][k].
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
    tile[r][threadIdx.x] = (i < d && j < ncol) ? Y[i * ldy + j] : (TY)0;
  }
  __syncthreads();
  for (int c = threadIdx.y; c < 32; c += blockDim.y) {
    const int j = j0 + c;
    const int64_t i = i0 + threadIdx.x;
    if (j < ncol && i < d) W[(int64_t)j * d + i] = tile[threadIdx.x][c];
  }
}

// Fixed-order block sum for float or double.
template <typename T>
__device__ __forceinline__ T block_sum_t(T v, T* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  T s = 0;
  for (int i = 0; i < nw; ++i) s += scratch[i];
  __syncthreads();
  return s;
}

// TW = double (plain form) or float (mixed form: FP32 factorisation).
template <typename TW>
__global__ void __launch_bounds__(256) k_householder(TW* __restrict__ W, int64_t d, int n, int ncol,
                                                     double* __restrict__ rdiag, GridBarrier* bar, uint32_t* status) {
  __shared__ TW scratch[32];
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nw = gridDim.x * (blockDim.x >> 5);
  const int kmax = n < d ? n : (int)d;
  for (int k = 0; k < kmax; ++k) {
    if (!grid_sync(bar, status)) return;
    const TW* wk = W + (int64_t)k * d;
    TW part = 0;
    for (int64_t i = k + 1 + threadIdx.x; i < d; i += blockDim.x) part = fma(wk[i], wk[i], part);
    const TW sigma = block_sum_t<TW>(part, scratch);
    const TW alpha = wk[k];
    TW beta = alpha, tau = 0, inv_v0 = 0;
    if (sigma != (TW)0) {
      const TW nrm = sqrt(fma(alpha, alpha, sigma));
      beta = alpha >= (TW)0 ? -nrm : nrm;
      tau = (beta - alpha) / beta;
      inv_v0 = (TW)1 / (alpha - beta);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rdiag[k] = (double)beta;
    if (tau == (TW)0) continue;
    for (int j = k + 1 + gw; j < ncol; j += nw) {
      TW* wj = W + (int64_t)j * d;
      // two partial sums shorten the dependent chain
      TW s0 = 0, s1 = 0;
      int64_t i = k + 1 + lane;
      for (; i + 32 < d; i += 64) {
        s0 = fma(wk[i], wj[i], s0);
        s1 = fma(wk[i + 32], wj[i + 32], s1);
      }
      if (i < d) s0 = fma(wk[i], wj[i], s0);
      TW s = s0 + s1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const TW f = tau * fma(inv_v0, s, wj[k]);
      const TW fv = f * inv_v0;
      if (lane == 0) wj[k] -= f;
      for (int64_t i2 = k + 1 + lane; i2 < d; i2 += 32) wj[i2] = fma(-fv, wk[i2], wj[i2]);
    }
  }
  grid_sync(bar, status);
}

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

// Column c of M = R^{-1} by back substitution, one warp per column, written
// as row c of Mt (contiguous).  R is row-major n x n.
__global__ void __launch_bounds__(256) k_tri_inverse(const double* __restrict__ R, int n,
                                                     double* __restrict__ Mt) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= n) return;
  double* mc = Mt + (int64_t)c * n;
  for (int i = c + 1 + lane; i < n; i += 32) mc[i] = 0.0;
  if (lane == 0) mc[c] = 1.0 / R[(int64_t)c * n + c];
  __syncwarp();
  for (int i = c - 1; i >= 0; --i) {
    // s = sum_{k=i+1..c} R[i][k] M[k][c]
    const double* Ri = R + (int64_t)i * n;
    double s = 0.0;
    for (int k = i + 1 + lane; k <= c; k += 32) s = fma(Ri[k], mc[k], s);
    s = warp_allreduce_sum(s);
    if (lane == 0) mc[i] = -s / Ri[i];
    __syncwarp();
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
  if ((e = cudaMemsetAsync(buf.bar, 0, sizeof(GridBarrier), st)) != cudaSuccess) return e;
  {
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_householder<TY>, 256, 0)) != cudaSuccess)
      return e;
    int blocks = (ncol + 7) / 8;
    blocks = blocks < sms ? blocks : sms;
    if (blocks > per_sm * sms) blocks = per_sm * sms;
    if (blocks < 1) blocks = 1;
    int64_t dd = d;
    int nn = n, nc = ncol;
    double* rd = buf.rdiag;
    GridBarrier* bar = buf.bar;
    uint32_t* status = buf.status;
    void* args[] = {&W, &dd, &nn, &nc, &rd, &bar, &status};
    if ((e = cudaLaunchCooperativeKernel((const void*)k_householder<TY>, blocks, 256, args, 0, st)) != cudaSuccess)
      return e;
  }
  double* Rw = R ? R : buf.R;
  k_extract_r<TY><<<(unsigned)std::min<int64_t>(((int64_t)n * n + 255) / 256, 1024), 256, 0, st>>>(
      W, d, n, buf.rdiag, Rw, nullptr, 0, buf.status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_tri_inverse<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(Rw, n, buf.Mt);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32)), block(32, 8);
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
