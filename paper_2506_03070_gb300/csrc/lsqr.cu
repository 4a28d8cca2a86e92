// lsqr.cu -- preconditioned LSQR (Algorithm 2) as one persistent cooperative
// kernel, in the one-synchronisation order of App. D.5.1:
//
//   pass over A:  uhat = A wv - (alpha/beta) uhat_prev   (wv = M v, uhat = beta u)
//                 partial sums of ||uhat||^2 and of A^T uhat, while each row is
//                 in registers (one read of A per iteration)
//   barrier; g = sum of per-block partials (fixed order)
//   barrier; beta = ||uhat||; vhat = M^T g / beta - beta v; partial ||vhat||^2
//   barrier; alpha = ||vhat||; Givens scalars; v = vhat / alpha;
//            wv = M v; x += (phi/rho) w; w = wv - (theta/rho) w; stopping test
//   barrier
//
// Every block derives the same scalars from the same partial sums in the same
// order, so all blocks take the same branch at the stopping test.  Modes 3
// and 4 run heavy-ball momentum (Algorithm 6) over the same passes instead.  After the
// loop the same pass structure computes r = b - A x, A^T r and ||A||_F (the
// accuracy check) and the backward-error bounds.
#include "lsqr_device.cuh"

namespace lsq {

namespace {

template <int T, bool VEC>
__global__ void __launch_bounds__(kThreads, 2) k_lsqr_native(LsqrParams p) {
  __shared__ double s_g[kWarps * 64 * T];
  __shared__ double s_scal[kWarps * 4];
  NativePass<T, VEC> pass{s_g, s_scal};
  p.gidx = blockIdx.x;
  p.gcount = gridDim.x;
  if (p.mode >= 3)
    hbm_body(p, pass, s_scal);
  else
    lsqr_body(p, pass, s_scal);
}

template <int T>
__global__ void __launch_bounds__(kThreads, 2) k_lsqr_df(LsqrParams p) {
  extern __shared__ __align__(128) double s_ring[];
  __shared__ __align__(8) uint64_t s_bars[kWarps * kNbuf];
  __shared__ double s_scal[kWarps * 4];
  __shared__ __align__(16) float2 s_w[64 * T];
  if ((threadIdx.x & 31) == 0) {
    for (int b = 0; b < kNbuf; ++b) mbar_init(&s_bars[(threadIdx.x >> 5) * kNbuf + b], 1u);
    fence_proxy_async_smem();
  }
  __syncthreads();
  DfPass<32, T> pass{s_ring, s_bars, s_scal, 0u, s_w};
  p.gidx = blockIdx.x;
  p.gcount = gridDim.x;
  if (p.mode >= 3)
    hbm_body(p, pass, s_scal);
  else
    lsqr_body(p, pass, s_scal);
}

// n > 512: PW warps per row (column panels of at most 512); ring of panel
// slices, then the pass vector as float pairs, in dynamic shared memory.
template <int PW>
__global__ void __launch_bounds__(kThreads, 2) k_lsqr_dfp(LsqrParams p) {
  extern __shared__ __align__(128) double s_ring[];
  __shared__ __align__(8) uint64_t s_bars[kWarps * kNbuf];
  __shared__ __align__(16) double s_scal[kWarps * 6];
  if ((threadIdx.x & 31) == 0) {
    for (int b = 0; b < kNbuf; ++b) mbar_init(&s_bars[(threadIdx.x >> 5) * kNbuf + b], 1u);
    fence_proxy_async_smem();
  }
  __syncthreads();
  float2* s_w = reinterpret_cast<float2*>(s_ring + (size_t)kWarps * kNbuf * 512);
  DfPass<32, 8, false, PW> pass{s_ring, s_bars, s_scal, 0u, s_w};
  p.gidx = blockIdx.x;
  p.gcount = gridDim.x;
  if (p.mode >= 3)
    hbm_body(p, pass, s_scal);
  else
    lsqr_body(p, pass, s_scal);
}

size_t dfp_smem(int n) { return (size_t)kWarps * kNbuf * 512 * sizeof(double) + (size_t)((n + 1) / 2 * 2) * 8; }

template <int PW>
int grid_dfp(int n, int sms) {
  const size_t smem = dfp_smem(n);
  if (cudaFuncSetAttribute(k_lsqr_dfp<PW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lsqr_dfp<PW>, kThreads, smem) != cudaSuccess ||
      per_sm < 1)
    return 0;
  if (per_sm > 2) per_sm = 2;
  return per_sm * sms;
}

template <int PW>
cudaError_t launch_dfp(const LsqrParams& p, int grid, cudaStream_t st) {
  LsqrParams q = p;
  void* args[] = {&q};
  const size_t smem = dfp_smem(p.n);
  cudaError_t e = cudaFuncSetAttribute(k_lsqr_dfp<PW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel((const void*)k_lsqr_dfp<PW>, grid, kThreads, args, smem, st);
}

size_t df_smem(int T, int n) {
  const size_t ring = (size_t)kWarps * kNbuf * (size_t)((n + 1) / 2 * 2) * sizeof(double);  // one row per step
  const size_t red = (size_t)kWarps * 64 * T * sizeof(double);
  return ring > red ? ring : red;
}

template <int T, bool VEC>
int grid_native(int sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lsqr_native<T, VEC>, kThreads, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  if (per_sm > 2) per_sm = 2;
  return per_sm * sms;
}

template <int T>
int grid_df(int n, int sms) {
  const size_t smem = df_smem(T, n);
  if (cudaFuncSetAttribute(k_lsqr_df<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lsqr_df<T>, kThreads, smem) != cudaSuccess ||
      per_sm < 1)
    return 0;
  if (per_sm > 2) per_sm = 2;
  return per_sm * sms;
}

template <int T, bool VEC>
cudaError_t launch_native(const LsqrParams& p, int grid, cudaStream_t st) {
  LsqrParams q = p;
  void* args[] = {&q};
  return cudaLaunchCooperativeKernel((const void*)k_lsqr_native<T, VEC>, grid, kThreads, args, 0, st);
}

template <int T>
cudaError_t launch_df(const LsqrParams& p, int grid, cudaStream_t st) {
  LsqrParams q = p;
  void* args[] = {&q};
  const size_t smem = df_smem(T, p.n);
  cudaError_t e = cudaFuncSetAttribute(k_lsqr_df<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel((const void*)k_lsqr_df<T>, grid, kThreads, args, smem, st);
}

// column pairs per lane of the one-warp-per-row kernels (n <= 512)
int chunks_for(int n) {
  if (n <= 64) return 1;
  if (n <= 128) return 2;
  if (n <= 256) return 4;
  if (n <= 512) return 8;
  return 0;
}
// warps per row of the panel kernel (512 < n <= 4096)
int panels_for(int n) {
  if (n <= 512) return 0;
  if (n <= 1024) return 2;
  if (n <= 2048) return 4;
  if (n <= 4096) return 8;
  return 0;
}

// Self-test kernels of the bounded waits (wait_selftest).  Kind 0: every
// block arrives at one grid barrier that expects gridDim.x + 1 arrivals, so
// the round never fills and every block gives up after the barrier's limit.
// Kind 1: one thread waits on phase 0 of a fresh mbarrier on which nothing
// arrives.  Neither touches memory other than the status word and the
// barrier it was given.
__global__ void k_wait_grid(GridBarrier* bar, uint32_t* status) { grid_sync(bar, status, gridDim.x + 1u); }

__global__ void k_wait_mbar(const GridBarrier* bar, uint32_t* status) {
  __shared__ __align__(8) uint64_t mb;
  if (threadIdx.x == 0) {
    mbar_init(&mb, 1u);
    fence_proxy_async_smem();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_bounded(&mb, 0u, wait_limit_ns(bar))) atomicOr(status, DS_TIMEOUT);
}

}  // namespace

cudaError_t wait_selftest(int kind, GridBarrier* bar, uint32_t* status, int blocks, cudaStream_t st) {
  if (kind == 1) {
    k_wait_mbar<<<1, 32, 0, st>>>(bar, status);
    return cudaGetLastError();
  }
  GridBarrier* b = bar;
  uint32_t* s = status;
  void* args[] = {&b, &s};
  return cudaLaunchCooperativeKernel((const void*)k_wait_grid, blocks, 32, args, 0, st);
}

int lsqr_gparts(int grid) { return grid * kWarps; }

bool lsqr_df_ok(const double* A, int64_t n, int64_t lda) {
  (void)A;
  (void)lda;
  return n >= 1 && n <= kLsqrMaxN;
}

bool lsqr_native_ok(int64_t n) { return n >= 1 && n <= 512; }

int lsqr_grid(int n, bool vec, bool native, int sms) {
  if (!native && n > 512) {
    switch (panels_for(n)) {
      case 2: return grid_dfp<2>(n, sms);
      case 4: return grid_dfp<4>(n, sms);
      case 8: return grid_dfp<8>(n, sms);
      default: return 0;
    }
  }
  if (!native) {
    switch (chunks_for(n)) {
      case 1: return grid_df<1>(n, sms);
      case 2: return grid_df<2>(n, sms);
      case 4: return grid_df<4>(n, sms);
      case 8: return grid_df<8>(n, sms);
      default: return 0;
    }
  }
  switch (chunks_for(n)) {
    case 1: return vec ? grid_native<1, true>(sms) : grid_native<1, false>(sms);
    case 2: return vec ? grid_native<2, true>(sms) : grid_native<2, false>(sms);
    case 4: return vec ? grid_native<4, true>(sms) : grid_native<4, false>(sms);
    case 8: return vec ? grid_native<8, true>(sms) : grid_native<8, false>(sms);
    default: return 0;
  }
}

cudaError_t lsqr_run(const LsqrParams& p, bool vec, bool native, int grid, cudaStream_t st) {
  if (!native && p.n > 512) {
    switch (panels_for(p.n)) {
      case 2: return launch_dfp<2>(p, grid, st);
      case 4: return launch_dfp<4>(p, grid, st);
      case 8: return launch_dfp<8>(p, grid, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (!native) {
    switch (chunks_for(p.n)) {
      case 1: return launch_df<1>(p, grid, st);
      case 2: return launch_df<2>(p, grid, st);
      case 4: return launch_df<4>(p, grid, st);
      case 8: return launch_df<8>(p, grid, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (chunks_for(p.n)) {
    case 1: return vec ? launch_native<1, true>(p, grid, st) : launch_native<1, false>(p, grid, st);
    case 2: return vec ? launch_native<2, true>(p, grid, st) : launch_native<2, false>(p, grid, st);
    case 4: return vec ? launch_native<4, true>(p, grid, st) : launch_native<4, false>(p, grid, st);
    case 8: return vec ? launch_native<8, true>(p, grid, st) : launch_native<8, false>(p, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lsq
