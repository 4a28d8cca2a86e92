// lsqr_rows.cu -- the double-float LSQR kernels for n <= 512 (one warp per row); see lsqr.cu for the iteration.
#include "lsqr_device.cuh"

namespace lsq {

namespace {

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

size_t df_smem(int T, int n) {
  const size_t ring = (size_t)kWarps * kNbuf * (size_t)((n + 1) / 2 * 2) * sizeof(double);  // one row per step
  const size_t red = (size_t)kWarps * 64 * T * sizeof(double);
  return ring > red ? ring : red;
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

template <int T>
cudaError_t launch_df(const LsqrParams& p, int grid, cudaStream_t st) {
  LsqrParams q = p;
  void* args[] = {&q};
  const size_t smem = df_smem(T, p.n);
  cudaError_t e = cudaFuncSetAttribute(k_lsqr_df<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel((const void*)k_lsqr_df<T>, grid, kThreads, args, smem, st);
}

}  // namespace

int lsqr_rows_grid(int chunks, int n, int sms) {
  switch (chunks) {
    case 1: return grid_df<1>(n, sms);
    case 2: return grid_df<2>(n, sms);
    case 4: return grid_df<4>(n, sms);
    case 8: return grid_df<8>(n, sms);
    default: return 0;
  }
}

cudaError_t lsqr_rows_run(int chunks, const LsqrParams& p, int grid, cudaStream_t st) {
  switch (chunks) {
    case 1: return launch_df<1>(p, grid, st);
    case 2: return launch_df<2>(p, grid, st);
    case 4: return launch_df<4>(p, grid, st);
    case 8: return launch_df<8>(p, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lsq
