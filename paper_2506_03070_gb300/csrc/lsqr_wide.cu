// lsqr_wide.cu -- the double-float LSQR kernels for 512 < n <= 4096 (PW warps per row); see lsqr.cu for the iteration.
#include "lsqr_device.cuh"

namespace lsq {

namespace {

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

// ring, then the pass vector (8 bytes per column of the image's row)
size_t dfp_smem(int n, int pw) {
  (void)pw;
  return (size_t)kWarps * kNbuf * 512 * sizeof(double) + (size_t)((n + 1) / 2 * 2) * 8;
}

template <int PW>
int grid_dfp(int n, int sms) {
  const size_t smem = dfp_smem(n, PW);
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
  const size_t smem = dfp_smem(p.n, PW);
  cudaError_t e = cudaFuncSetAttribute(k_lsqr_dfp<PW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel((const void*)k_lsqr_dfp<PW>, grid, kThreads, args, smem, st);
}

}  // namespace

int lsqr_wide_grid(int panels, int n, int sms) {
  switch (panels) {
    case 2: return grid_dfp<2>(n, sms);
    case 4: return grid_dfp<4>(n, sms);
    case 8: return grid_dfp<8>(n, sms);
    default: return 0;
  }
}

cudaError_t lsqr_wide_run(int panels, const LsqrParams& p, int grid, cudaStream_t st) {
  switch (panels) {
    case 2: return launch_dfp<2>(p, grid, st);
    case 4: return launch_dfp<4>(p, grid, st);
    case 8: return launch_dfp<8>(p, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lsq
