// lsqr_native.cu -- the native-FP64 LSQR kernels (LSQ_FLAG_NATIVE_FP64): one warp per row for n <= 512, column
// panels of PW warps per row up to n = 4096; see lsqr.cu for the iteration.
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

template <int T, bool VEC>
int grid_native(int sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lsqr_native<T, VEC>, kThreads, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  if (per_sm > 2) per_sm = 2;
  return per_sm * sms;
}

template <int T, bool VEC>
cudaError_t launch_native(const LsqrParams& p, int grid, cudaStream_t st) {
  LsqrParams q = p;
  void* args[] = {&q};
  return cudaLaunchCooperativeKernel((const void*)k_lsqr_native<T, VEC>, grid, kThreads, args, 0, st);
}

// n > 512 (LSQ_FLAG_NATIVE_FP64): PW warps per row in column panels, every
// pass in FP64 (NativePanelPass); no ring, rows are read directly.
template <int PW>
__global__ void __launch_bounds__(kThreads, 2) k_lsqr_native_wide(LsqrParams p) {
  __shared__ __align__(16) double s_scal[kWarps * 6];
  NativePanelPass<PW> pass{s_scal};
  p.gidx = blockIdx.x;
  p.gcount = gridDim.x;
  if (p.mode >= 3)
    hbm_body(p, pass, s_scal);
  else
    lsqr_body(p, pass, s_scal);
}

template <int PW>
int grid_native_wide(int sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lsqr_native_wide<PW>, kThreads, 0) != cudaSuccess ||
      per_sm < 1)
    return 0;
  if (per_sm > 2) per_sm = 2;
  return per_sm * sms;
}

template <int PW>
cudaError_t launch_native_wide(const LsqrParams& p, int grid, cudaStream_t st) {
  LsqrParams q = p;
  void* args[] = {&q};
  return cudaLaunchCooperativeKernel((const void*)k_lsqr_native_wide<PW>, grid, kThreads, args, 0, st);
}

}  // namespace

int lsqr_native_wide_grid(int panels, int sms) {
  switch (panels) {
    case 2: return grid_native_wide<2>(sms);
    case 4: return grid_native_wide<4>(sms);
    case 8: return grid_native_wide<8>(sms);
    default: return 0;
  }
}

cudaError_t lsqr_native_wide_run(int panels, const LsqrParams& p, int grid, cudaStream_t st) {
  switch (panels) {
    case 2: return launch_native_wide<2>(p, grid, st);
    case 4: return launch_native_wide<4>(p, grid, st);
    case 8: return launch_native_wide<8>(p, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

int lsqr_native_grid(int chunks, bool vec, int sms) {
  switch (chunks) {
    case 1: return vec ? grid_native<1, true>(sms) : grid_native<1, false>(sms);
    case 2: return vec ? grid_native<2, true>(sms) : grid_native<2, false>(sms);
    case 4: return vec ? grid_native<4, true>(sms) : grid_native<4, false>(sms);
    case 8: return vec ? grid_native<8, true>(sms) : grid_native<8, false>(sms);
    default: return 0;
  }
}

cudaError_t lsqr_native_run(int chunks, bool vec, const LsqrParams& p, int grid, cudaStream_t st) {
  switch (chunks) {
    case 1: return vec ? launch_native<1, true>(p, grid, st) : launch_native<1, false>(p, grid, st);
    case 2: return vec ? launch_native<2, true>(p, grid, st) : launch_native<2, false>(p, grid, st);
    case 4: return vec ? launch_native<4, true>(p, grid, st) : launch_native<4, false>(p, grid, st);
    case 8: return vec ? launch_native<8, true>(p, grid, st) : launch_native<8, false>(p, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lsq
