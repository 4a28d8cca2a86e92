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
// The kernels are instantiated in lsqr_rows.cu (double-float, n <= 512),
// lsqr_wide.cu (double-float, 512 < n <= 4096) and lsqr_native.cu (native
// FP64: one warp per row for n <= 512, column panels up to 4096); this file
// dispatches to them and holds the wait self-tests.
#include "lsqr_device.cuh"

namespace lsq {

namespace {

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
  if (native && n > 512) return lsqr_native_wide_grid(panels_for(n), sms);
  if (!native && n > 512) {
    return lsqr_wide_grid(panels_for(n), n, sms);
  }
  if (!native) {
    return lsqr_rows_grid(chunks_for(n), n, sms);
  }
  return lsqr_native_grid(chunks_for(n), vec, sms);
}

cudaError_t lsqr_run(const LsqrParams& p, bool vec, bool native, int grid, cudaStream_t st) {
  if (native && p.n > 512) return lsqr_native_wide_run(panels_for(p.n), p, grid, st);
  if (!native && p.n > 512) {
    return lsqr_wide_run(panels_for(p.n), p, grid, st);
  }
  if (!native) {
    return lsqr_rows_run(chunks_for(p.n), p, grid, st);
  }
  return lsqr_native_run(chunks_for(p.n), vec, p, grid, st);
}

}  // namespace lsq
