// sparse.cu -- sparse A in CSR form: the sketch Y = S [A | b] (Sec. 2.1,
// Sec. 3.1.2; the sketch applied to A's nonzeros only, O(zeta nnz) work as
// the paper notes for sparse sign sketches) and the LSQR passes (Algorithm 2,
// one-sync order of App. D.5.1) over the nonzeros.
//
// Sketch: a warp owns 32 rows at a time; lane l draws the sketch column of
// row base+l in registers (the same sketch_column as the dense path, so the
// sketch of a CSR matrix equals that of its dense form), then the warp walks
// each row's nonzeros and adds +-a/sqrt(zeta) into the zeta rows of Y with L2
// reductions; lane 0 adds the row's b entry into column n.
//
// LSQR pass: one warp per row.  Lanes stride over the row's nonzeros for the
// dot with the pass vector (gathered through the read-only path), the warp
// sum gives y_i = s A_i . w - gamma u_i, and the lanes add y_i a into the
// block's own partial row of A^T y with FP64 L2 reductions (blocks never
// share a partial row); the fixed-order sum over blocks (reduce_g) follows as
// in the dense kernels.  u is FP64.
#include "lsqr_device.cuh"
#include "sketch.cuh"

namespace lsq {
namespace {

__global__ void __launch_bounds__(256) k_sketch_csr(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                    const double* __restrict__ va, const double* __restrict__ b,
                                                    int64_t m, int n, uint64_t d, int zeta, uint64_t seed,
                                                    double* __restrict__ Y, int64_t ldy, double scale,
                                                    uint32_t* status, int32_t* max_rounds) {
  __shared__ int32_t s_idx[8][32][8];
  __shared__ uint64_t s_sgn[8][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  bool bad = false;
  for (int64_t base = ((int64_t)blockIdx.x * 8 + wib) * 32; base < m; base += (int64_t)gridDim.x * 8 * 32) {
    const int64_t row = base + lane;
    if (row < m) {
      int32_t c[8];
      uint64_t signs;
      const int r = sketch_column<8>(seed, (uint64_t)row, d, zeta, c, signs);
      if (r < 0) atomicOr(status, DS_SKETCH);
      if (r > 0) atomicMax(max_rounds, r);
#pragma unroll
      for (int k = 0; k < 8; ++k) s_idx[wib][lane][k] = c[k];
      s_sgn[wib][lane] = signs;
    }
    __syncwarp();
    const int nrows = (int)min((int64_t)32, m - base);
    for (int rr = 0; rr < nrows; ++rr) {
      const int64_t i = base + rr;
      const uint64_t sg = s_sgn[wib][rr];
      const int64_t p0 = __ldg(rp + i), p1 = __ldg(rp + i + 1);
      for (int64_t q = p0 + lane; q < p1 + (b ? 1 : 0); q += 32) {
        double a;
        int64_t j;
        if (q < p1) {
          a = __ldcs(va + q);
          j = __ldcs(ci + q);
        } else {
          a = __ldcs(b + i);
          j = n;
        }
        bad |= !isfinite(a);
        const double sa = a * scale;
        for (int k = 0; k < zeta; ++k) {
          const double v =
              __longlong_as_double(__double_as_longlong(sa) ^ ((long long)(((sg >> k) & 1ull) == 0ull) << 63));
          atomicAdd(Y + (int64_t)s_idx[wib][rr][k] * ldy + j, v);
        }
      }
    }
    __syncwarp();
  }
  if (bad) atomicOr(status, DS_NONFINITE);
}

struct CsrPass {
  const int64_t* rp;
  const int32_t* ci;
  const double* va;
  double* s_scal;

  // y_i = wsign A_i . wvec - gamma uin_i for the block's rows; uout_i = y_i
  // (optional); sums of y^2, uin^2 (UIN2) and A_ij^2 (FRO); A^T y into the
  // block's partial row.
  template <bool UIN2, bool FRO>
  __device__ void run(LsqrParams& p, const double* __restrict__ wvec, double wsign, const double* __restrict__ uin,
                      double gamma, double* __restrict__ uout) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int G = p.gcount, blk = p.gidx;
    p.gparts = G;
    double* gp = p.gpart + (int64_t)blk * p.npad;
    for (int j = threadIdx.x; j < p.n; j += kThreads) gp[j] = 0.0;
    __syncthreads();
    const int64_t r0 = (p.m * blk) / G, r1 = (p.m * (blk + 1)) / G;
    double ss = 0.0, bb = 0.0, fro = 0.0;
    for (int64_t i = r0 + wib; i < r1; i += kWarps) {
      const int64_t q0 = __ldg(rp + i), q1 = __ldg(rp + i + 1);
      double dot = 0.0;
      for (int64_t q = q0 + lane; q < q1; q += 32) dot = fma(__ldg(va + q), __ldg(wvec + __ldg(ci + q)), dot);
      dot = warp_allreduce_sum(dot);
      const double ui = uin[i];
      const double y = fma(-gamma, ui, wsign * dot);
      if (uout && lane == 0) uout[i] = y;
      ss = fma(y, y, ss);
      if (UIN2) bb = fma(ui, ui, bb);
      for (int64_t q = q0 + lane; q < q1; q += 32) {
        const double a = __ldg(va + q);
        atomicAdd(gp + __ldg(ci + q), y * a);
        if (FRO) fro = fma(a, a, fro);
      }
    }
    if (FRO) fro = warp_allreduce_sum(fro);
    if (lane == 0) {
      s_scal[wib * 4 + 0] = ss;
      s_scal[wib * 4 + 1] = bb;
      s_scal[wib * 4 + 2] = fro;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      double s = 0.0;
      for (int w = 0; w < kWarps; ++w) s += s_scal[w * 4 + threadIdx.x];
      p.part[(int64_t)blk * 4 + threadIdx.x] = s;
    }
    __syncthreads();
  }
  __device__ void init(LsqrParams& p) { run<true, false>(p, p.x, -1.0, p.b, -1.0, p.u); }
  __device__ void iter(LsqrParams& p, double gamma) { run<false, false>(p, p.wv, 1.0, p.u, gamma, p.u); }
  __device__ void check(LsqrParams& p) { run<true, true>(p, p.x, -1.0, p.b, -1.0, nullptr); }
  __device__ void residual(LsqrParams& p, bool) { run<true, false>(p, p.x, -1.0, p.b, -1.0, nullptr); }
};

struct CsrArgs {
  const int64_t* rp;
  const int32_t* ci;
  const double* va;
};

__global__ void __launch_bounds__(kThreads, 2) k_lsqr_csr(LsqrParams p, CsrArgs c) {
  __shared__ double s_scal[kWarps * 4];
  CsrPass pass{c.rp, c.ci, c.va, s_scal};
  p.gidx = blockIdx.x;
  p.gcount = gridDim.x;
  if (p.mode >= 3)
    hbm_body(p, pass, s_scal);
  else
    lsqr_body(p, pass, s_scal);
}

}  // namespace

cudaError_t sketch_csr(const int64_t* rp, const int32_t* ci, const double* va, const double* b, int64_t m, int64_t n,
                       int64_t d, int zeta, uint64_t seed, double* Y, int64_t ldy, uint32_t* status,
                       int32_t* max_rounds, int sms, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((m + 255) / 256, (int64_t)sms * 8);
  k_sketch_csr<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(rp, ci, va, b, m, (int)n, (uint64_t)d, zeta, seed, Y, ldy,
                                                        1.0 / sqrt((double)zeta), status, max_rounds);
  return cudaGetLastError();
}

int lsqr_csr_grid(int sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lsqr_csr, kThreads, 0) != cudaSuccess || per_sm < 1)
    return 0;
  return (per_sm > 2 ? 2 : per_sm) * sms;
}

cudaError_t lsqr_csr_run(const LsqrParams& p, const int64_t* rp, const int32_t* ci, const double* va, int grid,
                         cudaStream_t st) {
  LsqrParams q = p;
  CsrArgs c{rp, ci, va};
  void* args[] = {&q, &c};
  return cudaLaunchCooperativeKernel((const void*)k_lsqr_csr, grid, kThreads, args, 0, st);
}

}  // namespace lsq
