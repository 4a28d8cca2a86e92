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
// LSQR pass: L lanes per row (1, 4 or 32 by the mean row length).  A row's
// lanes stride over its nonzeros for the dot with the pass vector (gathered
// through the read-only path), their sum gives y_i = s A_i . w - gamma u_i,
// and the lanes add y_i a into the
// block's own partial row of A^T y with FP64 L2 reductions (blocks never
// share a partial row); the fixed-order sum over blocks (reduce_g) follows as
// in the dense kernels.  u is FP64.
#include "lsqr_device.cuh"
#include "sketch.cuh"

namespace lsq {
namespace {

// The structure every later kernel indexes by: row_ptr[0] = 0, nondecreasing,
// row_ptr[m] = nnz, and every column index in [0, n).
__global__ void __launch_bounds__(256) k_check_csr(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                   int64_t m, int64_t n, int64_t nnz, uint32_t* status) {
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= m; i += stride) {
    const int64_t r = __ldcs(rp + i);
    if (i == 0) bad |= r != 0;
    if (i == m) bad |= r != nnz;
    if (i < m) bad |= __ldcs(rp + i + 1) < r;
  }
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += stride) {
    const int32_t j = __ldcs(ci + q);
    bad |= j < 0 || (int64_t)j >= n;
  }
  if (bad) atomicOr(status, DS_CSR);
}

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

// A pass over the rows with L lanes per row (32 / L rows per warp at a time):
// few nonzeros per row leave most of a warp idle and a warp's rows latency
// bound one after another, so short rows take one lane each (L = 1), medium
// rows four and long rows the whole warp.  Each lane gathers up to four
// nonzeros at a time so their loads overlap.
template <int L>
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
    constexpr int R = 32 / L;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int sub = lane / L, sl = lane % L;
    const int G = p.gcount, blk = p.gidx;
    p.gparts = G;
    double* gp = p.gpart + (int64_t)blk * p.npad;
    for (int j = threadIdx.x; j < p.n; j += kThreads) gp[j] = 0.0;
    __syncthreads();
    const int64_t r0 = (p.m * blk) / G, r1 = (p.m * (blk + 1)) / G;
    double ss = 0.0, bb = 0.0, fro = 0.0;
    for (int64_t i0 = r0 + (int64_t)wib * R; i0 < r1; i0 += (int64_t)kWarps * R) {
      const int64_t i = i0 + sub;
      const bool live = i < r1;
      int64_t q0 = 0, q1 = 0;
      if (live) {
        q0 = __ldg(rp + i);
        q1 = __ldg(rp + i + 1);
      }
      double dot = 0.0;
      for (int64_t q = q0 + sl; q < q1; q += 4 * L) {
        int32_t c[4];
        double a[4], w[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int64_t qq = q + (int64_t)t * L;
          c[t] = qq < q1 ? __ldg(ci + qq) : -1;
          a[t] = qq < q1 ? __ldg(va + qq) : 0.0;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) w[t] = c[t] >= 0 ? __ldg(wvec + c[t]) : 0.0;
#pragma unroll
        for (int t = 0; t < 4; ++t) dot = fma(a[t], w[t], dot);
      }
#pragma unroll
      for (int o = L / 2; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
      if (live) {
        const double ui = uin[i];
        const double y = fma(-gamma, ui, wsign * dot);
        if (sl == 0) {
          if (uout) uout[i] = y;
          ss = fma(y, y, ss);
          if (UIN2) bb = fma(ui, ui, bb);
        }
        for (int64_t q = q0 + sl; q < q1; q += L) {
          const double a = __ldg(va + q);
          atomicAdd(gp + __ldg(ci + q), y * a);
          if (FRO) fro = fma(a, a, fro);
        }
      }
    }
    ss = warp_allreduce_sum(ss);
    if (UIN2) bb = warp_allreduce_sum(bb);
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

template <int L>
__global__ void __launch_bounds__(kThreads, 2) k_lsqr_csr(LsqrParams p, CsrArgs c) {
  __shared__ double s_scal[kWarps * 4];
  CsrPass<L> pass{c.rp, c.ci, c.va, s_scal};
  p.gidx = blockIdx.x;
  p.gcount = gridDim.x;
  if (p.mode >= 3)
    hbm_body(p, pass, s_scal);
  else
    lsqr_body(p, pass, s_scal);
}

const void* csr_kernel(int lanes) {
  return lanes == 1 ? (const void*)k_lsqr_csr<1> : lanes == 4 ? (const void*)k_lsqr_csr<4> : (const void*)k_lsqr_csr<32>;
}

}  // namespace

cudaError_t check_csr(const int64_t* rp, const int32_t* ci, int64_t m, int64_t n, int64_t nnz, uint32_t* status,
                      int sms, cudaStream_t st) {
  const int64_t work = (m > nnz ? m : nnz) + 1;
  const int blocks = (int)std::min<int64_t>((work + 255) / 256, (int64_t)sms * 8);
  k_check_csr<<<blocks, 256, 0, st>>>(rp, ci, m, n, nnz, status);
  return cudaGetLastError();
}

cudaError_t sketch_csr(const int64_t* rp, const int32_t* ci, const double* va, const double* b, int64_t m, int64_t n,
                       int64_t d, int zeta, uint64_t seed, double* Y, int64_t ldy, uint32_t* status,
                       int32_t* max_rounds, int sms, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((m + 255) / 256, (int64_t)sms * 8);
  k_sketch_csr<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(rp, ci, va, b, m, (int)n, (uint64_t)d, zeta, seed, Y, ldy,
                                                        1.0 / sqrt((double)zeta), status, max_rounds);
  return cudaGetLastError();
}

int csr_lanes(int64_t m, int64_t nnz) {
  const int64_t avg = m > 0 ? nnz / m : 0;
  return avg <= 8 ? 1 : avg <= 48 ? 4 : 32;
}

int lsqr_csr_grid(int sms, int lanes) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, csr_kernel(lanes), kThreads, 0) != cudaSuccess ||
      per_sm < 1)
    return 0;
  return (per_sm > 2 ? 2 : per_sm) * sms;
}

cudaError_t lsqr_csr_run(const LsqrParams& p, const int64_t* rp, const int32_t* ci, const double* va, int grid,
                         int lanes, cudaStream_t st) {
  LsqrParams q = p;
  CsrArgs c{rp, ci, va};
  void* args[] = {&q, &c};
  return cudaLaunchCooperativeKernel(csr_kernel(lanes), grid, kThreads, args, 0, st);
}

}  // namespace lsq
