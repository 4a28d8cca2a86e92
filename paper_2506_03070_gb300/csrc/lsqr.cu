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
// order, so all blocks take the same branch at the stopping test.  After the
// loop the same pass structure computes r = b - A x, A^T r and ||A||_F (the
// accuracy check) and the backward-error bounds.
#include "kernels.h"

namespace lsq {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;

// --------------------------------------------------------------------------
// The pass over A.  Block `blk` owns rows [m*blk/G, m*(blk+1)/G); its warp k
// takes rows start+k, start+k+8, ...  Lane l holds columns 2l+64t, 2l+64t+1
// (t < T) of the current row and of the vector wvec.  For each row:
//   y_i = wsign * (A_i . wvec) - gamma * uin_i;  uout_i = y_i (optional)
//   sum y_i^2, sum uin_i^2 (optional), sum A_ij^2 (optional), g += y_i A_i
// Per-block results: gpart[blk][0..n), part[blk][slot...].
// --------------------------------------------------------------------------
template <int T, bool VEC, bool FRO, bool UIN2>
__device__ void pass_native(const LsqrParams& p, const double* __restrict__ wvec, double wsign,
                            const double* __restrict__ uin, double gamma, double* __restrict__ uout, double* s_g,
                            double* s_scal) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int G = gridDim.x, blk = blockIdx.x;
  const int n = p.n;
  const int64_t r0 = (p.m * blk) / G, r1 = (p.m * (blk + 1)) / G;
  double wr[2 * T], g[2 * T];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int j = 2 * lane + 64 * t;
    wr[2 * t] = j < n ? wsign * wvec[j] : 0.0;
    wr[2 * t + 1] = j + 1 < n ? wsign * wvec[j + 1] : 0.0;
    g[2 * t] = g[2 * t + 1] = 0.0;
  }
  double ss = 0.0, bb = 0.0, fro = 0.0;
  for (int64_t i = r0 + wib; i < r1; i += kWarps) {
    const double* Ai = p.A + i * p.lda;
    double2 a[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const int j = 2 * lane + 64 * t;
      if (j + 1 < n) {
        if (VEC) {
          a[t] = __ldcs(reinterpret_cast<const double2*>(Ai + j));
        } else {
          a[t].x = __ldcs(Ai + j);
          a[t].y = __ldcs(Ai + j + 1);
        }
      } else if (j < n) {
        a[t].x = __ldcs(Ai + j);
        a[t].y = 0.0;
      } else {
        a[t].x = a[t].y = 0.0;
      }
    }
    double dot = 0.0;
#pragma unroll
    for (int t = 0; t < T; ++t) {
      dot = fma(a[t].x, wr[2 * t], dot);
      dot = fma(a[t].y, wr[2 * t + 1], dot);
    }
    dot = warp_allreduce_sum(dot);
    const double ui = uin[i];
    const double y = fma(-gamma, ui, dot);
    if (uout && lane == 0) uout[i] = y;
    ss = fma(y, y, ss);
    if (UIN2) bb = fma(ui, ui, bb);
#pragma unroll
    for (int t = 0; t < T; ++t) {
      g[2 * t] = fma(y, a[t].x, g[2 * t]);
      g[2 * t + 1] = fma(y, a[t].y, g[2 * t + 1]);
      if (FRO) {
        fro = fma(a[t].x, a[t].x, fro);
        fro = fma(a[t].y, a[t].y, fro);
      }
    }
  }
  // block reduction of g (warp order), ss, bb, fro
  double* sg = s_g + wib * (64 * T);
#pragma unroll
  for (int t = 0; t < T; ++t) {
    sg[2 * lane + 64 * t] = g[2 * t];
    sg[2 * lane + 64 * t + 1] = g[2 * t + 1];
  }
  if (FRO) fro = warp_allreduce_sum(fro);
  if (lane == 0) {
    s_scal[wib * 4 + 0] = ss;
    s_scal[wib * 4 + 1] = bb;
    s_scal[wib * 4 + 2] = fro;
  }
  __syncthreads();
  double* gp = p.gpart + (int64_t)blk * p.npad;
  for (int j = threadIdx.x; j < n; j += kThreads) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += s_g[w * (64 * T) + j];
    gp[j] = s;
  }
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += s_scal[w * 4 + threadIdx.x];
    p.part[(int64_t)blk * 4 + threadIdx.x] = s;
  }
  __syncthreads();
}

// g[j] = sum over blocks of gpart[blk][j], block order.
__device__ void reduce_g(const LsqrParams& p) {
  const int G = gridDim.x;
  for (int j = blockIdx.x * kThreads + threadIdx.x; j < p.n; j += G * kThreads) {
    double s = 0.0;
    for (int c = 0; c < G; ++c) s += p.gpart[(int64_t)c * p.npad + j];
    p.g[j] = s;
  }
}

// sum over blocks of part[blk][slot], block order (same value in every thread).
__device__ __forceinline__ double sum_part(const LsqrParams& p, int slot) {
  double s = 0.0;
  for (int c = 0; c < (int)gridDim.x; ++c) s += p.part[(int64_t)c * 4 + slot];
  return s;
}

// vhat_k = (M^T g)_k * ginv - cv * v_k, one warp per k; per-block sum of
// vhat_k^2 into part[blk][slot].  M^T g uses rows of Mt (contiguous).
__device__ void mt_apply(const LsqrParams& p, double ginv, double cv, int slot, double* s_scal) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = blockIdx.x * kWarps + wib, nw = gridDim.x * kWarps;
  double acc = 0.0;
  for (int k = gw; k < p.n; k += nw) {
    const double* mk = p.Mt + (int64_t)k * p.n;
    double s = 0.0;
    for (int i = lane; i <= k; i += 32) s = fma(mk[i], p.g[i], s);
    s = warp_allreduce_sum(s);
    const double vh = cv != 0.0 ? fma(s, ginv, -cv * p.v[k]) : s * ginv;
    if (lane == 0) p.vhat[k] = vh;
    acc = fma(vh, vh, acc);
  }
  if (lane == 0) s_scal[wib] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += s_scal[w];
    p.part[(int64_t)blockIdx.x * 4 + slot] = s;
  }
  __syncthreads();
}

// v = vhat * ainv; wv = M v; x += cx * w; w = wv - cw * w  (one warp per row i)
__device__ void m_apply_update(const LsqrParams& p, double ainv, double cx, double cw, bool first) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = blockIdx.x * kWarps + wib, nw = gridDim.x * kWarps;
  for (int i = gw; i < p.n; i += nw) {
    const double* mi = p.M + (int64_t)i * p.n;
    double s = 0.0;
    for (int k = i + lane; k < p.n; k += 32) s = fma(mi[k], p.vhat[k], s);
    s = warp_allreduce_sum(s);
    if (lane == 0) {
      const double wvi = s * ainv;
      p.v[i] = p.vhat[i] * ainv;
      p.wv[i] = wvi;
      if (first) {
        p.w[i] = wvi;
      } else {
        const double wi = p.w[i];
        p.x[i] = fma(cx, wi, p.x[i]);
        p.w[i] = fma(-cw, wi, wvi);
      }
    }
  }
}

template <int T, bool VEC>
__global__ void __launch_bounds__(kThreads, 2) k_lsqr_native(LsqrParams p) {
  __shared__ double s_g[kWarps * 64 * T];
  __shared__ double s_scal[kWarps * 4];
  uint32_t* status = p.status;
  double alpha = 0.0, beta = 0.0, rhobar = 0.0, phibar = 0.0, anorm2 = 0.0, bnorm = 0.0, normal_rel = 0.0;
  int64_t iters = 0;
  int stop = 0;

  if (p.mode != 1) {
    // ---- beta_1 u_1 = b - A x0 : pass with wvec = x0, wsign = -1, uin = b, gamma = -1
    pass_native<T, VEC, false, true>(p, p.x, -1.0, p.b, -1.0, p.u, s_g, s_scal);
    if (!grid_sync(p.bar, status)) return;
    reduce_g(p);
    if (!grid_sync(p.bar, status)) return;
    beta = sqrt(sum_part(p, 0));
    bnorm = sqrt(sum_part(p, 1));
    // ---- alpha_1 v_1 = M^T A^T u_1
    mt_apply(p, beta > 0.0 ? 1.0 / beta : 0.0, 0.0, 2, s_scal);
    if (!grid_sync(p.bar, status)) return;
    alpha = sqrt(sum_part(p, 2));
    // ---- w_1 = M v_1
    m_apply_update(p, alpha > 0.0 ? 1.0 / alpha : 0.0, 0.0, 0.0, true);
    rhobar = alpha;
    phibar = beta;
    anorm2 = alpha * alpha;
    if (beta == 0.0 || alpha == 0.0) stop = 4;
    if (!grid_sync(p.bar, status)) return;

    while (stop == 0) {
      if (iters >= p.maxit) {
        stop = 3;
        break;
      }
      ++iters;
      // uhat_{t+1} = A (M v_t) - alpha_t u_t = A wv - (alpha/beta) uhat_t
      pass_native<T, VEC, false, false>(p, p.wv, 1.0, p.u, alpha / beta, p.u, s_g, s_scal);
      if (!grid_sync(p.bar, status)) return;
      reduce_g(p);
      if (!grid_sync(p.bar, status)) return;
      const double beta1 = sqrt(sum_part(p, 0));
      // vhat_{t+1} = M^T A^T uhat / beta_{t+1} - beta_{t+1} v_t
      mt_apply(p, beta1 > 0.0 ? 1.0 / beta1 : 0.0, beta1, 2, s_scal);
      if (!grid_sync(p.bar, status)) return;
      const double alpha1 = beta1 > 0.0 ? sqrt(sum_part(p, 2)) : 0.0;
      // Givens rotation
      const double rho = sqrt(fma(rhobar, rhobar, beta1 * beta1));
      const double c = rhobar / rho, s = beta1 / rho;
      const double theta = s * alpha1;
      rhobar = -c * alpha1;
      const double phi = c * phibar;
      phibar = s * phibar;
      m_apply_update(p, alpha1 > 0.0 ? 1.0 / alpha1 : 0.0, phi / rho, theta / rho, false);
      anorm2 += alpha1 * alpha1 + beta1 * beta1;
      normal_rel = alpha1 * fabs(c) / sqrt(anorm2);
      alpha = alpha1;
      beta = beta1;
      if (normal_rel <= p.tol) stop = 1;
      else if (phibar <= p.tol * bnorm) stop = 2;
      else if (beta == 0.0 || alpha == 0.0) stop = 4;
      if (!grid_sync(p.bar, status)) return;
    }
  }

  if (p.mode == 2) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      p.out[OUT_ITERS] = (double)iters;
      p.out[OUT_STOP] = (double)stop;
      p.out[OUT_NORMAL_REL] = normal_rel;
      p.out[OUT_BNORM] = bnorm;
      p.out[OUT_ANORM_EST] = sqrt(anorm2);
      if (stop == 3) atomicOr(status, DS_NOCONV);
    }
    return;
  }
  // ---- accuracy pass: y = b - A x, g = A^T y, ||A||_F
  pass_native<T, VEC, true, true>(p, p.x, -1.0, p.b, -1.0, nullptr, s_g, s_scal);
  if (!grid_sync(p.bar, status)) return;
  reduce_g(p);
  if (!grid_sync(p.bar, status)) return;
  if (p.M) mt_apply(p, 1.0, 0.0, 3, s_scal);
  if (!grid_sync(p.bar, status)) return;
  if (blockIdx.x == 0) {
    __shared__ double scratch[32];
    double gx = 0.0, xx = 0.0;
    for (int j = threadIdx.x; j < p.n; j += kThreads) {
      gx = fma(p.g[j], p.g[j], gx);
      xx = fma(p.x[j], p.x[j], xx);
    }
    gx = block_sum(gx, scratch);
    xx = block_sum(xx, scratch);
    if (threadIdx.x == 0) {
      const double rnorm = sqrt(sum_part(p, 0));
      const double bn = sqrt(sum_part(p, 1));
      const double fro = sqrt(sum_part(p, 2));
      const double marn = p.M ? sqrt(sum_part(p, 3)) : 0.0;
      const double arn = sqrt(gx), xn = sqrt(xx);
      p.out[OUT_ITERS] = (double)iters;
      p.out[OUT_STOP] = (double)stop;
      p.out[OUT_NORMAL_REL] = normal_rel;
      p.out[OUT_RNORM] = rnorm;
      p.out[OUT_ARNORM] = arn;
      p.out[OUT_FRO] = fro;
      p.out[OUT_XNORM] = xn;
      p.out[OUT_BNORM] = bn;
      p.out[OUT_ETA_NE] = (fro > 0.0 && rnorm > 0.0) ? arn / (fro * rnorm) : 0.0;
      p.out[OUT_ETA_PRE] = (fro > 0.0 && xn > 0.0) ? marn / (fro * xn) : 0.0;
      p.out[OUT_MARNORM] = marn;
      p.out[OUT_ANORM_EST] = sqrt(anorm2);
      if (stop == 3) atomicOr(status, DS_NOCONV);
    }
  }
}

template <int T, bool VEC>
int grid_for(int sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lsqr_native<T, VEC>, kThreads, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  if (per_sm > 2) per_sm = 2;
  return per_sm * sms;
}

template <int T, bool VEC>
cudaError_t launch(const LsqrParams& p, int grid, cudaStream_t st) {
  LsqrParams q = p;
  void* args[] = {&q};
  return cudaLaunchCooperativeKernel((const void*)k_lsqr_native<T, VEC>, grid, kThreads, args, 0, st);
}

int chunks_for(int n) {
  if (n <= 64) return 1;
  if (n <= 128) return 2;
  if (n <= 256) return 4;
  if (n <= 512) return 8;
  return 0;
}

}  // namespace

int lsqr_grid(int n, bool vec, bool /*native*/, int sms) {
  switch (chunks_for(n)) {
    case 1: return vec ? grid_for<1, true>(sms) : grid_for<1, false>(sms);
    case 2: return vec ? grid_for<2, true>(sms) : grid_for<2, false>(sms);
    case 4: return vec ? grid_for<4, true>(sms) : grid_for<4, false>(sms);
    case 8: return vec ? grid_for<8, true>(sms) : grid_for<8, false>(sms);
    default: return 0;
  }
}

cudaError_t lsqr_run(const LsqrParams& p, bool vec, bool /*native*/, int grid, cudaStream_t st) {
  switch (chunks_for(p.n)) {
    case 1: return vec ? launch<1, true>(p, grid, st) : launch<1, false>(p, grid, st);
    case 2: return vec ? launch<2, true>(p, grid, st) : launch<2, false>(p, grid, st);
    case 4: return vec ? launch<4, true>(p, grid, st) : launch<4, false>(p, grid, st);
    case 8: return vec ? launch<8, true>(p, grid, st) : launch<8, false>(p, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lsq
