// lsqr_device.cuh -- device side of preconditioned LSQR (Algorithm 2) in the
// one-synchronisation order of App. D.5.1, shared by the single-problem
// persistent kernel (lsqr.cu) and the batched kernel (batch.cu).  Everything
// here works on a "group" of blocks that share one problem: the whole grid
// (grid barriers) or one block (block barriers).
#pragma once
#include "dfloat.cuh"
#include "kernels.h"

namespace lsq {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kNbuf = 3;  // bulk-copy ring depth per warp (rows in flight)

// Barrier over the blocks that share one problem: the whole grid (grid
// barrier with timeout) or a single block (batched problems).
__device__ __forceinline__ bool group_sync(const LsqrParams& p) {
  if (p.gcount == 1) {
    __syncthreads();
    return true;
  }
  return grid_sync(p.bar, p.status, (unsigned int)p.gcount);
}

// Exponent shifts of the double-float passes (see split2s).  A's entries are
// split as A 2^-sa, sa from the largest exponent of A (p.range, written by the
// sketch or by a range scan before the LSQR kernel), so the image holds values
// up to 1 in magnitude.  A pass that forms y = A w - gamma u (or b - A x)
// works on y' = y 2^-e with an output exponent e chosen for it: sb (from the
// largest entry of b) for the residual passes b - A x, whose y has b's scale,
// and 0 for the LSQR iterations, whose uhat = A M v - alpha u has the scale of
// ||A M|| ~ 1 whatever the scale of A and b.  Then the pass vector is scaled
// by 2^(sa-e), b by 2^-e, the stored y' is y 2^-e (the caller rescales gamma
// by 2^(e_prev - e) for the stored vector it reads), and the FP64 outputs are
// scaled back by exact powers of two: A^T y by 2^(sa+e), sums of y^2 and b^2
// by 2^(2e), of A_ij^2 by 2^(2 sa).
__device__ __forceinline__ void range_exps(const LsqrParams& p, int& sa, int& sb) {
  sa = sb = 0;
  if (p.range) {
    const uint32_t ea = __ldcg(p.range) >> 20, eb = __ldcg(p.range + 1) >> 20;
    if (ea) sa = (int)ea - 1023;
    if (eb) sb = (int)eb - 1023;
  }
}

struct PassScale {
  SplitShift a, b;  // A's split (sa) and b's (e)
  double w, g, y2, a2;
};
__device__ __forceinline__ PassScale pass_scale(const LsqrParams& p, int e) {
  int sa, sb;
  range_exps(p, sa, sb);
  PassScale r;
  r.a = split_shift(sa);
  r.b = split_shift(e);
  r.w = ldexp(1.0, sa - e);
  r.g = ldexp(1.0, sa + e);
  r.y2 = ldexp(1.0, 2 * e);
  r.a2 = ldexp(1.0, 2 * sa);
  return r;
}

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
  const int G = p.gcount, blk = p.gidx;
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

template <int T, bool VEC>
struct NativePass {
  double* s_g;
  double* s_scal;
  __device__ void init(LsqrParams& p) {  // y = b - A x0 -> u; sum y^2, sum b^2
    p.gparts = p.gcount;
    pass_native<T, VEC, false, true>(p, p.x, -1.0, p.b, -1.0, p.u, s_g, s_scal);
  }
  __device__ void iter(LsqrParams& p, double gamma) {  // y = A wv - gamma u -> u
    p.gparts = p.gcount;
    pass_native<T, VEC, false, false>(p, p.wv, 1.0, p.u, gamma, p.u, s_g, s_scal);
  }
  __device__ void check(LsqrParams& p) {  // y = b - A x; sum y^2, b^2 (and A_ij^2 unless known)
    p.gparts = p.gcount;
    if (p.fro_in)
      pass_native<T, VEC, false, true>(p, p.x, -1.0, p.b, -1.0, nullptr, s_g, s_scal);
    else
      pass_native<T, VEC, true, true>(p, p.x, -1.0, p.b, -1.0, nullptr, s_g, s_scal);
  }
  __device__ void residual(LsqrParams& p, bool) {  // y = b - A x; sum y^2, b^2
    p.gparts = p.gcount;
    pass_native<T, VEC, false, true>(p, p.x, -1.0, p.b, -1.0, nullptr, s_g, s_scal);
  }
};

// g[j] = sum over blocks of gpart[blk][j], block order.
// Column j is summed by block j % G: thread t adds partials t, t+256, ...,
// then a fixed-order block reduction (deterministic for a given grid).
__device__ void reduce_g(const LsqrParams& p) {
  double* scratch = block_scratch();
  const int G = p.gcount;
  for (int j = p.gidx; j < p.n; j += G) {
    double s = 0.0;
    for (int c = threadIdx.x; c < p.gparts; c += kThreads) s += p.gpart[(int64_t)c * p.npad + j];
    s = block_sum(s, scratch);
    if (threadIdx.x == 0) p.g[j] = s;
  }
}

// Sum over blocks of part[blk][slot]: thread t adds blocks t, t+256, ...,
// then a fixed-order block reduction.  Every thread of every block calls it
// and gets the same value.
__device__ double sum_part(const LsqrParams& p, int slot) {
  double* scratch = block_scratch();
  double s = 0.0;
  for (int c = threadIdx.x; c < p.gcount; c += kThreads) s += p.part[(int64_t)c * 4 + slot];
  return block_sum(s, scratch);
}

// vhat_k = (M^T g)_k * ginv - cv * v_k, one warp per k; per-block sum of
// vhat_k^2 into part[blk][slot].  M^T g uses rows of Mt (contiguous).
__device__ void mt_apply(const LsqrParams& p, double ginv, double cv, int slot, double* s_scal) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = p.gidx * kWarps + wib, nw = p.gcount * kWarps;
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
    p.part[(int64_t)p.gidx * 4 + slot] = s;
  }
  __syncthreads();
}

// v = vhat * ainv; wv = M v; x += cx * w; w = wv - cw * w  (one warp per row i)
__device__ void m_apply_update(const LsqrParams& p, double ainv, double cx, double cw, bool first) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = p.gidx * kWarps + wib, nw = p.gcount * kWarps;
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

// Named barrier of one row group (PW warps that share a row; barrier 0 is
// __syncthreads).
template <int PW>
__device__ __forceinline__ void row_group_bar(int rg) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + rg), "r"(32 * PW) : "memory");
}

// --------------------------------------------------------------------------
// Native FP64 pass for wide rows (512 < n <= 4096), in the row-group/panel
// layout of the double-float panel pass: the block's warps form kWarps/PW row
// groups; warp pw of a group owns columns [c0, c0 + pwid), c0 = pw * pwid,
// pwid = ceil(n/PW) rounded up to 16 (lane l: columns c0 + 2l + 64t, t < 8).
// Per row: each warp's partial dot of its panel with wsign * wvec, the
// partials meet in shared memory at the group's named barrier
// (double-buffered by row parity), every warp sums them in panel order (the
// same y in all of them), y = dot - gamma uin_i (the check: wvec = x,
// wsign = gamma = -1, uin = b: y = b_i - A_i x), stored to uout when given, and
// each warp adds y A_ij into its panel's FP64 column sums.  FRO adds sum
// A_ij^2; UIN2 sums uin_i^2.  Rows are read directly (16-byte loads when A is
// aligned and lda even); the pass is bound by the FP64 pipe (two FMA per
// entry).  Outputs as the other passes: gpart row (block, row group), part
// slots 0 (y^2), 1 (uin^2), 2 (A_ij^2).
// --------------------------------------------------------------------------
template <int PW, bool FRO, bool UIN2>
__device__ void pass_native_panel(const LsqrParams& p, const double* __restrict__ wvec, double wsign,
                                  const double* __restrict__ uin, double gamma, double* __restrict__ uout,
                                  double* s_scal) {
  constexpr int NRG = kWarps / PW, PPL = 8;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int rg = wib / PW, pw = wib % PW;
  const int G = p.gcount, blk = p.gidx, n = p.n;
  const int pwid = ((n + PW - 1) / PW + 15) / 16 * 16;
  const int c0 = pw * pwid, cend = min(c0 + pwid, n);
  const int64_t r0 = (p.m * blk) / G, r1 = (p.m * (blk + 1)) / G;
  double* pdot = s_scal + kWarps * 4 + rg * 2 * PW;
  double xr[2 * PPL], g[2 * PPL];
#pragma unroll
  for (int t = 0; t < PPL; ++t) {
    const int c = c0 + 2 * lane + 64 * t;
    xr[2 * t] = c < cend ? wsign * wvec[c] : 0.0;
    xr[2 * t + 1] = c + 1 < cend ? wsign * wvec[c + 1] : 0.0;
    g[2 * t] = g[2 * t + 1] = 0.0;
  }
  double ss = 0.0, bb = 0.0, fro = 0.0;
  uint32_t par = 0;
  for (int64_t i = r0 + rg; i < r1; i += NRG, par ^= 1u) {
    const double* Ai = p.A + i * p.lda;
    double2 a[PPL];
#pragma unroll
    for (int t = 0; t < PPL; ++t) {
      const int c = c0 + 2 * lane + 64 * t;
      if (c + 1 < cend) {
        if (p.vec) {
          a[t] = __ldcs(reinterpret_cast<const double2*>(Ai + c));
        } else {
          a[t].x = __ldcs(Ai + c);
          a[t].y = __ldcs(Ai + c + 1);
        }
      } else if (c < cend) {
        a[t].x = __ldcs(Ai + c);
        a[t].y = 0.0;
      } else {
        a[t].x = a[t].y = 0.0;
      }
    }
    const double ui = uin[i];
    double dot = 0.0;
#pragma unroll
    for (int t = 0; t < PPL; ++t) {
      dot = fma(a[t].x, xr[2 * t], dot);
      dot = fma(a[t].y, xr[2 * t + 1], dot);
    }
    dot = warp_allreduce_sum(dot);
    double* slot = pdot + par * PW;
    if (lane == 0) slot[pw] = dot;
    row_group_bar<PW>(rg);
    double ax = slot[0];
#pragma unroll
    for (int q = 1; q < PW; ++q) ax += slot[q];
    const double y = fma(-gamma, ui, ax);
    if (pw == 0) {
      if (uout && lane == 0) uout[i] = y;
      ss = fma(y, y, ss);
      if (UIN2) bb = fma(ui, ui, bb);
    }
#pragma unroll
    for (int t = 0; t < PPL; ++t) {
      g[2 * t] = fma(y, a[t].x, g[2 * t]);
      g[2 * t + 1] = fma(y, a[t].y, g[2 * t + 1]);
      if (FRO) {
        fro = fma(a[t].x, a[t].x, fro);
        fro = fma(a[t].y, a[t].y, fro);
      }
    }
  }
  double* gw = p.gpart + ((int64_t)blk * NRG + rg) * p.npad;
#pragma unroll
  for (int t = 0; t < PPL; ++t) {
    const int c = c0 + 2 * lane + 64 * t;
    if (c < cend) gw[c] = g[2 * t];
    if (c + 1 < cend) gw[c + 1] = g[2 * t + 1];
  }
  if (FRO) fro = warp_allreduce_sum(fro);
  if (lane == 0) {
    s_scal[wib * 4 + 0] = ss;
    s_scal[wib * 4 + 1] = bb;
    s_scal[wib * 4 + 2] = fro;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double sum = 0.0;
    for (int w = 0; w < kWarps; ++w) sum += s_scal[w * 4 + threadIdx.x];
    p.part[(int64_t)blk * 4 + threadIdx.x] = sum;
  }
  __syncthreads();
}

// The native FP64 passes for wide rows (512 < n <= 4096, LSQ_FLAG_NATIVE_FP64),
// PW warps per row in column panels: pass_native_panel above.
template <int PW>
struct NativePanelPass {
  double* s_scal;  // kWarps * 6 doubles: per-warp sums, then the row groups' partial dots
  __device__ void init(LsqrParams& p) {  // y = b - A x0 -> u; sum y^2, sum b^2
    p.gparts = p.gcount * (kWarps / PW);
    pass_native_panel<PW, false, true>(p, p.x, -1.0, p.b, -1.0, p.u, s_scal);
  }
  __device__ void iter(LsqrParams& p, double gamma) {  // y = A wv - gamma u -> u
    p.gparts = p.gcount * (kWarps / PW);
    pass_native_panel<PW, false, false>(p, p.wv, 1.0, p.u, gamma, p.u, s_scal);
  }
  __device__ void check(LsqrParams& p) {  // y = b - A x; sum y^2, b^2 (and A_ij^2 unless known)
    p.gparts = p.gcount * (kWarps / PW);
    if (p.fro_in)
      pass_native_panel<PW, false, true>(p, p.x, -1.0, p.b, -1.0, nullptr, s_scal);
    else
      pass_native_panel<PW, true, true>(p, p.x, -1.0, p.b, -1.0, nullptr, s_scal);
  }
  __device__ void residual(LsqrParams& p, bool) {  // y = b - A x; sum y^2, b^2
    p.gparts = p.gcount * (kWarps / PW);
    pass_native_panel<PW, false, true>(p, p.x, -1.0, p.b, -1.0, nullptr, s_scal);
  }
};


// --------------------------------------------------------------------------
// The double-float pass (FP32/INT pipes only in the per-entry and per-row
// work).  A warp handles R = 32/L rows per step, L lanes per row; lane l
// (segment l/L, column lane l%L) owns column pairs 2(l%L) + 2L t, t < PPL.
// Rows arrive through a per-warp ring of kNbuf shared-memory buffers of R rows
// filled by cp.async.bulk (one elected lane issues, an mbarrier per buffer
// signals completion), so a warp keeps kNbuf steps in flight while it computes.
//
// Per step: each lane splits its entries into (hi, mid) floats (or reads them
// from the float-pair image), accumulates its row's dot in two independent
// float-pair accumulators, sums them and butterflies over its segment (every
// lane of a segment ends with the same pair), forms y = dot - gamma * u_i in
// pair arithmetic, stores y (the u buffer holds float pairs in this kernel)
// and adds y * A_i into its column accumulators.  Column pairs are
// renormalised every second step and flushed -- summed over the segments,
// then into the warp's FP64 partial row of gpart -- every 32 steps.  gpart
// holds one row per warp.
//
// The first pass reads A (through the ring when n and lda are even and A is
// aligned, by direct loads otherwise) and, when p.asplit is set, stores every
// split row as a (hi, mid) float-pair image of A (ldi entries per row, 8 bytes
// each, as FP64), pair-major per column pair: hi_c, hi_c+1, mid_c, mid_c+1;
// later passes stream the image: identical values, and the per-entry integer
// split leaves the hot loop.  The pass vector sits in shared memory the same
// way (w1_c, w1_c+1, w2_c, w2_c+1), so the packed FP32x2 instructions take two
// columns' operands straight from one 16-byte load.
// --------------------------------------------------------------------------
template <int L, int PPL, bool CHUNKED = false, int PW = 1>
struct DfPass {
  static constexpr int R = 32 / L;
  static_assert(PW == 1 || (L == 32 && PPL == 8 && !CHUNKED), "panel pass: one row per step, 512 columns a warp");
  double* ring;     // dynamic shared memory [kWarps][kNbuf][p.ring_k * R * ldi]
  uint64_t* bars;   // [kWarps][kNbuf]
  double* s_scal;
  uint32_t seq;     // ring buffers this warp has consumed (all passes)
  float2* s_w;      // shared [>= ldi]: the pass vector as float pairs
  int u_exp = 0;    // output exponent of the stored vector u (see range_exps)

  // Chunk c of the group's rows: K = p.ring_k consecutive steps of R rows.
  template <bool FROM_IMAGE>
  __device__ void issue(const LsqrParams& p, int64_t r0, int64_t r1, int wib, uint32_t jc, double* myring,
                        uint64_t* mybars) {
    const int K = CHUNKED ? p.ring_k : 1;
    const int64_t crow = r0 + ((int64_t)wib + (int64_t)kWarps * jc) * K * R;
    const int rows = (int)min((int64_t)K * R, r1 - crow);
    const uint32_t b = (seq + jc) % kNbuf;
    double* dst = myring + (size_t)b * K * R * p.ldi;
    if (FROM_IMAGE) {
      const uint32_t bytes = (uint32_t)(rows * p.ldi) * 8u;
      mbar_arrive_expect_tx(mybars + b, bytes);
      bulk_g2s(dst, p.asplit + crow * p.ldi, bytes, mybars + b);
    } else if (p.lda == p.n) {
      const uint32_t bytes = (uint32_t)(rows * p.n) * 8u;
      mbar_arrive_expect_tx(mybars + b, bytes);
      bulk_g2s(dst, p.A + crow * p.lda, bytes, mybars + b);
    } else {
      const uint32_t rb = (uint32_t)p.n * 8u;
      mbar_arrive_expect_tx(mybars + b, rb * (uint32_t)rows);
      for (int r = 0; r < rows; ++r) bulk_g2s(dst + (size_t)r * p.ldi, p.A + (crow + r) * p.lda, rb, mybars + b);
    }
  }

  // Wait (bounded by lim ns) for the buffer of chunk jc.  Returns false on
  // timeout (warp-uniform).
  __device__ bool wait(uint32_t jc, uint64_t* mybars, unsigned long long lim) {
    const uint32_t s = seq + jc, b = s % kNbuf, par = (s / kNbuf) & 1u;
    const bool timed_out = !mbar_wait_bounded(mybars + b, par, lim);
    return !__any_sync(0xffffffffu, timed_out);
  }

  // column pairs summed over the R segments, then added to the warp's FP64 row
  __device__ void flush(float2 (&Gh)[PPL], float2 (&Gl)[PPL], double* gw, int cl, int seg, int n, bool& first,
                        double gmul) {
#pragma unroll
    for (int t = 0; t < PPL; ++t) {
#pragma unroll
      for (int o = L; o < 32; o <<= 1) {
        const df a = df_add(df{Gh[t].x, Gl[t].x}, shfl_xor_df(df{Gh[t].x, Gl[t].x}, o));
        const df b = df_add(df{Gh[t].y, Gl[t].y}, shfl_xor_df(df{Gh[t].y, Gl[t].y}, o));
        Gh[t] = make_float2(a.hi, b.hi);
        Gl[t] = make_float2(a.lo, b.lo);
      }
    }
    if (seg == 0) {
#pragma unroll
      for (int t = 0; t < PPL; ++t) {
        const int c = 2 * cl + 2 * L * t;
        if (c < n) {
          double2 g = first ? make_double2(0.0, 0.0) : *reinterpret_cast<const double2*>(gw + c);
          g.x += df_to_double(df{Gh[t].x, Gl[t].x}) * gmul;
          g.y += df_to_double(df{Gh[t].y, Gl[t].y}) * gmul;
          *reinterpret_cast<double2*>(gw + c) = g;
        }
      }
    }
#pragma unroll
    for (int t = 0; t < PPL; ++t) Gh[t] = Gl[t] = make_float2(0.f, 0.f);
    first = false;
  }

  // FROM_IMAGE: rows come from the image through the ring; else from A (split
  // on the fly) -- through the ring when p.a_ring, by direct loads otherwise --
  // and, when WRITE_IMAGE, the split rows are stored to the image.  FRO adds
  // sum A_ij^2 (in pair arithmetic) to slot 2.  Warp w takes chunks
  // w, w+8, ... of K steps (K*R consecutive rows), one ring buffer per chunk.
  template <bool UIN_B, bool UIN2, bool STORE, bool FROM_IMAGE, bool WRITE_IMAGE, bool FRO>
  __device__ void run(const LsqrParams& p, const double* __restrict__ wvec, double wsign, double gamma, int e_out) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int seg = lane / L, cl = lane % L;
    const int G = p.gcount, blk = p.gidx;
    const int n = p.n, K = CHUNKED ? p.ring_k : 1;
    const int64_t r0 = (p.m * blk) / G, r1 = (p.m * (blk + 1)) / G;
    const int64_t crows = (int64_t)K * R;
    const int64_t nchunks = (r1 - r0 + crows - 1) / crows;
    const uint32_t count = nchunks > wib ? (uint32_t)((nchunks - wib + kWarps - 1) / kWarps) : 0u;
    const bool use_ring = FROM_IMAGE || p.a_ring;
    double* myring = ring + (size_t)wib * kNbuf * crows * p.ldi;
    uint64_t* mybars = bars + wib * kNbuf;
    float2* ubuf = reinterpret_cast<float2*>(p.u);
    double* gw = p.gpart + ((int64_t)blk * kWarps + wib) * p.npad;
    const PassScale sc = pass_scale(p, e_out);
    const unsigned long long lim = wait_limit_ns(p.bar);

    // the pass vector (scaled by 2^(sa-sb)) as float pairs in shared memory (read per entry)
    for (int c = 2 * threadIdx.x; c < p.ldi; c += 2 * kThreads) {
      const double v0 = c < n ? wsign * wvec[c] * sc.w : 0.0;
      const double v1 = c + 1 < n ? wsign * wvec[c + 1] * sc.w : 0.0;
      const float a0 = __double2float_rn(v0), a1 = __double2float_rn(v1);
      *reinterpret_cast<float4*>(s_w + c) =
          make_float4(a0, a1, __double2float_rn(v0 - (double)a0), __double2float_rn(v1 - (double)a1));
    }
    __syncthreads();
    // column accumulators of the lane's column pairs (entries 2t, 2t+1 packed)
    float2 Gh[PPL], Gl[PPL];
#pragma unroll
    for (int t = 0; t < PPL; ++t) Gh[t] = Gl[t] = make_float2(0.f, 0.f);
    const float g1 = __double2float_rn(gamma);
    const df gdf{g1, __double2float_rn(gamma - (double)g1)};
    df ss{0.f, 0.f}, bb{0.f, 0.f}, fro{0.f, 0.f};
    bool first_flush = true;
    uint32_t steps = 0;

    if (lane == 0 && use_ring) {
      fence_proxy_async_smem();
      for (uint32_t jc = 0; jc < count && jc < (uint32_t)kNbuf; ++jc)
        issue<FROM_IMAGE>(p, r0, r1, wib, jc, myring, mybars);
    }
    bool ok = true;
    uint32_t jc = 0;
    for (; jc < count; ++jc) {
      if (use_ring && !wait(jc, mybars, lim)) {
        ok = false;
        break;
      }
      const int64_t crow = r0 + ((int64_t)wib + (int64_t)kWarps * jc) * crows;
      const double* cbuf = myring + (size_t)((seq + jc) % kNbuf) * crows * p.ldi;
      for (int s = 0; s < K; ++s, ++steps) {
        const int64_t row = crow + (int64_t)s * R + seg;
        // unchunked single-row steps: every issued step is a real row
        const bool valid = (CHUNKED || R > 1) ? row < r1 : true;
        if (CHUNKED && !__any_sync(0xffffffffu, valid)) break;  // past the end of the group's rows
        const double* buf = cbuf + (size_t)(s * R + seg) * p.ldi;
        // u_i (or b_i) is needed only after the row dot: load it first
        double bi = 0.0;
        float2 uu = make_float2(0.f, 0.f);
        if (valid) {
          if (UIN_B)
            bi = p.b[row];
          else
            uu = ubuf[row];
        }
        // the lane's column pairs, pair-major: H[t] = (hi_c, hi_c+1), Mm[t] = (mid_c, mid_c+1)
        float2 H[PPL], Mm[PPL];
#pragma unroll
        for (int t = 0; t < PPL; ++t) {
          const int c = 2 * cl + 2 * L * t;
          const bool in = valid && c < n;
          if (FROM_IMAGE) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (in) v = *reinterpret_cast<const float4*>(buf + c);
            H[t] = make_float2(v.x, v.y);
            Mm[t] = make_float2(v.z, v.w);
          } else {
            double2 v = make_double2(0.0, 0.0);
            if (p.a_ring) {
              if (in) v = *reinterpret_cast<const double2*>(buf + c);
            } else if (in) {
              const double* Ar = p.A + row * p.lda;
              v.x = __ldcs(Ar + c);
              if (c + 1 < n) v.y = __ldcs(Ar + c + 1);
            }
            split2s(v.x, H[t].x, Mm[t].x, sc.a);
            split2s(v.y, H[t].y, Mm[t].y, sc.a);
            if (WRITE_IMAGE && in)
              *reinterpret_cast<float4*>(p.asplit + row * p.ldi + c) = make_float4(H[t].x, H[t].y, Mm[t].x, Mm[t].y);
          }
        }
        // row dot: two independent pair accumulators (even and odd columns),
        // advanced together by the packed FP32x2 instructions
        float2 avh = make_float2(0.f, 0.f), avl = make_float2(0.f, 0.f);
#pragma unroll
        for (int t = 0; t < PPL; ++t) {
          const int c = 2 * cl + 2 * L * t;
          float4 ww = make_float4(0.f, 0.f, 0.f, 0.f);
          if (c < n) ww = *reinterpret_cast<const float4*>(s_w + c);
          df2_fma_acc(avh, avl, H[t], Mm[t], make_float2(ww.x, ww.y), make_float2(ww.z, ww.w));
        }
        df dot = df_add(df{avh.x, avl.x}, df{avh.y, avl.y});
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) dot = df_add_unnorm(dot, shfl_xor_df(dot, o));
        dot = df_renorm(dot);
        df y{0.f, 0.f};
        if (valid) {
          const df ui = UIN_B ? df_from_double_s(bi, sc.b) : df{uu.x, uu.y};
          y = df_add(dot, df_neg(df_mul(gdf, ui)));
          if (STORE && cl == 0) ubuf[row] = make_float2(y.hi, y.lo);
          ss = df_add(ss, df_mul(y, y));
          if (UIN2) bb = df_add(bb, df_mul(ui, ui));
        }
        const float2 y1 = make_float2(y.hi, y.hi), y2 = make_float2(y.lo, y.lo);
#pragma unroll
        for (int t = 0; t < PPL; ++t) {
          df2_fma_acc(Gh[t], Gl[t], H[t], Mm[t], y1, y2);
          if (steps & 1u) df2_renorm(Gh[t], Gl[t]);
          if (FRO) {
            df_fma_acc(fro, H[t].x, Mm[t].x, H[t].x, Mm[t].x);
            df_fma_acc(fro, H[t].y, Mm[t].y, H[t].y, Mm[t].y);
          }
        }
        if (FRO) fro = df_renorm(fro);
        if ((steps & 31u) == 31u) flush(Gh, Gl, gw, cl, seg, n, first_flush, sc.g);
      }
      __syncwarp();
      if (lane == 0 && use_ring && jc + kNbuf < count) {
        fence_proxy_async_smem();
        issue<FROM_IMAGE>(p, r0, r1, wib, jc + kNbuf, myring, mybars);
      }
    }
    if (!ok) {
      // give up: flag, then let the copies already issued land before leaving
      if (lane == 0) {
        atomicOr(p.status, DS_TIMEOUT);
        barrier_abort(p.bar);
      }
      for (uint32_t k = jc; k < count && k < jc + kNbuf; ++k) wait(k, mybars, lim);
    }
    if (use_ring) seq += count;  // ring phases advance only when rows went through it
    flush(Gh, Gl, gw, cl, seg, n, first_flush, sc.g);
    // ss and bb: one copy per segment (lanes of a segment agree); fro per lane
#pragma unroll
    for (int o = L; o < 32; o <<= 1) {
      ss = df_add(ss, shfl_xor_df(ss, o));
      bb = df_add(bb, shfl_xor_df(bb, o));
    }
    double frow = 0.0;
    if (FRO) frow = warp_allreduce_sum(df_to_double(fro)) * sc.a2;
    if (lane == 0) {
      s_scal[wib * 4 + 0] = df_to_double(ss) * sc.y2;
      s_scal[wib * 4 + 1] = df_to_double(bb) * sc.y2;
      s_scal[wib * 4 + 2] = frow;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      double sum = 0.0;
      for (int w = 0; w < kWarps; ++w) sum += s_scal[w * 4 + threadIdx.x];
      p.part[(int64_t)blk * 4 + threadIdx.x] = sum;
    }
    __syncthreads();
  }

  // ------------------------------------------------------------------------
  // Wide rows (n > 512): PW warps share each row.  The block's warps form
  // kWarps/PW row groups; warp pw of a group owns the column panel
  // [c0, c0 + pwid), c0 = pw * pwid, pwid = ceil(n/PW) rounded up to 16, and
  // keeps its own bulk-copy ring of panel slices.  Per row: every warp forms
  // its panel's partial dot, writes it to shared memory, the group meets at a
  // named barrier, and every warp sums the PW partials in panel order (the
  // same value in all of them), forms y and adds y * A_i into its own panel's
  // column accumulators.  Only panel 0 stores y and sums y^2 and u_i^2.  A
  // warp whose copy wait gives up keeps meeting its group's barriers (on
  // stale data, with DS_TIMEOUT raised) so the group never waits on it.
  // ------------------------------------------------------------------------
  __device__ __forceinline__ void group_bar(int rg) { row_group_bar<PW>(rg); }

  template <bool FROM_IMAGE>
  __device__ void issue_panel(const LsqrParams& p, int64_t row, int c0, int cols, uint32_t jc, double* myring,
                              uint64_t* mybars) {
    const uint32_t b = (seq + jc) % kNbuf;
    double* dst = myring + (size_t)b * 512;
    const uint32_t bytes = (uint32_t)cols * 8u;
    mbar_arrive_expect_tx(mybars + b, bytes);
    if (FROM_IMAGE)
      bulk_g2s(dst, p.asplit + row * p.ldi + c0, bytes, mybars + b);
    else
      bulk_g2s(dst, p.A + row * p.lda + c0, bytes, mybars + b);
  }

  template <bool UIN_B, bool UIN2, bool STORE, bool FROM_IMAGE, bool WRITE_IMAGE, bool FRO>
  __device__ void run_panel(const LsqrParams& p, const double* __restrict__ wvec, double wsign, double gamma,
                            int e_out) {
    constexpr int NRG = kWarps / PW;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int rg = wib / PW, pw = wib % PW;
    const int G = p.gcount, blk = p.gidx, n = p.n;
    const int pwid = ((n + PW - 1) / PW + 15) / 16 * 16;
    const int c0 = pw * pwid;
    const int cend = min(c0 + pwid, n);
    // bulk-copied slice: the panel's columns, padded to the image's even row
    const int cols = FROM_IMAGE ? (int)min((int64_t)pwid, p.ldi - c0) : cend - c0;
    const int64_t r0 = (p.m * blk) / G, r1 = (p.m * (blk + 1)) / G;
    const int64_t nrows = r1 - r0;
    const uint32_t count = nrows > rg ? (uint32_t)((nrows - rg + NRG - 1) / NRG) : 0u;
    const bool use_ring = FROM_IMAGE || p.a_ring;
    double* myring = ring + (size_t)wib * kNbuf * 512;
    uint64_t* mybars = bars + wib * kNbuf;
    float2* ubuf = reinterpret_cast<float2*>(p.u);
    double* gw = p.gpart + ((int64_t)blk * NRG + rg) * p.npad;
    // s_scal holds kWarps * 6 doubles here: 4 per warp, then [row group][2 parities][PW] pairs
    df* pdot = reinterpret_cast<df*>(s_scal + kWarps * 4) + rg * 2 * PW;
    const PassScale sc = pass_scale(p, e_out);
    const unsigned long long lim = wait_limit_ns(p.bar);

    for (int c = 2 * threadIdx.x; c < p.ldi; c += 2 * kThreads) {
      const double v0 = c < n ? wsign * wvec[c] * sc.w : 0.0;
      const double v1 = c + 1 < n ? wsign * wvec[c + 1] * sc.w : 0.0;
      const float a0 = __double2float_rn(v0), a1 = __double2float_rn(v1);
      *reinterpret_cast<float4*>(s_w + c) =
          make_float4(a0, a1, __double2float_rn(v0 - (double)a0), __double2float_rn(v1 - (double)a1));
    }
    __syncthreads();
    float2 Gh[PPL], Gl[PPL];
#pragma unroll
    for (int t = 0; t < PPL; ++t) Gh[t] = Gl[t] = make_float2(0.f, 0.f);
    const float g1 = __double2float_rn(gamma);
    const df gdf{g1, __double2float_rn(gamma - (double)g1)};
    df ss{0.f, 0.f}, bb{0.f, 0.f}, fro{0.f, 0.f};
    bool first_flush = true;

    if (lane == 0 && use_ring) {
      fence_proxy_async_smem();
      for (uint32_t jc = 0; jc < count && jc < (uint32_t)kNbuf; ++jc)
        issue_panel<FROM_IMAGE>(p, r0 + rg + (int64_t)NRG * jc, c0, cols, jc, myring, mybars);
    }
    bool ok = true;
    uint32_t failed_at = count;
    for (uint32_t jc = 0; jc < count; ++jc) {
      if (use_ring && ok && !wait(jc, mybars, lim)) {
        ok = false;
        failed_at = jc;
        if (lane == 0) {
          atomicOr(p.status, DS_TIMEOUT);
          barrier_abort(p.bar);
        }
      }
      const int64_t row = r0 + rg + (int64_t)NRG * jc;
      const double* buf = myring + (size_t)((seq + jc) % kNbuf) * 512;
      double bi = 0.0;
      float2 uu = make_float2(0.f, 0.f);
      if (UIN_B)
        bi = p.b[row];
      else
        uu = ubuf[row];
      float2 H[PPL], Mm[PPL];  // pair-major, as in run()
#pragma unroll
      for (int t = 0; t < PPL; ++t) {
        const int c = c0 + 2 * lane + 64 * t;
        const bool in = c < cend;
        if (FROM_IMAGE) {
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if (in) v = *reinterpret_cast<const float4*>(buf + (c - c0));
          H[t] = make_float2(v.x, v.y);
          Mm[t] = make_float2(v.z, v.w);
        } else {
          double2 v = make_double2(0.0, 0.0);
          if (p.a_ring) {
            if (in) v = *reinterpret_cast<const double2*>(buf + (c - c0));
          } else if (in) {
            const double* Ar = p.A + row * p.lda;
            v.x = __ldcs(Ar + c);
            if (c + 1 < n) v.y = __ldcs(Ar + c + 1);
          }
          split2s(v.x, H[t].x, Mm[t].x, sc.a);
          split2s(v.y, H[t].y, Mm[t].y, sc.a);
          if (WRITE_IMAGE && in)
            *reinterpret_cast<float4*>(p.asplit + row * p.ldi + c) = make_float4(H[t].x, H[t].y, Mm[t].x, Mm[t].y);
        }
      }
      // four pair chains (even / odd t, each packed over two columns): two
      // independent dependency chains per lane
      float2 h0 = make_float2(0.f, 0.f), l0 = h0, h1 = h0, l1 = h0;
#pragma unroll
      for (int t = 0; t < PPL; ++t) {
        const int c = c0 + 2 * lane + 64 * t;
        float4 ww = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c < cend) ww = *reinterpret_cast<const float4*>(s_w + c);
        if (t & 1)
          df2_fma_acc(h1, l1, H[t], Mm[t], make_float2(ww.x, ww.y), make_float2(ww.z, ww.w));
        else
          df2_fma_acc(h0, l0, H[t], Mm[t], make_float2(ww.x, ww.y), make_float2(ww.z, ww.w));
      }
      df dot = df_add(df_add(df{h0.x, l0.x}, df{h0.y, l0.y}), df_add(df{h1.x, l1.x}, df{h1.y, l1.y}));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dot = df_add_unnorm(dot, shfl_xor_df(dot, o));
      dot = df_renorm(dot);
      df* slot = pdot + (jc & 1u) * PW;
      if (lane == 0) slot[pw] = dot;
      group_bar(rg);
      dot = slot[0];
#pragma unroll
      for (int q = 1; q < PW; ++q) dot = df_add(dot, slot[q]);
      const df ui = UIN_B ? df_from_double_s(bi, sc.b) : df{uu.x, uu.y};
      const df y = df_add(dot, df_neg(df_mul(gdf, ui)));
      if (pw == 0) {
        if (STORE && lane == 0) ubuf[row] = make_float2(y.hi, y.lo);
        ss = df_add(ss, df_mul(y, y));
        if (UIN2) bb = df_add(bb, df_mul(ui, ui));
      }
      const float2 y1 = make_float2(y.hi, y.hi), y2 = make_float2(y.lo, y.lo);
#pragma unroll
      for (int t = 0; t < PPL; ++t) {
        df2_fma_acc(Gh[t], Gl[t], H[t], Mm[t], y1, y2);
        if (jc & 1u) df2_renorm(Gh[t], Gl[t]);
        if (FRO) {
          df_fma_acc(fro, H[t].x, Mm[t].x, H[t].x, Mm[t].x);
          df_fma_acc(fro, H[t].y, Mm[t].y, H[t].y, Mm[t].y);
        }
      }
      if (FRO) fro = df_renorm(fro);
      if ((jc & 31u) == 31u) flush_panel(Gh, Gl, gw, c0, cend, first_flush, sc.g);
      __syncwarp();
      if (lane == 0 && use_ring && ok && jc + kNbuf < count) {
        fence_proxy_async_smem();
        issue_panel<FROM_IMAGE>(p, r0 + rg + (int64_t)NRG * (jc + kNbuf), c0, cols, jc + kNbuf, myring, mybars);
      }
    }
    if (!ok) {
      // let the copies already issued land before the ring is reused
      for (uint32_t k = failed_at; k < count && k < failed_at + kNbuf; ++k) wait(k, mybars, lim);
    }
    if (use_ring) seq += count;
    flush_panel(Gh, Gl, gw, c0, cend, first_flush, sc.g);
    double frow = 0.0;
    if (FRO) frow = warp_allreduce_sum(df_to_double(fro)) * sc.a2;
    if (lane == 0) {
      s_scal[wib * 4 + 0] = df_to_double(ss) * sc.y2;
      s_scal[wib * 4 + 1] = df_to_double(bb) * sc.y2;
      s_scal[wib * 4 + 2] = frow;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      double sum = 0.0;
      for (int w = 0; w < kWarps; ++w) sum += s_scal[w * 4 + threadIdx.x];
      p.part[(int64_t)blk * 4 + threadIdx.x] = sum;
    }
    __syncthreads();
  }

  __device__ void flush_panel(float2 (&Gh)[PPL], float2 (&Gl)[PPL], double* gw, int c0, int cend, bool& first,
                              double gmul) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int t = 0; t < PPL; ++t) {
      const int c = c0 + 2 * lane + 64 * t;
      if (c < cend) {
        double2 g = first ? make_double2(0.0, 0.0) : *reinterpret_cast<const double2*>(gw + c);
        g.x += df_to_double(df{Gh[t].x, Gl[t].x}) * gmul;
        g.y += df_to_double(df{Gh[t].y, Gl[t].y}) * gmul;
        *reinterpret_cast<double2*>(gw + c) = g;
      }
      Gh[t] = Gl[t] = make_float2(0.f, 0.f);
    }
    first = false;
  }

  __device__ void init(LsqrParams& p) {
    int sa, sb;
    range_exps(p, sa, sb);
    u_exp = sb;  // u = b - A x0 carries b's scale
    if (PW > 1) {
      p.gparts = p.gcount * (kWarps / PW);
      if (p.asplit) {
        run_panel<true, true, true, false, true, false>(p, p.x, -1.0, -1.0, sb);
        asm volatile("fence.proxy.async.global;" ::: "memory");
      } else {
        run_panel<true, true, true, false, false, false>(p, p.x, -1.0, -1.0, sb);
      }
      return;
    }
    p.gparts = p.gcount * kWarps;
    if (p.asplit) {
      run<true, true, true, false, true, false>(p, p.x, -1.0, -1.0, sb);
      // the image was written through the generic proxy and is read by bulk
      // copies (async proxy) after the next barrier
      asm volatile("fence.proxy.async.global;" ::: "memory");
    } else {
      run<true, true, true, false, false, false>(p, p.x, -1.0, -1.0, sb);
    }
  }
  // uhat = A wv - gamma uhat_prev at output exponent 0; the stored vector has
  // exponent u_exp, so gamma is applied as gamma 2^u_exp
  __device__ void iter(LsqrParams& p, double gamma) {
    const double g = ldexp(gamma, u_exp);
    u_exp = 0;
    if (PW > 1) {
      p.gparts = p.gcount * (kWarps / PW);
      if (p.asplit)
        run_panel<false, false, true, true, false, false>(p, p.wv, 1.0, g, 0);
      else
        run_panel<false, false, true, false, false, false>(p, p.wv, 1.0, g, 0);
      return;
    }
    p.gparts = p.gcount * kWarps;
    if (p.asplit)
      run<false, false, true, true, false, false>(p, p.wv, 1.0, g, 0);
    else
      run<false, false, true, false, false, false>(p, p.wv, 1.0, g, 0);
  }
  // y = b - A x with A^T y, sum y^2 and sum b^2 (heavy-ball momentum); the
  // first call writes the float-pair image, later ones stream it.
  __device__ void residual(LsqrParams& p, bool first) {
    int sa, sb;
    range_exps(p, sa, sb);
    if (PW > 1) {
      p.gparts = p.gcount * (kWarps / PW);
      if (p.asplit && first) {
        run_panel<true, true, false, false, true, false>(p, p.x, -1.0, -1.0, sb);
        asm volatile("fence.proxy.async.global;" ::: "memory");
      } else if (p.asplit) {
        run_panel<true, true, false, true, false, false>(p, p.x, -1.0, -1.0, sb);
      } else {
        run_panel<true, true, false, false, false, false>(p, p.x, -1.0, -1.0, sb);
      }
      return;
    }
    p.gparts = p.gcount * kWarps;
    if (p.asplit && first) {
      run<true, true, false, false, true, false>(p, p.x, -1.0, -1.0, sb);
      asm volatile("fence.proxy.async.global;" ::: "memory");
    } else if (p.asplit) {
      run<true, true, false, true, false, false>(p, p.x, -1.0, -1.0, sb);
    } else {
      run<true, true, false, false, false, false>(p, p.x, -1.0, -1.0, sb);
    }
  }
  // Accuracy pass (Algorithm 1's final check; App. A.3): always native FP64
  // on the original A -- one warp per row for n <= 512, the panel layout of
  // the wide-row pass above.
  __device__ void check(LsqrParams& p) {
    // sum A_ij^2 is skipped when the sketch already formed it (p.fro_in):
    // the pass is bound by the FP64 pipe, two FMA per entry instead of three
    if (PW > 1) {
      p.gparts = p.gcount * (kWarps / PW);
      if (p.fro_in)
        pass_native_panel<PW, false, true>(p, p.x, -1.0, p.b, -1.0, nullptr, s_scal);
      else
        pass_native_panel<PW, true, true>(p, p.x, -1.0, p.b, -1.0, nullptr, s_scal);
      return;
    }
    p.gparts = p.gcount;
    constexpr int TN = (2 * L * PPL + 63) / 64;
    if (p.vec) {
      if (p.fro_in)
        pass_native<TN, true, false, true>(p, p.x, -1.0, p.b, -1.0, nullptr, ring, s_scal);
      else
        pass_native<TN, true, true, true>(p, p.x, -1.0, p.b, -1.0, nullptr, ring, s_scal);
    } else {
      if (p.fro_in)
        pass_native<TN, false, false, true>(p, p.x, -1.0, p.b, -1.0, nullptr, ring, s_scal);
      else
        pass_native<TN, false, true, true>(p, p.x, -1.0, p.b, -1.0, nullptr, ring, s_scal);
    }
  }
};

// --------------------------------------------------------------------------
// Algorithm 2 around a pass policy (see the file header for the order).
// --------------------------------------------------------------------------
template <class Pass>
__device__ void finish_body(LsqrParams& p, Pass& pass, double* s_scal, int64_t iters, int stop, double normal_rel,
                            double bnorm, double anorm_est, bool skip_check);

template <class Pass>
__device__ void lsqr_body(LsqrParams& p, Pass& pass, double* s_scal) {
  double alpha = 0.0, beta = 0.0, rhobar = 0.0, phibar = 0.0, anorm2 = 0.0, bnorm = 0.0, normal_rel = 0.0;
  int64_t iters = 0;
  int stop = 0;

  if (p.mode != 1) {
    // ---- beta_1 u_1 = b - A x0
    pass.init(p);
    if (!group_sync(p)) return;
    reduce_g(p);
    if (!group_sync(p)) return;
    beta = sqrt(sum_part(p, 0));
    bnorm = sqrt(sum_part(p, 1));
    // ---- alpha_1 v_1 = M^T A^T u_1
    mt_apply(p, beta > 0.0 ? 1.0 / beta : 0.0, 0.0, 2, s_scal);
    if (!group_sync(p)) return;
    alpha = sqrt(sum_part(p, 2));
    // ---- w_1 = M v_1
    m_apply_update(p, alpha > 0.0 ? 1.0 / alpha : 0.0, 0.0, 0.0, true);
    rhobar = alpha;
    phibar = beta;
    anorm2 = alpha * alpha;
    if (beta == 0.0 || alpha == 0.0) stop = 4;
    if (!group_sync(p)) return;

    while (stop == 0) {
      if (iters >= p.maxit) {
        stop = 3;
        break;
      }
      ++iters;
      // uhat_{t+1} = A (M v_t) - alpha_t u_t = A wv - (alpha/beta) uhat_t
      pass.iter(p, alpha / beta);
      if (!group_sync(p)) return;
      reduce_g(p);
      if (!group_sync(p)) return;
      const double beta1 = sqrt(sum_part(p, 0));
      // vhat_{t+1} = M^T A^T uhat / beta_{t+1} - beta_{t+1} v_t
      mt_apply(p, beta1 > 0.0 ? 1.0 / beta1 : 0.0, beta1, 2, s_scal);
      if (!group_sync(p)) return;
      const double a2 = sum_part(p, 2);
      const double alpha1 = beta1 > 0.0 ? sqrt(a2) : 0.0;
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
      if (!group_sync(p)) return;
    }
  }

  finish_body(p, pass, s_scal, iters, stop, normal_rel, bnorm, sqrt(anorm2), p.mode == 2);
}

// Outputs of an iteration (LSQR or heavy-ball momentum), then -- unless
// skip_check -- the accuracy pass: y = b - A x, g = A^T y, ||A||_F and the
// backward-error bounds.
template <class Pass>
__device__ void finish_body(LsqrParams& p, Pass& pass, double* s_scal, int64_t iters, int stop, double normal_rel,
                            double bnorm, double anorm_est, bool skip_check) {
  uint32_t* status = p.status;
  if (skip_check) {
    if (p.gidx == 0 && threadIdx.x == 0) {
      p.out[OUT_ITERS] = (double)iters;
      p.out[OUT_STOP] = (double)stop;
      p.out[OUT_NORMAL_REL] = normal_rel;
      p.out[OUT_BNORM] = bnorm;
      p.out[OUT_ANORM_EST] = anorm_est;
      if (stop == 3) atomicOr(status, DS_NOCONV);
    }
    return;
  }
  // ---- accuracy pass: y = b - A x, g = A^T y, ||A||_F
  const bool stamp = p.gidx == 0 && threadIdx.x == 0;
  if (stamp) p.out[OUT_T_CHECK0] = (double)globaltimer_ns();
  pass.check(p);
  if (!group_sync(p)) return;
  if (stamp) p.out[OUT_T_CHECK1] = (double)globaltimer_ns();
  reduce_g(p);
  if (!group_sync(p)) return;
  if (p.M) mt_apply(p, 1.0, 0.0, 3, s_scal);
  if (!group_sync(p)) return;
  if (p.gidx == 0) {
    double* scratch = block_scratch();
    double gx = 0.0, xx = 0.0;
    for (int j = threadIdx.x; j < p.n; j += kThreads) {
      gx = fma(p.g[j], p.g[j], gx);
      xx = fma(p.x[j], p.x[j], xx);
    }
    gx = block_sum(gx, scratch);
    xx = block_sum(xx, scratch);
    const double rnorm = sqrt(sum_part(p, 0));
    const double bn = sqrt(sum_part(p, 1));
    const double fro = p.fro_in ? sqrt(__ldcg(p.fro_in)) : sqrt(sum_part(p, 2));
    const double marn = p.M ? sqrt(sum_part(p, 3)) : 0.0;
    if (threadIdx.x == 0) {
      const double arn = sqrt(gx), xn = sqrt(xx);
      p.out[OUT_ITERS] = (double)iters;
      p.out[OUT_STOP] = (double)stop;
      p.out[OUT_NORMAL_REL] = normal_rel;
      p.out[OUT_RNORM] = rnorm;
      p.out[OUT_ARNORM] = arn;
      p.out[OUT_FRO] = fro;
      p.out[OUT_XNORM] = xn;
      p.out[OUT_BNORM] = bn;
      const double eta_ne = (fro > 0.0 && rnorm > 0.0) ? arn / (fro * rnorm) : 0.0;
      const double eta_pre = (fro > 0.0 && xn > 0.0) ? marn / (fro * xn) : 0.0;
      p.out[OUT_ETA_NE] = eta_ne;
      p.out[OUT_ETA_PRE] = eta_pre;
      p.out[OUT_MARNORM] = marn;
      p.out[OUT_ANORM_EST] = anorm_est;
      if (stop == 3) atomicOr(status, DS_NOCONV);
      // accuracy gate: the smaller of the two backward-error bounds (NaN fails)
      if (p.gate > 0.0) {
        const double eta = p.M ? fmin(eta_ne, eta_pre) : eta_ne;
        if (!(eta <= p.gate)) atomicOr(status, DS_ACCURACY);
      }
    }
  }
}

// x_t = x_{t-1} + alpha M q + beta (x_{t-1} - x_{t-2}) with q = vhat = M^T A^T r
// (one warp per row i of the upper triangular M); w holds x_{t-2}.
__device__ void hbm_update(const LsqrParams& p) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = p.gidx * kWarps + wib, nw = p.gcount * kWarps;
  for (int i = gw; i < p.n; i += nw) {
    const double* mi = p.M + (int64_t)i * p.n;
    double s = 0.0;
    for (int k = i + lane; k < p.n; k += 32) s = fma(mi[k], p.vhat[k], s);
    s = warp_allreduce_sum(s);
    if (lane == 0) {
      const double xi = p.x[i];
      p.x[i] = fma(p.hbm_alpha, s, fma(p.hbm_beta, xi - p.w[i], xi));
      p.w[i] = xi;
    }
  }
}

// Algorithm 6 (gradient descent with heavy-ball momentum) from x0:
//   x_{-1} = x_0;  g_t = M M^T A^T (b - A x_{t-1});
//   x_t = x_{t-1} + alpha g_t + beta (x_{t-1} - x_{t-2}).
// Per iteration one pass over A forms r = b - A x_{t-1} and, with each row on
// chip, A^T r and ||r||^2; then q = M^T A^T r and the update.  Test before each
// update: ||q|| <= tol ||b|| (bounds ||A (x - x_*)|| by tol ||b|| / sigma_min(AM),
// the Sec. 4.3 accuracy target), ||r|| <= tol ||b||, or maxit updates.
template <class Pass>
__device__ void hbm_body(LsqrParams& p, Pass& pass, double* s_scal) {
  for (int i = p.gidx * kThreads + threadIdx.x; i < p.n; i += p.gcount * kThreads) p.w[i] = p.x[i];
  if (!group_sync(p)) return;
  int64_t iters = 0;
  int stop = 0;
  double rel = 0.0, bn = 0.0;
  bool first = true;
  for (;;) {
    pass.residual(p, first);
    first = false;
    if (!group_sync(p)) return;
    reduce_g(p);
    if (!group_sync(p)) return;
    mt_apply(p, 1.0, 0.0, 2, s_scal);  // vhat = M^T g; ||vhat||^2 -> part slot 2
    if (!group_sync(p)) return;
    const double rn = sqrt(sum_part(p, 0)), qn = sqrt(sum_part(p, 2));
    bn = sqrt(sum_part(p, 1));
    rel = bn > 0.0 ? qn / bn : 0.0;
    if (qn <= p.tol * bn) {
      stop = 1;
      break;
    }
    if (rn <= p.tol * bn) {
      stop = 2;
      break;
    }
    if (iters >= p.maxit) {
      stop = 3;
      break;
    }
    hbm_update(p);
    ++iters;
    if (!group_sync(p)) return;
  }
  if (!group_sync(p)) return;
  finish_body(p, pass, s_scal, iters, stop, rel, bn, 0.0, p.mode == 4);
}

}  // namespace
}  // namespace lsq
