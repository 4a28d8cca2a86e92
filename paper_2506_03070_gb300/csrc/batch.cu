// batch.cu -- many independent least-squares problems in one persistent launch.
//
// Every block takes whole problems from a device work counter (problems
// sorted by descending cost on the host, so the tail is short) and runs all
// of Algorithm 1 for a problem by itself: the sparse sign sketch (Sec. 2.1,
// Sec. 3.1.2) scattered into its own Y, a block-local Householder QR
// (Algorithm 1 "QR(Y)"), M = R^{-1} and x0 (Sec. 3.2), then preconditioned
// LSQR (Algorithm 2, one-sync order of App. D.5.1) with block barriers instead
// of grid barriers.  The LSQR pass is the double-float pass of lsqr_device.cuh
// with a lanes-per-row shape chosen for the problem's n (several rows per warp
// for small n), picked by the autotuner in lsq_solve_batch.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "lsqr_device.cuh"
#include "sketch.cuh"

namespace lsq {
namespace {

constexpr int kBatchShapes = 7;
// (lanes per row, column pairs per lane) of the double-float pass
__host__ __device__ constexpr int shape_L(int s) { return s == 0 ? 8 : s == 1 ? 8 : s == 2 ? 16 : s == 3 ? 16 : s == 4 ? 32 : s == 5 ? 32 : 32; }
__host__ __device__ constexpr int shape_P(int s) { return s == 0 ? 2 : s == 1 ? 4 : s == 2 ? 2 : s == 3 ? 4 : s == 4 ? 2 : s == 5 ? 4 : 8; }
__host__ __device__ constexpr int shape_maxn(int s) { return 2 * shape_L(s) * shape_P(s); }

struct BatchItem {
  const double* A;
  const double* b;
  double* x;
  int64_t m, lda;
  int32_t n, d, zeta, shape;
  uint64_t seed;
};

struct BatchParams {
  const BatchItem* items;
  const int32_t* order;
  int32_t count;
  int32_t* next;
  char* ws;
  size_t slab;  // bytes of workspace per block
  // slab layout (byte offsets)
  size_t oY, oW, oR, oM, oMt, oRd, oU, oVec, oGpart, oPart, oImg;
  int npad_max;
  double tol;
  int64_t maxit;  // <= 0: per-problem default
  int mode;       // 0: LSQR + accuracy pass, 2: LSQR only
  double* out;    // count x kOutSlots
  uint32_t* status;  // count
  GridBarrier* bar;  // abort flag holder (never waited on)
};

__device__ int64_t default_maxit_dev(int n, int d, double tol) {
  const double rate = sqrt((double)n / (double)d);
  if (!(tol > 0.0) || !(rate < 1.0)) return 1000;
  return (int64_t)(10.0 * ceil(log(tol) / log(rate)));
}

// Block-local sketch: warps take 32 rows at a time; lane l draws the column of
// S for row base+l; the warp then adds +-A_ij/sqrt(zeta) into Y (L2 reductions).
__device__ void sketch_block(const BatchItem& it, double* Y, int ldy, int32_t* s_idx, uint64_t* s_sgn,
                             uint32_t* status) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* my_idx = s_idx + wib * 32 * 8;
  const int n = it.n, ncol = n + 1;
  const double scale = 1.0 / sqrt((double)it.zeta);
  bool bad = false;
  for (int64_t base = (int64_t)wib * 32; base < it.m; base += (int64_t)kWarps * 32) {
    const int64_t row = base + lane;
    if (row < it.m) {
      int32_t c[8];
      uint64_t signs;
      const int r = sketch_column<8>(it.seed, (uint64_t)row, (uint64_t)it.d, it.zeta, c, signs);
      if (r < 0) atomicOr(status, DS_SKETCH);
#pragma unroll
      for (int k = 0; k < 8; ++k) my_idx[lane * 8 + k] = c[k];
      s_sgn[wib * 32 + lane] = signs;
    }
    __syncwarp();
    const int nrows = (int)min((int64_t)32, it.m - base);
    for (int rr = 0; rr < nrows; ++rr) {
      const int64_t i = base + rr;
      const double* Ai = it.A + i * it.lda;
      const uint64_t sg = s_sgn[wib * 32 + rr];
      const int32_t* ci = my_idx + rr * 8;
      for (int j = lane; j < ncol; j += 32) {
        const double a = j < n ? __ldcs(Ai + j) : it.b[i];
        bad |= !isfinite(a);
        const double sa = a * scale;
        for (int k = 0; k < it.zeta; ++k) {
          const double v = __longlong_as_double(__double_as_longlong(sa) ^ ((long long)(((sg >> k) & 1ull) == 0ull) << 63));
          atomicAdd(Y + (int64_t)ci[k] * ldy + j, v);
        }
      }
    }
    __syncwarp();
  }
  if (bad) atomicOr(status, DS_NONFINITE);
}

// Block-local Householder QR of the d x ncol column-major W (same reflector
// convention as the single-problem kernel); rdiag gets R's diagonal, R[k][j]
// stays in W[j][k].
__device__ void householder_block(double* W, int d, int n, int ncol, double* rdiag, double* scratch) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  for (int k = 0; k < n; ++k) {
    const double* wk = W + (int64_t)k * d;
    double part = 0.0;
    for (int i = k + 1 + threadIdx.x; i < d; i += kThreads) part = fma(__ldcg(wk + i), __ldcg(wk + i), part);
    const double sigma = block_sum(part, scratch);
    const double alpha = __ldcg(wk + k);
    double beta = alpha, tau = 0.0, inv_v0 = 0.0;
    if (sigma != 0.0) {
      const double nrm = sqrt(fma(alpha, alpha, sigma));
      beta = alpha >= 0.0 ? -nrm : nrm;
      tau = (beta - alpha) / beta;
      inv_v0 = 1.0 / (alpha - beta);
    }
    if (threadIdx.x == 0) rdiag[k] = beta;
    if (tau != 0.0) {
      for (int j = k + 1 + wib; j < ncol; j += kWarps) {
        double* wj = W + (int64_t)j * d;
        double s0 = 0.0, s1 = 0.0;
        int i = k + 1 + lane;
        for (; i + 32 < d; i += 64) {
          s0 = fma(__ldcg(wk + i), __ldcg(wj + i), s0);
          s1 = fma(__ldcg(wk + i + 32), __ldcg(wj + i + 32), s1);
        }
        if (i < d) s0 = fma(__ldcg(wk + i), __ldcg(wj + i), s0);
        const double s = warp_allreduce_sum(s0 + s1);
        const double f = tau * fma(inv_v0, s, __ldcg(wj + k));
        const double fv = f * inv_v0;
        if (lane == 0) wj[k] = __ldcg(wj + k) - f;
        for (int i2 = k + 1 + lane; i2 < d; i2 += 32) wj[i2] = fma(-fv, __ldcg(wk + i2), __ldcg(wj + i2));
      }
    }
    __syncthreads();
  }
}

// Doubles of ring per buffer in the batched kernel: chunks of about 4 KB.
constexpr int kBatchChunk = 512;

template <int S>
__device__ void lsqr_shape(LsqrParams& p, double* ring, uint64_t* bars, double* s_scal, uint32_t& seq,
                           float2* s_w) {
  constexpr int R = 32 / shape_L(S);
  const int kk = kBatchChunk / (R * (int)p.ldi);
  p.ring_k = kk > 1 ? kk : 1;
  DfPass<shape_L(S), shape_P(S), true> pass{ring, bars, s_scal, seq, s_w};
  lsqr_body(p, pass, s_scal);
  seq = pass.seq;
}

__global__ void __launch_bounds__(kThreads, 2) k_batch(BatchParams bp) {
  extern __shared__ __align__(128) double s_ring[];
  __shared__ __align__(8) uint64_t s_bars[kWarps * kNbuf];
  __shared__ double s_scal[kWarps * 4];
  __shared__ double scratch[32];
  __shared__ uint64_t s_sgn[kWarps * 32];
  __shared__ int s_prob;
  __shared__ __align__(16) float2 s_w[512];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (lane == 0) {
    for (int b = 0; b < kNbuf; ++b) mbar_init(&s_bars[wib * kNbuf + b], 1u);
    fence_proxy_async_smem();
  }
  __syncthreads();
  uint32_t seq = 0;  // ring steps of this warp (persist across problems)
  char* slab = bp.ws + (size_t)blockIdx.x * bp.slab;
  for (;;) {
    if (threadIdx.x == 0) s_prob = atomicAdd(bp.next, 1);
    __syncthreads();
    const int prob = s_prob;
    __syncthreads();
    if (prob >= bp.count) break;
    const int idx = bp.order[prob];
    const BatchItem it = bp.items[idx];
    uint32_t* status = bp.status + idx;
    const int n = it.n, d = it.d, ncol = n + 1, ldy = ncol;
    double* Y = reinterpret_cast<double*>(slab + bp.oY);
    double* W = reinterpret_cast<double*>(slab + bp.oW);
    double* R = reinterpret_cast<double*>(slab + bp.oR);
    double* M = reinterpret_cast<double*>(slab + bp.oM);
    double* Mt = reinterpret_cast<double*>(slab + bp.oMt);
    double* rdiag = reinterpret_cast<double*>(slab + bp.oRd);
    double* vec = reinterpret_cast<double*>(slab + bp.oVec);

    // ---- sketch Y = S [A | b]
    for (int e = threadIdx.x; e < d * ldy; e += kThreads) Y[e] = 0.0;
    __syncthreads();
    sketch_block(it, Y, ldy, reinterpret_cast<int32_t*>(s_ring), s_sgn, status);
    __threadfence_block();
    __syncthreads();
    // ---- Householder QR of Y (column-major copy), R, M = R^{-1}, x0 = M z
    for (int e = threadIdx.x; e < d * ncol; e += kThreads) {
      const int i = e / ncol, j = e % ncol;
      W[(int64_t)j * d + i] = __ldcg(Y + e);
    }
    __syncthreads();
    householder_block(W, d, n, ncol, rdiag, scratch);
    double mx = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) mx = fmax(mx, fabs(rdiag[i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) scratch[wib] = mx;
    __syncthreads();
    mx = 0.0;
    for (int w = 0; w < kWarps; ++w) mx = fmax(mx, scratch[w]);
    __syncthreads();
    const double thr = (double)n * 2.220446049250313e-16 * mx;
    for (int e = threadIdx.x; e < n * n; e += kThreads) {
      const int i = e / n, j = e % n;
      R[e] = j < i ? 0.0 : (j == i ? rdiag[i] : __ldcg(W + (int64_t)j * d + i));
      if (i == j && !(fabs(rdiag[i]) > thr)) atomicOr(status, DS_RANK);
    }
    __syncthreads();
    for (int c = wib; c < n; c += kWarps) {  // column c of M by back substitution, as row c of Mt
      double* mc = Mt + (int64_t)c * n;
      for (int i = c + 1 + lane; i < n; i += 32) mc[i] = 0.0;
      if (lane == 0) mc[c] = 1.0 / R[(int64_t)c * n + c];
      __syncwarp();
      for (int i = c - 1; i >= 0; --i) {
        const double* Ri = R + (int64_t)i * n;
        double s = 0.0;
        for (int k = i + 1 + lane; k <= c; k += 32) s = fma(Ri[k], mc[k], s);
        s = warp_allreduce_sum(s);
        if (lane == 0) mc[i] = -s / Ri[i];
        __syncwarp();
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += kThreads) {
      const int i = e / n, k = e % n;
      M[e] = Mt[(int64_t)k * n + i];
    }
    __syncthreads();
    for (int i = wib; i < n; i += kWarps) {
      double s = 0.0;
      for (int k = i + lane; k < n; k += 32) s = fma(M[(int64_t)i * n + k], __ldcg(W + (int64_t)n * d + k), s);
      s = warp_allreduce_sum(s);
      if (lane == 0) it.x[i] = s;
    }
    __syncthreads();
    if (*(volatile uint32_t*)status & (DS_RANK | DS_SKETCH | DS_NONFINITE)) continue;

    // ---- preconditioned LSQR from x0, block-local
    LsqrParams p;
    p.A = it.A;
    p.m = it.m;
    p.n = n;
    p.npad = bp.npad_max;
    p.lda = it.lda;
    p.b = it.b;
    p.asplit = reinterpret_cast<float2*>(slab + bp.oImg);
    p.ldi = (n + 1) / 2 * 2;
    p.vec = ((uintptr_t)it.A % 16 == 0) && (it.lda % 2 == 0);
    p.a_ring = p.vec && (n % 2 == 0);
    p.check_df = true;
    p.M = M;
    p.Mt = Mt;
    p.x = it.x;
    p.u = reinterpret_cast<double*>(slab + bp.oU);
    p.v = vec;
    p.vhat = vec + bp.npad_max;
    p.w = vec + 2 * bp.npad_max;
    p.wv = vec + 3 * bp.npad_max;
    p.g = vec + 4 * bp.npad_max;
    p.gpart = reinterpret_cast<double*>(slab + bp.oGpart);
    p.part = reinterpret_cast<double*>(slab + bp.oPart);
    p.tol = bp.tol;
    p.maxit = bp.maxit > 0 ? bp.maxit : default_maxit_dev(n, d, bp.tol);
    p.mode = bp.mode;
    p.gidx = 0;
    p.gcount = 1;
    p.bar = bp.bar;
    p.status = status;
    p.out = bp.out + (int64_t)idx * kOutSlots;
    switch (it.shape) {
      case 0: lsqr_shape<0>(p, s_ring, s_bars, s_scal, seq, s_w); break;
      case 1: lsqr_shape<1>(p, s_ring, s_bars, s_scal, seq, s_w); break;
      case 2: lsqr_shape<2>(p, s_ring, s_bars, s_scal, seq, s_w); break;
      case 3: lsqr_shape<3>(p, s_ring, s_bars, s_scal, seq, s_w); break;
      case 4: lsqr_shape<4>(p, s_ring, s_bars, s_scal, seq, s_w); break;
      default: lsqr_shape<5>(p, s_ring, s_bars, s_scal, seq, s_w); break;
    }
    __syncthreads();
  }
}

// shapes able to take n, fastest-first default order
void shape_candidates(int n, std::vector<int>& out) {
  out.clear();
  if (n <= 32) out = {0, 2};
  else if (n <= 64) out = {1, 2};
  else if (n <= 128) out = {3, 4};
  else out = {5};
}
int bucket_of(int n) { return n <= 32 ? 0 : n <= 64 ? 1 : n <= 128 ? 2 : 3; }

}  // namespace

// ---------------------------------------------------------------------------
// Host side (called from api.cu)
// ---------------------------------------------------------------------------
struct BatchTuning {
  int shape_for_bucket[5] = {-1, -1, -1, -1, -1};
  std::mutex mu;
};

BatchTuning* batch_tuning_new() { return new BatchTuning(); }
void batch_tuning_free(BatchTuning* t) { delete t; }

// Ring doubles per buffer a problem with n columns can need: a chunk of
// about kBatchChunk doubles, or one step (rows per step x padded row) if larger.
int batch_ring_elems(int n) {
  const int ldi = (n + 1) / 2 * 2;
  const int step = (n <= 64 ? 4 : n <= 128 ? 2 : 1) * ldi;
  return step > kBatchChunk ? step : kBatchChunk;
}

size_t batch_smem_bytes(int ring_elems) {
  size_t ring = (size_t)kWarps * kNbuf * (size_t)ring_elems * sizeof(double);
  const size_t sk = (size_t)kWarps * 32 * 8 * sizeof(int32_t);
  const size_t red = (size_t)kWarps * 64 * 8 * sizeof(double);
  ring = std::max(ring, std::max(sk, red));
  return ring;
}

static size_t al(size_t v) { return (v + 255) / 256 * 256; }

BatchLayout batch_layout(int64_t m_max, int n_max, int d_max) {
  BatchLayout L;
  const int npad = (n_max + 31) / 32 * 32;
  const int ldi = (n_max + 1) / 2 * 2;
  size_t o = 0;
  L.oY = o; o += al((size_t)d_max * (n_max + 1) * 8);
  L.oW = o; o += al((size_t)d_max * (n_max + 1) * 8);
  L.oR = o; o += al((size_t)n_max * n_max * 8);
  L.oM = o; o += al((size_t)n_max * n_max * 8);
  L.oMt = o; o += al((size_t)n_max * n_max * 8);
  L.oRd = o; o += al((size_t)npad * 8);
  L.oU = o; o += al((size_t)m_max * 8);
  L.oVec = o; o += al((size_t)5 * npad * 8);
  L.oGpart = o; o += al((size_t)kWarps * npad * 8);
  L.oPart = o; o += al(4 * 8);
  L.oImg = o; o += al((size_t)m_max * ldi * 8);
  L.slab = o;
  L.npad_max = npad;
  return L;
}

int batch_grid(int ring_elems, int sms) {
  const size_t smem = batch_smem_bytes(ring_elems);
  if (cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, kThreads, smem) != cudaSuccess || per_sm < 1)
    return 0;
  return per_sm * sms;
}

// One launch over `count` problems (items in device memory, order = indices
// by descending cost).  ws: grid * L.slab bytes.
cudaError_t batch_launch(const void* items_dev, const int32_t* order_dev, int count, int32_t* next_dev, char* ws,
                         const BatchLayout& L, double tol, int64_t maxit, int mode, double* out, uint32_t* status,
                         GridBarrier* bar, int grid, int ring_elems, cudaStream_t st) {
  BatchParams bp;
  bp.items = static_cast<const BatchItem*>(items_dev);
  bp.order = order_dev;
  bp.count = count;
  bp.next = next_dev;
  bp.ws = ws;
  bp.slab = L.slab;
  bp.oY = L.oY;
  bp.oW = L.oW;
  bp.oR = L.oR;
  bp.oM = L.oM;
  bp.oMt = L.oMt;
  bp.oRd = L.oRd;
  bp.oU = L.oU;
  bp.oVec = L.oVec;
  bp.oGpart = L.oGpart;
  bp.oPart = L.oPart;
  bp.oImg = L.oImg;
  bp.npad_max = L.npad_max;
  bp.tol = tol;
  bp.maxit = maxit;
  bp.mode = mode;
  bp.out = out;
  bp.status = status;
  bp.bar = bar;
  cudaError_t e = cudaMemsetAsync(next_dev, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  const size_t smem = batch_smem_bytes(ring_elems);
  k_batch<<<grid, kThreads, smem, st>>>(bp);
  return cudaGetLastError();
}

size_t batch_item_bytes() { return sizeof(BatchItem); }

// Fill device-layout items from the public descriptors; shapes from the tuning.
void batch_items_fill(void* dst, const lsq_batch_item* src, int64_t count, const BatchTuning* tune) {
  BatchItem* out = static_cast<BatchItem*>(dst);
  for (int64_t i = 0; i < count; ++i) {
    BatchItem b;
    b.A = src[i].A;
    b.b = src[i].b;
    b.x = src[i].x;
    b.m = src[i].m;
    b.lda = src[i].lda;
    b.n = (int32_t)src[i].n;
    b.d = (int32_t)src[i].d;
    b.zeta = src[i].zeta;
    b.seed = src[i].seed;
    const int bk = bucket_of(b.n);
    std::vector<int> c;
    shape_candidates(b.n, c);
    const int tuned = tune ? tune->shape_for_bucket[bk] : -1;
    b.shape = tuned >= 0 ? tuned : c.back();
    out[i] = b;
  }
}

void batch_shape_candidates(int n, std::vector<int>& out) { shape_candidates(n, out); }
int batch_bucket_of(int n) { return bucket_of(n); }
void batch_set_shape(BatchTuning* t, int bucket, int shape) { t->shape_for_bucket[bucket] = shape; }
int batch_get_shape(const BatchTuning* t, int bucket) { return t->shape_for_bucket[bucket]; }
void batch_set_item_shape(void* items, int64_t i, int shape) { static_cast<BatchItem*>(items)[i].shape = shape; }

}  // namespace lsq
