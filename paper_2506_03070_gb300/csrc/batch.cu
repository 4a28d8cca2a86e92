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

#include "problem_device.cuh"

namespace lsq {
namespace {

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
  size_t oY, oW, oR, oM, oMt, oRd, oU, oVec, oGpart, oPart, oImg, oRange;
  int npad_max;
  double tol;
  int64_t maxit;  // <= 0: per-problem default
  int mode;       // 0: LSQR + accuracy pass, 2: LSQR only
  double* out;    // count x kOutSlots
  uint32_t* status;  // count
  GridBarrier* bar;  // abort flag holder (never waited on)
};

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

    uint32_t* range = reinterpret_cast<uint32_t*>(slab + bp.oRange);
    const Group g{0, 1, bp.bar, status, range};
    // ---- sketch Y = S [A | b]
    zero_group(Y, (int64_t)d * ldy, g);
    if (threadIdx.x < 2) range[threadIdx.x] = 0u;
    __syncthreads();
    sketch_group(it.A, it.b, it.m, n, it.lda, d, it.zeta, it.seed, Y, ldy, reinterpret_cast<int32_t*>(s_ring), s_sgn,
                 g);
    __threadfence_block();
    __syncthreads();
    // ---- Householder QR of Y (column-major copy), R, M = R^{-1}, x0 = M z
    for (int e = threadIdx.x; e < d * ncol; e += kThreads) {
      const int i = e / ncol, j = e % ncol;
      W[(int64_t)j * d + i] = __ldcg(Y + e);
    }
    householder_group(W, d, n, ncol, rdiag, scratch, g);
    precond_group(W, d, n, rdiag, R, M, Mt, it.x, scratch, g);
    const int failed = threadIdx.x == 0 ? ((*(volatile uint32_t*)status & (DS_RANK | DS_SKETCH | DS_NONFINITE)) != 0)
                                        : 0;
    if (__syncthreads_or(failed)) continue;

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
    p.range = range;
    p.gate = bp.mode == 0 ? fmax(1e-10, bp.tol) : 0.0;
    p.fro_in = nullptr;
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

// shapes able to take n, the one measured fastest on the batched mix first
// (the default when the n-range is not tuned)
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
// about kChunkDoubles doubles, or one step (rows per step x padded row) if larger.
int batch_ring_elems(int n) {
  const int ldi = (n + 1) / 2 * 2;
  const int step = (n <= 64 ? 4 : n <= 128 ? 2 : 1) * ldi;
  return step > kChunkDoubles ? step : kChunkDoubles;
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
  L.oRange = o; o += al(2 * 4);
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
  bp.oRange = L.oRange;
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
    b.shape = tuned >= 0 ? tuned : c.front();
    out[i] = b;
  }
}

void batch_shape_candidates(int n, std::vector<int>& out) { shape_candidates(n, out); }
int batch_bucket_of(int n) { return bucket_of(n); }
void batch_set_shape(BatchTuning* t, int bucket, int shape) { t->shape_for_bucket[bucket] = shape; }
int batch_get_shape(const BatchTuning* t, int bucket) { return t->shape_for_bucket[bucket]; }
void batch_set_item_shape(void* items, int64_t i, int shape) { static_cast<BatchItem*>(items)[i].shape = shape; }
int batch_shape_maxn(int shape) { return shape >= 0 && shape < kShapes ? shape_maxn(shape) : 0; }

}  // namespace lsq
