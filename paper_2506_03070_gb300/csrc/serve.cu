// serve.cu -- lsq_submit / lsq_poll: a persistent request loop.
//
// Device side: k_serve is one cooperative launch with every block resident
// (2 per SM).  Requests sit in a ring in device memory.  The host publishes
// an entry with two copy-engine copies on one stream -- the entry, then the
// new `tail` -- so an entry has always landed before `tail` covers it, with
// no reliance on the host CPU's memory ordering towards the GPU; each entry
// also carries its sequence number, which a block checks before trusting
// it.  A block claims the
// request at the queue head with a compare-and-swap on a device word
// (head << 16 | joined): a request of group size G stays at the head until G
// blocks have joined, each getting its index in the group.  Requests are
// therefore claimed strictly in arrival order; only the head can be partly
// joined, and every earlier request already has its full group, so a
// waiting group always fills once earlier requests finish.  The group runs
// Algorithm 1 for the request on its own slot of device memory (sketch, QR,
// M, x0, LSQR, accuracy pass; problem_device.cuh) with group barriers
// scoped to the request.  The last block to leave the request copies the
// results into the request's completion record (mapped host memory) and
// releases its `done` flag.
//
// Host side: one scheduler thread per context admits queued requests in
// arrival order while their slot fits in the arena (first-fit allocator),
// stages host problems and zeroes the slot's control words with copy-engine
// copies only (no kernel may need SMs while the server holds them),
// publishes staged requests, watches completion flags, copies host results
// back, and frees slots.  It launches the server when work is published and
// none is running, and closes it (a flag the idle blocks read) 2 ms after the
// last published request completed -- also while requests are still staged,
// since their callers' earlier GPU work (which they are ordered after) cannot
// run while the server holds every SM.
//
// Every device wait is bounded: group barriers and bulk-copy waits by
// kBarrierTimeoutNs, an idle block by kServeIdleNs, after which it retires the
// whole launch (kRetired) so that no group can form on a half-exited server.
// A block whose request hit a timeout leaves the loop (its copy ring may be
// out of phase); the host relaunches the server once the rest has drained.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ctx.h"
#include "problem_device.cuh"

namespace lsq {
namespace {

constexpr int kServeMaxN = 1024;
constexpr int kServeRingDoubles = kWarps * kNbuf * 512;  // per-warp rings of 3 x 4 KB
constexpr unsigned long long kServeIdleNs = 10ull * 1000ull * 1000ull * 1000ull;
constexpr uint32_t kServeCap = 4096;  // queue entries
// Bit of the queue word that retires the running launch: set (by a block
// that waited kServeIdleNs with no work) only by compare-and-swap on the
// same word that claims carry, so no group is joined once it is set; every
// block leaves on seeing it, and the last block out clears it.
constexpr unsigned long long kRetired = 1ull << 63;

// Pass variants: 0..5 chunked shapes (n <= 256), 6: one warp per row with
// 8 column pairs per lane (n <= 512), 7: two warps per row (n <= 1024).
constexpr int kVarWarpRow = 6, kVarPanel2 = 7;

struct ServeItem {  // written by the host into mapped memory; 8-byte words only
  const double* A;
  const double* b;
  double* x;
  int64_t m, lda;
  int32_t n, d, zeta, variant;
  int32_t G, mode;
  uint64_t seed;
  double tol;
  int64_t maxit;
  double gate;  // accuracy gate of the final pass (0: none)
  char* slot;
  uint64_t oCtl, oY, oW, oR, oM, oMt, oRd, oU, oVec, oGpart, oPart, oImg;
  int64_t npad;
  uint64_t seq;  // queue index + 1
};
constexpr int kItemWords = sizeof(ServeItem) / 8;
static_assert(sizeof(ServeItem) % 8 == 0, "item is copied as 8-byte words");

struct ServeCtl {  // per request, in its slot; reset by the host before publishing
  GridBarrier bar;     // bar.limit_us: the context's wait limit when the request was staged
  uint32_t status;
  uint32_t exit;
  uint32_t range[2];   // exponent maxima of A and b (the double-float passes' shifts)
  double out[kOutSlots];
};

struct ServeDone {  // per queue entry, mapped host memory
  unsigned long long done;  // the entry's sequence number once its request is complete
  uint32_t status;
  uint32_t pad;
  double out[kOutSlots];
};

struct ServeArgs {
  const unsigned long long* tail;  // device: entries published
  const unsigned int* closed;      // device: 1 = idle blocks leave
  const ServeItem* ring;
  ServeDone* done;
  unsigned long long* qstate;  // device: head << 16 | joined, plus kRetired
  uint32_t* srv_status;        // device: DS_TIMEOUT when a block left early
  unsigned int* exits;         // device: blocks of this launch that have left
  uint32_t cap;
};

__device__ __forceinline__ void st_release_sys_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Thread 0: claim the next request (or learn that the server is to stop).
// Returns 0 with (idx, gidx) and the item copied into s_item, 1 to exit.
__device__ int claim(const ServeArgs& a, unsigned long long& idx, int& gidx, unsigned long long* s_item) {
  unsigned long long idle0 = 0;
  unsigned int ns = 128;
  for (;;) {
    const unsigned long long st = atomicAdd(a.qstate, 0ull);
    if (st & kRetired) return 1;
    const unsigned long long head = st >> 16;
    const unsigned int joined = (unsigned int)(st & 0xFFFFull);
    const unsigned long long tail = *(volatile const unsigned long long*)a.tail;
    const ServeItem* e = a.ring + (head % a.cap);
    // an entry counts once its own sequence number has landed (always true
    // after `tail` covers it; checked rather than assumed)
    const bool ready = head < tail && *(volatile const unsigned long long*)&e->seq == head + 1;
    if (!ready) {
      if (head >= tail && *(volatile const unsigned int*)a.closed) return 1;
      const unsigned long long now = globaltimer_ns();
      if (idle0 == 0) {
        idle0 = now;
      } else if (now - idle0 > kServeIdleNs) {
        // the host stopped closing the server: retire the whole launch,
        // unless a claim changed the queue word meanwhile
        if (atomicCAS(a.qstate, st, st | kRetired) == st) return 1;
        idle0 = 0;
        continue;
      }
      __nanosleep(ns);
      if (ns < 4096) ns <<= 1;
      continue;
    }
    idle0 = 0;
    ns = 128;
    const unsigned int G = (unsigned int)*(volatile const int32_t*)&e->G;
    const unsigned long long next = (joined + 1 >= G) ? ((head + 1) << 16) : (st + 1);
    if (atomicCAS(a.qstate, st, next) == st) {
      idx = head;
      gidx = (int)joined;
      const volatile unsigned long long* src = reinterpret_cast<const volatile unsigned long long*>(e);
      for (int w = 0; w < kItemWords; ++w) s_item[w] = src[w];
      return 0;
    }
  }
}

template <int PW>
__device__ __noinline__ void lsqr_wide(LsqrParams& p, double* ring, uint64_t* bars, double* s_scal, uint32_t& seq, float2* s_w) {
  p.ring_k = 1;
  DfPass<32, 8, false, PW> pass{ring, bars, s_scal, seq, s_w};
  lsqr_body(p, pass, s_scal);
  seq = pass.seq;
}

// Algorithm 1 for one request on group (gidx of it.G blocks).
__device__ void serve_solve(const ServeItem& it, int gidx, double* s_ring, uint64_t* s_bars, double* s_scal,
                            double* scratch, uint64_t* s_sgn, float2* s_w, uint32_t& seq) {
  char* slot = it.slot;
  ServeCtl* ctl = reinterpret_cast<ServeCtl*>(slot + it.oCtl);
  const Group g{gidx, it.G, &ctl->bar, &ctl->status, ctl->range};
  const int n = it.n, d = it.d, ncol = n + 1, ldy = ncol;
  double* Y = reinterpret_cast<double*>(slot + it.oY);
  double* W = reinterpret_cast<double*>(slot + it.oW);
  double* R = reinterpret_cast<double*>(slot + it.oR);
  double* M = reinterpret_cast<double*>(slot + it.oM);
  double* Mt = reinterpret_cast<double*>(slot + it.oMt);
  double* rdiag = reinterpret_cast<double*>(slot + it.oRd);
  double* vec = reinterpret_cast<double*>(slot + it.oVec);
  const int npad = (int)it.npad;

  const bool stamp = gidx == 0 && threadIdx.x == 0;
  if (stamp) ctl->out[OUT_T_JOIN] = (double)globaltimer_ns();
  // ---- Y = S [A | b]
  zero_group(Y, (int64_t)d * ldy, g);
  if (!gsync(g)) return;
  if (stamp) ctl->out[OUT_T_START] = (double)globaltimer_ns();
  sketch_group(it.A, it.b, it.m, n, it.lda, d, it.zeta, it.seed, Y, ldy, reinterpret_cast<int32_t*>(s_ring), s_sgn, g);
  __threadfence();
  if (!gsync(g)) return;
  if (stamp) ctl->out[OUT_T_SKETCH] = (double)globaltimer_ns();
  // ---- QR of Y, R, M = R^{-1}, x0 = M z
  {
    const int64_t tid = (int64_t)gidx * kThreads + threadIdx.x, ts = (int64_t)it.G * kThreads;
    for (int64_t e = tid; e < (int64_t)d * ncol; e += ts) {
      const int64_t i = e / ncol, j = e % ncol;
      W[j * d + i] = __ldcg(Y + e);
    }
  }
  if (!householder_group(W, d, n, ncol, rdiag, scratch, g)) return;
  if (!precond_group(W, d, n, rdiag, R, M, Mt, it.x, scratch, g)) return;
  if (stamp) ctl->out[OUT_T_PRECOND] = (double)globaltimer_ns();
  // one reader, so the whole block takes the same branch
  const int failed = threadIdx.x == 0 ? ((*(volatile uint32_t*)&ctl->status &
                                          (DS_RANK | DS_SKETCH | DS_NONFINITE | DS_TIMEOUT)) != 0)
                                      : 0;
  if (__syncthreads_or(failed)) return;

  // ---- preconditioned LSQR from x0 and the accuracy pass
  LsqrParams p;
  p.A = it.A;
  p.m = it.m;
  p.n = n;
  p.npad = npad;
  p.lda = it.lda;
  p.b = it.b;
  p.asplit = reinterpret_cast<float2*>(slot + it.oImg);
  p.ldi = (n + 1) / 2 * 2;
  p.vec = ((uintptr_t)it.A % 16 == 0) && (it.lda % 2 == 0);
  p.a_ring = p.vec && (n % 2 == 0);
  p.ring_k = 1;
  p.range = ctl->range;
  p.gate = it.gate;
  p.fro_in = nullptr;
  p.M = M;
  p.Mt = Mt;
  p.x = it.x;
  p.u = reinterpret_cast<double*>(slot + it.oU);
  p.v = vec;
  p.vhat = vec + npad;
  p.w = vec + 2 * npad;
  p.wv = vec + 3 * npad;
  p.g = vec + 4 * npad;
  p.gpart = reinterpret_cast<double*>(slot + it.oGpart);
  p.part = reinterpret_cast<double*>(slot + it.oPart);
  p.tol = it.tol;
  p.maxit = it.maxit > 0 ? it.maxit : default_maxit_dev(n, d, it.tol);
  p.mode = it.mode;
  p.gidx = gidx;
  p.gcount = it.G;
  p.bar = &ctl->bar;
  p.status = &ctl->status;
  p.out = ctl->out;
  switch (it.variant) {
    case 0: lsqr_shape<0>(p, s_ring, s_bars, s_scal, seq, s_w); break;
    case 1: lsqr_shape<1>(p, s_ring, s_bars, s_scal, seq, s_w); break;
    case 2: lsqr_shape<2>(p, s_ring, s_bars, s_scal, seq, s_w); break;
    case 3: lsqr_shape<3>(p, s_ring, s_bars, s_scal, seq, s_w); break;
    case 4: lsqr_shape<4>(p, s_ring, s_bars, s_scal, seq, s_w); break;
    case 5: lsqr_shape<5>(p, s_ring, s_bars, s_scal, seq, s_w); break;
    case kVarWarpRow: lsqr_wide<1>(p, s_ring, s_bars, s_scal, seq, s_w); break;
    default: lsqr_wide<2>(p, s_ring, s_bars, s_scal, seq, s_w); break;
  }
  if (stamp) ctl->out[OUT_T_END] = (double)globaltimer_ns();
}

__global__ void __launch_bounds__(kThreads, 2) k_serve(ServeArgs a) {
  extern __shared__ __align__(128) double s_ring[];  // rings, then the pass vector (float2[kServeMaxN])
  __shared__ __align__(8) uint64_t s_bars[kWarps * kNbuf];
  __shared__ __align__(16) double s_scal[kWarps * 6];
  __shared__ double scratch[32];
  __shared__ uint64_t s_sgn[kWarps * 32];
  __shared__ __align__(16) unsigned long long s_item[kItemWords];
  __shared__ unsigned long long s_idx;
  __shared__ int s_cmd, s_gidx, s_leave;
  if ((threadIdx.x & 31) == 0) {
    for (int b = 0; b < kNbuf; ++b) mbar_init(&s_bars[(threadIdx.x >> 5) * kNbuf + b], 1u);
    fence_proxy_async_smem();
  }
  __syncthreads();
  float2* s_w = reinterpret_cast<float2*>(s_ring + kServeRingDoubles);
  uint32_t seq = 0;  // ring phases of this warp, carried across requests
  for (;;) {
    if (threadIdx.x == 0) {
      unsigned long long idx = 0;
      int gidx = 0;
      s_cmd = claim(a, idx, gidx, s_item);
      s_idx = idx;
      s_gidx = gidx;
    }
    __syncthreads();
    if (s_cmd != 0) break;
    const ServeItem& it = *reinterpret_cast<const ServeItem*>(s_item);
    serve_solve(it, s_gidx, s_ring, s_bars, s_scal, scratch, s_sgn, s_w, seq);
    __syncthreads();
    if (threadIdx.x == 0) {
      bool leave = false;
      ServeCtl* ctl = reinterpret_cast<ServeCtl*>(it.slot + it.oCtl);
      const uint32_t bits = *(volatile uint32_t*)&ctl->status;
      leave = (bits & DS_TIMEOUT) != 0;
      __threadfence();
      if (atomicAdd(&ctl->exit, 1u) == (uint32_t)it.G - 1u) {
        // last block of the group: publish the results
        __threadfence();
        ServeDone* dn = a.done + (s_idx % a.cap);
        for (int k = 0; k < kOutSlots; ++k) dn->out[k] = __ldcg(&ctl->out[k]);
        dn->status = *(volatile uint32_t*)&ctl->status;
        __threadfence_system();
        st_release_sys_u64(&dn->done, s_idx + 1ull);
      }
      if (leave) atomicOr(a.srv_status, DS_TIMEOUT);
      s_leave = leave ? 1 : 0;
    }
    __syncthreads();
    // s_cmd is rewritten only after the next request's first barrier, s_leave
    // only after its second: every thread has read both by then
    if (s_leave != 0) break;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(a.exits, 1u) == gridDim.x - 1u) {  // last block out: reset for the next launch
      atomicExch(a.exits, 0u);
      atomicAnd(a.qstate, ~kRetired);
      __threadfence();
    }
  }
}

size_t serve_smem() { return (size_t)kServeRingDoubles * sizeof(double) + (size_t)kServeMaxN * sizeof(float2); }

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int variant_for(int n, const BatchTuning* tune) {
  if (n > 512) return kVarPanel2;
  if (n > 256) return kVarWarpRow;
  std::vector<int> c;
  batch_shape_candidates(n, c);
  const int tuned = tune ? batch_get_shape(tune, batch_bucket_of(n)) : -1;
  return tuned >= 0 ? tuned : c.front();
}

lsq_status status_of_bits(uint32_t bits) {
  if (bits & DS_TIMEOUT) return LSQ_ERR_TIMEOUT;
  if (bits & DS_NONFINITE) return LSQ_ERR_NONFINITE;
  if (bits & DS_SKETCH) return LSQ_ERR_SKETCH;
  if (bits & DS_RANK) return LSQ_ERR_RANK;
  if (bits & DS_NOCONV) return LSQ_ERR_NOCONV;
  if (bits & DS_ACCURACY) return LSQ_ERR_ACCURACY;
  return LSQ_OK;
}

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct ServeRequest {
  lsq_ticket ticket = 0;
  lsq_problem pr{};
  lsq_opts o{};
  double* x_user = nullptr;
  ServeItem item{};
  size_t bytes = 0, off = 0;
  size_t oA = 0, oB = 0, oX = 0;  // host problems: device copies in the slot
  uint64_t qidx = 0;
  cudaEvent_t ev = nullptr;
  cudaEvent_t ready = nullptr;  // recorded on the caller's stream at submission, or null
  enum { kPending, kStaging, kPublished, kDraining, kDone } state = kPending;
  lsq_status status = LSQ_PENDING;
  double out[kOutSlots] = {0};
  double t_submit = 0, t_start = 0, t_done = 0;
};

struct Server {
  lsq_ctx* ctx = nullptr;
  int device = 0;
  // device memory
  char* arena = nullptr;
  size_t arena_bytes = 0, arena_used = 0, arena_peak = 0;
  std::map<size_t, size_t> free_blocks;  // offset -> size
  // device memory: queue words and the ring of entries
  char* d_q = nullptr;
  unsigned long long* d_tail = nullptr;
  unsigned int* d_closed = nullptr;
  unsigned int* d_exits = nullptr;
  unsigned long long* d_qstate = nullptr;
  uint32_t* d_srv_status = nullptr;
  ServeItem* d_ring = nullptr;
  // pinned host memory: staged entries and tail values (sources of the
  // publishing copies), constant words, the control-word template (zero but
  // for the wait limit)
  char* h_pin = nullptr;
  ServeItem* h_items = nullptr;
  unsigned long long* h_tails = nullptr;
  unsigned int* h_words = nullptr;  // {0, 1}
  void* h_zero = nullptr;
  // mapped host memory: completion records written by the device
  char* hmem = nullptr;
  ServeDone* done = nullptr;
  ServeDone* d_done = nullptr;
  cudaEvent_t ev_pub = nullptr;
  cudaStream_t s_srv = nullptr, s_copy = nullptr;
  cudaEvent_t ev_srv = nullptr;
  std::vector<cudaEvent_t> ev_pool;
  int grid = 0;
  int max_group = 0;
  double cta_bytes = 64.0 * 1024 * 1024;
  bool running = false, closing = false;
  double idle_since = 0;
  uint64_t tail = 0;
  std::set<uint64_t> inflight_q;  // queue indices published and not yet seen complete
  std::deque<ServeRequest*> pending, staging;
  std::map<uint64_t, ServeRequest*> published;
  std::vector<ServeRequest*> draining;
  std::unordered_map<lsq_ticket, ServeRequest*> tickets;
  lsq_ticket next_ticket = 1;
  int64_t n_submitted = 0, n_completed = 0, n_launches = 0;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::string err;
  std::thread th;

  bool arena_alloc(size_t bytes, size_t* off) {
    for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t noff = it->first + bytes;
        free_blocks.erase(it);
        if (rest) free_blocks[noff] = rest;
        arena_used += bytes;
        if (arena_used > arena_peak) arena_peak = arena_used;
        return true;
      }
    }
    return false;
  }
  void arena_free(size_t off, size_t bytes) {
    arena_used -= bytes;
    auto it = free_blocks.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_blocks.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_blocks.erase(nx);
    }
    if (it != free_blocks.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_blocks.erase(it);
      }
    }
  }
  cudaEvent_t get_event() {
    if (!ev_pool.empty()) {
      cudaEvent_t e = ev_pool.back();
      ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
  }
  void put_event(cudaEvent_t e) {
    if (e) ev_pool.push_back(e);
  }

  void finalize(ServeRequest* r) {
    arena_free(r->off, r->bytes);
    if (r->ev) put_event(r->ev);
    r->ev = nullptr;
    r->state = ServeRequest::kDone;
    r->t_done = now_s();
    ++n_completed;
  }

  // One pass of the scheduler (mutex held).  Returns true if anything moved.
  bool step() {
    bool moved = false;
    // (1) completions
    for (auto it = published.begin(); it != published.end();) {
      ServeRequest* r = it->second;
      ServeDone* dn = done + (r->qidx % kServeCap);
      if (*(volatile unsigned long long*)&dn->done == r->qidx + 1) {
        std::atomic_thread_fence(std::memory_order_acquire);
        const uint32_t bits = *(volatile uint32_t*)&dn->status;
        for (int k = 0; k < kOutSlots; ++k) r->out[k] = ((volatile double*)dn->out)[k];
        r->status = status_of_bits(bits);
        inflight_q.erase(r->qidx);
        it = published.erase(it);
        moved = true;
        if (r->pr.mem == LSQ_MEM_HOST) {
          r->ev = get_event();
          cudaMemcpyAsync(r->x_user, arena + r->off + r->oX, sizeof(double) * r->pr.n, cudaMemcpyDeviceToHost,
                          s_copy);
          cudaEventRecord(r->ev, s_copy);
          r->state = ServeRequest::kDraining;
          draining.push_back(r);
        } else {
          finalize(r);
        }
      } else {
        ++it;
      }
    }
    for (size_t i = 0; i < draining.size();) {
      ServeRequest* r = draining[i];
      if (cudaEventQuery(r->ev) == cudaSuccess) {
        finalize(r);
        draining[i] = draining.back();
        draining.pop_back();
        moved = true;
      } else {
        ++i;
      }
    }
    // (2) server state
    if (running && cudaEventQuery(ev_srv) == cudaSuccess) {
      running = false;
      closing = false;
    }
    // (3) admission in arrival order
    while (!pending.empty()) {
      ServeRequest* r = pending.front();
      size_t off = 0;
      if (!arena_alloc(r->bytes, &off)) break;
      pending.pop_front();
      r->off = off;
      char* slot = arena + off;
      if (r->ready) cudaStreamWaitEvent(s_copy, r->ready, 0);  // the caller's earlier work first
      r->item.slot = slot;
      if (r->pr.mem == LSQ_MEM_HOST) {
        double* Ad = reinterpret_cast<double*>(slot + r->oA);
        double* bd = reinterpret_cast<double*>(slot + r->oB);
        r->item.A = Ad;
        r->item.b = bd;
        r->item.x = reinterpret_cast<double*>(slot + r->oX);
        r->item.lda = r->pr.n;
        if (r->pr.lda == r->pr.n)
          cudaMemcpyAsync(Ad, r->pr.A, sizeof(double) * (size_t)r->pr.m * r->pr.n, cudaMemcpyHostToDevice, s_copy);
        else
          cudaMemcpy2DAsync(Ad, sizeof(double) * r->pr.n, r->pr.A, sizeof(double) * r->pr.lda,
                            sizeof(double) * r->pr.n, r->pr.m, cudaMemcpyHostToDevice, s_copy);
        cudaMemcpyAsync(bd, r->pr.b, sizeof(double) * r->pr.m, cudaMemcpyHostToDevice, s_copy);
      }
      cudaMemcpyAsync(slot + r->item.oCtl, h_zero, sizeof(ServeCtl), cudaMemcpyHostToDevice, s_copy);
      r->ev = get_event();
      cudaEventRecord(r->ev, s_copy);
      r->state = ServeRequest::kStaging;
      staging.push_back(r);
      moved = true;
    }
    // (4) publish staged requests (in order) once their copies landed
    if (!closing) {
      while (!staging.empty()) {
        ServeRequest* r = staging.front();
        if (cudaEventQuery(r->ev) != cudaSuccess) break;
        if (!inflight_q.empty() && tail >= *inflight_q.begin() + kServeCap) break;  // queue entry still in use
        staging.pop_front();
        put_event(r->ev);
        r->ev = nullptr;
        put_event(r->ready);
        r->ready = nullptr;
        r->qidx = tail;
        const uint32_t q = (uint32_t)(tail % kServeCap);
        h_items[q] = r->item;
        h_items[q].seq = tail + 1;
        h_tails[q] = tail + 1;
        cudaMemcpyAsync(d_ring + q, h_items + q, sizeof(ServeItem), cudaMemcpyHostToDevice, s_copy);
        cudaMemcpyAsync(d_tail, h_tails + q, sizeof(unsigned long long), cudaMemcpyHostToDevice, s_copy);
        ++tail;
        r->state = ServeRequest::kPublished;
        r->t_start = now_s();
        published[r->qidx] = r;
        inflight_q.insert(r->qidx);
        moved = true;
      }
    }
    // (5) launch or close the server
    const bool work = !published.empty();
    if (work && !running) {
      // the open flag and every entry published so far land before the launch
      cudaMemcpyAsync(d_closed, h_words + 0, sizeof(unsigned int), cudaMemcpyHostToDevice, s_copy);
      cudaEventRecord(ev_pub, s_copy);
      cudaStreamWaitEvent(s_srv, ev_pub, 0);
      ServeArgs a;
      a.tail = d_tail;
      a.closed = d_closed;
      a.ring = d_ring;
      a.done = d_done;
      a.qstate = d_qstate;
      a.srv_status = d_srv_status;
      a.exits = d_exits;
      a.cap = kServeCap;
      void* args[] = {&a};
      cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_serve, grid, kThreads, args, serve_smem(), s_srv);
      if (e == cudaSuccess) e = cudaEventRecord(ev_srv, s_srv);
      if (e != cudaSuccess) {
        err = std::string("server launch failed: ") + cudaGetErrorString(e);
        // fail everything published: nothing will run it
        for (auto& kv : published) {
          kv.second->status = LSQ_ERR_CUDA;
          inflight_q.erase(kv.first);
          finalize(kv.second);
        }
        published.clear();
      } else {
        running = true;
        closing = false;
        ++n_launches;
      }
      moved = true;
    }
    // close as soon as nothing is published: staged requests may be waiting
    // for other work on the GPU (their callers' streams), which cannot run
    // while the server holds every SM
    const bool idle = published.empty();
    if (running && !closing && idle) {
      if (idle_since == 0) idle_since = now_s();
      if (now_s() - idle_since > 0.002) {  // linger 2 ms, then let the blocks leave
        cudaMemcpyAsync(d_closed, h_words + 1, sizeof(unsigned int), cudaMemcpyHostToDevice, s_copy);
        closing = true;
        moved = true;
      }
    } else if (!idle) {
      idle_since = 0;
    }
    return moved;
  }

  void loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
      const bool moved = step();
      const bool busy = running || !pending.empty() || !staging.empty() || !draining.empty();
      if (moved) continue;
      if (busy) {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      } else {
        cv.wait_for(lk, std::chrono::milliseconds(50));
      }
    }
    // shut down: close the server and let it drain (published work completes)
    cudaMemcpyAsync(d_closed, h_words + 1, sizeof(unsigned int), cudaMemcpyHostToDevice, s_copy);
  }
};

void server_set_wait_limit(Server* s, uint32_t limit_us) {
  if (s && s->h_zero) reinterpret_cast<volatile uint32_t*>(&reinterpret_cast<ServeCtl*>(s->h_zero)->bar.limit_us)[0] = limit_us;
}

void server_destroy(Server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  cudaSetDevice(s->device);
  if (s->s_copy) cudaStreamSynchronize(s->s_copy);
  if (s->s_srv) cudaStreamSynchronize(s->s_srv);  // bounded: idle blocks leave once closed
  for (auto& kv : s->tickets) {
    if (kv.second->ev) cudaEventDestroy(kv.second->ev);
    if (kv.second->ready) cudaEventDestroy(kv.second->ready);
    delete kv.second;
  }
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  if (s->ev_srv) cudaEventDestroy(s->ev_srv);
  if (s->ev_pub) cudaEventDestroy(s->ev_pub);
  if (s->s_srv) cudaStreamDestroy(s->s_srv);
  if (s->s_copy) cudaStreamDestroy(s->s_copy);
  if (s->arena) cudaFree(s->arena);
  if (s->d_q) cudaFree(s->d_q);
  if (s->hmem) cudaFreeHost(s->hmem);
  if (s->h_pin) cudaFreeHost(s->h_pin);
  delete s;
}

namespace {

lsq_status server_create(lsq_ctx* ctx, Server** out) {
  Server* s = new Server();
  s->ctx = ctx;
  s->device = ctx->device;
  if (ctx->serve_cta_bytes > 0) s->cta_bytes = ctx->serve_cta_bytes;
  s->max_group = ctx->serve_max_group;
  size_t want = ctx->serve_arena ? ctx->serve_arena : (ctx->budget > ctx->ws_size ? ctx->budget - ctx->ws_size : 0);
  want = want / 256 * 256;
  auto bail = [&](lsq_status st, const std::string& m) {
    ctx->err = m;
    server_destroy(s);
    return st;
  };
  if (want < (1u << 20)) return bail(LSQ_ERR_BUDGET, "serving arena below 1 MiB");
  if (cudaFuncSetAttribute(k_serve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)serve_smem()) != cudaSuccess)
    return bail(LSQ_ERR_CUDA, "server kernel: shared memory attribute refused");
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_serve, kThreads, serve_smem()) != cudaSuccess ||
      per_sm < 1)
    return bail(LSQ_ERR_CUDA, "server kernel does not fit an SM");
  if (per_sm > 2) per_sm = 2;
  s->grid = per_sm * ctx->sms;
  if (s->max_group <= 0 || s->max_group > s->grid) s->max_group = s->max_group > 0 ? s->grid : s->grid / 8;
  if (s->max_group < 1) s->max_group = 1;
  if (cudaMalloc(&s->arena, want) != cudaSuccess) {
    cudaGetLastError();
    return bail(LSQ_ERR_OOM, "serving arena allocation failed");
  }
  s->arena_bytes = want;
  s->free_blocks[0] = want;
  const size_t qbytes = 256 + sizeof(ServeItem) * kServeCap;
  if (cudaMalloc(&s->d_q, qbytes) != cudaSuccess) return bail(LSQ_ERR_OOM, "server queue");
  cudaMemset(s->d_q, 0, qbytes);
  s->d_tail = reinterpret_cast<unsigned long long*>(s->d_q);
  s->d_closed = reinterpret_cast<unsigned int*>(s->d_q + 8);
  s->d_qstate = reinterpret_cast<unsigned long long*>(s->d_q + 64);
  s->d_srv_status = reinterpret_cast<uint32_t*>(s->d_q + 128);
  s->d_exits = reinterpret_cast<unsigned int*>(s->d_q + 192);
  s->d_ring = reinterpret_cast<ServeItem*>(s->d_q + 256);
  const size_t pbytes = sizeof(ServeItem) * kServeCap + sizeof(unsigned long long) * kServeCap + 256 + 4096;
  if (cudaHostAlloc(&s->h_pin, pbytes, cudaHostAllocDefault) != cudaSuccess) return bail(LSQ_ERR_OOM, "pinned queue");
  std::memset(s->h_pin, 0, pbytes);
  s->h_items = reinterpret_cast<ServeItem*>(s->h_pin);
  s->h_tails = reinterpret_cast<unsigned long long*>(s->h_pin + sizeof(ServeItem) * kServeCap);
  s->h_words = reinterpret_cast<unsigned int*>(s->h_pin + sizeof(ServeItem) * kServeCap +
                                               sizeof(unsigned long long) * kServeCap);
  s->h_words[0] = 0u;
  s->h_words[1] = 1u;
  s->h_zero = s->h_pin + sizeof(ServeItem) * kServeCap + sizeof(unsigned long long) * kServeCap + 256;
  server_set_wait_limit(s, ctx->wait_limit_us);
  const size_t hbytes = sizeof(ServeDone) * kServeCap;
  if (cudaHostAlloc(&s->hmem, hbytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess)
    return bail(LSQ_ERR_OOM, "mapped completion records");
  std::memset(s->hmem, 0, hbytes);
  s->done = reinterpret_cast<ServeDone*>(s->hmem);
  void* dp = nullptr;
  if (cudaHostGetDevicePointer(&dp, s->hmem, 0) != cudaSuccess) return bail(LSQ_ERR_CUDA, "mapped record pointer");
  s->d_done = reinterpret_cast<ServeDone*>(dp);
  if (cudaStreamCreateWithFlags(&s->s_srv, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->s_copy, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_srv, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_pub, cudaEventDisableTiming) != cudaSuccess)
    return bail(LSQ_ERR_CUDA, "server streams");
  if (cudaDeviceSynchronize() != cudaSuccess) return bail(LSQ_ERR_CUDA, "server setup");
  s->th = std::thread([s] { s->loop(); });
  *out = s;
  return LSQ_OK;
}

// Slot layout and group size of a request; false if it cannot be served.
void plan_request(ServeRequest* r, int max_group, double cta_bytes, const BatchTuning* tune) {
  const int64_t m = r->pr.m, n = r->pr.n, d = r->o.d;
  const int64_t npad = (n + 31) / 32 * 32, ldi = (n + 1) / 2 * 2, ncol = n + 1;
  const double abytes = 8.0 * (double)m * (double)n;
  const double qr_flops = 2.0 * (double)d * (double)ncol * (double)ncol;
  int64_t G = (int64_t)std::ceil(abytes / cta_bytes);
  const int64_t Gq = (int64_t)std::ceil(qr_flops / 2.5e8);  // ~40 ms of one SM's FP64 per block
  if (Gq > G) G = Gq;
  const int64_t rows_cap = (m + 31) / 32;  // at least one 32-row sketch block per block
  if (G > rows_cap) G = rows_cap;
  if (G < 1) G = 1;
  if (G > max_group) G = max_group;
  ServeItem& it = r->item;
  it.A = r->pr.A;
  it.b = r->pr.b;
  it.x = r->x_user;
  it.m = m;
  it.lda = r->pr.lda;
  it.n = (int32_t)n;
  it.d = (int32_t)d;
  it.zeta = r->o.zeta;
  it.variant = variant_for((int)n, tune);
  it.G = (int32_t)G;
  it.mode = (r->o.flags & LSQ_FLAG_NO_CHECK) ? 2 : 0;
  it.seed = r->o.seed;
  it.tol = r->o.tol;
  it.maxit = r->o.maxit;
  it.gate = it.mode == 0 ? (r->o.gate < 0.0 ? 0.0 : r->o.gate > 0.0 ? r->o.gate : std::max(1e-10, r->o.tol)) : 0.0;
  it.npad = npad;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += al256(bytes);
    return (uint64_t)at;
  };
  it.oCtl = take(sizeof(ServeCtl));
  it.oY = take((size_t)d * ncol * 8);
  it.oW = take((size_t)d * ncol * 8);
  it.oR = take((size_t)n * n * 8);
  it.oM = take((size_t)n * n * 8);
  it.oMt = take((size_t)n * n * 8);
  it.oRd = take((size_t)npad * 8);
  it.oU = take((size_t)m * 8);
  it.oVec = take((size_t)5 * npad * 8);
  it.oGpart = take((size_t)G * kWarps * npad * 8);
  it.oPart = take((size_t)G * 4 * 8);
  it.oImg = take((size_t)m * ldi * 8);
  if (r->pr.mem == LSQ_MEM_HOST) {
    r->oA = take((size_t)m * n * 8);
    r->oB = take((size_t)m * 8);
    r->oX = take((size_t)npad * 8);
  }
  r->bytes = o;
}

}  // namespace
}  // namespace lsq

using namespace lsq;

extern "C" {

lsq_status lsq_serve_config(lsq_ctx* ctx, size_t arena_bytes, double cta_bytes, int32_t max_group) {
  if (!ctx) return LSQ_ERR_ARG;
  if (ctx->server) {
    ctx->err = "serving is already running on this context";
    return LSQ_ERR_ARG;
  }
  if (cta_bytes < 0 || max_group < 0) {
    ctx->err = "cta_bytes and max_group must be >= 0";
    return LSQ_ERR_ARG;
  }
  ctx->serve_arena = arena_bytes;
  ctx->serve_cta_bytes = cta_bytes;
  ctx->serve_max_group = max_group;
  return LSQ_OK;
}

lsq_status lsq_submit(lsq_ctx* ctx, const lsq_problem* pr, const lsq_opts* o, double* x, lsq_ticket* out,
                      void* stream) {
  if (!ctx) return LSQ_ERR_ARG;
  if (!pr || !o || !x || !out) {
    ctx->err = "null problem, options, x or ticket";
    return LSQ_ERR_ARG;
  }
  *out = 0;
  const int64_t m = pr->m, n = pr->n, lda = pr->lda, d = o->d;
  if (m < 1 || n < 1 || lda < n || !pr->A || !pr->b) {
    ctx->err = "need m, n >= 1, lda >= n, A, b";
    return LSQ_ERR_ARG;
  }
  if (o->zeta < 1 || o->zeta > kGroupZeta || (int64_t)o->zeta > d) {
    ctx->err = "serving takes 1 <= zeta <= min(8, d)";
    return LSQ_ERR_ARG;
  }
  if (d < n + 1 || d > 2147483647LL) {
    ctx->err = "need n + 1 <= d <= 2^31-1";
    return LSQ_ERR_ARG;
  }
  if (pr->mem != LSQ_MEM_DEVICE && pr->mem != LSQ_MEM_HOST) {
    ctx->err = "unknown memory kind";
    return LSQ_ERR_ARG;
  }
  if (n > kServeMaxN || o->prec != LSQ_PREC_FP64 || (o->flags & LSQ_FLAG_NATIVE_FP64)) {
    ctx->err = "serving is built for the FP64 form with n <= 1024";
    return LSQ_ERR_UNSUPPORTED;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    ctx->err = "cudaSetDevice failed";
    return LSQ_ERR_CUDA;
  }
  if (!ctx->server) {
    lsq_status s = server_create(ctx, &ctx->server);
    if (s != LSQ_OK) {
      ctx->server = nullptr;
      return s;
    }
  }
  Server* srv = ctx->server;
  ServeRequest* r = new ServeRequest();
  r->pr = *pr;
  r->o = *o;
  r->x_user = x;
  plan_request(r, srv->max_group, srv->cta_bytes, ctx->tuning);
  if (r->bytes > srv->arena_bytes) {
    ctx->err = "request needs " + std::to_string(r->bytes) + " bytes; the serving arena holds " +
               std::to_string(srv->arena_bytes);
    delete r;
    return LSQ_ERR_BUDGET;
  }
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    {
      r->ready = srv->get_event();
      if (!r->ready || cudaEventRecord(r->ready, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        if (r->ready) srv->put_event(r->ready);
        delete r;
        ctx->err = "could not record the ordering event on the caller's stream";
        return LSQ_ERR_CUDA;
      }
    }
    r->ticket = srv->next_ticket++;
    r->t_submit = now_s();
    srv->tickets[r->ticket] = r;
    srv->pending.push_back(r);
    ++srv->n_submitted;
    *out = r->ticket;
  }
  srv->cv.notify_all();
  return LSQ_OK;
}

lsq_status lsq_poll(lsq_ctx* ctx, lsq_ticket ticket, lsq_info* info) {
  if (!ctx) return LSQ_ERR_ARG;
  Server* srv = ctx->server;
  if (!srv) {
    ctx->err = "no request was submitted on this context";
    return LSQ_ERR_ARG;
  }
  ServeRequest* r = nullptr;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->tickets.find(ticket);
    if (it == srv->tickets.end()) {
      ctx->err = "unknown ticket";
      return LSQ_ERR_ARG;
    }
    r = it->second;
    if (r->state != ServeRequest::kDone) return LSQ_PENDING;
    srv->tickets.erase(it);
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->status = r->status;
    info->iters = (int64_t)r->out[OUT_ITERS];
    info->stop = (int32_t)r->out[OUT_STOP];
    info->normal_rel_est = r->out[OUT_NORMAL_REL];
    info->backward_error_ne = r->out[OUT_ETA_NE];
    info->backward_error_pre = r->out[OUT_ETA_PRE];
    info->rnorm = r->out[OUT_RNORM];
    info->arnorm = r->out[OUT_ARNORM];
    info->anorm_fro = r->out[OUT_FRO];
    info->xnorm = r->out[OUT_XNORM];
    info->bnorm = r->out[OUT_BNORM];
    info->t_submit_s = r->t_submit;
    info->t_start_s = r->t_start;
    info->t_done_s = r->t_done;
    info->group_blocks = r->item.G;
    const double* t = r->out;
    if (t[OUT_T_START] > 0) info->t_group_wait_ms = (float)((t[OUT_T_START] - t[OUT_T_JOIN]) * 1e-6);
    if (t[OUT_T_SKETCH] > 0) info->t_sketch_ms = (float)((t[OUT_T_SKETCH] - t[OUT_T_START]) * 1e-6);
    if (t[OUT_T_PRECOND] > 0) info->t_precond_ms = (float)((t[OUT_T_PRECOND] - t[OUT_T_SKETCH]) * 1e-6);
    if (t[OUT_T_END] > 0) info->t_lsqr_ms = (float)((t[OUT_T_END] - t[OUT_T_PRECOND]) * 1e-6);
  }
  const lsq_status s = r->status;
  delete r;
  return s;
}

lsq_status lsq_serve_stats_get(lsq_ctx* ctx, lsq_serve_stats* out) {
  if (!ctx || !out) return LSQ_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  Server* srv = ctx->server;
  if (!srv) return LSQ_OK;
  std::lock_guard<std::mutex> lk(srv->mu);
  out->submitted = srv->n_submitted;
  out->completed = srv->n_completed;
  out->pending = (int64_t)(srv->pending.size() + srv->staging.size());
  out->in_flight = (int64_t)(srv->published.size() + srv->draining.size());
  out->server_launches = srv->n_launches;
  out->grid_blocks = srv->grid;
  out->arena_bytes = srv->arena_bytes;
  out->arena_peak_bytes = srv->arena_peak;
  return LSQ_OK;
}

}  // extern "C"
