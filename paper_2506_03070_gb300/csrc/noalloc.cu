// noalloc.cu -- lsq_check_noalloc: the accuracy pass of lsq_check for callers
// that cannot allocate device memory.
//
// Who needs it: code that runs where it may not call cudaMalloc -- inside a
// framework whose caching allocator owns all device memory, in a process with
// a fixed memory plan decided at start-up, or in latency-critical loops where
// an allocation (which can synchronise the device) is not acceptable.  Such
// callers cannot create an lsq_ctx either (lsq_create allocates), so this entry
// point takes no context.
//
// All of its scratch lives in the file-scope array below, which every GPU that
// loads the library holds for the life of the process (about 4.1 MB).  The
// caller passes only inputs and outputs.  Host code never uses the array's
// name as an address: the device address comes from cudaGetSymbolAddress,
// looked up once per device (and per driver context, for callers that make
// their own context current), with that device current, on the first call
// made there (make that first call before any stream capture).  Every call on a
// device reuses the same array and leaves its contents behind; the barrier
// and status words are cleared at the start of each call and every other
// region is fully rewritten before it is read.  Two calls whose work overlaps
// on the GPU (different streams, or different host threads) race on the
// array: serialise them.
#include <cstring>
#include <mutex>

#include "kernels.h"

namespace lsq {
namespace {

constexpr int kNoallocMaxN = 512;      // columns of A
constexpr int kNoallocMaxGrid = 512;   // co-resident blocks of the pass kernel
constexpr int kNoallocMaxDevices = 64;

// Layout of the scratch array (bytes, 256-aligned regions).
constexpr size_t kOffSmall = 0;                                                // status, barrier, out: 4 KB
constexpr size_t kOffVec = 4096;                                               // 5 vectors of kNoallocMaxN
constexpr size_t kOffPart = kOffVec + 5 * kNoallocMaxN * sizeof(double);       // kNoallocMaxGrid x 4
constexpr size_t kOffGpart = kOffPart + (size_t)kNoallocMaxGrid * 4 * sizeof(double);
constexpr size_t kOffMt = kOffGpart + (size_t)kNoallocMaxGrid * kNoallocMaxN * sizeof(double);
constexpr size_t kScratchBytes = kOffMt + (size_t)kNoallocMaxN * kNoallocMaxN * sizeof(double);

static __device__ __align__(256) unsigned char g_check_scratch[kScratchBytes];

std::mutex g_setup_mutex;
// (device, CUDA context) -> device address of g_check_scratch in that context.
// The runtime uses the device's primary context unless the caller made
// another context current through the driver API; the array has a separate
// copy (and address) in every context that loaded the library.
struct ScratchEntry {
  int dev;
  void* cuctx;
  void* addr;
};
ScratchEntry g_entries[kNoallocMaxDevices];
int g_nentries = 0;

// The current driver context (cuCtxGetCurrent through the runtime's entry
// point query: the library links no driver library).
void* current_cuctx() {
  typedef int (*GetCurrent)(void**);
  static GetCurrent fn = nullptr;
  static bool looked = false;
  if (!looked) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<GetCurrent>(f);
    looked = true;
  }
  void* c = nullptr;
  if (fn && fn(&c) != 0) c = nullptr;
  return c;
}

// Device address of g_check_scratch for the current device and context
// (looked up once per pair, with that device current).
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  void* cctx = current_cuctx();
  for (int i = 0; i < g_nentries; ++i)
    if (g_entries[i].dev == dev && g_entries[i].cuctx == cctx) {
      *out = g_entries[i].addr;
      return cudaSuccess;
    }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_check_scratch);
  if (e != cudaSuccess) return e;
  if (g_nentries < kNoallocMaxDevices) g_entries[g_nentries++] = ScratchEntry{dev, cctx, p};
  *out = p;
  return cudaSuccess;
}

}  // namespace
}  // namespace lsq

using namespace lsq;

extern "C" lsq_status lsq_check_noalloc(const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                                        const double* x, const double* M, lsq_info* info, void* stream) {
  if (m < 1 || n < 1 || lda < n || !A || !b || !x) return LSQ_ERR_ARG;
  if (n > kNoallocMaxN) return LSQ_ERR_ARG;  // beyond the static scratch
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return LSQ_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LSQ_ERR_CUDA;
  const int ni = (int)n, npad = (int)((n + 31) / 32 * 32);
  const bool vec = ((uintptr_t)A % 16 == 0) && (lda % 2 == 0);
  const int grid = lsqr_grid(ni, vec, true, sms);
  if (grid < 1 || grid > kNoallocMaxGrid) return LSQ_ERR_UNSUPPORTED;
  void* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess) return LSQ_ERR_CUDA;
  char* s = static_cast<char*>(base);
  cudaStream_t st = (cudaStream_t)stream;

  uint32_t* status = reinterpret_cast<uint32_t*>(s + kOffSmall);
  GridBarrier* bar = reinterpret_cast<GridBarrier*>(s + kOffSmall + 128);
  double* out = reinterpret_cast<double*>(s + kOffSmall + 256);
  double* vecs = reinterpret_cast<double*>(s + kOffVec);
  LsqrParams p;
  p.A = A;
  p.m = m;
  p.n = ni;
  p.npad = npad;
  p.lda = lda;
  p.b = b;
  p.M = M;
  p.Mt = M ? reinterpret_cast<double*>(s + kOffMt) : nullptr;
  p.x = const_cast<double*>(x);  // read only in the check pass
  p.u = nullptr;                 // not touched by the check pass
  p.v = vecs;
  p.vhat = vecs + kNoallocMaxN;
  p.w = vecs + 2 * kNoallocMaxN;
  p.wv = vecs + 3 * kNoallocMaxN;
  p.g = vecs + 4 * kNoallocMaxN;
  p.part = reinterpret_cast<double*>(s + kOffPart);
  p.gpart = reinterpret_cast<double*>(s + kOffGpart);
  p.tol = 0.0;
  p.maxit = 0;
  p.mode = 1;
  p.asplit = nullptr;
  p.ldi = (n + 1) / 2 * 2;
  p.vec = vec;
  p.a_ring = false;
  p.ring_k = 1;
  p.range = nullptr;
  p.gate = 0.0;
  p.fro_in = nullptr;
  p.bar = bar;
  p.status = status;
  p.out = out;

  // status, barrier and result words start at zero on every call
  if (cudaMemsetAsync(s + kOffSmall, 0, 4096, st) != cudaSuccess) return LSQ_ERR_CUDA;
  if (M && transpose_square(M, ni, const_cast<double*>(p.Mt), st) != cudaSuccess) return LSQ_ERR_CUDA;
  if (lsqr_run(p, vec, true, grid, st) != cudaSuccess) return LSQ_ERR_CUDA;
  uint32_t bits = 0;
  double h_out[kOutSlots];
  if (cudaMemcpyAsync(&bits, status, sizeof(bits), cudaMemcpyDeviceToHost, st) != cudaSuccess) return LSQ_ERR_CUDA;
  if (cudaMemcpyAsync(h_out, out, sizeof(h_out), cudaMemcpyDeviceToHost, st) != cudaSuccess) return LSQ_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return LSQ_ERR_CUDA;
  lsq_status rc = LSQ_OK;
  if (bits & DS_TIMEOUT) rc = LSQ_ERR_TIMEOUT;
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->status = rc;
    info->backward_error_ne = h_out[OUT_ETA_NE];
    info->backward_error_pre = h_out[OUT_ETA_PRE];
    info->rnorm = h_out[OUT_RNORM];
    info->arnorm = h_out[OUT_ARNORM];
    info->anorm_fro = h_out[OUT_FRO];
    info->xnorm = h_out[OUT_XNORM];
    info->bnorm = h_out[OUT_BNORM];
  }
  return rc;
}
