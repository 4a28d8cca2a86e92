// api.cu -- the C ABI declared in include/lsq.h: context, workspace under an
// HBM budget, argument checking, status mapping and the Algorithm 1 chain
// sketch -> preconditioner -> LSQR -> accuracy pass on one stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>
#include <cstring>
#include <string>

#include "ctx.h"

using namespace lsq;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kSmallBytes = 4096;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

lsq_status fail(lsq_ctx* c, lsq_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}
lsq_status cuda_fail(lsq_ctx* c, cudaError_t e, const char* where) {
  return fail(c, e == cudaErrorMemoryAllocation ? LSQ_ERR_OOM : LSQ_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}
#define CK(call)                                        \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

// CUDA events destroyed on every return path.
template <int N>
struct Events {
  cudaEvent_t e[N] = {};
  cudaError_t create() {
    for (auto& x : e)
      if (cudaError_t r = cudaEventCreate(&x); r != cudaSuccess) return r;
    return cudaSuccess;
  }
  cudaEvent_t& operator[](int i) { return e[i]; }
  ~Events() {
    for (auto x : e)
      if (x) cudaEventDestroy(x);
  }
};

struct Carver {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += align_up(count * sizeof(T));
    return p;
  }
};

lsq_status ensure_ws(lsq_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_size) return LSQ_OK;
  if (bytes > ctx->budget)
    return fail(ctx, LSQ_ERR_BUDGET,
                "workspace of " + std::to_string(bytes) + " bytes exceeds the HBM budget of " +
                    std::to_string(ctx->budget));
  if (ctx->ws) {
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_size = 0;
  }
  cudaError_t e = cudaMalloc(&ctx->ws, bytes);
  if (e != cudaSuccess) {
    ctx->ws = nullptr;
    cudaGetLastError();
    return fail(ctx, LSQ_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  ctx->ws_size = bytes;
  return LSQ_OK;
}

lsq_status status_from_bits(lsq_ctx* ctx, uint32_t bits) {
  if (bits & DS_TIMEOUT) return fail(ctx, LSQ_ERR_TIMEOUT, "a device-side wait gave up (grid barrier or bulk copy)");
  if (bits & DS_NONFINITE) return fail(ctx, LSQ_ERR_NONFINITE, "A or b contains NaN or Inf");
  if (bits & DS_SKETCH) return fail(ctx, LSQ_ERR_SKETCH, "rejection sampling exceeded its round cap");
  if (bits & DS_RANK) return fail(ctx, LSQ_ERR_RANK, "R has a negligible diagonal entry (rank-deficient sketch)");
  if (bits & DS_NOCONV) return fail(ctx, LSQ_ERR_NOCONV, "LSQR reached maxit before the stopping test held");
  if (bits & DS_ACCURACY)
    return fail(ctx, LSQ_ERR_ACCURACY, "the accuracy pass's backward-error bound exceeds the gate (x is written)");
  return LSQ_OK;
}

// Gate of the accuracy pass for a solve with tolerance tol: the gate in
// opts when set (> 0; < 0 disables it), else max(1e-10, tol).
double solve_gate(double tol, double opt_gate) {
  if (opt_gate < 0.0) return 0.0;
  if (opt_gate > 0.0) return opt_gate;
  return std::max(1e-10, tol);
}

lsq_status check_ctx(lsq_ctx* ctx) {
  if (!ctx) return LSQ_ERR_ARG;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  return LSQ_OK;
}

lsq_status check_sketch_args(lsq_ctx* ctx, int64_t d, int32_t zeta) {
  if (zeta < 1 || zeta > kMaxZeta) return fail(ctx, LSQ_ERR_ARG, "zeta must be in [1, 64]");
  if (d < 1 || d > 2147483647LL) return fail(ctx, LSQ_ERR_ARG, "d must be in [1, 2^31-1]");
  if ((int64_t)zeta > d) return fail(ctx, LSQ_ERR_ARG, "zeta must not exceed d");
  return LSQ_OK;
}

// reset the small device words on the stream, except the barrier's wait
// limit (a context setting, lsq_set_wait_limit)
lsq_status reset_small(lsq_ctx* ctx, cudaStream_t st) {
  char* base = reinterpret_cast<char*>(ctx->d_status);
  const size_t lim = reinterpret_cast<char*>(&ctx->d_bar->limit_us) - base;
  CK(cudaMemsetAsync(base, 0, lim, st));
  CK(cudaMemsetAsync(base + lim + sizeof(uint32_t), 0, kSmallBytes - lim - sizeof(uint32_t), st));
  return LSQ_OK;
}

// copy status + max_rounds + out back and synchronise
lsq_status read_small(lsq_ctx* ctx, cudaStream_t st, uint32_t* bits, int32_t* rounds, double* out) {
  CK(cudaMemcpyAsync(ctx->h_small, ctx->d_status, kSmallBytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const char* h = static_cast<const char*>(ctx->h_small);
  const size_t off_rounds = (const char*)ctx->d_max_rounds - (const char*)ctx->d_status;
  const size_t off_out = (const char*)ctx->d_out - (const char*)ctx->d_status;
  if (bits) std::memcpy(bits, h, sizeof(uint32_t));
  if (rounds) std::memcpy(rounds, h + off_rounds, sizeof(int32_t));
  if (out) std::memcpy(out, h + off_out, sizeof(double) * kOutSlots);
  return LSQ_OK;
}

bool vec_ok(const double* A, int64_t lda) { return ((uintptr_t)A % 16 == 0) && (lda % 2 == 0); }

// The address at which kernels read host memory p, when p lies in pinned or
// registered host memory (page-locked, mapped into the device's address
// space); nullptr for pageable memory, which is copied instead.
const void* host_device_view(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

int64_t default_maxit(int64_t n, int64_t d, double tol) {
  const double rate = std::sqrt((double)n / (double)d);
  if (!(tol > 0.0) || !(rate < 1.0)) return 1000;
  return (int64_t)(10.0 * std::ceil(std::log(tol) / std::log(rate)));
}

struct LsqrWork {
  double *u, *v, *vhat, *w, *wv, *g, *gpart, *part, *Mt;
  float2* image;  // (hi, mid) float-pair image of A for the double-float pass, or null
};

LsqrWork carve_lsqr(Carver& cv, int64_t m, int n, int npad, int grid, bool image = false) {
  LsqrWork w;
  w.image = image ? cv.take<float2>((size_t)m * ((n + 1) / 2 * 2)) : nullptr;
  w.u = cv.take<double>((size_t)m);
  w.v = cv.take<double>(npad);
  w.vhat = cv.take<double>(npad);
  w.w = cv.take<double>(npad);
  w.wv = cv.take<double>(npad);
  w.g = cv.take<double>(npad);
  w.gpart = cv.take<double>((size_t)lsqr_gparts(grid) * npad);
  w.part = cv.take<double>((size_t)grid * 4);
  w.Mt = cv.take<double>((size_t)n * n);
  return w;
}

void fill_info(lsq_info* info, const double* out, lsq_status st, int32_t rounds) {
  if (!info) return;
  std::memset(info, 0, sizeof(*info));
  info->status = st;
  info->iters = (int64_t)out[OUT_ITERS];
  info->stop = (int32_t)out[OUT_STOP];
  info->normal_rel_est = out[OUT_NORMAL_REL];
  info->backward_error_ne = out[OUT_ETA_NE];
  info->backward_error_pre = out[OUT_ETA_PRE];
  info->rnorm = out[OUT_RNORM];
  info->arnorm = out[OUT_ARNORM];
  info->anorm_fro = out[OUT_FRO];
  info->xnorm = out[OUT_XNORM];
  info->bnorm = out[OUT_BNORM];
  info->sketch_rounds_max = rounds;
  if (out[OUT_T_CHECK1] > out[OUT_T_CHECK0] && out[OUT_T_CHECK0] > 0.0)
    info->t_check_ms = (float)((out[OUT_T_CHECK1] - out[OUT_T_CHECK0]) * 1e-6);
}

// Launch the LSQR / check kernel (native: FP64-pipe pass; else double-float pass).
lsq_status run_lsqr(lsq_ctx* ctx, const double* A, int64_t m, int n, int64_t lda, const double* b, const double* M,
                    const double* Mt, double* x, double tol, int64_t maxit, int mode, const LsqrWork& w, int grid,
                    int npad, bool native, cudaStream_t st, double hbm_alpha = 0.0, double hbm_beta = 0.0,
                    double gate = 0.0, const double* fro_in = nullptr) {
  LsqrParams p;
  p.A = A;
  p.m = m;
  p.n = n;
  p.npad = npad;
  p.lda = lda;
  p.b = b;
  p.asplit = native ? nullptr : w.image;
  p.ldi = (n + 1) / 2 * 2;
  p.vec = vec_ok(A, lda);
  p.a_ring = p.vec && (n % 2 == 0);
  p.ring_k = 1;
  p.range = ctx->d_range;
  p.gate = gate;
  p.fro_in = fro_in;
  p.M = M;
  p.Mt = Mt;
  p.x = x;
  p.u = w.u;
  p.v = w.v;
  p.vhat = w.vhat;
  p.w = w.w;
  p.wv = w.wv;
  p.g = w.g;
  p.gpart = w.gpart;
  p.part = w.part;
  p.tol = tol;
  p.maxit = maxit;
  p.mode = mode;
  p.hbm_alpha = hbm_alpha;
  p.hbm_beta = hbm_beta;
  p.bar = ctx->d_bar;
  p.status = ctx->d_status;
  p.out = ctx->d_out;
  CK(cudaMemsetAsync(&ctx->d_bar->count, 0, sizeof(unsigned int), st));
  CK(lsqr_run(p, vec_ok(A, lda), native, grid, st));
  return LSQ_OK;
}

// ---------------------------------------------------------------------------
// Embedding dimension (Sec. 4.3 "Selecting the embedding dimension").  The
// solve time is modelled as T(d) = T_qr(d) + (t(d) + 2) T_iter(m) with the
// Sec. 4.3 rate estimate (n/d)^{t/2} <= tol, i.e. t(d) = 2 |ln tol| / ln(d/n)
// iterations, a preconditioner cost linear in d (t_qr_per_d per sketch row)
// and an iteration cost linear in m (t_iter_per_row).  The constants are this
// GPU's, measured by calibrate_d on synthetic data of the problem's width.
// ---------------------------------------------------------------------------
lsq_status calibrate_d(lsq_ctx* ctx, int64_t n64, lsq_ctx::DCalib* out) {
  auto it = ctx->dcalib.find(n64);
  if (it != ctx->dcalib.end()) {
    *out = it->second;
    return LSQ_OK;
  }
  const int n = (int)n64, npad = (int)((n64 + 31) / 32 * 32), ncol = n + 1;
  int64_t mc = (int64_t)1 << 18;
  const int64_t mmax = ((int64_t)1 << 30) / (8 * n64);
  if (mc > mmax) mc = mmax;
  if (mc < 8192) mc = 8192;
  const int64_t d1 = std::max<int64_t>(n64 + 1, 2 * n64), d2 = std::max<int64_t>(8 * n64, d1 + n64);
  const bool native = !lsqr_df_ok(nullptr, n64, n64);
  const int grid = lsqr_grid(n, n % 2 == 0, native, ctx->sms);
  if (grid < 1) return fail(ctx, LSQ_ERR_CUDA, "no launchable LSQR configuration");
  auto carve = [&](Carver& cv, double** A, double** b, double** x, double** M, LsqrWork* lw, double** Y,
                   PrecondBuffers* pb, double** R2, double** M2, double** x0) {
    *A = cv.take<double>((size_t)mc * n);
    *b = cv.take<double>((size_t)mc);
    *x = cv.take<double>(npad);
    *M = cv.take<double>((size_t)n * n);
    *lw = carve_lsqr(cv, mc, n, npad, grid, !native);
    *Y = cv.take<double>((size_t)d2 * ncol);
    pb->W = cv.take<double>((size_t)d2 * ncol);
    pb->rdiag = cv.take<double>(npad);
    pb->R = cv.take<double>((size_t)n * n);
    pb->Mt = cv.take<double>((size_t)n * n);
    pb->blk = cv.take<char>(precond_blocked_bytes(d2, n));
    *R2 = cv.take<double>((size_t)n * n);
    *M2 = cv.take<double>((size_t)n * n);
    *x0 = cv.take<double>(npad);
  };
  double *A, *b, *x, *M, *Y, *R2, *M2, *x0;
  LsqrWork lw;
  PrecondBuffers pb;
  {
    Carver probe{nullptr};
    carve(probe, &A, &b, &x, &M, &lw, &Y, &pb, &R2, &M2, &x0);
    lsq_status s = ensure_ws(ctx, probe.off);
    if (s != LSQ_OK) return s;
  }
  Carver cv{ctx->ws};
  carve(cv, &A, &b, &x, &M, &lw, &Y, &pb, &R2, &M2, &x0);
  pb.bar = ctx->d_bar;
  pb.status = ctx->d_status;
  pb.mode = ctx->qr_mode;
  cudaStream_t st = nullptr;
  CK(fill_hash(A, mc, n, n, 11, ctx->sms, st));
  CK(fill_hash(b, mc, 1, 1, 12, ctx->sms, st));
  CK(fill_identity(M, n, ctx->sms, st));
  CK(transpose_square(M, n, lw.Mt, st));
  Events<2> ce;
  CK(ce.create());
  cudaEvent_t e0 = ce[0], e1 = ce[1];
  auto timed = [&](auto&& fn) -> float {
    float ms = -1.f;
    if (cudaEventRecord(e0, st) != cudaSuccess) return ms;
    if (fn() != LSQ_OK) return ms;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return ms;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  auto lsqr_k = [&](int64_t k) {
    lsq_status s = reset_small(ctx, st);
    if (s != LSQ_OK) return s;
    if (cudaMemsetAsync(x, 0, sizeof(double) * npad, st) != cudaSuccess) return LSQ_ERR_CUDA;
    return run_lsqr(ctx, A, mc, n, n, b, M, lw.Mt, x, 0.0, k, 2, lw, grid, npad, native, st);
  };
  auto qr_d = [&](int64_t d) {
    if (fill_hash(Y, d, ncol, ncol, 13, ctx->sms, st) != cudaSuccess) return LSQ_ERR_CUDA;
    if (reset_small(ctx, st) != LSQ_OK) return LSQ_ERR_CUDA;
    return precond<double>(Y, d, n, ncol, 1, R2, M2, x0, pb, ctx->sms, st) == cudaSuccess ? LSQ_OK
                                                                                          : LSQ_ERR_CUDA;
  };
  timed([&] { return lsqr_k(1); });  // warm-up (module load, image)
  const float t2 = timed([&] { return lsqr_k(2); });
  const float t6 = timed([&] { return lsqr_k(6); });
  timed([&] { return qr_d(d1); });
  const float q1 = timed([&] { return qr_d(d1); });
  const float q2 = timed([&] { return qr_d(d2); });
  if (t2 < 0 || t6 < 0 || q1 < 0 || q2 < 0) return fail(ctx, LSQ_ERR_CUDA, "embedding-dimension calibration failed");
  lsq_ctx::DCalib cal;
  cal.t_iter_per_row = std::max(1e-15, (double)(t6 - t2) * 1e-3 / 4.0 / (double)mc);
  // the QR's cost per extra sketch row, floored at its FP64 flop time (2 n^2 at ~1 TFLOP/s)
  cal.t_qr_per_d = std::max(2.0 * (double)n * n * 1e-12, (double)(q2 - q1) * 1e-3 / (double)(d2 - d1));
  ctx->dcalib[n64] = cal;
  *out = cal;
  return reset_small(ctx, st);
}

}  // namespace

extern "C" {

lsq_status lsq_create(lsq_ctx** out, int device, size_t hbm_budget_bytes) {
  if (!out) return LSQ_ERR_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return LSQ_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return LSQ_ERR_CUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return LSQ_ERR_CUDA;
  if (!prop.cooperativeLaunch) return LSQ_ERR_CUDA;
  lsq_ctx* ctx = new lsq_ctx();
  ctx->device = device;
  ctx->sms = prop.multiProcessorCount;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    delete ctx;
    return LSQ_ERR_CUDA;
  }
  ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)fr);
  char* small = nullptr;
  if (cudaMalloc(&small, kSmallBytes) != cudaSuccess) {
    delete ctx;
    return LSQ_ERR_OOM;
  }
  ctx->d_status = reinterpret_cast<uint32_t*>(small);
  ctx->d_max_rounds = reinterpret_cast<int32_t*>(small + 64);
  ctx->d_bar = reinterpret_cast<GridBarrier*>(small + 128);
  ctx->d_out = reinterpret_cast<double*>(small + 256);
  ctx->d_range = reinterpret_cast<uint32_t*>(small + 1024);
  ctx->d_fro = reinterpret_cast<double*>(small + 1040);
  if (cudaMallocHost(&ctx->h_small, kSmallBytes) != cudaSuccess) {
    cudaFree(small);
    delete ctx;
    return LSQ_ERR_OOM;
  }
  cudaMemset(small, 0, kSmallBytes);
  ctx->tuning = batch_tuning_new();
  *out = ctx;
  return LSQ_OK;
}

lsq_status lsq_destroy(lsq_ctx* ctx) {
  if (!ctx) return LSQ_ERR_ARG;
  cudaSetDevice(ctx->device);
  if (ctx->server) server_destroy(ctx->server);
  ctx->server = nullptr;
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->h_small) cudaFreeHost(ctx->h_small);
  if (ctx->tuning) batch_tuning_free(ctx->tuning);
  delete ctx;
  return LSQ_OK;
}

const char* lsq_last_error(const lsq_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

const char* lsq_status_string(lsq_status s) {
  switch (s) {
    case LSQ_OK: return "LSQ_OK";
    case LSQ_PENDING: return "LSQ_PENDING";
    case LSQ_ERR_ARG: return "LSQ_ERR_ARG";
    case LSQ_ERR_CUDA: return "LSQ_ERR_CUDA";
    case LSQ_ERR_OOM: return "LSQ_ERR_OOM";
    case LSQ_ERR_BUDGET: return "LSQ_ERR_BUDGET";
    case LSQ_ERR_SKETCH: return "LSQ_ERR_SKETCH";
    case LSQ_ERR_RANK: return "LSQ_ERR_RANK";
    case LSQ_ERR_NOCONV: return "LSQ_ERR_NOCONV";
    case LSQ_ERR_TIMEOUT: return "LSQ_ERR_TIMEOUT";
    case LSQ_ERR_NONFINITE: return "LSQ_ERR_NONFINITE";
    case LSQ_ERR_UNSUPPORTED: return "LSQ_ERR_UNSUPPORTED";
    case LSQ_ERR_ACCURACY: return "LSQ_ERR_ACCURACY";
    default: return "LSQ_UNKNOWN";
  }
}

size_t lsq_workspace_bytes(const lsq_ctx* ctx) { return ctx ? ctx->ws_size + kSmallBytes : 0; }

double lsq_lambert_w0(double x) {
  // principal branch on [-1/e, inf): Halley's iteration on f(w) = w e^w - x
  const double em1 = 0.36787944117144233;  // 1/e
  if (!(x >= -em1) || std::isinf(x)) return std::isinf(x) && x > 0 ? x : NAN;
  if (x == 0.0) return 0.0;
  double w;
  if (x < -0.32) {
    const double p = std::sqrt(2.0 * (1.0 + x / em1));  // series about the branch point
    w = -1.0 + p - p * p / 3.0;
  } else if (x < 3.0) {
    w = std::log1p(x) * 0.75;
  } else {
    const double l = std::log(x);
    w = l - std::log(l);
  }
  for (int k = 0; k < 64; ++k) {
    const double ew = std::exp(w);
    const double f = w * ew - x;
    const double wp1 = w + 1.0;
    if (wp1 == 0.0) break;
    const double dw = f / (ew * wp1 - (w + 2.0) * f / (2.0 * wp1));
    w -= dw;
    if (std::fabs(dw) <= 4e-16 * (1.0 + std::fabs(w))) break;
  }
  return w;
}

int64_t lsq_d_from_model(int64_t m, int64_t n, double tol, double t_iter_per_row, double t_qr_per_d) {
  // minimise T(d) = t_qr_per_d d + (2 |ln tol| / ln(d/n) + 2) t_iter_per_row m over d > n:
  // with d = n e^u, dT/du = 0 gives u^2 e^u = C, C = 2 |ln tol| t_iter_per_row m / (t_qr_per_d n),
  // so u/2 = W0(sqrt(C) / 2)
  if (m < 1 || n < 1 || !(tol > 0.0 && tol < 1.0) || !(t_iter_per_row > 0.0) || !(t_qr_per_d > 0.0)) return 0;
  const double C = 2.0 * std::fabs(std::log(tol)) * t_iter_per_row * (double)m / (t_qr_per_d * (double)n);
  const double u = 2.0 * lsq_lambert_w0(std::sqrt(C) / 2.0);
  const double d = (double)n * std::exp(u);
  if (!(d < 2147483647.0)) return 2147483647LL;
  return (int64_t)std::ceil(d);
}

lsq_status lsq_choose_d(lsq_ctx* ctx, int64_t m, int64_t n, double tol, int64_t* d) {
  lsq_status s;
  if ((s = check_ctx(ctx)) != LSQ_OK) return s;
  if (!d || m < 1 || n < 1 || n > kLsqrMaxN || !(tol > 0.0 && tol < 1.0))
    return fail(ctx, LSQ_ERR_ARG, "need d, m >= 1, 1 <= n <= 4096, 0 < tol < 1");
  lsq_ctx::DCalib cal;
  if ((s = calibrate_d(ctx, n, &cal)) != LSQ_OK) return s;
  int64_t v = lsq_d_from_model(m, n, tol, cal.t_iter_per_row, cal.t_qr_per_d);
  // keep the rate below 0.9 and the sketch within m rows and an eighth of the budget
  const int64_t lo = std::max<int64_t>(n + 1, (n * 5 + 3) / 4);
  int64_t hi = std::min<int64_t>(m, 2147483647LL);
  hi = std::min<int64_t>(hi, (int64_t)(ctx->budget / 8 / (16 * (size_t)(n + 1))));
  if (hi < lo) hi = lo;
  *d = std::min(std::max(v, lo), hi);
  return LSQ_OK;
}

lsq_status lsq_set_wait_limit(lsq_ctx* ctx, double seconds) {
  lsq_status s;
  if ((s = check_ctx(ctx)) != LSQ_OK) return s;
  if (!(seconds >= 0.0) || seconds > 4000.0) return fail(ctx, LSQ_ERR_ARG, "need 0 <= seconds <= 4000");
  uint32_t us = (uint32_t)std::llround(seconds * 1e6);
  if (seconds > 0.0 && us == 0) us = 1;
  // stream-ordered after all earlier work of the device (a synchronous copy)
  CK(cudaMemcpy(&ctx->d_bar->limit_us, &us, sizeof(us), cudaMemcpyHostToDevice));
  ctx->wait_limit_us = us;
  if (ctx->server) server_set_wait_limit(ctx->server, us);
  return LSQ_OK;
}

lsq_status lsq_selftest_wait(lsq_ctx* ctx, int32_t kind, void* stream) {
  lsq_status s;
  if ((s = check_ctx(ctx)) != LSQ_OK) return s;
  if (kind != 0 && kind != 1) return fail(ctx, LSQ_ERR_ARG, "kind must be 0 (grid barrier) or 1 (mbarrier)");
  cudaStream_t st = (cudaStream_t)stream;
  if ((s = reset_small(ctx, st)) != LSQ_OK) return s;
  CK(wait_selftest(kind, ctx->d_bar, ctx->d_status, 2, st));
  uint32_t bits = 0;
  if ((s = read_small(ctx, st, &bits, nullptr, nullptr)) != LSQ_OK) return s;
  // the barrier's abort bit stays set until the next launch zeroes the counter
  return status_from_bits(ctx, bits);
}

lsq_status lsq_batch_shape_set(lsq_ctx* ctx, int32_t bucket, int32_t shape) {
  lsq_status s;
  if ((s = check_ctx(ctx)) != LSQ_OK) return s;
  static const int kBucketMaxN[4] = {32, 64, 128, 256};
  if (bucket < 0 || bucket > 3) return fail(ctx, LSQ_ERR_ARG, "bucket must be 0..3");
  if (shape != -1 && batch_shape_maxn(shape) < kBucketMaxN[bucket])
    return fail(ctx, LSQ_ERR_ARG, "shape " + std::to_string(shape) + " cannot take n <= " +
                                      std::to_string(kBucketMaxN[bucket]));
  batch_set_shape(ctx->tuning, bucket, shape);
  return LSQ_OK;
}

lsq_status lsq_batch_shape_get(lsq_ctx* ctx, int32_t bucket, int32_t* shape) {
  lsq_status s;
  if ((s = check_ctx(ctx)) != LSQ_OK) return s;
  if (bucket < 0 || bucket > 3 || !shape) return fail(ctx, LSQ_ERR_ARG, "bucket must be 0..3, shape non-null");
  *shape = batch_get_shape(ctx->tuning, bucket);
  return LSQ_OK;
}

lsq_status lsq_set_qr_mode(lsq_ctx* ctx, int32_t mode) {
  if (!ctx) return LSQ_ERR_ARG;
  if (mode != LSQ_QR_AUTO && mode != LSQ_QR_UNBLOCKED && mode != LSQ_QR_BLOCKED)
    return fail(ctx, LSQ_ERR_ARG, "unknown QR mode");
  ctx->qr_mode = mode;
  return LSQ_OK;
}

lsq_status lsq_sketch_indices(lsq_ctx* ctx, uint64_t seed, int64_t row0, int64_t rows, int64_t d, int32_t zeta,
                              int32_t* idx, int8_t* sign, int32_t* rounds, void* stream) {
  lsq_status s;
  if ((s = check_ctx(ctx)) != LSQ_OK) return s;
  if ((s = check_sketch_args(ctx, d, zeta)) != LSQ_OK) return s;
  if (rows < 0 || row0 < 0) return fail(ctx, LSQ_ERR_ARG, "rows and row0 must be >= 0");
  if (rows > 0 && (!idx || !sign)) return fail(ctx, LSQ_ERR_ARG, "idx and sign must not be null");
  cudaStream_t st = (cudaStream_t)stream;
  if ((s = reset_small(ctx, st)) != LSQ_OK) return s;
  CK(sketch_indices(seed, row0, rows, d, zeta, idx, sign, rounds, ctx->d_status, ctx->d_max_rounds, ctx->sms, st));
  uint32_t bits = 0;
  if ((s = read_small(ctx, st, &bits, nullptr, nullptr)) != LSQ_OK) return s;
  return status_from_bits(ctx, bits);
}

lsq_status lsq_sketch(lsq_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda, const double* b, int64_t d,
                      int32_t zeta, uint64_t seed, int32_t prec, void* Y, int64_t ldy, void* stream) {
  lsq_status s;
  if ((s = check_ctx(ctx)) != LSQ_OK) return s;
  if ((s = check_sketch_args(ctx, d, zeta)) != LSQ_OK) return s;
  if (m < 0 || n < 1 || n > 2147483647LL || lda < n) return fail(ctx, LSQ_ERR_ARG, "need m >= 0, n >= 1, lda >= n");
  if (ldy < n + (b ? 1 : 0)) return fail(ctx, LSQ_ERR_ARG, "ldy must be >= n + (b != NULL)");
  if (!Y || (m > 0 && !A)) return fail(ctx, LSQ_ERR_ARG, "null pointer");
  if (prec != LSQ_PREC_FP64 && prec != LSQ_PREC_MIXED) return fail(ctx, LSQ_ERR_ARG, "unknown precision");
  cudaStream_t st = (cudaStream_t)stream;
  if ((s = reset_small(ctx, st)) != LSQ_OK) return s;
  if (prec == LSQ_PREC_FP64) {
    CK(cudaMemsetAsync(Y, 0, (size_t)d * ldy * sizeof(double), st));
    CK(sketch_apply<double>(A, m, n, lda, b, d, zeta, seed, 0, (double*)Y, ldy, ctx->d_status, ctx->d_max_rounds,
                            nullptr, nullptr, ctx->sms, st));
  } else {
    // blocked FP32 accumulation (chunk sums in FP32, folded into float
    // pairs in workspace), rounded once into the FP32 output
    const int64_t ncol = n + (b ? 1 : 0), ldc = (ncol + 3) / 4 * 4;
    const size_t y64 = align_up((size_t)d * ncol * sizeof(double));
    if ((s = ensure_ws(ctx, y64 + align_up(2 * (size_t)d * ldc * sizeof(float)))) != LSQ_OK) return s;
    float2* Yp = reinterpret_cast<float2*>(ctx->ws);
    float* Yc = reinterpret_cast<float*>(static_cast<char*>(ctx->ws) + y64);
    CK(cudaMemsetAsync(Yp, 0, (size_t)d * ncol * sizeof(float2), st));
    CK(cudaMemsetAsync(Yc, 0, 2 * (size_t)d * ldc * sizeof(float), st));
    CK(sketch_apply_fold(A, m, n, lda, b, d, zeta, seed, Yc, ldc, Yp, ncol, ctx->d_status, ctx->d_max_rounds,
                         nullptr, nullptr, ctx->d_bar, ctx->sms, st));
    CK(round_to_float(Yp, ncol, static_cast<float*>(Y), ldy, d, ncol, ctx->sms, st));
  }
  uint32_t bits = 0;
  if ((s = read_small(ctx, st, &bits, nullptr, nullptr)) != LSQ_OK) return s;
  return status_from_bits(ctx, bits);
}

lsq_status lsq_precond(lsq_ctx* ctx, const void* Y, int64_t d, int64_t n, int64_t ldy, int32_t has_b, int32_t prec,
                       double* R, double* M, double* x0, void* stream) {
  lsq_status s;
  if ((s = check_ctx(ctx)) != LSQ_OK) return s;
  const int64_t ncol = n + (has_b ? 1 : 0);
  if (n < 1 || n > 65536 || d < ncol || d > 2147483647LL || ldy < ncol)
    return fail(ctx, LSQ_ERR_ARG, "need 1 <= n <= 65536, d >= n + has_b, ldy >= n + has_b");
  if (!Y || !M) return fail(ctx, LSQ_ERR_ARG, "Y and M must not be null");
  if (x0 && !has_b) return fail(ctx, LSQ_ERR_ARG, "x0 needs the sketched b column (has_b)");
  if (prec != LSQ_PREC_FP64 && prec != LSQ_PREC_MIXED) return fail(ctx, LSQ_ERR_ARG, "unknown precision");
  cudaStream_t st = (cudaStream_t)stream;
  Carver probe{nullptr};
  probe.take<double>((size_t)ncol * d);
  probe.take<double>(n);
  probe.take<double>((size_t)n * n);
  probe.take<double>((size_t)n * n);
  probe.take<char>(precond_blocked_bytes(d, n));
  if ((s = ensure_ws(ctx, probe.off)) != LSQ_OK) return s;
  Carver cv{ctx->ws};
  PrecondBuffers buf;
  buf.W = cv.take<double>((size_t)ncol * d);  // large enough for either precision
  buf.rdiag = cv.take<double>(n);
  buf.R = cv.take<double>((size_t)n * n);
  buf.Mt = cv.take<double>((size_t)n * n);
  buf.blk = cv.take<char>(precond_blocked_bytes(d, n));
  buf.mode = ctx->qr_mode;
  buf.bar = ctx->d_bar;
  buf.status = ctx->d_status;
  if ((s = reset_small(ctx, st)) != LSQ_OK) return s;
  if (prec == LSQ_PREC_FP64)
    CK(precond<double>((const double*)Y, d, n, ldy, has_b, R, M, x0, buf, ctx->sms, st));
  else
    CK(precond<float>((const float*)Y, d, n, ldy, has_b, R, M, x0, buf, ctx->sms, st));
  uint32_t bits = 0;
  if ((s = read_small(ctx, st, &bits, nullptr, nullptr)) != LSQ_OK) return s;
  return status_from_bits(ctx, bits);
}

lsq_status lsq_lsqr(lsq_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                    const double* M, const double* x0, double tol, int64_t maxit, int32_t flags, double* x,
                    lsq_info* info, void* stream) {
  lsq_status s;
  if ((s = check_ctx(ctx)) != LSQ_OK) return s;
  if (m < 1 || n < 1 || lda < n) return fail(ctx, LSQ_ERR_ARG, "need m >= 1, n >= 1, lda >= n");
  if (!A || !b || !M || !x0 || !x) return fail(ctx, LSQ_ERR_ARG, "null pointer");
  if (n > kLsqrMaxN) return fail(ctx, LSQ_ERR_UNSUPPORTED, "LSQR kernels built for n <= 4096");
  if ((flags & LSQ_FLAG_NATIVE_FP64) && n > kLsqrMaxN)
    return fail(ctx, LSQ_ERR_UNSUPPORTED, "native FP64 LSQR kernels built for n <= 4096");
  cudaStream_t st = (cudaStream_t)stream;
  const int ni = (int)n, npad = (int)((n + 31) / 32 * 32);
  bool native = (flags & LSQ_FLAG_NATIVE_FP64) || !lsqr_df_ok(A, n, lda);
  int grid = lsqr_grid(ni, vec_ok(A, lda), native, ctx->sms);
  if (grid < 1) return fail(ctx, LSQ_ERR_CUDA, "no launchable LSQR configuration");
  bool image = !native && !(flags & LSQ_FLAG_NO_IMAGE);
  Carver probe{nullptr};
  carve_lsqr(probe, m, ni, npad, grid, image);
  if (image && probe.off > ctx->budget) {
    image = false;  // fall back to splitting A on the fly in every pass
    probe = Carver{nullptr};
    carve_lsqr(probe, m, ni, npad, grid, false);
  }
  if (!native && !image && !(vec_ok(A, lda) && n % 2 == 0) && lsqr_native_ok(n)) {
    // without the image every pass streams A through the bulk-copy ring,
    // which needs even n and lda and an aligned A (wide rows load directly)
    native = true;
    grid = lsqr_grid(ni, vec_ok(A, lda), native, ctx->sms);
    probe = Carver{nullptr};
    carve_lsqr(probe, m, ni, npad, grid, false);
  }
  if ((s = ensure_ws(ctx, probe.off)) != LSQ_OK) return s;
  Carver cv{ctx->ws};
  LsqrWork w = carve_lsqr(cv, m, ni, npad, grid, image);
  if ((s = reset_small(ctx, st)) != LSQ_OK) return s;
  // exponent range of A and b for the double-float passes (and a finiteness check)
  if (!native) CK(range_scan(A, m, n, lda, b, ctx->d_range, ctx->d_status, ctx->sms, st));
  CK(transpose_square(M, ni, w.Mt, st));
  if (x != x0) CK(cudaMemcpyAsync(x, x0, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  if (maxit <= 0) maxit = 1000;
  if ((s = run_lsqr(ctx, A, m, ni, lda, b, M, w.Mt, x, tol, maxit, 2, w, grid, npad, native, st)) != LSQ_OK)
    return s;
  uint32_t bits = 0;
  double out[kOutSlots];
  if ((s = read_small(ctx, st, &bits, nullptr, out)) != LSQ_OK) return s;
  s = status_from_bits(ctx, bits);
  fill_info(info, out, s, 0);
  return s;
}

lsq_status lsq_hbm(lsq_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                   const double* M, const double* x0, double tol, int64_t maxit, double eta_hat, int32_t flags,
                   double* x, lsq_info* info, void* stream) {
  lsq_status s;
  if ((s = check_ctx(ctx)) != LSQ_OK) return s;
  if (m < 1 || n < 1 || lda < n) return fail(ctx, LSQ_ERR_ARG, "need m >= 1, n >= 1, lda >= n");
  if (!A || !b || !M || !x0 || !x) return fail(ctx, LSQ_ERR_ARG, "null pointer");
  if (!(eta_hat >= 0.0 && eta_hat < 1.0)) return fail(ctx, LSQ_ERR_ARG, "need 0 <= eta_hat < 1");
  if (n > kLsqrMaxN) return fail(ctx, LSQ_ERR_UNSUPPORTED, "LSQR kernels built for n <= 4096");
  if ((flags & LSQ_FLAG_NATIVE_FP64) && n > kLsqrMaxN)
    return fail(ctx, LSQ_ERR_UNSUPPORTED, "native FP64 LSQR kernels built for n <= 4096");
  cudaStream_t st = (cudaStream_t)stream;
  const int ni = (int)n, npad = (int)((n + 31) / 32 * 32);
  bool native = (flags & LSQ_FLAG_NATIVE_FP64) || !lsqr_df_ok(A, n, lda);
  int grid = lsqr_grid(ni, vec_ok(A, lda), native, ctx->sms);
  if (grid < 1) return fail(ctx, LSQ_ERR_CUDA, "no launchable LSQR configuration");
  bool image = !native && !(flags & LSQ_FLAG_NO_IMAGE);
  Carver probe{nullptr};
  carve_lsqr(probe, m, ni, npad, grid, image);
  if (image && probe.off > ctx->budget) {
    image = false;  // fall back to splitting A on the fly in every pass
    probe = Carver{nullptr};
    carve_lsqr(probe, m, ni, npad, grid, false);
  }
  if (!native && !image && !(vec_ok(A, lda) && n % 2 == 0) && lsqr_native_ok(n)) {
    // without the image every pass streams A through the bulk-copy ring,
    // which needs even n and lda and an aligned A (wide rows load directly)
    native = true;
    grid = lsqr_grid(ni, vec_ok(A, lda), native, ctx->sms);
    probe = Carver{nullptr};
    carve_lsqr(probe, m, ni, npad, grid, false);
  }
  if ((s = ensure_ws(ctx, probe.off)) != LSQ_OK) return s;
  Carver cv{ctx->ws};
  LsqrWork w = carve_lsqr(cv, m, ni, npad, grid, image);
  if ((s = reset_small(ctx, st)) != LSQ_OK) return s;
  if (!native) CK(range_scan(A, m, n, lda, b, ctx->d_range, ctx->d_status, ctx->sms, st));
  CK(transpose_square(M, ni, w.Mt, st));
  if (x != x0) CK(cudaMemcpyAsync(x, x0, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  if (maxit <= 0) maxit = 1000;
  // App. C.2: alpha = (1 - eta^2)^2, beta = eta^2
  const double e2 = eta_hat * eta_hat;
  const int hmode = (flags & LSQ_FLAG_NO_CHECK) ? 4 : 3;
  if ((s = run_lsqr(ctx, A, m, ni, lda, b, M, w.Mt, x, tol, maxit, hmode, w, grid, npad, native, st,
                    (1.0 - e2) * (1.0 - e2), e2, solve_gate(tol, 0.0))) != LSQ_OK)
    return s;
  uint32_t bits = 0;
  double out[kOutSlots];
  if ((s = read_small(ctx, st, &bits, nullptr, out)) != LSQ_OK) return s;
  s = status_from_bits(ctx, bits);
  fill_info(info, out, s, 0);
  return s;
}

lsq_status lsq_check(lsq_ctx* ctx, const double* A, int64_t m, int64_t n, int64_t lda, const double* b,
                     const double* x, const double* M, lsq_info* info, void* stream) {
  lsq_status s;
  if ((s = check_ctx(ctx)) != LSQ_OK) return s;
  if (m < 1 || n < 1 || lda < n) return fail(ctx, LSQ_ERR_ARG, "need m >= 1, n >= 1, lda >= n");
  if (!A || !b || !x) return fail(ctx, LSQ_ERR_ARG, "null pointer");
  if (n > kLsqrMaxN) return fail(ctx, LSQ_ERR_UNSUPPORTED, "check kernels built for n <= 4096");
  cudaStream_t st = (cudaStream_t)stream;
  const int ni = (int)n, npad = (int)((n + 31) / 32 * 32);
  // native FP64 pass: one warp per row for n <= 512, the panel kernel's
  // FP64 check pass for wider rows
  const bool native = lsqr_native_ok(n);
  const int grid = lsqr_grid(ni, vec_ok(A, lda), native, ctx->sms);
  if (grid < 1) return fail(ctx, LSQ_ERR_CUDA, "no launchable check configuration");
  Carver probe{nullptr};
  carve_lsqr(probe, m, ni, npad, grid);
  if ((s = ensure_ws(ctx, probe.off)) != LSQ_OK) return s;
  Carver cv{ctx->ws};
  LsqrWork w = carve_lsqr(cv, m, ni, npad, grid);
  if ((s = reset_small(ctx, st)) != LSQ_OK) return s;
  if (M) CK(transpose_square(M, ni, w.Mt, st));
  if ((s = run_lsqr(ctx, A, m, ni, lda, b, M, M ? w.Mt : nullptr, const_cast<double*>(x), 0.0, 0, 1, w, grid, npad,
                    native, st)) != LSQ_OK)
    return s;
  uint32_t bits = 0;
  double out[kOutSlots];
  if ((s = read_small(ctx, st, &bits, nullptr, out)) != LSQ_OK) return s;
  s = status_from_bits(ctx, bits);
  fill_info(info, out, s, 0);
  return s;
}

static lsq_status solve_once(lsq_ctx* ctx, const lsq_problem* pr, const lsq_opts* o, double* x, lsq_info* info,
                             void* stream) {
  lsq_status s;
  if ((s = check_ctx(ctx)) != LSQ_OK) return s;
  if (!pr || !o || !x) return fail(ctx, LSQ_ERR_ARG, "null problem, options or x");
  const int64_t m = pr->m, n = pr->n, lda = pr->lda, d = o->d;
  if (m < 1 || n < 1 || lda < n || !pr->A || !pr->b) return fail(ctx, LSQ_ERR_ARG, "need m, n >= 1, lda >= n, A, b");
  if ((s = check_sketch_args(ctx, d, o->zeta)) != LSQ_OK) return s;
  if (d < n + 1) return fail(ctx, LSQ_ERR_ARG, "need d >= n + 1");
  if (o->prec != LSQ_PREC_FP64 && o->prec != LSQ_PREC_MIXED) return fail(ctx, LSQ_ERR_ARG, "unknown precision");
  if (pr->mem != LSQ_MEM_DEVICE && pr->mem != LSQ_MEM_HOST) return fail(ctx, LSQ_ERR_ARG, "unknown memory kind");
  if (n > kLsqrMaxN) return fail(ctx, LSQ_ERR_UNSUPPORTED, "LSQR kernels built for n <= 4096");
  if ((o->flags & LSQ_FLAG_NATIVE_FP64) && n > kLsqrMaxN)
    return fail(ctx, LSQ_ERR_UNSUPPORTED, "native FP64 LSQR kernels built for n <= 4096");
  cudaStream_t st = (cudaStream_t)stream;
  const bool host = pr->mem == LSQ_MEM_HOST;
  // host problems in pinned or registered memory are read in place by the
  // FP64 sketch, which writes the device copy in the same pass (no separate
  // copy before it); pageable memory is copied first
  const double* hA = nullptr;
  const double* hb = nullptr;
  if (host && o->prec == LSQ_PREC_FP64) {
    hA = static_cast<const double*>(host_device_view(pr->A));
    hb = static_cast<const double*>(host_device_view(pr->b));
  }
  const bool tee = hA && hb;
  const bool timing = (o->flags & LSQ_FLAG_TIMING) != 0;
  const int ni = (int)n, npad = (int)((n + 31) / 32 * 32);
  // Y is FP64 in both forms; the mixed form accumulates its terms in FP32
  // chunk sums (Yc, rows padded to 4 floats for the 4-wide reductions)
  const int64_t ncol = n + 1, ldy = ncol, ldc = (ncol + 3) / 4 * 4;
  const size_t yes = 8;
  const bool mixed = o->prec == LSQ_PREC_MIXED;
  const int64_t lda_dev = host ? n : lda;
  const bool vec = host ? (n % 2 == 0) : vec_ok(pr->A, lda);
  // host problems are copied into 256-byte aligned workspace with lda = n
  bool native = (o->flags & LSQ_FLAG_NATIVE_FP64) || !lsqr_df_ok(pr->A, n, lda);
  int grid = lsqr_grid(ni, vec, native, ctx->sms);
  if (grid < 1) return fail(ctx, LSQ_ERR_CUDA, "no launchable LSQR configuration");
  const int64_t maxit = o->maxit > 0 ? o->maxit : default_maxit(n, d, o->tol);

  bool image = !native && !(o->flags & LSQ_FLAG_NO_IMAGE);
  float* Yc = nullptr;
  auto carve = [&](Carver& cv, const double** A, const double** b, double** xd, void** Y, PrecondBuffers* pb,
                   double** R, double** M, LsqrWork* lw) {
    if (host) {
      *A = cv.take<double>((size_t)m * n);
      *b = cv.take<double>((size_t)m);
      *xd = cv.take<double>(npad);
    } else {
      *A = pr->A;
      *b = pr->b;
      *xd = x;
    }
    *Y = cv.take<char>((size_t)d * ldy * yes);
    Yc = mixed ? cv.take<float>(2 * (size_t)d * ldc) : nullptr;
    pb->W = cv.take<double>((size_t)ncol * d);
    pb->rdiag = cv.take<double>(npad);
    pb->blk = cv.take<char>(precond_blocked_bytes(d, n));
    pb->R = nullptr;
    pb->Mt = nullptr;
    *R = cv.take<double>((size_t)n * n);
    *M = cv.take<double>((size_t)n * n);
    *lw = carve_lsqr(cv, m, ni, npad, grid, image);
    pb->Mt = lw->Mt;
  };
  {
    Carver probe{nullptr};
    const double *A0, *b0;
    double *x0, *R0, *M0;
    void* Y0;
    PrecondBuffers pb0;
    LsqrWork lw0;
    carve(probe, &A0, &b0, &x0, &Y0, &pb0, &R0, &M0, &lw0);
    if (image && probe.off > ctx->budget) {
      image = false;  // no room for the float-pair image: split A on the fly
      if (!(vec && n % 2 == 0) && lsqr_native_ok(n)) {
        // every pass would stream A through the bulk-copy ring: needs even n, lda
        native = true;
        grid = lsqr_grid(ni, vec, native, ctx->sms);
      }
      probe = Carver{nullptr};
      carve(probe, &A0, &b0, &x0, &Y0, &pb0, &R0, &M0, &lw0);
    }
    if (!native && !image && !(vec && n % 2 == 0) && lsqr_native_ok(n)) {
      native = true;
      grid = lsqr_grid(ni, vec, native, ctx->sms);
      probe = Carver{nullptr};
      carve(probe, &A0, &b0, &x0, &Y0, &pb0, &R0, &M0, &lw0);
    }
    if ((s = ensure_ws(ctx, probe.off)) != LSQ_OK) return s;
  }
  Carver cv{ctx->ws};
  const double *A, *b;
  double *xd, *R, *M;
  void* Y;
  PrecondBuffers pb;
  LsqrWork lw;
  carve(cv, &A, &b, &xd, &Y, &pb, &R, &M, &lw);
  pb.bar = ctx->d_bar;
  pb.status = ctx->d_status;
  pb.mode = ctx->qr_mode;

  Events<6> ev;
  if (timing) CK(ev.create());
  if (timing) CK(cudaEventRecord(ev[0], st));
  if (host && !tee) {
    if (lda == n)  // packed rows: one flat copy
      CK(cudaMemcpyAsync((void*)A, pr->A, sizeof(double) * (size_t)m * n, cudaMemcpyHostToDevice, st));
    else
      CK(cudaMemcpy2DAsync((void*)A, sizeof(double) * n, pr->A, sizeof(double) * lda, sizeof(double) * n, m,
                           cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync((void*)b, pr->b, sizeof(double) * m, cudaMemcpyHostToDevice, st));
  }
  if (timing) CK(cudaEventRecord(ev[1], st));
  if ((s = reset_small(ctx, st)) != LSQ_OK) return s;
  CK(cudaMemsetAsync(Y, 0, (size_t)d * ldy * yes, st));
  // the sketch also records the exponent range of A and b (ctx->d_range) for
  // the double-float LSQR passes
  if (tee) {
    CK(sketch_apply_tee(hA, m, n, lda, hb, d, o->zeta, o->seed, (double*)Y, ldy, const_cast<double*>(A), lda_dev,
                        const_cast<double*>(b), ctx->d_status, ctx->d_max_rounds, ctx->d_range, ctx->d_fro,
                        ctx->sms, st));
  } else if (o->prec == LSQ_PREC_FP64) {
    CK(sketch_apply<double>(A, m, n, lda_dev, b, d, o->zeta, o->seed, 0, (double*)Y, ldy, ctx->d_status,
                            ctx->d_max_rounds, ctx->d_range, ctx->d_fro, ctx->sms, st));
  } else {
    // blocked FP32 accumulation: chunk sums in Yc, folded into float pairs in
    // Y's memory, then turned into the FP64 sketch in place
    CK(cudaMemsetAsync(Yc, 0, 2 * (size_t)d * ldc * sizeof(float), st));
    CK(sketch_apply_fold(A, m, n, lda_dev, b, d, o->zeta, o->seed, Yc, ldc, (float2*)Y, ldy, ctx->d_status,
                         ctx->d_max_rounds, ctx->d_range, ctx->d_fro, ctx->d_bar, ctx->sms, st));
    CK(pairs_to_double((float2*)Y, d * ldy, ctx->sms, st));
  }
  if (timing) CK(cudaEventRecord(ev[2], st));
  // both forms factor the FP64 sketch (the tensor-core trailing updates
  // accumulate bf16 slice products in FP32 either way)
  CK(precond<double>((const double*)Y, d, n, ldy, 1, R, M, xd, pb, ctx->sms, st));
  if (timing) CK(cudaEventRecord(ev[3], st));
  // status after the preconditioner (sketch failure, rank) before iterating
  uint32_t bits = 0;
  int32_t rounds = 0;
  double out[kOutSlots] = {0};
  if ((s = read_small(ctx, st, &bits, &rounds, nullptr)) != LSQ_OK) return s;
  if (o->prec == LSQ_PREC_MIXED && !bits) {
    // the FP32 sketch needs max|A| and max|b| well inside the FP32 range
    // (sums of many terms must not overflow, entries far below the largest
    // may flush): exponents in [-60, 100], else the plain form solves it
    const char* h = static_cast<const char*>(ctx->h_small);
    const size_t off = (const char*)ctx->d_range - (const char*)ctx->d_status;
    uint32_t rg[2];
    std::memcpy(rg, h + off, sizeof(rg));
    for (uint32_t w : rg) {
      const int e = (int)(w >> 20) - 1023;
      if (w && (e < -60 || e > 100))
        return fail(ctx, LSQ_ERR_UNSUPPORTED, "mixed form: A or b outside the FP32 sketch's range (|max| exponent " +
                                                  std::to_string(e) + ")");
    }
  }
  if (bits) {
    s = status_from_bits(ctx, bits);
    if (info) {
      fill_info(info, out, s, rounds);
    }
    return s;
  }
  const bool hbm = (o->flags & LSQ_FLAG_HBM) != 0;
  const bool nocheck = (o->flags & LSQ_FLAG_NO_CHECK) != 0;
  const int mode = hbm ? (nocheck ? 4 : 3) : (nocheck ? 2 : 0);
  // heavy-ball momentum: App. C.2 parameters with the distortion estimate sqrt(n/d)
  const double e2 = (double)n / (double)d;
  if ((s = run_lsqr(ctx, A, m, ni, lda_dev, b, M, lw.Mt, xd, o->tol, maxit, mode, lw, grid, npad, native, st,
                    hbm ? (1.0 - e2) * (1.0 - e2) : 0.0, hbm ? e2 : 0.0, solve_gate(o->tol, o->gate),
                    ctx->d_fro)) != LSQ_OK)
    return s;
  if (timing) CK(cudaEventRecord(ev[4], st));
  if (host) CK(cudaMemcpyAsync(x, xd, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  if (timing) CK(cudaEventRecord(ev[5], st));
  if ((s = read_small(ctx, st, &bits, nullptr, out)) != LSQ_OK) return s;
  s = status_from_bits(ctx, bits);
  fill_info(info, out, s, rounds);
  if (info && timing) {
    float t;
    cudaEventElapsedTime(&t, ev[0], ev[1]);
    info->t_h2d_ms = t;
    cudaEventElapsedTime(&t, ev[1], ev[2]);
    info->t_sketch_ms = t;
    cudaEventElapsedTime(&t, ev[2], ev[3]);
    info->t_precond_ms = t;
    cudaEventElapsedTime(&t, ev[3], ev[4]);
    info->t_lsqr_ms = t;
    cudaEventElapsedTime(&t, ev[4], ev[5]);
    info->t_d2h_ms = t;
  }
  return s;
}

// Mixed form: FP32 sketch and QR give a good preconditioner only while
// cond(A) * u_fp32 * sqrt(m zeta / d) stays well below 1.  The mixed solve is
// therefore capped at twice the iteration count the Sec. 4.3 rate estimate
// predicts; if the cap is hit, the plain FP64 form solves the problem again.
static lsq_status lsq_solve_d(lsq_ctx* ctx, const lsq_problem* pr, const lsq_opts* o, double* x, lsq_info* info,
                              void* stream);

lsq_status lsq_solve(lsq_ctx* ctx, const lsq_problem* pr, const lsq_opts* o_in, double* x, lsq_info* info,
                     void* stream) {
  lsq_opts oa;
  const lsq_opts* o = o_in;
  if (o_in && pr && o_in->d == 0) {  // automatic embedding dimension
    oa = *o_in;
    lsq_status s = lsq_choose_d(ctx, pr->m, pr->n, o_in->tol, &oa.d);
    if (s != LSQ_OK) return s;
    o = &oa;
  }
  lsq_status s0 = lsq_solve_d(ctx, pr, o, x, info, stream);
  if (info && o) info->d_used = o->d;
  return s0;
}

static lsq_status lsq_solve_d(lsq_ctx* ctx, const lsq_problem* pr, const lsq_opts* o, double* x, lsq_info* info,
                              void* stream) {
  if (!o || o->prec != LSQ_PREC_MIXED || (o->flags & LSQ_FLAG_NO_FALLBACK) || !pr)
    return solve_once(ctx, pr, o, x, info, stream);
  lsq_opts om = *o;
  const int64_t full = o->maxit > 0 ? o->maxit : default_maxit(pr->n, o->d, o->tol);
  const int64_t cap = 2 * (default_maxit(pr->n, o->d, o->tol) / 10) + 5;
  om.maxit = cap < full ? cap : full;
  lsq_status s = solve_once(ctx, pr, &om, x, info, stream);
  // fall back to the plain form when the FP32 preconditioner stalled LSQR, the
  // accuracy gate failed, or the data is outside the FP32 sketch's range
  const bool retry = s == LSQ_ERR_ACCURACY || s == LSQ_ERR_UNSUPPORTED || (s == LSQ_ERR_NOCONV && om.maxit < full);
  if (!retry) return s;
  lsq_opts op = *o;
  op.prec = LSQ_PREC_FP64;
  s = solve_once(ctx, pr, &op, x, info, stream);
  if (info) info->precond_fallback = 1;
  return s;
}

lsq_status lsq_solve_csr(lsq_ctx* ctx, const lsq_csr_problem* pr, const lsq_opts* o_in, double* x, lsq_info* info,
                         void* stream) {
  lsq_status s;
  if ((s = check_ctx(ctx)) != LSQ_OK) return s;
  if (!pr || !o_in || !x) return fail(ctx, LSQ_ERR_ARG, "null problem, options or x");
  const int64_t m = pr->m, n = pr->n;
  if (m < 1 || n < 1 || n > kLsqrMaxN || pr->nnz < 0 || !pr->row_ptr || !pr->b || (pr->nnz > 0 && (!pr->col_idx ||
      !pr->values)))
    return fail(ctx, LSQ_ERR_ARG, "need m >= 1, 1 <= n <= 4096, nnz >= 0 and the CSR arrays");
  if (o_in->prec != LSQ_PREC_FP64) return fail(ctx, LSQ_ERR_UNSUPPORTED, "sparse A: FP64 form only");
  lsq_opts o = *o_in;
  if (o.d == 0 && (s = lsq_choose_d(ctx, m, n, o.tol, &o.d)) != LSQ_OK) return s;
  const int64_t d = o.d;
  if ((s = check_sketch_args(ctx, d, o.zeta)) != LSQ_OK) return s;
  if (d < n + 1) return fail(ctx, LSQ_ERR_ARG, "need d >= n + 1");
  cudaStream_t st = (cudaStream_t)stream;
  const bool timing = (o.flags & LSQ_FLAG_TIMING) != 0;
  const int ni = (int)n, npad = (int)((n + 31) / 32 * 32);
  const int64_t ncol = n + 1;
  const int lanes = csr_lanes(m, pr->nnz);
  const int grid = lsqr_csr_grid(ctx->sms, lanes);
  if (grid < 1) return fail(ctx, LSQ_ERR_CUDA, "no launchable CSR LSQR configuration");
  const int64_t maxit = o.maxit > 0 ? o.maxit : default_maxit(n, d, o.tol);
  auto carve = [&](Carver& cv, double** Y, PrecondBuffers* pb, double** R, double** M, LsqrWork* lw) {
    *Y = cv.take<double>((size_t)d * ncol);
    pb->W = cv.take<double>((size_t)ncol * d);
    pb->rdiag = cv.take<double>(npad);
    pb->blk = cv.take<char>(precond_blocked_bytes(d, n));
    pb->R = nullptr;
    *R = cv.take<double>((size_t)n * n);
    *M = cv.take<double>((size_t)n * n);
    *lw = carve_lsqr(cv, m, ni, npad, grid, false);
    pb->Mt = lw->Mt;
  };
  double *Y, *R, *M;
  PrecondBuffers pb;
  LsqrWork lw;
  {
    Carver probe{nullptr};
    carve(probe, &Y, &pb, &R, &M, &lw);
    if ((s = ensure_ws(ctx, probe.off)) != LSQ_OK) return s;
  }
  Carver cv{ctx->ws};
  carve(cv, &Y, &pb, &R, &M, &lw);
  pb.bar = ctx->d_bar;
  pb.status = ctx->d_status;
  pb.mode = ctx->qr_mode;
  Events<4> ev;
  if (timing) CK(ev.create());
  if (timing) CK(cudaEventRecord(ev[0], st));
  if ((s = reset_small(ctx, st)) != LSQ_OK) return s;
  {
    // no kernel indexes by row_ptr or col_idx before they are known to be well formed
    CK(check_csr(pr->row_ptr, pr->col_idx, m, n, pr->nnz, ctx->d_status, ctx->sms, st));
    uint32_t cbits = 0;
    if ((s = read_small(ctx, st, &cbits, nullptr, nullptr)) != LSQ_OK) return s;
    if (cbits & DS_CSR)
      return fail(ctx, LSQ_ERR_ARG, "malformed CSR: need row_ptr[0] = 0, nondecreasing, row_ptr[m] = nnz, col_idx in [0, n)");
  }
  CK(cudaMemsetAsync(Y, 0, sizeof(double) * (size_t)d * ncol, st));
  CK(sketch_csr(pr->row_ptr, pr->col_idx, pr->values, pr->b, m, n, d, o.zeta, o.seed, Y, ncol, ctx->d_status,
                ctx->d_max_rounds, ctx->sms, st));
  if (timing) CK(cudaEventRecord(ev[1], st));
  CK(precond<double>(Y, d, n, ncol, 1, R, M, x, pb, ctx->sms, st));
  if (timing) CK(cudaEventRecord(ev[2], st));
  uint32_t bits = 0;
  int32_t rounds = 0;
  double out[kOutSlots] = {0};
  if ((s = read_small(ctx, st, &bits, &rounds, nullptr)) != LSQ_OK) return s;
  if (bits) {
    s = status_from_bits(ctx, bits);
    fill_info(info, out, s, rounds);
    return s;
  }
  LsqrParams p;
  std::memset(&p, 0, sizeof(p));
  p.m = m;
  p.n = ni;
  p.npad = npad;
  p.lda = n;
  p.b = pr->b;
  p.ldi = (n + 1) / 2 * 2;
  p.ring_k = 1;
  p.M = M;
  p.Mt = lw.Mt;
  p.x = x;
  p.u = lw.u;
  p.v = lw.v;
  p.vhat = lw.vhat;
  p.w = lw.w;
  p.wv = lw.wv;
  p.g = lw.g;
  p.gpart = lw.gpart;
  p.part = lw.part;
  p.tol = o.tol;
  p.maxit = maxit;
  const bool hbm = (o.flags & LSQ_FLAG_HBM) != 0, nocheck = (o.flags & LSQ_FLAG_NO_CHECK) != 0;
  p.mode = hbm ? (nocheck ? 4 : 3) : (nocheck ? 2 : 0);
  const double e2 = (double)n / (double)d;
  p.hbm_alpha = hbm ? (1.0 - e2) * (1.0 - e2) : 0.0;
  p.hbm_beta = hbm ? e2 : 0.0;
  p.gate = solve_gate(o.tol, o.gate);
  p.bar = ctx->d_bar;
  p.status = ctx->d_status;
  p.out = ctx->d_out;
  CK(transpose_square(M, ni, lw.Mt, st));
  CK(cudaMemsetAsync(&ctx->d_bar->count, 0, sizeof(unsigned int), st));
  CK(lsqr_csr_run(p, pr->row_ptr, pr->col_idx, pr->values, grid, lanes, st));
  if (timing) CK(cudaEventRecord(ev[3], st));
  if ((s = read_small(ctx, st, &bits, nullptr, out)) != LSQ_OK) return s;
  s = status_from_bits(ctx, bits);
  fill_info(info, out, s, rounds);
  if (info) {
    info->d_used = d;
    if (timing) {
      float t;
      cudaEventElapsedTime(&t, ev[0], ev[1]);
      info->t_sketch_ms = t;
      cudaEventElapsedTime(&t, ev[1], ev[2]);
      info->t_precond_ms = t;
      cudaEventElapsedTime(&t, ev[2], ev[3]);
      info->t_lsqr_ms = t;
    }
  }
  return s;
}

lsq_status lsq_solve_batch(lsq_ctx* ctx, const lsq_batch_item* items, int64_t count, double tol, int64_t maxit,
                           int32_t flags, lsq_batch_result* results, void* stream) {
  lsq_status s;
  if ((s = check_ctx(ctx)) != LSQ_OK) return s;
  if (count < 0 || (count > 0 && !items)) return fail(ctx, LSQ_ERR_ARG, "bad batch");
  if (count == 0) return LSQ_OK;
  if (count > 2147483647LL) return fail(ctx, LSQ_ERR_ARG, "too many problems");
  cudaStream_t st = (cudaStream_t)stream;
  int64_t m_max = 0;
  int n_max = 0, d_max = 0, ring_elems = 0;
  for (int64_t i = 0; i < count; ++i) {
    const lsq_batch_item& it = items[i];
    if (it.m < 1 || it.n < 1 || it.n > 256 || it.lda < it.n || it.d < it.n + 1 || it.d > (1 << 20) || it.zeta < 1 ||
        it.zeta > 8 || it.zeta > it.d || !it.A || !it.b || !it.x)
      return fail(ctx, LSQ_ERR_ARG, "batch item " + std::to_string(i) +
                                        ": need 1 <= n <= 256, lda >= n, n+1 <= d, 1 <= zeta <= min(8, d), pointers");
    m_max = std::max(m_max, it.m);
    n_max = std::max(n_max, (int)it.n);
    ring_elems = std::max(ring_elems, batch_ring_elems((int)it.n));
    d_max = std::max(d_max, (int)it.d);
  }
  const BatchLayout L = batch_layout(m_max, n_max, d_max);
  const int grid = batch_grid(ring_elems, ctx->sms);
  if (grid < 1) return fail(ctx, LSQ_ERR_CUDA, "batch kernel does not fit on the device");
  const size_t ib = batch_item_bytes();
  Carver probe{nullptr};
  probe.take<char>((size_t)grid * L.slab);
  probe.take<char>((size_t)count * ib);
  probe.take<int32_t>((size_t)count);
  probe.take<double>((size_t)count * kOutSlots);
  probe.take<uint32_t>((size_t)count);
  probe.take<int32_t>(1);
  if ((s = ensure_ws(ctx, probe.off)) != LSQ_OK) return s;
  Carver cv{ctx->ws};
  char* ws = cv.take<char>((size_t)grid * L.slab);
  void* items_dev = cv.take<char>((size_t)count * ib);
  int32_t* order_dev = cv.take<int32_t>((size_t)count);
  double* out_dev = cv.take<double>((size_t)count * kOutSlots);
  uint32_t* status_dev = cv.take<uint32_t>((size_t)count);
  int32_t* next_dev = cv.take<int32_t>(1);

  std::vector<char> host_items((size_t)count * ib);
  std::vector<int32_t> order((size_t)count);
  for (int64_t i = 0; i < count; ++i) order[i] = (int32_t)i;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return items[a].m * items[a].n > items[b].m * items[b].n;
  });
  const int mode = (flags & LSQ_FLAG_NO_CHECK) ? 2 : 0;
  if ((s = reset_small(ctx, st)) != LSQ_OK) return s;

  // ---- autotuner: time each candidate shape on the largest problems of an untuned n-range
  if (flags & LSQ_FLAG_AUTOTUNE) {
    for (int bk = 0; bk < 4; ++bk) {
      if (batch_get_shape(ctx->tuning, bk) >= 0) continue;
      std::vector<int32_t> sub;
      for (int32_t i : order)
        if (batch_bucket_of((int)items[i].n) == bk && (int)sub.size() < grid) sub.push_back(i);
      if (sub.empty()) continue;
      std::vector<int> cand;
      batch_shape_candidates((int)items[sub[0]].n, cand);
      if (cand.size() == 1) {
        batch_set_shape(ctx->tuning, bk, cand[0]);
        continue;
      }
      float best_ms = 1e30f;
      int best = cand.back();
      Events<2> te;
      CK(te.create());
      cudaEvent_t e0 = te[0], e1 = te[1];
      for (int shp : cand) {
        batch_items_fill(host_items.data(), items, count, nullptr);
        for (int32_t i : sub) batch_set_item_shape(host_items.data(), i, shp);
        CK(cudaMemcpyAsync(items_dev, host_items.data(), host_items.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(order_dev, sub.data(), sub.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(status_dev, 0, (size_t)count * sizeof(uint32_t), st));
        CK(cudaEventRecord(e0, st));
        CK(batch_launch(items_dev, order_dev, (int)sub.size(), next_dev, ws, L, tol, maxit, 2, out_dev, status_dev,
                        ctx->d_bar, grid, ring_elems, st));
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) {
          best_ms = ms;
          best = shp;
        }
      }
      batch_set_shape(ctx->tuning, bk, best);
    }
  }

  batch_items_fill(host_items.data(), items, count, ctx->tuning);
  CK(cudaMemcpyAsync(items_dev, host_items.data(), host_items.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(order_dev, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(status_dev, 0, (size_t)count * sizeof(uint32_t), st));
  CK(batch_launch(items_dev, order_dev, (int)count, next_dev, ws, L, tol, maxit, mode, out_dev, status_dev,
                  ctx->d_bar, grid, ring_elems, st));
  std::vector<double> hout((size_t)count * kOutSlots);
  std::vector<uint32_t> hst((size_t)count);
  CK(cudaMemcpyAsync(hout.data(), out_dev, hout.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hst.data(), status_dev, hst.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  lsq_status worst = LSQ_OK;
  std::string msg;
  for (int64_t i = 0; i < count; ++i) {
    const lsq_status si = status_from_bits(nullptr, hst[i]);
    if (si != LSQ_OK && worst == LSQ_OK) {
      worst = si;
      msg = "batch item " + std::to_string(i) + ": " + lsq_status_string(si);
    }
    if (results) {
      lsq_batch_result& r = results[i];
      const double* o = hout.data() + (size_t)i * kOutSlots;
      r.status = si;
      r.stop = (int32_t)o[OUT_STOP];
      r.iters = (int64_t)o[OUT_ITERS];
      r.backward_error_ne = o[OUT_ETA_NE];
      r.rnorm = o[OUT_RNORM];
      r.anorm_fro = o[OUT_FRO];
      r.xnorm = o[OUT_XNORM];
      r.bnorm = o[OUT_BNORM];
    }
  }
  if (worst != LSQ_OK) return fail(ctx, worst, msg);
  return LSQ_OK;
}

}  // extern "C"
