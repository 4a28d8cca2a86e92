// ctx.h -- the library context behind the opaque lsq_ctx handle (internal).
#pragma once
#include <map>
#include <string>

#include "kernels.h"

namespace lsq {
struct Server;
// Serving side (serve.cu): stop and free a context's server, if any.
void server_destroy(Server* s);
// Wait limit written into the control words of requests staged from now on.
void server_set_wait_limit(Server* s, uint32_t limit_us);
}  // namespace lsq

struct lsq_ctx {
  int device = 0;
  int sms = 0;
  size_t budget = 0;
  std::string err;
  // grown-on-demand workspace (one allocation, carved per call)
  char* ws = nullptr;
  size_t ws_size = 0;
  // small persistent device words
  uint32_t* d_status = nullptr;
  int32_t* d_max_rounds = nullptr;
  lsq::GridBarrier* d_bar = nullptr;
  double* d_out = nullptr;
  uint32_t* d_range = nullptr;  // [2] exponent maxima of A and b (pass_scale)
  double* d_fro = nullptr;      // sum of A_ij^2 formed by the sketch of lsq_solve
  uint32_t wait_limit_us = 0;   // limit of every device wait (0: the built-in 20 s)
  // pinned host mirror of the small words
  void* h_small = nullptr;
  // batched solves: tuned LSQR pass shapes per n-range
  lsq::BatchTuning* tuning = nullptr;
  int qr_mode = 0;  // LSQ_QR_AUTO / LSQ_QR_UNBLOCKED / LSQ_QR_BLOCKED
  // embedding-dimension calibration per width n: seconds per row of one LSQR
  // iteration, seconds per extra sketch row of the preconditioner
  struct DCalib {
    double t_iter_per_row = 0, t_qr_per_d = 0;
  };
  std::map<int64_t, DCalib> dcalib;
  // serving: persistent request loop, created by the first lsq_submit
  lsq::Server* server = nullptr;
  size_t serve_arena = 0;        // 0: the budget minus the synchronous workspace
  double serve_cta_bytes = 0.0;  // 0: default bytes of A per block of a request's group
  int serve_max_group = 0;       // 0: default cap on a request's group
};
