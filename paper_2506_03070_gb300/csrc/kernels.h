// kernels.h -- host-side launchers of the library's kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace lsq {

// Sketch (sketch.cu)
cudaError_t sketch_indices(uint64_t seed, int64_t row0, int64_t rows, int64_t d, int zeta, int32_t* idx, int8_t* sgn,
                           int32_t* rounds, uint32_t* status, int32_t* max_rounds, int sms, cudaStream_t st);
// range (nullable, [2] words, zeroed by the caller): atomic max of the
// exponent field (high word & 0x7FF00000) over A's and over b's finite entries.
// fro (nullable, zeroed by the caller): FP64 sum of A_ij^2 (atomic adds of warp partials).
template <typename TY>  // double
cudaError_t sketch_apply(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, int64_t d, int zeta,
                         uint64_t seed, int64_t row0, TY* Y, int64_t ldy, uint32_t* status, int32_t* max_rounds,
                         uint32_t* range, double* fro, int sms, cudaStream_t st);
// out (d x ncol floats, row stride ldo) = the float pairs Y (row stride ldy),
// each pair's sum rounded once to FP32.
cudaError_t round_to_float(const float2* Y, int64_t ldy, float* out, int64_t ldo, int64_t d, int64_t ncol, int sms,
                           cudaStream_t st);
// In place: each of the count float pairs becomes the double hi + lo.
cudaError_t pairs_to_double(float2* Y, int64_t count, int sms, cudaStream_t st);
// The mixed form's sketch with blocked FP32 accumulation: terms are added in
// FP32 into Yc (two buffers of d x ldc floats, ldc % 4 == 0, zero on entry and
// on exit) one chunk of rows at a time, each chunk's sums then added into the float-pair
// sketch Y (d x ldy pairs, zero on entry; pairs_to_double or round_to_float
// finish it).  Cooperative launch; bar's counter is reset.
cudaError_t sketch_apply_fold(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, int64_t d,
                              int zeta, uint64_t seed, float* Yc, int64_t ldc, float2* Y, int64_t ldy,
                              uint32_t* status, int32_t* max_rounds, uint32_t* range, double* fro, GridBarrier* bar,
                              int sms, cudaStream_t st);
// The FP64 sketch of a problem in host memory the device reads in place
// (A, b: device-usable addresses of pinned or registered host memory, row
// stride lda): the same Y as sketch_apply, and every entry is also stored to
// the device copy Aout (row stride ldo) and bout.
cudaError_t sketch_apply_tee(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, int64_t d,
                             int zeta, uint64_t seed, double* Y, int64_t ldy, double* Aout, int64_t ldo, double* bout,
                             uint32_t* status, int32_t* max_rounds, uint32_t* range, double* fro, int sms,
                             cudaStream_t st);
// The same range words (and DS_NONFINITE) from one read of A and b, for LSQR
// calls that do not sketch first.
cudaError_t range_scan(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, uint32_t* range,
                       uint32_t* status, int sms, cudaStream_t st);

// Preconditioner (qr.cu).  W: FP64 column-major working copy, ncol x d.
struct PrecondBuffers {
  void* W;         // ncol * d working copy (double, or float for the mixed form)
  double* rdiag;   // n
  double* R;       // n * n, row-major R when the caller passes none
  double* Mt;      // n * n, row-major transpose of M (working buffer)
  GridBarrier* bar;
  uint32_t* status;
  void* blk;       // precond_blocked_bytes(d, n) of scratch for the blocked QR, or null (unblocked)
  int mode;        // 0: choose by size, 1: unblocked, 2: blocked (LSQ_QR_*)
};
// Scratch the blocked Householder QR needs for a d x (n+1) sketch.
size_t precond_blocked_bytes(int64_t d, int64_t n);
// dst = src^T for a row-major n x n matrix.
cudaError_t transpose_square(const double* src, int n, double* dst, cudaStream_t st);
template <typename TY>
cudaError_t precond(const TY* Y, int64_t d, int64_t n, int64_t ldy, int has_b, double* R, double* M, double* x0,
                    const PrecondBuffers& buf, int sms, cudaStream_t st);

// Tensor-core GEMMs of the blocked QR's trailing updates (tc_gemm.cu): D = A B^T
// from exact bf16 slices of A's and B's rows ([S][rows][Kpad], K contiguous,
// row exponents ea/eb), S = 7 for FP64 data, 3 for FP32.
struct OzGemm {
  int S;
  const void* a;  // __nv_bfloat16 slices of A's M rows
  const void* b;  // __nv_bfloat16 slices of B's N rows
  int M, N, K, Kpad;
  int a_rows, b_rows;  // rows per slice in the slice arrays (>= M resp. N, >= the 128 / 64 row boxes)
  const int* ea;
  const int* eb;
  int mode;       // 0: out[a * ldo + b] += D (FP64 atomics, out zeroed by the caller); 1: out[b * ldo + a] -= D
  int out_f32;    // mode 1: out is float
  void* out;
  int64_t ldo;
  int k_split;    // mode 0: K per CTA, a multiple of 128
  uint32_t* status;
  const GridBarrier* bar;
};
int oz_kpad(int K);
// Slices of R rows of length K (row r at X + r ldx), or with T (b x b, K = b)
// of the rows of U T^T for column-major U (X, ld ldx); out is [S][Rpad][Kpad]
// with zero rows past R and zero columns past K.
template <typename TX>
cudaError_t oz_slice(const TX* X, int R, int K, int64_t ldx, const double* T, int S, void* out, int Kpad, int* ex,
                     int Rpad, int sms, cudaStream_t st);
cudaError_t oz_gemm(const OzGemm& g, cudaStream_t st);

// LSQR and the accuracy pass (lsqr.cu).
struct LsqrParams {
  const double* A;
  int64_t m;
  int n;
  int npad;
  int64_t lda;
  const double* b;
  float2* asplit;    // m x ldi float-pair image of A (pair-major per column pair) written by the first pass, or null
  int64_t ldi;       // image row length: n rounded up to even
  bool a_ring;       // A rows can come through bulk copies (n even, lda even, A 16-byte aligned)
  bool vec;          // A rows allow 16-byte vector loads (lda even, A aligned)
  int ring_k;        // consecutive row steps per ring buffer (1 for the single-problem kernel)
  const uint32_t* range;  // [2]: largest (high word & 0x7FF00000) over A's and b's entries, or null:
                          // exponent shifts of the double-float passes (pass_scale)
  const double* M;   // n x n row-major (upper triangular), may be null in check mode
  const double* Mt;  // transpose of M, row-major
  double* x;         // in: start, out: solution
  double* u;         // m
  double* v;         // n
  double* vhat;      // n
  double* w;         // n
  double* wv;        // n
  double* g;         // n
  double* gpart;     // gparts * npad partial sums of A^T y (per block or per warp)
  int gparts;        // rows of gpart in use (set by the pass)
  double* part;      // grid * 4
  double tol;
  int64_t maxit;
  int mode;          // 0 = LSQR then check, 1 = check only, 2 = LSQR only,
                     // 3 = heavy-ball momentum then check, 4 = heavy-ball momentum only
  double hbm_alpha, hbm_beta;  // step and momentum of modes 3 and 4
  double gate;       // > 0: the accuracy pass raises DS_ACCURACY when min(eta_ne, eta_pre) > gate
  const double* fro_in;  // sum of A_ij^2 formed by the sketch (FP64), or null: the accuracy pass forms it
  int gidx, gcount;  // this block's index among the blocks sharing the problem (set in-kernel)
  GridBarrier* bar;
  uint32_t* status;
  double* out;       // kOutSlots doubles of results
};
enum {
  OUT_ITERS = 0,
  OUT_STOP,
  OUT_NORMAL_REL,
  OUT_RNORM,
  OUT_ARNORM,
  OUT_FRO,
  OUT_XNORM,
  OUT_BNORM,
  OUT_ETA_NE,
  OUT_ETA_PRE,
  OUT_MARNORM,
  OUT_ANORM_EST,
  // serving only: %globaltimer (ns) when the group's first block joined, when
  // the group was complete, and after the sketch, the preconditioner and LSQR
  OUT_T_JOIN = 12,
  OUT_T_START,
  OUT_T_SKETCH,
  OUT_T_PRECOND,
  OUT_T_END,
  // %globaltimer (ns) when block 0 started the final accuracy pass and when
  // the pass had finished on every block (the first barrier after it)
  OUT_T_CHECK0 = 17,
  OUT_T_CHECK1,
  kOutSlots = 24
};
// Widest problem of the LSQR kernels (the panel kernel shares a row among
// up to 8 warps of 512 columns each).
constexpr int kLsqrMaxN = 4096;
// True when the double-float LSQR kernel applies (1 <= n <= kLsqrMaxN).
bool lsqr_df_ok(const double* A, int64_t n, int64_t lda);
// True when the one-warp-per-row native-FP64 LSQR kernel applies: n <= 512
// (LSQ_FLAG_NATIVE_FP64 runs the column-panel native kernel beyond that).
bool lsqr_native_ok(int64_t n);
// Rows of gpart the LSQR kernel needs for a grid (per-warp partials).
int lsqr_gparts(int grid);
// Grid size the LSQR kernel will use for n (co-resident blocks).
int lsqr_grid(int n, bool vec, bool native, int sms);
cudaError_t lsqr_run(const LsqrParams& p, bool vec, bool native, int grid, cudaStream_t st);
// The kernel families behind lsqr_grid / lsqr_run (lsqr_rows.cu: double-float,
// one warp per row, `chunks` column pairs per lane; lsqr_wide.cu: double-float,
// `panels` warps per row; lsqr_native.cu: native FP64).  Grid 0 = unusable.
int lsqr_rows_grid(int chunks, int n, int sms);
cudaError_t lsqr_rows_run(int chunks, const LsqrParams& p, int grid, cudaStream_t st);
int lsqr_wide_grid(int panels, int n, int sms);
cudaError_t lsqr_wide_run(int panels, const LsqrParams& p, int grid, cudaStream_t st);
int lsqr_native_grid(int chunks, bool vec, int sms);
// Native FP64 kernels for 512 < n <= 4096 (panels = 2, 4 or 8 warps per row).
int lsqr_native_wide_grid(int panels, int sms);
cudaError_t lsqr_native_wide_run(int panels, const LsqrParams& p, int grid, cudaStream_t st);
cudaError_t lsqr_native_run(int chunks, bool vec, const LsqrParams& p, int grid, cudaStream_t st);
// Self-test of the bounded device waits: kind 0 -- a grid barrier of `blocks`
// co-resident blocks that expects one block more (it can never fill); kind 1
// -- an mbarrier phase that nothing completes.  Both give up after the
// barrier word's limit_us and raise DS_TIMEOUT in *status.
cudaError_t wait_selftest(int kind, GridBarrier* bar, uint32_t* status, int blocks, cudaStream_t st);

// Sparse A in CSR form (sparse.cu): structure check (sets DS_CSR), sketch of the nonzeros (Y zeroed by the
// caller, ldy >= n + 1 with b), and the LSQR kernel over the nonzeros.
cudaError_t check_csr(const int64_t* rp, const int32_t* ci, int64_t m, int64_t n, int64_t nnz, uint32_t* status,
                      int sms, cudaStream_t st);
cudaError_t sketch_csr(const int64_t* rp, const int32_t* ci, const double* va, const double* b, int64_t m, int64_t n,
                       int64_t d, int zeta, uint64_t seed, double* Y, int64_t ldy, uint32_t* status,
                       int32_t* max_rounds, int sms, cudaStream_t st);
// lanes: lanes per row of the LSQR pass (csr_lanes picks it from the mean row length).
int csr_lanes(int64_t m, int64_t nnz);
int lsqr_csr_grid(int sms, int lanes);
cudaError_t lsqr_csr_run(const LsqrParams& p, const int64_t* rp, const int32_t* ci, const double* va, int grid,
                         int lanes, cudaStream_t st);

// Calibration fills (calib.cu): hash values in [-1, 1) into rows x cols (ld), M = I.
cudaError_t fill_hash(double* p, int64_t rows, int64_t cols, int64_t ld, uint64_t seed, int sms, cudaStream_t st);
cudaError_t fill_identity(double* M, int n, int sms, cudaStream_t st);

// Batched solves (batch.cu).
struct BatchTuning;
BatchTuning* batch_tuning_new();
void batch_tuning_free(BatchTuning* t);
struct BatchLayout {
  size_t oY, oW, oR, oM, oMt, oRd, oU, oVec, oGpart, oPart, oImg, oRange, slab;
  int npad_max;
};
BatchLayout batch_layout(int64_t m_max, int n_max, int d_max);
int batch_ring_elems(int n);
int batch_grid(int ring_elems, int sms);
size_t batch_item_bytes();
void batch_items_fill(void* dst, const lsq_batch_item* src, int64_t count, const BatchTuning* tune);
cudaError_t batch_launch(const void* items_dev, const int32_t* order_dev, int count, int32_t* next_dev, char* ws,
                         const BatchLayout& L, double tol, int64_t maxit, int mode, double* out, uint32_t* status,
                         GridBarrier* bar, int grid, int ring_elems, cudaStream_t st);
void batch_shape_candidates(int n, std::vector<int>& out);
int batch_bucket_of(int n);
void batch_set_shape(BatchTuning* t, int bucket, int shape);
int batch_get_shape(const BatchTuning* t, int bucket);
void batch_set_item_shape(void* items, int64_t i, int shape);
// Largest n a pass shape takes (0: no such shape).
int batch_shape_maxn(int shape);

}  // namespace lsq
