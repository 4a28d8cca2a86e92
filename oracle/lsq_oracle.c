/*
 * lsq_oracle.c -- CPU oracle for sparse-sign sketch-and-precondition least
 * squares (arXiv 2506.03070).  TEST INFRASTRUCTURE ONLY: the tests, the smoke
 * check and the benchmark's CPU-baseline leg use it to check and time the CUDA
 * library; the library itself never links, loads or calls anything here.
 *
 * Plain, slow, obviously correct, single-threaded, FP64 throughout.  No
 * blocking, no fusion, no reordering beyond what each cited definition or
 * algorithm states.  It shares no code with the CUDA path.
 *
 * Conventions: every matrix is row-major with an explicit leading dimension;
 * indices are 0-based (the paper's [d] = {1..d} read as {0..d-1}).
 *
 * Functions and the passages they follow:
 *   orc_philox4x64_10   Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11).
 *   orc_sketch_row      Sec. 3.1.2 rejection sampling of one sketch column
 *                       (steps (i)-(iv)) and the random signs of Algorithm 3.
 *   orc_sketch_indices  the same over a range of columns of S.
 *   orc_sketch_apply    Y = S [A | b], Sec. 2.1 (Def. of the sparse sign
 *                       sketch) and Algorithm 1 step "Form Y = SA".
 *   orc_householder_qr  Algorithm 1 step "Factor Q, R = QR(Y)" as textbook
 *                       unblocked Householder QR (Golub & Van Loan 5.2.1).
 *   orc_tri_inverse     Algorithm 1 step "M = R^{-1}" (Sec. 3.2: explicit inverse).
 *   orc_lsqr            Algorithm 2 (preconditioned LSQR), two-pass matvecs.
 *   orc_backward_error  normwise backward error of a least-squares solution.
 *   orc_solve           Algorithm 1 end to end.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Built two ways.  The checker build (tests, smoke) is plain single-threaded
 * C: every loop runs in the order written here.  The CPU-baseline build adds
 * -fopenmp: the row loops of the sketch and of the matvecs, the trailing
 * columns of each Householder step and the columns of the inverse run on all
 * host threads (partial sums of per-thread copies added in thread order), the
 * same operations in a different summation order.  Nothing else changes. */

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_SKETCH (-2) /* rejection sampling exceeded the round cap */
#define ORC_ERR_RANK (-3)
#define ORC_ERR_NOCONV (-4)
#define ORC_ERR_OOM (-5)

#define ORC_MAX_ZETA 64
#define ORC_MAX_ROUNDS 10000

/* ---------------------------------------------------------------------------
 * Philox4x64-10.  State: four 64-bit counter words, two 64-bit key words.
 * One round: two 64x64->128 multiplies of counter words 0 and 2 by fixed odd
 * multipliers; the outputs are (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2),
 * hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)).  Between rounds the key is advanced by
 * the two Weyl constants.  Ten rounds.
 * ------------------------------------------------------------------------- */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint64_t k[2] = {key_in[0], key_in[1]};
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k[0] += W0;
      k[1] += W1;
    }
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(M0, c[0], &hi0, &lo0);
    mulhilo64(M1, c[2], &hi1, &lo1);
    uint64_t n0 = hi1 ^ c[1] ^ k[0];
    uint64_t n1 = lo1;
    uint64_t n2 = hi0 ^ c[3] ^ k[1];
    uint64_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Random stream layout (our reading; the paper's CuPy generator is unnamed):
 *   key = (seed, 0).
 *   index draw for column i of S, redraw round r, slot j:
 *       counter (i, r, j/4, 0), word j%4, mapped to [0,d) as floor(u*d/2^64).
 *   sign for column i, sorted slot k (k < 64):
 *       counter (i, 0, 0, 1), bit k of word 0; 1 -> +1/sqrt(zeta), 0 -> -1/sqrt(zeta).
 */
static uint64_t draw_word(uint64_t seed, uint64_t i, uint64_t r, int j) {
  uint64_t ctr[4] = {i, r, (uint64_t)(j / 4), 0};
  uint64_t key[2] = {seed, 0};
  uint64_t out[4];
  orc_philox4x64_10(ctr, key, out);
  return out[j % 4];
}

static int32_t draw_index(uint64_t seed, uint64_t i, uint64_t r, int j, int64_t d) {
  uint64_t u = draw_word(seed, i, r, j);
  uint64_t hi, lo;
  mulhilo64(u, (uint64_t)d, &hi, &lo);
  return (int32_t)hi;
}

static uint64_t sign_word(uint64_t seed, uint64_t i) {
  uint64_t ctr[4] = {i, 0, 0, 1};
  uint64_t key[2] = {seed, 0};
  uint64_t out[4];
  orc_philox4x64_10(ctr, key, out);
  return out[0];
}

/* insertion sort, ascending */
static void sort_ints(int32_t* c, int n) {
  for (int a = 1; a < n; ++a) {
    int32_t v = c[a];
    int b = a - 1;
    while (b >= 0 && c[b] > v) {
      c[b + 1] = c[b];
      --b;
    }
    c[b + 1] = v;
  }
}

/* One column of S (Sec. 3.1.2): (i) draw zeta indices with replacement;
 * (ii) sort and compare neighbours; (iii) replace each duplicate -- the
 * earlier position j of every equal pair (j, j+1) -- with a fresh draw;
 * (iv) repeat until all entries differ.  Then the signs of Algorithm 3, one
 * per sorted slot.  Returns the number of redraw rounds used, or
 * ORC_ERR_SKETCH past the cap. */
int orc_sketch_row(uint64_t seed, int64_t i, int64_t d, int zeta, int32_t* idx, int8_t* sgn) {
  int32_t c[ORC_MAX_ZETA];
  int dup[ORC_MAX_ZETA];
  for (int j = 0; j < zeta; ++j) c[j] = draw_index(seed, (uint64_t)i, 0, j, d);
  sort_ints(c, zeta);
  int r = 0;
  for (;;) {
    int ndup = 0;
    for (int j = 0; j + 1 < zeta; ++j) {
      dup[j] = (c[j] == c[j + 1]);
      ndup += dup[j];
    }
    if (ndup == 0) break;
    ++r;
    if (r > ORC_MAX_ROUNDS) return ORC_ERR_SKETCH;
    for (int j = 0; j + 1 < zeta; ++j)
      if (dup[j]) c[j] = draw_index(seed, (uint64_t)i, (uint64_t)r, j, d);
    sort_ints(c, zeta);
  }
  uint64_t sw = sign_word(seed, (uint64_t)i);
  for (int k = 0; k < zeta; ++k) {
    idx[k] = c[k];
    sgn[k] = ((sw >> k) & 1ULL) ? (int8_t)1 : (int8_t)-1;
  }
  return r;
}

static int check_sketch_args(int64_t d, int zeta) {
  if (zeta < 1 || zeta > ORC_MAX_ZETA || d < 1 || (int64_t)zeta > d || d > 2147483647LL) return ORC_ERR_ARG;
  return ORC_OK;
}

/* Columns row0 .. row0+rows-1 of S: idx and sgn are rows x zeta row-major. */
int orc_sketch_indices(uint64_t seed, int64_t row0, int64_t rows, int64_t d, int zeta, int32_t* idx, int8_t* sgn,
                       int32_t* rounds) {
  if (check_sketch_args(d, zeta) != ORC_OK || rows < 0 || row0 < 0) return ORC_ERR_ARG;
  for (int64_t t = 0; t < rows; ++t) {
    int r = orc_sketch_row(seed, row0 + t, d, zeta, idx + t * zeta, sgn + t * zeta);
    if (r < 0) return r;
    if (rounds) rounds[t] = r;
  }
  return ORC_OK;
}

/* Y (d x ldy, row-major) = sum over rows i of A of s_ik [A_i, b_i] placed in
 * row c_ik of Y.  The sketch uses global column index row0 + i so a row
 * partition of A reproduces slices of the same S (App. B, sketching).
 * b may be NULL (then only n columns are written).  Y is overwritten. */
int orc_sketch_apply(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, int64_t d, int zeta,
                     uint64_t seed, int64_t row0, double* Y, int64_t ldy) {
  int64_t ncol = n + (b ? 1 : 0);
  if (check_sketch_args(d, zeta) != ORC_OK || m < 0 || n < 1 || lda < n || ldy < ncol) return ORC_ERR_ARG;
  for (int64_t r = 0; r < d; ++r)
    for (int64_t j = 0; j < ldy; ++j) Y[r * ldy + j] = 0.0;
  const double scale = 1.0 / sqrt((double)zeta);
#ifdef _OPENMP
  /* CPU-baseline build: each thread sketches a contiguous block of rows into
   * its own copy of Y; the copies are added in thread order */
  const int nt = omp_get_max_threads();
  double* priv = nt > 1 ? (double*)calloc((size_t)nt * (size_t)d * (size_t)ldy, sizeof(double)) : NULL;
  if (priv) {
    int fail = 0;
#pragma omp parallel num_threads(nt)
    {
      double* Yt = priv + (size_t)omp_get_thread_num() * (size_t)d * (size_t)ldy;
      int32_t idx[ORC_MAX_ZETA];
      int8_t sgn[ORC_MAX_ZETA];
#pragma omp for schedule(static)
      for (int64_t i = 0; i < m; ++i) {
        if (orc_sketch_row(seed, row0 + i, d, zeta, idx, sgn) < 0) {
#pragma omp atomic write
          fail = 1;
          continue;
        }
        for (int k = 0; k < zeta; ++k) {
          double s = sgn[k] > 0 ? scale : -scale;
          double* y = Yt + (int64_t)idx[k] * ldy;
          for (int64_t j = 0; j < n; ++j) y[j] += s * A[i * lda + j];
          if (b) y[n] += s * b[i];
        }
      }
    }
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < d; ++r)
      for (int t = 0; t < nt; ++t)
        for (int64_t j = 0; j < ldy; ++j) Y[r * ldy + j] += priv[((size_t)t * d + r) * ldy + j];
    free(priv);
    return fail ? ORC_ERR_SKETCH : ORC_OK;
  }
#endif
  int32_t idx[ORC_MAX_ZETA];
  int8_t sgn[ORC_MAX_ZETA];
  for (int64_t i = 0; i < m; ++i) {
    int rc = orc_sketch_row(seed, row0 + i, d, zeta, idx, sgn);
    if (rc < 0) return rc;
    for (int k = 0; k < zeta; ++k) {
      double s = sgn[k] > 0 ? scale : -scale;
      double* y = Y + (int64_t)idx[k] * ldy;
      for (int64_t j = 0; j < n; ++j) y[j] += s * A[i * lda + j];
      if (b) y[n] += s * b[i];
    }
  }
  return ORC_OK;
}

/* In-place Householder QR of the rows x cols matrix Y (row-major, ld).
 * For k = 0..min(rows,cols)-1: build the reflector H_k = I - tau_k v v^T that
 * maps Y[k:,k] to beta*e_1 with beta = -sign(Y[k][k]) * ||Y[k:,k]|| (the sign
 * avoids cancellation), apply it to columns k+1.., store beta in Y[k][k] and
 * v[1:] below it (v[0] = 1 implicit).  If Y[k+1:,k] is already zero, tau_k = 0.
 * Afterwards the upper triangle of Y holds R. */
int orc_householder_qr(double* Y, int64_t rows, int64_t cols, int64_t ld, double* tau) {
  if (rows < 1 || cols < 1 || ld < cols) return ORC_ERR_ARG;
  int64_t kmax = rows < cols ? rows : cols;
  for (int64_t k = 0; k < kmax; ++k) {
    double alpha = Y[k * ld + k];
    double sigma = 0.0;
    for (int64_t i = k + 1; i < rows; ++i) sigma += Y[i * ld + k] * Y[i * ld + k];
    if (sigma == 0.0) {
      tau[k] = 0.0;
      continue;
    }
    double norm = sqrt(alpha * alpha + sigma);
    double beta = alpha >= 0.0 ? -norm : norm;
    double v0 = alpha - beta;
    tau[k] = (beta - alpha) / beta;
    for (int64_t i = k + 1; i < rows; ++i) Y[i * ld + k] /= v0;
    Y[k * ld + k] = beta;
#pragma omp parallel for schedule(static)
    for (int64_t j = k + 1; j < cols; ++j) {
      double dot = Y[k * ld + j];
      for (int64_t i = k + 1; i < rows; ++i) dot += Y[i * ld + k] * Y[i * ld + j];
      double f = tau[k] * dot;
      Y[k * ld + j] -= f;
      for (int64_t i = k + 1; i < rows; ++i) Y[i * ld + j] -= f * Y[i * ld + k];
    }
  }
  return ORC_OK;
}

/* M = R^{-1} for upper-triangular R (n x n, ldr): column c of M solves
 * R m_c = e_c by back substitution.  M is upper triangular (ldm).
 * Returns ORC_ERR_RANK if a diagonal entry of R is zero. */
int orc_tri_inverse(const double* R, int64_t n, int64_t ldr, double* M, int64_t ldm) {
  if (n < 1 || ldr < n || ldm < n) return ORC_ERR_ARG;
  for (int64_t i = 0; i < n; ++i)
    if (R[i * ldr + i] == 0.0) return ORC_ERR_RANK;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t c = 0; c < n; ++c) M[i * ldm + c] = 0.0;
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t c = 0; c < n; ++c) {
    M[c * ldm + c] = 1.0 / R[c * ldr + c];
    for (int64_t i = c - 1; i >= 0; --i) {
      double s = 0.0;
      for (int64_t k = i + 1; k <= c; ++k) s += R[i * ldr + k] * M[k * ldm + c];
      M[i * ldm + c] = -s / R[i * ldr + i];
    }
  }
  return ORC_OK;
}

/* y = A x (m), y = A^T z (n), y = M x, y = M^T x : plain loops */
static void mv_A(const double* A, int64_t m, int64_t n, int64_t lda, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += A[i * lda + j] * x[j];
    y[i] = s;
  }
}
static void mv_At(const double* A, int64_t m, int64_t n, int64_t lda, const double* z, double* y) {
  for (int64_t j = 0; j < n; ++j) y[j] = 0.0;
#ifdef _OPENMP
  /* CPU-baseline build: per-thread partial sums over contiguous row blocks,
   * added in thread order */
  const int nt = omp_get_max_threads();
  double* part = nt > 1 ? (double*)calloc((size_t)nt * (size_t)n, sizeof(double)) : NULL;
  if (part) {
#pragma omp parallel num_threads(nt)
    {
      double* yt = part + (size_t)omp_get_thread_num() * (size_t)n;
#pragma omp for schedule(static)
      for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) yt[j] += A[i * lda + j] * z[i];
    }
    for (int t = 0; t < nt; ++t)
      for (int64_t j = 0; j < n; ++j) y[j] += part[(size_t)t * n + j];
    free(part);
    return;
  }
#endif
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) y[j] += A[i * lda + j] * z[i];
}
static void mv_M(const double* M, int64_t n, const double* x, double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = 0; k < n; ++k) s += M[i * n + k] * x[k];
    y[i] = s;
  }
}
static void mv_Mt(const double* M, int64_t n, const double* x, double* y) {
  for (int64_t k = 0; k < n; ++k) y[k] = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = 0; k < n; ++k) y[k] += M[i * n + k] * x[i];
}
static double nrm2(const double* x, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += x[i] * x[i];
  return sqrt(s);
}

typedef struct {
  int64_t iters;      /* iterations t performed */
  int32_t stop;       /* 1 normal-equation test, 2 residual test, 3 maxit, 4 breakdown */
  int32_t pad;
  double anorm_est;   /* sqrt(sum alpha^2 + beta^2): estimate of ||A M||_F */
  double normal_rel;  /* last ||(AM)^T r|| / (||AM|| ||r||) estimate */
  double rnorm_est;   /* last phibar estimate of ||r|| */
} orc_lsqr_info;

/* Algorithm 2 (preconditioned LSQR), the paper's order of updates, with the
 * matvecs A(Mv) and M^T(A^T u) as separate passes.  The stopping test
 * (Algorithm 2 leaves it open) is, on the preconditioned problem,
 *   phibar_{t+1} alpha_{t+1} |c_t| <= tol * anorm_est * phibar_{t+1}
 *       (normal-equation residual ||(AM)^T r_t|| relative to ||AM|| ||r_t||), or
 *   phibar_{t+1} <= tol * ||b||                 (consistent systems), or t = maxit.
 * M is n x n row-major (ld n).  x receives the final iterate.  trace, if not
 * NULL, receives x_t for t = 1..iters (iters x n row-major); alpha_beta, if not
 * NULL, receives (alpha_t, beta_t) for t = 1..iters+1. */
int orc_lsqr(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, const double* M, const double* x0,
             double tol, int64_t maxit, double* x, orc_lsqr_info* info, double* trace, double* alpha_beta) {
  if (m < 1 || n < 1 || lda < n || maxit < 0) return ORC_ERR_ARG;
  double* u = (double*)malloc(sizeof(double) * m);
  double* v = (double*)malloc(sizeof(double) * n);
  double* w = (double*)malloc(sizeof(double) * n);
  double* tn = (double*)malloc(sizeof(double) * n);
  double* tn2 = (double*)malloc(sizeof(double) * n);
  double* tm = (double*)malloc(sizeof(double) * m);
  if (!u || !v || !w || !tn || !tn2 || !tm) {
    free(u); free(v); free(w); free(tn); free(tn2); free(tm);
    return ORC_ERR_OOM;
  }
  double bnorm = nrm2(b, m);
  /* beta_1 u_1 = b - A x_0 */
  for (int64_t j = 0; j < n; ++j) x[j] = x0[j];
  mv_A(A, m, n, lda, x, tm);
  for (int64_t i = 0; i < m; ++i) u[i] = b[i] - tm[i];
  double beta = nrm2(u, m);
  double alpha = 0.0;
  if (beta > 0.0) {
    for (int64_t i = 0; i < m; ++i) u[i] /= beta;
    /* alpha_1 v_1 = M^T A^T u_1 */
    mv_At(A, m, n, lda, u, tn);
    mv_Mt(M, n, tn, v);
    alpha = nrm2(v, n);
    if (alpha > 0.0)
      for (int64_t j = 0; j < n; ++j) v[j] /= alpha;
  }
  if (alpha_beta) { alpha_beta[0] = alpha; alpha_beta[1] = beta; }
  /* w_1 = M v_1, phibar_1 = beta_1, rhobar_1 = alpha_1 */
  mv_M(M, n, v, w);
  double phibar = beta, rhobar = alpha;
  double anorm2 = alpha * alpha;
  int32_t stop = 3;
  int64_t t = 0;
  double normal_rel = 0.0;
  if (beta == 0.0 || alpha == 0.0) {
    stop = 4;
  } else {
    for (t = 1; t <= maxit; ++t) {
      /* uhat = A M v_t - alpha_t u_t ; beta_{t+1} = ||uhat|| ; u_{t+1} = uhat / beta */
      mv_M(M, n, v, tn);
      mv_A(A, m, n, lda, tn, tm);
      for (int64_t i = 0; i < m; ++i) u[i] = tm[i] - alpha * u[i];
      beta = nrm2(u, m);
      if (beta > 0.0)
        for (int64_t i = 0; i < m; ++i) u[i] /= beta;
      /* vhat = M^T A^T u_{t+1} - beta_{t+1} v_t ; alpha_{t+1} = ||vhat|| */
      mv_At(A, m, n, lda, u, tn);
      mv_Mt(M, n, tn, tn2);
      for (int64_t j = 0; j < n; ++j) v[j] = tn2[j] - beta * v[j];
      alpha = nrm2(v, n);
      if (alpha > 0.0)
        for (int64_t j = 0; j < n; ++j) v[j] /= alpha;
      if (alpha_beta) { alpha_beta[2 * t] = alpha; alpha_beta[2 * t + 1] = beta; }
      anorm2 += alpha * alpha + beta * beta;
      /* Givens rotation */
      double rho = sqrt(rhobar * rhobar + beta * beta);
      double c = rhobar / rho;
      double s = beta / rho;
      double theta = s * alpha;
      rhobar = -c * alpha;
      double phi = c * phibar;
      phibar = s * phibar;
      /* x_t = x_{t-1} + (phi/rho) w_t ; w_{t+1} = M v_{t+1} - (theta/rho) w_t */
      for (int64_t j = 0; j < n; ++j) x[j] += (phi / rho) * w[j];
      mv_M(M, n, v, tn);
      for (int64_t j = 0; j < n; ++j) w[j] = tn[j] - (theta / rho) * w[j];
      if (trace)
        for (int64_t j = 0; j < n; ++j) trace[(t - 1) * n + j] = x[j];
      double anorm = sqrt(anorm2);
      normal_rel = alpha * fabs(c) / anorm;
      if (normal_rel <= tol) { stop = 1; break; }
      if (phibar <= tol * bnorm) { stop = 2; break; }
      if (beta == 0.0 || alpha == 0.0) { stop = 4; break; }
    }
    if (t > maxit) t = maxit;
  }
  if (info) {
    info->iters = t;
    info->stop = stop;
    info->anorm_est = sqrt(anorm2);
    info->normal_rel = normal_rel;
    info->rnorm_est = phibar;
  }
  free(u); free(v); free(w); free(tn); free(tn2); free(tm);
  return stop == 3 && maxit > 0 ? ORC_ERR_NOCONV : ORC_OK;
}

/* Normwise backward error of x as a least-squares solution of min ||b - A x||:
 *   eta = ||A^T r|| / (||A||_F ||r||),  r = b - A x  (FP64),
 * and, when ||r|| <= tol ||b|| (consistent case),
 *   eta = ||r|| / (||A||_F ||x|| + ||b||).
 * Also returns ||r||, ||A^T r|| and ||A||_F through out[0..2] if out != NULL. */
double orc_backward_error(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, const double* x,
                          double tol, double* out) {
  double* r = (double*)malloc(sizeof(double) * m);
  double* g = (double*)malloc(sizeof(double) * n);
  if (!r || !g) { free(r); free(g); return -1.0; }
  mv_A(A, m, n, lda, x, r);
  for (int64_t i = 0; i < m; ++i) r[i] = b[i] - r[i];
  mv_At(A, m, n, lda, r, g);
  double fro = 0.0;
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) fro += A[i * lda + j] * A[i * lda + j];
  fro = sqrt(fro);
  double rn = nrm2(r, m), gn = nrm2(g, n), bn = nrm2(b, m), xn = nrm2(x, n);
  double eta;
  if (rn <= tol * bn)
    eta = rn / (fro * xn + bn);
  else
    eta = gn / (fro * rn);
  if (out) { out[0] = rn; out[1] = gn; out[2] = fro; }
  free(r); free(g);
  return eta;
}

typedef struct {
  int64_t iters;
  int32_t stop;
  int32_t sketch_rounds_max;
  double backward_error;
  double anorm_est;
} orc_solve_info;

/* Algorithm 1 with the sparse sign sketch and LSQR:
 *   Y = S [A | b] (d x (n+1)); Householder QR of Y gives R_aug = [[R, z],[0, rho]]
 *   with z = (Q^T S b)[:n]; M = R^{-1}; x0 = M z (the sketch-and-solve
 *   solution argmin ||S b - S A x||); then Algorithm 2 from x0.
 * x (n) receives the solution; R and M (n x n each, ld n) if not NULL. */
int orc_solve(const double* A, int64_t m, int64_t n, int64_t lda, const double* b, int64_t d, int zeta, uint64_t seed,
              double tol, int64_t maxit, double* x, double* R_out, double* M_out, double* x0_out,
              orc_solve_info* info) {
  if (d < n + 1) return ORC_ERR_ARG;
  int64_t ldy = n + 1;
  double* Y = (double*)malloc(sizeof(double) * d * ldy);
  double* tau = (double*)malloc(sizeof(double) * ldy);
  double* R = (double*)malloc(sizeof(double) * n * n);
  double* M = (double*)malloc(sizeof(double) * n * n);
  double* z = (double*)malloc(sizeof(double) * n);
  double* x0 = (double*)malloc(sizeof(double) * n);
  int rc = ORC_OK;
  if (!Y || !tau || !R || !M || !z || !x0) { rc = ORC_ERR_OOM; goto done; }
  rc = orc_sketch_apply(A, m, n, lda, b, d, zeta, seed, 0, Y, ldy);
  if (rc != ORC_OK) goto done;
  rc = orc_householder_qr(Y, d, ldy, ldy, tau);
  if (rc != ORC_OK) goto done;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j < n; ++j) R[i * n + j] = j >= i ? Y[i * ldy + j] : 0.0;
    z[i] = Y[i * ldy + n];
  }
  rc = orc_tri_inverse(R, n, n, M, n);
  if (rc != ORC_OK) goto done;
  mv_M(M, n, z, x0);
  {
    orc_lsqr_info li;
    rc = orc_lsqr(A, m, n, lda, b, M, x0, tol, maxit, x, &li, NULL, NULL);
    if (info) {
      info->iters = li.iters;
      info->stop = li.stop;
      info->anorm_est = li.anorm_est;
      info->sketch_rounds_max = 0;
      info->backward_error = orc_backward_error(A, m, n, lda, b, x, tol, NULL);
    }
  }
  if (R_out) memcpy(R_out, R, sizeof(double) * n * n);
  if (M_out) memcpy(M_out, M, sizeof(double) * n * n);
  if (x0_out) memcpy(x0_out, x0, sizeof(double) * n);
done:
  free(Y); free(tau); free(R); free(M); free(z); free(x0);
  return rc;
}

/* Threads of the CPU-baseline build's parallel loops (no effect on the
 * single-threaded checker build).  Not arithmetic: the per-thread partial
 * sums are added in thread order either way. */
void orc_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}
