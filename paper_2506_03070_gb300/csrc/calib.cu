// calib.cu -- synthetic fills for the embedding-dimension calibration: the
// library times its own QR and LSQR kernels on data of a problem's width
// before choosing d (see lsq_choose_d).  Values come from a 64-bit integer
// hash of (seed, row, column) mapped to [-1, 1): dense, full rank in practice,
// and independent of any RNG library.
#include "kernels.h"

namespace lsq {
namespace {

__device__ __forceinline__ double hash_unit(uint64_t seed, uint64_t i, uint64_t j) {
  uint64_t z = seed ^ (i * 0x9E3779B97F4A7C15ull) ^ (j * 0xC2B2AE3D27D4EB4Full);
  z ^= z >> 33;
  z *= 0xFF51AFD7ED558CCDull;
  z ^= z >> 33;
  z *= 0xC4CEB9FE1A85EC53ull;
  z ^= z >> 33;
  return (double)(z >> 11) * (1.0 / 4503599627370496.0) - 1.0;  // [0, 2^53) / 2^52 - 1
}

__global__ void k_fill_hash(double* __restrict__ p, int64_t rows, int64_t cols, int64_t ld, uint64_t seed) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e % cols;
    p[i * ld + j] = hash_unit(seed, (uint64_t)i, (uint64_t)j);
  }
}

__global__ void k_fill_identity(double* __restrict__ M, int n) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    M[e] = (e / n == e % n) ? 1.0 : 0.0;
}

}  // namespace

cudaError_t fill_hash(double* p, int64_t rows, int64_t cols, int64_t ld, uint64_t seed, int sms, cudaStream_t st) {
  k_fill_hash<<<sms * 8, 256, 0, st>>>(p, rows, cols, ld, seed);
  return cudaGetLastError();
}

cudaError_t fill_identity(double* M, int n, int sms, cudaStream_t st) {
  k_fill_identity<<<sms * 2, 256, 0, st>>>(M, n);
  return cudaGetLastError();
}

}  // namespace lsq
