// Shared device helpers for the sWLR kernels (Dutta & Li, arXiv 1703.06303).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace wlr {

// Error word bits set by kernels and read back by the host.
enum : int {
  ERRBIT_NOT_SPD = 1,        // a row system diag(W1(i,:)^2) + C C^T broke down
  ERRBIT_RANK_DEFICIENT = 2, // Cholesky of X1^T X1 (or Q1^T Q1) broke down
  ERRBIT_BAD_WEIGHT = 4,     // W1 <= 0 or not finite
  ERRBIT_EIG = 8,            // the small eigensolver met a non-finite value
};

// Host: set the message that wlr_last_error(NULL) returns (calls without a handle).
void set_global_error(const char* msg);

// Round to the nearest TF32 number (10 explicit mantissa bits, ties away from zero).
__device__ __forceinline__ float round_tf32(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ float  wsqrt(float x)  { return sqrtf(x); }
__device__ __forceinline__ double wsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ bool   wfinite(float x)  { return isfinite(x); }
__device__ __forceinline__ bool   wfinite(double x) { return isfinite(x); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of one double per thread; result valid in thread 0.
__device__ __forceinline__ double block_sum_double(double v, double* sh /*>=32*/) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    r = lane < nw ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

// SplitMix64 output number n for a given seed (Steele, Lea & Flood 2014):
// state = seed + (n + 1) * gamma, then the finaliser with shifts 30/27/31.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t n) {
  uint64_t z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// N(0,1) number t of the stream: Box-Muller on outputs 2t and 2t+1.
__device__ __forceinline__ double normal_at(uint64_t seed, uint64_t t) {
  const double u1 = (double)(splitmix64_at(seed, 2ull * t) >> 11) * 0x1.0p-53;
  const double u2 = (double)(splitmix64_at(seed, 2ull * t + 1ull) >> 11) * 0x1.0p-53;
  return sqrt(-2.0 * log1p(-u1)) * cospi(2.0 * u2);
}

}  // namespace wlr
