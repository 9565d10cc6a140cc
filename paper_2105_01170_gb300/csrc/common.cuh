// Shared device helpers for the sma kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sma.h"

#define SMA_STATUS_BIT(s) (1 << (int)(s))

namespace sma {

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr double v = 5.9604644775390625e-08; };
template <> struct Eps<double> { static constexpr double v = 1.1102230246251565e-16; };

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum of a double; `red` must hold >= 32 doubles.  Every thread
// gets the result.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = (threadIdx.x < (unsigned)nw) ? red[threadIdx.x] : 0.0;
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}

}  // namespace sma

// ---------------------------------------------------------------------------
// Launchers implemented in the .cu files (host side, enqueue on `st`).
// ---------------------------------------------------------------------------
namespace sma {

// Generic strided, two-level-batched GEMM on CUDA cores:
//   C(i,j) = alpha * sum_k A(i,k) B(k,j) + beta * C(i,j)
// with A(i,k) = A[i*a_rs + k*a_cs], B(k,j) = B[k*b_rs + j*b_cs],
// C(i,j) = C[i*c_rs + j*c_cs]; batch index z = b1 + nb1*b2 adds
// b1*x_b1 + b2*x_b2 to each pointer.  Optional device-side per-b1 sizes
// dM/dN/dK clamp M/N/K (entries read at run time, so the launch can be
// enqueued before they are known).  c_off, if set, replaces the batch offset
// of C by c_off[b1]*c_off_mul.
template <typename T>
struct GemmParams {
  int M = 0, N = 0, K = 0;
  const int* dM = nullptr;
  const int* dN = nullptr;
  const int* dK = nullptr;
  const int* dKoff = nullptr;  // optional: K range starts at dKoff[dstride * b1]
  int dstride = 1;   // dM/dN/dK/dKoff are read at [dstride * b1] (0 = one shared value)
  const T* A = nullptr; int64_t a_rs = 0, a_cs = 0, a_b1 = 0, a_b2 = 0;
  const T* B = nullptr; int64_t b_rs = 0, b_cs = 0, b_b1 = 0, b_b2 = 0;
  T* C = nullptr; int64_t c_rs = 0, c_cs = 0, c_b1 = 0, c_b2 = 0;
  const int* c_off = nullptr; int64_t c_off_mul = 0;
  // optional (fp32 only): write C as three bf16 planes (hi, mid, lo) at the
  // same offsets, plane p at Cs + p*cs_plane, instead of writing C
  void* Cs = nullptr; int64_t cs_plane = 0;
  int nb1 = 1, nb2 = 1;
  T alpha = T(1), beta = T(0);
  // > 0: split K, batch index b1 takes the range [b1 kchunk, (b1 + 1) kchunk)
  // (A and B then usually have no b1 offset; each b1 writes its own partial C)
  int kchunk = 0;
};

template <typename T> cudaError_t gemm(const GemmParams<T>& p, cudaStream_t st);

}  // namespace sma
