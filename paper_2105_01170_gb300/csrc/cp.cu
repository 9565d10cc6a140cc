// CP (Kruskal) compressor by alternating least squares (Section 2.3; the
// matrix forms of Theorem tildeA and Corollary kronsumcp): the kernels the
// least-squares steps need besides the contractions, which go through gemm.
//   khatri_rao   columnwise Kronecker product of two factors
//   cp_solve     one factor update: the normal-equations matrix (Hadamard
//                product of the other two factors' Gram matrices) factored
//                in fp64 in one CTA, then every row of the contracted tensor
//                solved against it
//   sum_slabs_t  fixed-order sum of per-block partial products
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.cuh"

namespace sma {
namespace {

constexpr int CP_THREADS = 256;

// out[(a + ra b), j] = A[a, j] B[b, j] (A ra x r, B rb x r, both ld = rows).
template <typename T>
__global__ void khatri_rao_kernel(const T* __restrict__ A, int ra, const T* __restrict__ B, int rb,
                                  int r, T* __restrict__ out) {
  const int64_t rows = (int64_t)ra * rb, total = rows * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e % rows;
    const int j = (int)(e / rows);
    const int a = (int)(row % ra), b = (int)(row / ra);
    out[e] = A[a + (int64_t)j * ra] * B[b + (int64_t)j * rb];
  }
}

// out (rows x r, ld ldo) = M (rows x r, ld rows) V^-1 with
// V = (B1^T B1) .* (B2^T B2) (r x r, SPD when the factors have full column
// rank).  V is formed and Cholesky-factored in fp64 in shared memory (right-
// looking, the trailing update spread over the CTA); each thread then solves
// the rows assigned to it (L y = m, L^T x = y).  A pivot that is not finite
// or not above 64 eps times the largest diagonal entry (a numerically
// singular system) sets SMA_ERR_NONFINITE and writes zeros.
template <typename T>
__global__ void __launch_bounds__(CP_THREADS)
    cp_solve_kernel(const T* __restrict__ B1, int n1, const T* __restrict__ B2, int n2, int r,
                    const T* __restrict__ M, int rows, T* __restrict__ out, int64_t ldo,
                    int* __restrict__ status) {
  extern __shared__ double Ls[];   // r x r, column-major
  __shared__ int s_bad;
  __shared__ double s_floor;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) s_bad = 0;
  for (int e = tid; e < r * r; e += nt) {
    const int i = e % r, j = e / r;
    if (i < j) continue;
    double g1 = 0.0, g2 = 0.0;
    for (int a = 0; a < n1; ++a)
      g1 = fma((double)B1[a + (int64_t)i * n1], (double)B1[a + (int64_t)j * n1], g1);
    for (int b = 0; b < n2; ++b)
      g2 = fma((double)B2[b + (int64_t)i * n2], (double)B2[b + (int64_t)j * n2], g2);
    Ls[i + j * r] = g1 * g2;
  }
  __syncthreads();
  if (tid == 0) {
    // pivots at the rounding level of the largest diagonal entry mean a
    // numerically singular system (e.g. two equal columns in both factors)
    double dmax = 0.0;
    for (int j = 0; j < r; ++j) dmax = fmax(dmax, Ls[j + j * r]);
    s_floor = 64.0 * 2.220446049250313e-16 * dmax;
  }
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    if (tid == 0) {
      const double d = Ls[j + j * r];
      if (!(d > s_floor) || !isfinite(d)) {
        s_bad = 1;
      } else {
        Ls[j + j * r] = sqrt(d);
      }
    }
    __syncthreads();
    if (s_bad) break;
    const double piv = Ls[j + j * r];
    for (int i = j + 1 + tid; i < r; i += nt) Ls[i + j * r] /= piv;
    __syncthreads();
    // trailing lower triangle: L(i, k) -= L(i, j) L(k, j), j < k <= i
    const int t = r - j - 1;
    for (int e = tid; e < t * t; e += nt) {
      const int i = j + 1 + e % t, k = j + 1 + e / t;
      if (k <= i) Ls[i + k * r] -= Ls[i + j * r] * Ls[k + j * r];
    }
    __syncthreads();
  }
  if (s_bad) {
    for (int64_t e = tid; e < (int64_t)rows * r; e += nt) {
      const int64_t i = e % rows, j = e / rows;
      out[i + j * ldo] = T(0);
    }
    if (tid == 0) atomicOr(status, SMA_STATUS_BIT(SMA_ERR_NONFINITE));
    return;
  }
  double y[kCpMaxRank];
  for (int row = tid; row < rows; row += nt) {
    for (int i = 0; i < r; ++i) {
      double acc = (double)M[row + (int64_t)i * rows];
      for (int k = 0; k < i; ++k) acc = fma(-Ls[i + k * r], y[k], acc);
      y[i] = acc / Ls[i + i * r];
    }
    for (int i = r - 1; i >= 0; --i) {
      double acc = y[i];
      for (int k = i + 1; k < r; ++k) acc = fma(-Ls[k + i * r], y[k], acc);
      y[i] = acc / Ls[i + i * r];
    }
    for (int i = 0; i < r; ++i) out[row + (int64_t)i * ldo] = (T)y[i];
  }
}

template <typename T>
__global__ void sum_slabs_t_kernel(const T* __restrict__ part, int nslab, int64_t count,
                                   T* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < nslab; ++s) acc += (double)part[e + s * count];
    out[e] = (T)acc;
  }
}

__global__ void set_int_kernel(int* dst, int v) { *dst = v; }

int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

template <typename T>
cudaError_t khatri_rao(const T* A, int ra, const T* B, int rb, int r, T* out, cudaStream_t st) {
  khatri_rao_kernel<T><<<grid_for((int64_t)ra * rb * r), 256, 0, st>>>(A, ra, B, rb, r, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t cp_solve(const T* B1, int n1, const T* B2, int n2, int r, const T* M, int rows, T* out,
                     int64_t ldo, int* status, cudaStream_t st) {
  if (r < 1 || r > kCpMaxRank) return cudaErrorInvalidValue;
  cp_solve_kernel<T><<<1, CP_THREADS, (size_t)r * r * sizeof(double), st>>>(B1, n1, B2, n2, r, M,
                                                                             rows, out, ldo, status);
  return cudaGetLastError();
}

template <typename T>
cudaError_t sum_slabs_t(const T* part, int nslab, int64_t count, T* out, cudaStream_t st) {
  sum_slabs_t_kernel<T><<<grid_for(count), 256, 0, st>>>(part, nslab, count, out);
  return cudaGetLastError();
}

cudaError_t set_int(int* dst, int v, cudaStream_t st) {
  set_int_kernel<<<1, 1, 0, st>>>(dst, v);
  return cudaGetLastError();
}

template cudaError_t khatri_rao<float>(const float*, int, const float*, int, int, float*,
                                       cudaStream_t);
template cudaError_t khatri_rao<double>(const double*, int, const double*, int, int, double*,
                                        cudaStream_t);
template cudaError_t cp_solve<float>(const float*, int, const float*, int, int, const float*, int,
                                     float*, int64_t, int*, cudaStream_t);
template cudaError_t cp_solve<double>(const double*, int, const double*, int, int, const double*,
                                      int, double*, int64_t, int*, cudaStream_t);
template cudaError_t sum_slabs_t<float>(const float*, int, int64_t, float*, cudaStream_t);
template cudaError_t sum_slabs_t<double>(const double*, int, int64_t, double*, cudaStream_t);

}  // namespace sma
