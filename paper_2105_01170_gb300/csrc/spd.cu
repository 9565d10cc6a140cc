// Section 5.2, preserving positive definiteness: the diagonal block T_0 of
// T = I (x) T_0 + sum_k E_k (x) T_k is factored T_0 = L L^T, the remaining
// blocks are compressed as A_k = L^-1 T_k L^-T, and the approximation is
// T_hat = (I (x) L)(I + M_E[T])(I (x) L^T).  This file holds the small
// kernels that wrap the shared-U Tucker path with that congruence: the
// factorization and inverse of the diagonal block, and two elementwise
// helpers of the reconstruction and the matvec.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.cuh"

namespace sma {
namespace {

constexpr int CHOL_THREADS = 1024;

// T_0 = L L^T (right-looking, column by column) followed by L^-1 (row-wise
// forward substitution applied to the identity), one CTA, in the element
// type T.  L and Linv are m x m column-major (ld m) in global memory, which
// stays in L2 for the sizes this is used at; the current column of L (or row
// of L^-1) is staged in shared memory.  A pivot that is not positive and
// finite stops the factorization: L and Linv are then set to zero (so the
// compression that follows runs on finite data) and the status word gets
// SMA_ERR_NOT_SPD.
template <typename T>
__global__ void __launch_bounds__(CHOL_THREADS)
    chol_inv_kernel(const T* __restrict__ T0, int64_t ld0, int m, T* __restrict__ L,
                    T* __restrict__ Linv, int* __restrict__ status) {
  extern __shared__ unsigned char sm_raw[];
  T* vec = reinterpret_cast<T*>(sm_raw);  // m entries
  __shared__ T s_piv;
  __shared__ int s_bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  const int64_t mm = (int64_t)m * m;
  if (tid == 0) s_bad = 0;
  for (int64_t e = tid; e < mm; e += nt) {
    const int i = (int)(e % m), j = (int)(e / m);
    L[e] = i >= j ? T0[i + j * ld0] : T(0);
    Linv[e] = i == j ? T(1) : T(0);
  }
  __syncthreads();
  // ---- Cholesky: column j is scaled by 1/sqrt(pivot); the trailing lower
  // triangle loses the outer product of the scaled column with itself.
  for (int j = 0; j < m; ++j) {
    if (tid == 0) {
      const T d = L[j + (int64_t)j * m];
      const bool ok = d > T(0) && isfinite(d);
      s_piv = ok ? sqrt(d) : T(0);
      if (!ok) s_bad = 1;
    }
    __syncthreads();
    if (s_bad) break;  // uniform: every thread reads the same flag
    const T piv = s_piv;
    const T inv = T(1) / piv;
    for (int i = j + tid; i < m; i += nt) {
      const T v = i == j ? piv : L[i + (int64_t)j * m] * inv;
      vec[i] = v;
      L[i + (int64_t)j * m] = v;
    }
    __syncthreads();
    // columns k > j to warps, rows i >= k to lanes (coalesced down a column)
    for (int k = j + 1 + warp; k < m; k += nwarps) {
      const T lk = vec[k];
      T* colk = L + (int64_t)k * m;
      for (int i = k + lane; i < m; i += 32) colk[i] -= vec[i] * lk;
    }
    __syncthreads();
  }
  if (s_bad) {
    for (int64_t e = tid; e < mm; e += nt) {
      L[e] = T(0);
      Linv[e] = T(0);
    }
    if (tid == 0) atomicOr(status, SMA_STATUS_BIT(SMA_ERR_NOT_SPD));
    return;
  }
  // ---- L^-1: X = I, then for i = 0..m-1 row i of X is divided by L(i,i)
  // and rows r > i lose L(r,i) times it (only columns c <= i are nonzero).
  for (int i = 0; i < m; ++i) {
    const T inv = T(1) / L[i + (int64_t)i * m];
    for (int c = tid; c <= i; c += nt) {
      const T v = Linv[i + (int64_t)c * m] * inv;
      vec[c] = v;
      Linv[i + (int64_t)c * m] = v;
    }
    __syncthreads();
    const T* coli = L + (int64_t)i * m;
    for (int c = warp; c <= i; c += nwarps) {
      const T xc = vec[c];
      T* colc = Linv + (int64_t)c * m;
      for (int r = i + 1 + lane; r < m; r += 32) colc[r] -= coli[r] * xc;
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void add_identity_kernel(T* A, int64_t ld, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    A[i + i * ld] += T(1);
}

// Y[:, s] += X[:, s] for s < cols, rows entries per column.
template <typename T>
__global__ void add_into_kernel(const T* __restrict__ X, int64_t ldx, T* __restrict__ Y,
                                int64_t ldy, int64_t rows, int cols) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % rows, s = e / rows;
    Y[r + s * ldy] += X[r + s * ldx];
  }
}

int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  const int64_t cap = 152 * 16;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

size_t chol_inv_smem(int m, size_t elem) { return (size_t)m * elem; }

template <typename T>
cudaError_t chol_inv(const T* T0, int64_t ld0, int m, T* L, T* Linv, int* status,
                     cudaStream_t st) {
  const size_t smem = chol_inv_smem(m, sizeof(T));
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(chol_inv_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  chol_inv_kernel<T><<<1, CHOL_THREADS, smem, st>>>(T0, ld0, m, L, Linv, status);
  return cudaGetLastError();
}

template <typename T>
cudaError_t add_identity(T* A, int64_t ld, int64_t n, cudaStream_t st) {
  add_identity_kernel<T><<<grid_for(n, 256), 256, 0, st>>>(A, ld, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t add_into(const T* X, int64_t ldx, T* Y, int64_t ldy, int64_t rows, int cols,
                     cudaStream_t st) {
  add_into_kernel<T><<<grid_for(rows * cols, 256), 256, 0, st>>>(X, ldx, Y, ldy, rows, cols);
  return cudaGetLastError();
}

template cudaError_t chol_inv<float>(const float*, int64_t, int, float*, float*, int*, cudaStream_t);
template cudaError_t chol_inv<double>(const double*, int64_t, int, double*, double*, int*,
                                      cudaStream_t);
template cudaError_t add_identity<float>(float*, int64_t, int64_t, cudaStream_t);
template cudaError_t add_identity<double>(double*, int64_t, int64_t, cudaStream_t);
template cudaError_t add_into<float>(const float*, int64_t, float*, int64_t, int64_t, int,
                                     cudaStream_t);
template cudaError_t add_into<double>(const double*, int64_t, double*, int64_t, int64_t, int,
                                      cudaStream_t);

}  // namespace sma
