// Matvec of the three-level structured approximation (Section 7.5) in the
// factors' structured form.
//
// The compressed operator is
//   A_hat = sum_{j1, j2, j3} G[j1, j2, j3] C1_j1 (x) C2_j2 (x) C3_j3,
//   Ct_j[a, b] = U_t[k, j] / sqrt(eta_k),  k = map_t(a, b)  (zero where
//   map_t(a, b) = -1),
// applied to volumes x[b3 + q3 (b2 + q2 b1)] (level 3 innermost).  Every
// Ct_j has the sparsity of its level's map (for the 3-D blur a band of 15
// diagonals out of 64), so the factors are applied through the map's
// nonzero positions (one compressed-row list per level) instead of as dense
// l x q matrices, with the core folded into the innermost factor:
//   B_{j1 j2} = sum_j3 G[j1, j2, j3] C3_j3   (the sparsity of map 3),
//   W_{j1}(b1)  = sum_j2 C2_j2 (x) B_{j1 j2}  applied to plane b1 of x,
//   y           = sum_j1 C1_j1 (x) I          applied along level 1 to W.
// ml_xy_kernel: one CTA per (plane b1, volume): the plane and the level-3
// and level-2 passes in shared memory, W_{j1} planes out.  ml_z_kernel: one
// thread per (a3, a2) position, the level-1 pass over the W planes.
// Both are bound by their shared-memory and L1 traffic; the algorithmic
// work is 2 nnz-per-row (k2 (q2 l3 + l2 l3) + l2 l3) k1 flops per plane.
#include "common.cuh"
#include "kernels.cuh"

namespace sma {
namespace {

constexpr int ML_THREADS = 256;

// coefficient e of level t's compressed-row list for factor column j
template <typename T>
__device__ __forceinline__ T level_coef(const MlApply<T>& P, int t, int j, int e) {
  const int k = P.kk[t][e];
  return (T)((double)P.U[t][k + (int64_t)P.p[t] * j] * P.isq[t][k]);
}

// c1[j1 nnz1 + e], c2[j2 nnz2 + e] and b[(j1 + r1 j2) nnz3 + e]
template <typename T>
__global__ void ml_coef_kernel(const MlApply<T> P) {
  const int n1 = P.r[0] * P.nnz[0], n2 = P.r[1] * P.nnz[1];
  const int n3 = P.r[0] * P.r[1] * P.nnz[2];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n1 + n2 + n3;
       i += gridDim.x * blockDim.x) {
    if (i < n1) {
      P.c1[i] = level_coef(P, 0, i / P.nnz[0], i % P.nnz[0]);
    } else if (i < n1 + n2) {
      const int t = i - n1;
      P.c2[t] = level_coef(P, 1, t / P.nnz[1], t % P.nnz[1]);
    } else {
      const int t = i - n1 - n2;
      const int e = t % P.nnz[2], jj = t / P.nnz[2];
      const int j1 = jj % P.r[0], j2 = jj / P.r[0];
      const int k = P.kk[2][e];
      double acc = 0.0;
      for (int j3 = 0; j3 < P.r[2]; ++j3)
        acc += (double)P.G[j1 + (int64_t)P.p[0] * (j2 + (int64_t)P.p[1] * j3)] *
               (double)P.U[2][k + (int64_t)P.p[2] * j3];
      P.b[t] = (T)(acc * P.isq[2][k]);
    }
  }
}

// One CTA per (plane b1, volume v).  Shared memory: the plane Xp[b3 + q3 b2],
// the level-3 pass Tp[a3 + l3 b2], the accumulator Acc[a3 + l3 a2], the
// coefficients of the current (j1, j2) and the two levels' row lists.  G
// outputs per thread share each row's coefficient and column loads (G = 4
// when q2 and l3 are multiples of 4, else 1).
template <typename T, int G>
__global__ void __launch_bounds__(ML_THREADS)
ml_xy_kernel(const MlApply<T> P, const T* __restrict__ X, int64_t ldx, T* __restrict__ W) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int l2 = P.l[1], l3 = P.l[2], q2 = P.q[1], q3 = P.q[2];
  const int nnz2 = P.nnz[1], nnz3 = P.nnz[2];
  T* Xp = reinterpret_cast<T*>(sm_raw);
  T* Tp = Xp + q2 * q3;
  T* Acc = Tp + q2 * l3;
  T* cb = Acc + l2 * l3;
  T* c2s = cb + nnz3;
  int* ptr3 = reinterpret_cast<int*>(c2s + nnz2);
  int* col3 = ptr3 + l3 + 1;
  int* ptr2 = col3 + nnz3;
  int* col2 = ptr2 + l2 + 1;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int b1 = blockIdx.x, v = blockIdx.y;
  const T* x = X + (int64_t)v * ldx + (int64_t)q3 * q2 * b1;
  for (int i = tid; i < q2 * q3; i += nth) Xp[i] = x[i];
  for (int i = tid; i <= l3; i += nth) ptr3[i] = P.ptr[2][i];
  for (int i = tid; i < nnz3; i += nth) col3[i] = P.col[2][i];
  for (int i = tid; i <= l2; i += nth) ptr2[i] = P.ptr[1][i];
  for (int i = tid; i < nnz2; i += nth) col2[i] = P.col[1][i];
  for (int j1 = 0; j1 < P.r[0]; ++j1) {
    for (int i = tid; i < l2 * l3; i += nth) Acc[i] = T(0);
    for (int j2 = 0; j2 < P.r[1]; ++j2) {
      __syncthreads();   // Tp and the coefficients of the previous (j1, j2) are consumed
      for (int i = tid; i < nnz3; i += nth) cb[i] = P.b[(int64_t)(j1 + P.r[0] * j2) * nnz3 + i];
      for (int i = tid; i < nnz2; i += nth) c2s[i] = P.c2[(int64_t)j2 * nnz2 + i];
      __syncthreads();
      // level 3: Tp[a3, b2] = sum over row a3 of map 3 of B_{j1 j2}[a3, b3] x[b3, b2];
      // a thread takes G values of b2 (q2 / G apart) on one row a3, so each
      // coefficient and column index is read once for G products
      {
        const int qg = q2 / G;
        for (int i = tid; i < l3 * qg; i += nth) {
          const int a3 = i % l3, bg = i / l3;
          T acc[G];
#pragma unroll
          for (int u = 0; u < G; ++u) acc[u] = T(0);
          for (int e = ptr3[a3]; e < ptr3[a3 + 1]; ++e) {
            const T cf = cb[e];
            const T* xc = Xp + col3[e] + q3 * bg;
#pragma unroll
            for (int u = 0; u < G; ++u) acc[u] = fma(cf, xc[q3 * qg * u], acc[u]);
          }
#pragma unroll
          for (int u = 0; u < G; ++u) Tp[a3 + l3 * (bg + qg * u)] = acc[u];
        }
      }
      __syncthreads();
      // level 2: Acc[a3, a2] += sum over row a2 of map 2 of C2_j2[a2, b2] Tp[a3, b2];
      // a thread takes G values of a3 (l3 / G apart) on one row a2
      {
        const int lg = l3 / G;
        for (int i = tid; i < lg * l2; i += nth) {
          const int ag = i % lg, a2 = i / lg;
          T* ac = Acc + ag + l3 * a2;
          T acc[G];
#pragma unroll
          for (int u = 0; u < G; ++u) acc[u] = ac[lg * u];
          for (int e = ptr2[a2]; e < ptr2[a2 + 1]; ++e) {
            const T cf = c2s[e];
            const T* tc = Tp + ag + l3 * col2[e];
#pragma unroll
            for (int u = 0; u < G; ++u) acc[u] = fma(cf, tc[lg * u], acc[u]);
          }
#pragma unroll
          for (int u = 0; u < G; ++u) ac[lg * u] = acc[u];
        }
      }
    }
    __syncthreads();   // Acc is read in another thread-to-element order
    T* w = W + (int64_t)l3 * l2 * (j1 + (int64_t)P.r[0] * (b1 + (int64_t)P.q[0] * v));
    for (int i = tid; i < l3 * l2; i += nth) w[i] = Acc[i];
  }
}

// y[pos + l3 l2 a1] = sum_j1 sum over row a1 of map 1 of C1_j1[a1, b1]
// W_j1[pos, b1], one thread per position pos = a3 + l3 a2 and volume.
template <typename T>
__global__ void __launch_bounds__(ML_THREADS)
ml_z_kernel(const MlApply<T> P, const T* __restrict__ W, T* __restrict__ Y, int64_t ldy) {
  const int l1 = P.l[0], plane = P.l[1] * P.l[2], q1 = P.q[0], r1 = P.r[0];
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (pos >= plane) return;
  const T* w = W + pos + (int64_t)plane * r1 * q1 * v;
  T* y = Y + (int64_t)v * ldy + pos;
  for (int a1 = 0; a1 < l1; ++a1) {
    T acc = T(0);
    const int e0 = P.ptr[0][a1], e1 = P.ptr[0][a1 + 1];
    for (int j1 = 0; j1 < r1; ++j1)
      for (int e = e0; e < e1; ++e)
        acc = fma(P.c1[(int64_t)j1 * P.nnz[0] + e],
                  __ldg(w + (int64_t)plane * (j1 + (int64_t)r1 * P.col[0][e])), acc);
    y[(int64_t)plane * a1] = acc;
  }
}

}  // namespace

template <typename T>
size_t ml_apply_smem(const MlApply<T>& P) {
  return sizeof(T) * ((size_t)P.q[1] * P.q[2] + (size_t)P.q[1] * P.l[2] + (size_t)P.l[1] * P.l[2] +
                      P.nnz[2] + P.nnz[1]) +
         sizeof(int) * ((size_t)P.l[2] + 1 + P.nnz[2] + P.l[1] + 1 + P.nnz[1]);
}

template <typename T>
cudaError_t ml_apply(const MlApply<T>& P, bool coef, const T* X, int64_t ldx, T* W, T* Y,
                     int64_t ldy, int nv, cudaStream_t st) {
  if (nv <= 0) return cudaSuccess;
  if (coef) {
    const int n = P.r[0] * P.nnz[0] + P.r[1] * P.nnz[1] + P.r[0] * P.r[1] * P.nnz[2];
    ml_coef_kernel<T><<<(n + 255) / 256, 256, 0, st>>>(P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t smem = ml_apply_smem(P);
  void (*kern)(const MlApply<T>, const T*, int64_t, T*) =
      (P.q[1] % 4 == 0 && P.l[2] % 4 == 0) ? ml_xy_kernel<T, 4> : ml_xy_kernel<T, 1>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3(P.q[0], nv), ML_THREADS, smem, st>>>(P, X, ldx, W);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int plane = P.l[1] * P.l[2];
  ml_z_kernel<T><<<dim3((plane + ML_THREADS - 1) / ML_THREADS, nv), ML_THREADS, 0, st>>>(P, W, Y,
                                                                                          ldy);
  return cudaGetLastError();
}

template size_t ml_apply_smem<float>(const MlApply<float>&);
template size_t ml_apply_smem<double>(const MlApply<double>&);
template cudaError_t ml_apply<float>(const MlApply<float>&, bool, const float*, int64_t, float*,
                                     float*, int64_t, int, cudaStream_t);
template cudaError_t ml_apply<double>(const MlApply<double>&, bool, const double*, int64_t,
                                      double*, double*, int64_t, int, cudaStream_t);

}  // namespace sma
