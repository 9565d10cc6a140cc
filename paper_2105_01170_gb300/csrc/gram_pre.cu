// Preconditioning of the mixed path's Gram eigen-solve.
//
// The Tucker variants (Sections 5.1, 6.2, 6.3, 7) need the eigenpairs of a
// Gram G = Y Y^T of an unfolding Y.  One-sided Jacobi on G itself sees the
// squared condition number of Y: in fp32 it needs many sweeps and leaves the
// small eigenvalues unresolved.  Here G (fp64) is factored by a Cholesky
// decomposition with diagonal pivoting,
//   P^T G P = R^T R,   pivot of step k = the largest remaining diagonal entry,
// which in exact arithmetic is the R factor of the column-pivoted QR of Y^T
// (the slice SVD's preconditioner), and returned as L = P R^T, a square
// factor G = L L^T in the original row order: L[c, k] = R[k, c'] for the
// original index c at pivoted position c'.  The one-sided Jacobi of L (the
// Jacobi of R^T with its rows permuted, so the same rotations) converges like
// that of a QR-preconditioned slice; L V = U Sigma gives G = U Sigma^2 U^T.
//
// pchol_kernel: a cluster of PCHOL_CTAS CTAs (the fp64 rate of one SM bounds
// a single CTA).  The trailing matrix is kept in pivoted order in a global
// fp64 workspace (lower triangle, n^2 doubles, L2-resident, read with
// ld.global.cg): a pivot swaps its row and column with those of position k
// (O(n) moves, spread over the cluster), so the rank-1 update of each step
// runs over contiguous columns, the columns dealt round-robin to the CTAs and
// one warp per column.  Every CTA keeps its own copy of the remaining
// diagonal, the position -> index map and the pivot's row of R in shared
// memory and updates them identically (so every CTA picks the same pivot
// without communicating); the hardware cluster barrier orders the steps'
// workspace accesses.  L is written by original index.  L is written in fp64 and, scaled
// by 1 / sqrt(max_j G_jj) (entries at most 1 in magnitude), in fp32.  A pivot
// at or below n eps max_j G_jj (the rounding level of the elimination) is
// raised to that floor, so R stays nonsingular; that changes G by about the
// floor, far below what the eigen-solve resolves.
#include <algorithm>
#include <cfloat>

#include "common.cuh"
#include "kernels.cuh"

namespace sma {
namespace {

constexpr int PCHOL_THREADS = 256;
constexpr int PCHOL_CTAS = 8;

__device__ __forceinline__ void pchol_cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}

__global__ void __launch_bounds__(PCHOL_THREADS)
    pchol_kernel(const double* __restrict__ G, int n, double* __restrict__ A,
                 double* __restrict__ L, float* __restrict__ L32, int* __restrict__ status) {
  __shared__ double d[kPcholMaxRows];    // remaining diagonal, by position
  __shared__ double rk[kPcholMaxRows];   // the current row of R, by position
  __shared__ int ord[kPcholMaxRows];     // position -> original index
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ double s_scale, s_floor;
  __shared__ int s_q;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nw = (nt + 31) >> 5;
  const int cta = blockIdx.x, ncta = gridDim.x;
  const int gt = cta * nt + tid, gn = ncta * nt;   // thread index over the cluster
  const int64_t nn = (int64_t)n * n;
  for (int64_t e = gt; e < nn; e += gn) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (i >= j) __stcg(A + e, G[e]);
    L[e] = 0.0;
    L32[e] = 0.f;
  }
  double mx = 0.0;
  bool bad = false;
  for (int j = tid; j < n; j += nt) {
    const double v = G[j + (int64_t)n * j];
    d[j] = v;
    ord[j] = j;
    bad |= !isfinite(v);
    mx = fmax(mx, v);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  bad = __syncthreads_or(bad);
  if (lane == 0) red_v[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int w = 0; w < nw; ++w) m = fmax(m, red_v[w]);
    s_scale = m > 0.0 ? 1.0 / sqrt(m) : 1.0;
    s_floor = fmax((double)n * DBL_EPSILON * m, DBL_MIN);
    if (bad && cta == 0) atomicOr(status, SMA_STATUS_BIT(SMA_ERR_NONFINITE));
  }
  __syncthreads();
  const double scale = s_scale, flo = s_floor;
  pchol_cluster_barrier();   // the workspace is filled
  for (int k = 0; k < n; ++k) {
    // pivot: the largest remaining diagonal entry, the lowest position on ties
    double bv = -DBL_MAX;
    int bq = n;
    for (int q = k + tid; q < n; q += nt) {
      const double v = d[q];
      if (v > bv || (v == bv && q < bq)) {
        bv = v;
        bq = q;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oq = __shfl_xor_sync(0xffffffffu, bq, o);
      if (ov > bv || (ov == bv && oq < bq)) {
        bv = ov;
        bq = oq;
      }
    }
    if (lane == 0) {
      red_v[warp] = bv;
      red_i[warp] = bq;
    }
    __syncthreads();
    if (warp == 0) {
      double v = lane < nw ? red_v[lane] : -DBL_MAX;
      int q = lane < nw ? red_i[lane] : n;
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oq = __shfl_xor_sync(0xffffffffu, q, o);
        if (ov > v || (ov == v && oq < q)) {
          v = ov;
          q = oq;
        }
      }
      if (lane == 0) s_q = (q < k || q >= n) ? k : q;   // no comparable entry (NaN): keep the order
    }
    __syncthreads();
    const int q = s_q;   // the same in every CTA (identical copies of d)
    if (q != k) {
      // swap positions k and q in the trailing lower triangle: (i, k) with
      // (q, i) for k < i < q, (i, k) with (i, q) for i > q; the entry (q, k)
      // stays and the diagonals move with d
      for (int i = k + 1 + gt; i < n; i += gn) {
        if (i == q) continue;
        double* a = A + i + (int64_t)n * k;
        double* b = i < q ? A + q + (int64_t)n * i : A + i + (int64_t)n * q;
        const double t = __ldcg(a);
        __stcg(a, __ldcg(b));
        __stcg(b, t);
      }
      if (tid == 0) {
        const double t = d[k];
        d[k] = d[q];
        d[q] = t;
        const int o = ord[k];
        ord[k] = ord[q];
        ord[q] = o;
      }
      pchol_cluster_barrier();   // (also a block barrier)
    }
    const double rkk = sqrt(fmax(d[k], flo));
    // row k of R (column k of A below the diagonal) in every CTA; column k
    // of L, by original index, written by the CTA that owns the entry
    for (int i = k + 1 + tid; i < n; i += nt) {
      const double r = __ldcg(A + i + (int64_t)n * k) / rkk;
      rk[i] = r;
      if (i % ncta == cta) {
        const int c = ord[i];
        L[c + (int64_t)n * k] = r;
        L32[c + (int64_t)n * k] = (float)(r * scale);
      }
    }
    if (tid == 0 && cta == 0) {
      L[ord[k] + (int64_t)n * k] = rkk;
      L32[ord[k] + (int64_t)n * k] = (float)(rkk * scale);
    }
    __syncthreads();
    // rank-1 update of the trailing lower triangle: column j to CTA
    // (j - k - 1) mod ncta, one warp per column, two 32-row chunks in flight
    for (int j = k + 1 + cta + ncta * warp; j < n; j += ncta * nw) {
      const double rj = rk[j];
      double* col = A + (int64_t)n * j;
      int i = j + lane;
      for (; i + 32 < n; i += 64) {
        const double a0 = __ldcg(col + i), a1 = __ldcg(col + i + 32);
        __stcg(col + i, fma(-rk[i], rj, a0));
        __stcg(col + i + 32, fma(-rk[i + 32], rj, a1));
      }
      if (i < n) __stcg(col + i, fma(-rk[i], rj, __ldcg(col + i)));
    }
    for (int i = k + 1 + tid; i < n; i += nt) d[i] = fma(-rk[i], rk[i], d[i]);
    pchol_cluster_barrier();   // the update is complete everywhere (also a block barrier)
  }
}

// From the fp64 Jacobi of L V: U[:, j] = Wf[:, j] / sigma_j (e_j where sigma_j
// is 0 or not finite, only for an all-zero G) and the eigenvalue sigma_j^2.
__global__ void pchol_finish_kernel(const double* __restrict__ Wf, double* __restrict__ sig,
                                    int n, double* __restrict__ U) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e % n), j = (int)(e / n);
    const double s = sig[j];
    U[e] = (s > 0.0 && isfinite(s)) ? Wf[e] / s : (q == j ? 1.0 : 0.0);
  }
}

__global__ void square_kernel(double* __restrict__ v, int n) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    v[j] = v[j] * v[j];
}

}  // namespace

cudaError_t gram_pchol(const double* G, int n, double* work, double* L, float* L32, int* status,
                       cudaStream_t st) {
  if (n < 1 || n > kPcholMaxRows) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(PCHOL_CTAS);
  cfg.blockDim = dim3(PCHOL_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = PCHOL_CTAS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, pchol_kernel, G, n, work, L, L32, status);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t gram_pchol_finish(const double* Wf, double* sig, int n, double* U, cudaStream_t st) {
  if (n < 1) return cudaErrorInvalidValue;
  const int64_t nn = (int64_t)n * n;
  const int blocks = (int)std::min<int64_t>((nn + 255) / 256, 1024);
  pchol_finish_kernel<<<blocks, 256, 0, st>>>(Wf, sig, n, U);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  square_kernel<<<(n + 255) / 256, 256, 0, st>>>(sig, n);
  return cudaGetLastError();
}

}  // namespace sma
