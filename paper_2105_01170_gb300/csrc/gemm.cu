// Generic strided batched GEMM on CUDA cores (fp32 / fp64).
//
// Used for the small and irregular contractions of the path (per-slice
// projections with run-time ranks, the Kronecker-sum middle contraction) and
// as the fp64 form of every contraction.  The large fp32 contractions of the
// mixed path go to the tcgen05 kernel in tc_gemm.cu instead.
#include <cuda_bf16.h>

#include "common.cuh"

namespace sma {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

// three-plane bf16 split of an fp32 result (hi = bf16(v), mid = bf16(v - hi),
// lo = bf16(v - hi - mid)); base_off is the batch offset applied to C
__device__ __forceinline__ void store_split(const GemmParams<float>& p, int64_t base_off,
                                            int64_t off, float v) {
  __nv_bfloat16* d = static_cast<__nv_bfloat16*>(p.Cs) + base_off + off;
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(hi);
  const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
  d[0] = hi;
  d[p.cs_plane] = mid;
  d[2 * p.cs_plane] = __float2bfloat16_rn(r1 - __bfloat162float(mid));
}
__device__ __forceinline__ void store_split(const GemmParams<double>&, int64_t, int64_t, double) {}

template <typename T>
__global__ void __launch_bounds__(NT) gemm_kernel(const GemmParams<T> p) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int b1 = blockIdx.y, b2 = blockIdx.z;
  const int di = p.dstride * b1;
  const int M = p.dM ? min(p.M, p.dM[di]) : p.M;
  const int N = p.dN ? min(p.N, p.dN[di]) : p.N;
  int K = p.dK ? min(p.K, p.dK[di]) : p.K;
  const int tiles_m = (p.M + BM - 1) / BM;
  const int m0 = (blockIdx.x % tiles_m) * BM;
  const int n0 = (blockIdx.x / tiles_m) * BN;
  if (m0 >= M || n0 >= N) return;
  const T* A = p.A + b1 * p.a_b1 + b2 * p.a_b2;
  const T* B = p.B + b1 * p.b_b1 + b2 * p.b_b2;
  const int64_t cbo = (p.c_off ? (int64_t)p.c_off[b1] * p.c_off_mul : b1 * p.c_b1) + b2 * p.c_b2;
  T* C = p.C + cbo;

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  const bool a_col = (p.a_rs == 1);
  const bool b_col = (p.b_rs == 1);
  // 16-row (column) groups of the tile that hold output (block-uniform): a
  // tile of a small product skips the multiply-adds of its empty groups,
  // which matters in fp64 (2 FMA per clock per SM): a 15 x 15 Gram does 1/16
  // of the padded tile's work
  const int gm = min(4, (M - m0 + 15) / 16), gn = min(4, (N - n0 + 15) / 16);
  int kbeg = p.dKoff ? p.dKoff[di] : 0;
  if (p.kchunk > 0) {
    kbeg = b1 * p.kchunk;
    K = min(K, kbeg + p.kchunk);
  }
  // an empty K range with beta = 1 leaves C as it is (the truncated rebuild
  // of a slice that discards nothing): nothing to read or write
  if (kbeg >= K && p.beta == T(1) && !p.Cs) return;
  for (int k0 = kbeg; k0 < K; k0 += BK) {
#pragma unroll
    for (int t = 0; t < (BM * BK) / NT; ++t) {
      const int e = tid + t * NT;
      int i, k;
      if (a_col) { i = e % BM; k = e / BM; } else { k = e % BK; i = e / BK; }
      const int gi = m0 + i, gk = k0 + k;
      As[k][i] = (gi < M && gk < K) ? A[(int64_t)gi * p.a_rs + (int64_t)gk * p.a_cs] : T(0);
    }
#pragma unroll
    for (int t = 0; t < (BN * BK) / NT; ++t) {
      const int e = tid + t * NT;
      int j, k;
      if (b_col) { k = e % BK; j = e / BK; } else { j = e % BN; k = e / BN; }
      const int gj = n0 + j, gk = k0 + k;
      Bs[k][j] = (gj < N && gk < K) ? B[(int64_t)gk * p.b_rs + (int64_t)gj * p.b_cs] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T a[4], b[4];
      // rows follow tx so that consecutive threads write consecutive rows of
      // the (column-major) output
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][ty + 16 * j];
      if (gm == 4 && gn == 4) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (i < gm && j < gn) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = m0 + tx + 16 * i;
    if (gi >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = n0 + ty + 16 * j;
      if (gj >= N) continue;
      const int64_t off = (int64_t)gi * p.c_rs + (int64_t)gj * p.c_cs;
      T v = p.alpha * acc[i][j];
      if (p.Cs) {
        store_split(p, cbo, off, v);
        continue;
      }
      T* c = C + off;
      if (p.beta != T(0)) v += p.beta * *c;
      *c = v;
    }
  }
}

}  // namespace

template <typename T>
cudaError_t gemm(const GemmParams<T>& p, cudaStream_t st) {
  if (p.M <= 0 || p.N <= 0 || p.nb1 <= 0 || p.nb2 <= 0) return cudaSuccess;
  if (p.nb1 > 65535 || p.nb2 > 65535) return cudaErrorInvalidValue;
  const int64_t tiles = (int64_t)((p.M + BM - 1) / BM) * ((p.N + BN - 1) / BN);
  if (tiles > 0x7fffffff) return cudaErrorInvalidValue;
  dim3 grid((unsigned)tiles, p.nb1, p.nb2);
  gemm_kernel<T><<<grid, NT, 0, st>>>(p);
  return cudaGetLastError();
}

template cudaError_t gemm<float>(const GemmParams<float>&, cudaStream_t);
template cudaError_t gemm<double>(const GemmParams<double>&, cudaStream_t);

}  // namespace sma
