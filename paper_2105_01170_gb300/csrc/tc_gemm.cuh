// tcgen05 (5th-generation tensor core) GEMM for the large fp32 contractions
// of the mixed path, computed as 3-piece bf16 split products with fp32
// accumulation in tensor memory.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace sma {
// True when the device can run the tcgen05 kernel (compute capability 10.3)
// and the driver exposes cuTensorMapEncodeTiled.
bool tc_gemm_available(int major, int minor);
// K padded to the kernel's K tile (64).
int64_t tc_pad_k(int64_t K);
// fp32 (element (j, k) at src[j*s_rs + k*s_cs], j < R, k < K) -> three bf16
// planes dst[p*R*Kp + j*Kp + k] (hi, mid, lo); columns K..Kp-1 untouched.
cudaError_t tc_split_transpose(const float* src, int64_t s_rs, int64_t s_cs, int R, int K,
                               int64_t Kp, __nv_bfloat16* dst, cudaStream_t st);
// C(i, j) = sum_k A(i,k) B(j,k) over the six split products, A given as
// three planes [M][Kp], B as three planes [N][Kp] (Kp % 64 == 0,
// padding columns zero); C(i, j) at C[i*ldc + j], or C[i + j*ldc] when
// col_major.  Timeouts set SMA_ERR_TIMEOUT in *err.
cudaError_t tc_gemm_planes(const __nv_bfloat16* A, const __nv_bfloat16* B, int M, int N,
                           int64_t Kp, float* C, int64_t ldc, int* err, cudaStream_t st,
                           bool col_major = false);
// Batched form: nbatch copies, source offset src_bs and destination offset
// dst_bs per batch, plane stride `plane` (elements) for all of them.
cudaError_t tc_split_transpose_batched(const float* src, int64_t s_rs, int64_t s_cs, int R, int K,
                                       int64_t Kp, int nbatch, int64_t src_bs, int64_t dst_bs,
                                       int64_t plane, __nv_bfloat16* dst, cudaStream_t st);
// Short-K product written as split planes in the long-K operand layout:
// Z(i, j) = sum_k A(i,k) B(j,k) (A planes [M][Kq], B planes [N][Kq], Kq % 64
// == 0), with i = c + n s and j = a + ell t stored at
// Z[p*zplane + (a + ell s)*Kp + c + n t] for the hi, mid, lo parts p.
cudaError_t tc_mid_planes(const __nv_bfloat16* A, int M, const __nv_bfloat16* B, int N, int64_t Kq,
                          __nv_bfloat16* Z, int64_t Kp, int64_t zplane, int n, int ell, int* err,
                          cudaStream_t st);
bool tc_gemm_eligible(const GemmParams<float>& g);
cudaError_t tc_gemm_bf16x3(const GemmParams<float>& g, cudaStream_t st);
}  // namespace sma
