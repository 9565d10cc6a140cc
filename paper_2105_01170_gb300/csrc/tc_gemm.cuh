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
// fp16 two-piece form (x s = hi + lo, s a power of two that puts x s below
// 2^15, three products hi hi, hi lo, lo hi): planes as uint16_t fp16 bit
// patterns, two per operand.  C is multiplied by *scale (device).
cudaError_t tc_gemm_planes_f16(const uint16_t* A, const uint16_t* B, int M, int N, int64_t Kp,
                               float* C, int64_t ldc, const float* scale, int* err,
                               cudaStream_t st, bool col_major = false);
// The mid-index product in the fp16 form: Z is multiplied by *mult (device)
// and written as two fp16 planes.
cudaError_t tc_mid_planes_f16(const uint16_t* A, int M, const uint16_t* B, int N, int64_t Kq,
                              uint16_t* Z, int64_t Kp, int64_t zplane, int n, int ell,
                              const float* mult, int* err, cudaStream_t st);
// fp32 -> two fp16 planes of x * (*scale) (device scalar), layout as
// tc_split_transpose_batched.
cudaError_t tc_split2_transpose_batched(const float* src, int64_t s_rs, int64_t s_cs, int R, int K,
                                        int64_t Kp, int nbatch, int64_t src_bs, int64_t dst_bs,
                                        int64_t plane, const float* scale, uint16_t* dst,
                                        cudaStream_t st);
// *out = max |a[r + ld c]| (r < rows, c < cols) as the bit pattern of a float
cudaError_t tc_absmax(const float* a, int64_t rows, int64_t cols, int64_t ld, unsigned* out,
                      cudaStream_t st);
// *out = max |a[r rs + c cs]| (r < rows, c < cols) as the bit pattern of a float
cudaError_t tc_absmax_strided(const float* a, int64_t rows, int64_t cols, int64_t rs, int64_t cs,
                              unsigned* out, cudaStream_t st);
// *s = the power-of-two scale for the maximum *mx; out = {s_B, 1 / (s_A s_B)}
cudaError_t tc_f16_scale1(const unsigned* mx, float* s, cudaStream_t st);
cudaError_t tc_f16_scale_out(const unsigned* mxA, const unsigned* mxB, float* out,
                             cudaStream_t st);
// *out = max over (a, j) of sum_b |C[a + ell b + ell q j]|
cudaError_t tc_rowl1max(const float* C, int ell, int q, int nt, unsigned* out, cudaStream_t st);
// sc[0..5] = s_X, s_C, s_D, s_Z, s_Z / (s_X s_C), 1 / (s_Z s_D) from mx[0..3] =
// max |X|, max |C|, max row L1 of C, max |D| (powers of two, 2^(14 - e))
cudaError_t tc_f16_scales(const unsigned* mx, float* sc, cudaStream_t st);
bool tc_gemm_eligible(const GemmParams<float>& g);
cudaError_t tc_gemm_bf16x3(const GemmParams<float>& g, cudaStream_t st);
}  // namespace sma
