// tcgen05 (5th-generation tensor core) GEMM for the fp32 contractions of the
// mixed path, computed as 3-piece bf16 split products with fp32 accumulation
// in tensor memory.
#pragma once
#include "common.cuh"

namespace sma {
// True when the device can run the tcgen05 kernel (compute capability 10.3).
bool tc_gemm_available(int major, int minor);
// True when the strided problem maps onto the kernel's operand layouts.
bool tc_gemm_eligible(const GemmParams<float>& g);
cudaError_t tc_gemm_bf16x3(const GemmParams<float>& g, cudaStream_t st);
}  // namespace sma
