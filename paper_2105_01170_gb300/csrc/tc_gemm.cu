#include "tc_gemm.cuh"

namespace sma {
bool tc_gemm_available(int major, int minor) { return false && major == 10 && minor == 3; }
bool tc_gemm_eligible(const GemmParams<float>&) { return false; }
cudaError_t tc_gemm_bf16x3(const GemmParams<float>& g, cudaStream_t st) { return gemm<float>(g, st); }
}  // namespace sma
