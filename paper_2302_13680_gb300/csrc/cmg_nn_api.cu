// C ABI of the warm-start network kernels (include/cmg.h, "learned warm
// start" section).
#include <cstdint>

#include "cmg_internal.h"

using namespace cmg;

namespace {
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
}  // namespace

extern "C" cmg_status cmg_nn_gemm_bf16(const void* A, const void* B, int M, int N, int K, const float* bias,
                                       int relu, float* C32, void* C16, int ldc, int* status, void* stream) {
  if (!A || !B || !status || (!C32 && !C16)) return CMG_ERR_INVALID_ARG;
  if (M < 1 || N < 1 || K < 64 || K % 64 != 0 || ldc < N) return CMG_ERR_INVALID_ARG;
  if (!aligned16(A) || !aligned16(B)) return CMG_ERR_INVALID_ARG;
  const cudaError_t e = launch_gemm_bf16_tn(A, B, M, N, K, bias, relu, C32, C16, ldc, status,
                                            static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return CMG_ERR_CUDA;
  }
  return CMG_OK;
}
