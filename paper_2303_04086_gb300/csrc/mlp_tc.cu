// Tensor-core MLP variants of the shade step (BF16 / FP8 e4m3 operands, FP32
// accumulation in tensor memory).
#include <cuda_runtime.h>

#include "inolf_internal.h"
#include "kernels_common.cuh"

namespace inolf {

inolf_status prepare_tc_weights(Object& obj, const float* w1, const float* w2, const float* w3, void* stream) {
  (void)obj; (void)w1; (void)w2; (void)w3; (void)stream;
  return INOLF_OK;
}

inolf_status launch_shade_tc(const Params& p, inolf_precision prec, cudaStream_t st) {
  (void)p; (void)prec; (void)st;
  return fail(INOLF_E_UNSUPPORTED, "tensor-core MLP not built yet");
}

}  // namespace inolf
