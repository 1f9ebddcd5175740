// recon32.cu -- FP32 Riemann states of the mixed-precision path (placeholder until built).
#include <cuda_runtime.h>

#include "common.cuh"

namespace kfvm {

cudaError_t launch_recon32(kfvm_ctx*, const double*, const float*, float*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace kfvm
