// gate.cu -- learned smooth-cell gate (placeholder until built).
#include <cuda_runtime.h>

#include "common.cuh"

namespace kfvm {

cudaError_t launch_gate_mask(kfvm_ctx*, const double*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_gate_features(kfvm_ctx*, const double*, float*, float*, double, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_gate_forward(kfvm_ctx*, const float*, float*, size_t, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_gate_train(kfvm_ctx*, const float*, const float*, size_t, float, float*, float*, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace kfvm

extern "C" {
size_t kfvm_gate_param_count(const kfvm_ctx* ctx) { return ctx ? ctx->gate.count() : 0; }
kfvm_status kfvm_gate_set_params(kfvm_ctx*, const float*, size_t) { return KFVM_ERR_STATE; }
kfvm_status kfvm_gate_get_params(kfvm_ctx*, float*, size_t) { return KFVM_ERR_STATE; }
kfvm_status kfvm_gate_features(kfvm_ctx*, const double*, float*, float*, double, void*) { return KFVM_ERR_STATE; }
kfvm_status kfvm_gate_forward(kfvm_ctx*, const float*, float*, size_t, void*) { return KFVM_ERR_STATE; }
kfvm_status kfvm_gate_train_step(kfvm_ctx*, const float*, const float*, size_t, float, float*, float*, void*) {
  return KFVM_ERR_STATE;
}
}
