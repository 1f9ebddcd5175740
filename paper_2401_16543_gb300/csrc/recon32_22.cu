// recon32_22.cu -- FP32 Riemann states for d = 2, R = 2 (one instantiation per
// translation unit so that the library compiles in parallel).
#include "recon32.cuh"

namespace kfvm {
cudaError_t launch_recon32_22(kfvm_ctx* ctx, const double* U, const float* shadow, float* faces,
                                cudaStream_t st, int zf_first, int zf_count) {
  return r32::launch<2, 2>(ctx, U, shadow, faces, st, zf_first, zf_count);
}
cudaError_t launch_labels_22(kfvm_ctx* ctx, const double* U, float* y, float thresh, cudaStream_t st) {
  return r32::launch_labels<2, 2>(ctx, U, y, thresh, st);
}
}  // namespace kfvm
