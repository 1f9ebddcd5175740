// recon64_23.cu -- FP64 Riemann states for d = 2, R = 3 (one instantiation per
// translation unit so that the library compiles in parallel).
#include "recon64.cuh"

namespace kfvm {
cudaError_t launch_recon64_23(kfvm_ctx* ctx, const double* U, double* faces, cudaStream_t st, int zf_first,
                              int zf_count) {
  return r64::launch_dr<2, 3>(ctx, U, faces, st, zf_first, zf_count);
}
}  // namespace kfvm
