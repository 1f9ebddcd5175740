// recon64.cu -- dispatch of the FP64 Riemann-state kernels over (d, R).
#include "internal.h"

namespace kfvm {

cudaError_t launch_recon64_22(kfvm_ctx*, const double*, double*, cudaStream_t);
cudaError_t launch_recon64_23(kfvm_ctx*, const double*, double*, cudaStream_t);
cudaError_t launch_recon64_32(kfvm_ctx*, const double*, double*, cudaStream_t);
cudaError_t launch_recon64_33(kfvm_ctx*, const double*, double*, cudaStream_t);

cudaError_t launch_recon64(kfvm_ctx* ctx, const double* U, double* faces, cudaStream_t st) {
  if (ctx->dims == 2 && ctx->R == 2) return launch_recon64_22(ctx, U, faces, st);
  if (ctx->dims == 2 && ctx->R == 3) return launch_recon64_23(ctx, U, faces, st);
  if (ctx->dims == 3 && ctx->R == 2) return launch_recon64_32(ctx, U, faces, st);
  return launch_recon64_33(ctx, U, faces, st);
}

}  // namespace kfvm
