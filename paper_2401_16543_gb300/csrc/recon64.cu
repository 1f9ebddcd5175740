// recon64.cu -- dispatch of the FP64 Riemann-state kernels over (d, R).
#include "internal.h"

namespace kfvm {

cudaError_t launch_recon64_22(kfvm_ctx*, const double*, double*, cudaStream_t, int, int);
cudaError_t launch_recon64_23(kfvm_ctx*, const double*, double*, cudaStream_t, int, int);
cudaError_t launch_recon64_32(kfvm_ctx*, const double*, double*, cudaStream_t, int, int);
cudaError_t launch_recon64_33(kfvm_ctx*, const double*, double*, cudaStream_t, int, int);

cudaError_t launch_recon64(kfvm_ctx* ctx, const double* U, double* faces, cudaStream_t st, int zf_first,
                           int zf_count) {
  if (zf_count <= 0) {
    zf_first = 0;
    zf_count = ctx->n[2];
  }
  if (ctx->dims == 2 && ctx->R == 2) return launch_recon64_22(ctx, U, faces, st, 0, 1);
  if (ctx->dims == 2 && ctx->R == 3) return launch_recon64_23(ctx, U, faces, st, 0, 1);
  if (ctx->dims == 3 && ctx->R == 2) return launch_recon64_32(ctx, U, faces, st, zf_first, zf_count);
  return launch_recon64_33(ctx, U, faces, st, zf_first, zf_count);
}

}  // namespace kfvm
