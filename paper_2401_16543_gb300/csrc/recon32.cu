// recon32.cu -- dispatch of the FP32 Riemann-state kernels over (d, R).
#include "internal.h"

namespace kfvm {

cudaError_t launch_recon32_22(kfvm_ctx*, const double*, const float*, float*, cudaStream_t, int, int);
cudaError_t launch_recon32_23(kfvm_ctx*, const double*, const float*, float*, cudaStream_t, int, int);
cudaError_t launch_recon32_32(kfvm_ctx*, const double*, const float*, float*, cudaStream_t, int, int);
cudaError_t launch_recon32_33(kfvm_ctx*, const double*, const float*, float*, cudaStream_t, int, int);

cudaError_t launch_labels_22(kfvm_ctx*, const double*, float*, float, cudaStream_t);
cudaError_t launch_labels_23(kfvm_ctx*, const double*, float*, float, cudaStream_t);
cudaError_t launch_labels_32(kfvm_ctx*, const double*, float*, float, cudaStream_t);
cudaError_t launch_labels_33(kfvm_ctx*, const double*, float*, float, cudaStream_t);

cudaError_t launch_labels(kfvm_ctx* ctx, const double* U, float* y, float thresh, cudaStream_t st) {
  if (ctx->dims == 2 && ctx->R == 2) return launch_labels_22(ctx, U, y, thresh, st);
  if (ctx->dims == 2 && ctx->R == 3) return launch_labels_23(ctx, U, y, thresh, st);
  if (ctx->dims == 3 && ctx->R == 2) return launch_labels_32(ctx, U, y, thresh, st);
  return launch_labels_33(ctx, U, y, thresh, st);
}

cudaError_t launch_recon32(kfvm_ctx* ctx, const double* U, const float* shadow, float* faces, cudaStream_t st,
                           int zf_first, int zf_count) {
  if (ctx->dims == 2 && ctx->R == 2) return launch_recon32_22(ctx, U, shadow, faces, st, 0, 0);
  if (ctx->dims == 2 && ctx->R == 3) return launch_recon32_23(ctx, U, shadow, faces, st, 0, 0);
  if (ctx->dims == 3 && ctx->R == 2) return launch_recon32_32(ctx, U, shadow, faces, st, zf_first, zf_count);
  return launch_recon32_33(ctx, U, shadow, faces, st, zf_first, zf_count);
}

}  // namespace kfvm
