// internal.h -- context and launch interfaces shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <vector>

#include "../../include/kfvm.h"
#include "geometry.h"

namespace kfvm {

// Device-side status bits (OR-ed into ctx->d_status).
enum : int { kFlagNonphysical = 1, kFlagTimeout = 2 };

// Scalars the kernels exchange through device memory.
struct DevScalars {
  unsigned long long rate_bits;  // max over cells of sum_d (|u_d| + c)/dx_d, as ordered bits
  unsigned int blocks_done;      // arrival counter of the reduction's last-block pattern
  unsigned int pad;
  double dt;                     // current step size
  double cfl, t_rem;             // inputs of the dt rule
};

// Kernel families timed by the "profile" option.
enum ProfKernel : int { kProfMaxRate = 0, kProfRecon64, kProfRecon32, kProfFaceFlux, kProfUpdate, kProfGateMask,
                        kProfShadow, kProfKxrcf, kProfCount };

struct ProfPair {
  cudaEvent_t start, stop;
  int kernel;
};

struct GateNet {
  int in = 0;
  static constexpr int H = 32;
  size_t count() const { return (size_t)H * in + H + H * H + H + H + 1; }
};

}  // namespace kfvm

struct kfvm_ctx {
  // geometry and physics
  int dims = 2, R = 2, nv = 4, nq = 6, n0 = 13, F = 8, M = 5, NT = 2;
  int n[3] = {1, 1, 1};
  double dx[3] = {1, 1, 1};
  int bc[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  double gamma = 1.4, ell = 5.0;
  long long ncell = 0;
  int sizes[kfvm::kMaxNQ] = {0};
  int degrees[kfvm::kMaxNQ] = {0};
  // options
  int precision = 64, recon = 0, riemann = 0, positivity = 1;
  int tensor_cores = 1;  // d = 3, R = 3 FP32 contraction on tcgen05 (0: the CUDA-core kernel)
  int timeout_probe = 0;  // test hook: the next tensor-core launch waits on nothing and times out
  double kappa = 0.1, eta = 0.0, eps = 1e-40, gate_threshold = 0.5;
  double kxrcf_m = 1.5;  // power m of the KXRCF threshold Delta^m (recon mode 4)
  int vars = 0;          // WENO-AO variables: 0 linearized primitive, 1 characteristic (FP64 path)
  // weights
  size_t wcount = 0;
  bool weights_built = false;
  std::vector<double> w_host;  // float64 tables (kernel-parameter copies are made from these)
  double* d_w64 = nullptr;
  float* d_w32 = nullptr;
  void* d_w33tc = nullptr;       // d = 3, R = 3: FP16 hi/lo weight image of the tensor-core kernel
  // scratch owned by the library
  void* d_faces = nullptr;       // F * nv * ncell values (float64 or float32)
  double* d_flux = nullptr;      // face-averaged fluxes, per direction nv * (n_d + 1) * prod(n_other)
  size_t flux_off[3] = {0, 0, 0};
  double* d_stage = nullptr;     // one intermediate RK state, nv * ncell
  double* d_stage2 = nullptr;    // second intermediate state (only when the step runs in z-slabs)
  float* d_shadow2 = nullptr;    // second float32 shadow (slabs)
  size_t face_bytes = 0;         // bytes of the Riemann-state buffer d_faces
  int slab_user = 0;             // z-planes per slab set by the "slab_planes" option (0: automatic)
  double* d_L = nullptr;         // optional dUdt scratch for kfvm_rhs-style calls
  float* d_shadow = nullptr;     // float32 copy of the state for the FP32 path, nv * ncell
  unsigned char* d_gate_mask = nullptr;  // per cell: 1 = smooth (linear), 0 = WENO
  kfvm::DevScalars* d_scalars = nullptr;
  int* d_status = nullptr;
  // gate
  kfvm::GateNet gate;
  float* d_gate = nullptr;        // float32 master parameters
  float* d_gate_adam = nullptr;   // Adam moments m, v (2 * count)
  float* d_gate_grad = nullptr;   // gradient accumulator (+1 float: the batch loss sum)
  void* d_gate_pack = nullptr;    // BF16 working copy of the weights + float32 biases
  long long gate_step = 0;
  bool gate_loaded = false;
  // accounting and tracing
  long long launches = 0;
  int profile = 0;
  std::vector<kfvm::ProfPair> prof_pairs;   // recorded, not yet folded into the totals
  std::vector<cudaEvent_t> prof_free;       // event pool
  long long prof_launches[kfvm::kProfCount] = {0};
  double prof_ms[kfvm::kProfCount] = {0};
};

namespace kfvm {

// Launch helpers implemented per translation unit.  Every launcher returns a
// cudaError_t from cudaGetLastError() after its launches and adds the number
// of kernels it launched to ctx->launches.
cudaError_t launch_build_weights(kfvm_ctx* ctx, cudaStream_t st, int* d_err);
cudaError_t launch_max_rate(kfvm_ctx* ctx, const double* U, double cfl, double t_rem, cudaStream_t st);
// zf_first / zf_count select the z-planes whose Riemann states go to `faces` (3D slabs);
// zf_count = 0 means the whole grid.
cudaError_t launch_recon64(kfvm_ctx* ctx, const double* U, double* faces, cudaStream_t st, int zf_first = 0,
                           int zf_count = 0);
// d = 3, R = 3 FP32 weights: padded row table (floats) and its fill from the float64 tables
size_t recon33_table_floats();
void recon33_fill_table(const double* w, float* out);
size_t recon33_tc_image_bytes();
void recon33_tc_fill_image(const double* w, unsigned char* out);
cudaError_t launch_recon32(kfvm_ctx* ctx, const double* U, const float* shadow, float* faces, cudaStream_t st,
                           int zf_first = 0, int zf_count = 0);
cudaError_t launch_face_flux(kfvm_ctx* ctx, const void* faces, cudaStream_t st);
// stage: 0 -> dUdt only (to out), 1/2/3 -> SSP-RK3 stages writing the new state to out.
cudaError_t launch_update(kfvm_ctx* ctx, int stage, const double* U0, const double* Us, double* out, cudaStream_t st);
cudaError_t launch_shadow(kfvm_ctx* ctx, const double* U, float* shadow, cudaStream_t st);
// Fused face fluxes + divergence + stage update (stage 0: write dUdt to out).
// zc_lo..zc_hi: planes of cells to update (zc_hi = 0: all); the faces hold planes zf_first.. (slabs).
cudaError_t launch_flux_update(kfvm_ctx* ctx, int stage, const void* faces, const double* U0, const double* Us,
                               double* out, cudaStream_t st, float* shadow_out = nullptr, int zc_lo = 0,
                               int zc_hi = 0, int zf_first = 0, int zf_count = 0);
// shadow != nullptr: features from the float32 shadow (mixed path), else from U
cudaError_t launch_gate_mask(kfvm_ctx* ctx, const double* U, const float* shadow, cudaStream_t st);
// KXRCF troubled-cell mask of U (shadow != nullptr: from the float32 shadow, the FP32 path).
cudaError_t launch_kxrcf(kfvm_ctx* ctx, const double* U, const float* shadow, unsigned char* mask, cudaStream_t st);
// The reconstruction kernels' mode: the KXRCF mode (4) runs them on the indicator's mask (3).
inline int kernel_recon_mode(const kfvm_ctx* c) { return c->recon == 4 ? 3 : c->recon; }
// WENO-AO training labels of the gate (float32 shadow input).
cudaError_t launch_labels(kfvm_ctx* ctx, const double* U, float* y, float thresh, cudaStream_t st);
cudaError_t launch_gate_features(kfvm_ctx* ctx, const double* U, float* X, float* y, double tau, cudaStream_t st);
cudaError_t launch_gate_forward(kfvm_ctx* ctx, const float* X, float* prob, size_t n, cudaStream_t st);
cudaError_t launch_gate_train(kfvm_ctx* ctx, const float* X, const float* y, size_t n, float lr, float* loss,
                              float* grads_out, cudaStream_t st);
cudaError_t fma_peak(int bits, double* flops);

// Tracing helpers (no-ops unless ctx->profile): bracket one launcher call.
cudaEvent_t prof_begin(kfvm_ctx* ctx, cudaStream_t st);
void prof_end(kfvm_ctx* ctx, int kernel, cudaEvent_t start, cudaStream_t st);

}  // namespace kfvm
