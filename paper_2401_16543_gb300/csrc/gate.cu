// gate.cu -- the learned smooth-cell gate: features, BF16 tensor-core MLP
// inference and training (forward, backward, Adam), and the per-cell mask the
// gated reconstruction reads.
//
// The gate plays the role of the paper's troubled-cell indicator (Sec. 3.5,
// Sec. 5.3 step 2): cells it marks smooth take the unlimited linear
// reconstruction, the others WENO-AO.  It has no counterpart in the paper; its
// training labels come from the method's own WENO-AO weights (label_kernel in
// recon32.cuh).
//
// Network: NIN -> 32 -> 32 -> 1 (ReLU, ReLU, sigmoid).  Input: the radius-2
// full stencil of rho and of the cell-average pressure, each as deviations from
// the central cell divided by max(max |deviation|, 1e-4 |central value|), so a
// feature vector describes the shape of the data and not its amplitude (as the
// WENO weights do) and is exactly zero on constant data in any precision.  Matrix products run on the tensor cores with
// mma.sync.m16n8k16 (BF16 operands, FP32 accumulation) on 32-row warp tiles;
// the weight gradients are FP32 sums of products of the BF16-rounded operands;
// parameters are FP32 masters updated by Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <utility>
#include <vector>

#include "gate.cuh"

namespace kfvm {
namespace gate {

__constant__ ShellTable c_shell = make_shell();

template <int D, int L>
struct Off2 {
  static constexpr int x = Geo<D, 2>::tab.off[L][0], y = Geo<D, 2>::tab.off[L][1], z = Geo<D, 2>::tab.off[L][2];
};

// Gate features of cell (x, y, z) from the state (float64, or its float32
// shadow on the mixed-precision path), written to f[NIN]; in 3D the two shell
// inputs are computed when `shell` (radius-3 reconstruction), else zero.
template <int D, typename TU, int... Ls>
__device__ __forceinline__ void features(const GridArgs& a, const TU* __restrict__ U, long long ncell, int x,
                                         int y, int z, float* f, bool shell, std::integer_sequence<int, Ls...>) {
  constexpr int N0 = Dims<D>::N0;
  const float gm1 = a.gammaf - 1.0f;
  auto load = [&](int ox, int oy, int oz, float& rho, float& p) {
    const int gx = map_index(x + ox, a.n[0], a.bc[0][0], a.bc[0][1]);
    const int gy = map_index(y + oy, a.n[1], a.bc[1][0], a.bc[1][1]);
    const int gz = (D == 3) ? map_index(z + oz, a.n[2], a.bc[2][0], a.bc[2][1]) : 0;
    const long long gc = ((long long)gz * a.n[1] + gy) * a.n[0] + gx;
    const float r = (float)U[gc];
    float m2 = 0.0f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float m = (float)U[(1 + k) * ncell + gc];
      m2 = fmaf(m, m, m2);
    }
    rho = r;
    p = gm1 * fmaf(-0.5f * m2, __frcp_rn(r), (float)U[(D + 1) * ncell + gc]);
  };
  ((load(Off2<D, Ls>::x, Off2<D, Ls>::y, Off2<D, Ls>::z, f[Ls], f[N0 + Ls])), ...);
  constexpr int C = Geo<D, 2>::center();
  const float rc = f[C], pc = f[N0 + C];
  const float dr = normalise_block<N0, C>(f);
  const float dp = normalise_block<N0, C>(f + N0);
  if (D == 3) {
    float mr = 0.0f, mp = 0.0f;
    if (shell) {
#pragma unroll 6
      for (int l = 0; l < 90; ++l) {
        float r, p;
        load(c_shell.off[l][0], c_shell.off[l][1], c_shell.off[l][2], r, p);
        mr = fmaxf(mr, fabsf(r - rc));
        mp = fmaxf(mp, fabsf(p - pc));
      }
    }
    f[2 * N0] = shell_feature(mr, dr);
    f[2 * N0 + 1] = shell_feature(mp, dp);
  }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(256) features_kernel(GridArgs a, const double* __restrict__ U,
                                                       float* __restrict__ X, bool shell) {
  constexpr int NIN = Dims<D>::NIN;
  const long long ncell = (long long)a.n[0] * a.n[1] * a.n[2];
  const long long c = blockIdx.x * 256LL + threadIdx.x;
  if (c >= ncell) return;
  const int x = (int)(c % a.n[0]), y = (int)((c / a.n[0]) % a.n[1]), z = (int)(c / ((long long)a.n[0] * a.n[1]));
  float f[NIN];
  features<D>(a, U, ncell, x, y, z, f, shell, std::make_integer_sequence<int, Dims<D>::N0>{});
#pragma unroll
  for (int i = 0; i < NIN; ++i) X[c * NIN + i] = f[i];
}

// rows of X (float32 [n][NIN]) -> bf16 smem tile of one warp
template <int D>
__device__ __forceinline__ void stage_rows(const float* __restrict__ X, long long row0, long long n,
                                           __nv_bfloat16* xs) {
  constexpr int NIN = Dims<D>::NIN, KIN = Dims<D>::KIN, LDX = Dims<D>::LDX;
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < 32 * KIN; i += 32) {
    const int r = i / KIN, k = i % KIN;
    const long long row = row0 + r;
    const float v = (row < n && k < NIN) ? X[row * NIN + k] : 0.0f;
    xs[r * LDX + k] = __float2bfloat16_rn(v);
  }
  __syncwarp();
}

template <int D>
__global__ void __launch_bounds__(32 * kWarps) forward_kernel(const Pack<D>* __restrict__ pack,
                                                              const float* __restrict__ X, float* __restrict__ prob,
                                                              long long n) {
  __shared__ Pack<D> P;
  __shared__ __align__(16) __nv_bfloat16 xs_all[kWarps][32 * Dims<D>::LDX];
  load_pack<D>(pack, &P);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  __nv_bfloat16* xs = xs_all[warp];
  for (long long row0 = (blockIdx.x * (long long)kWarps + warp) * 32; row0 < n;
       row0 += (long long)gridDim.x * kWarps * 32) {
    stage_rows<D>(X, row0, n, xs);
    float h1[2][4][4], h2[2][4][4], z[2][4];
    forward32<D>(P, xs, h1, h2, z);
    if (t == 0) {
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const long long r0 = row0 + 16 * mt + g, r1 = r0 + 8;
        if (r0 < n) prob[r0] = 1.0f / (1.0f + __expf(-z[mt][0]));
        if (r1 < n) prob[r1] = 1.0f / (1.0f + __expf(-z[mt][2]));
      }
    }
    __syncwarp();
  }
}

// Per-cell smooth mask of the gated reconstruction: features of 32 consecutive
// cells per warp, the MLP on the tensor cores, logit > logit(threshold).
template <int D, typename TU>
__global__ void __launch_bounds__(32 * kWarps) mask_kernel(GridArgs a, const Pack<D>* __restrict__ pack,
                                                           const TU* __restrict__ U,
                                                           unsigned char* __restrict__ mask, float zthresh,
                                                           bool shell) {
  constexpr int NIN = Dims<D>::NIN, KIN = Dims<D>::KIN, LDX = Dims<D>::LDX;
  __shared__ Pack<D> P;
  __shared__ __align__(16) __nv_bfloat16 xs_all[kWarps][32 * LDX];
  load_pack<D>(pack, &P);
  __syncthreads();
  const long long ncell = (long long)a.n[0] * a.n[1] * a.n[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  __nv_bfloat16* xs = xs_all[warp];
  for (long long row0 = (blockIdx.x * (long long)kWarps + warp) * 32; row0 < ncell;
       row0 += (long long)gridDim.x * kWarps * 32) {
    const long long c = row0 + lane;
    float f[NIN];
    if (c < ncell) {
      const int x = (int)(c % a.n[0]), y = (int)((c / a.n[0]) % a.n[1]);
      const int z = (int)(c / ((long long)a.n[0] * a.n[1]));
      features<D>(a, U, ncell, x, y, z, f, shell, std::make_integer_sequence<int, Dims<D>::N0>{});
    } else {
#pragma unroll
      for (int i = 0; i < NIN; ++i) f[i] = 0.0f;
    }
#pragma unroll
    for (int k = 0; k < KIN; ++k) xs[lane * LDX + k] = __float2bfloat16_rn(k < NIN ? f[k] : 0.0f);
    __syncwarp();
    float h1[2][4][4], h2[2][4][4], z[2][4];
    forward32<D>(P, xs, h1, h2, z);
    if (t == 0) {
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const long long r0 = row0 + 16 * mt + g, r1 = r0 + 8;
        if (r0 < ncell) mask[r0] = z[mt][0] > zthresh ? 1 : 0;
        if (r1 < ncell) mask[r1] = z[mt][2] > zthresh ? 1 : 0;
      }
    }
    __syncwarp();
  }
}

// One training pass over a batch: forward, backward of the mean binary
// cross-entropy, weight gradients accumulated into grad (+ loss sum at grad[COUNT]).
template <int D>
__global__ void __launch_bounds__(32 * kTrainWarps) train_kernel(const Pack<D>* __restrict__ pack,
                                                            const float* __restrict__ X, const float* __restrict__ y,
                                                            long long n, float* __restrict__ grad) {
  using DM = Dims<D>;
  constexpr int NIN = DM::NIN, LDX = DM::LDX, LDH = H + 2;
  __shared__ Pack<D> P;
  __shared__ __align__(16) __nv_bfloat16 xs_all[kTrainWarps][32 * LDX];
  // per-warp operands of the weight gradients, bf16 as the tensor-core products see them
  __shared__ __align__(16) __nv_bfloat16 sh1[kTrainWarps][32 * LDH], sh2[kTrainWarps][32 * LDH],
      sd1[kTrainWarps][32 * LDH], sd2[kTrainWarps][32 * LDH];
  __shared__ float sdz[kTrainWarps][32];
  load_pack<D>(pack, &P);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  __nv_bfloat16* xs = xs_all[warp];
  __nv_bfloat16* H1 = sh1[warp];
  __nv_bfloat16* H2 = sh2[warp];
  __nv_bfloat16* D1 = sd1[warp];
  __nv_bfloat16* D2 = sd2[warp];
  float* DZ = sdz[warp];
  const float invn = 1.0f / (float)n;
  // per-lane gradient partials: lane owns row `lane` of W1, W2 and element `lane` of b1, b2, W3
  float gW1[NIN], gW2[H], gb1 = 0.f, gb2 = 0.f, gW3 = 0.f, gb3 = 0.f, loss = 0.f;
#pragma unroll
  for (int i = 0; i < NIN; ++i) gW1[i] = 0.f;
#pragma unroll
  for (int i = 0; i < H; ++i) gW2[i] = 0.f;

  for (long long row0 = (blockIdx.x * (long long)kTrainWarps + warp) * 32; row0 < n;
       row0 += (long long)gridDim.x * kTrainWarps * 32) {
    stage_rows<D>(X, row0, n, xs);
    float h1[2][4][4], h2[2][4][4], z[2][4];
    forward32<D>(P, xs, h1, h2, z);
    // output layer: p = sigmoid(z), dz = (p - y)/n, BCE loss (rows beyond n contribute nothing)
    float dzr[2][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const long long row = row0 + 16 * mt + g + 8 * hh;
        float dz = 0.0f;
        if (t == 0 && row < n) {
          const float zz = z[mt][2 * hh];
          const float yy = y[row];
          const float p = 1.0f / (1.0f + __expf(-zz));
          dz = (p - yy) * invn;
          loss += fmaxf(zz, 0.0f) - zz * yy + log1pf(__expf(-fabsf(zz)));
        }
        dzr[mt][hh] = __shfl_sync(0xffffffffu, dz, lane & ~3);  // broadcast across the quad
      }
    // dH2 = dz w3^T masked by ReLU; dH1 = (dH2 W2) masked by ReLU
    float d2[2][4][4], d1[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int col = 8 * nt + 2 * t + (j & 1);
          const float w3 = __bfloat162float(P.W3[col]);
          d2[mt][nt][j] = h2[mt][nt][j] > 0.0f ? dzr[mt][j >> 1] * w3 : 0.0f;
          d1[mt][nt][j] = 0.0f;
        }
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        uint32_t af[4];
        af[0] = pack_bf16(d2[mt][2 * kk][0], d2[mt][2 * kk][1]);
        af[1] = pack_bf16(d2[mt][2 * kk][2], d2[mt][2 * kk][3]);
        af[2] = pack_bf16(d2[mt][2 * kk + 1][0], d2[mt][2 * kk + 1][1]);
        af[3] = pack_bf16(d2[mt][2 * kk + 1][2], d2[mt][2 * kk + 1][3]);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const __nv_bfloat16* w = P.W2T + (8 * nt + g) * H + 16 * kk + 2 * t;
          mma16816(d1[mt][nt], af, ld_pair(w), ld_pair(w + 8));
        }
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (!(h1[mt][nt][j] > 0.0f)) d1[mt][nt][j] = 0.0f;
          const int row = 16 * mt + g + 8 * (j >> 1), col = 8 * nt + 2 * t + (j & 1);
          H1[row * LDH + col] = __float2bfloat16_rn(h1[mt][nt][j]);
          H2[row * LDH + col] = __float2bfloat16_rn(h2[mt][nt][j]);
          D1[row * LDH + col] = __float2bfloat16_rn(d1[mt][nt][j]);
          D2[row * LDH + col] = __float2bfloat16_rn(d2[mt][nt][j]);
        }
      if (t == 0) {
        DZ[16 * mt + g] = dzr[mt][0];
        DZ[16 * mt + g + 8] = dzr[mt][1];
      }
    }
    __syncwarp();
    // weight gradients in FP32: sums over the 32 rows
#pragma unroll 4
    for (int r = 0; r < 32; ++r) {
      const float dh2 = __bfloat162float(D2[r * LDH + lane]), dh1 = __bfloat162float(D1[r * LDH + lane]);
      const float dz = DZ[r];
      gb2 += dh2;
      gb1 += dh1;
      gW3 = fmaf(dz, __bfloat162float(H2[r * LDH + lane]), gW3);
      if (lane == 0) gb3 += dz;
#pragma unroll
      for (int i = 0; i < H; ++i) gW2[i] = fmaf(dh2, __bfloat162float(H1[r * LDH + i]), gW2[i]);
#pragma unroll
      for (int i = 0; i < NIN; ++i) gW1[i] = fmaf(dh1, __bfloat162float(xs[r * LDX + i]), gW1[i]);
    }
    __syncwarp();
  }
#pragma unroll
  for (int i = 0; i < NIN; ++i) atomicAdd(grad + DM::oW1 + lane * NIN + i, gW1[i]);
#pragma unroll
  for (int i = 0; i < H; ++i) atomicAdd(grad + DM::oW2 + lane * H + i, gW2[i]);
  atomicAdd(grad + DM::ob1 + lane, gb1);
  atomicAdd(grad + DM::ob2 + lane, gb2);
  atomicAdd(grad + DM::oW3 + lane, gW3);
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, o);
  if (lane == 0) {
    atomicAdd(grad + DM::ob3, gb3);
    atomicAdd(grad + DM::COUNT, loss);
  }
}

// Write the BF16 working copy (and the float32 biases) from the float32 masters.
template <int D>
__device__ __forceinline__ void pack_one(const float* __restrict__ prm, Pack<D>* __restrict__ P, int i) {
  using DM = Dims<D>;
  const float v = prm[i];
  if (i < DM::ob1) {
    const int h = i / DM::NIN, k = i % DM::NIN;
    P->W1[h * DM::KIN + k] = __float2bfloat16_rn(v);
  } else if (i < DM::oW2) {
    P->b1[i - DM::ob1] = v;
  } else if (i < DM::ob2) {
    const int o = (i - DM::oW2) / H, j = (i - DM::oW2) % H;
    P->W2[o * H + j] = __float2bfloat16_rn(v);
    P->W2T[j * H + o] = __float2bfloat16_rn(v);
  } else if (i < DM::oW3) {
    P->b2[i - DM::ob2] = v;
  } else if (i < DM::ob3) {
    P->W3[i - DM::oW3] = __float2bfloat16_rn(v);
  } else {
    P->b3 = v;
  }
}

template <int D>
__global__ void pack_kernel(const float* __restrict__ prm, Pack<D>* __restrict__ P) {
  using DM = Dims<D>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < DM::COUNT) pack_one<D>(prm, P, i);
}

template <int D>
__global__ void zero_pack_kernel(Pack<D>* __restrict__ P) {
  uint32_t* w = reinterpret_cast<uint32_t*>(P);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (int)(sizeof(Pack<D>) / 4); i += gridDim.x * blockDim.x)
    w[i] = 0u;
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the float32 masters, then repack.
template <int D>
__global__ void adam_kernel(float* __restrict__ prm, float* __restrict__ mv, float* __restrict__ grad,
                            Pack<D>* __restrict__ P, float lr, float bc1, float bc2, long long n,
                            float* __restrict__ grads_out, float* __restrict__ loss_out) {
  using DM = Dims<D>;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && loss_out) *loss_out = grad[DM::COUNT] / (float)n;
  if (i >= DM::COUNT) return;
  const float gr = grad[i];
  if (grads_out) grads_out[i] = gr;
  float m = mv[i], v = mv[DM::COUNT + i];
  m = 0.9f * m + 0.1f * gr;
  v = 0.999f * v + 0.001f * gr * gr;
  mv[i] = m;
  mv[DM::COUNT + i] = v;
  prm[i] -= lr * (m / bc1) / (sqrtf(v / bc2) + 1e-8f);
  grad[i] = 0.0f;
  pack_one<D>(prm, P, i);
}

__global__ void clear_loss_kernel(float* __restrict__ grad, int count) {
  if (blockIdx.x == 0 && threadIdx.x == 0) grad[count] = 0.0f;
}

inline int grid_for(long long rows, int warps_per_cta) {
  long long warps = (rows + 31) / 32;
  long long blocks = (warps + warps_per_cta - 1) / warps_per_cta;
  return (int)(blocks < 152LL * 16 ? (blocks > 0 ? blocks : 1) : 152LL * 16);
}

}  // namespace gate

using namespace gate;

template <int D>
static cudaError_t gate_mask_d(kfvm_ctx* ctx, const double* U, const float* shadow, cudaStream_t st) {
  const GridArgs a = make_grid_args(ctx);
  const float th = (float)ctx->gate_threshold;
  const float zth = logf(th / (1.0f - th));
  const Pack<D>* P = (const Pack<D>*)ctx->d_gate_pack;
  const bool shell = D == 3 && ctx->R >= 3;
  if (shadow)
    mask_kernel<D, float><<<grid_for(ctx->ncell, kWarps), 32 * kWarps, 0, st>>>(a, P, shadow, ctx->d_gate_mask, zth,
                                                                                 shell);
  else
    mask_kernel<D, double><<<grid_for(ctx->ncell, kWarps), 32 * kWarps, 0, st>>>(a, P, U, ctx->d_gate_mask, zth,
                                                                                  shell);
  ctx->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_gate_mask(kfvm_ctx* ctx, const double* U, const float* shadow, cudaStream_t st) {
  if (!ctx->gate_loaded) return cudaErrorNotReady;
  return ctx->dims == 2 ? gate_mask_d<2>(ctx, U, shadow, st) : gate_mask_d<3>(ctx, U, shadow, st);
}

template <int D>
static cudaError_t gate_features_d(kfvm_ctx* ctx, const double* U, float* X, float* y, double tau, cudaStream_t st) {
  const GridArgs a = make_grid_args(ctx);
  features_kernel<D><<<(unsigned)((ctx->ncell + 255) / 256), 256, 0, st>>>(a, U, X, D == 3 && ctx->R >= 3);
  ctx->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_labels(ctx, U, y, (float)(1.0 - tau), st);
}

cudaError_t launch_gate_features(kfvm_ctx* ctx, const double* U, float* X, float* y, double tau, cudaStream_t st) {
  return ctx->dims == 2 ? gate_features_d<2>(ctx, U, X, y, tau, st) : gate_features_d<3>(ctx, U, X, y, tau, st);
}

template <int D>
static cudaError_t gate_forward_d(kfvm_ctx* ctx, const float* X, float* prob, size_t n, cudaStream_t st) {
  forward_kernel<D><<<grid_for((long long)n, kWarps), 32 * kWarps, 0, st>>>((const Pack<D>*)ctx->d_gate_pack, X, prob,
                                                                        (long long)n);
  ctx->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_gate_forward(kfvm_ctx* ctx, const float* X, float* prob, size_t n, cudaStream_t st) {
  return ctx->dims == 2 ? gate_forward_d<2>(ctx, X, prob, n, st) : gate_forward_d<3>(ctx, X, prob, n, st);
}

template <int D>
static cudaError_t gate_train_d(kfvm_ctx* ctx, const float* X, const float* y, size_t n, float lr, float* loss,
                                float* grads_out, cudaStream_t st) {
  using DM = Dims<D>;
  clear_loss_kernel<<<1, 32, 0, st>>>(ctx->d_gate_grad, DM::COUNT);
  train_kernel<D><<<grid_for((long long)n, kTrainWarps), 32 * kTrainWarps, 0, st>>>((const Pack<D>*)ctx->d_gate_pack, X, y,
                                                                      (long long)n, ctx->d_gate_grad);
  ctx->gate_step += 1;
  const float bc1 = 1.0f - powf(0.9f, (float)ctx->gate_step), bc2 = 1.0f - powf(0.999f, (float)ctx->gate_step);
  adam_kernel<D><<<(DM::COUNT + 255) / 256, 256, 0, st>>>(ctx->d_gate, ctx->d_gate_adam, ctx->d_gate_grad,
                                                          (Pack<D>*)ctx->d_gate_pack, lr, bc1, bc2, (long long)n,
                                                          grads_out, loss);
  ctx->launches += 3;
  return cudaGetLastError();
}

cudaError_t launch_gate_train(kfvm_ctx* ctx, const float* X, const float* y, size_t n, float lr, float* loss,
                              float* grads_out, cudaStream_t st) {
  return ctx->dims == 2 ? gate_train_d<2>(ctx, X, y, n, lr, loss, grads_out, st)
                        : gate_train_d<3>(ctx, X, y, n, lr, loss, grads_out, st);
}

template <int D>
static cudaError_t gate_upload_d(kfvm_ctx* ctx, const float* host) {
  using DM = Dims<D>;
  cudaError_t e = cudaSuccess;
  if (!ctx->d_gate) e = cudaMalloc(&ctx->d_gate, sizeof(float) * DM::COUNT);
  if (e == cudaSuccess && !ctx->d_gate_adam) e = cudaMalloc(&ctx->d_gate_adam, sizeof(float) * 2 * DM::COUNT);
  if (e == cudaSuccess && !ctx->d_gate_grad) e = cudaMalloc(&ctx->d_gate_grad, sizeof(float) * (DM::COUNT + 1));
  if (e == cudaSuccess && !ctx->d_gate_pack) e = cudaMalloc(&ctx->d_gate_pack, sizeof(Pack<D>));
  if (e == cudaSuccess) e = cudaMemcpy(ctx->d_gate, host, sizeof(float) * DM::COUNT, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_gate_adam, 0, sizeof(float) * 2 * DM::COUNT);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_gate_grad, 0, sizeof(float) * (DM::COUNT + 1));
  if (e != cudaSuccess) return e;
  zero_pack_kernel<D><<<8, 256>>>((Pack<D>*)ctx->d_gate_pack);
  pack_kernel<D><<<(DM::COUNT + 255) / 256, 256>>>(ctx->d_gate, (Pack<D>*)ctx->d_gate_pack);
  ctx->launches += 2;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  ctx->gate_step = 0;
  return e;
}

}  // namespace kfvm

using namespace kfvm;

extern "C" {

size_t kfvm_gate_param_count(const kfvm_ctx* ctx) {
  if (!ctx) return 0;
  return ctx->dims == 2 ? (size_t)Dims<2>::COUNT : (size_t)Dims<3>::COUNT;
}

kfvm_status kfvm_gate_set_params(kfvm_ctx* ctx, const float* host, size_t count) {
  if (!ctx || !host || count != kfvm_gate_param_count(ctx)) return KFVM_ERR_ARG;
  const cudaError_t e = ctx->dims == 2 ? gate_upload_d<2>(ctx, host) : gate_upload_d<3>(ctx, host);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? KFVM_ERR_NOMEM : KFVM_ERR_CUDA;
  ctx->gate_loaded = true;
  return KFVM_OK;
}

kfvm_status kfvm_gate_get_params(kfvm_ctx* ctx, float* host, size_t count) {
  if (!ctx || !host || count != kfvm_gate_param_count(ctx)) return KFVM_ERR_ARG;
  if (!ctx->gate_loaded) return KFVM_ERR_STATE;
  if (cudaDeviceSynchronize() != cudaSuccess) return KFVM_ERR_CUDA;
  if (cudaMemcpy(host, ctx->d_gate, sizeof(float) * count, cudaMemcpyDeviceToHost) != cudaSuccess)
    return KFVM_ERR_CUDA;
  return KFVM_OK;
}

kfvm_status kfvm_gate_features(kfvm_ctx* ctx, const double* U, float* X, float* y, double tau, void* stream) {
  if (!ctx || !U || !X || !y || !(tau >= 0 && tau < 1)) return KFVM_ERR_ARG;
  if (!ctx->weights_built) return KFVM_ERR_STATE;
  return launch_gate_features(ctx, U, X, y, tau, (cudaStream_t)stream) == cudaSuccess ? KFVM_OK : KFVM_ERR_CUDA;
}

kfvm_status kfvm_gate_mask(kfvm_ctx* ctx, const double* U, unsigned char* mask_out, void* stream) {
  if (!ctx || !U || !mask_out) return KFVM_ERR_ARG;
  if (!ctx->gate_loaded) return KFVM_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (ctx->precision == 32) {
    e = launch_shadow(ctx, U, ctx->d_shadow, st);
    if (e == cudaSuccess) e = launch_gate_mask(ctx, U, ctx->d_shadow, st);
  } else {
    e = launch_gate_mask(ctx, U, nullptr, st);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(mask_out, ctx->d_gate_mask, (size_t)ctx->ncell, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? KFVM_OK : KFVM_ERR_CUDA;
}

kfvm_status kfvm_set_smooth_mask(kfvm_ctx* ctx, const unsigned char* mask, void* stream) {
  if (!ctx || !mask) return KFVM_ERR_ARG;
  if (cudaMemcpyAsync(ctx->d_gate_mask, mask, (size_t)ctx->ncell, cudaMemcpyDeviceToDevice, (cudaStream_t)stream) !=
      cudaSuccess)
    return KFVM_ERR_CUDA;
  ctx->recon = 3;
  return KFVM_OK;
}

kfvm_status kfvm_gate_forward(kfvm_ctx* ctx, const float* X, float* prob, size_t n, void* stream) {
  if (!ctx || !X || !prob) return KFVM_ERR_ARG;
  if (!ctx->gate_loaded) return KFVM_ERR_STATE;
  return launch_gate_forward(ctx, X, prob, n, (cudaStream_t)stream) == cudaSuccess ? KFVM_OK : KFVM_ERR_CUDA;
}

kfvm_status kfvm_gate_train_step(kfvm_ctx* ctx, const float* X, const float* y, size_t n, float lr, float* loss_dev,
                                 float* grads_out, void* stream) {
  if (!ctx || !X || !y || n == 0 || !(lr >= 0)) return KFVM_ERR_ARG;
  if (!ctx->gate_loaded) return KFVM_ERR_STATE;
  return launch_gate_train(ctx, X, y, n, lr, loss_dev, grads_out, (cudaStream_t)stream) == cudaSuccess
             ? KFVM_OK
             : KFVM_ERR_CUDA;
}

kfvm_status kfvm_gate_load(kfvm_ctx* ctx, const void* host_weights, size_t bytes) {
  if (!ctx || !host_weights) return KFVM_ERR_ARG;
  const size_t count = kfvm_gate_param_count(ctx);
  if (bytes == 4 * count) return kfvm_gate_set_params(ctx, static_cast<const float*>(host_weights), count);
  if (bytes != 2 * count) return KFVM_ERR_ARG;
  // bfloat16 parameters: widen to the float32 masters (exact)
  std::vector<float> w(count);
  const uint16_t* b = static_cast<const uint16_t*>(host_weights);
  for (size_t i = 0; i < count; ++i) {
    const uint32_t bits = (uint32_t)b[i] << 16;
    std::memcpy(&w[i], &bits, 4);
  }
  return kfvm_gate_set_params(ctx, w.data(), count);
}

kfvm_status kfvm_gate_train(kfvm_ctx* ctx, const float* X, const float* y, size_t n, int epochs, float lr,
                            void* stream) {
  if (!ctx || !X || !y || n == 0 || epochs < 1 || !(lr >= 0)) return KFVM_ERR_ARG;
  if (!ctx->gate_loaded) return KFVM_ERR_STATE;
  const size_t nin = ctx->dims == 2 ? (size_t)Dims<2>::NIN : (size_t)Dims<3>::NIN;
  constexpr size_t kBatch = 2048;
  cudaStream_t st = (cudaStream_t)stream;
  for (int e = 0; e < epochs; ++e)
    for (size_t r0 = 0; r0 < n; r0 += kBatch) {
      const size_t nb = n - r0 < kBatch ? n - r0 : kBatch;
      if (launch_gate_train(ctx, X + r0 * nin, y + r0, nb, lr, nullptr, nullptr, st) != cudaSuccess)
        return KFVM_ERR_CUDA;
    }
  return KFVM_OK;
}

}  // extern "C"
