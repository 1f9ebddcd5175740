// gate.cuh -- device pieces of the learned gate shared by gate.cu and the fused
// gated reconstruction in recon32.cuh: parameter packing, mma.sync helpers and the
// 32-row forward pass on the tensor cores.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace kfvm {
namespace gate {

constexpr int H = 32;
constexpr int kWarps = 4;       // warps per CTA in the inference kernels
constexpr int kTrainWarps = 2;  // warps per CTA in the training kernel (shared-memory bound)

template <int D>
struct Dims {
  static constexpr int N0 = Geo<D, 2>::N0;       // radius-2 stencil
  static constexpr int NSH = (D == 3) ? 2 : 0;   // 3D: radius-3 shell inputs of rho and p
  static constexpr int NIN = 2 * N0 + NSH;       // rho and p blocks (+ shell)
  static constexpr int KIN = (NIN + 15) / 16 * 16;
  static constexpr int LDX = KIN + 8;            // padded smem row (bank-conflict free fragment loads)
  // float32 master parameter offsets
  static constexpr int oW1 = 0, ob1 = H * NIN, oW2 = ob1 + H, ob2 = oW2 + H * H, oW3 = ob2 + H, ob3 = oW3 + H;
  static constexpr int COUNT = ob3 + 1;
};

template <int D>
struct __align__(16) Pack {
  __nv_bfloat16 W1[H * Dims<D>::KIN];  // [h][k], zero for k >= NIN
  __nv_bfloat16 W2[H * H];             // [o][i]
  __nv_bfloat16 W2T[H * H];            // [i][o]
  __nv_bfloat16 W3[8 * H];             // row 0 = W3, rows 1..7 zero
  float b1[H], b2[H], b3, pad[3];
};

// ---------------------------------------------------------------------------
// mma.sync m16n8k16 BF16 x BF16 -> FP32 on warp fragments
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// Forward pass of 32 rows held in shared memory (xs[row * LDX + k], bf16).
// h1, h2: post-ReLU C fragments [m-tile][n-tile][4]; z: layer-3 C fragments.
template <int D>
__device__ __forceinline__ void forward32(const Pack<D>& P, const __nv_bfloat16* xs, float (&h1)[2][4][4],
                                          float (&h2)[2][4][4], float (&z)[2][4]) {
  constexpr int KIN = Dims<D>::KIN, LDX = Dims<D>::LDX;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    // layer 1
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      h1[mt][nt][0] = h1[mt][nt][2] = P.b1[8 * nt + 2 * t];
      h1[mt][nt][1] = h1[mt][nt][3] = P.b1[8 * nt + 2 * t + 1];
    }
#pragma unroll
    for (int kk = 0; kk < KIN / 16; ++kk) {
      uint32_t af[4];
      const __nv_bfloat16* r0 = xs + (16 * mt + g) * LDX + 16 * kk + 2 * t;
      af[0] = ld_pair(r0);
      af[1] = ld_pair(r0 + 8 * LDX);
      af[2] = ld_pair(r0 + 8);
      af[3] = ld_pair(r0 + 8 * LDX + 8);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const __nv_bfloat16* w = P.W1 + (8 * nt + g) * KIN + 16 * kk + 2 * t;
        mma16816(h1[mt][nt], af, ld_pair(w), ld_pair(w + 8));
      }
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int j = 0; j < 4; ++j) h1[mt][nt][j] = fmaxf(h1[mt][nt][j], 0.0f);
    // layer 2
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      h2[mt][nt][0] = h2[mt][nt][2] = P.b2[8 * nt + 2 * t];
      h2[mt][nt][1] = h2[mt][nt][3] = P.b2[8 * nt + 2 * t + 1];
    }
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      uint32_t af[4];
      af[0] = pack_bf16(h1[mt][2 * kk][0], h1[mt][2 * kk][1]);
      af[1] = pack_bf16(h1[mt][2 * kk][2], h1[mt][2 * kk][3]);
      af[2] = pack_bf16(h1[mt][2 * kk + 1][0], h1[mt][2 * kk + 1][1]);
      af[3] = pack_bf16(h1[mt][2 * kk + 1][2], h1[mt][2 * kk + 1][3]);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const __nv_bfloat16* w = P.W2 + (8 * nt + g) * H + 16 * kk + 2 * t;
        mma16816(h2[mt][nt], af, ld_pair(w), ld_pair(w + 8));
      }
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int j = 0; j < 4; ++j) h2[mt][nt][j] = fmaxf(h2[mt][nt][j], 0.0f);
    // layer 3 (N padded to 8; column 0 is the logit)
    z[mt][0] = z[mt][1] = z[mt][2] = z[mt][3] = P.b3;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      uint32_t af[4];
      af[0] = pack_bf16(h2[mt][2 * kk][0], h2[mt][2 * kk][1]);
      af[1] = pack_bf16(h2[mt][2 * kk][2], h2[mt][2 * kk][3]);
      af[2] = pack_bf16(h2[mt][2 * kk + 1][0], h2[mt][2 * kk + 1][1]);
      af[3] = pack_bf16(h2[mt][2 * kk + 1][2], h2[mt][2 * kk + 1][3]);
      const __nv_bfloat16* w = P.W3 + g * H + 16 * kk + 2 * t;
      mma16816(z[mt], af, ld_pair(w), ld_pair(w + 8));
    }
  }
}

template <int D>
__device__ __forceinline__ void load_pack(const Pack<D>* __restrict__ src, Pack<D>* dst) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(Pack<D>) / 16); i += blockDim.x) d[i] = s[i];
}

// Normalise a feature block in place: deviations from the central value divided by
// d = max(max |deviation|, 1e-4 |central value|) (+1e-30); returns d.  The floor is the
// amplitude below which the training labels call a component smooth, so smaller variations
// show as small inputs (and the rounding of a float32 pressure stays below 0.01).
template <int N0, int C>
__device__ __forceinline__ float normalise_block(float* v) {
  const float vc = v[C];
  float mx = 0.0f;
#pragma unroll
  for (int l = 0; l < N0; ++l) mx = fmaxf(mx, fabsf(v[l] - vc));
  const float d = fmaxf(mx, 1e-4f * fabsf(vc) + 1e-30f);
  const float inv = __frcp_rn(d);
#pragma unroll
  for (int l = 0; l < N0; ++l) v[l] = (v[l] - vc) * inv;
  return d;
}

// 3D shell 4 < |o|^2 <= 9 (the radius-3 stencil minus the radius-2 one), z-outer, x fastest
struct ShellTable {
  int n;
  int off[90][3];
};
constexpr ShellTable make_shell() {
  ShellTable t{};
  t.n = 0;
  for (int k = -3; k <= 3; ++k)
    for (int j = -3; j <= 3; ++j)
      for (int i = -3; i <= 3; ++i) {
        const int r2 = i * i + j * j + k * k;
        if (r2 > 4 && r2 <= 9) {
          t.off[t.n][0] = i;
          t.off[t.n][1] = j;
          t.off[t.n][2] = k;
          ++t.n;
        }
      }
  return t;
}
static_assert(make_shell().n == 90, "the radius-3 shell has 90 cells");
template <int L>
struct Shell {
  static constexpr int x = make_shell().off[L][0], y = make_shell().off[L][1], z = make_shell().off[L][2];
};

// shell input of one block: m / (m + d), m = max |v_shell - v_c|, d = the block's normaliser
__device__ __forceinline__ float shell_feature(float m, float d) { return m * __frcp_rn(m + d); }

}  // namespace gate
}  // namespace kfvm
