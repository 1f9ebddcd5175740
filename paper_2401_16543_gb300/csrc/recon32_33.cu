// recon32_33.cu -- FP32 Riemann states for d = 3, R = 3 (Sec. 3, Sec. 4, Sec. 5.3 steps 1-3).
//
// The same mathematics as recon32.cuh, arranged for the size of this case: S0 has
// 123 cells, there are 8 stencils with 348 (stencil, cell) pairs, 54 face points
// and 19 derivative multi-indices, i.e. 25,404 multiply-adds per variable and
// cell.  Two kernels: recon33_tc_kernel (the default) runs the contraction on the
// tcgen05 tensor cores (described at its namespace below); recon33_kernel runs it
// on the FP32 pipe.  Unrolling the contraction with compile-time weights, as the
// smaller cases do, would give a kernel of ~10^5 instructions, so in recon33_kernel
//   * the weights are a float32 row table in global memory, one row of 56 face
//     values + 20 derivative values (zero padded, float4 aligned) per (stencil,
//     cell) pair; every thread of a warp reads the same row, so the loads are
//     broadcasts served by L1;
//   * the tile offsets of the 348 pairs sit in constant memory;
//   * a (cell, variable) is reconstructed in two passes: derivative values of
//     every stencil -> beta_q -> WENO-AO coefficients, then the face values of all
//     stencils accumulated with the coefficient folded into the stencil value;
//   * the reconstructed dW (54 points x 5 variables) is parked in the cell's own
//     slots of the output buffer and read back by the tail (limiter, primitive
//     states), which overwrites them: no shared-memory copy of 270 values per cell.
// The gated mode evaluates the learned gate on the tile (features of the radius-2
// stencil, MLP on the tensor cores) and compacts the WENO cells as recon32 does.
#include <cuda_fp16.h>

#include <cmath>

#include "internal.h"
#include "recon32.cuh"
#include "tc.cuh"

namespace kfvm {
namespace r33 {

using G = Geo<3, 3>;
using T = r32::T32<3, 3>;
constexpr int NV = 5, NQ = G::NQ, F = G::F, M = G::M, SN = T::SN, TH = T::THREADS;
constexpr int FP = 56, MP = 20, ROW = FP + MP;  // floats per weight row
constexpr int ROW4 = ROW / 4;                   // float4 per row
static_assert(F <= FP && M <= MP && FP % 4 == 0 && MP % 4 == 0, "row padding");

struct Pairs {
  int start[NQ + 1];  // first pair of each stencil
  int off[G::N0 * 3];  // tile offset of the cell of each pair
};

constexpr Pairs make_pairs() {
  Pairs p{};
  int k = 0;
  for (int q = 0; q < NQ; ++q) {
    p.start[q] = k;
    for (int j = 0; j < G::tab.len[q]; ++j, ++k) {
      const int l = G::tab.idx[q][j];
      p.off[k] = G::tab.off[l][0] + T::SX * (G::tab.off[l][1] + T::SY * G::tab.off[l][2]);
    }
  }
  p.start[NQ] = k;
  return p;
}
constexpr Pairs kPairs = make_pairs();
constexpr int NP = kPairs.start[NQ];
static_assert(NP == 348, "3D R=3 has 348 (stencil, cell) pairs");

__constant__ Pairs c_pairs = make_pairs();

// shared memory layout (floats)
struct Smem {
  static constexpr int base = (NV + 1) * SN;                   // cell averages + pressures
  static constexpr int list_off = base;                        // [TH] ints
  static constexpr int pack_off = (list_off + TH + 3) / 4 * 4;  // gate parameters (16-byte aligned)
  static constexpr int pack_floats = (int)(sizeof(gate::Pack<3>) / 4);
  static constexpr int xs_off = pack_off + pack_floats;
  static constexpr int xs_floats = TH * gate::Dims<3>::LDX / 2;
  static constexpr int z_off = xs_off + xs_floats;
  static constexpr int plain = pack_off;
  static constexpr int gated = z_off + TH;
};

// address of the dW slot (point s, variable v) of buffer cell fc: the variable's own
// place in the float32 Riemann-state layout ([s][cell] float4 (rho,u,v,p), plane of w)
__device__ __forceinline__ float* slot(float* faces, long long ncell_f, long long fc, int s, int v) {
  if (v == 3) return faces + 4LL * F * ncell_f + (long long)s * ncell_f + fc;
  const int comp = v == 4 ? 3 : v;
  return faces + (((long long)s * ncell_f + fc) << 2) + comp;
}

// reference state of a tile cell and the lin-prim delta of one variable (Eq. 33, relative to
// the centre: row v of Phi applied to U_o - U_c)
struct Ref {
  float uc[NV], ut[3], kin, irt, uv, ucv, gm1;  // ucv = uc[v], kept out of the runtime-indexed array
  int v;
  __device__ __forceinline__ Ref(const float* __restrict__ sm, int cc, int var, float gm1_) : gm1(gm1_), v(var) {
    r32::cell_ref<3, 3>(sm, cc, uc, ut, kin, irt);
    uv = v == 1 ? ut[0] : (v == 2 ? ut[1] : ut[2]);
    ucv = v == 1 ? uc[1] : (v == 2 ? uc[2] : uc[3]);
  }
  __device__ __forceinline__ float delta(const float* __restrict__ sm, int o) const {
    const float dr = sm[o] - uc[0];
    if (v == 0) return dr;
    if (v <= 3) return fmaf(-uv, dr, sm[v * SN + o] - ucv) * irt;
    float t = fmaf(kin, dr, sm[4 * SN + o] - uc[4]);
    t = fmaf(-ut[0], sm[SN + o] - uc[1], t);
    t = fmaf(-ut[1], sm[2 * SN + o] - uc[2], t);
    t = fmaf(-ut[2], sm[3 * SN + o] - uc[3], t);
    return gm1 * t;
  }
  __device__ __forceinline__ float fold(float inv_s) const {
    return v == 0 ? inv_s : (v <= 3 ? irt * inv_s : gm1 * inv_s);
  }
  // delta(o) times a power of two inv_s of the variable V (= v, known at compile time) at the four tile
  // offsets o of cell cc, the scale folded into the row's last factor (fs = fold(inv_s): the same
  // bits as delta(o) * inv_s)
  template <int V>
  __device__ __forceinline__ void deltas4(const float* __restrict__ sm, int cc, int4 o, float fs,
                                          float (&x)[4]) const {
    const int oo[4] = {cc + o.x, cc + o.y, cc + o.z, cc + o.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float dr = sm[oo[e]] - uc[0];
      if constexpr (V == 0) {
        x[e] = dr * fs;
      } else if constexpr (V <= 3) {
        x[e] = fmaf(-ut[V - 1], dr, sm[V * SN + oo[e]] - uc[V]) * fs;
      } else {
        float t = fmaf(kin, dr, sm[4 * SN + oo[e]] - uc[4]);
        t = fmaf(-ut[0], sm[SN + oo[e]] - uc[1], t);
        t = fmaf(-ut[1], sm[2 * SN + oo[e]] - uc[2], t);
        t = fmaf(-ut[2], sm[3 * SN + oo[e]] - uc[3], t);
        x[e] = t * fs;
      }
    }
  }
};

// smoothness indicators beta_q (Eq. 22) of every stencil for one (cell, variable)
template <class Delta>
__device__ __forceinline__ void betas(int cc, Delta delta, const float4* __restrict__ Wt, float (&beta)[NQ]) {
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    float d[MP];
#pragma unroll
    for (int m = 0; m < MP; ++m) d[m] = 0.0f;
#pragma unroll 2
    for (int k = c_pairs.start[q]; k < c_pairs.start[q + 1]; ++k) {
      const float g = delta(cc + c_pairs.off[k]);
      const float4* wr = Wt + k * ROW4 + FP / 4;
#pragma unroll
      for (int m4 = 0; m4 < MP / 4; ++m4) {
        const float4 w = __ldg(wr + m4);
        d[4 * m4] = fmaf(w.x, g, d[4 * m4]);
        d[4 * m4 + 1] = fmaf(w.y, g, d[4 * m4 + 1]);
        d[4 * m4 + 2] = fmaf(w.z, g, d[4 * m4 + 2]);
        d[4 * m4 + 3] = fmaf(w.w, g, d[4 * m4 + 3]);
      }
    }
    float bq = 0.0f;
#pragma unroll
    for (int m = 0; m < M; ++m) bq = fmaf(d[m], d[m], bq);
    beta[q] = bq;
  }
}

// stage the float32 shadow of a tile (+ halo 3) and its float32 pressures
__device__ __forceinline__ void stage_tile(const GridArgs& a, const float* __restrict__ S, float* sm, float* sp,
                                           int x0, int y0, int z0, int nthreads = TH) {
  const long long ncell = (long long)a.n[0] * a.n[1] * a.n[2];
  const float gm1 = a.gammaf - 1.0f;
  for (int i = threadIdx.x; i < SN; i += nthreads) {
    const int sx = i % T::SX, sy = (i / T::SX) % T::SY, sz = i / (T::SX * T::SY);
    const int gx = map_index(x0 + sx, a.n[0], a.bc[0][0], a.bc[0][1]);
    const int gy = map_index(y0 + sy, a.n[1], a.bc[1][0], a.bc[1][1]);
    const int gz = map_index(z0 + sz, a.n[2], a.bc[2][0], a.bc[2][1]);
    const long long gc = ((long long)gz * a.n[1] + gy) * a.n[0] + gx;
    float u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      u[v] = S[v * ncell + gc];
      sm[v * SN + i] = u[v];
    }
    const float m2 = fmaf(u[1], u[1], fmaf(u[2], u[2], u[3] * u[3]));
    sp[i] = gm1 * fmaf(-0.5f * m2, __frcp_rn(u[0]), u[4]);
  }
}

__global__ void __launch_bounds__(TH, 3) recon33_kernel(GridArgs a, int mode, const double* __restrict__ U,
                                                        const float* __restrict__ S, float* faces,
                                                        const unsigned char* __restrict__ gate_mask,
                                                        const gate::Pack<3>* __restrict__ gpack, float zthresh,
                                                        const float4* __restrict__ Wt) {
  extern __shared__ float smem33[];
  float* sm = smem33;        // [NV][SN] shadow cell averages
  float* sp = sm + NV * SN;  // [SN] float32 pressures
  int* list = reinterpret_cast<int*>(smem33 + Smem::list_off);
  __shared__ int s_count;
  const long long ncell = (long long)a.n[0] * a.n[1] * a.n[2];
  const float gm1 = a.gammaf - 1.0f;
  const int tiles_x = (a.n[0] + T::TX - 1) / T::TX, tiles_y = (a.n[1] + T::TY - 1) / T::TY;
  int b = blockIdx.x;
  const int bx = b % tiles_x;
  b /= tiles_x;
  const int by = b % tiles_y;
  const int bz = b / tiles_y;
  const int x0 = bx * T::TX - T::H, y0 = by * T::TY - T::H, z0 = a.zf_first + bz * T::TZ - T::H;
  const int tid = threadIdx.x;
  if (tid == 0) s_count = 0;
  const long long ncell_f = face_ncell(a);

  stage_tile(a, S, sm, sp, x0, y0, z0);
  __syncthreads();

  // which cell of the tile this thread owns
  auto locate = [&](int t, int& cc, long long& cell, long long& fcell) {
    const int lx = t % T::TX, ly = (t / T::TX) % T::TY, lz = t / (T::TX * T::TY);
    const int x = bx * T::TX + lx, y = by * T::TY + ly, l = bz * T::TZ + lz;
    const int z = l < a.zf_count ? slab_plane(a, l) : -1;
    cc = (lx + T::H) + T::SX * ((ly + T::H) + T::SY * (lz + T::H));
    const bool ok = x < a.n[0] && y < a.n[1] && z >= 0;
    cell = ok ? ((long long)z * a.n[1] + y) * a.n[0] + x : -1;
    fcell = ok ? ((long long)l * a.n[1] + y) * a.n[0] + x : -1;
    return ok;
  };
  int c;
  long long cell, fcell;
  const bool active = locate(tid, c, cell, fcell);

  bool smooth = false;
  if (mode == 2) {
    using DM = gate::Dims<3>;
    gate::Pack<3>* P = reinterpret_cast<gate::Pack<3>*>(smem33 + Smem::pack_off);
    __nv_bfloat16* xs_all = reinterpret_cast<__nv_bfloat16*>(smem33 + Smem::xs_off);
    float* zs = smem33 + Smem::z_off;
    gate::load_pack<3>(gpack, P);
    float f[DM::NIN];
    r32::gate_features_tile<3, 3>(sm, sp, c, f, std::make_integer_sequence<int, Geo<3, 2>::N0>{});
    const int warp = tid >> 5, lane = tid & 31;
    __nv_bfloat16* xs = xs_all + warp * 32 * DM::LDX;
#pragma unroll
    for (int k = 0; k < DM::KIN; ++k) xs[lane * DM::LDX + k] = __float2bfloat16_rn(k < DM::NIN ? f[k] : 0.0f);
    __syncthreads();
    float h1[2][4][4], h2[2][4][4], zf[2][4];
    gate::forward32<3>(*P, xs, h1, h2, zf);
    if ((lane & 3) == 0) {
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        zs[warp * 32 + 16 * mt + (lane >> 2)] = zf[mt][0];
        zs[warp * 32 + 16 * mt + (lane >> 2) + 8] = zf[mt][2];
      }
    }
    __syncwarp();
    smooth = zs[tid] > zthresh;
  }

  // one reconstruction variable of one cell; linear = S0 only with coefficient 1
  auto recon_var = [&](int cc, long long fc, int v, bool linear) {
    const Ref r(sm, cc, v, gm1);
    float coef[NQ];
    coef[0] = 1.0f;
#pragma unroll
    for (int q = 1; q < NQ; ++q) coef[q] = 0.0f;
    if (!linear) {
      float beta[NQ];
      betas(cc, [&](int o) { return r.delta(sm, o); }, Wt, beta);
      // nonlinear weights in the scaled form (Eq. 24) and the WENO-AO coefficients (Eq. 25)
      float bmax = 0.0f;
#pragma unroll
      for (int q = 0; q < NQ; ++q) bmax = fmaxf(bmax, beta[q]);
      if (bmax > 0.0f) {
        const float ib = __frcp_rn(bmax);
        const float e = fmaxf(a.epsf * ib * ib, 1e-30f);
        float om[NQ], sum = 0.0f;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const float bq = beta[q] * ib;
          om[q] = __fdividef((float)linear_weight<3>(q), fmaf(bq, bq, e));
          sum += om[q];
        }
        const float inv = __frcp_rn(sum);
        const float w0 = om[0] * inv;
        coef[0] = w0 / (float)linear_weight<3>(0);
#pragma unroll
        for (int q = 1; q < NQ; ++q)
          coef[q] = fmaf(-w0, (float)(linear_weight<3>(q) / linear_weight<3>(0)), om[q] * inv);
      }
    }
    // pass 2: face values, sum over stencils of coef_q r_q(s) . g_q
    float acc[FP];
#pragma unroll
    for (int s = 0; s < FP; ++s) acc[s] = 0.0f;
    const int kend = linear ? c_pairs.start[1] : NP;
#pragma unroll 1
    for (int q = 0; q < NQ; ++q) {
      const int k0 = c_pairs.start[q], k1 = c_pairs.start[q + 1];
      if (k0 >= kend) break;
      float cq = coef[0];
#pragma unroll
      for (int qq = 1; qq < NQ; ++qq) cq = (q == qq) ? coef[qq] : cq;
#pragma unroll 2
      for (int k = k0; k < k1; ++k) {
        const float g = cq * r.delta(sm, cc + c_pairs.off[k]);
        const float4* wr = Wt + k * ROW4;
#pragma unroll
        for (int s4 = 0; s4 < FP / 4; ++s4) {
          const float4 w = __ldg(wr + s4);
          acc[4 * s4] = fmaf(w.x, g, acc[4 * s4]);
          acc[4 * s4 + 1] = fmaf(w.y, g, acc[4 * s4 + 1]);
          acc[4 * s4 + 2] = fmaf(w.z, g, acc[4 * s4 + 2]);
          acc[4 * s4 + 3] = fmaf(w.w, g, acc[4 * s4 + 3]);
        }
      }
    }
#pragma unroll
    for (int s = 0; s < F; ++s) *slot(faces, ncell_f, fc, s, v) = acc[s];
  };

  // phase 1: linear cells, each thread its own cell
  const bool weno_here = active && (mode == 0 || (mode == 2 && !smooth) || (mode == 3 && !gate_mask[cell]));
  if (active && !weno_here) {
#pragma unroll 1
    for (int v = 0; v < NV; ++v) recon_var(c, fcell, v, true);
  }
  // phase 2: WENO-AO (cell, variable) pairs; compacted in the gated modes
  if (mode == 0) {
    if (active) {
#pragma unroll 1
      for (int v = 0; v < NV; ++v) recon_var(c, fcell, v, false);
    }
  } else {
    __syncthreads();
    if (weno_here) list[atomicAdd(&s_count, 1)] = tid;
    __syncthreads();
    const int npairs = s_count * NV;
#pragma unroll 1
    for (int k = tid; k < npairs; k += TH) {
      int oc;
      long long ocell, ofc;
      locate(list[k / NV], oc, ocell, ofc);
      recon_var(oc, ofc, k % NV, false);
    }
  }
  __syncthreads();  // every dW slot of the tile written
  if (!active) return;
  r32::write_states<3, 3>(a, sm, sp, c, U, ncell, cell, fcell, ncell_f, faces,
                          [&](int s, int v) { return *slot(faces, ncell_f, fcell, s, v); });
}

// Training labels of the learned gate for d = 3, R = 3: the rule of r32::label_kernel
// (density and pressure components; float64 lin-prim deltas, float32 indicators), with the
// rolled contraction above.
__global__ void __launch_bounds__(TH) label33_kernel(GridArgs a, const double* __restrict__ U, float* __restrict__ y,
                                                     float thresh, const float4* __restrict__ Wt) {
  extern __shared__ double smem33l[];
  const int tiles_x = (a.n[0] + T::TX - 1) / T::TX, tiles_y = (a.n[1] + T::TY - 1) / T::TY;
  int b = blockIdx.x;
  const int bx = b % tiles_x;
  b /= tiles_x;
  const int by = b % tiles_y;
  const int bz = b / tiles_y;
  r32::stage64<3, 3>(a, U, smem33l, bx * T::TX - T::H, by * T::TY - T::H, bz * T::TZ - T::H);
  __syncthreads();
  const int tid = threadIdx.x;
  const int lx = tid % T::TX, ly = (tid / T::TX) % T::TY, lz = tid / (T::TX * T::TY);
  const int x = bx * T::TX + lx, yy = by * T::TY + ly, z = bz * T::TZ + lz;
  if (x >= a.n[0] || yy >= a.n[1] || z >= a.n[2]) return;
  const long long cell = ((long long)z * a.n[1] + yy) * a.n[0] + x;
  const int c = (lx + T::H) + T::SX * ((ly + T::H) + T::SY * (lz + T::H));
  const r32::Ref64<3, 3> r(smem33l, c, a.gamma);
  float worst = 1.0f;
#pragma unroll 1
  for (int iv = 0; iv < 2; ++iv) {
    const int v = iv == 0 ? 0 : NV - 1;  // density, pressure
    auto delta = [&](int o) { return r.delta(smem33l, o, v); };
    float amp = 0.0f;
#pragma unroll 4
    for (int k = 0; k < c_pairs.start[1]; ++k) amp = fmaxf(amp, fabsf(delta(c + c_pairs.off[k])));
    if ((double)amp <= 1e-4 * r.scale_of(v)) continue;
    float beta[NQ];
    betas(c, delta, Wt, beta);
    worst = fminf(worst, r32::omega0_ratio<3, NQ>(beta, a.epsf));
  }
  y[cell] = worst >= thresh ? 1.0f : 0.0f;
}

// Tail of one cell shared by its four threads of the tensor-core kernel (quarter h owns the face
// points 16 h ... 16 h + 15): the same arithmetic as r32::write_states -- central pressure (float64
// where E/p shows cancellation), positivity limiter (Sec. 4) on the reconstructed dW, float32
// primitive Riemann states -- with the limiter's theta_rho and theta_p, minima over all 54 points,
// combined through shared memory (xch: 2 x 4 x 128 floats).  The quarter's dW come from two loaders
// that every thread calls (they may read tensor memory, which takes the whole warp): ld_rho(d) the
// density deltas of its 16 points, ld_half(m0, dw) all variables of points m0 ... m0 + 7.  Every
// thread of the CTA calls it (it holds two CTA barriers); inactive rows only take part.
template <class LdRho, class LdHalf>
__device__ __forceinline__ void write_states_split(const GridArgs& a, const float* __restrict__ sm,
                                                   const float* __restrict__ sp, int c, const double* __restrict__ U,
                                                   long long ncell, long long cell, long long fcell, long long ncell_f,
                                                   float* faces, bool active, int r, int h, float* xch, LdRho ld_rho,
                                                   LdHalf ld_half) {
  constexpr int P = 16, HP = 8;  // face points per quarter (the last quarter has F - 48 = 6), half
  const int s_lo = P * h;
  const float gm1 = a.gammaf - 1.0f;
  float uc[NV], ut[3] = {0.f, 0.f, 0.f}, kin = 0.0f, irt = 1.0f;
  float pt = 0.0f, rt = 1.0f, cq = 0.0f, th = 1.0f, thp = 1.0f;
  float p_min = 0.0f;
  float d0[P];
  ld_rho(d0);
  if (active) {
    r32::cell_ref<3, 3>(sm, c, uc, ut, kin, irt);
    // central pressure: float32 where E/p < 8, else recovered in float64 from the state
    pt = sp[c];
    if (!(pt > 0.125f * uc[NV - 1])) {
      double m2 = 0.0, u8[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) u8[v] = U[v * ncell + cell];
#pragma unroll
      for (int k = 0; k < 3; ++k) m2 = fma(u8[1 + k], u8[1 + k], m2);
      const double p8 = (a.gamma - 1.0) * fma(-0.5 * m2, recip64(u8[0]), u8[NV - 1]);
      pt = (float)p8;
      if (!(u8[0] > 0.0) || !(p8 > 0.0)) raise_flag(a.status, kFlagNonphysical);
    }
    rt = uc[0];
    cq = 0.5f * gm1 * rt * rt;  // (gamma-1) rho~^2 / 2
    if (a.positivity) {
      float rmax = -3.0e38f, rmin = 3.0e38f, pmin = 3.0e38f;
#pragma unroll
      for (int k = -1; k <= 1; ++k)
#pragma unroll
        for (int j = -1; j <= 1; ++j)
#pragma unroll
          for (int i = -1; i <= 1; ++i) {
            const int o = c + i + T::SX * (j + T::SY * k);
            rmax = fmaxf(rmax, sm[o]);
            rmin = fminf(rmin, sm[o]);
            pmin = fminf(pmin, sp[o]);
          }
      const float rho_max = rmax * a.hi_f, rho_min = rmin * a.lo_f;
      p_min = pmin * a.lo_f;
#pragma unroll
      for (int m = 0; m < P; ++m) {
        if (s_lo + m >= F) continue;
        const float rs = rt + d0[m];
        if (rs < rho_min) th = fminf(th, (rt - rho_min) / (rt - rs));
        if (rs > rho_max) th = fminf(th, (rho_max - rt) / (rs - rt));
      }
    }
  }
  xch[h * 128 + r] = th;
  __syncthreads();
  th = fminf(fminf(xch[r], xch[128 + r]), fminf(xch[256 + r], xch[384 + r]));
  float dw[NV][HP];
  if (a.positivity) {
    // p(theta) >= p_min  <=>  (pt + theta dpi - p_min) (rt + theta drho) >= cq theta^2 |du|^2
    auto admissible = [&](float t, float dr, float dp, float du2) {
      const float rr = fmaf(t, dr, rt);
      return rr > 0.0f && (fmaf(t, dp, pt) - p_min) * rr >= cq * t * t * du2;
    };
#pragma unroll
    for (int m0 = 0; m0 < P; m0 += HP) {
      ld_half(m0, dw);
      if (!active) continue;
#pragma unroll
      for (int m = 0; m < HP; ++m) {
        if (s_lo + m0 + m >= F) continue;
        const float dr = th * dw[0][m];
        const float dp = th * dw[NV - 1][m];
        float du2 = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float du = th * dw[1 + k][m];
          du2 = fmaf(du, du, du2);
        }
        if (admissible(1.0f, dr, dp, du2)) continue;
        float lo = 0.0f, hi = 1.0f;
#pragma unroll 1
        for (int it = 0; it < 40; ++it) {
          const float mid = 0.5f * (lo + hi);
          if (admissible(mid, dr, dp, du2)) lo = mid; else hi = mid;
        }
        thp = fminf(thp, lo);
      }
    }
  }
  xch[512 + h * 128 + r] = thp;
  __syncthreads();
  thp = fminf(fminf(xch[512 + r], xch[640 + r]), fminf(xch[768 + r], xch[896 + r]));
  const float scl = th * thp;
  float4* out4 = reinterpret_cast<float4*>(faces);
#pragma unroll
  for (int m0 = 0; m0 < P; m0 += HP) {
    ld_half(m0, dw);
    if (!active) continue;
#pragma unroll
    for (int m = 0; m < HP; ++m) {
      const int s = s_lo + m0 + m;
      if (s >= F) continue;
      const float dr = scl * dw[0][m];
      const float rs = rt + dr;
      const float irs = __frcp_rn(rs);
      float du2 = 0.0f, uo[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float du = scl * dw[1 + k][m];
        du2 = fmaf(du, du, du2);
        uo[k] = fmaf(rt * du, irs, ut[k]);
      }
      const float dp = scl * dw[NV - 1][m];
      const float ps = fmaf(-cq * du2, irs, pt + dp);
      // float32 layout: [s][cell] float4 (rho, u, v, p), then the plane [s][cell] of w
      out4[(long long)s * ncell_f + fcell] = make_float4(rs, uo[0], uo[1], ps);
      faces[4LL * F * ncell_f + (long long)s * ncell_f + fcell] = uo[2];
    }
  }
}

// ===========================================================================
// Tensor-core variant (tcgen05): the contraction as a GEMM per (tile of 128 cells, variable).
//
// Rows of A are the 128 cells of a tile (M = 128, one TMEM lane per cell); its K
// columns are the (stencil, cell) pairs, each stencil's block padded to a multiple
// of 16 (128 + 48 + 6 x 32 = 368, 23 MMA k-steps).  A holds the lin-prim deltas
// divided by a per-(cell, variable) power of two s, split into two FP16 halves
// (hi + lo); B holds the weights split the same way (each output column scaled by a
// power of two).  Three kind::f16 MMAs per k-step (hi.hi + hi.lo + lo.hi, FP32
// accumulation in TMEM) carry ~22 bits, close to the FP32 contraction.
//
// Each chunk of A is built once per (tile, variable) and feeds one GEMM per product
// with N = 96 columns: the 32 derivative columns of its stencil (Eq. 23 rows, 19 used)
// and the 64 face columns (Eq. 18 rows, 54 used), one B block per k-step.  A stencil's
// accumulators occupy one of two TMEM regions (columns 128 i ... 128 i + 95); the stencils
// are consumed in order as soon as their MMAs complete: beta_q (Eq. 22) -> the
// unnormalised WENO weight w~_q = gamma_q / (beta'^2 + eps') (Eq. 24, beta' = beta / s^2,
// eps' = eps / s^4, the same weights as gamma_q / (beta^2 + eps) after normalisation) ->
// the WENO-AO coefficient of Eq. 19 times the stencil's face values, added to a running
// blend (S0 first, so w~_0 is known for every later stencil); the blend is divided by
// sum_q w~_q at the end.  The region is then handed back to the MMA-issuing thread.
// Denominators are floored at 1e-30: stencils whose beta' is below 1e-15 (a relative
// variation under the float32 resolution of the state) count as equally smooth.
// Tiles whose cells are all linear (gated modes) run the 8 face k-steps of S0 only.
// The CTA is persistent (one per SM): B (138 KB, FP16 hi/lo) is loaded into shared
// memory once; 512 threads build A chunks (cell r = t % 128, quarter h = t / 128 of each
// 16-wide k-step) in a ring of 2 chunks of 2 k-steps.  Each warp signals a written chunk
// on the chunk's "full" mbarrier (no CTA-wide barrier: only the issuer waits for every
// warp); thread 0 issues the MMAs and commits the buffer to its "free" mbarrier.  The scale s of a (cell, variable) is the
// power of two at or above the central cell's own scale (rho~, sound speed, p~), so A
// stays O(1) (FP16 subnormals cost at most ~3e-8 of that scale).  Every wait has an
// iteration limit; on expiry the kernel raises the timeout flag and stops.
// ===========================================================================
namespace tcg {

constexpr int KS = 23;                     // k-steps of 16
constexpr int KT = KS * 16;                // padded K = 368
constexpr int TCT = 512;                   // threads per CTA: 4 per cell row (a quarter of each k-step)
constexpr int KPC = 2;                     // MMA k-steps per ring chunk (one full / free hand-off each)
constexpr int NB = 2;                      // A ring buffers
constexpr int NREG = 2;                    // TMEM regions, one stencil's accumulators each
constexpr int NOUT = 96;                   // MMA columns per k-step: 32 derivative + 64 face values
constexpr int BB_BLOCK = NOUT * 16 * 2 * 2;  // B block of one k-step: 96 x 16 FP16, hi + lo
constexpr int BB_BYTES = KS * BB_BLOCK;
constexpr int CS_FLOATS = NQ * 32 + 64;    // column scales (derivatives per stencil, faces)
constexpr int B_BYTES = BB_BYTES + CS_FLOATS * 4;
constexpr int A_KS = 8192;                 // one k-step of A: 128 x 16 FP16, hi + lo
constexpr int A_BUF = KPC * A_KS;          // one ring chunk
constexpr int WAIT_LIMIT = 1 << 22;

// TMEM columns of region i (128 apart): the 32 derivative columns, then the 64 face columns
__host__ __device__ constexpr uint32_t der_col(int i) { return 128u * (uint32_t)i; }
__host__ __device__ constexpr uint32_t face_col(int i) { return 128u * (uint32_t)i + 32u; }
// where quarter h parks the blended dW of variable v until the tail: columns 256 + 64 v + 16 h for
// v < 4; the last variable in the 32 columns each region leaves free (96 ... 127, 224 ... 255)
__host__ __device__ constexpr uint32_t park_col(int v, int h) {
  return v < NV - 1 ? 256u + 64u * (uint32_t)v + 16u * (uint32_t)h
                    : 96u + 128u * (uint32_t)(h >> 1) + 16u * (uint32_t)(h & 1);
}
static_assert(NREG == 2 && der_col(1) + NOUT <= 224 && park_col(NV - 2, 3) + 16 <= 512, "TMEM columns");

struct KMap {
  int kq[KS];       // stencil of each k-step
  int first[KS];    // 1 on the first k-step of a stencil
  int last_of[NQ];  // last k-step of each stencil
  int off[KT];      // tile offset of each padded K column (0 for padding: the row's own cell, whose
                    // delta is exactly zero; the padding's B rows are zero too)
};

constexpr KMap make_kmap() {
  KMap m{};
  int kk = 0;
  for (int q = 0; q < NQ; ++q) {
    const int len = G::tab.len[q];
    const int padded = (len + 15) / 16 * 16;
    for (int j = 0; j < padded; ++j, ++kk) {
      if (j % 16 == 0) {
        m.kq[kk / 16] = q;
        m.first[kk / 16] = j == 0 ? 1 : 0;
      }
      if (j < len) {
        const int l = G::tab.idx[q][j];
        m.off[kk] = G::tab.off[l][0] + T::SX * (G::tab.off[l][1] + T::SY * G::tab.off[l][2]);
      } else {
        m.off[kk] = 0;
      }
    }
    m.last_of[q] = kk / 16 - 1;
  }
  return m;
}
static_assert(make_kmap().kq[KS - 1] == NQ - 1, "23 k-steps");
static_assert(make_kmap().last_of[0] == 7, "S0 takes 8 k-steps");
__constant__ KMap c_kmap = make_kmap();

// per-k-step facts for the issuing thread and the consumers as compile-time bit patterns (no
// constant-memory loads on the issue path): bit j of kFirst / kLast marks the first / last k-step
// of a stencil, kLastPacked holds each stencil's last k-step in 5 bits
constexpr uint32_t first_mask() {
  uint32_t v = 0;
  for (int j = 0; j < KS; ++j) v |= (uint32_t)make_kmap().first[j] << j;
  return v;
}
constexpr uint32_t last_mask() {
  uint32_t v = 0;
  for (int q = 0; q < NQ; ++q) v |= 1u << make_kmap().last_of[q];
  return v;
}
constexpr unsigned long long last_packed() {
  unsigned long long v = 0;
  for (int q = 0; q < NQ; ++q) v |= (unsigned long long)make_kmap().last_of[q] << (5 * q);
  return v;
}
constexpr uint32_t kFirst = first_mask(), kLast = last_mask();
constexpr unsigned long long kLastPacked = last_packed();
static_assert(KS <= 31 && NQ * 5 <= 64, "bit patterns");
__device__ __forceinline__ int last_kstep(int q) { return (int)((kLastPacked >> (5 * q)) & 31u); }
__device__ __forceinline__ int kstep_stencil(int j) { return __popc(kFirst & ((2u << j) - 1u)) - 1; }

// shared memory (bytes)
struct TSmem {
  static constexpr int b_off = 0;
  static constexpr int a_off = B_BYTES;                          // ring of NB A buffers
  static constexpr int tile_off = a_off + NB * A_BUF;            // (NV + 1) x SN floats
  static constexpr int koff_off = tile_off + (NV + 1) * SN * 4;  // tile offsets of the K columns
  static constexpr int pack_off = koff_off + KT * 4;              // gate parameters
  static constexpr int bar_off = (pack_off + (int)sizeof(gate::Pack<3>) + 15) / 16 * 16;
  static constexpr int nbar = 2 * NB + 2 * NREG + 1;  // chunk_full, chunk_free, sten_done, reg_free, drain
  static constexpr int total = bar_off + 8 * nbar + 16;
};
static_assert(TSmem::total <= 232448, "shared memory of one CTA");
static_assert(128 * gate::Dims<3>::LDX * 2 + 128 * 4 <= NB * A_BUF, "gate staging fits in the A ring");

// byte offset of (row, k) in a K-major FP16 tile of 16 columns (core matrices 8 x 16 B)
__host__ __device__ constexpr int tile_byte(int row, int k) {
  return (row / 8) * 256 + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2;
}

__device__ __forceinline__ uint32_t pack_half2(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__global__ void __launch_bounds__(TCT, 1) recon33_tc_kernel(GridArgs a, int mode, int ntiles,
                                                             const double* __restrict__ U,
                                                             const float* __restrict__ S, float* faces,
                                                             const unsigned char* __restrict__ gate_mask,
                                                             const gate::Pack<3>* __restrict__ gpack, float zthresh,
                                                             const uint4* __restrict__ bimg, int timeout_probe) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* Bs = tsm + TSmem::b_off;
  unsigned char* As = tsm + TSmem::a_off;
  float* sm = reinterpret_cast<float*>(tsm + TSmem::tile_off);
  float* sp = sm + NV * SN;
  const float* cs1 = reinterpret_cast<const float*>(Bs + BB_BYTES);
  const float* cs2 = cs1 + NQ * 32;
  uint64_t* chunk_full = reinterpret_cast<uint64_t*>(tsm + TSmem::bar_off);  // every warp wrote its rows
  uint64_t* chunk_free = chunk_full + NB;  // the chunk's MMAs have completed
  uint64_t* sten_done = chunk_free + NB;  // one commit per stencil occupying region i
  uint64_t* reg_free = sten_done + NREG;  // every warp has read region i's occupant
  uint64_t* drain = reg_free + NREG;      // exit after a failed wait
  uint32_t* tbase_s = reinterpret_cast<uint32_t*>(drain + 1);
  int* koff = reinterpret_cast<int*>(tsm + TSmem::koff_off);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = tid & 127, h = tid >> 7;
  const float gm1 = a.gammaf - 1.0f;
  const long long ncell_f = face_ncell(a);
  const int tiles_x = (a.n[0] + T::TX - 1) / T::TX, tiles_y = (a.n[1] + T::TY - 1) / T::TY;

  // ---- once per CTA: B image, gate parameters, barriers, TMEM ----
  for (int i = tid; i < B_BYTES / 16; i += TCT) reinterpret_cast<uint4*>(Bs)[i] = __ldg(bimg + i);
  for (int i = tid; i < KT; i += TCT) koff[i] = c_kmap.off[i];
  gate::Pack<3>* P = reinterpret_cast<gate::Pack<3>*>(tsm + TSmem::pack_off);
  if (mode == 2) gate::load_pack<3>(gpack, P);
  if (tid == 0) {
    for (int i = 0; i < NB; ++i) {
      tc::mbar_init(chunk_full + i, TCT / 32);
      tc::mbar_init(chunk_free + i, 1);
    }
    for (int i = 0; i < NREG; ++i) {
      tc::mbar_init(sten_done + i, 1);
      tc::mbar_init(reg_free + i, TCT / 32);
    }
    tc::mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(tbase_s, 512);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tbase_s;
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  const uint32_t id96 = tc::idesc_f16_f32(128, NOUT);
  const uint32_t a_addr = tc::smem_addr(As), b_addr = tc::smem_addr(Bs);

  uint32_t it = 0;                // A ring chunks used so far
  uint32_t sd_ph = 0;             // next parity of each sten_done barrier (bit i)
  uint32_t rf_ph = 0, rf_used = 0;  // issuer: next parity of each reg_free barrier, regions used once
  bool ok = true;

  // test hook of the bounded waits: wait on a phase that nothing completes (an mbarrier no thread
  // arrives on), give up after a short limit, raise the timeout flag and do no work
  if (timeout_probe) {
    bool got = true;
    if (tid == 0) got = tc::mbar_wait(reg_free, 0u, 1 << 10);  // phase 0 of a fresh barrier
    ok = __syncthreads_and(got) != 0;
  }
  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    int b = tile;
    const int bx = b % tiles_x;
    b /= tiles_x;
    const int by = b % tiles_y;
    const int bz = b / tiles_y;
    __syncthreads();  // the previous tile's tail is done with the staged cells
    stage_tile(a, S, sm, sp, bx * T::TX - T::H, by * T::TY - T::H, a.zf_first + bz * T::TZ - T::H, TCT);
    __syncthreads();
    // the cell of row r: a warp holds one y row of the tile across its four z planes (conflict-free
    // shared-memory gathers, see T32<3, 3>)
    const int lx = r % T::TX, lz = (r / T::TX) % T::TZ, ly = r / (T::TX * T::TZ);
    const int x = bx * T::TX + lx, y = by * T::TY + ly, l = bz * T::TZ + lz;
    const int z = l < a.zf_count ? slab_plane(a, l) : -1;
    const int c = (lx + T::H) + T::SX * ((ly + T::H) + T::SY * (lz + T::H));
    const bool active = x < a.n[0] && y < a.n[1] && z >= 0;
    const long long cell = active ? ((long long)z * a.n[1] + y) * a.n[0] + x : 0;
    const long long fcell = active ? ((long long)l * a.n[1] + y) * a.n[0] + x : 0;

    // which rows are linear (gated modes); the gate's staging lives in the A ring (free here:
    // every MMA of the previous tile has completed)
    bool smooth = false;
    if (mode == 2) {
      using DM = gate::Dims<3>;
      __nv_bfloat16* xs_all = reinterpret_cast<__nv_bfloat16*>(As);
      float* zs = reinterpret_cast<float*>(As + 128 * DM::LDX * 2);
      if (h == 0) {
        float f[DM::NIN];
        r32::gate_features_tile<3, 3>(sm, sp, c, f, std::make_integer_sequence<int, Geo<3, 2>::N0>{});
        __nv_bfloat16* xs = xs_all + warp * 32 * DM::LDX;
#pragma unroll
        for (int k = 0; k < DM::KIN; ++k) xs[lane * DM::LDX + k] = __float2bfloat16_rn(k < DM::NIN ? f[k] : 0.0f);
        __syncwarp();
        float h1[2][4][4], h2[2][4][4], zf[2][4];
        gate::forward32<3>(*P, xs, h1, h2, zf);
        if ((lane & 3) == 0) {
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            zs[warp * 32 + 16 * mt + (lane >> 2)] = zf[mt][0];
            zs[warp * 32 + 16 * mt + (lane >> 2) + 8] = zf[mt][2];
          }
        }
      }
      __syncthreads();
      smooth = zs[r] > zthresh;
      __syncthreads();  // the ring is written from here on
    }
    const bool weno_row = active && (mode == 0 || (mode == 2 && !smooth) || (mode == 3 && !gate_mask[cell]));
    const bool weno_tile = __syncthreads_or(weno_row) != 0;
    const int ks_end = weno_tile ? KS : last_kstep(0) + 1;
    const int nq_used = weno_tile ? NQ : 1;

#pragma unroll 1
    for (int v = 0; v < NV; ++v) {
      const Ref ref(sm, c, v, gm1);
      // s = power of two at or above the central cell's scale of this variable
      const float pc = sp[c];
      const float scale = v == 0 ? ref.uc[0] : (v == NV - 1 ? pc : sqrtf(fmaxf(a.gammaf * pc * ref.irt, 0.0f)));
      int ex = 0;
      if (scale > 0.0f && scale < 3.0e38f) frexpf(scale, &ex);
      const float inv_s = ldexpf(1.0f, -ex), sc = ldexpf(1.0f, ex);
      const float fs = ref.fold(inv_s);
      const float eps_s = fminf(ldexpf(a.epsf, -4 * ex), 1.0e30f);  // eps / s^4

      float acc[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) acc[m] = 0.0f;
      float wsum = 0.0f, w0g = 0.0f;  // sum of w~_q; w~_0 / gamma_0
      int nc = 0;                     // stencils consumed

      // stencil q's accumulators -> running WENO-AO blend of this thread's 16 face columns; the
      // region goes back to the issuer once every warp has read it
      auto consume = [&](int q) {
        const int i = q % NREG;
        if (!tc::mbar_wait(sten_done + i, (sd_ph >> i) & 1u, WAIT_LIMIT)) ok = false;
        sd_ph ^= 1u << i;
        tc::fence_after_sync();
        float cq = q == 0 ? 1.0f : 0.0f;  // linear rows: S0 alone
        float f[16];
        if (weno_tile) {
          static_assert(M > 16 && M <= 20, "19 derivative columns: 16 + 4 loaded");
          float d0[16], d1[4];
          tc::tmem_ld16_4_16(tbase + lane_base + der_col(i), tbase + lane_base + der_col(i) + 16u,
                             tbase + lane_base + face_col(i) + 16u * h, d0, d1, f);
          if (weno_row) {
            float bq = 0.0f;
#pragma unroll
            for (int m = 0; m < 16; ++m) {
              const float dm = d0[m] * cs1[q * 32 + m];
              bq = fmaf(dm, dm, bq);
            }
#pragma unroll
            for (int m = 16; m < M; ++m) {
              const float dm = d1[m - 16] * cs1[q * 32 + m];
              bq = fmaf(dm, dm, bq);
            }
            float gq = (float)linear_weight<3>(0);
#pragma unroll
            for (int qq = 1; qq < NQ; ++qq) gq = (q == qq) ? (float)linear_weight<3>(qq) : gq;
            const float wq = __fdividef(gq, fmaxf(fmaf(bq, bq, eps_s), 1.0e-30f));
            wsum += wq;
            if (q == 0) {
              w0g = wq * (float)(1.0 / linear_weight<3>(0));
              cq = w0g;
            } else {
              cq = fmaf(-w0g, gq, wq);  // w~_q - w~_0 gamma_q / gamma_0
            }
          }
        } else {
          tc::tmem_ld16(tbase + lane_base + face_col(i) + 16u * h, f);
        }
#pragma unroll
        for (int m = 0; m < 16; ++m) acc[m] = fmaf(cq, f[m], acc[m]);
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(reg_free + i);
      };

#pragma unroll 1
      for (int j0 = 0; j0 < ks_end; j0 += KPC) {
        const int nj = ks_end - j0 < KPC ? ks_end - j0 : KPC;
        // build the chunk: every thread writes its 4 columns (hi, lo) of row r per k-step
        const int buf = (int)(it % NB);
        const uint32_t use = it / NB;
        if (use > 0 && !tc::mbar_wait(chunk_free + buf, (use - 1) & 1u, WAIT_LIMIT)) ok = false;
        unsigned char* base = As + buf * A_BUF;
        const int ob = tile_byte(r, 4 * h);
#pragma unroll
        for (int jj = 0; jj < KPC; ++jj) {
          if (jj < nj) {
            // a linear row takes S0 alone and no smoothness indicator: its substencil columns stay zero
            // (a warp whose rows are all linear skips their gathers)
            const bool row_needs = active && (weno_row || j0 + jj <= last_kstep(0));
            float xv[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            if (row_needs) {
              const int4 o4 = *reinterpret_cast<const int4*>(koff + 16 * (j0 + jj) + 4 * h);
              switch (v) {  // uniform: the variable's arithmetic chosen once per k-step
                case 0: ref.deltas4<0>(sm, c, o4, fs, xv); break;
                case 1: ref.deltas4<1>(sm, c, o4, fs, xv); break;
                case 2: ref.deltas4<2>(sm, c, o4, fs, xv); break;
                case 3: ref.deltas4<3>(sm, c, o4, fs, xv); break;
                default: ref.deltas4<4>(sm, c, o4, fs, xv); break;
              }
            }
            // hi = FP16 rounding of each value (one rounding per pair), lo = FP16 of the remainder
            const __half2 h01 = __floats2half2_rn(xv[0], xv[1]), h23 = __floats2half2_rn(xv[2], xv[3]);
            const float2 f01 = __half22float2(h01), f23 = __half22float2(h23);
            uint2 hi, lo;
            hi.x = *reinterpret_cast<const uint32_t*>(&h01);
            hi.y = *reinterpret_cast<const uint32_t*>(&h23);
            lo.x = pack_half2(xv[0] - f01.x, xv[1] - f01.y);
            lo.y = pack_half2(xv[2] - f23.x, xv[3] - f23.y);
            *reinterpret_cast<uint2*>(base + jj * A_KS + ob) = hi;
            *reinterpret_cast<uint2*>(base + jj * A_KS + A_KS / 2 + ob) = lo;
          }
        }
        // hand the chunk to the issuing thread: no CTA barrier, only the issuer waits for all warps
        tc::fence_proxy_async();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(chunk_full + buf);
        // stencils whose MMAs were issued in earlier chunks, before this chunk's MMAs (which may
        // need their regions)
        while (nc < nq_used && last_kstep(nc) < j0) consume(nc++);
        if (tid == 0) {
          if (!tc::mbar_wait(chunk_full + buf, use & 1u, WAIT_LIMIT)) ok = false;
          tc::fence_after_sync();
          // descriptors: the chunk's and the weight image's base, plus the k-step's offset (>> 4, the
          // address field's unit; every address stays below 2^18)
          const uint64_t abase = tc::smem_desc(a_addr + buf * A_BUF, 128, 256);
          const uint64_t bbase = tc::smem_desc(b_addr, 128, 256);
#pragma unroll
          for (int jj = 0; jj < KPC; ++jj) {
            if (jj >= nj) break;
            const int j = j0 + jj, q = kstep_stencil(j), i = q % NREG;
            const bool first = (kFirst >> j) & 1u;
            if (first) {
              if ((rf_used >> i) & 1u) {
                if (!tc::mbar_wait(reg_free + i, (rf_ph >> i) & 1u, WAIT_LIMIT)) ok = false;
                rf_ph ^= 1u << i;
                tc::fence_after_sync();
              }
              rf_used |= 1u << i;
            }
            // derivative and face columns of stencil q in one N = 96 MMA per product (all-linear
            // tiles compute the derivative columns too and ignore them)
            const uint32_t acc0 = first ? 0u : 1u;
            const uint64_t ahi = abase + (uint64_t)((jj * A_KS) >> 4), alo = ahi + (uint64_t)((A_KS / 2) >> 4);
            const uint64_t bhi = bbase + (uint64_t)((j * BB_BLOCK) >> 4), blo = bhi + (uint64_t)((BB_BLOCK / 2) >> 4);
            tc::mma_f16(tbase + der_col(i), ahi, bhi, id96, acc0);
            tc::mma_f16(tbase + der_col(i), ahi, blo, id96, 1u);
            tc::mma_f16(tbase + der_col(i), alo, bhi, id96, 1u);
            if ((kLast >> j) & 1u) tc::commit(sten_done + i);
          }
          tc::commit(chunk_free + buf);
        }
        ++it;
      }
      while (nc < nq_used) consume(nc++);
      // blended face values / sum_q w~_q, back in the variable's units, parked in tensor memory (the
      // last variable in registers) until the tail
      const float inv_w = weno_row ? __frcp_rn(wsum) : 1.0f;
#pragma unroll
      for (int m = 0; m < 16; ++m) acc[m] = 16 * h + m < F ? acc[m] * inv_w * cs2[16 * h + m] * sc : 0.0f;
      tc::tmem_st16(tbase + lane_base + park_col(v, h), acc);
    }
    // one CTA-wide check per tile (nothing between the variables needs a CTA barrier: the ring and
    // the TMEM regions have their own hand-offs, and each thread parks and reads back its own dW)
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
    // the tail, four threads per cell, on the dW each thread parked itself in tensor memory; the A
    // ring (every MMA consumed) holds the limiter's exchange
    tc::fence_after_sync();
    auto ld_rho = [&](float (&d)[16]) { tc::tmem_ld16(tbase + lane_base + park_col(0, h), d); };
    auto ld_half = [&](int m0, float (&d)[NV][8]) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        float t8[8];
        tc::tmem_ld8(tbase + lane_base + park_col(v, h) + (uint32_t)m0, t8);
#pragma unroll
        for (int m = 0; m < 8; ++m) d[v][m] = t8[m];
      }
    };
    write_states_split(a, sm, sp, c, U, (long long)a.n[0] * a.n[1] * a.n[2], cell, fcell, ncell_f, faces, active, r,
                       h, reinterpret_cast<float*>(As), ld_rho, ld_half);
  }
  if (!ok) {
    if (tid == 0) raise_flag(a.status, kFlagTimeout);
    // let whatever is still in flight finish (bounded) before the TMEM goes back
    if (tid == 0) tc::commit(drain);
    tc::mbar_wait(drain, 0u, WAIT_LIMIT);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tbase, 512);
}
}  // namespace tcg
}  // namespace r33

size_t recon33_table_floats() { return (size_t)r33::NP * r33::ROW; }

// row table from the float64 weights (layout of kfvm_get_weights: per stencil q,
// F face rows then M derivative rows, each over the stencil's cells)
void recon33_fill_table(const double* w, float* out) {
  using namespace r33;
  constexpr StencilTable tab = make_stencil(3, 3);
  for (int q = 0, k = 0, wo = 0; q < NQ; wo += tab.len[q] * (F + M), ++q) {
    const int n = tab.len[q];
    for (int j = 0; j < n; ++j, ++k) {
      float* row = out + (size_t)k * ROW;
      for (int i = 0; i < ROW; ++i) row[i] = 0.0f;
      for (int s = 0; s < F; ++s) row[s] = (float)w[wo + s * n + j];
      for (int m = 0; m < M; ++m) row[FP + m] = (float)w[wo + F * n + m * n + j];
    }
  }
}

size_t recon33_tc_image_bytes() { return (size_t)r33::tcg::B_BYTES; }

// FP16 hi/lo image of the weights in the tensor-core kernel's shared-memory layout: per k-step one
// block of 96 columns x 16 K (the 32 derivative columns of its stencil, then the 64 face columns),
// hi then lo, then the power-of-two column scales (derivatives per stencil, faces)
void recon33_tc_fill_image(const double* w, unsigned char* out) {
  using namespace r33;
  using namespace r33::tcg;
  constexpr StencilTable tab = make_stencil(3, 3);
  constexpr KMap km = make_kmap();
  int woffq[NQ], kstart[NQ];
  for (int q = 0, wo = 0, ks = 0; q < NQ; ++q) {
    woffq[q] = wo;
    kstart[q] = ks;
    wo += tab.len[q] * (F + M);
    ks += (tab.len[q] + 15) / 16 * 16;
  }
  // weight of output column n (kind 1: derivative n of the k-step's stencil; kind 2: face point n) at
  // padded K kk
  auto weight = [&](int pass, int n, int kk) -> double {
    const int q = km.kq[kk / 16];
    const int jin = kk - kstart[q], len = tab.len[q];
    if (jin >= len) return 0.0;
    if (pass == 1) return n < M ? w[woffq[q] + F * len + n * len + jin] : 0.0;
    return n < F ? w[woffq[q] + n * len + jin] : 0.0;
  };
  float* cs = reinterpret_cast<float*>(out + BB_BYTES);
  float scale1[NQ][32], scale2[64];
  for (int q = 0; q < NQ; ++q)
    for (int n = 0; n < 32; ++n) {
      double mx = 0.0;
      for (int kk = 0; kk < KT; ++kk)
        if (km.kq[kk / 16] == q) mx = std::fmax(mx, std::fabs(weight(1, n, kk)));
      int e = 0;
      if (mx > 0.0) std::frexp(mx, &e);
      scale1[q][n] = (float)std::ldexp(1.0, -e);
      cs[q * 32 + n] = (float)std::ldexp(1.0, e);
    }
  for (int n = 0; n < 64; ++n) {
    double mx = 0.0;
    for (int kk = 0; kk < KT; ++kk) mx = std::fmax(mx, std::fabs(weight(2, n, kk)));
    int e = 0;
    if (mx > 0.0) std::frexp(mx, &e);
    scale2[n] = (float)std::ldexp(1.0, -e);
    cs[NQ * 32 + n] = (float)std::ldexp(1.0, e);
  }
  auto put = [&](unsigned char* blk, int n, int k, float v) {
    const __half hi = __float2half_rn(v);
    const __half lo = __float2half_rn(v - __half2float(hi));
    *reinterpret_cast<__half*>(blk + tile_byte(n, k)) = hi;
    *reinterpret_cast<__half*>(blk + BB_BLOCK / 2 + tile_byte(n, k)) = lo;
  };
  for (int j = 0; j < KS; ++j) {
    const int q = km.kq[j];
    unsigned char* blk = out + j * BB_BLOCK;
    for (int k = 0; k < 16; ++k) {
      for (int n = 0; n < 32; ++n) put(blk, n, k, (float)(weight(1, n, 16 * j + k) * scale1[q][n]));
      for (int n = 0; n < 64; ++n) put(blk, 32 + n, k, (float)(weight(2, n, 16 * j + k) * scale2[n]));
    }
  }
}

cudaError_t launch_recon32_33_tc(kfvm_ctx* ctx, const double* U, const float* shadow, float* faces, cudaStream_t st,
                                 int zf_first, int zf_count) {
  using namespace r33;
  GridArgs a = make_grid_args(ctx);
  if (zf_count > 0) {
    a.zf_first = zf_first;
    a.zf_count = zf_count;
  }
  const int ntiles = ((ctx->n[0] + T::TX - 1) / T::TX) * ((ctx->n[1] + T::TY - 1) / T::TY) *
                     ((a.zf_count + T::TZ - 1) / T::TZ);
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tcg::recon33_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tcg::TSmem::total);
  if (e != cudaSuccess) return e;
  const int grid = ntiles < nsm ? ntiles : nsm;
  const float th = (float)ctx->gate_threshold;
  const float zth = logf(th / (1.0f - th));
  tcg::recon33_tc_kernel<<<grid, tcg::TCT, tcg::TSmem::total, st>>>(
      a, kernel_recon_mode(ctx), ntiles, U, shadow, faces, ctx->d_gate_mask, (const gate::Pack<3>*)ctx->d_gate_pack, zth,
      reinterpret_cast<const uint4*>(ctx->d_w33tc), ctx->timeout_probe);
  ctx->timeout_probe = 0;
  ctx->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_recon32_33(kfvm_ctx* ctx, const double* U, const float* shadow, float* faces, cudaStream_t st,
                              int zf_first, int zf_count) {
  using namespace r33;
  if (ctx->tensor_cores && ctx->d_w33tc) return launch_recon32_33_tc(ctx, U, shadow, faces, st, zf_first, zf_count);
  GridArgs a = make_grid_args(ctx);
  if (zf_count > 0) {
    a.zf_first = zf_first;
    a.zf_count = zf_count;
  }
  const int tiles = ((ctx->n[0] + T::TX - 1) / T::TX) * ((ctx->n[1] + T::TY - 1) / T::TY) *
                    ((a.zf_count + T::TZ - 1) / T::TZ);
  const bool learned = ctx->recon == 2;
  const size_t smem = sizeof(float) * (learned ? Smem::gated : Smem::plain);
  cudaError_t e = cudaFuncSetAttribute(recon33_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(float) * Smem::gated));
  if (e != cudaSuccess) return e;
  const float th = (float)ctx->gate_threshold;
  const float zth = logf(th / (1.0f - th));
  recon33_kernel<<<tiles, TH, smem, st>>>(a, kernel_recon_mode(ctx), U, shadow, faces, ctx->d_gate_mask,
                                          (const gate::Pack<3>*)ctx->d_gate_pack, zth,
                                          reinterpret_cast<const float4*>(ctx->d_w32));
  ctx->launches += 1;
  return cudaGetLastError();
}

}  // namespace kfvm

namespace kfvm {
cudaError_t launch_labels_33(kfvm_ctx* ctx, const double* U, float* y, float thresh, cudaStream_t st) {
  using namespace r33;
  const GridArgs a = make_grid_args(ctx);
  const int tiles = ((ctx->n[0] + T::TX - 1) / T::TX) * ((ctx->n[1] + T::TY - 1) / T::TY) *
                    ((ctx->n[2] + T::TZ - 1) / T::TZ);
  const size_t smem = sizeof(double) * NV * SN;
  cudaError_t e = cudaFuncSetAttribute(label33_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  label33_kernel<<<tiles, TH, smem, st>>>(a, U, y, thresh, reinterpret_cast<const float4*>(ctx->d_w32));
  ctx->launches += 1;
  return cudaGetLastError();
}
}  // namespace kfvm
