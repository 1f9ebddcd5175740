// recon32.cuh -- FP32 Riemann states of the mixed-precision path (Sec. 5.3 steps 1-3).
//
// Same mathematics as recon64 (Sec. 3, Sec. 4), arranged for the FP32 pipe:
//   * the CTA stages a float32 shadow of its tile of cell averages (+ halo R);
//   * the stencil is transformed to linearized primitive variables RELATIVE
//     to the central cell, dW_h = Phi (U_h - U_c) (Eq. 33); since every
//     reconstruction vector sums to one and the WENO-AO coefficients sum to
//     one, w_s = W_c + (reconstruction of dW), with W_c = (rho~, 0, p~);
//   * contractions with compile-time indices (C++17 fold expressions over the
//     stencil tables) so the stencil stays in registers and the weights are
//     constant-bank operands;
//   * nonlinear weights in the scaled form omega_q ~ gamma_q/((beta_q/beta_max)^2
//     + eps/beta_max^2), identical in exact arithmetic to Eq. 24 (eps = 1e-40 is
//     subnormal in float32);
//   * the pressure at a face point follows without cancellation from the
//     linearized primitive values: p_s = pi_s - (gamma-1) rho~^2 |du_s|^2 / (2 rho_s),
//     and the positivity limiter (Sec. 4) works on the same quantities
//     (the blend toward the cell average is linear, so it is a scaling of dW);
//   * the central pressure p~ is recovered in float64 (with a float32 reciprocal
//     refined by one Newton step) wherever E/p >= 8, i.e. where E - |m|^2/(2 rho)
//     cancels (high Mach numbers, near vacuum); elsewhere float32 suffices.
// Output: float32 primitive (rho, u, [v, w,] p) Riemann states.
// In the gated mode the cells the gate marks smooth take the linear S0
// reconstruction; the others are compacted within the CTA so that whole warps
// run WENO-AO.
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <utility>

#include "common.cuh"
#include "gate.cuh"

namespace kfvm {
namespace r32 {

template <int D, int R>
struct T32 {
  static constexpr int TX = (D == 2) ? 32 : 8;
  static constexpr int TY = (D == 2) ? 8 : 8;
  static constexpr int TZ = (D == 2) ? 1 : 2;
  static constexpr int H = R;
  static constexpr int SX = TX + 2 * H, SY = TY + 2 * H, SZ = (D == 2) ? 1 : TZ + 2 * H;
  static constexpr int SN = SX * SY * SZ;
  static constexpr int THREADS = TX * TY * TZ;
};
// d = 3, R = 3: an 8 x 4 x 4 tile keeps the radius-3 halo at 1400 cells; the planes are padded
// from 14 x 10 to 14 x 12 = 168 cells (= 8 mod 32 banks), so that 32 cells of one y row and
// four z planes read 32 different banks at any common stencil offset
template <>
struct T32<3, 3> {
  static constexpr int TX = 8, TY = 4, TZ = 4, H = 3;
  static constexpr int SX = TX + 2 * H, SY = TY + 2 * H + 2, SZ = TZ + 2 * H;
  static constexpr int SN = SX * SY * SZ;
  static constexpr int THREADS = TX * TY * TZ;
};

// compile-time views of the stencil tables (scalar constexpr members are usable in device code)
template <int D, int R, int Q, int J>
struct SIdx {
  static constexpr int v = Geo<D, R>::tab.idx[Q][J];
};
template <int D, int R, int Q>
struct SLen {
  static constexpr int v = Geo<D, R>::tab.len[Q];
};
template <int D, int R, int Q>
struct WOff {
  static constexpr int v = Geo<D, R>::woff(Q);
};
template <int D, int R, int L>
struct Dlt {
  static constexpr int v = Geo<D, R>::tab.off[L][0] +
                           T32<D, R>::SX * (Geo<D, R>::tab.off[L][1] + T32<D, R>::SY * Geo<D, R>::tab.off[L][2]);
};

// offsets of the radius-2 stencil (the gate's input) in the tile of radius R
template <int D, int R, int L>
struct Dlt2 {
  static constexpr int v = Geo<D, 2>::tab.off[L][0] +
                           T32<D, R>::SX * (Geo<D, 2>::tab.off[L][1] + T32<D, R>::SY * Geo<D, 2>::tab.off[L][2]);
};

// offsets of the 3D radius-3 shell (the gate's shell inputs) in the tile of radius R >= 3
template <int D, int R, int L>
struct DltS {
  static constexpr int v = gate::Shell<L>::x + T32<D, R>::SX * (gate::Shell<L>::y + T32<D, R>::SY * gate::Shell<L>::z);
};

template <int D, int R, int... Ss>
__device__ __forceinline__ void shell_max(const float* __restrict__ sm, const float* __restrict__ sp, int c, float rc,
                                          float pc, float& mr, float& mp, std::integer_sequence<int, Ss...>) {
  ((mr = fmaxf(mr, fabsf(sm[c + DltS<D, R, Ss>::v] - rc)), mp = fmaxf(mp, fabsf(sp[c + DltS<D, R, Ss>::v] - pc))),
   ...);
}

template <int D, int R, int... Ls>
__device__ __forceinline__ void gate_features_tile(const float* __restrict__ sm, const float* __restrict__ sp, int c,
                                                   float* f, std::integer_sequence<int, Ls...>) {
  constexpr int N0 = Geo<D, 2>::N0;
  ((f[Ls] = sm[c + Dlt2<D, R, Ls>::v]), ...);
  ((f[N0 + Ls] = sp[c + Dlt2<D, R, Ls>::v]), ...);
  const float rc = sm[c], pc = sp[c];
  const float dr = gate::normalise_block<N0, Geo<D, 2>::center()>(f);
  const float dp = gate::normalise_block<N0, Geo<D, 2>::center()>(f + N0);
  if constexpr (D == 3) {
    float mr = 0.0f, mp = 0.0f;
    if constexpr (R >= 3) shell_max<D, R>(sm, sp, c, rc, pc, mr, mp, std::make_integer_sequence<int, 90>{});
    f[2 * N0] = gate::shell_feature(mr, dr);
    f[2 * N0 + 1] = gate::shell_feature(mp, dp);
  }
}

// dynamic shared memory of recon32_kernel (floats), and where the gate's pieces sit
template <int D, int R>
struct Smem32 {
  using T = T32<D, R>;
  using G = Geo<D, R>;
  static constexpr int base = (G::NV + 1) * T::SN + G::F * G::NV * T::THREADS + T::THREADS;  // + list (ints)
  static constexpr int pack_off = (base + 3) / 4 * 4;                                           // 16-byte aligned
  static constexpr int pack_floats = (int)(sizeof(gate::Pack<D>) / 4);
  static constexpr int total_gate = pack_off + pack_floats;
  // the gate's input rows and logits live in the dW region, which phase 1 writes only after them
  static constexpr int dw_off = (G::NV + 1) * T::SN;
  static constexpr int xs_off = (dw_off + 3) / 4 * 4;
  static constexpr int xs_floats = T::THREADS * gate::Dims<D>::LDX / 2;
  static constexpr int z_off = xs_off + xs_floats;
  static_assert(z_off + T::THREADS <= dw_off + G::F * G::NV * T::THREADS, "gate staging must fit in dW");
};

template <int D, int R>
struct W32 {
  float w[Geo<D, R>::WCOUNT];
};

// r . g over substencil Q with the weight row starting at OFF
template <int D, int R, int Q, int OFF, int... J>
__device__ __forceinline__ float dot_q(const W32<D, R>& W, const float (&g)[Geo<D, R>::N0],
                                       std::integer_sequence<int, J...>) {
  float acc = 0.0f;
  ((acc = fmaf(W.w[OFF + J], g[SIdx<D, R, Q, J>::v], acc)), ...);
  return acc;
}

template <int D, int R, int Q, int M_>
__device__ __forceinline__ float deriv(const W32<D, R>& W, const float (&g)[Geo<D, R>::N0]) {
  constexpr int n = SLen<D, R, Q>::v;
  return dot_q<D, R, Q, WOff<D, R, Q>::v + Geo<D, R>::F * n + M_ * n>(W, g, std::make_integer_sequence<int, n>{});
}

template <int D, int R, int Q, int... Ms>
__device__ __forceinline__ float beta_q(const W32<D, R>& W, const float (&g)[Geo<D, R>::N0],
                                        std::integer_sequence<int, Ms...>) {
  float b = 0.0f, t = 0.0f;
  ((t = deriv<D, R, Q, Ms>(W, g), b = fmaf(t, t, b)), ...);
  return b;
}

template <int D, int R, int Q, int S>
__device__ __forceinline__ float face_q(const W32<D, R>& W, const float (&g)[Geo<D, R>::N0]) {
  constexpr int n = SLen<D, R, Q>::v;
  return dot_q<D, R, Q, WOff<D, R, Q>::v + S * n>(W, g, std::make_integer_sequence<int, n>{});
}

template <int D, int R, int S, int... Qs>
__device__ __forceinline__ float face_blend(const W32<D, R>& W, const float (&g)[Geo<D, R>::N0],
                                            const float (&coef)[Geo<D, R>::NQ], std::integer_sequence<int, Qs...>) {
  float acc = 0.0f;
  ((acc = fmaf(coef[Qs], face_q<D, R, Qs, S>(W, g), acc)), ...);
  return acc;
}

template <int D, int R, int... Qs>
__device__ __forceinline__ void all_betas(const W32<D, R>& W, const float (&g)[Geo<D, R>::N0],
                                          float (&beta)[Geo<D, R>::NQ], std::integer_sequence<int, Qs...>) {
  ((beta[Qs] = beta_q<D, R, Qs>(W, g, std::make_integer_sequence<int, Geo<D, R>::M>{})), ...);
}

template <int D, int R, int... Ss>
__device__ __forceinline__ void all_faces_weno(const W32<D, R>& W, const float (&g)[Geo<D, R>::N0],
                                               const float (&coef)[Geo<D, R>::NQ], float* out, int stride,
                                               std::integer_sequence<int, Ss...>) {
  ((out[Ss * stride] = face_blend<D, R, Ss>(W, g, coef, std::make_integer_sequence<int, Geo<D, R>::NQ>{})), ...);
}

template <int D, int R, int... Ss>
__device__ __forceinline__ void all_faces_linear(const W32<D, R>& W, const float (&g)[Geo<D, R>::N0], float* out,
                                                 int stride, std::integer_sequence<int, Ss...>) {
  ((out[Ss * stride] = face_q<D, R, 0, Ss>(W, g)), ...);
}

// load dW (row v of Phi applied to U_l - U_c) for every S0 cell into g
template <int D, int R, int... Ls>
__device__ __forceinline__ void gather_row(const float* __restrict__ sm, int c, int v, float (&g)[Geo<D, R>::N0],
                                           const float* uc, const float* ut, float kin, float irt, float gm1,
                                           std::integer_sequence<int, Ls...>) {
  constexpr int SN = T32<D, R>::SN;
  if (v == 0) {
    ((g[Ls] = sm[c + Dlt<D, R, Ls>::v] - uc[0]), ...);
  } else if (v <= D) {
    const float uv = (v == 1) ? ut[0] : (v == 2 ? ut[1] : ut[D == 3 ? 2 : 1]);
    ((g[Ls] = (fmaf(-uv, sm[c + Dlt<D, R, Ls>::v] - uc[0], sm[v * SN + c + Dlt<D, R, Ls>::v] - uc[v])) * irt), ...);
  } else {
    auto pr = [&](int o) {
      float t = fmaf(kin, sm[o] - uc[0], sm[(D + 1) * SN + o] - uc[D + 1]);
#pragma unroll
      for (int k = 0; k < D; ++k) t = fmaf(-ut[k], sm[(1 + k) * SN + o] - uc[1 + k], t);
      return gm1 * t;
    };
    ((g[Ls] = pr(c + Dlt<D, R, Ls>::v)), ...);
  }
}

// reference state of a tile cell: averages, velocity, kinetic energy per mass, 1/rho
template <int D, int R>
__device__ __forceinline__ void cell_ref(const float* __restrict__ sm, int cc, float* uc, float* ut, float& kin,
                                         float& irt) {
  constexpr int NV = D + 2, SN = T32<D, R>::SN;
#pragma unroll
  for (int v = 0; v < NV; ++v) uc[v] = sm[v * SN + cc];
  irt = __frcp_rn(uc[0]);
  kin = 0.0f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    ut[k] = uc[1 + k] * irt;
    kin = fmaf(ut[k], ut[k], kin);
  }
  kin *= 0.5f;
}

// Tail of the FP32 reconstruction of one cell: central pressure (float64 where E/p shows
// cancellation), positivity limiter (Sec. 4) on the reconstructed dW = dwget(s, v), and the
// float32 primitive Riemann states.
template <int D, int R, class DW>
__device__ __forceinline__ void write_states(const GridArgs& a, const float* __restrict__ sm,
                                             const float* __restrict__ sp, int c, const double* __restrict__ U,
                                             long long ncell, long long cell, long long fcell, long long ncell_f,
                                             float* faces, DW dwget) {
  using G = Geo<D, R>;
  using T = T32<D, R>;
  constexpr int NV = G::NV, F = G::F;
  const float gm1 = a.gammaf - 1.0f;
  float uc[NV], ut[3] = {0.f, 0.f, 0.f}, kin, irt;
  cell_ref<D, R>(sm, c, uc, ut, kin, irt);
  // central pressure: float32 where E/p < 8 (the cancellation E - |m|^2/(2 rho) then costs
  // under 3 bits, relative error below 6e-7), else recovered in float64 from the state
  float pt = sp[c];
  if (!(pt > 0.125f * uc[D + 1])) {
    double m2 = 0.0, u8[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) u8[v] = U[v * ncell + cell];
#pragma unroll
    for (int k = 0; k < D; ++k) m2 = fma(u8[1 + k], u8[1 + k], m2);
    const double p8 = (a.gamma - 1.0) * fma(-0.5 * m2, recip64(u8[0]), u8[D + 1]);
    pt = (float)p8;
    if (!(u8[0] > 0.0) || !(p8 > 0.0)) raise_flag(a.status, kFlagNonphysical);
  }
  const float rt = uc[0];
  const float cq = 0.5f * gm1 * rt * rt;  // (gamma-1) rho~^2 / 2
  float th = 1.0f, thp = 1.0f;
  if (a.positivity) {
    float rmax = -3.0e38f, rmin = 3.0e38f, pmin = 3.0e38f;
#pragma unroll
    for (int k = (D == 3 ? -1 : 0); k <= (D == 3 ? 1 : 0); ++k)
#pragma unroll
      for (int j = -1; j <= 1; ++j)
#pragma unroll
        for (int i = -1; i <= 1; ++i) {
          const int o = c + i + T::SX * (j + T::SY * k);
          rmax = fmaxf(rmax, sm[o]);
          rmin = fminf(rmin, sm[o]);
          pmin = fminf(pmin, sp[o]);
        }
    const float rho_max = rmax * a.hi_f, rho_min = rmin * a.lo_f, p_min = pmin * a.lo_f;
#pragma unroll
    for (int s = 0; s < F; ++s) {
      const float drs = dwget(s, 0);
      const float rs = rt + drs;
      if (rs < rho_min) th = fminf(th, (rt - rho_min) / (rt - rs));
      if (rs > rho_max) th = fminf(th, (rho_max - rt) / (rs - rt));
    }
    // p(theta) >= p_min  <=>  (pt + theta dpi - p_min) (rt + theta drho) >= cq theta^2 |du|^2
    auto admissible = [&](float t, float dr, float dp, float du2) {
      const float rr = fmaf(t, dr, rt);
      return rr > 0.0f && (fmaf(t, dp, pt) - p_min) * rr >= cq * t * t * du2;
    };
#pragma unroll 1
    for (int s = 0; s < F; ++s) {
      const float dr = th * dwget(s, 0);
      const float dp = th * dwget(s, NV - 1);
      float du2 = 0.0f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float du = th * dwget(s, 1 + k);
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
  const float sc = th * thp;
  float4* out4 = reinterpret_cast<float4*>(faces);
#pragma unroll 1
  for (int s = 0; s < F; ++s) {
    const float dr = sc * dwget(s, 0);
    const float rs = rt + dr;
    const float irs = __frcp_rn(rs);
    float du2 = 0.0f, uo[3];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float du = sc * dwget(s, 1 + k);
      du2 = fmaf(du, du, du2);
      uo[k] = fmaf(rt * du, irs, ut[k]);
    }
    const float dp = sc * dwget(s, NV - 1);
    const float ps = fmaf(-cq * du2, irs, pt + dp);
    // float32 layout: [s][cell] float4 (rho, u, v, p), then (3D) the plane [s][cell] of w
    out4[(long long)s * ncell_f + fcell] = make_float4(rs, uo[0], uo[1], ps);
    if (D == 3) faces[4LL * F * ncell_f + (long long)s * ncell_f + fcell] = uo[D == 3 ? 2 : 0];
  }
}

// Characteristic variables of direction dir (Sec. 3.4.1) in float32 at the central average uc, from
// its velocity ut, kinetic energy per mass kin and 1/rho irt: L (rows: left eigenvectors of the flux
// Jacobian of dir) and Rm (columns: right eigenvectors).  Waves u_n - c, entropy, the shear waves of
// the tangential axes in increasing order, u_n + c; b1 = (gamma-1)/c^2, b2 = b1 |u|^2/2,
// H = (E+p)/rho.
template <int D>
__device__ __forceinline__ void char_matrices32(const float* uc, const float* ut, float kin, float irt, float pc,
                                                float gamma, int dir, float (&L)[D + 2][D + 2],
                                                float (&Rm)[D + 2][D + 2]) {
  constexpr int NV = D + 2;
  const float c = sqrtf(gamma * pc * irt), ic = __frcp_rn(c), H = (uc[NV - 1] + pc) * irt;
  const float q2 = 2.0f * kin;
  const float b1 = (gamma - 1.0f) * ic * ic, b2 = 0.5f * b1 * q2, un = ut[dir];
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int j = 0; j < NV; ++j) L[i][j] = Rm[i][j] = 0.0f;
  Rm[0][0] = Rm[0][1] = Rm[0][NV - 1] = 1.0f;
  L[0][0] = 0.5f * (b2 + un * ic);
  L[1][0] = 1.0f - b2;
  L[NV - 1][0] = 0.5f * (b2 - un * ic);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float nk = (k == dir) ? 1.0f : 0.0f;
    Rm[1 + k][0] = ut[k] - c * nk;
    Rm[1 + k][1] = ut[k];
    Rm[1 + k][NV - 1] = ut[k] + c * nk;
    L[0][1 + k] = 0.5f * (-b1 * ut[k] - nk * ic);
    L[1][1 + k] = b1 * ut[k];
    L[NV - 1][1 + k] = 0.5f * (-b1 * ut[k] + nk * ic);
  }
  Rm[NV - 1][0] = H - c * un;
  Rm[NV - 1][1] = 0.5f * q2;
  Rm[NV - 1][NV - 1] = H + c * un;
  L[0][NV - 1] = 0.5f * b1;
  L[1][NV - 1] = -b1;
  L[NV - 1][NV - 1] = 0.5f * b1;
  int w = 2;
#pragma unroll
  for (int t = 0; t < D; ++t) {
    if (t == dir) continue;
    Rm[1 + t][w] = 1.0f;
    Rm[NV - 1][w] = ut[t];
    L[w][0] = -ut[t];
    L[w][1 + t] = 1.0f;
    ++w;
  }
}

// row Lv of L applied to U_l - U_c for every S0 cell l (characteristic deltas relative to the centre)
template <int D, int R, int... Ls>
__device__ __forceinline__ void gather_char(const float* __restrict__ sm, int c, const float* Lv, const float* uc,
                                            float (&g)[Geo<D, R>::N0], std::integer_sequence<int, Ls...>) {
  constexpr int SN = T32<D, R>::SN, NV = D + 2;
  auto one = [&](int o) {
    float t = 0.0f;
#pragma unroll
    for (int j = 0; j < NV; ++j) t = fmaf(Lv[j], sm[j * SN + o] - uc[j], t);
    return t;
  };
  ((g[Ls] = one(c + Dlt<D, R, Ls>::v)), ...);
}

// WENO-AO values (Eq. 19) at the face points S0 + k, k < 2 NT: the two faces normal to one direction
template <int D, int R, int S0, int... Ks>
__device__ __forceinline__ void faces_weno_range(const W32<D, R>& W, const float (&g)[Geo<D, R>::N0],
                                                 const float (&coef)[Geo<D, R>::NQ], float* out, int stride,
                                                 std::integer_sequence<int, Ks...>) {
  ((out[(S0 + Ks) * stride] = face_blend<D, R, S0 + Ks>(W, g, coef, std::make_integer_sequence<int, Geo<D, R>::NQ>{})),
   ...);
}

// nonlinear weights in the scaled form (reading of Eq. 24 for float32) and the WENO-AO coefficients
// of Eq. 19 from the smoothness indicators of one (cell, variable)
template <int D, int NQ>
__device__ __forceinline__ void weno_coefficients(const float (&beta)[NQ], float epsf, float (&coef)[NQ]) {
  float bmax = 0.0f;
#pragma unroll
  for (int q = 0; q < NQ; ++q) bmax = fmaxf(bmax, beta[q]);
  if (bmax > 0.0f) {
    const float ib = __frcp_rn(bmax);
    const float e = fmaxf(epsf * ib * ib, 1e-30f);
    float om[NQ], sum = 0.0f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const float bq = beta[q] * ib;
      om[q] = __fdividef((float)linear_weight<D>(q), fmaf(bq, bq, e));
      sum += om[q];
    }
    const float inv = __frcp_rn(sum);
    const float w0 = om[0] * inv;
    coef[0] = w0 / (float)linear_weight<D>(0);
#pragma unroll
    for (int q = 1; q < NQ; ++q) coef[q] = fmaf(-w0, (float)(linear_weight<D>(q) / linear_weight<D>(0)), om[q] * inv);
  } else {
    coef[0] = 1.0f;
#pragma unroll
    for (int q = 1; q < NQ; ++q) coef[q] = 0.0f;
  }
}

// CH: WENO-AO cells in characteristic variables (Sec. 3.4.1), a separate instantiation; the values
// at a direction's face points are reconstructed in that direction's characteristic deltas with their
// own weights, then taken back (R, then Phi) to the linearized primitive deltas the tail expects.
template <int D, int R, bool CH = false>
__global__ void __launch_bounds__(T32<D, R>::THREADS, (D == 2 && R == 2) ? 3 : 1) recon32_kernel(GridArgs a, int mode,
                                                                     const double* __restrict__ U,
                                                                     const float* __restrict__ S,
                                                                     float* __restrict__ faces,
                                                                     const unsigned char* __restrict__ gate_mask,
                                                                     const gate::Pack<D>* __restrict__ gpack,
                                                                     float zthresh,
                                                                     const __grid_constant__ W32<D, R> W) {
  using G = Geo<D, R>;
  using T = T32<D, R>;
  constexpr int NV = G::NV, SN = T::SN, F = G::F, NQ = G::NQ, N0 = G::N0, TH = T::THREADS;
  extern __shared__ float smem32[];
  float* sm = smem32;                 // [NV][SN] shadow cell averages
  float* sp = sm + NV * SN;           // [SN] float32 pressures (limiter bounds)
  float* dw = sp + SN;                // [F*NV][TH] reconstructed dW per cell of the tile
  int* list = reinterpret_cast<int*>(dw + F * NV * TH);  // [TH] compacted WENO cells
  __shared__ int s_count;
  const long long ncell = (long long)a.n[0] * a.n[1] * a.n[2];
  const float gm1 = a.gammaf - 1.0f;

  const int tiles_x = (a.n[0] + T::TX - 1) / T::TX, tiles_y = (a.n[1] + T::TY - 1) / T::TY;
  int b = blockIdx.x;
  const int bx = b % tiles_x;
  b /= tiles_x;
  const int by = b % tiles_y;
  const int bz = b / tiles_y;
  const int x0 = bx * T::TX - T::H, y0 = by * T::TY - T::H, z0 = (D == 3) ? a.zf_first + bz * T::TZ - T::H : 0;
  const int tid = threadIdx.x;
  if (tid == 0) s_count = 0;
  const long long ncell_f = face_ncell(a);

  for (int i = tid; i < SN; i += TH) {
    const int sx = i % T::SX, sy = (i / T::SX) % T::SY, sz = i / (T::SX * T::SY);
    const int gx = map_index(x0 + sx, a.n[0], a.bc[0][0], a.bc[0][1]);
    const int gy = map_index(y0 + sy, a.n[1], a.bc[1][0], a.bc[1][1]);
    const int gz = (D == 3) ? map_index(z0 + sz, a.n[2], a.bc[2][0], a.bc[2][1]) : 0;
    const long long gc = ((long long)gz * a.n[1] + gy) * a.n[0] + gx;
    float u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      u[v] = S[v * ncell + gc];
      sm[v * SN + i] = u[v];
    }
    float m2 = 0.0f;
#pragma unroll
    for (int k = 0; k < D; ++k) m2 = fmaf(u[1 + k], u[1 + k], m2);
    sp[i] = gm1 * fmaf(-0.5f * m2, __frcp_rn(u[0]), u[D + 1]);
  }
  __syncthreads();

  const int lx = tid % T::TX, ly = (tid / T::TX) % T::TY, lz = tid / (T::TX * T::TY);
  const int x = bx * T::TX + lx, y = by * T::TY + ly, l = (D == 3) ? bz * T::TZ + lz : 0;
  const int z = (D == 3) ? (l < a.zf_count ? slab_plane(a, l) : -1) : 0;
  const bool active = x < a.n[0] && y < a.n[1] && z >= 0;
  const long long cell = active ? ((long long)z * a.n[1] + y) * a.n[0] + x : 0;
  const long long fcell = active ? ((long long)l * a.n[1] + y) * a.n[0] + x : 0;
  const int c = (lx + T::H) + T::SX * ((ly + T::H) + T::SY * (D == 3 ? lz + T::H : 0));
  float* mydw = dw + tid;

  // ---- learned gate, fused: features from the tile, the MLP on the tensor cores per warp ----
  bool smooth = false;
  if (mode == 2) {
    using SM = Smem32<D, R>;
    using DM = gate::Dims<D>;
    gate::Pack<D>* P = reinterpret_cast<gate::Pack<D>*>(smem32 + SM::pack_off);
    __nv_bfloat16* xs_all = reinterpret_cast<__nv_bfloat16*>(smem32 + SM::xs_off);
    float* zs = smem32 + SM::z_off;
    gate::load_pack<D>(gpack, P);
    float f[DM::NIN];
    gate_features_tile<D, R>(sm, sp, c, f, std::make_integer_sequence<int, Geo<D, 2>::N0>{});
    const int warp = tid >> 5, lane = tid & 31;
    __nv_bfloat16* xs = xs_all + warp * 32 * DM::LDX;
#pragma unroll
    for (int k = 0; k < DM::KIN; ++k) xs[lane * DM::LDX + k] = __float2bfloat16_rn(k < DM::NIN ? f[k] : 0.0f);
    __syncthreads();  // pack and rows in place
    float h1[2][4][4], h2[2][4][4], zf[2][4];
    gate::forward32<D>(*P, xs, h1, h2, zf);
    if ((lane & 3) == 0) {
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        zs[warp * 32 + 16 * mt + (lane >> 2)] = zf[mt][0];
        zs[warp * 32 + 16 * mt + (lane >> 2) + 8] = zf[mt][2];
      }
    }
    __syncwarp();
    smooth = zs[tid] > zthresh;
    __syncthreads();  // the dW region is reused from here on
  }
  constexpr auto SEQ_L = std::make_integer_sequence<int, N0>{};
  constexpr auto SEQ_S = std::make_integer_sequence<int, F>{};


  // ---- phase 1: linear cells (all cells in the linear mode) ----
  bool weno_here = active && (mode == 0 || (mode == 2 && !smooth) || (mode == 3 && !gate_mask[cell]));
  if (active && !weno_here) {
    float uc[NV], ut[3] = {0.f, 0.f, 0.f}, kin, irt;
    cell_ref<D, R>(sm, c, uc, ut, kin, irt);
    float g[N0];
#pragma unroll 1
    for (int v = 0; v < NV; ++v) {
      gather_row<D, R>(sm, c, v, g, uc, ut, kin, irt, gm1, SEQ_L);
      all_faces_linear<D, R>(W, g, mydw + v * TH, NV * TH, SEQ_S);
    }
  }
  // ---- phase 2: WENO-AO cells, compacted within the CTA ----
  if (mode == 0) {
    // every active cell is a WENO cell: no compaction needed
  } else {
    if (weno_here) list[atomicAdd(&s_count, 1)] = tid;
  }
  __syncthreads();
  // one WENO-AO reconstruction variable of one cell (the variables are independent)
  auto weno_var = [&](int owner, int v) {
    const int olx = owner % T::TX, oly = (owner / T::TX) % T::TY, olz = owner / (T::TX * T::TY);
    const int oc = (olx + T::H) + T::SX * ((oly + T::H) + T::SY * (D == 3 ? olz + T::H : 0));
    float uc[NV], ut[3] = {0.f, 0.f, 0.f}, kin, irt;
    cell_ref<D, R>(sm, oc, uc, ut, kin, irt);
    float g[N0], beta[NQ], coef[NQ];
    if constexpr (!CH) {
      gather_row<D, R>(sm, oc, v, g, uc, ut, kin, irt, gm1, SEQ_L);
      all_betas<D, R>(W, g, beta, std::make_integer_sequence<int, NQ>{});
      weno_coefficients<D, NQ>(beta, a.epsf, coef);
      all_faces_weno<D, R>(W, g, coef, dw + owner + v * TH, NV * TH, SEQ_S);
    } else {
      // component v of each direction's characteristic variables, weights per direction, values at
      // that direction's two faces (slots of the characteristic component v until the back transform)
      constexpr int NT = G::NT;
      constexpr auto SEQ_F = std::make_integer_sequence<int, 2 * NT>{};
#pragma unroll
      for (int dir = 0; dir < D; ++dir) {
        float L[NV][NV], Rm[NV][NV];
        char_matrices32<D>(uc, ut, kin, irt, sp[oc], a.gammaf, dir, L, Rm);
        float Lv[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) Lv[j] = L[v][j];
        gather_char<D, R>(sm, oc, Lv, uc, g, SEQ_L);
        all_betas<D, R>(W, g, beta, std::make_integer_sequence<int, NQ>{});
        weno_coefficients<D, NQ>(beta, a.epsf, coef);
        float* out = dw + owner + v * TH;
        if (dir == 0) faces_weno_range<D, R, 0>(W, g, coef, out, NV * TH, SEQ_F);
        if (dir == 1) faces_weno_range<D, R, 2 * NT>(W, g, coef, out, NV * TH, SEQ_F);
        if constexpr (D == 3)
          if (dir == 2) faces_weno_range<D, R, 4 * NT>(W, g, coef, out, NV * TH, SEQ_F);
      }
    }
  };
  if (mode == 0) {
    // every active cell is a WENO cell: each thread its own cell, variable by variable
    if (active) {
#pragma unroll 1
      for (int v = 0; v < NV; ++v) weno_var(tid, v);
    }
  } else {
    // compacted WENO cells, one (cell, variable) pair per thread so that several warps share them
    const int npairs = s_count * NV;
#pragma unroll 1
    for (int k = tid; k < npairs; k += TH) weno_var(list[k / NV], k % NV);
  }
  __syncthreads();
  if (!active) return;
  if constexpr (CH) {
    // characteristic values of this WENO-AO cell back to conservative deltas (R) and to the
    // linearized primitive deltas of the tail (Phi): dW = Phi R w at every face point
    if (weno_here) {
      constexpr int NT = G::NT;
      float uc[NV], ut[3] = {0.f, 0.f, 0.f}, kin, irt;
      cell_ref<D, R>(sm, c, uc, ut, kin, irt);
#pragma unroll 1
      for (int dir = 0; dir < D; ++dir) {
        float L[NV][NV], Rm[NV][NV];
        char_matrices32<D>(uc, ut, kin, irt, sp[c], a.gammaf, dir, L, Rm);
#pragma unroll 1
        for (int k = 0; k < 2 * NT; ++k) {
          const int s = 2 * dir * NT + k;
          float w[NV], du[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) w[v] = mydw[(s * NV + v) * TH];
#pragma unroll
          for (int i = 0; i < NV; ++i) {
            float t = 0.0f;
#pragma unroll
            for (int j = 0; j < NV; ++j) t = fmaf(Rm[i][j], w[j], t);
            du[i] = t;
          }
          mydw[(s * NV + 0) * TH] = du[0];
          float pi = fmaf(kin, du[0], du[NV - 1]);
#pragma unroll
          for (int k2 = 0; k2 < D; ++k2) {
            mydw[(s * NV + 1 + k2) * TH] = fmaf(-ut[k2], du[0], du[1 + k2]) * irt;
            pi = fmaf(-ut[k2], du[1 + k2], pi);
          }
          mydw[(s * NV + NV - 1) * TH] = gm1 * pi;
        }
      }
    }
  }

  // ---- tail: central pressure in float64, limiter, primitive Riemann states ----
  write_states<D, R>(a, sm, sp, c, U, ncell, cell, fcell, ncell_f, faces,
                     [&](int s, int v) { return mydw[(s * NV + v) * TH]; });
}

// Training labels of the learned gate, from the cell's own WENO-AO weights
// (Eqs. 22, 24, 25): y = 1 when the density and the pressure components of the
// linearized primitive variables (the quantities the gate's inputs describe)
// are both smooth by the weights (omega_0/gamma_0 >= thresh = 1 - tau) or vary
// over the stencil by less than 1e-4 of their scale (rho~, p~), where WENO-AO
// and the linear reconstruction differ by less than that; else 0.  The lin-prim deltas are
// formed in float64 from the float64 state (a float32 shadow would leave
// rounding noise of ~1e-7 of E in components that are constant, and the
// weights of noise are random); the indicators then run in float32 as in the
// reconstruction.
template <int D, int R>
__device__ __forceinline__ float delta64(const double* __restrict__ sm, int o, int v, const double* uc,
                                         const double* ut, double kin, double irt, double gm1) {
  constexpr int SN = T32<D, R>::SN;
  const double dr = sm[o] - uc[0];
  if (v == 0) return (float)dr;
  if (v <= D) return (float)(fma(-ut[v - 1], dr, sm[v * SN + o] - uc[v]) * irt);
  double t = fma(kin, dr, sm[(D + 1) * SN + o] - uc[D + 1]);
#pragma unroll
  for (int k = 0; k < D; ++k) t = fma(-ut[k], sm[(1 + k) * SN + o] - uc[1 + k], t);
  return (float)(gm1 * t);
}

// float64 tile of the state (+ halo R); every label kernel stages it the same way
template <int D, int R>
__device__ __forceinline__ void stage64(const GridArgs& a, const double* __restrict__ U, double* sm, int x0, int y0,
                                        int z0) {
  using T = T32<D, R>;
  constexpr int NV = D + 2;
  const long long ncell = (long long)a.n[0] * a.n[1] * a.n[2];
  for (int i = threadIdx.x; i < T::SN; i += T::THREADS) {
    const int sx = i % T::SX, sy = (i / T::SX) % T::SY, sz = i / (T::SX * T::SY);
    const int gx = map_index(x0 + sx, a.n[0], a.bc[0][0], a.bc[0][1]);
    const int gy = map_index(y0 + sy, a.n[1], a.bc[1][0], a.bc[1][1]);
    const int gz = (D == 3) ? map_index(z0 + sz, a.n[2], a.bc[2][0], a.bc[2][1]) : 0;
    const long long gc = ((long long)gz * a.n[1] + gy) * a.n[0] + gx;
#pragma unroll
    for (int v = 0; v < NV; ++v) sm[v * T::SN + i] = U[v * ncell + gc];
  }
}

// reference quantities of a cell from the float64 tile: state, velocity, kinetic energy per
// mass, 1/rho, and the amplitude scales (rho, sound speed, p)
template <int D, int R>
struct Ref64 {
  double uc[D + 2], ut[3] = {0.0, 0.0, 0.0}, kin = 0.0, irt, gm1, scale[3];
  __device__ __forceinline__ Ref64(const double* __restrict__ sm, int c, double gamma) : gm1(gamma - 1.0) {
    constexpr int SN = T32<D, R>::SN;
#pragma unroll
    for (int v = 0; v < D + 2; ++v) uc[v] = sm[v * SN + c];
    irt = 1.0 / uc[0];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      ut[k] = uc[1 + k] * irt;
      kin = fma(ut[k], ut[k], kin);
    }
    kin *= 0.5;
    const double p = gm1 * (uc[D + 1] - uc[0] * kin);
    scale[0] = uc[0];
    scale[1] = sqrt(fmax(gamma * p * irt, 0.0));
    scale[2] = p;
  }
  __device__ __forceinline__ double scale_of(int v) const { return v == 0 ? scale[0] : (v == D + 1 ? scale[2] : scale[1]); }
  __device__ __forceinline__ float delta(const double* __restrict__ sm, int o, int v) const {
    return delta64<D, R>(sm, o, v, uc, ut, kin, irt, gm1);
  }
};

// lin-prim deltas of variable v over S0 (float64, rounded to float32); returns max |delta|
template <int D, int R, int... Ls>
__device__ __forceinline__ float load_deltas64(const Ref64<D, R>& r, const double* __restrict__ sm, int c, int v,
                                               float (&g)[Geo<D, R>::N0], std::integer_sequence<int, Ls...>) {
  float amp = 0.0f;
  ((g[Ls] = r.delta(sm, c + Dlt<D, R, Ls>::v, v), amp = fmaxf(amp, fabsf(g[Ls]))), ...);
  return amp;
}

// omega_0 / gamma_0 from the indicators (Eq. 24, scaled form)
template <int D, int NQ>
__device__ __forceinline__ float omega0_ratio(const float (&beta)[NQ], float epsf) {
  float bmax = 0.0f;
#pragma unroll
  for (int q = 0; q < NQ; ++q) bmax = fmaxf(bmax, beta[q]);
  if (!(bmax > 0.0f)) return 1.0f;
  const float ib = __frcp_rn(bmax);
  const float e = fmaxf(epsf * ib * ib, 1e-30f);
  float om0 = 0.0f, sum = 0.0f;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const float bq = beta[q] * ib;
    const float o = __fdividef((float)linear_weight<D>(q), fmaf(bq, bq, e));
    if (q == 0) om0 = o;
    sum += o;
  }
  return om0 / (sum * (float)linear_weight<D>(0));
}

template <int D, int R>
__global__ void __launch_bounds__(T32<D, R>::THREADS) label_kernel(GridArgs a, const double* __restrict__ U,
                                                                   float* __restrict__ y, float thresh,
                                                                   const __grid_constant__ W32<D, R> W) {
  using G = Geo<D, R>;
  using T = T32<D, R>;
  constexpr int NV = G::NV, NQ = G::NQ, N0 = G::N0;
  extern __shared__ double smem64l[];
  const int tiles_x = (a.n[0] + T::TX - 1) / T::TX, tiles_y = (a.n[1] + T::TY - 1) / T::TY;
  int b = blockIdx.x;
  const int bx = b % tiles_x;
  b /= tiles_x;
  const int by = b % tiles_y;
  const int bz = b / tiles_y;
  stage64<D, R>(a, U, smem64l, bx * T::TX - T::H, by * T::TY - T::H, (D == 3) ? bz * T::TZ - T::H : 0);
  __syncthreads();
  const int tid = threadIdx.x;
  const int lx = tid % T::TX, ly = (tid / T::TX) % T::TY, lz = tid / (T::TX * T::TY);
  const int x = bx * T::TX + lx, yy = by * T::TY + ly, z = (D == 3) ? bz * T::TZ + lz : 0;
  if (x >= a.n[0] || yy >= a.n[1] || z >= a.n[2]) return;
  const long long cell = ((long long)z * a.n[1] + yy) * a.n[0] + x;
  const int c = (lx + T::H) + T::SX * ((ly + T::H) + T::SY * (D == 3 ? lz + T::H : 0));
  const Ref64<D, R> r(smem64l, c, a.gamma);
  float worst = 1.0f;
#pragma unroll 1
  for (int iv = 0; iv < 2; ++iv) {
    const int v = iv == 0 ? 0 : NV - 1;  // density, pressure
    float g[N0];
    const float amp = load_deltas64<D, R>(r, smem64l, c, v, g, std::make_integer_sequence<int, N0>{});
    if ((double)amp <= 1e-4 * r.scale_of(v)) continue;  // negligible variation: smooth whatever the weights
    float beta[NQ];
    all_betas<D, R>(W, g, beta, std::make_integer_sequence<int, NQ>{});
    worst = fminf(worst, omega0_ratio<D, NQ>(beta, a.epsf));
  }
  y[cell] = worst >= thresh ? 1.0f : 0.0f;
}

template <int D, int R>
cudaError_t launch_labels(kfvm_ctx* ctx, const double* U, float* y, float thresh, cudaStream_t st) {
  using T = T32<D, R>;
  using G = Geo<D, R>;
  const GridArgs a = make_grid_args(ctx);
  const int tiles = ((ctx->n[0] + T::TX - 1) / T::TX) * ((ctx->n[1] + T::TY - 1) / T::TY) *
                    ((D == 3) ? (ctx->n[2] + T::TZ - 1) / T::TZ : 1);
  const size_t smem = sizeof(double) * G::NV * T::SN;
  cudaError_t e = cudaFuncSetAttribute(label_kernel<D, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  std::unique_ptr<W32<D, R>> wp(new W32<D, R>);
  for (int i = 0; i < G::WCOUNT; ++i) wp->w[i] = (float)ctx->w_host[i];
  label_kernel<D, R><<<tiles, T::THREADS, smem, st>>>(a, U, y, thresh, *wp);
  ctx->launches += 1;
  return cudaGetLastError();
}

template <int D, int R>
cudaError_t launch(kfvm_ctx* ctx, const double* U, const float* shadow, float* faces, cudaStream_t st,
                   int zf_first, int zf_count) {
  using T = T32<D, R>;
  using G = Geo<D, R>;
  GridArgs a = make_grid_args(ctx);
  if (D == 3 && zf_count > 0) {
    a.zf_first = zf_first;
    a.zf_count = zf_count;
  }
  const int tiles = ((ctx->n[0] + T::TX - 1) / T::TX) * ((ctx->n[1] + T::TY - 1) / T::TY) *
                    ((D == 3) ? (a.zf_count + T::TZ - 1) / T::TZ : 1);
  const bool learned = ctx->recon == 2;
  const size_t smem = sizeof(float) * (learned ? Smem32<D, R>::total_gate : Smem32<D, R>::base);
  auto kern = ctx->vars == 1 ? recon32_kernel<D, R, true> : recon32_kernel<D, R, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(float) * Smem32<D, R>::total_gate));
  if (e != cudaSuccess) return e;
  std::unique_ptr<W32<D, R>> wp(new W32<D, R>);
  for (int i = 0; i < G::WCOUNT; ++i) wp->w[i] = (float)ctx->w_host[i];
  const float th = (float)ctx->gate_threshold;
  const float zth = logf(th / (1.0f - th));
  kern<<<tiles, T::THREADS, smem, st>>>(a, kernel_recon_mode(ctx), U, shadow, faces, ctx->d_gate_mask,
                                        (const gate::Pack<D>*)ctx->d_gate_pack, zth, *wp);
  ctx->launches += 1;
  return cudaGetLastError();
}

}  // namespace r32
}  // namespace kfvm
