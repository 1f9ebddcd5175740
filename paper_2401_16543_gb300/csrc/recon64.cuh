// recon64.cuh -- FP64 Riemann states (Sec. 5.3 steps 1-3) of the plain path.
//
// One thread per cell; a CTA stages its tile of cell averages plus a halo of R
// cells in shared memory through the ghost-cell map (periodic wrap / outflow
// clamp).  Per cell, in float64 throughout:
//   * Phi from the central cell average (appendix A): W_h = Phi U_h over S0,
//     applied row by row with Phi's zeros skipped (Eq. 33);
//   * for each reconstruction variable: derivative values d_q(alpha).g_q and
//     beta_q = sum_alpha (d_q(alpha).g_q)^2 for q = 0..N_S (Eq. 22, unit-cell
//     coordinates), omega_q = gamma_q/(beta_q^2 + eps) normalised (Eqs. 24-25),
//     then the WENO-AO face values (ω0/γ0) r_0.g_0 + sum_q (ω_q - ω0 γ_q/γ0) r_q.g_q
//     at every face Gauss point (Eq. 19);
//   * back to conservative variables with the exact inverse Phi^{-1}
//     (Eq. 28; energy row rho*u_i);
//   * the positivity-preserving limiter of Sec. 4 (bounds from the 3^d
//     neighbourhood, theta_rho, theta_p by 60 bisection steps).
// With "variables" = 1 the WENO-AO cells reconstruct in characteristic
// variables instead (Sec. 3.4.1, recon_cell_char): one set of nonlinear weights
// per direction, serving that direction's faces.
// In the linear mode the conservative variables are reconstructed with r_0.
// The weight tables travel as a kernel parameter (constant bank, at most
// 28 KB: d = 2, and d = 3 with R = 2) or are read from global memory
// (d = 3, R = 3, 203 KB).
#pragma once
#include <cuda_runtime.h>

#include <memory>

#include "common.cuh"

namespace kfvm {
namespace r64 {

// Stencil plan in constant memory (geometry only, identical for every context
// with the same (d, R)): S0 cell offsets in the shared-memory tile, and for
// each (sub)stencil its length, its block in the weight table and its cells.
template <int D, int R>
struct Plan {
  int delta[kMaxN0];
  int len[kMaxNQ];
  int woff[kMaxNQ];
  int start[kMaxNQ];
  int idx[kMaxNQ * kMaxN0];
};

template <int D, int R>
__constant__ Plan<D, R> c_plan;

template <int D, int R>
Plan<D, R> make_plan() {
  Plan<D, R> p{};
  constexpr StencilTable t = make_stencil(D, R);
  using T = Tile<D, R>;
  for (int l = 0; l < t.n0; ++l) p.delta[l] = t.off[l][0] + T::SX * (t.off[l][1] + T::SY * t.off[l][2]);
  int w = 0, st = 0;
  for (int q = 0; q < t.nq; ++q) {
    p.len[q] = t.len[q];
    p.woff[q] = w;
    p.start[q] = st;
    for (int j = 0; j < t.len[q]; ++j) p.idx[st + j] = t.idx[q][j];
    st += t.len[q];
    w += t.len[q] * (Geo<D, R>::F + Geo<D, R>::M);
  }
  return p;
}

template <int D, int R>
struct W64 {
  double w[Geo<D, R>::WCOUNT];
};

// Weight source: the kernel-parameter copy (constant bank; d = 2 and d = 3
// with R = 2, at most 28 KB) or the global table (d = 3, R = 3).
template <int D, int R>
constexpr bool params_fit() {
  return Geo<D, R>::WCOUNT * 8 <= 28 * 1024;
}
template <int D, int R, bool P>
struct WParam {
  double w[P ? Geo<D, R>::WCOUNT : 1];
};

template <int D, int R>
struct Cfg64 {
  using T = Tile<D, R>;
  static constexpr int kThreads = (D == 3 && R == 3) ? 128 : T::THREADS;
};

// Pressure of a conservative state.
__device__ __forceinline__ double pressure_of(const double* u, int D, double gm1) {
  double m2 = 0.0;
  for (int k = 0; k < D; ++k) m2 = fma(u[1 + k], u[1 + k], m2);
  return gm1 * (u[D + 1] - 0.5 * m2 / u[0]);
}

// p(u) >= pmin, for rho > 0, evaluated without a division: gm1 (E rho - |m|^2/2) >= pmin rho
template <int D>
__device__ __forceinline__ bool p_at_least(const double* u, double gm1, double pmin) {
  double m2 = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) m2 = fma(u[1 + k], u[1 + k], m2);
  return gm1 * fma(u[D + 1], u[0], -0.5 * m2) >= pmin * u[0];
}

// Riemann states of one cell.  g (the stencil in reconstruction variables) is
// staged per thread in shared memory, gs[l * kThreads].  FP64 arithmetic is the
// bottleneck here (2 DFMA/clk/SM), so the loops stay rolled and read their
// indices from constant memory.
template <int D, int R, bool LINEAR, class WF>
__device__ __forceinline__ void recon_cell(const GridArgs& a, const WF& W, const double* __restrict__ sm, int c,
                                           double* __restrict__ gs, double* __restrict__ faces, long long cell,
                                           long long ncell) {
  using G = Geo<D, R>;
  using T = Tile<D, R>;
  constexpr int NV = G::NV, N0 = G::N0, NQ = G::NQ, F = G::F, M = G::M, SN = T::SN;
  constexpr int TS = Cfg64<D, R>::kThreads;
  const Plan<D, R>& P = c_plan<D, R>;
  const double gm1 = a.gamma - 1.0;

  if constexpr (LINEAR) {
    // unlimited linear S0 reconstruction of the conservative variables
    for (int v = 0; v < NV; ++v) {
      const double* s = sm + v * SN + c;
      for (int sp = 0; sp < F; ++sp) {
        double acc = 0.0;
        for (int l = 0; l < N0; ++l) acc = fma(W(sp * N0 + l), s[P.delta[l]], acc);
        faces[((long long)sp * NV + v) * ncell + cell] = acc;
      }
    }
  } else {
    const double rt = sm[c];
    double ut[3] = {0.0, 0.0, 0.0}, kin = 0.0;
    const double irt = 1.0 / rt;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      ut[k] = sm[(1 + k) * SN + c] * irt;
      kin = fma(ut[k], ut[k], kin);
    }
    kin *= 0.5;
    double wrho[F], eacc[F];
#pragma unroll 1
    for (int v = 0; v < NV; ++v) {
      // velocity component of this row (uniform across the warp)
      const double uv = (v == 1) ? ut[0] : (v == 2 ? ut[1] : (v == 3 && D == 3 ? ut[2] : 0.0));
      // ---- g = row v of Phi applied to every stencil cell (Eq. 33) ----
#pragma unroll 4
      for (int l = 0; l < N0; ++l) {
        const int o = c + P.delta[l];
        double val;
        if (v == 0) {
          val = sm[o];
        } else if (v <= D) {
          val = fma(-uv, sm[o], sm[v * SN + o]) * irt;
        } else {
          double t = fma(kin, sm[o], sm[(D + 1) * SN + o]);
#pragma unroll
          for (int k = 0; k < D; ++k) t = fma(-ut[k], sm[(1 + k) * SN + o], t);
          val = gm1 * t;
        }
        gs[l * TS] = val;
      }
      // ---- smoothness indicators (Eq. 22) and nonlinear weights (Eqs. 24, 25) ----
      double om[NQ], sum = 0.0;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int nq = P.len[q], base = P.woff[q] + F * nq;
        const int* idx = P.idx + P.start[q];
        double b = 0.0;
#pragma unroll 1
        for (int m = 0; m < M; ++m) {
          double d = 0.0;
#pragma unroll 4
          for (int j = 0; j < nq; ++j) d = fma(W(base + m * nq + j), gs[idx[j] * TS], d);
          b = fma(d, d, b);
        }
        om[q] = linear_weight<D>(q) / fma(b, b, a.eps);
        sum += om[q];
      }
      // ---- WENO-AO coefficients (Eq. 19) ----
      double coef[NQ];
      {
        const double inv = 1.0 / sum;
        const double w0 = om[0] * inv;
        coef[0] = w0 / linear_weight<D>(0);
#pragma unroll
        for (int q = 1; q < NQ; ++q) coef[q] = om[q] * inv - w0 * (linear_weight<D>(q) / linear_weight<D>(0));
      }
      // ---- face values and the back transform, accumulated variable by variable ----
#pragma unroll 1
      for (int sp = 0; sp < F; ++sp) {
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int nq = P.len[q], base = P.woff[q] + sp * nq;
          const int* idx = P.idx + P.start[q];
          double val = 0.0;
#pragma unroll 4
          for (int j = 0; j < nq; ++j) val = fma(W(base + j), gs[idx[j] * TS], val);
          acc = fma(coef[q], val, acc);
        }
        // Phi^{-1}: rho = w_rho; m_k = u_k w_rho + rho w_uk; E = kin w_rho + rho u.w_u + w_p/(gamma-1)
        double out;
        if (v == 0) {
          wrho[sp] = acc;
          eacc[sp] = kin * acc;
          out = acc;
        } else if (v <= D) {
          out = fma(uv, wrho[sp], rt * acc);
          eacc[sp] = fma(rt * uv, acc, eacc[sp]);
        } else {
          out = fma(acc, 1.0 / gm1, eacc[sp]);
        }
        faces[((long long)sp * NV + v) * ncell + cell] = out;
      }
    }
  }
}

// Characteristic variables of direction dir at the reference state ut (conservative; Sec. 3.4.1):
// the flux Jacobian A = R Lambda L of that direction, Phi = L (rows: left eigenvectors) and
// Phi^{-1} = R (columns: right eigenvectors).  Waves u_n - c, entropy, the shear waves of the
// tangential axes in increasing order, u_n + c; b1 = (gamma-1)/c^2, b2 = b1 |u|^2/2, H = (E+p)/rho.
template <int D>
__device__ __forceinline__ void char_matrices(const double* ut, double gamma, int dir, double (&L)[D + 2][D + 2],
                                              double (&Rm)[D + 2][D + 2]) {
  constexpr int NV = D + 2;
  const double rho = ut[0], irho = 1.0 / rho;
  double u[3] = {0.0, 0.0, 0.0}, q2 = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    u[k] = ut[1 + k] * irho;
    q2 = fma(u[k], u[k], q2);
  }
  const double p = (gamma - 1.0) * fma(-0.5 * rho, q2, ut[NV - 1]);
  const double c = sqrt(gamma * p * irho), ic = 1.0 / c, H = (ut[NV - 1] + p) * irho;
  const double b1 = (gamma - 1.0) * ic * ic, b2 = 0.5 * b1 * q2, un = u[dir];
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int j = 0; j < NV; ++j) L[i][j] = Rm[i][j] = 0.0;
  Rm[0][0] = Rm[0][1] = Rm[0][NV - 1] = 1.0;
  L[0][0] = 0.5 * (b2 + un * ic);
  L[1][0] = 1.0 - b2;
  L[NV - 1][0] = 0.5 * (b2 - un * ic);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double nk = (k == dir) ? 1.0 : 0.0;
    Rm[1 + k][0] = u[k] - c * nk;
    Rm[1 + k][1] = u[k];
    Rm[1 + k][NV - 1] = u[k] + c * nk;
    L[0][1 + k] = 0.5 * (-b1 * u[k] - nk * ic);
    L[1][1 + k] = b1 * u[k];
    L[NV - 1][1 + k] = 0.5 * (-b1 * u[k] + nk * ic);
  }
  Rm[NV - 1][0] = H - c * un;
  Rm[NV - 1][1] = 0.5 * q2;
  Rm[NV - 1][NV - 1] = H + c * un;
  L[0][NV - 1] = 0.5 * b1;
  L[1][NV - 1] = -b1;
  L[NV - 1][NV - 1] = 0.5 * b1;
  int w = 2;
#pragma unroll
  for (int t = 0; t < D; ++t) {
    if (t == dir) continue;
    Rm[1 + t][w] = 1.0;
    Rm[NV - 1][w] = u[t];
    L[w][0] = -u[t];
    L[w][1 + t] = 1.0;
    ++w;
  }
}

// WENO-AO Riemann states of one cell in characteristic variables (Sec. 3.4.1): for each direction,
// the stencil in that direction's characteristic variables, smoothness indicators and nonlinear
// weights per characteristic component (Eqs. 22, 24, 25), the WENO-AO values (Eq. 19) at the Gauss
// points of the two faces normal to it only, and the back transform with R.  The weights are
// computed once per direction: d times the work of the linearized primitive variables.
template <int D, int R, class WF>
__device__ __forceinline__ void recon_cell_char(const GridArgs& a, const WF& W, const double* __restrict__ sm, int c,
                                                double* __restrict__ gs, double* __restrict__ faces, long long cell,
                                                long long ncell) {
  using G = Geo<D, R>;
  using T = Tile<D, R>;
  constexpr int NV = G::NV, NQ = G::NQ, F = G::F, M = G::M, NT = G::NT, SN = T::SN;
  constexpr int TS = Cfg64<D, R>::kThreads;
  const Plan<D, R>& P = c_plan<D, R>;
  double ut[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) ut[v] = sm[v * SN + c];
#pragma unroll 1
  for (int dir = 0; dir < D; ++dir) {
    double L[NV][NV], Rm[NV][NV];
    char_matrices<D>(ut, a.gamma, dir, L, Rm);
    double wv[2 * NT][NV];  // characteristic values at this direction's face points
#pragma unroll 1
    for (int v = 0; v < NV; ++v) {
      // ---- g = row v of L applied to every stencil cell ----
#pragma unroll 4
      for (int l = 0; l < G::N0; ++l) {
        const int o = c + P.delta[l];
        double val = 0.0;
#pragma unroll
        for (int j = 0; j < NV; ++j) val = fma(L[v][j], sm[j * SN + o], val);
        gs[l * TS] = val;
      }
      // ---- smoothness indicators and nonlinear weights of this component ----
      double om[NQ], sum = 0.0;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int nq = P.len[q], base = P.woff[q] + F * nq;
        const int* idx = P.idx + P.start[q];
        double b = 0.0;
#pragma unroll 1
        for (int m = 0; m < M; ++m) {
          double d = 0.0;
#pragma unroll 4
          for (int j = 0; j < nq; ++j) d = fma(W(base + m * nq + j), gs[idx[j] * TS], d);
          b = fma(d, d, b);
        }
        om[q] = linear_weight<D>(q) / fma(b, b, a.eps);
        sum += om[q];
      }
      double coef[NQ];
      {
        const double inv = 1.0 / sum;
        const double w0 = om[0] * inv;
        coef[0] = w0 / linear_weight<D>(0);
#pragma unroll
        for (int q = 1; q < NQ; ++q) coef[q] = om[q] * inv - w0 * (linear_weight<D>(q) / linear_weight<D>(0));
      }
      // ---- WENO-AO values at the Gauss points of the faces normal to dir ----
#pragma unroll 1
      for (int k = 0; k < 2 * NT; ++k) {
        const int sp = 2 * dir * NT + k;
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int nq = P.len[q], base = P.woff[q] + sp * nq;
          const int* idx = P.idx + P.start[q];
          double val = 0.0;
#pragma unroll 4
          for (int j = 0; j < nq; ++j) val = fma(W(base + j), gs[idx[j] * TS], val);
          acc = fma(coef[q], val, acc);
        }
        wv[k][v] = acc;
      }
    }
    // ---- back to conservative variables, u_s = R w_s ----
#pragma unroll 1
    for (int k = 0; k < 2 * NT; ++k) {
      const int sp = 2 * dir * NT + k;
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        double out = 0.0;
#pragma unroll
        for (int v = 0; v < NV; ++v) out = fma(Rm[j][v], wv[k][v], out);
        faces[((long long)sp * NV + j) * ncell + cell] = out;
      }
    }
  }
}

// Positivity-preserving limiter of Sec. 4 on the F Riemann states of one cell.
template <int D, int R>
__device__ __forceinline__ void limit_cell(const GridArgs& a, const double* __restrict__ sm,
                                           const double* __restrict__ sp_tile, int c, double* __restrict__ faces,
                                           long long cell, long long ncell) {
  using G = Geo<D, R>;
  using T = Tile<D, R>;
  constexpr int NV = G::NV, F = G::F, SN = T::SN;
  const double gm1 = a.gamma - 1.0;
  double ut[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) ut[v] = sm[v * SN + c];
  double rmax = -1e300, rmin = 1e300, pmin = 1e300;
#pragma unroll
  for (int k = (D == 3 ? -1 : 0); k <= (D == 3 ? 1 : 0); ++k)
#pragma unroll
    for (int j = -1; j <= 1; ++j)
#pragma unroll
      for (int i = -1; i <= 1; ++i) {
        const int o = c + i + T::SX * (j + T::SY * k);
        rmax = fmax(rmax, sm[o]);
        rmin = fmin(rmin, sm[o]);
        pmin = fmin(pmin, sp_tile[o]);
      }
  const double lo_f = 1.0 - a.kappa + a.kappa * a.eta, hi_f = 1.0 + a.kappa - a.kappa * a.eta;
  const double rho_max = rmax * hi_f, rho_min = rmin * lo_f, p_min = pmin * lo_f;
  double th = 1.0;
#pragma unroll
  for (int s = 0; s < F; ++s) {
    const double rs = faces[((long long)s * NV) * ncell + cell];
    if (rs < rho_min) th = fmin(th, (ut[0] - rho_min) / (ut[0] - rs));
    if (rs > rho_max) th = fmin(th, (rho_max - ut[0]) / (rs - ut[0]));
  }
  double thp = 1.0;
#pragma unroll 1
  for (int s = 0; s < F; ++s) {
    double u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double f = faces[((long long)s * NV + v) * ncell + cell];
      u[v] = th < 1.0 ? ut[v] + th * (f - ut[v]) : f;
    }
    if (p_at_least<D>(u, gm1, p_min)) continue;
    double lo = 0.0, hi = 1.0;
#pragma unroll 1
    for (int it = 0; it < 60; ++it) {
      const double mid = 0.5 * (lo + hi);
      double t[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) t[v] = ut[v] + mid * (u[v] - ut[v]);
      if (p_at_least<D>(t, gm1, p_min))
        lo = mid;
      else
        hi = mid;
    }
    thp = fmin(thp, lo);
  }
  if (th < 1.0 || thp < 1.0) {
#pragma unroll 1
    for (int s = 0; s < F; ++s)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        double* f = faces + ((long long)s * NV + v) * ncell + cell;
        double u = *f;
        if (th < 1.0) u = ut[v] + th * (u - ut[v]);
        if (thp < 1.0) u = ut[v] + thp * (u - ut[v]);
        *f = u;
      }
  }
}

template <int D, int R, bool P>
struct WFun {
  const double* __restrict__ g;
  const WParam<D, R, P>& p;
  __device__ __forceinline__ double operator()(int i) const {
    if constexpr (P)
      return p.w[i];
    else
      return __ldg(g + i);
  }
};

// CHAR: WENO-AO cells in characteristic variables (a separate instantiation, so that the
// linearized-primitive kernel keeps its register allocation)
template <int D, int R, bool P, bool CHAR>
__global__ void __launch_bounds__(Cfg64<D, R>::kThreads) recon64_kernel(GridArgs a, int mode,
                                                                        const double* __restrict__ U,
                                                                        double* __restrict__ faces,
                                                                        const unsigned char* __restrict__ gate_mask,
                                                                        const double* __restrict__ wglob,
                                                                        const __grid_constant__ WParam<D, R, P> wpar) {
  using G = Geo<D, R>;
  using T = Tile<D, R>;
  constexpr int NV = G::NV, SN = T::SN, TS = Cfg64<D, R>::kThreads;
  extern __shared__ double smem[];
  double* sm = smem;            // [NV][SN] cell averages
  double* sp = smem + NV * SN;  // [SN] cell-average pressures
  double* gs = sp + SN;         // [N0][TS] per-thread stencil in reconstruction variables
  const long long ncell = (long long)a.n[0] * a.n[1] * a.n[2];
  const double gm1 = a.gamma - 1.0;

  const int tiles_x = (a.n[0] + T::TX - 1) / T::TX, tiles_y = (a.n[1] + T::TY - 1) / T::TY;
  int b = blockIdx.x;
  const int bx = b % tiles_x;
  b /= tiles_x;
  const int by = b % tiles_y;
  const int bz = b / tiles_y;
  const int x0 = bx * T::TX - T::H, y0 = by * T::TY - T::H, z0 = (D == 3) ? a.zf_first + bz * T::TZ - T::H : 0;
  const int tid = threadIdx.x;
  const long long ncell_f = face_ncell(a);

  for (int i = tid; i < SN; i += TS) {
    const int sx = i % T::SX, sy = (i / T::SX) % T::SY, sz = i / (T::SX * T::SY);
    const int gx = map_index(x0 + sx, a.n[0], a.bc[0][0], a.bc[0][1]);
    const int gy = map_index(y0 + sy, a.n[1], a.bc[1][0], a.bc[1][1]);
    const int gz = (D == 3) ? map_index(z0 + sz, a.n[2], a.bc[2][0], a.bc[2][1]) : 0;
    const long long gc = ((long long)gz * a.n[1] + gy) * a.n[0] + gx;
    double u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      u[v] = U[v * ncell + gc];
      sm[v * SN + i] = u[v];
    }
    sp[i] = pressure_of(u, D, gm1);
  }
  __syncthreads();

  const WFun<D, R, P> W{wglob, wpar};
  for (int lc = tid; lc < T::THREADS; lc += TS) {
    const int lx = lc % T::TX, ly = (lc / T::TX) % T::TY, lz = lc / (T::TX * T::TY);
    const int x = bx * T::TX + lx, y = by * T::TY + ly, l = (D == 3) ? bz * T::TZ + lz : 0;
    if (x >= a.n[0] || y >= a.n[1] || l >= a.zf_count) continue;
    const int z = (D == 3) ? slab_plane(a, l) : 0;
    if (z < 0) continue;
    const int c = (lx + T::H) + T::SX * ((ly + T::H) + T::SY * (D == 3 ? lz + T::H : 0));
    const long long cell = ((long long)z * a.n[1] + y) * a.n[0] + x;
    const long long fc = ((long long)l * a.n[1] + y) * a.n[0] + x;
    if (!(sm[c] > 0.0) || !(sp[c] > 0.0)) raise_flag(a.status, kFlagNonphysical);
    const bool linear = (mode == 1) || (mode >= 2 && gate_mask[cell]);
    if (linear)
      recon_cell<D, R, true>(a, W, sm, c, gs + tid, faces, fc, ncell_f);
    else if constexpr (CHAR)
      recon_cell_char<D, R>(a, W, sm, c, gs + tid, faces, fc, ncell_f);
    else
      recon_cell<D, R, false>(a, W, sm, c, gs + tid, faces, fc, ncell_f);
    if (a.positivity) limit_cell<D, R>(a, sm, sp, c, faces, fc, ncell_f);
  }
}

template <int D, int R>
cudaError_t launch_dr(kfvm_ctx* ctx, const double* U, double* faces, cudaStream_t st, int zf_first, int zf_count) {
  using T = Tile<D, R>;
  constexpr bool P = params_fit<D, R>();
  constexpr int TS = Cfg64<D, R>::kThreads;
  static bool plan_ready[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !plan_ready[dev]) {
    const Plan<D, R> plan = make_plan<D, R>();
    cudaError_t e = cudaMemcpyToSymbol(c_plan<D, R>, &plan, sizeof(plan));
    if (e != cudaSuccess) return e;
    plan_ready[dev] = true;
  }
  GridArgs a = make_grid_args(ctx);
  a.zf_first = zf_first;
  a.zf_count = zf_count;
  const int tiles = ((ctx->n[0] + T::TX - 1) / T::TX) * ((ctx->n[1] + T::TY - 1) / T::TY) *
                    ((D == 3) ? (zf_count + T::TZ - 1) / T::TZ : 1);
  const size_t smem = sizeof(double) * ((Geo<D, R>::NV + 1) * T::SN + Geo<D, R>::N0 * TS);
  auto kern = ctx->vars == 1 ? recon64_kernel<D, R, P, true> : recon64_kernel<D, R, P, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  std::unique_ptr<WParam<D, R, P>> wp(new WParam<D, R, P>);  // host staging of the parameter copy
  if constexpr (P)
    for (int i = 0; i < Geo<D, R>::WCOUNT; ++i) wp->w[i] = ctx->w_host[i];
  else
    wp->w[0] = 0.0;
  kern<<<tiles, TS, smem, st>>>(a, kernel_recon_mode(ctx), U, faces, ctx->d_gate_mask, ctx->d_w64, *wp);
  ctx->launches += 1;
  return cudaGetLastError();
}

}  // namespace r64
}  // namespace kfvm
