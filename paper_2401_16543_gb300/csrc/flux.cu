// flux.cu -- Riemann solves, flux divergence, SSP-RK3 stage update and the
// CFL time step (Sec. 5.3 steps 4-6, Sec. 5.4).
//
//   max_rate_kernel   dt = cfl / max_cells sum_d (|u_d| + c)/Delta_d clipped to
//                     the time left: warp shuffles, one atomicMax per CTA on
//                     the ordered bits of the (non-negative) rate, and the
//                     last CTA to arrive (arrival counter, no waiting) writes
//                     dt and re-arms the reduction.  In the FP32 mode it also
//                     writes the float32 shadow of the state.
//   face_flux_kernel  one thread per face of one direction: the Riemann states
//                     on both sides at the R^(d-1) Gauss points (outflow:
//                     the exterior state copies the interior one; periodic:
//                     the wrapped neighbour), HLLC (Toro) or HLL with Batten
//                     wave speeds (Roe-averaged u and c), Gauss-Legendre
//                     average over the face.
//   update_kernel     L = -sum_d (F_{d,+} - F_{d,-})/Delta_d and the Shu-Osher
//                     stage combination in float64.
//   flux_update_kernel  the hot path's fusion of the two: a CTA computes every
//                     face flux of its tile once into shared memory, then the
//                     divergence and the stage update of its cells.
// The face-flux buffer kernels serve kfvm_flux_static.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

namespace kfvm {
namespace {

constexpr int kBlock = 256;

// ---------------------------------------------------------------------------
// CFL rate reduction and dt
// ---------------------------------------------------------------------------
template <int D, bool SHADOW>
__global__ void __launch_bounds__(kBlock) max_rate_kernel(GridArgs a, const double* __restrict__ U,
                                                          float* __restrict__ shadow, double cfl, double t_rem) {
  const long long ncell = (long long)a.n[0] * a.n[1] * a.n[2];
  const double gm1 = a.gamma - 1.0;
  double best = 0.0;
  for (long long c = blockIdx.x * (long long)kBlock + threadIdx.x; c < ncell; c += (long long)gridDim.x * kBlock) {
    double u[D + 2];
#pragma unroll
    for (int v = 0; v < D + 2; ++v) {
      u[v] = U[v * ncell + c];
      if (SHADOW) shadow[v * ncell + c] = (float)u[v];
    }
    double rate;
    if constexpr (SHADOW) {
      // mixed-precision path: float32 where E/p < 8; the pressure is recovered in float64 only
      // where E - |m|^2/(2 rho) cancels (high Mach numbers, near vacuum)
      float uf[D + 2];
#pragma unroll
      for (int v = 0; v < D + 2; ++v) uf[v] = (float)u[v];
      const float irf = __frcp_rn(uf[0]);
      float m2f = 0.0f;
#pragma unroll
      for (int k = 0; k < D; ++k) m2f = fmaf(uf[1 + k], uf[1 + k], m2f);
      float pf = (float)gm1 * fmaf(-0.5f * m2f, irf, uf[D + 1]);
      if (!(pf > 0.125f * uf[D + 1])) {
        const double ir = recip64(u[0]);
        double m2 = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) m2 = fma(u[1 + k], u[1 + k], m2);
        const double p = gm1 * fma(-0.5 * m2, ir, u[D + 1]);
        pf = (p > 0.0 && u[0] > 0.0) ? (float)p : __int_as_float(0x7fc00000);
      }
      const float cs = sqrtf(a.gammaf * pf * irf);
      float r = 0.0f;
#pragma unroll
      for (int k = 0; k < D; ++k) r += (fabsf(uf[1 + k] * irf) + cs) * a.idxf[k];
      rate = (double)r;
    } else {
      const double ir = 1.0 / u[0];
      double m2 = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) m2 = fma(u[1 + k], u[1 + k], m2);
      const double p = gm1 * (u[D + 1] - 0.5 * m2 * ir);
      const double cs = sqrt(a.gamma * p * ir);
      rate = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) rate += (fabs(u[1 + k] * ir) + cs) / a.dx[k];
    }
    if (!(rate <= best)) best = rate;  // NaN propagates
  }
  unsigned long long bits = __double_as_longlong(best);
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long ob = __shfl_down_sync(0xffffffffu, bits, o);
    bits = ob > bits ? ob : bits;
  }
  __shared__ unsigned long long s_max[kBlock / 32];
  __shared__ bool s_last;
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = bits;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = s_max[0];
    for (int w = 1; w < kBlock / 32; ++w) m = s_max[w] > m ? s_max[w] : m;
    atomicMax(&a.scalars->rate_bits, m);
    __threadfence();
    const unsigned int done = atomicAdd(&a.scalars->blocks_done, 1u);
    s_last = (done == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    const unsigned long long m = atomicAdd(&a.scalars->rate_bits, 0ull);
    const double rate = __longlong_as_double((long long)m);
    double dt = cfl / rate;
    if (dt > t_rem) dt = t_rem;
    if (!(rate > 0.0) || !(dt > 0.0) || !(dt <= t_rem)) {
      raise_flag(a.status, kFlagNonphysical);
      dt = 0.0;
    }
    a.scalars->dt = dt;
    a.scalars->rate_bits = 0ull;
    a.scalars->blocks_done = 0u;
  }
}

__global__ void shadow_kernel(const double* __restrict__ U, float* __restrict__ S, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    S[i] = (float)U[i];
}

// ---------------------------------------------------------------------------
// Riemann solvers
// ---------------------------------------------------------------------------
// Float64 states are conservative (rho, m, E); float32 states are primitive (rho, u, p).
template <int D>
__device__ __forceinline__ bool riemann64(const double* uL, const double* uR, int dir, double gamma, int solver,
                                          double* f) {
  constexpr int NV = D + 2;
  const double gm1 = gamma - 1.0;
  const double rL = uL[0], rR = uR[0];
  const double irL = 1.0 / rL, irR = 1.0 / rR;
  double vL[D], vR[D], m2L = 0.0, m2R = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    vL[k] = uL[1 + k] * irL;
    vR[k] = uR[1 + k] * irR;
    m2L = fma(uL[1 + k], vL[k], m2L);
    m2R = fma(uR[1 + k], vR[k], m2R);
  }
  const double EL = uL[NV - 1], ER = uR[NV - 1];
  const double pL = gm1 * (EL - 0.5 * m2L), pR = gm1 * (ER - 0.5 * m2R);
  if (!(rL > 0.0) || !(rR > 0.0) || !(pL > 0.0) || !(pR > 0.0)) {
#pragma unroll
    for (int v = 0; v < NV; ++v) f[v] = 0.0;
    return false;
  }
  const double cL = sqrt(gamma * pL * irL), cR = sqrt(gamma * pR * irR);
  const double sL = sqrt(rL), sR = sqrt(rR), isum = 1.0 / (sL + sR);
  double ut2 = 0.0, utn = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double ut = (sL * vL[k] + sR * vR[k]) * isum;
    ut2 = fma(ut, ut, ut2);
    if (k == dir) utn = ut;
  }
  const double HL = (EL + pL) * irL, HR = (ER + pR) * irR;
  const double Ht = (sL * HL + sR * HR) * isum;
  const double ct2 = gm1 * (Ht - 0.5 * ut2);
  const double ct = sqrt(ct2 > 0.0 ? ct2 : 0.0);
  const double unL = vL[dir], unR = vR[dir];
  const double SL = fmin(unL - cL, utn - ct), SR = fmax(unR + cR, utn + ct);
  double FL[NV], FR[NV];
  FL[0] = uL[1 + dir];
  FR[0] = uR[1 + dir];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    FL[1 + k] = uL[1 + k] * unL + (k == dir ? pL : 0.0);
    FR[1 + k] = uR[1 + k] * unR + (k == dir ? pR : 0.0);
  }
  FL[NV - 1] = unL * (EL + pL);
  FR[NV - 1] = unR * (ER + pR);
  if (SL >= 0.0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) f[v] = FL[v];
    return true;
  }
  if (SR <= 0.0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) f[v] = FR[v];
    return true;
  }
  if (solver == 1) {
    const double idn = 1.0 / (SR - SL);
#pragma unroll
    for (int v = 0; v < NV; ++v) f[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (uR[v] - uL[v])) * idn;
    return true;
  }
  const double Ss = (pR - pL + rL * unL * (SL - unL) - rR * unR * (SR - unR)) / (rL * (SL - unL) - rR * (SR - unR));
  const bool left = Ss >= 0.0;
  const double* uK = left ? uL : uR;
  const double* FK = left ? FL : FR;
  const double SK = left ? SL : SR, rK = left ? rL : rR, unK = left ? unL : unR, pK = left ? pL : pR;
  const double irK = left ? irL : irR;
  const double fac = rK * (SK - unK) / (SK - Ss);
  double us[NV];
  us[0] = fac;
#pragma unroll
  for (int k = 0; k < D; ++k) us[1 + k] = fac * (k == dir ? Ss : uK[1 + k] * irK);
  us[NV - 1] = fac * (uK[NV - 1] * irK + (Ss - unK) * (Ss + pK / (rK * (SK - unK))));
#pragma unroll
  for (int v = 0; v < NV; ++v) f[v] = FK[v] + SK * (us[v] - uK[v]);
  return true;
}

// Reciprocal and square root of the FP32 solver.  FAST: single PTX instructions, rcp.approx.f32 (at
// most 1 ulp) and sqrt.approx.f32 (relative error ~2^-23), instead of the IEEE-rounded __frcp_rn /
// sqrtf (a few instructions each and a slow path); the flux/update kernel is partly issue-bound (five
// square roots and four reciprocals per Riemann solve), 2D 1024^2: 0.077 -> 0.069 ms per stage.  Used
// at radius 2 only: the radius-3 linear reconstructions amplify high-wavenumber perturbations weakly
// (a von Neumann symbol with max Re(lambda) dx > 0), and the extra rounding raised the 3D radius-3
// gated path's L1 error on the 32^3 sine translation from ~1.08 to 1.21 times FP64 WENO-AO's.
template <bool FAST>
__device__ __forceinline__ float rcp32(float x) {
  if constexpr (FAST) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  } else {
    return __frcp_rn(x);
  }
}
template <bool FAST>
__device__ __forceinline__ float sqrt32(float x) {
  if constexpr (FAST) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  } else {
    return sqrtf(x);
  }
}

template <int D, bool FAST>
__device__ __forceinline__ bool riemann32(const float* wL, const float* wR, int dir, float gamma, int solver,
                                          float* f) {
  constexpr int NV = D + 2;
  const float gm1 = gamma - 1.0f;
  const float rL = wL[0], rR = wR[0], pL = wL[NV - 1], pR = wR[NV - 1];
  if (!(rL > 0.0f) || !(rR > 0.0f) || !(pL > 0.0f) || !(pR > 0.0f)) {
#pragma unroll
    for (int v = 0; v < NV; ++v) f[v] = 0.0f;
    return false;
  }
  float v2L = 0.0f, v2R = 0.0f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    v2L = fmaf(wL[1 + k], wL[1 + k], v2L);
    v2R = fmaf(wR[1 + k], wR[1 + k], v2R);
  }
  const float igm1 = rcp32<FAST>(gm1);
  const float EL = fmaf(pL, igm1, 0.5f * rL * v2L), ER = fmaf(pR, igm1, 0.5f * rR * v2R);
  const float irL = rcp32<FAST>(rL), irR = rcp32<FAST>(rR);
  const float cL = sqrt32<FAST>(gamma * pL * irL), cR = sqrt32<FAST>(gamma * pR * irR);
  const float sL = sqrt32<FAST>(rL), sR = sqrt32<FAST>(rR), isum = rcp32<FAST>(sL + sR);
  float ut2 = 0.0f, utn = 0.0f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float ut = (sL * wL[1 + k] + sR * wR[1 + k]) * isum;
    ut2 = fmaf(ut, ut, ut2);
    if (k == dir) utn = ut;
  }
  const float HL = (EL + pL) * irL, HR = (ER + pR) * irR;
  const float Ht = (sL * HL + sR * HR) * isum;
  const float ct2 = gm1 * (Ht - 0.5f * ut2);
  const float ct = sqrt32<FAST>(ct2 > 0.0f ? ct2 : 0.0f);
  const float unL = wL[1 + dir], unR = wR[1 + dir];
  const float SL = fminf(unL - cL, utn - ct), SR = fmaxf(unR + cR, utn + ct);
  float UL[NV], UR[NV], FL[NV], FR[NV];
  UL[0] = rL;
  UR[0] = rR;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    UL[1 + k] = rL * wL[1 + k];
    UR[1 + k] = rR * wR[1 + k];
  }
  UL[NV - 1] = EL;
  UR[NV - 1] = ER;
  FL[0] = UL[1 + dir];
  FR[0] = UR[1 + dir];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    FL[1 + k] = UL[1 + k] * unL + (k == dir ? pL : 0.0f);
    FR[1 + k] = UR[1 + k] * unR + (k == dir ? pR : 0.0f);
  }
  FL[NV - 1] = unL * (EL + pL);
  FR[NV - 1] = unR * (ER + pR);
  if (SL >= 0.0f) {
#pragma unroll
    for (int v = 0; v < NV; ++v) f[v] = FL[v];
    return true;
  }
  if (SR <= 0.0f) {
#pragma unroll
    for (int v = 0; v < NV; ++v) f[v] = FR[v];
    return true;
  }
  if (solver == 1) {
    const float idn = rcp32<FAST>(SR - SL);
#pragma unroll
    for (int v = 0; v < NV; ++v) f[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) * idn;
    return true;
  }
  const float Ss = __fdividef(pR - pL + rL * unL * (SL - unL) - rR * unR * (SR - unR), rL * (SL - unL) - rR * (SR - unR));
  const bool left = Ss >= 0.0f;
  const float* uK = left ? UL : UR;
  const float* wK = left ? wL : wR;
  const float* FK = left ? FL : FR;
  const float SK = left ? SL : SR, rK = left ? rL : rR, unK = left ? unL : unR, pK = left ? pL : pR;
  const float fac = __fdividef(rK * (SK - unK), SK - Ss);
  float us[NV];
  us[0] = fac;
#pragma unroll
  for (int k = 0; k < D; ++k) us[1 + k] = fac * (k == dir ? Ss : wK[1 + k]);
  us[NV - 1] = fac * (uK[NV - 1] * (left ? irL : irR) + (Ss - unK) * (Ss + __fdividef(pK, rK * (SK - unK))));
#pragma unroll
  for (int v = 0; v < NV; ++v) f[v] = FK[v] + SK * (us[v] - uK[v]);
  return true;
}

// ---------------------------------------------------------------------------
// Face fluxes
// ---------------------------------------------------------------------------
struct FluxLayout {
  long long off[3];  // start of each direction's block (in elements)
  long long nface[3];
};

// Riemann state of point s of cell `cell`.  Float64 faces: conservative
// [s][v][cell].  Float32 faces: primitive, [s][cell] float4 (rho, u, v, p)
// followed in 3D by the plane [s][cell] of w.
template <int D, int R>
__device__ __forceinline__ void load_face(const double* __restrict__ f, int s, long long cell, long long ncell,
                                          double* u) {
#pragma unroll
  for (int v = 0; v < D + 2; ++v) u[v] = f[((long long)s * (D + 2) + v) * ncell + cell];
}
template <int D, int R>
__device__ __forceinline__ void load_face(const float* __restrict__ f, int s, long long cell, long long ncell,
                                          float* u) {
  constexpr int F = 2 * D * ipow(R, D - 1);
  const float4 q = __ldg(reinterpret_cast<const float4*>(f) + (long long)s * ncell + cell);
  u[0] = q.x;
  u[1] = q.y;
  u[2] = q.z;
  if (D == 3) u[3] = __ldg(f + 4LL * F * ncell + (long long)s * ncell + cell);
  u[D + 1] = q.w;
}

// Face-averaged numerical flux on the face between cell c - e_dir and cell c
// (c[dir] in [0, n_dir]): exterior states at outflow boundaries copy the
// interior one, periodic faces see the wrapped neighbour; R^(d-1) Gauss points.
template <int D, int R, typename Real>
__device__ __forceinline__ bool face_flux_at(const GridArgs& a, const Real* __restrict__ faces, int dir, const int* c,
                                             long long ncell, Real* acc) {
  constexpr int NV = D + 2, NT = ipow(R, D - 1);
  const int nd = a.n[dir];
  const int i = c[dir];
  int cl[3] = {c[0], c[1], c[2]}, cr[3] = {c[0], c[1], c[2]};
  cl[dir] = i - 1;
  cr[dir] = i;
  bool has_l = true, has_r = true;
  if (i == 0) {
    if (a.bc[dir][0] == KFVM_BC_PERIODIC) cl[dir] = nd - 1; else { has_l = false; cl[dir] = 0; }
  }
  if (i == nd) {
    if (a.bc[dir][1] == KFVM_BC_PERIODIC) cr[dir] = 0; else { has_r = false; cr[dir] = nd - 1; }
  }
  // positions in the Riemann-state buffer (which may hold a slab of z-planes)
  const long long lcell = face_cell(a, cl[0], cl[1], cl[2]);
  const long long rcell = face_cell(a, cr[0], cr[1], cr[2]);
  ncell = face_ncell(a);
  constexpr double w2[2] = {0.5, 0.5};
  constexpr double w3[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = Real(0);
  bool ok = true;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int s_hi = (dir * 2 + 1) * NT + t, s_lo = (dir * 2) * NT + t;
    Real uL[NV], uR[NV], fl[NV];
    if (has_l) load_face<D, R>(faces, s_hi, lcell, ncell, uL);
    if (has_r) load_face<D, R>(faces, s_lo, rcell, ncell, uR);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if (!has_l) uL[v] = uR[v];
      if (!has_r) uR[v] = uL[v];
    }
    if constexpr (sizeof(Real) == 8)
      ok &= riemann64<D>(uL, uR, dir, a.gamma, a.riemann, fl);
    else
      ok &= riemann32<D, R == 2>(uL, uR, dir, (float)a.gamma, a.riemann, fl);
    const double wt = (R == 2 ? w2[t % R] : w3[t % R]) * (D == 3 ? (R == 2 ? w2[t / R] : w3[t / R]) : 1.0);
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] += Real(wt) * fl[v];
  }
  return ok;
}

template <int D, int R, typename Real>
__global__ void __launch_bounds__(kBlock) face_flux_kernel(GridArgs a, FluxLayout L, const Real* __restrict__ faces,
                                                           Real* __restrict__ flux) {
  constexpr int NV = D + 2;
  const int dir = blockIdx.y;
  const long long nf = L.nface[dir];
  const long long f = blockIdx.x * (long long)kBlock + threadIdx.x;
  if (f >= nf) return;
  const long long ncell = (long long)a.n[0] * a.n[1] * a.n[2];
  // face coordinates in the grid extended by one along dir
  int e[3] = {a.n[0], a.n[1], a.n[2]};
  e[dir] += 1;
  long long r = f;
  int c[3];
  c[0] = (int)(r % e[0]);
  r /= e[0];
  c[1] = (int)(r % e[1]);
  c[2] = (int)(r / e[1]);
  Real acc[NV];
  if (!face_flux_at<D, R, Real>(a, faces, dir, c, ncell, acc)) raise_flag(a.status, kFlagNonphysical);
#pragma unroll
  for (int v = 0; v < NV; ++v) flux[L.off[dir] + v * nf + f] = acc[v];
}

// ---------------------------------------------------------------------------
// Fused flux divergence and SSP-RK3 stage (the hot-path version): a CTA owns a
// tile of cells, computes every face flux touching the tile exactly once into
// shared memory (the faces, the tile's high faces included, dealt out evenly to
// its threads), then each thread forms L = -sum_d (F_hi - F_lo)/Delta_d for its
// cell and the stage update.
// Float64 faces: L and the update in float64 (the plain path).  Float32 faces:
// L in float32, the stage combination accumulated in float64.
// ---------------------------------------------------------------------------
template <int D>
struct FTile {
  static constexpr int TX = (D == 2) ? 32 : 8, TY = 8, TZ = (D == 2) ? 1 : 4;
  static constexpr int THREADS = TX * TY * TZ;
  static constexpr int NF0 = (TX + 1) * TY * TZ, NF1 = TX * (TY + 1) * TZ, NF2 = (D == 3) ? TX * TY * (TZ + 1) : 0;
  static constexpr int NF = NF0 + NF1 + NF2;
  __host__ __device__ static constexpr int off(int d) { return d == 0 ? 0 : (d == 1 ? NF0 : NF0 + NF1); }
  // faces of direction d, and where direction d starts in the warp-padded order
  // the threads deal them out in
  __host__ __device__ static constexpr int nfd(int d) { return d == 0 ? NF0 : (d == 1 ? NF1 : NF2); }
  __host__ __device__ static constexpr int pad(int n) { return (n + 31) / 32 * 32; }
  __host__ __device__ static constexpr int eoff(int d) {
    return d == 0 ? 0 : (d == 1 ? pad(NF0) : pad(NF0) + pad(NF1));
  }
  static constexpr int NE = pad(NF0) + pad(NF1) + pad(NF2);
  // index of face with local coordinates (x, y, z) in direction d's array
  __device__ static int idx(int d, int x, int y, int z) {
    const int ex = TX + (d == 0), ey = TY + (d == 1);
    return off(d) + x + ex * (y + ey * z);
  }
};

template <int D, int R, typename Real, bool SHADOW>
__global__ void __launch_bounds__(FTile<D>::THREADS, sizeof(Real) == 8 ? 3 : 5) flux_update_kernel(GridArgs a, const Real* __restrict__ faces,
                                                                        int stage, const double* __restrict__ U0,
                                                                        const double* __restrict__ Us,
                                                                        double* __restrict__ out,
                                                                        float* __restrict__ shadow) {
  using T = FTile<D>;
  constexpr int NV = D + 2;
  __shared__ Real sflux[NV][T::NF];
  const long long ncell = (long long)a.n[0] * a.n[1] * a.n[2];
  const int tiles_x = (a.n[0] + T::TX - 1) / T::TX, tiles_y = (a.n[1] + T::TY - 1) / T::TY;
  int b = blockIdx.x;
  const int bx = b % tiles_x;
  b /= tiles_x;
  const int by = b % tiles_y;
  const int bz = b / tiles_y;
  const int tid = threadIdx.x;
  const int l[3] = {tid % T::TX, (tid / T::TX) % T::TY, tid / (T::TX * T::TY)};
  const int c[3] = {bx * T::TX + l[0], by * T::TY + l[1], (D == 3) ? a.zc_lo + bz * T::TZ + l[2] : 0};
  const bool active = c[0] < a.n[0] && c[1] < a.n[1] && c[2] < (D == 3 ? a.zc_hi : 1);
  const int last[3] = {a.n[0] - 1, a.n[1] - 1, (D == 3 ? a.zc_hi : 1) - 1};
  // Every face flux touching the tile, each once.  The faces are dealt out in
  // direction blocks padded to whole warps, so a warp works on one direction and
  // the CTA's threads share the tile's faces evenly (a tile has more faces than
  // cells: its high faces along each direction).
  {
    bool ok = true;
    const int org[3] = {bx * T::TX, by * T::TY, (D == 3) ? a.zc_lo + bz * T::TZ : 0};
    for (int e = tid; e < T::NE; e += T::THREADS) {
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int j = e - T::eoff(d);
        const int ex = T::TX + (d == 0), ey = T::TY + (d == 1);
        if (j >= 0 && j < T::nfd(d)) {
          int fc[3] = {org[0] + j % ex, org[1] + (j / ex) % ey, org[2] + j / (ex * ey)};
          bool need = true;
#pragma unroll
          for (int k = 0; k < 3; ++k) need &= fc[k] <= last[k] + (k == d);
          if (need) {
            Real f[NV];
            ok &= face_flux_at<D, R, Real>(a, faces, d, fc, ncell, f);
#pragma unroll
            for (int v = 0; v < NV; ++v) sflux[v][T::off(d) + j] = f[v];
          }
        }
      }
    }
    if (!ok) raise_flag(a.status, kFlagNonphysical);
  }
  __syncthreads();
  if (!active) return;
  const long long cidx = ((long long)c[2] * a.n[1] + c[1]) * a.n[0] + c[0];
  Real Lv[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Lv[v] = Real(0);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    int lh[3] = {l[0], l[1], l[2]};
    lh[d] += 1;
    const int ilo = T::idx(d, l[0], l[1], l[2]), ihi = T::idx(d, lh[0], lh[1], lh[2]);
    const Real idx = sizeof(Real) == 8 ? Real(a.idx[d]) : Real(a.idxf[d]);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Lv[v] = fma(sflux[v][ilo], idx, Lv[v]);
      Lv[v] = fma(-sflux[v][ihi], idx, Lv[v]);
    }
  }
  if (stage == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v * ncell + cidx] = (double)Lv[v];
    return;
  }
  const double dt = a.scalars->dt;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const long long i = v * ncell + cidx;
    double res;
    if constexpr (sizeof(Real) == 8) {
      if (stage == 1) res = fma(dt, Lv[v], U0[i]);
      else if (stage == 2) res = 0.75 * U0[i] + 0.25 * fma(dt, Lv[v], Us[i]);
      else res = (1.0 / 3.0) * U0[i] + (2.0 / 3.0) * fma(dt, Lv[v], Us[i]);
    } else {
      // increment dt*L formed in float32, accumulated in float64
      const double inc = (double)((float)dt * Lv[v]);
      if (stage == 1) res = U0[i] + inc;
      else if (stage == 2) res = fma(0.75, U0[i], 0.25 * (Us[i] + inc));
      else res = fma(1.0 / 3.0, U0[i], (2.0 / 3.0) * (Us[i] + inc));
    }
    out[i] = res;
    if (SHADOW) shadow[i] = (float)res;
  }
}

// ---------------------------------------------------------------------------
// Flux divergence and the SSP-RK3 stages
// ---------------------------------------------------------------------------
template <int D, typename Real, bool SHADOW>
__global__ void __launch_bounds__(kBlock) update_kernel(GridArgs a, FluxLayout L, const Real* __restrict__ flux,
                                                        int stage, const double* __restrict__ U0,
                                                        const double* __restrict__ Us, double* __restrict__ out,
                                                        float* __restrict__ shadow) {
  constexpr int NV = D + 2;
  const long long ncell = (long long)a.n[0] * a.n[1] * a.n[2];
  const long long cidx = blockIdx.x * (long long)kBlock + threadIdx.x;
  if (cidx >= ncell) return;
  long long r = cidx;
  int c[3];
  c[0] = (int)(r % a.n[0]);
  r /= a.n[0];
  c[1] = (int)(r % a.n[1]);
  c[2] = (int)(r / a.n[1]);
  double Lv[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Lv[v] = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    int e[3] = {a.n[0], a.n[1], a.n[2]};
    e[d] += 1;
    const long long flo = ((long long)c[2] * e[1] + c[1]) * e[0] + c[0];
    const long long stride = d == 0 ? 1 : (d == 1 ? e[0] : (long long)e[0] * e[1]);
    const long long fhi = flo + stride;
    const long long nf = L.nface[d];
    const double idx = a.idx[d];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double lo = (double)flux[L.off[d] + v * nf + flo];
      const double hi = (double)flux[L.off[d] + v * nf + fhi];
      Lv[v] = fma(lo, idx, Lv[v]);
      Lv[v] = fma(-hi, idx, Lv[v]);
    }
  }
  if (stage == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v * ncell + cidx] = Lv[v];
    return;
  }
  const double dt = a.scalars->dt;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const long long i = v * ncell + cidx;
    double res;
    if (stage == 1) {
      res = fma(dt, Lv[v], U0[i]);
    } else if (stage == 2) {
      res = 0.75 * U0[i] + 0.25 * fma(dt, Lv[v], Us[i]);
    } else {
      res = (1.0 / 3.0) * U0[i] + (2.0 / 3.0) * fma(dt, Lv[v], Us[i]);
    }
    out[i] = res;
    if (SHADOW) shadow[i] = (float)res;
  }
}

FluxLayout flux_layout(const kfvm_ctx* ctx) {
  FluxLayout L{};
  for (int d = 0; d < 3; ++d) {
    L.off[d] = (long long)ctx->flux_off[d];
    L.nface[d] = d < ctx->dims ? (long long)(ctx->n[d] + 1) * (ctx->ncell / ctx->n[d]) : 0;
  }
  return L;
}

template <int D, int R>
cudaError_t face_flux_dr(kfvm_ctx* ctx, const void* faces, cudaStream_t st) {
  const GridArgs a = make_grid_args(ctx);
  const FluxLayout L = flux_layout(ctx);
  long long mx = 0;
  for (int d = 0; d < D; ++d) mx = L.nface[d] > mx ? L.nface[d] : mx;
  dim3 grid((unsigned)((mx + kBlock - 1) / kBlock), D);
  if (ctx->precision == 64)
    face_flux_kernel<D, R, double><<<grid, kBlock, 0, st>>>(a, L, (const double*)faces, ctx->d_flux);
  else
    face_flux_kernel<D, R, float><<<grid, kBlock, 0, st>>>(a, L, (const float*)faces, (float*)ctx->d_flux);
  ctx->launches += 1;
  return cudaGetLastError();
}

template <int D, int R>
cudaError_t flux_update_dr(kfvm_ctx* ctx, int stage, const void* faces, const double* U0, const double* Us,
                           double* out, cudaStream_t st, float* shadow_out, int zc_lo, int zc_hi, int zf_first,
                           int zf_count) {
  using T = FTile<D>;
  GridArgs a = make_grid_args(ctx);
  if (D == 3 && zc_hi > 0) {
    a.zc_lo = zc_lo;
    a.zc_hi = zc_hi;
    a.zf_first = zf_first;
    a.zf_count = zf_count;
  }
  const unsigned tiles = (unsigned)(((ctx->n[0] + T::TX - 1) / T::TX) * ((ctx->n[1] + T::TY - 1) / T::TY) *
                                    ((D == 3) ? (a.zc_hi - a.zc_lo + T::TZ - 1) / T::TZ : 1));
  const bool shadow = ctx->precision == 32 && stage >= 1 && stage <= 2;
  if (!shadow_out) shadow_out = ctx->d_shadow;
  if (ctx->precision == 64)
    flux_update_kernel<D, R, double, false><<<tiles, T::THREADS, 0, st>>>(a, (const double*)faces, stage, U0, Us, out,
                                                                         nullptr);
  else if (shadow)
    flux_update_kernel<D, R, float, true><<<tiles, T::THREADS, 0, st>>>(a, (const float*)faces, stage, U0, Us, out,
                                                                       shadow_out);
  else
    flux_update_kernel<D, R, float, false><<<tiles, T::THREADS, 0, st>>>(a, (const float*)faces, stage, U0, Us, out,
                                                                        nullptr);
  ctx->launches += 1;
  return cudaGetLastError();
}

template <int D>
cudaError_t update_d(kfvm_ctx* ctx, int stage, const double* U0, const double* Us, double* out, cudaStream_t st) {
  const GridArgs a = make_grid_args(ctx);
  const FluxLayout L = flux_layout(ctx);
  const unsigned blocks = (unsigned)((ctx->ncell + kBlock - 1) / kBlock);
  const bool shadow = ctx->precision == 32 && stage >= 1 && stage <= 2;
  if (ctx->precision == 64)
    update_kernel<D, double, false><<<blocks, kBlock, 0, st>>>(a, L, ctx->d_flux, stage, U0, Us, out, nullptr);
  else if (shadow)
    update_kernel<D, float, true><<<blocks, kBlock, 0, st>>>(a, L, (const float*)ctx->d_flux, stage, U0, Us, out,
                                                             ctx->d_shadow);
  else
    update_kernel<D, float, false><<<blocks, kBlock, 0, st>>>(a, L, (const float*)ctx->d_flux, stage, U0, Us, out,
                                                              nullptr);
  ctx->launches += 1;
  return cudaGetLastError();
}

// register-only multiply-add loop for the FMA peak measurement
template <typename T>
__global__ void fma_loop(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
      x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T>
cudaError_t fma_peak_t(double* flops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = sms * 4, threads = 256, iters = sizeof(T) == 8 ? 2000 : 40000;
  T* out = nullptr;
  e = cudaMalloc(&out, sizeof(T) * blocks * threads);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_loop<T><<<blocks, threads>>>(out, iters / 10, (T)0.999, (T)0.001);
  cudaEventRecord(e0);
  fma_loop<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);
  cudaEventRecord(e1);
  e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  *flops = 2.0 * 8 * 16 * (double)iters * blocks * threads / (ms * 1e-3);
  return e;
}

}  // namespace

cudaError_t launch_max_rate(kfvm_ctx* ctx, const double* U, double cfl, double t_rem, cudaStream_t st) {
  const GridArgs a = make_grid_args(ctx);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long want = (ctx->ncell + kBlock - 1) / kBlock;
  unsigned blocks = (unsigned)(want < 8LL * sms ? want : 8LL * sms);
  if (blocks == 0) blocks = 1;
  const bool sh = ctx->precision == 32;
  if (ctx->dims == 2) {
    if (sh) max_rate_kernel<2, true><<<blocks, kBlock, 0, st>>>(a, U, ctx->d_shadow, cfl, t_rem);
    else max_rate_kernel<2, false><<<blocks, kBlock, 0, st>>>(a, U, nullptr, cfl, t_rem);
  } else {
    if (sh) max_rate_kernel<3, true><<<blocks, kBlock, 0, st>>>(a, U, ctx->d_shadow, cfl, t_rem);
    else max_rate_kernel<3, false><<<blocks, kBlock, 0, st>>>(a, U, nullptr, cfl, t_rem);
  }
  ctx->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_shadow(kfvm_ctx* ctx, const double* U, float* shadow, cudaStream_t st) {
  const long long n = ctx->ncell * ctx->nv;
  unsigned blocks = (unsigned)((n + kBlock - 1) / kBlock);
  if (blocks > 65535u * 8u) blocks = 65535u * 8u;
  shadow_kernel<<<blocks, kBlock, 0, st>>>(U, shadow, n);
  ctx->launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_face_flux(kfvm_ctx* ctx, const void* faces, cudaStream_t st) {
  if (ctx->dims == 2 && ctx->R == 2) return face_flux_dr<2, 2>(ctx, faces, st);
  if (ctx->dims == 2 && ctx->R == 3) return face_flux_dr<2, 3>(ctx, faces, st);
  if (ctx->dims == 3 && ctx->R == 2) return face_flux_dr<3, 2>(ctx, faces, st);
  return face_flux_dr<3, 3>(ctx, faces, st);
}

cudaError_t launch_update(kfvm_ctx* ctx, int stage, const double* U0, const double* Us, double* out,
                          cudaStream_t st) {
  if (ctx->dims == 2) return update_d<2>(ctx, stage, U0, Us, out, st);
  return update_d<3>(ctx, stage, U0, Us, out, st);
}

cudaError_t launch_flux_update(kfvm_ctx* ctx, int stage, const void* faces, const double* U0, const double* Us,
                               double* out, cudaStream_t st, float* shadow_out, int zc_lo, int zc_hi, int zf_first,
                               int zf_count) {
  if (ctx->dims == 2 && ctx->R == 2) return flux_update_dr<2, 2>(ctx, stage, faces, U0, Us, out, st, shadow_out, 0, 0, 0, 0);
  if (ctx->dims == 2 && ctx->R == 3) return flux_update_dr<2, 3>(ctx, stage, faces, U0, Us, out, st, shadow_out, 0, 0, 0, 0);
  if (ctx->dims == 3 && ctx->R == 2)
    return flux_update_dr<3, 2>(ctx, stage, faces, U0, Us, out, st, shadow_out, zc_lo, zc_hi, zf_first, zf_count);
  return flux_update_dr<3, 3>(ctx, stage, faces, U0, Us, out, st, shadow_out, zc_lo, zc_hi, zf_first, zf_count);
}

cudaError_t fma_peak(int bits, double* flops) {
  return bits == 64 ? fma_peak_t<double>(flops) : fma_peak_t<float>(flops);
}

}  // namespace kfvm

// ===========================================================================
// Allocation-free flux divergence (kfvm_flux_static).
//
// Some callers must not allocate device memory at all: plug-ins whose host
// application owns the device memory budget through its own pool, and
// latency-sensitive loops where cudaMalloc/cudaFree (which may synchronise
// the device) are not allowed.  For them kfvm_flux_static runs the same face
// flux and divergence kernels as kfvm_flux without a context, keeping the
// face-averaged fluxes in the fixed array below instead of in buffers that
// kfvm_init allocates.  The array lives in every device that loads this
// library until the process exits.  Its device address is looked up once per
// device, on the first call made with that device current.
// ===========================================================================
namespace kfvm {
namespace {
constexpr size_t kStaticHeader = 256;             // status word of the last call
constexpr size_t kStaticFluxBytes = 16u << 20;    // 16 MiB of face fluxes
}  // namespace
}  // namespace kfvm

static __device__ __align__(256) unsigned char kfvm_static_scratch[kfvm::kStaticHeader + kfvm::kStaticFluxBytes];

namespace kfvm {
namespace {

std::mutex g_static_mu;
void* g_static_addr[128] = {nullptr};

cudaError_t static_scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, kfvm_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return cudaSuccess;
}

template <int D, int R>
cudaError_t flux_static_dr(const GridArgs& a, const FluxLayout& L, const double* faces, double* flux, double* dUdt,
                           cudaStream_t st) {
  long long mx = 0;
  for (int d = 0; d < D; ++d) mx = L.nface[d] > mx ? L.nface[d] : mx;
  dim3 grid((unsigned)((mx + kBlock - 1) / kBlock), D);
  face_flux_kernel<D, R, double><<<grid, kBlock, 0, st>>>(a, L, faces, flux);
  const long long ncell = (long long)a.n[0] * a.n[1] * a.n[2];
  update_kernel<D, double, false><<<(unsigned)((ncell + kBlock - 1) / kBlock), kBlock, 0, st>>>(
      a, L, flux, 0, nullptr, nullptr, dUdt, nullptr);
  return cudaGetLastError();
}

}  // namespace
}  // namespace kfvm

extern "C" kfvm_status kfvm_flux_static(const kfvm_grid* grid, int dims, int radius, double gamma, int riemann,
                                        const double* faces, double* dUdt, int* status_out, void* stream) {
  using namespace kfvm;
  if (!grid || !faces || !dUdt || (dims != 2 && dims != 3) || (radius != 2 && radius != 3)) return KFVM_ERR_ARG;
  if (!(gamma > 1.0) || (riemann != 0 && riemann != 1)) return KFVM_ERR_ARG;
  GridArgs a{};
  long long ncell = 1;
  for (int d = 0; d < 3; ++d) {
    const bool used = d < dims;
    a.n[d] = used ? grid->n[d] : 1;
    if (a.n[d] < 1 || (used && !(grid->hi[d] > grid->lo[d]))) return KFVM_ERR_ARG;
    a.dx[d] = used ? (grid->hi[d] - grid->lo[d]) / grid->n[d] : 1.0;
    a.idx[d] = 1.0 / a.dx[d];
    a.idxf[d] = (float)a.idx[d];
    for (int s = 0; s < 2; ++s) {
      a.bc[d][s] = used ? grid->bc[d][s] : KFVM_BC_PERIODIC;
      if (a.bc[d][s] != KFVM_BC_PERIODIC && a.bc[d][s] != KFVM_BC_OUTFLOW) return KFVM_ERR_ARG;
    }
    ncell *= a.n[d];
  }
  FluxLayout L{};
  long long total = 0;
  for (int d = 0; d < 3; ++d) {
    L.off[d] = total;
    L.nface[d] = d < dims ? (long long)(a.n[d] + 1) * (ncell / a.n[d]) : 0;
    total += (long long)(dims + 2) * L.nface[d];
  }
  if ((unsigned long long)total * sizeof(double) > kStaticFluxBytes) return KFVM_ERR_TOO_LARGE;
  void* base = nullptr;
  if (static_scratch_address(&base) != cudaSuccess) return KFVM_ERR_CUDA;
  int* status = reinterpret_cast<int*>(base);
  double* flux = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + kStaticHeader);
  a.gamma = gamma;
  a.riemann = riemann;
  a.status = status;
  a.scalars = nullptr;
  a.zf_first = 0;
  a.zf_count = a.n[2];
  a.zc_lo = 0;
  a.zc_hi = a.n[2];
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return KFVM_ERR_CUDA;
  cudaError_t e;
  if (dims == 2 && radius == 2) e = flux_static_dr<2, 2>(a, L, faces, flux, dUdt, st);
  else if (dims == 2) e = flux_static_dr<2, 3>(a, L, faces, flux, dUdt, st);
  else if (radius == 2) e = flux_static_dr<3, 2>(a, L, faces, flux, dUdt, st);
  else e = flux_static_dr<3, 3>(a, L, faces, flux, dUdt, st);
  if (e != cudaSuccess) return KFVM_ERR_CUDA;
  if (status_out && cudaMemcpyAsync(status_out, status, sizeof(int), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return KFVM_ERR_CUDA;
  return KFVM_OK;
}
