// common.cuh -- device helpers shared by the hot-path kernels.
#pragma once

#include <cuda_runtime.h>

#include "geometry.h"
#include "internal.h"

namespace kfvm {

// Grid, boundary conditions and scheme options passed to every hot-path kernel.
struct GridArgs {
  int n[3];
  int bc[3][2];
  double dx[3];
  double gamma;
  double eps;
  double kappa, eta;
  int positivity;
  int riemann;
  int vars;  // WENO-AO variables: 0 linearized primitive (Sec. 3.4.2), 1 characteristic (Sec. 3.4.1)
  int* status;
  DevScalars* scalars;
  // float32 copies for the mixed-precision kernels
  float gammaf, epsf, lo_f, hi_f;
  // reciprocal cell sizes (host-computed: a float64 division costs ~10 FP64 issue slots here)
  double idx[3];
  float idxf[3];
  // slabs (3D): the Riemann-state buffer holds the z-planes zf_first .. zf_first + zf_count - 1
  // (wrapped periodically); a launch processes the cells of planes zc_lo .. zc_hi - 1
  int zf_first, zf_count, zc_lo, zc_hi;
};

inline GridArgs make_grid_args(const kfvm_ctx* c) {
  GridArgs g{};
  for (int a = 0; a < 3; ++a) {
    g.n[a] = c->n[a];
    g.dx[a] = c->dx[a];
    g.bc[a][0] = c->bc[a][0];
    g.bc[a][1] = c->bc[a][1];
  }
  g.gamma = c->gamma;
  g.eps = c->eps;
  g.kappa = c->kappa;
  g.eta = c->eta;
  g.positivity = c->positivity;
  g.riemann = c->riemann;
  g.vars = c->vars;
  g.status = c->d_status;
  g.scalars = c->d_scalars;
  g.gammaf = (float)c->gamma;
  g.epsf = (float)c->eps;
  g.lo_f = (float)(1.0 - c->kappa + c->kappa * c->eta);
  g.hi_f = (float)(1.0 + c->kappa - c->kappa * c->eta);
  for (int a = 0; a < 3; ++a) {
    g.idx[a] = 1.0 / c->dx[a];
    g.idxf[a] = (float)g.idx[a];
  }
  g.zf_first = 0;
  g.zf_count = c->n[2];
  g.zc_lo = 0;
  g.zc_hi = c->n[2];
  return g;
}

// Index of grid cell (x, y, z) in the Riemann-state buffer (see zf_first / zf_count).
__device__ __forceinline__ long long face_cell(const GridArgs& a, int x, int y, int z) {
  // z is a wrapped grid index; the buffer's planes run from zf_first (possibly -1) upwards
  int l = z - a.zf_first;
  if (l < 0) l += a.n[2];
  if (l >= a.zf_count) l -= a.n[2];
  return ((long long)l * a.n[1] + y) * a.n[0] + x;
}
__device__ __forceinline__ long long face_ncell(const GridArgs& a) {
  return (long long)a.zf_count * a.n[0] * a.n[1];
}
// Global z of plane l of the Riemann-state buffer, or -1 when that plane lies
// outside a non-periodic grid.
__device__ __forceinline__ int slab_plane(const GridArgs& a, int l) {
  int z = a.zf_first + l;
  if (z >= 0 && z < a.n[2]) return z;
  if (a.bc[2][0] != KFVM_BC_PERIODIC) return -1;
  return ((z % a.n[2]) + a.n[2]) % a.n[2];
}

// Ghost-cell index map (Sec. 5.3 step 1): periodic wraps, outflow clamps.
__device__ __forceinline__ int map_index(int i, int n, int bclo, int bchi) {
  if (i < 0) return bclo == KFVM_BC_PERIODIC ? ((i % n) + n) % n : 0;
  if (i >= n) return bchi == KFVM_BC_PERIODIC ? i % n : n - 1;
  return i;
}

// Shared-memory tile of one CTA: TX x TY x TZ cells plus a halo of H cells.
template <int D, int R>
struct Tile {
  static constexpr int TX = (D == 2) ? 32 : 8;
  static constexpr int TY = (D == 2) ? 8 : 8;
  static constexpr int TZ = (D == 2) ? 1 : 2;
  static constexpr int H = R;
  static constexpr int SX = TX + 2 * H, SY = TY + 2 * H, SZ = (D == 2) ? 1 : TZ + 2 * H;
  static constexpr int SN = SX * SY * SZ;
  static constexpr int THREADS = TX * TY * TZ;
  // smem offset of S0 cell l relative to the centre; device code reads it
  // through a local copy: `constexpr auto DL = Tile<D,R>::deltas;`
  __host__ __device__ static constexpr IntArr make_deltas() {
    IntArr a{};
    constexpr StencilTable t = make_stencil(D, R);
    for (int l = 0; l < t.n0; ++l) a.v[l] = t.off[l][0] + SX * (t.off[l][1] + SY * t.off[l][2]);
    return a;
  }
  static constexpr IntArr deltas = make_deltas();
};

// Linear weights of WENO-AO (Sec. 3.2): gamma_hi = gamma_lo = 0.8; gamma_0 = gamma_hi,
// gamma_1 = (1 - gamma_hi) gamma_lo, biased gamma_q = (1 - gamma_hi)(1 - gamma_lo) / (2d).
template <int D>
__host__ __device__ constexpr double linear_weight(int q) {
  constexpr double ghi = 0.8, glo = 0.8;
  return q == 0 ? ghi : (q == 1 ? (1.0 - ghi) * glo : (1.0 - ghi) * (1.0 - glo) / (2 * D));
}

// 1/x in float64 from a float32 reciprocal refined by one Newton-Raphson step
// (relative error below 1e-14 for normal x; Newton's iteration for 1/x).
__device__ __forceinline__ double recip64(double x) {
  const double r0 = (double)__frcp_rn((float)x);
  return r0 * fma(-x, r0, 2.0);
}

__device__ __forceinline__ void raise_flag(int* status, int bit) {
  if (status) atomicOr(status, bit);
}

}  // namespace kfvm
