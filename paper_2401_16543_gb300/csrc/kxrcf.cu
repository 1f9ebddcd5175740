// kxrcf.cu -- the KXRCF troubled-cell indicator (Sec. 3.5; Sec. 5.3 step 2, items 1-2).
//
// The unlimited linear S0 reconstruction of the conservative variables gives
// every cell a state at each of its face Gauss points.  At every point s on the
// faces of cell c, q = p / rho^gamma (the entropy) of c's own state and of the
// state reconstructed at the same point by the cell across that face are
// compared; c is smooth (mask 1: it keeps the linear reconstruction) when
//     max_s |q+_s - q-_s| / <Q>  <  Delta^m,   <Q> = p(Ubar_c) / rhobar_c^gamma,
// Delta the largest cell width and m = 3/2 by default; otherwise it is flagged
// for WENO-AO (mask 0).  Faces on an outflow boundary carry no jump (the
// exterior state copies the interior one, Sec. 5.3 step 4); periodic faces
// compare with the wrapped neighbour.  A state that is not admissible
// (rho <= 0, p <= 0 or not finite) on either side of a point, or such a cell
// average, flags the cell.
//
// A CTA owns a TX x TY x TZ tile whose cell averages (halo R + 1, through the
// ghost-cell map) sit in shared memory.  The directions are taken one at a
// time: the tile's cells and the ring of cells just outside it along that
// direction (one thread each: the block has as many threads as the largest such
// set, so the ring is no second wave) reconstruct their two faces normal to it
// in one pass over the stencil (a ring cell keeps only the face it shares with
// the tile) and park q at those points in shared memory, numbered with x
// fastest so that a warp reads consecutive cells; then every tile cell compares
// its two faces with its neighbours'.  Each face state is computed once per
// direction instead of once per side.  T = double
// reads the float64 state (FP64 mode); T = float reads its float32 shadow (FP32
// mode), so the decision is taken in the precision of the path it serves.
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"

namespace kfvm {
namespace kx {

template <int D, int R>
struct KT {
  static constexpr int TX = (D == 2) ? 32 : 8;
  static constexpr int TY = 8;
  static constexpr int TZ = (D == 2) ? 1 : 4;
  static constexpr int H = R + 1;
  static constexpr int SX = TX + 2 * H, SY = TY + 2 * H, SZ = (D == 2) ? 1 : TZ + 2 * H;
  static constexpr int SN = SX * SY * SZ;
  static constexpr int THREADS = TX * TY * TZ;
  __host__ __device__ static constexpr int tdim(int k) { return k == 0 ? TX : (k == 1 ? TY : TZ); }
};

// S0 offsets in the shared-memory tile (geometry only: one table per (d, R)).
template <int D, int R>
__constant__ int c_delta[kMaxN0];

// cells of the tile plus the ring along dir (phase 1 of a direction)
template <int D, int R>
__host__ __device__ constexpr int ext_count(int dir) {
  using K = KT<D, R>;
  return K::THREADS / K::tdim(dir) * (K::tdim(dir) + 2);
}
// extent of axis k in the ring-extended numbering of direction dir
template <int D, int R>
__host__ __device__ constexpr int ext_dim(int dir, int k) {
  return KT<D, R>::tdim(k) + (k == dir ? 2 : 0);
}

template <int D, int R>
__host__ __device__ constexpr int max_ext() {
  int m = 0;
  for (int d = 0; d < D; ++d) m = ext_count<D, R>(d) > m ? ext_count<D, R>(d) : m;
  return m;
}

// rho^-gamma: float64 through pow; float32 as 2^(-gamma log2 rho) with the hardware log2 and exp2
// (relative error ~2e-7, below the float32 copy's own rounding of the states it is applied to)
__device__ __forceinline__ double rho_pow_neg(double rho, double gamma) { return 1.0 / pow(rho, gamma); }
__device__ __forceinline__ float rho_pow_neg(float rho, float gamma) { return exp2f(-gamma * __log2f(rho)); }

// q = p / rho^gamma of a conservative state; +inf when it is not admissible
template <int D, class T>
__device__ __forceinline__ T entropy(const T* u, T gamma) {
  T m2 = T(0);
#pragma unroll
  for (int k = 0; k < D; ++k) m2 = fma(u[1 + k], u[1 + k], m2);
  const T p = (gamma - T(1)) * (u[D + 1] - T(0.5) * m2 / u[0]);
  const bool ok = u[0] > T(0) && p > T(0) && isfinite(p) && isfinite(u[0]);
  return ok ? p * rho_pow_neg(u[0], gamma) : T(INFINITY);
}

template <class T>
__device__ __forceinline__ T jump(T a, T b) {
  return (isinf(a) || isinf(b)) ? T(INFINITY) : fabs(a - b);
}

template <int D, int R, class T>
__global__ void __launch_bounds__(max_ext<D, R>()) kxrcf_kernel(GridArgs a, const T* __restrict__ U,
                                                                   const double* __restrict__ w64, T thresh,
                                                                   unsigned char* __restrict__ mask) {
  using K = KT<D, R>;
  using G = Geo<D, R>;
  constexpr int NV = G::NV, N0 = G::N0, NT = G::NT, F = G::F, SN = K::SN;
  constexpr int EX = max_ext<D, R>(), TH = EX;  // threads = the largest tile + ring set
  // both faces of a direction in one pass over the stencil while their accumulators fit in ~80
  // registers (not for d = 3, R = 3: 2 x 9 points x 5 variables), and full unrolling up to 33 cells
  constexpr int SP = (2 * NT * NV * sizeof(T) <= 320) ? 2 : 1;
  constexpr int UL = N0 <= 33 ? N0 : 4;
  extern __shared__ unsigned char kx_smem[];
  T* sm = reinterpret_cast<T*>(kx_smem);  // [NV][SN] cell averages
  T* ws = sm + NV * SN;                    // [F][N0] r_0 face rows
  T* qb = ws + F * N0;                     // [2 * NT][EX] q at the faces of the current direction
  const long long ncell = (long long)a.n[0] * a.n[1] * a.n[2];
  const T gamma = (T)a.gamma;

  const int tiles_x = (a.n[0] + K::TX - 1) / K::TX, tiles_y = (a.n[1] + K::TY - 1) / K::TY;
  int b = blockIdx.x;
  const int bx = b % tiles_x;
  b /= tiles_x;
  const int by = b % tiles_y;
  const int bz = b / tiles_y;
  const int org[3] = {bx * K::TX, by * K::TY, (D == 3) ? bz * K::TZ : 0};
  const int tid = threadIdx.x;

  for (int i = tid; i < SN; i += TH) {
    const int sx = i % K::SX, sy = (i / K::SX) % K::SY, sz = i / (K::SX * K::SY);
    const int gx = map_index(org[0] - K::H + sx, a.n[0], a.bc[0][0], a.bc[0][1]);
    const int gy = map_index(org[1] - K::H + sy, a.n[1], a.bc[1][0], a.bc[1][1]);
    const int gz = (D == 3) ? map_index(org[2] - K::H + sz, a.n[2], a.bc[2][0], a.bc[2][1]) : 0;
    const long long gc = ((long long)gz * a.n[1] + gy) * a.n[0] + gx;
#pragma unroll
    for (int v = 0; v < NV; ++v) sm[v * SN + i] = U[v * ncell + gc];
  }
  for (int i = tid; i < F * N0; i += TH) ws[i] = (T)w64[i];  // q = 0 face rows lead the table
  __syncthreads();

  // this thread's tile cell
  const int lx = tid % K::TX, ly = (tid / K::TX) % K::TY, lz = tid / (K::TX * K::TY);
  const int me[3] = {lx, ly, lz};
  const bool active = tid < K::THREADS && org[0] + lx < a.n[0] && org[1] + ly < a.n[1] &&
                      (D == 2 || org[2] + lz < a.n[2]);
  const int c_me = (lx + K::H) + K::SX * ((ly + K::H) + K::SY * (D == 3 ? lz + K::H : 0));
  T jmax = T(0);

#pragma unroll 1
  for (int dir = 0; dir < D; ++dir) {
    const int td = K::tdim(dir);
    const int e0 = ext_dim<D, R>(dir, 0), e1 = ext_dim<D, R>(dir, 1);
    const int E = e0 * e1 * ext_dim<D, R>(dir, 2);
    // phase 1: q at the faces normal to dir of the tile cells and the ring along dir
    if (tid < E) {
      const int e = tid;
      // e -> (x, y, z) with x fastest; the coordinate along dir runs over -1..td
      int loc[3] = {e % e0, (e / e0) % e1, e / (e0 * e1)};
      loc[dir] -= 1;
      const int ld = loc[dir];
      const int c = (loc[0] + K::H) + K::SX * ((loc[1] + K::H) + K::SY * (D == 3 ? loc[2] + K::H : 0));
#pragma unroll 1
      for (int s0 = 0; s0 < 2; s0 += SP) {
        // the ring cell before the tile needs its high face only, the one after it its low face
        // (the other face of a ring cell is computed when SP = 2 but not stored)
        if (SP == 1 && ((ld < 0 && s0 == 0) || (ld >= td && s0 == 1))) continue;
        T acc[SP][NT][NV];
#pragma unroll
        for (int si = 0; si < SP; ++si)
#pragma unroll
          for (int t = 0; t < NT; ++t)
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[si][t][v] = T(0);
        const T* wrow = ws + ((dir * 2 + s0) * NT) * N0;
#pragma unroll UL
        for (int l = 0; l < N0; ++l) {
          const int o = c + c_delta<D, R>[l];
          T g[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) g[v] = sm[v * SN + o];
#pragma unroll
          for (int si = 0; si < SP; ++si)
#pragma unroll
            for (int t = 0; t < NT; ++t) {
              const T w = wrow[(si * NT + t) * N0 + l];
#pragma unroll
              for (int v = 0; v < NV; ++v) acc[si][t][v] = fma(w, g[v], acc[si][t][v]);
            }
        }
#pragma unroll
        for (int si = 0; si < SP; ++si) {
          const int side = s0 + si;
          if ((ld < 0 && side == 0) || (ld >= td && side == 1)) continue;
#pragma unroll
          for (int t = 0; t < NT; ++t) qb[(side * NT + t) * EX + e] = entropy<D, T>(acc[si][t], gamma);
        }
      }
    }
    __syncthreads();
    // phase 2: jumps across this thread's two faces normal to dir
    if (active) {
      const int ld = me[dir];
      // this cell and its neighbours along dir in the ring-extended numbering of phase 1
      const int e_me = (me[0] + (dir == 0)) + e0 * ((me[1] + (dir == 1)) + e1 * (me[2] + (dir == 2)));
      const int stride = dir == 0 ? 1 : (dir == 1 ? e0 : e0 * e1);
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int g_nb = org[dir] + ld + (side ? 1 : -1);
        if ((g_nb < 0 || g_nb >= a.n[dir]) && a.bc[dir][side] != KFVM_BC_PERIODIC) continue;
        const int e_nb = e_me + (side ? stride : -stride);
#pragma unroll
        for (int t = 0; t < NT; ++t)
          jmax = fmax(jmax, jump(qb[(side * NT + t) * EX + e_me], qb[((1 - side) * NT + t) * EX + e_nb]));
      }
    }
    __syncthreads();
  }

  if (active) {
    T ub[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) ub[v] = sm[v * SN + c_me];
    const T Q = entropy<D, T>(ub, gamma);
    const T ratio = isinf(Q) ? T(INFINITY) : jmax / Q;
    const long long cell = ((long long)(D == 3 ? org[2] + lz : 0) * a.n[1] + org[1] + ly) * a.n[0] + org[0] + lx;
    mask[cell] = ratio < thresh ? 1 : 0;
  }
}

template <int D, int R, class T>
cudaError_t launch_dr(kfvm_ctx* ctx, const T* U, unsigned char* mask, cudaStream_t st) {
  using K = KT<D, R>;
  using G = Geo<D, R>;
  static bool ready[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !ready[dev]) {
    constexpr StencilTable t = make_stencil(D, R);
    int d[kMaxN0] = {0};
    for (int l = 0; l < t.n0; ++l) d[l] = t.off[l][0] + K::SX * (t.off[l][1] + K::SY * t.off[l][2]);
    cudaError_t e = cudaMemcpyToSymbol(c_delta<D, R>, d, sizeof(d));
    if (e != cudaSuccess) return e;
    ready[dev] = true;
  }
  GridArgs a = make_grid_args(ctx);
  double delta = 0.0;
  for (int k = 0; k < D; ++k) delta = ctx->dx[k] > delta ? ctx->dx[k] : delta;
  const T thresh = (T)std::pow(delta, ctx->kxrcf_m);
  const int tiles = ((ctx->n[0] + K::TX - 1) / K::TX) * ((ctx->n[1] + K::TY - 1) / K::TY) *
                    ((D == 3) ? (ctx->n[2] + K::TZ - 1) / K::TZ : 1);
  const size_t smem = sizeof(T) * ((size_t)G::NV * K::SN + (size_t)G::F * G::N0 + 2 * G::NT * max_ext<D, R>());
  auto kern = kxrcf_kernel<D, R, T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<tiles, max_ext<D, R>(), smem, st>>>(a, U, ctx->d_w64, thresh, mask);
  ctx->launches += 1;
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_t(kfvm_ctx* ctx, const T* U, unsigned char* mask, cudaStream_t st) {
  if (ctx->dims == 2 && ctx->R == 2) return launch_dr<2, 2, T>(ctx, U, mask, st);
  if (ctx->dims == 2 && ctx->R == 3) return launch_dr<2, 3, T>(ctx, U, mask, st);
  if (ctx->dims == 3 && ctx->R == 2) return launch_dr<3, 2, T>(ctx, U, mask, st);
  return launch_dr<3, 3, T>(ctx, U, mask, st);
}

}  // namespace kx

cudaError_t launch_kxrcf(kfvm_ctx* ctx, const double* U, const float* shadow, unsigned char* mask, cudaStream_t st) {
  return shadow ? kx::launch_t<float>(ctx, shadow, mask, st) : kx::launch_t<double>(ctx, U, mask, st);
}

}  // namespace kfvm
