// recon32_33.cu -- FP32 Riemann states for d = 3, R = 3 (Sec. 3, Sec. 4, Sec. 5.3 steps 1-3).
//
// The same mathematics as recon32.cuh, arranged for the size of this case: S0 has
// 123 cells, there are 8 stencils with 348 (stencil, cell) pairs, 54 face points
// and 19 derivative multi-indices, i.e. 25,404 multiply-adds per variable and
// cell.  Unrolling that with compile-time weights, as the smaller cases do, would
// give a kernel of ~10^5 instructions, so here
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
#include "internal.h"
#include "recon32.cuh"

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
  float uc[NV], ut[3], kin, irt, uv, gm1;
  int v;
  __device__ __forceinline__ Ref(const float* __restrict__ sm, int cc, int var, float gm1_) : gm1(gm1_), v(var) {
    r32::cell_ref<3, 3>(sm, cc, uc, ut, kin, irt);
    uv = v == 1 ? ut[0] : (v == 2 ? ut[1] : ut[2]);
  }
  __device__ __forceinline__ float delta(const float* __restrict__ sm, int o) const {
    const float dr = sm[o] - uc[0];
    if (v == 0) return dr;
    if (v <= 3) return fmaf(-uv, dr, sm[v * SN + o] - uc[v]) * irt;
    float t = fmaf(kin, dr, sm[4 * SN + o] - uc[4]);
    t = fmaf(-ut[0], sm[SN + o] - uc[1], t);
    t = fmaf(-ut[1], sm[2 * SN + o] - uc[2], t);
    t = fmaf(-ut[2], sm[3 * SN + o] - uc[3], t);
    return gm1 * t;
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
                                           int x0, int y0, int z0) {
  const long long ncell = (long long)a.n[0] * a.n[1] * a.n[2];
  const float gm1 = a.gammaf - 1.0f;
  for (int i = threadIdx.x; i < SN; i += TH) {
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

cudaError_t launch_recon32_33(kfvm_ctx* ctx, const double* U, const float* shadow, float* faces, cudaStream_t st,
                              int zf_first, int zf_count) {
  using namespace r33;
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
  recon33_kernel<<<tiles, TH, smem, st>>>(a, ctx->recon, U, shadow, faces, ctx->d_gate_mask,
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
