// api.cu -- the C ABI of include/kfvm.h: context lifetime, host-side set-up
// (stencils, polynomial degrees, options) and the orchestration of the
// device kernels for reconstruct / flux / rhs / SSP-RK3 step.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

using namespace kfvm;

namespace {

// ---------------------------------------------------------------------------
// Polynomial degree of a (sub)stencil: the largest p whose cell-average
// monomial matrix P is unisolvent (full column rank) over the stencil
// (Sec. 2.1).  Column v of P scaled by prod_k 2^(a_k+1) (a_k+1) is the integer
// prod_k [(2o_k+1)^(a_k+1) - (2o_k-1)^(a_k+1)], so the rank is exact integer
// arithmetic; it is computed modulo two 61-bit primes (the rank over Q is at
// least the rank mod p, and equal unless p divides every nonzero maximal
// minor).
// ---------------------------------------------------------------------------
constexpr uint64_t kPrimes[2] = {2305843009213693951ULL, 4611686018427387847ULL};

uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)((unsigned __int128)a * b % p); }

uint64_t powmod(uint64_t a, uint64_t e, uint64_t p) {
  uint64_t r = 1;
  while (e) {
    if (e & 1) r = mulmod(r, a, p);
    a = mulmod(a, a, p);
    e >>= 1;
  }
  return r;
}

int rank_mod(std::vector<std::vector<int64_t>> rows, uint64_t p) {
  const size_t nr = rows.size(), nc = nr ? rows[0].size() : 0;
  std::vector<std::vector<uint64_t>> m(nr, std::vector<uint64_t>(nc));
  for (size_t i = 0; i < nr; ++i)
    for (size_t j = 0; j < nc; ++j) {
      int64_t v = rows[i][j] % (int64_t)p;  // both primes are below 2^63
      m[i][j] = v < 0 ? (uint64_t)(v + (int64_t)p) : (uint64_t)v;
    }
  int rank = 0;
  for (size_t c = 0; c < nc && (size_t)rank < nr; ++c) {
    size_t piv = nr;
    for (size_t r = rank; r < nr; ++r)
      if (m[r][c]) { piv = r; break; }
    if (piv == nr) continue;
    std::swap(m[rank], m[piv]);
    uint64_t inv = powmod(m[rank][c], p - 2, p);
    for (size_t r = 0; r < nr; ++r) {
      if ((int)r == rank || !m[r][c]) continue;
      uint64_t f = mulmod(m[r][c], inv, p);
      for (size_t j = c; j < nc; ++j) m[r][j] = (m[r][j] + p - mulmod(f, m[rank][j], p)) % p;
    }
    ++rank;
  }
  return rank;
}

int64_t ipow64(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// multi-indices with |alpha| <= p, by total degree then alpha_x descending (3 ints each)
std::vector<int> monomials(int dim, int p, bool skip_constant) {
  std::vector<int> out;
  for (int n = skip_constant ? 1 : 0; n <= p; ++n) {
    if (dim == 2) {
      for (int a = n; a >= 0; --a) { out.push_back(a); out.push_back(n - a); out.push_back(0); }
    } else {
      for (int a = n; a >= 0; --a)
        for (int b = n - a; b >= 0; --b) { out.push_back(a); out.push_back(b); out.push_back(n - a - b); }
    }
  }
  return out;
}

int max_unisolvent_degree(int dim, const std::vector<int>& offs /* n x 3 */) {
  const int n = (int)offs.size() / 3;
  int p = 0;
  for (;;) {
    std::vector<int> mons = monomials(dim, p + 1, false);
    const int D = (int)mons.size() / 3;
    if (D > n) return p;
    std::vector<std::vector<int64_t>> P(n, std::vector<int64_t>(D));
    for (int h = 0; h < n; ++h)
      for (int v = 0; v < D; ++v) {
        int64_t e = 1;
        for (int k = 0; k < dim; ++k) {
          int o = offs[3 * h + k], a = mons[3 * v + k];
          e *= ipow64(2 * o + 1, a + 1) - ipow64(2 * o - 1, a + 1);
        }
        P[h][v] = e;
      }
    int r = 0;
    for (uint64_t pr : kPrimes) {
      int rr = rank_mod(P, pr);
      if (rr > r) r = rr;
    }
    if (r < D) return p;
    ++p;
  }
}

const StencilTable* table_for(int dims, int R) {
  static const StencilTable t22 = make_stencil(2, 2), t23 = make_stencil(2, 3), t32 = make_stencil(3, 2),
                            t33 = make_stencil(3, 3);
  if (dims == 2 && R == 2) return &t22;
  if (dims == 2 && R == 3) return &t23;
  if (dims == 3 && R == 2) return &t32;
  if (dims == 3 && R == 3) return &t33;
  return nullptr;
}

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, sizeof(T) * count);
}

kfvm_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return KFVM_OK;
  if (e == cudaErrorMemoryAllocation) return KFVM_ERR_NOMEM;
  return KFVM_ERR_CUDA;
}

#define KFVM_TRY(expr)                                 \
  do {                                                 \
    cudaError_t e_ = (expr);                           \
    if (e_ != cudaSuccess) return cuda_status(e_);     \
  } while (0)

cudaEvent_t pool_event(kfvm_ctx* c) {
  if (!c->prof_free.empty()) {
    cudaEvent_t e = c->prof_free.back();
    c->prof_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Fold completed event pairs into the per-kernel totals; returns false if one is still pending.
bool prof_fold(kfvm_ctx* c) {
  bool all = true;
  std::vector<ProfPair> keep;
  for (const ProfPair& p : c->prof_pairs) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p.start, p.stop) == cudaSuccess) {
      c->prof_ms[p.kernel] += ms;
      c->prof_launches[p.kernel] += 1;
      c->prof_free.push_back(p.start);
      c->prof_free.push_back(p.stop);
    } else {
      (void)cudaGetLastError();
      keep.push_back(p);
      all = false;
    }
  }
  c->prof_pairs.swap(keep);
  return all;
}

// A launcher call bracketed by tracing events.
#define KFVM_LAUNCH(ctx, kernel, st, call)             \
  do {                                                 \
    cudaEvent_t ev_ = prof_begin((ctx), (st));         \
    cudaError_t e_ = (call);                           \
    prof_end((ctx), (kernel), ev_, (st));              \
    if (e_ != cudaSuccess) return cuda_status(e_);     \
  } while (0)

kfvm_status check_ready(kfvm_ctx* ctx) {
  if (!ctx) return KFVM_ERR_ARG;
  if (!ctx->weights_built) return KFVM_ERR_STATE;
  if (ctx->recon == 2 && !ctx->gate_loaded) return KFVM_ERR_STATE;
  // characteristic variables in float32: d = 2 and d = 3 radius 2 (the radius-3 3D kernels are lin-prim only)
  if (ctx->vars == 1 && ctx->precision == 32 && ctx->dims == 3 && ctx->R == 3) return KFVM_ERR_STATE;
  return KFVM_OK;
}

// Bytes of the Riemann-state buffer: 3D grids whose float64 states exceed it are stepped in z-slabs.
constexpr size_t kFaceBudget = (size_t)24 << 30;

// Bytes the Riemann states of one z-plane take in the current precision: float64 conservative
// values, or float32 primitive values (a float4 per point plus, in 3D, a float of w).
size_t face_plane_bytes(const kfvm_ctx* c) {
  const size_t per_point = c->precision == 64 ? (size_t)c->nv * sizeof(double) : (c->dims == 3 ? 20 : 16);
  return per_point * c->F * c->n[0] * c->n[1];
}

// z-planes per slab of a 3D step (= n[2]: one pass over the whole grid).  A slab of S planes
// reconstructs S + 2 (one on each side for its boundary faces), so the automatic choice takes as
// few slabs as the buffer allows, makes them even, and rounds S + 2 up to a multiple of the
// reconstruction's z-tile when the buffer still holds it (no partly empty tiles).
int slab_planes(const kfvm_ctx* c) {
  const int nz = c->n[2];
  if (c->dims != 3) return nz;
  const long long P = (long long)(c->face_bytes / face_plane_bytes(c));  // >= 3 (see kfvm_init)
  if (c->slab_user > 0) {
    if (c->slab_user >= nz && P >= nz) return nz;
    return (int)(c->slab_user < P - 2 ? c->slab_user : P - 2);
  }
  if (P >= nz) return nz;
  const long long smax = P - 2, ns = (nz + smax - 1) / smax;
  long long s = (nz + ns - 1) / ns;
  const int tz = (c->precision == 32 && c->R == 3) ? 4 : 2;
  const long long sa = (s + 2 + tz - 1) / tz * tz - 2;
  return (int)(sa <= smax ? sa : s);
}

}  // namespace

namespace kfvm {

cudaEvent_t prof_begin(kfvm_ctx* ctx, cudaStream_t st) {
  if (!ctx->profile) return nullptr;
  cudaEvent_t e = pool_event(ctx);
  if (e) cudaEventRecord(e, st);
  return e;
}

void prof_end(kfvm_ctx* ctx, int kernel, cudaEvent_t start, cudaStream_t st) {
  if (!ctx->profile || !start) return;
  cudaEvent_t e = pool_event(ctx);
  if (!e) return;
  cudaEventRecord(e, st);
  ctx->prof_pairs.push_back(ProfPair{start, e, kernel});
}

}  // namespace kfvm

extern "C" {

int kfvm_stencil_info(int dims, int radius, int* sizes, int* degrees, int* nface, int* nderiv) {
  const StencilTable* t = table_for(dims, radius);
  if (!t) return -1;
  for (int q = 0; q < t->nq; ++q) {
    std::vector<int> offs;
    for (int l = 0; l < t->len[q]; ++l)
      for (int k = 0; k < 3; ++k) offs.push_back(t->off[t->idx[q][l]][k]);
    if (sizes) sizes[q] = t->len[q];
    if (degrees) degrees[q] = max_unisolvent_degree(dims, offs);
  }
  if (nface) *nface = 2 * dims * ipow(radius, dims - 1);
  if (nderiv) *nderiv = n_multi(dims, radius);
  return t->nq;
}

const char* kfvm_status_string(kfvm_status s) {
  switch (s) {
    case KFVM_OK: return "ok";
    case KFVM_ERR_ARG: return "invalid argument";
    case KFVM_ERR_CUDA: return "CUDA error";
    case KFVM_ERR_SINGULAR: return "singular weight system";
    case KFVM_ERR_NONPHYSICAL: return "non-admissible state (rho <= 0, p <= 0 or NaN)";
    case KFVM_ERR_STATE: return "call out of order";
    case KFVM_ERR_TIMEOUT: return "bounded device wait timed out";
    case KFVM_ERR_NOMEM: return "out of memory";
    case KFVM_ERR_TOO_LARGE: return "problem exceeds the fixed-size scratch of kfvm_flux_static";
  }
  return "unknown status";
}

kfvm_status kfvm_init(kfvm_ctx** out, const kfvm_grid* g, int dims, int radius, double ell_over_dx, double gamma) {
  if (!out) return KFVM_ERR_ARG;
  *out = nullptr;
  if (!g || (dims != 2 && dims != 3) || (radius != 2 && radius != 3)) return KFVM_ERR_ARG;
  if (!(ell_over_dx > 0) || !(gamma > 1)) return KFVM_ERR_ARG;
  for (int a = 0; a < dims; ++a) {
    if (g->n[a] < 1 || !(g->hi[a] > g->lo[a])) return KFVM_ERR_ARG;
    for (int s = 0; s < 2; ++s)
      if (g->bc[a][s] != KFVM_BC_PERIODIC && g->bc[a][s] != KFVM_BC_OUTFLOW) return KFVM_ERR_ARG;
    if ((g->bc[a][0] == KFVM_BC_PERIODIC) != (g->bc[a][1] == KFVM_BC_PERIODIC)) return KFVM_ERR_ARG;
  }
  kfvm_ctx* c = new (std::nothrow) kfvm_ctx();
  if (!c) return KFVM_ERR_NOMEM;
  c->dims = dims;
  c->R = radius;
  c->nv = dims + 2;
  c->gamma = gamma;
  c->ell = ell_over_dx;
  for (int a = 0; a < 3; ++a) {
    c->n[a] = a < dims ? g->n[a] : 1;
    c->dx[a] = a < dims ? (g->hi[a] - g->lo[a]) / g->n[a] : 1.0;
    for (int s = 0; s < 2; ++s) c->bc[a][s] = a < dims ? g->bc[a][s] : 0;
  }
  c->ncell = (long long)c->n[0] * c->n[1] * c->n[2];
  int F = 0, M = 0;
  c->nq = kfvm_stencil_info(dims, radius, c->sizes, c->degrees, &F, &M);
  c->F = F;
  c->M = M;
  c->NT = ipow(radius, dims - 1);
  c->n0 = c->sizes[0];
  c->wcount = 0;
  for (int q = 0; q < c->nq; ++q) c->wcount += (size_t)c->sizes[q] * (F + M);
  c->gate.in = 2 * make_stencil(dims, 2).n0;

  const size_t nc = (size_t)c->ncell, nv = (size_t)c->nv;
  cudaError_t e = cudaSuccess;
  size_t flux_total = 0;
  for (int a = 0; a < dims; ++a) {
    c->flux_off[a] = flux_total;
    size_t faces = (size_t)(c->n[a] + 1) * (nc / c->n[a]);
    flux_total += nv * faces;
  }
  if (e == cudaSuccess) e = dalloc(&c->d_w64, c->wcount);
  // float32 weights: the packed table, or for d = 3, R = 3 the padded row table of recon32_33
  if (e == cudaSuccess)
    e = dalloc(&c->d_w32, (dims == 3 && radius == 3) ? recon33_table_floats() : c->wcount);
  if (e == cudaSuccess && dims == 3 && radius == 3) e = cudaMalloc(&c->d_w33tc, recon33_tc_image_bytes());
  // Riemann-state buffer: the whole grid's float64 states if they fit in kFaceBudget, else
  // kFaceBudget (at least three planes); 3D steps then run in z-slabs (slab_planes below)
  {
    const size_t plane = (size_t)F * nv * c->n[0] * c->n[1];  // float64 values per z-plane
    size_t count = plane * c->n[2];
    if (dims == 3 && count * sizeof(double) > kFaceBudget) {
      count = kFaceBudget / sizeof(double);
      if (count < 3 * plane) count = 3 * plane;
    }
    c->face_bytes = count * sizeof(double);
    if (e == cudaSuccess) e = dalloc((double**)&c->d_faces, count);
  }
  if (e == cudaSuccess) e = dalloc(&c->d_flux, flux_total);
  if (e == cudaSuccess) e = dalloc(&c->d_stage, nv * nc);
  if (e == cudaSuccess) e = dalloc(&c->d_shadow, nv * nc);
  if (e == cudaSuccess) e = dalloc(&c->d_gate_mask, nc);
  if (e == cudaSuccess) e = dalloc(&c->d_scalars, 1);
  if (e == cudaSuccess) e = dalloc(&c->d_status, 1);
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_scalars, 0, sizeof(DevScalars));
  if (e != cudaSuccess) {
    kfvm_destroy(c);
    return cuda_status(e);
  }
  *out = c;
  return KFVM_OK;
}

void kfvm_destroy(kfvm_ctx* c) {
  if (!c) return;
  for (const ProfPair& p : c->prof_pairs) {
    cudaEventDestroy(p.start);
    cudaEventDestroy(p.stop);
  }
  for (cudaEvent_t e : c->prof_free) cudaEventDestroy(e);
  cudaFree(c->d_w64);
  cudaFree(c->d_w32);
  cudaFree(c->d_w33tc);
  cudaFree(c->d_faces);
  cudaFree(c->d_flux);
  cudaFree(c->d_stage);
  cudaFree(c->d_stage2);
  cudaFree(c->d_shadow2);
  cudaFree(c->d_L);
  cudaFree(c->d_shadow);
  cudaFree(c->d_gate_mask);
  cudaFree(c->d_scalars);
  cudaFree(c->d_status);
  cudaFree(c->d_gate);
  cudaFree(c->d_gate_adam);
  cudaFree(c->d_gate_grad);
  delete c;
}

size_t kfvm_weights_count(const kfvm_ctx* ctx) { return ctx ? ctx->wcount : 0; }

long long kfvm_launch_count(const kfvm_ctx* ctx) { return ctx ? ctx->launches : 0; }

kfvm_status kfvm_build_weights(kfvm_ctx* ctx, void* stream) {
  if (!ctx) return KFVM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int* d_err = nullptr;
  KFVM_TRY(cudaMalloc(&d_err, sizeof(int)));
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = launch_build_weights(ctx, st, d_err);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_err);
  if (e != cudaSuccess) return cuda_status(e);
  if (herr) return KFVM_ERR_SINGULAR;
  ctx->w_host.assign(ctx->wcount, 0.0);
  KFVM_TRY(cudaMemcpy(ctx->w_host.data(), ctx->d_w64, sizeof(double) * ctx->wcount, cudaMemcpyDeviceToHost));
  const bool rows = ctx->dims == 3 && ctx->R == 3;
  std::vector<float> w32(rows ? recon33_table_floats() : ctx->wcount);
  if (rows)
    recon33_fill_table(ctx->w_host.data(), w32.data());
  else
    for (size_t i = 0; i < ctx->wcount; ++i) w32[i] = (float)ctx->w_host[i];
  KFVM_TRY(cudaMemcpy(ctx->d_w32, w32.data(), sizeof(float) * w32.size(), cudaMemcpyHostToDevice));
  if (ctx->d_w33tc) {
    std::vector<unsigned char> img(recon33_tc_image_bytes(), 0);
    recon33_tc_fill_image(ctx->w_host.data(), img.data());
    KFVM_TRY(cudaMemcpy(ctx->d_w33tc, img.data(), img.size(), cudaMemcpyHostToDevice));
  }
  ctx->weights_built = true;
  return KFVM_OK;
}

kfvm_status kfvm_get_weights(kfvm_ctx* ctx, double* host, size_t count) {
  if (!ctx || !host || count != ctx->wcount) return KFVM_ERR_ARG;
  if (!ctx->weights_built) return KFVM_ERR_STATE;
  std::memcpy(host, ctx->w_host.data(), sizeof(double) * count);
  return KFVM_OK;
}

kfvm_status kfvm_set_option(kfvm_ctx* ctx, const char* key, double v) {
  if (!ctx || !key) return KFVM_ERR_ARG;
  std::string k(key);
  if (k == "precision") {
    if (v != 64 && v != 32) return KFVM_ERR_ARG;
    ctx->precision = (int)v;
  } else if (k == "recon") {
    if (v != 0 && v != 1 && v != 2 && v != 4) return KFVM_ERR_ARG;
    ctx->recon = (int)v;
  } else if (k == "riemann") {
    if (v != 0 && v != 1) return KFVM_ERR_ARG;
    ctx->riemann = (int)v;
  } else if (k == "positivity") {
    if (v != 0 && v != 1) return KFVM_ERR_ARG;
    ctx->positivity = (int)v;
  } else if (k == "kappa") {
    if (!(v >= 0 && v < 1)) return KFVM_ERR_ARG;
    ctx->kappa = v;
  } else if (k == "eta") {
    if (!(v >= 0 && v <= 1)) return KFVM_ERR_ARG;
    ctx->eta = v;
  } else if (k == "eps") {
    if (!(v > 0)) return KFVM_ERR_ARG;
    ctx->eps = v;
  } else if (k == "tensor_cores") {
    if (v != 0 && v != 1) return KFVM_ERR_ARG;
    ctx->tensor_cores = (int)v;
  } else if (k == "timeout_probe") {
    if (v != 0 && v != 1) return KFVM_ERR_ARG;
    ctx->timeout_probe = (int)v;
  } else if (k == "slab_planes") {
    // split 3D steps into z-slabs of this many planes (at most what the buffer holds)
    if (!(v >= 1) || ctx->dims != 3) return KFVM_ERR_ARG;
    ctx->slab_user = v < ctx->n[2] ? (int)v : ctx->n[2];
  } else if (k == "profile") {
    if (v != 0 && v != 1) return KFVM_ERR_ARG;
    ctx->profile = (int)v;
  } else if (k == "variables") {
    if (v != 0 && v != 1) return KFVM_ERR_ARG;
    ctx->vars = (int)v;
  } else if (k == "kxrcf_m") {
    if (!(v > 0 && v <= 16)) return KFVM_ERR_ARG;
    ctx->kxrcf_m = v;
  } else if (k == "gate_threshold") {
    if (!(v > 0 && v < 1)) return KFVM_ERR_ARG;
    ctx->gate_threshold = v;
  } else {
    return KFVM_ERR_ARG;
  }
  return KFVM_OK;
}

kfvm_status kfvm_reconstruct(kfvm_ctx* ctx, const double* U, void* faces, void* stream) {
  kfvm_status s = check_ready(ctx);
  if (s) return s;
  if (!U || !faces) return KFVM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (ctx->precision == 64) {
    if (ctx->recon == 2) KFVM_LAUNCH(ctx, kProfGateMask, st, launch_gate_mask(ctx, U, nullptr, st));
    if (ctx->recon == 4) KFVM_LAUNCH(ctx, kProfKxrcf, st, launch_kxrcf(ctx, U, nullptr, ctx->d_gate_mask, st));
    KFVM_LAUNCH(ctx, kProfRecon64, st, launch_recon64(ctx, U, (double*)faces, st));
  } else {
    KFVM_LAUNCH(ctx, kProfShadow, st, launch_shadow(ctx, U, ctx->d_shadow, st));
    if (ctx->recon == 4)
      KFVM_LAUNCH(ctx, kProfKxrcf, st, launch_kxrcf(ctx, U, ctx->d_shadow, ctx->d_gate_mask, st));
    // the FP32 reconstruction evaluates the learned gate itself (fused)
    KFVM_LAUNCH(ctx, kProfRecon32, st, launch_recon32(ctx, U, ctx->d_shadow, (float*)faces, st));
  }
  return KFVM_OK;
}

kfvm_status kfvm_flux(kfvm_ctx* ctx, const void* faces, double* dUdt, void* stream) {
  kfvm_status s = check_ready(ctx);
  if (s) return s;
  if (!faces || !dUdt) return KFVM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  KFVM_LAUNCH(ctx, kProfUpdate, st, launch_flux_update(ctx, 0, faces, nullptr, nullptr, dUdt, st));
  return KFVM_OK;
}

namespace {

// One RK stage (or, with stage 0, dUdt) over the grid, in z-slabs when the step was sized for them:
// Riemann states of the planes zc_lo - 1 .. zc_hi (wrapped or skipped at the ends), then the fused
// flux divergence / stage update of the planes zc_lo .. zc_hi - 1.
kfvm_status stage_pass(kfvm_ctx* ctx, int stage, const double* in, const double* U0, double* out,
                       const float* shadow_in, float* shadow_out, cudaStream_t st) {
  const bool fp32 = ctx->precision == 32;
  const int nz = ctx->n[2], S = slab_planes(ctx);
  const bool multi = ctx->dims == 3 && S < nz;
  for (int z0 = 0; z0 < (multi ? nz : 1); z0 += (multi ? S : 1)) {
    const int zc_lo = multi ? z0 : 0, zc_hi = multi ? (z0 + S < nz ? z0 + S : nz) : 0;
    const int zf_first = multi ? z0 - 1 : 0, zf_count = multi ? zc_hi - zc_lo + 2 : 0;
    if (fp32)
      KFVM_LAUNCH(ctx, kProfRecon32, st,
                  launch_recon32(ctx, in, shadow_in, (float*)ctx->d_faces, st, zf_first, zf_count));
    else
      KFVM_LAUNCH(ctx, kProfRecon64, st, launch_recon64(ctx, in, (double*)ctx->d_faces, st, zf_first, zf_count));
    KFVM_LAUNCH(ctx, kProfUpdate, st,
                launch_flux_update(ctx, stage, ctx->d_faces, U0, in, out, st, shadow_out, zc_lo, zc_hi, zf_first,
                                   zf_count));
  }
  return KFVM_OK;
}

kfvm_status ensure_slab_buffers(kfvm_ctx* ctx) {
  if (!(ctx->dims == 3 && slab_planes(ctx) < ctx->n[2])) return KFVM_OK;
  const size_t n = (size_t)ctx->nv * ctx->ncell;
  if (!ctx->d_stage2) KFVM_TRY(cudaMalloc(&ctx->d_stage2, sizeof(double) * n));
  if (!ctx->d_shadow2) KFVM_TRY(cudaMalloc(&ctx->d_shadow2, sizeof(float) * n));
  return KFVM_OK;
}

}  // namespace

kfvm_status kfvm_rhs(kfvm_ctx* ctx, const double* U, double* dUdt, void* stream) {
  kfvm_status s = check_ready(ctx);
  if (s) return s;
  if (!U || !dUdt) return KFVM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (ctx->precision == 64) {
    if (ctx->recon == 2) KFVM_LAUNCH(ctx, kProfGateMask, st, launch_gate_mask(ctx, U, nullptr, st));
    if (ctx->recon == 4) KFVM_LAUNCH(ctx, kProfKxrcf, st, launch_kxrcf(ctx, U, nullptr, ctx->d_gate_mask, st));
  } else {
    KFVM_LAUNCH(ctx, kProfShadow, st, launch_shadow(ctx, U, ctx->d_shadow, st));
    if (ctx->recon == 4)
      KFVM_LAUNCH(ctx, kProfKxrcf, st, launch_kxrcf(ctx, U, ctx->d_shadow, ctx->d_gate_mask, st));
  }
  return stage_pass(ctx, 0, U, nullptr, dUdt, ctx->d_shadow, nullptr, st);
}

kfvm_status kfvm_step(kfvm_ctx* ctx, double* U, double cfl, double t_remaining, double* dt_out, void* stream) {
  kfvm_status s = check_ready(ctx);
  if (s) return s;
  if (!U || !(cfl > 0) || !(t_remaining > 0)) return KFVM_ERR_ARG;
  if (U == ctx->d_stage || U == ctx->d_stage2) return KFVM_ERR_ARG;
  s = ensure_slab_buffers(ctx);
  if (s) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const bool fp32 = ctx->precision == 32;
  const bool multi = ctx->dims == 3 && slab_planes(ctx) < ctx->n[2];
  // dt from U (and, in the FP32 mode, the float32 shadow of U for the first stage)
  KFVM_LAUNCH(ctx, kProfMaxRate, st, launch_max_rate(ctx, U, cfl, t_remaining, st));
  // Shu-Osher stages; with slabs no stage writes the state its own reconstruction still reads
  double* A = ctx->d_stage;
  double* B = multi ? ctx->d_stage2 : ctx->d_stage;
  float* s0 = ctx->d_shadow;
  float* s1 = multi ? ctx->d_shadow2 : ctx->d_shadow;
  const double* in[3] = {U, A, B};
  double* outp[3] = {A, B, U};
  const float* sh_in[3] = {s0, s1, s0};
  float* sh_out[3] = {s1, s0, nullptr};
  for (int k = 0; k < 3; ++k) {
    if (ctx->recon == 2 && !fp32)  // the FP32 reconstruction evaluates the gate itself
      KFVM_LAUNCH(ctx, kProfGateMask, st, launch_gate_mask(ctx, in[k], nullptr, st));
    if (ctx->recon == 4)  // the indicator of this stage's input state, for the whole grid
      KFVM_LAUNCH(ctx, kProfKxrcf, st, launch_kxrcf(ctx, in[k], fp32 ? sh_in[k] : nullptr, ctx->d_gate_mask, st));
    s = stage_pass(ctx, k + 1, in[k], U, outp[k], sh_in[k], sh_out[k], st);
    if (s) return s;
  }
  if (dt_out) {
    KFVM_TRY(cudaMemcpyAsync(dt_out, &ctx->d_scalars->dt, sizeof(double), cudaMemcpyDeviceToHost, st));
    return kfvm_sync_status(ctx, stream);
  }
  return KFVM_OK;
}

kfvm_status kfvm_kxrcf_mask(kfvm_ctx* ctx, const double* U, unsigned char* mask_out, void* stream) {
  if (!ctx || !U || !mask_out) return KFVM_ERR_ARG;
  if (!ctx->weights_built) return KFVM_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  if (ctx->precision == 32) {
    KFVM_LAUNCH(ctx, kProfShadow, st, launch_shadow(ctx, U, ctx->d_shadow, st));
    KFVM_LAUNCH(ctx, kProfKxrcf, st, launch_kxrcf(ctx, U, ctx->d_shadow, mask_out, st));
  } else {
    KFVM_LAUNCH(ctx, kProfKxrcf, st, launch_kxrcf(ctx, U, nullptr, mask_out, st));
  }
  return KFVM_OK;
}

kfvm_status kfvm_sync_status(kfvm_ctx* ctx, void* stream) {
  if (!ctx) return KFVM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int h = 0;
  KFVM_TRY(cudaMemcpyAsync(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  KFVM_TRY(cudaStreamSynchronize(st));
  if (h) KFVM_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
  KFVM_TRY(cudaStreamSynchronize(st));
  if (h & kFlagNonphysical) return KFVM_ERR_NONPHYSICAL;
  if (h & kFlagTimeout) return KFVM_ERR_TIMEOUT;
  return KFVM_OK;
}

int kfvm_profile_count(void) { return kProfCount; }

kfvm_status kfvm_profile_get(kfvm_ctx* ctx, int index, const char** name, long long* launches, double* ms) {
  static const char* names[kProfCount] = {"max_rate", "recon64", "recon32", "face_flux", "flux_update",
                                          "gate_mask", "shadow", "kxrcf"};
  if (!ctx || index < 0 || index >= kProfCount) return KFVM_ERR_ARG;
  const bool done = prof_fold(ctx);
  if (name) *name = names[index];
  if (launches) *launches = ctx->prof_launches[index];
  if (ms) *ms = ctx->prof_ms[index];
  return done ? KFVM_OK : KFVM_ERR_CUDA;
}

kfvm_status kfvm_profile_reset(kfvm_ctx* ctx) {
  if (!ctx) return KFVM_ERR_ARG;
  prof_fold(ctx);
  for (const ProfPair& p : ctx->prof_pairs) {
    ctx->prof_free.push_back(p.start);
    ctx->prof_free.push_back(p.stop);
  }
  ctx->prof_pairs.clear();
  for (int i = 0; i < kProfCount; ++i) {
    ctx->prof_launches[i] = 0;
    ctx->prof_ms[i] = 0.0;
  }
  return KFVM_OK;
}

kfvm_status kfvm_measure_fma_peak(int bits, double* flops) {
  if (!flops || (bits != 32 && bits != 64)) return KFVM_ERR_ARG;
  KFVM_TRY(fma_peak(bits, flops));
  return KFVM_OK;
}

}  // extern "C"
