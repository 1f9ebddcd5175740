// weights.cu -- K0: the reconstruction and derivative vectors of every
// (sub)stencil, solved once on the GPU in double-double arithmetic.
//
// For stencil q with N cells (unit cells, Sec. 3.1) and D monomials of total
// degree <= p_q, one CTA assembles the (N + D) x (N + D) saddle-point matrix
//   [[Q^T, P], [P^T, 0]]                                   (Eq. 14)
// with Q_hl = lambda_h K(., x_l) (Eq. 7), the cell average of the squared
// exponential kernel K(x, y) = exp(-|x - y|^2 / (2 ell^2)) (Eq. 6; a product of
// 1D integrals ell sqrt(pi/2) [erf((d + 1/2)/(sqrt2 ell)) - erf((d - 1/2)/(sqrt2 ell))]),
// P_hv = lambda_h x^alpha_v (Eq. 8), and the right-hand sides
//   T_l = K(x_s, x_l), S_v = x_s^alpha_v                   (Eqs. 12-13)
// for every face Gauss point x_s, and
//   D_l = d^alpha K(x, x_l)|_0, S_v = d^alpha x^alpha_v|_0  (Eq. 23)
// for every indicator multi-index 0 < |alpha| <= R (1D factors through the
// probabilists' Hermite polynomials: d^n/dx^n exp(-t^2/2) with t = (x - c)/ell
// equals (-1)^n ell^-n He_n(t) exp(-t^2/2)).  Gaussian elimination with
// partial pivoting runs in double-double in global scratch; the solutions r
// (the first N unknowns) are rounded to float64.  The conditioning (up to
// ~1e17 for d = 3, R = 3) is why double precision alone is not enough.
#include <cuda_runtime.h>

#include <vector>

#include "dd.cuh"
#include "internal.h"

namespace kfvm {
namespace {

struct StencilJob {
  int N, Dm;          // cells, monomials
  int off_start;      // index into ints (3 per cell)
  int mon_start;      // index into ints (3 per monomial)
  int wout;           // offset of this stencil's block in the weight table
  long long scratch;  // offset (in dd elements) of this job's matrix + rhs in scratch
};

constexpr int kThreads = 256;

__device__ dd gl_node(int R, int i) {
  // Gauss-Legendre nodes on [-1/2, 1/2], ascending.
  if (R == 2) {
    dd a = dd_sqrt(dd_make(3.0)) / dd_make(6.0);
    return i == 0 ? -a : a;
  }
  dd a = dd_sqrt(dd_make(15.0)) / dd_make(10.0);
  return i == 0 ? -a : (i == 1 ? dd_make(0.0) : a);
}

__device__ dd dd_powi(dd x, int a) {
  dd r = dd_make(1.0);
  for (int i = 0; i < a; ++i) r = r * x;
  return r;
}

__global__ void __launch_bounds__(kThreads) build_weights_kernel(const StencilJob* jobs, const int* ints,
                                                                   const int* ders, int dim, int R, double ell_d,
                                                                   int F, int M, dd* scratch, double* wout,
                                                                   int* err) {
  const StencilJob job = jobs[blockIdx.x];
  const int N = job.N, Dm = job.Dm, n = N + Dm, nr = F + M;
  const int* offs = ints + job.off_start;
  const int* mons = ints + job.mon_start;
  dd* A = scratch + job.scratch;  // n x n
  dd* B = A + (long long)n * n;   // n x nr
  const int tid = threadIdx.x;

  __shared__ dd s_pts[54][3];      // face points
  __shared__ dd s_I[13];           // 1D cell integrals, offset difference -6..6
  __shared__ dd s_K[4][7];         // 1D kernel derivatives: order 0..3, centre -3..3
  __shared__ dd s_f[192];          // elimination factors of one step
  __shared__ double s_best[kThreads / 32];
  __shared__ int s_bidx[kThreads / 32];
  __shared__ int s_piv;

  const dd ell = dd_make(ell_d);
  const dd sq2l = dd_sqrt(dd_make(2.0)) * ell;
  if (tid < 13) {
    const int d = tid - 6;
    dd lo = dd_erf((dd_make((double)d) - dd_make(0.5)) / sq2l);
    dd hi = dd_erf((dd_make((double)d) + dd_make(0.5)) / sq2l);
    s_I[tid] = ell * dd_sqrt(dd_pi() / dd_make(2.0)) * (hi - lo);
  } else if (tid >= 32 && tid < 32 + 28) {
    const int a = (tid - 32) / 7, c = (tid - 32) % 7 - 3;
    if (a <= R) {
      dd t = -(dd_make((double)c) / ell);
      // He_a(t)
      dd h0 = dd_make(1.0), h1 = t;
      dd he = a == 0 ? h0 : h1;
      for (int k = 1; k < a; ++k) {
        dd h2 = t * h1 - h0 * (double)k;
        h0 = h1;
        h1 = h2;
        he = h2;
      }
      dd val = he * dd_exp(-(t * t) * 0.5) / dd_powi(ell, a);
      s_K[a][c + 3] = (a & 1) ? -val : val;
    }
  } else if (tid >= 64 && tid < 64 + F) {
    const int s = tid - 64, nt = dim == 2 ? R : R * R, dir = s / (2 * nt), side = (s / nt) % 2, t = s % nt;
    int tr[2], m = 0;
    for (int a = 0; a < dim; ++a)
      if (a != dir) tr[m++] = a;
    for (int a = 0; a < 3; ++a) s_pts[s][a] = dd_make(0.0);
    s_pts[s][dir] = dd_make(side ? 0.5 : -0.5);
    s_pts[s][tr[0]] = gl_node(R, t % R);
    if (dim == 3) s_pts[s][tr[1]] = gl_node(R, t / R);
  }
  __syncthreads();

  // ---- assemble the matrix ----
  for (long long e = tid; e < (long long)n * n; e += kThreads) {
    const int row = (int)(e / n), col = (int)(e % n);
    dd v = dd_make(0.0);
    if (row < N && col < N) {
      v = dd_make(1.0);  // (Q^T)_{row,col} = Q_{col,row} = prod_k I(off_col - off_row)
      for (int k = 0; k < dim; ++k) v = v * s_I[offs[3 * col + k] - offs[3 * row + k] + 6];
    } else if (row < N || col < N) {
      const int h = row < N ? row : col, vv = row < N ? col - N : row - N;
      v = dd_make(1.0);
      for (int k = 0; k < dim; ++k) {
        const int o = offs[3 * h + k], a = mons[3 * vv + k];
        double hi = 1.0, lo = 1.0;  // (o+1/2)^(a+1), (o-1/2)^(a+1): exact dyadic rationals
        for (int i = 0; i <= a; ++i) { hi *= (o + 0.5); lo *= (o - 0.5); }
        v = v * (dd_make(hi - lo) / dd_make((double)(a + 1)));
      }
    }
    A[e] = v;
  }
  // ---- assemble the right-hand sides ----
  const double inv2l2 = 1.0 / (2.0 * ell_d * ell_d);  // exact for ell = 5 (1/50 is not, so use dd below)
  (void)inv2l2;
  const dd two_l2 = dd_make(2.0) * ell * ell;
  for (long long e = tid; e < (long long)n * nr; e += kThreads) {
    const int row = (int)(e / nr), col = (int)(e % nr);
    dd v = dd_make(0.0);
    if (col < F) {
      if (row < N) {
        dd r2 = dd_make(0.0);
        for (int k = 0; k < dim; ++k) {
          dd d = s_pts[col][k] - dd_make((double)offs[3 * row + k]);
          r2 = r2 + d * d;
        }
        v = dd_exp(-(r2 / two_l2));
      } else {
        v = dd_make(1.0);
        for (int k = 0; k < dim; ++k) v = v * dd_powi(s_pts[col][k], mons[3 * (row - N) + k]);
      }
    } else {
      const int* a = ders + 3 * (col - F);
      if (row < N) {
        v = dd_make(1.0);
        for (int k = 0; k < dim; ++k) v = v * s_K[a[k]][offs[3 * row + k] + 3];
      } else {
        const int* b = mons + 3 * (row - N);
        bool same = true;
        double fact = 1.0;
        for (int k = 0; k < dim; ++k) {
          if (a[k] != b[k]) same = false;
          for (int i = 2; i <= a[k]; ++i) fact *= i;
        }
        v = dd_make(same ? fact : 0.0);
      }
    }
    B[e] = v;
  }
  __syncthreads();

  // ---- Gaussian elimination with partial pivoting ----
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bidx = k;
    for (int i = k + tid; i < n; i += kThreads) {
      double a = fabs(A[(long long)i * n + k].hi);
      if (a > best) { best = a; bidx = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_down_sync(0xffffffffu, best, o);
      int oi = __shfl_down_sync(0xffffffffu, bidx, o);
      if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    if ((tid & 31) == 0) { s_best[tid >> 5] = best; s_bidx[tid >> 5] = bidx; }
    __syncthreads();
    if (tid == 0) {
      double b = s_best[0];
      int bi = s_bidx[0];
      for (int w = 1; w < kThreads / 32; ++w)
        if (s_best[w] > b || (s_best[w] == b && s_bidx[w] < bi)) { b = s_best[w]; bi = s_bidx[w]; }
      s_piv = (b > 0.0) ? bi : -1;
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv < 0) {
      if (tid == 0) atomicOr(err, 1);
      return;  // uniform across the block
    }
    if (piv != k) {
      for (int j = tid; j < n; j += kThreads) {
        dd t = A[(long long)k * n + j];
        A[(long long)k * n + j] = A[(long long)piv * n + j];
        A[(long long)piv * n + j] = t;
      }
      for (int j = tid; j < nr; j += kThreads) {
        dd t = B[(long long)k * nr + j];
        B[(long long)k * nr + j] = B[(long long)piv * nr + j];
        B[(long long)piv * nr + j] = t;
      }
    }
    __syncthreads();
    const dd akk = A[(long long)k * n + k];
    for (int i = k + 1 + tid; i < n; i += kThreads) s_f[i - k - 1] = A[(long long)i * n + k] / akk;
    __syncthreads();
    const int rows = n - k - 1, wa = n - k - 1, wb = nr;
    for (long long e = tid; e < (long long)rows * (wa + wb); e += kThreads) {
      const int ii = (int)(e / (wa + wb)), jj = (int)(e % (wa + wb));
      const dd f = s_f[ii];
      if (f.hi == 0.0) continue;
      const int i = k + 1 + ii;
      if (jj < wa) {
        const int j = k + 1 + jj;
        A[(long long)i * n + j] = A[(long long)i * n + j] - f * A[(long long)k * n + j];
      } else {
        const int j = jj - wa;
        B[(long long)i * nr + j] = B[(long long)i * nr + j] - f * B[(long long)k * nr + j];
      }
    }
    __syncthreads();
  }
  // ---- back substitution, one right-hand side per thread ----
  for (int r = tid; r < nr; r += kThreads) {
    for (int k = n - 1; k >= 0; --k) {
      dd x = B[(long long)k * nr + r];
      for (int i = k + 1; i < n; ++i) x = x - A[(long long)k * n + i] * B[(long long)i * nr + r];
      B[(long long)k * nr + r] = x / A[(long long)k * n + k];
    }
    double* w = wout + job.wout;
    for (int l = 0; l < N; ++l) {
      const dd v = B[(long long)l * nr + r];
      const double rounded = v.hi + v.lo;  // nearest double of the double-double value
      if (r < F)
        w[r * N + l] = rounded;
      else
        w[F * N + (r - F) * N + l] = rounded;
    }
  }
}

}  // namespace

cudaError_t launch_build_weights(kfvm_ctx* ctx, cudaStream_t st, int* d_err) {
  const StencilTable t = make_stencil(ctx->dims, ctx->R);
  std::vector<StencilJob> jobs;
  std::vector<int> ints;
  // derivative multi-indices 0 < |alpha| <= R, by total degree then alpha_x descending
  std::vector<int> ders;
  for (int nn = 1; nn <= ctx->R; ++nn) {
    if (ctx->dims == 2) {
      for (int a = nn; a >= 0; --a) { ders.push_back(a); ders.push_back(nn - a); ders.push_back(0); }
    } else {
      for (int a = nn; a >= 0; --a)
        for (int b = nn - a; b >= 0; --b) { ders.push_back(a); ders.push_back(b); ders.push_back(nn - a - b); }
    }
  }
  long long scratch = 0;
  int wout = 0;
  for (int q = 0; q < t.nq; ++q) {
    StencilJob j{};
    j.N = t.len[q];
    j.off_start = (int)ints.size();
    for (int l = 0; l < t.len[q]; ++l)
      for (int k = 0; k < 3; ++k) ints.push_back(t.off[t.idx[q][l]][k]);
    j.mon_start = (int)ints.size();
    const int p = ctx->degrees[q];
    int Dm = 0;
    for (int nn = 0; nn <= p; ++nn) {
      if (ctx->dims == 2) {
        for (int a = nn; a >= 0; --a) { ints.push_back(a); ints.push_back(nn - a); ints.push_back(0); ++Dm; }
      } else {
        for (int a = nn; a >= 0; --a)
          for (int b = nn - a; b >= 0; --b) {
            ints.push_back(a); ints.push_back(b); ints.push_back(nn - a - b); ++Dm;
          }
      }
    }
    j.Dm = Dm;
    j.wout = wout;
    j.scratch = scratch;
    const long long n = j.N + Dm;
    scratch += n * n + n * (ctx->F + ctx->M);
    wout += t.len[q] * (ctx->F + ctx->M);
    jobs.push_back(j);
  }
  StencilJob* d_jobs = nullptr;
  int* d_ints = nullptr;
  int* d_ders = nullptr;
  dd* d_scratch = nullptr;
  cudaError_t e = cudaMalloc(&d_jobs, sizeof(StencilJob) * jobs.size());
  if (e == cudaSuccess) e = cudaMalloc(&d_ints, sizeof(int) * ints.size());
  if (e == cudaSuccess) e = cudaMalloc(&d_ders, sizeof(int) * ders.size());
  if (e == cudaSuccess) e = cudaMalloc(&d_scratch, sizeof(dd) * scratch);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(StencilJob) * jobs.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_ints, ints.data(), sizeof(int) * ints.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_ders, ders.data(), sizeof(int) * ders.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    build_weights_kernel<<<(unsigned)jobs.size(), kThreads, 0, st>>>(d_jobs, d_ints, d_ders, ctx->dims, ctx->R,
                                                                      ctx->ell, ctx->F, ctx->M, d_scratch,
                                                                      ctx->d_w64, d_err);
    ctx->launches += 1;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_jobs);
  cudaFree(d_ints);
  cudaFree(d_ders);
  cudaFree(d_scratch);
  return e;
}

}  // namespace kfvm
