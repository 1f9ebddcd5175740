// geometry.h -- compile-time stencil geometry of KFVM-WENO (host and device).
//
// Sec. 3.1 of May & Lee (arXiv 2401.16543): the full stencil
// S0 = {o in Z^d : |o|^2 <= R^2} around the reconstruction cell, the central
// substencil S1 of radius R-1 and 2d biased substencils (2D: |j| <= i,
// |j| <= -i, |i| <= j, |i| <= -j; 3D: both transverse offsets bounded by the
// biased one).  Cells with |j| = i belong to two biased substencils, as the
// paper's "<=" conditions say.  S0 is enumerated z-outer, x-fastest; each
// substencil is an ascending list of indices into S0.
//
// Face Gauss points (Sec. 5.1): R Gauss-Legendre points per face dimension on
// each of the 2d faces, F = 2d R^(d-1); point s = (dir*2+side)*R^(d-1) + t.
// Derivative multi-indices of the smoothness indicator (Eq. 22 with p = R):
// 0 < |alpha| <= R, by total degree then alpha_x descending; M of them.
#pragma once

#ifdef __CUDACC__
#define KFVM_HD __host__ __device__
#else
#define KFVM_HD
#endif

namespace kfvm {

constexpr int kMaxN0 = 123;  // |S0| for d = 3, R = 3
constexpr int kMaxNQ = 8;    // N_S + 1 for d = 3

struct StencilTable {
  int n0;
  int off[kMaxN0][3];
  int nq;
  int len[kMaxNQ];
  int idx[kMaxNQ][kMaxN0];
};

KFVM_HD constexpr bool in_sub(int dim, int R, int q, int i, int j, int k) {
  auto ab = [](int v) { return v < 0 ? -v : v; };
  if (q == 0) return true;
  if (q == 1) return i * i + j * j + k * k <= (R - 1) * (R - 1);
  if (dim == 2) {
    switch (q) {
      case 2: return ab(j) <= i;
      case 3: return ab(j) <= -i;
      case 4: return ab(i) <= j;
      default: return ab(i) <= -j;
    }
  }
  switch (q) {
    case 2: return ab(j) <= i && ab(k) <= i;
    case 3: return ab(j) <= -i && ab(k) <= -i;
    case 4: return ab(i) <= j && ab(k) <= j;
    case 5: return ab(i) <= -j && ab(k) <= -j;
    case 6: return ab(i) <= k && ab(j) <= k;
    default: return ab(i) <= -k && ab(j) <= -k;
  }
}

KFVM_HD constexpr StencilTable make_stencil(int dim, int R) {
  StencilTable t{};
  t.n0 = 0;
  const int kr = dim == 3 ? R : 0;
  for (int k = -kr; k <= kr; ++k)
    for (int j = -R; j <= R; ++j)
      for (int i = -R; i <= R; ++i)
        if (i * i + j * j + k * k <= R * R) {
          t.off[t.n0][0] = i;
          t.off[t.n0][1] = j;
          t.off[t.n0][2] = k;
          ++t.n0;
        }
  t.nq = 2 * dim + 2;
  for (int q = 0; q < t.nq; ++q) {
    t.len[q] = 0;
    for (int l = 0; l < t.n0; ++l)
      if (in_sub(dim, R, q, t.off[l][0], t.off[l][1], t.off[l][2])) t.idx[q][t.len[q]++] = l;
  }
  return t;
}

KFVM_HD constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }
KFVM_HD constexpr int binom(int n, int k) { return k == 0 ? 1 : binom(n - 1, k - 1) * n / k; }

// number of multi-indices with 0 < |alpha| <= p in dim dimensions
KFVM_HD constexpr int n_multi(int dim, int p) { return binom(p + dim, dim) - 1; }

// A small array usable in device code through a local constexpr copy.
struct IntArr {
  int v[kMaxN0 + 1];
};

template <int D, int R>
struct Geo {
  static constexpr StencilTable tab = make_stencil(D, R);
  static constexpr int NV = D + 2;
  static constexpr int N0 = tab.n0;
  static constexpr int NQ = 2 * D + 2;
  static constexpr int NT = ipow(R, D - 1);  // Gauss points per face
  static constexpr int F = 2 * D * NT;       // face points per cell
  static constexpr int M = n_multi(D, R);    // derivatives of the indicator
  KFVM_HD static constexpr int len(int q) { return tab.len[q]; }
  // offset of stencil q's block in the packed weight table
  KFVM_HD static constexpr int woff(int q) { return q == 0 ? 0 : woff(q - 1) + tab.len[q - 1] * (F + M); }
  static constexpr int WCOUNT = woff(NQ);
  KFVM_HD static constexpr IntArr make_woffs() {
    IntArr a{};
    for (int q = 0; q <= NQ; ++q) a.v[q] = woff(q);
    return a;
  }
  // device code reads these through `constexpr auto x = Geo<D,R>::woffs;`
  static constexpr IntArr woffs = make_woffs();
  // index of the central cell in S0
  KFVM_HD static constexpr int center() {
    int c = -1;
    for (int l = 0; l < tab.n0; ++l)
      if (tab.off[l][0] == 0 && tab.off[l][1] == 0 && tab.off[l][2] == 0) c = l;
    return c;
  }
};

}  // namespace kfvm
