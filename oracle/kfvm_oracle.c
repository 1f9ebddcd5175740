/*
 * kfvm_oracle.c -- the plain, slow CPU oracle of the KFVM-WENO hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code with
 * the CUDA path (no headers, helpers or tables) and must never serve as a
 * fallback for it.
 *
 * What it computes follows May & Lee, "KFVM-WENO: a high-order accurate
 * kernel-based finite volume method for compressible hydrodynamics"
 * (arXiv 2401.16543), step by step, one cell at a time, with no blocking,
 * fusion or reordering:
 *
 *   kfo_weights      Sec. 2.1 Eqs. (6)-(18): reconstruction vectors r from the
 *                    saddle-point system [[Q^T, P], [P^T, 0]] [r; w] = [T; S]
 *                    for every face Gauss point, and the derivative version of
 *                    Sec. 3.3 (sample vector D, Eq. 23) for every multi-index
 *                    0 < |alpha| <= R.  Solved in binary128 by Gaussian
 *                    elimination with partial pivoting, then rounded to double
 *                    (the system is ill-conditioned: cond up to ~1e17, so the
 *                    canonical weights are the high-precision solution).
 *   kfo_reconstruct  Sec. 3 and Sec. 5.3: linearized primitive transform
 *                    (Eqs. 27-33, appendix A with the corrected energy row of
 *                    Phi^{-1}), contractions with r for S0 and all substencils,
 *                    smoothness indicators beta_q = sum (d_q(alpha).g_q)^2 in
 *                    unit-cell coordinates (Eq. 22, read without the Delta
 *                    factors), nonlinear weights omega = gamma/(beta^2+eps)
 *                    normalised (Eqs. 24-25), WENO-AO blend (Eq. 19), back
 *                    transform (Eq. 28).  Mode 1 is the unlimited linear S0
 *                    reconstruction of the conservative variables.
 *   kfo_char         Sec. 3.4.1: characteristic variables of one direction,
 *                    Phi = L and Phi^{-1} = R from the eigenvectors of the
 *                    flux Jacobian at the central cell average; with them
 *                    the WENO-AO weights are computed once per direction and
 *                    serve only that direction's faces.
 *   kfo_kxrcf        Sec. 3.5 and Sec. 5.3 step 2 items 1-2: the KXRCF
 *                    troubled-cell indicator on the unlimited linear states,
 *                    which decides per cell between the linear and the WENO-AO
 *                    reconstruction (recon mode 3).
 *   kfo_limit        Sec. 4 (Sec. 5.3 step 3): positivity-preserving limiter of
 *                    the Riemann states with data-dependent density and
 *                    pressure bounds; theta_p by bisection.
 *   kfo_flux         Sec. 5.3 steps 4-6: exterior states at physical
 *                    boundaries (periodic: neighbour; outflow: copy of the
 *                    interior state), HLLC (Toro) or HLL with Batten wave
 *                    speeds at every face Gauss point, Gauss-Legendre face
 *                    integration and the flux divergence of Eq. (1).
 *   kfo_step         SSP-RK3 (Shu-Osher) with dt = CFL / max_cells
 *                    sum_d (|u_d| + c)/Delta_d, clipped to the time left.
 *
 * Threads: compiled as it is (the checker library) everything runs on one
 * thread.  The cell loops carry OpenMP work-sharing pragmas that only the
 * separate timing build (-fopenmp, used for the all-core CPU baseline) turns
 * on; every cell is still computed by the same statements in the same order,
 * so both builds give the same bits.
 *
 * Layouts: the state is SoA [var][z][y][x] (x fastest).  Face states are
 * [point][var][cell] with point = (dir*2 + side)*R^(dim-1) + t, side 0 the
 * low face (x_dir = -1/2), t = t0 + R*t1 over the transverse axes in
 * increasing order, Gauss-Legendre nodes ascending.
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#define KFO_MAX_THREADS() omp_get_max_threads()
#define KFO_THREAD() omp_get_thread_num()
#else
#define KFO_MAX_THREADS() 1
#define KFO_THREAD() 0
#endif

#if defined(__aarch64__) && (LDBL_MANT_DIG == 113)
typedef long double qreal;
static qreal q_erf(qreal x) { return erfl(x); }
static qreal q_exp(qreal x) { return expl(x); }
static qreal q_sqrt(qreal x) { return sqrtl(x); }
static qreal q_abs(qreal x) { return fabsl(x); }
#define QPI 3.141592653589793238462643383279502884L
#else
#include <quadmath.h>
typedef __float128 qreal;
static qreal q_erf(qreal x) { return erfq(x); }
static qreal q_exp(qreal x) { return expq(x); }
static qreal q_sqrt(qreal x) { return sqrtq(x); }
static qreal q_abs(qreal x) { return fabsq(x); }
#define QPI M_PIq
#endif

enum { KFO_OK = 0, KFO_ERR_ARG = 1, KFO_ERR_SINGULAR = 3, KFO_ERR_NONPHYSICAL = 4, KFO_ERR_NOMEM = 7 };

/* ------------------------------------------------------------------------- */
/* Gauss-Legendre rule on [-1/2, 1/2] with weights summing to one.           */
/* ------------------------------------------------------------------------- */
static int gl_nodes_q(int R, qreal* x) {
  if (R == 1) { x[0] = 0; return 0; }
  if (R == 2) { qreal a = q_sqrt((qreal)3) / 6; x[0] = -a; x[1] = a; return 0; }
  if (R == 3) { qreal a = q_sqrt((qreal)15) / 10; x[0] = -a; x[1] = 0; x[2] = a; return 0; }
  return -1;
}

int kfo_gl_weights(int R, double* w) {
  if (R == 1) { w[0] = 1.0; return 0; }
  if (R == 2) { w[0] = 0.5; w[1] = 0.5; return 0; }
  if (R == 3) { w[0] = 5.0 / 18.0; w[1] = 8.0 / 18.0; w[2] = 5.0 / 18.0; return 0; }
  return -1;
}

/* Face Gauss points in unit-cell coordinates, ordered as described above. */
static int face_points_q(int dim, int R, qreal* pts /* F x 3 */) {
  qreal node[3];
  if (gl_nodes_q(R, node)) return -1;
  int nt = (dim == 2) ? R : R * R;
  int s = 0;
  for (int dir = 0; dir < dim; ++dir) {
    int tr[2], m = 0;
    for (int a = 0; a < dim; ++a) if (a != dir) tr[m++] = a;
    for (int side = 0; side < 2; ++side) {
      for (int t = 0; t < nt; ++t) {
        qreal* x = pts + 3 * s;
        x[0] = x[1] = x[2] = 0;
        x[dir] = side ? (qreal)0.5 : (qreal)-0.5;
        x[tr[0]] = node[t % R];
        if (dim == 3) x[tr[1]] = node[t / R];
        ++s;
      }
    }
  }
  return s;
}

int kfo_face_points(int dim, int R, double* pts) {
  qreal q[3 * 54];
  int n = face_points_q(dim, R, q);
  for (int i = 0; i < 3 * n; ++i) pts[i] = (double)q[i];
  return n;
}

/* ------------------------------------------------------------------------- */
/* Kernel integrals (Sec. 2.1, unit cells, length scale ell = ell/Delta).    */
/* ------------------------------------------------------------------------- */
/* int_{c-1/2}^{c+1/2} exp(-x^2/(2 ell^2)) dx, closed form through erf. */
static qreal cell_int_1d(int c, qreal ell) {
  qreal s = q_sqrt((qreal)2) * ell;
  return ell * q_sqrt(QPI / 2) * (q_erf(((qreal)c + (qreal)0.5) / s) - q_erf(((qreal)c - (qreal)0.5) / s));
}

/* x^a, a >= 0 */
static qreal qpow(qreal x, int a) {
  qreal r = 1;
  for (int i = 0; i < a; ++i) r *= x;
  return r;
}

/* cell average of x^a over [c-1/2, c+1/2] */
static qreal cell_avg_mono_1d(int c, int a) {
  return (qpow((qreal)c + (qreal)0.5, a + 1) - qpow((qreal)c - (qreal)0.5, a + 1)) / (qreal)(a + 1);
}

/* probabilists' Hermite polynomial He_n(t): He_0 = 1, He_1 = t, He_{n+1} = t He_n - n He_{n-1} */
static qreal hermite_e(int n, qreal t) {
  qreal h0 = 1, h1 = t;
  if (n == 0) return h0;
  for (int k = 1; k < n; ++k) {
    qreal h2 = t * h1 - (qreal)k * h0;
    h0 = h1;
    h1 = h2;
  }
  return h1;
}

/* d^n/dx^n exp(-(x-c)^2/(2 ell^2)) at x = 0:
   with t = (x-c)/ell, d^n/dx^n exp(-t^2/2) = (-1)^n ell^{-n} He_n(t) exp(-t^2/2). */
static qreal kernel_deriv_1d(int n, int c, qreal ell) {
  qreal t = -(qreal)c / ell;
  qreal sgn = (n % 2) ? -1 : 1;
  return sgn * hermite_e(n, t) * q_exp(-t * t / 2) / qpow(ell, n);
}

/* ------------------------------------------------------------------------- */
/* Dense Gaussian elimination with partial pivoting, multiple right sides.  */
/* ------------------------------------------------------------------------- */
static int solve_q(int n, qreal* A /* n x n row-major, destroyed */, int nrhs, qreal* B /* n x nrhs */) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    qreal best = q_abs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      qreal v = q_abs(A[i * n + k]);
      if (v > best) { best = v; piv = i; }
    }
    if (best == 0) return KFO_ERR_SINGULAR;
    if (piv != k) {
      for (int j = 0; j < n; ++j) { qreal t = A[k * n + j]; A[k * n + j] = A[piv * n + j]; A[piv * n + j] = t; }
      for (int j = 0; j < nrhs; ++j) { qreal t = B[k * nrhs + j]; B[k * nrhs + j] = B[piv * nrhs + j]; B[piv * nrhs + j] = t; }
    }
    for (int i = k + 1; i < n; ++i) {
      qreal f = A[i * n + k] / A[k * n + k];
      if (f == 0) continue;
      for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      for (int j = 0; j < nrhs; ++j) B[i * nrhs + j] -= f * B[k * nrhs + j];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    for (int j = 0; j < nrhs; ++j) {
      qreal s = B[k * nrhs + j];
      for (int i = k + 1; i < n; ++i) s -= A[k * n + i] * B[i * nrhs + j];
      B[k * nrhs + j] = s / A[k * n + k];
    }
  }
  return KFO_OK;
}

/*
 * Reconstruction and derivative vectors of one (sub)stencil.
 *   offs   : n x 3 integer cell-centre offsets (unit cells)
 *   mons   : nmono x 3 monomial multi-indices, |alpha| <= p (D = nmono)
 *   ders   : nder x 3 derivative multi-indices (0 < |alpha| <= R)
 *   rface  : out, F x n  (one row per face Gauss point)
 *   rderiv : out, nder x n
 * Solves [[Q^T, P], [P^T, 0]] [r; w] = [T; S] (Eq. 14) with
 *   Q_hl = lambda_h K(., x_l) (Eq. 7), P_hv = lambda_h x^alpha_v (Eq. 8),
 *   T_l = K(x_s, x_l), S_v = x_s^alpha_v (Eqs. 12-13) for the face points and
 *   D_l = d^alpha K(x, x_l)|_0, S_v = d^alpha x^alpha_v |_0 (Eq. 23) for the
 *   derivatives.
 */
int kfo_weights(int dim, int R, double ell_d, int n, const int* offs, int nmono, const int* mons, int nder,
                const int* ders, double* rface, double* rderiv) {
  if ((dim != 2 && dim != 3) || n <= 0 || nmono < 0 || nmono > n) return KFO_ERR_ARG;
  qreal pts[3 * 54];
  int F = face_points_q(dim, R, pts);
  if (F <= 0) return KFO_ERR_ARG;
  qreal ell = (qreal)ell_d;
  int N = n + nmono;
  int nrhs = F + nder;
  qreal* A = (qreal*)calloc((size_t)N * N, sizeof(qreal));
  qreal* B = (qreal*)calloc((size_t)N * nrhs, sizeof(qreal));
  if (!A || !B) { free(A); free(B); return KFO_ERR_NOMEM; }

  /* Q_hl and P_hv */
  for (int h = 0; h < n; ++h) {
    for (int l = 0; l < n; ++l) {
      qreal q = 1;
      for (int k = 0; k < dim; ++k) q *= cell_int_1d(offs[3 * h + k] - offs[3 * l + k], ell);
      A[l * N + h] = q; /* row l of Q^T is column l of Q: (Q^T)_{lh} = Q_hl */
    }
    for (int v = 0; v < nmono; ++v) {
      qreal pv = 1;
      for (int k = 0; k < dim; ++k) pv *= cell_avg_mono_1d(offs[3 * h + k], mons[3 * v + k]);
      A[h * N + n + v] = pv;   /* P block */
      A[(n + v) * N + h] = pv; /* P^T block */
    }
  }
  /* right-hand sides: face points */
  for (int s = 0; s < F; ++s) {
    const qreal* x = pts + 3 * s;
    for (int l = 0; l < n; ++l) {
      qreal r2 = 0;
      for (int k = 0; k < dim; ++k) { qreal d = x[k] - (qreal)offs[3 * l + k]; r2 += d * d; }
      B[l * nrhs + s] = q_exp(-r2 / (2 * ell * ell));
    }
    for (int v = 0; v < nmono; ++v) {
      qreal m = 1;
      for (int k = 0; k < dim; ++k) m *= qpow(x[k], mons[3 * v + k]);
      B[(n + v) * nrhs + s] = m;
    }
  }
  /* right-hand sides: derivatives at the cell centre */
  for (int m = 0; m < nder; ++m) {
    const int* a = ders + 3 * m;
    for (int l = 0; l < n; ++l) {
      qreal dk = 1;
      for (int k = 0; k < dim; ++k) dk *= kernel_deriv_1d(a[k], offs[3 * l + k], ell);
      B[l * nrhs + F + m] = dk;
    }
    for (int v = 0; v < nmono; ++v) {
      const int* b = mons + 3 * v;
      int same = 1;
      qreal fact = 1;
      for (int k = 0; k < dim; ++k) {
        if (a[k] != b[k]) same = 0;
        for (int i = 2; i <= a[k]; ++i) fact *= i;
      }
      B[(n + v) * nrhs + F + m] = same ? fact : 0;
    }
  }
  int rc = solve_q(N, A, nrhs, B);
  if (rc == KFO_OK) {
    for (int s = 0; s < F; ++s)
      for (int l = 0; l < n; ++l) rface[s * n + l] = (double)B[l * nrhs + s];
    for (int m = 0; m < nder; ++m)
      for (int l = 0; l < n; ++l) rderiv[m * n + l] = (double)B[l * nrhs + F + m];
  }
  free(A);
  free(B);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Problem description shared with the Python side of the oracle.            */
/* ------------------------------------------------------------------------- */
typedef struct {
  int dim, R, nv;
  int n[3];
  double dx[3];
  int bc[3][2];         /* 0 periodic, 1 outflow */
  double gamma;
  double eps;
  int nq;               /* number of (sub)stencils, N_S + 1 */
  int n0;               /* |S0| */
  const int* offs;      /* n0 x 3 */
  const int* sub_len;   /* nq */
  const int* sub_idx;   /* concatenated index lists into S0 */
  const double* lin_w;  /* nq linear weights gamma_q */
  int nface, nderiv;    /* F, M */
  const double* wts;    /* per q: F*N_q face weights then M*N_q derivative weights */
  const double* gl_w;   /* R Gauss-Legendre weights on [-1/2,1/2] */
  int recon;            /* 0: WENO-AO in linearized primitive variables; 1: linear S0, conservative;
                           2: per-cell choice of the two by `mask` (the gated reconstruction);
                           3: per-cell choice by the KXRCF indicator of each stage's own state */
  int riemann;          /* 0: HLLC, 1: HLL */
  int positivity;       /* 1: apply the positivity-preserving limiter of Sec. 4 to the Riemann states */
  double kappa, eta;    /* bound relaxation kappa and flattener eta of Sec. 4.1 */
  const unsigned char* mask; /* recon 2: per cell, 1 = linear (smooth), 0 = WENO-AO */
  double kxrcf_m;       /* recon 3: power m of the KXRCF threshold Delta^m (Sec. 3.5: m = 3/2) */
  int vars;             /* WENO-AO variables: 0 linearized primitive (Sec. 3.4.2), 1 characteristic (Sec. 3.4.1) */
} kfo_problem;

static long ncell_of(const kfo_problem* pb) { return (long)pb->n[0] * pb->n[1] * pb->n[2]; }

/* ghost-cell index map of Sec. 5.3 step 1: periodic wraps, outflow clamps */
static int map_index(int i, int n, int bc_lo, int bc_hi) {
  if (i < 0) return bc_lo == 0 ? ((i % n) + n) % n : 0;
  if (i >= n) return bc_hi == 0 ? i % n : n - 1;
  return i;
}

static double pressure(const double* u, int dim, double gamma) {
  double ke = 0;
  for (int k = 0; k < dim; ++k) ke += u[1 + k] * u[1 + k];
  ke = 0.5 * ke / u[0];
  return (gamma - 1.0) * (u[dim + 1] - ke);
}

static int physical(const double* u, int dim, double gamma) {
  double p = pressure(u, dim, gamma);
  return u[0] > 0 && p > 0 && isfinite(u[0]) && isfinite(p);
}

/* Phi = dV/dU and Phi^{-1} = dU/dV at the reference state ut (appendix A).
   The energy row of Phi^{-1} uses rho*u_i (d E / d u_i), which makes Phi^{-1}
   the exact inverse that Sec. 3.4.1 requires; the printed row has u_i. */
void kfo_phi(int dim, double gamma, const double* ut, double* phi, double* phinv) {
  int nv = dim + 2;
  double rho = ut[0];
  double u[3] = {0, 0, 0}, u2 = 0;
  for (int k = 0; k < dim; ++k) { u[k] = ut[1 + k] / rho; u2 += u[k] * u[k]; }
  memset(phi, 0, sizeof(double) * nv * nv);
  memset(phinv, 0, sizeof(double) * nv * nv);
  phi[0] = 1;
  for (int k = 0; k < dim; ++k) {
    phi[(1 + k) * nv + 0] = -u[k] / rho;
    phi[(1 + k) * nv + 1 + k] = 1.0 / rho;
  }
  phi[(nv - 1) * nv + 0] = (gamma - 1.0) * u2 / 2.0;
  for (int k = 0; k < dim; ++k) phi[(nv - 1) * nv + 1 + k] = (1.0 - gamma) * u[k];
  phi[(nv - 1) * nv + nv - 1] = gamma - 1.0;

  phinv[0] = 1;
  for (int k = 0; k < dim; ++k) {
    phinv[(1 + k) * nv + 0] = u[k];
    phinv[(1 + k) * nv + 1 + k] = rho;
  }
  phinv[(nv - 1) * nv + 0] = u2 / 2.0;
  for (int k = 0; k < dim; ++k) phinv[(nv - 1) * nv + 1 + k] = rho * u[k];
  phinv[(nv - 1) * nv + nv - 1] = 1.0 / (gamma - 1.0);
}

/* Characteristic variables of direction dir at the reference state ut (Sec. 3.4.1): the flux
   Jacobian A = dF_dir/dU = R Lambda L, Phi = L (rows: left eigenvectors) and Phi^{-1} = R
   (columns: right eigenvectors), L R = I.  Waves in the order u_n - c, entropy, the shear waves of
   the tangential axes in increasing order, u_n + c.  With b1 = (gamma-1)/c^2, b2 = b1 |u|^2/2,
   H = (E + p)/rho and n the unit normal:
     R: (1, u - c n, H - c u_n), (1, u, |u|^2/2), (0, e_a, u_a), (1, u + c n, H + c u_n);
     L: (b2 + u_n/c, -b1 u - n/c, b1)/2, (1 - b2, b1 u, -b1), (-u_a, e_a, 0), (b2 - u_n/c, -b1 u + n/c, b1)/2. */
void kfo_char(int dim, double gamma, const double* ut, int dir, double* L, double* Rm) {
  const int nv = dim + 2;
  const double rho = ut[0];
  double u[3] = {0, 0, 0}, q2 = 0;
  for (int k = 0; k < dim; ++k) { u[k] = ut[1 + k] / rho; q2 += u[k] * u[k]; }
  const double p = (gamma - 1.0) * (ut[nv - 1] - 0.5 * rho * q2);
  const double c = sqrt(gamma * p / rho), H = (ut[nv - 1] + p) / rho;
  const double b1 = (gamma - 1.0) / (c * c), b2 = 0.5 * b1 * q2, un = u[dir];
  memset(L, 0, sizeof(double) * nv * nv);
  memset(Rm, 0, sizeof(double) * nv * nv);
  /* columns of R */
  Rm[0 * nv + 0] = 1.0;
  Rm[0 * nv + 1] = 1.0;
  Rm[0 * nv + nv - 1] = 1.0;
  for (int k = 0; k < dim; ++k) {
    const double nk = (k == dir) ? 1.0 : 0.0;
    Rm[(1 + k) * nv + 0] = u[k] - c * nk;
    Rm[(1 + k) * nv + 1] = u[k];
    Rm[(1 + k) * nv + nv - 1] = u[k] + c * nk;
  }
  Rm[(nv - 1) * nv + 0] = H - c * un;
  Rm[(nv - 1) * nv + 1] = 0.5 * q2;
  Rm[(nv - 1) * nv + nv - 1] = H + c * un;
  /* rows of L */
  L[0 * nv + 0] = 0.5 * (b2 + un / c);
  L[1 * nv + 0] = 1.0 - b2;
  L[(nv - 1) * nv + 0] = 0.5 * (b2 - un / c);
  for (int k = 0; k < dim; ++k) {
    const double nk = (k == dir) ? 1.0 : 0.0;
    L[0 * nv + 1 + k] = 0.5 * (-b1 * u[k] - nk / c);
    L[1 * nv + 1 + k] = b1 * u[k];
    L[(nv - 1) * nv + 1 + k] = 0.5 * (-b1 * u[k] + nk / c);
  }
  L[0 * nv + nv - 1] = 0.5 * b1;
  L[1 * nv + nv - 1] = -b1;
  L[(nv - 1) * nv + nv - 1] = 0.5 * b1;
  /* shear waves: one per tangential axis a, in increasing order */
  int w = 2;
  for (int a = 0; a < dim; ++a) {
    if (a == dir) continue;
    Rm[(1 + a) * nv + w] = 1.0;
    Rm[(nv - 1) * nv + w] = u[a];
    L[w * nv + 0] = -u[a];
    L[w * nv + 1 + a] = 1.0;
    ++w;
  }
}

/* offset of the weights of stencil q inside pb->wts */
static long wts_offset(const kfo_problem* pb, int q) {
  long off = 0;
  for (int j = 0; j < q; ++j) off += (long)pb->sub_len[j] * (pb->nface + pb->nderiv);
  return off;
}

static long sub_start(const kfo_problem* pb, int q) {
  long off = 0;
  for (int j = 0; j < q; ++j) off += pb->sub_len[j];
  return off;
}

/*
 * Riemann states of every cell (Sec. 5.3 step 2).
 *   U     : [nv][ncell]
 *   faces : out, [F][nv][ncell]
 *   omega : optional out, [nq][nv][ncell] normalised nonlinear weights (WENO mode, linearized
 *           primitive variables)
 */
int kfo_kxrcf(const kfo_problem* pb, const double* U, double* ratio, unsigned char* mask);

int kfo_reconstruct(const kfo_problem* pb, const double* U, double* faces, double* omega) {
  const int dim = pb->dim, nv = pb->nv, n0 = pb->n0, F = pb->nface, M = pb->nderiv, nq = pb->nq;
  const long nc = ncell_of(pb);
  int status = KFO_OK;
  if (pb->recon == 3) {
    /* Sec. 5.3 step 2: the KXRCF indicator of this state picks each cell's reconstruction */
    unsigned char* kmask = (unsigned char*)malloc((size_t)nc);
    if (!kmask) return KFO_ERR_NOMEM;
    kfo_problem gated = *pb;
    int sk = kfo_kxrcf(pb, U, NULL, kmask);
    gated.recon = 2;
    gated.mask = kmask;
    if (sk == KFO_OK) sk = kfo_reconstruct(&gated, U, faces, omega);
    free(kmask);
    return sk;
  }
  /* per-thread scratch (one thread in the checker build) */
  const int nth = KFO_MAX_THREADS();
  double* sten_all = (double*)malloc(sizeof(double) * n0 * nv * nth); /* [l][var] conservative */
  double* W_all = (double*)malloc(sizeof(double) * n0 * nv * nth);    /* [var][l] reconstruction variables */
  double* vals_all = (double*)malloc(sizeof(double) * nq * F * nth);  /* v_q(s) for one variable */
  double* ws_all = (double*)malloc(sizeof(double) * F * nv * nth);    /* w_s [s][var] */
  if (!sten_all || !W_all || !vals_all || !ws_all) {
    free(sten_all); free(W_all); free(vals_all); free(ws_all);
    return KFO_ERR_NOMEM;
  }

#pragma omp parallel for collapse(2) schedule(dynamic, 1) reduction(max : status)
  for (int z = 0; z < pb->n[2]; ++z)
    for (int y = 0; y < pb->n[1]; ++y)
      for (int x = 0; x < pb->n[0]; ++x) {
        const long c = ((long)z * pb->n[1] + y) * pb->n[0] + x;
        const int th = KFO_THREAD();
        double* sten = sten_all + (long)th * n0 * nv;
        double* W = W_all + (long)th * n0 * nv;
        double* vals = vals_all + (long)th * nq * F;
        double* ws = ws_all + (long)th * F * nv;
        /* gather S0 through the ghost-cell map */
        for (int l = 0; l < n0; ++l) {
          int ix = map_index(x + pb->offs[3 * l + 0], pb->n[0], pb->bc[0][0], pb->bc[0][1]);
          int iy = map_index(y + pb->offs[3 * l + 1], pb->n[1], pb->bc[1][0], pb->bc[1][1]);
          int iz = dim == 3 ? map_index(z + pb->offs[3 * l + 2], pb->n[2], pb->bc[2][0], pb->bc[2][1]) : 0;
          long cl = ((long)iz * pb->n[1] + iy) * pb->n[0] + ix;
          for (int v = 0; v < nv; ++v) sten[l * nv + v] = U[v * nc + cl];
        }
        if (pb->recon == 1 || (pb->recon == 2 && pb->mask && pb->mask[c])) {
          /* unlimited linear reconstruction on S0 in conservative variables */
          const double* r0 = pb->wts;
          for (int s = 0; s < F; ++s)
            for (int v = 0; v < nv; ++v) {
              double acc = 0;
              for (int l = 0; l < n0; ++l) acc += r0[s * n0 + l] * sten[l * nv + v];
              ws[s * nv + v] = acc;
            }
        } else {
          /* the reference state: the central cell average (the l with offset 0) */
          int lc = -1;
          for (int l = 0; l < n0; ++l)
            if (pb->offs[3 * l] == 0 && pb->offs[3 * l + 1] == 0 && pb->offs[3 * l + 2] == 0) lc = l;
          /* linearized primitive variables: one Phi for every face (Sec. 3.4.2); characteristic
             variables: one Phi per direction, serving that direction's faces only (Sec. 3.4.1) */
          const int npass = pb->vars == 1 ? dim : 1;
          const int nt = F / (2 * dim);
          for (int pass = 0; pass < npass; ++pass) {
            double phi[25], phinv[25];
            if (pb->vars == 1)
              kfo_char(dim, pb->gamma, sten + lc * nv, pass, phi, phinv);
            else
              kfo_phi(dim, pb->gamma, sten + lc * nv, phi, phinv);
            const int s_lo = pb->vars == 1 ? 2 * pass * nt : 0, s_hi = pb->vars == 1 ? (2 * pass + 2) * nt : F;
            /* W_h = Phi U_h over the whole stencil (Eq. 33, or L U_h) */
            for (int v = 0; v < nv; ++v)
              for (int l = 0; l < n0; ++l) {
                double acc = 0;
                for (int j = 0; j < nv; ++j) acc += phi[v * nv + j] * sten[l * nv + j];
                W[v * n0 + l] = acc;
              }
            for (int v = 0; v < nv; ++v) {
              double beta[8], om[8];
              for (int q = 0; q < nq; ++q) {
                const int nl = pb->sub_len[q];
                const int* idx = pb->sub_idx + sub_start(pb, q);
                const double* rf = pb->wts + wts_offset(pb, q);
                const double* rd = rf + (long)F * nl;
                for (int s = s_lo; s < s_hi; ++s) {
                  double acc = 0;
                  for (int l = 0; l < nl; ++l) acc += rf[s * nl + l] * W[v * n0 + idx[l]];
                  vals[q * F + s] = acc;
                }
                double b = 0;
                for (int m = 0; m < M; ++m) {
                  double acc = 0;
                  for (int l = 0; l < nl; ++l) acc += rd[m * nl + l] * W[v * n0 + idx[l]];
                  b += acc * acc;
                }
                beta[q] = b;
              }
              double sum = 0;
              for (int q = 0; q < nq; ++q) { om[q] = pb->lin_w[q] / (beta[q] * beta[q] + pb->eps); sum += om[q]; }
              for (int q = 0; q < nq; ++q) om[q] /= sum;
              if (omega && pb->vars == 0)
                for (int q = 0; q < nq; ++q) omega[((long)q * nv + v) * nc + c] = om[q];
              const double g0 = pb->lin_w[0];
              for (int s = s_lo; s < s_hi; ++s) {
                double acc = om[0] / g0 * vals[s];
                for (int q = 1; q < nq; ++q) acc += (om[q] - om[0] * pb->lin_w[q] / g0) * vals[q * F + s];
                ws[s * nv + v] = acc;
              }
            }
            /* back to conservative variables, u_s = Phi^{-1} w_s */
            for (int s = s_lo; s < s_hi; ++s) {
              double u[5];
              for (int v = 0; v < nv; ++v) {
                double acc = 0;
                for (int j = 0; j < nv; ++j) acc += phinv[v * nv + j] * ws[s * nv + j];
                u[v] = acc;
              }
              for (int v = 0; v < nv; ++v) ws[s * nv + v] = u[v];
            }
          }
        }
        for (int s = 0; s < F; ++s) {
          if (!physical(ws + s * nv, dim, pb->gamma)) status = KFO_ERR_NONPHYSICAL;
          for (int v = 0; v < nv; ++v) faces[((long)s * nv + v) * nc + c] = ws[s * nv + v];
        }
      }
  free(sten_all);
  free(W_all);
  free(vals_all);
  free(ws_all);
  return status;
}

/* ------------------------------------------------------------------------- */
/* Positivity-preserving limiter (Sec. 4), applied to all Riemann states of  */
/* one cell at a time.                                                       */
/* ------------------------------------------------------------------------- */
static void blend(const double* ut, const double* us, double th, int nv, double* out) {
  for (int v = 0; v < nv; ++v) out[v] = ut[v] + th * (us[v] - ut[v]);
}

/*
 * faces [F][nv][ncell] are modified in place.  Bounds (Sec. 4.1) come from the
 * cell averages of the 3^dim neighbourhood (ghost-cell map as for the
 * stencil); theta_rho (Eq. 36) uses each fraction only where its bound is
 * violated; theta_p is the smallest per-point root of Eq. (39) found by 60
 * bisection steps on [0, 1], keeping the admissible end (Eq. 40).
 * Returns KFO_ERR_NONPHYSICAL when a cell average itself is not admissible.
 */
int kfo_limit(const kfo_problem* pb, const double* U, double* faces) {
  const int dim = pb->dim, nv = pb->nv, F = pb->nface;
  const long nc = ncell_of(pb);
  int status = KFO_OK;
#pragma omp parallel for collapse(2) schedule(dynamic, 1) reduction(max : status)
  for (int z = 0; z < pb->n[2]; ++z)
    for (int y = 0; y < pb->n[1]; ++y)
      for (int x = 0; x < pb->n[0]; ++x) {
        const long c = ((long)z * pb->n[1] + y) * pb->n[0] + x;
        double ut[5];
        for (int v = 0; v < nv; ++v) ut[v] = U[v * nc + c];
        double rmax = -INFINITY, rmin = INFINITY, pmin = INFINITY;
        int kz = dim == 3 ? 1 : 0;
        for (int k = -kz; k <= kz; ++k)
          for (int j = -1; j <= 1; ++j)
            for (int i = -1; i <= 1; ++i) {
              int ix = map_index(x + i, pb->n[0], pb->bc[0][0], pb->bc[0][1]);
              int iy = map_index(y + j, pb->n[1], pb->bc[1][0], pb->bc[1][1]);
              int iz = dim == 3 ? map_index(z + k, pb->n[2], pb->bc[2][0], pb->bc[2][1]) : 0;
              long cl = ((long)iz * pb->n[1] + iy) * pb->n[0] + ix;
              double u[5];
              for (int v = 0; v < nv; ++v) u[v] = U[v * nc + cl];
              double p = pressure(u, dim, pb->gamma);
              if (u[0] > rmax) rmax = u[0];
              if (u[0] < rmin) rmin = u[0];
              if (p < pmin) pmin = p;
            }
        const double relax_hi = 1.0 + pb->kappa - pb->kappa * pb->eta;
        const double relax_lo = 1.0 - pb->kappa + pb->kappa * pb->eta;
        const double rho_max = rmax * relax_hi, rho_min = rmin * relax_lo, p_min = pmin * relax_lo;
        if (!physical(ut, dim, pb->gamma)) { status = KFO_ERR_NONPHYSICAL; continue; }
        /* density: theta_rho */
        double th = 1.0;
        for (int s = 0; s < F; ++s) {
          double rs = faces[((long)s * nv + 0) * nc + c];
          if (rs < rho_min) { double t = (ut[0] - rho_min) / (ut[0] - rs); if (t < th) th = t; }
          if (rs > rho_max) { double t = (rho_max - ut[0]) / (rs - ut[0]); if (t < th) th = t; }
        }
        if (th < 1.0)
          for (int s = 0; s < F; ++s)
            for (int v = 0; v < nv; ++v) {
              double* f = faces + ((long)s * nv + v) * nc + c;
              *f = ut[v] + th * (*f - ut[v]);
            }
        /* pressure: theta_p */
        double thp = 1.0;
        for (int s = 0; s < F; ++s) {
          double us[5], tmp[5];
          for (int v = 0; v < nv; ++v) us[v] = faces[((long)s * nv + v) * nc + c];
          if (pressure(us, dim, pb->gamma) >= p_min) continue;
          double lo = 0.0, hi = 1.0;
          for (int it = 0; it < 60; ++it) {
            double mid = 0.5 * (lo + hi);
            blend(ut, us, mid, nv, tmp);
            if (pressure(tmp, dim, pb->gamma) >= p_min) lo = mid; else hi = mid;
          }
          if (lo < thp) thp = lo;
        }
        if (thp < 1.0)
          for (int s = 0; s < F; ++s)
            for (int v = 0; v < nv; ++v) {
              double* f = faces + ((long)s * nv + v) * nc + c;
              *f = ut[v] + thp * (*f - ut[v]);
            }
      }
  return status;
}

/* ------------------------------------------------------------------------- */
/* Riemann solvers (Sec. 5.4: HLLC and HLL with Batten wave speeds).         */
/* ------------------------------------------------------------------------- */
static void euler_flux(const double* u, int dir, int dim, double gamma, double* f) {
  double p = pressure(u, dim, gamma);
  double un = u[1 + dir] / u[0];
  f[0] = u[1 + dir];
  for (int k = 0; k < dim; ++k) f[1 + k] = u[1 + k] * un + (k == dir ? p : 0.0);
  f[dim + 1] = un * (u[dim + 1] + p);
}

/* Numerical flux in direction dir between left state uL and right state uR.
   Returns 0, or KFO_ERR_NONPHYSICAL if either state has rho <= 0 or p <= 0. */
int kfo_riemann(int dim, double gamma, int solver, int dir, const double* uL, const double* uR, double* fout) {
  const int nv = dim + 2;
  if (!physical(uL, dim, gamma) || !physical(uR, dim, gamma)) {
    for (int v = 0; v < nv; ++v) fout[v] = NAN;
    return KFO_ERR_NONPHYSICAL;
  }
  double rL = uL[0], rR = uR[0];
  double pL = pressure(uL, dim, gamma), pR = pressure(uR, dim, gamma);
  double unL = uL[1 + dir] / rL, unR = uR[1 + dir] / rR;
  double cL = sqrt(gamma * pL / rL), cR = sqrt(gamma * pR / rR);
  /* Roe averages */
  double sL = sqrt(rL), sR = sqrt(rR);
  double ut[3] = {0, 0, 0}, ut2 = 0;
  for (int k = 0; k < dim; ++k) {
    ut[k] = (sL * uL[1 + k] / rL + sR * uR[1 + k] / rR) / (sL + sR);
    ut2 += ut[k] * ut[k];
  }
  double HL = (uL[dim + 1] + pL) / rL, HR = (uR[dim + 1] + pR) / rR;
  double Ht = (sL * HL + sR * HR) / (sL + sR);
  double ct2 = (gamma - 1.0) * (Ht - 0.5 * ut2);
  double ct = sqrt(ct2 > 0 ? ct2 : 0.0);
  /* Batten wave speeds */
  double SL = fmin(unL - cL, ut[dir] - ct);
  double SR = fmax(unR + cR, ut[dir] + ct);
  double FL[5], FR[5];
  euler_flux(uL, dir, dim, gamma, FL);
  euler_flux(uR, dir, dim, gamma, FR);
  if (SL >= 0) { for (int v = 0; v < nv; ++v) fout[v] = FL[v]; return 0; }
  if (SR <= 0) { for (int v = 0; v < nv; ++v) fout[v] = FR[v]; return 0; }
  if (solver == 1) {
    for (int v = 0; v < nv; ++v) fout[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (uR[v] - uL[v])) / (SR - SL);
    return 0;
  }
  /* HLLC: contact speed and star states (Toro) */
  double Ss = (pR - pL + rL * unL * (SL - unL) - rR * unR * (SR - unR)) / (rL * (SL - unL) - rR * (SR - unR));
  const double* uK = (Ss >= 0) ? uL : uR;
  const double* FK = (Ss >= 0) ? FL : FR;
  double SK = (Ss >= 0) ? SL : SR;
  double rK = uK[0], unK = uK[1 + dir] / rK, pK = (Ss >= 0) ? pL : pR;
  double fac = rK * (SK - unK) / (SK - Ss);
  double us[5];
  us[0] = fac;
  for (int k = 0; k < dim; ++k) us[1 + k] = fac * (k == dir ? Ss : uK[1 + k] / rK);
  us[dim + 1] = fac * (uK[dim + 1] / rK + (Ss - unK) * (Ss + pK / (rK * (SK - unK))));
  for (int v = 0; v < nv; ++v) fout[v] = FK[v] + SK * (us[v] - uK[v]);
  return 0;
}

/*
 * Flux divergence (Sec. 5.3 steps 4-6): dUdt = -sum_d (F_{d,+} - F_{d,-}) / Delta_d
 * with F_{d,+/-} the Gauss-Legendre average of the point fluxes on that face.
 */
int kfo_flux(const kfo_problem* pb, const double* faces, double* dUdt) {
  const int dim = pb->dim, nv = pb->nv, R = pb->R;
  const long nc = ncell_of(pb);
  const int nt = (dim == 2) ? R : R * R;
  int status = KFO_OK;
  for (long i = 0; i < (long)nv * nc; ++i) dUdt[i] = 0;
#pragma omp parallel for collapse(2) schedule(dynamic, 1) reduction(max : status)
  for (int z = 0; z < pb->n[2]; ++z)
    for (int y = 0; y < pb->n[1]; ++y)
      for (int x = 0; x < pb->n[0]; ++x) {
        const long c = ((long)z * pb->n[1] + y) * pb->n[0] + x;
        const int ci[3] = {x, y, z};
        for (int dir = 0; dir < dim; ++dir) {
          for (int side = 0; side < 2; ++side) {
            /* the face of cell c on this side, and the cell across it */
            int nb[3] = {x, y, z};
            nb[dir] += side ? 1 : -1;
            int outside = nb[dir] < 0 || nb[dir] >= pb->n[dir];
            int bc = pb->bc[dir][side];
            long cn = -1;
            if (!outside || bc == 0) {
              nb[dir] = ((nb[dir] % pb->n[dir]) + pb->n[dir]) % pb->n[dir];
              cn = ((long)nb[2] * pb->n[1] + nb[1]) * pb->n[0] + nb[0];
            }
            (void)ci;
            double favg[5] = {0, 0, 0, 0, 0};
            for (int t = 0; t < nt; ++t) {
              int s_in = (dir * 2 + side) * nt + t;        /* this cell's point */
              int s_out = (dir * 2 + (1 - side)) * nt + t; /* the neighbour's matching point */
              double uin[5], uout[5], f[5];
              for (int v = 0; v < nv; ++v) {
                uin[v] = faces[((long)s_in * nv + v) * nc + c];
                uout[v] = (cn >= 0) ? faces[((long)s_out * nv + v) * nc + cn] : uin[v];
              }
              const double* uL = side ? uin : uout;
              const double* uR = side ? uout : uin;
              if (kfo_riemann(dim, pb->gamma, pb->riemann, dir, uL, uR, f)) status = KFO_ERR_NONPHYSICAL;
              double wt = pb->gl_w[t % R] * (dim == 3 ? pb->gl_w[t / R] : 1.0);
              for (int v = 0; v < nv; ++v) favg[v] += wt * f[v];
            }
            double sgn = side ? -1.0 : 1.0;
            for (int v = 0; v < nv; ++v) dUdt[v * nc + c] += sgn * favg[v] / pb->dx[dir];
          }
        }
      }
  return status;
}

/* max over cells of sum_d (|u_d| + c) / Delta_d */
double kfo_max_rate(const kfo_problem* pb, const double* U) {
  const int dim = pb->dim, nv = pb->nv;
  const long nc = ncell_of(pb);
  double mx = 0;
  for (long c = 0; c < nc; ++c) {
    double u[5];
    for (int v = 0; v < nv; ++v) u[v] = U[v * nc + c];
    double p = pressure(u, dim, pb->gamma);
    double cs = sqrt(pb->gamma * p / u[0]);
    double rate = 0;
    for (int d = 0; d < dim; ++d) rate += (fabs(u[1 + d] / u[0]) + cs) / pb->dx[d];
    if (!(rate <= mx)) mx = rate; /* a NaN rate propagates */
  }
  return mx;
}

/* ------------------------------------------------------------------------- */
/* KXRCF troubled-cell indicator (Sec. 3.5; Sec. 5.3 step 2, items 1-2).      */
/* ------------------------------------------------------------------------- */
static double entropy_q(const double* u, int dim, double gamma) {
  /* q = p / rho^gamma of one conservative state; +inf when it is not admissible */
  if (!physical(u, dim, gamma)) return INFINITY;
  return pressure(u, dim, gamma) / pow(u[0], gamma);
}

/*
 * Step 1: unlimited linear S0 reconstruction of the conservative variables on
 * every cell.  Step 2: for every cell c and every Gauss point s of each of its
 * faces, the entropy q = p / rho^gamma of c's own state at s (minus side) and of
 * the state the cell across that face reconstructs at the same point (plus
 * side); ratio[c] = max_s |q+ - q-| / <Q>, with <Q> = p(Ubar_c) / rhobar_c^gamma
 * from c's cell average.  The cell is smooth (mask 1: linear reconstruction)
 * when ratio < Delta^m, Delta the largest cell width over the axes; otherwise it
 * is flagged for WENO-AO (mask 0).
 * Faces on the physical boundary: periodic -> the wrapped neighbour; outflow ->
 * the exterior state is a copy of the interior one (Sec. 5.3 step 4), so the
 * face has no jump.  A state that is not admissible (rho <= 0, p <= 0 or not
 * finite) on either side of a point, or such a cell average, gives ratio = +inf.
 * ratio and mask may each be NULL.
 */
int kfo_kxrcf(const kfo_problem* pb, const double* U, double* ratio, unsigned char* mask) {
  const int dim = pb->dim, nv = pb->nv, R = pb->R;
  const long nc = ncell_of(pb);
  const int nt = (dim == 2) ? R : R * R;
  kfo_problem lin = *pb;
  lin.recon = 1;
  double* faces = (double*)malloc(sizeof(double) * (size_t)pb->nface * nv * nc);
  if (!faces) return KFO_ERR_NOMEM;
  kfo_reconstruct(&lin, U, faces, NULL); /* unlimited states may be inadmissible: handled below */
  double delta = 0;
  for (int d = 0; d < dim; ++d)
    if (pb->dx[d] > delta) delta = pb->dx[d];
  const double thresh = pow(delta, pb->kxrcf_m);
  for (int z = 0; z < pb->n[2]; ++z)
    for (int y = 0; y < pb->n[1]; ++y)
      for (int x = 0; x < pb->n[0]; ++x) {
        const long c = ((long)z * pb->n[1] + y) * pb->n[0] + x;
        double ubar[5];
        for (int v = 0; v < nv; ++v) ubar[v] = U[v * nc + c];
        const double Q = entropy_q(ubar, dim, pb->gamma);
        double jmax = 0;
        for (int dir = 0; dir < dim; ++dir)
          for (int side = 0; side < 2; ++side) {
            int nb[3] = {x, y, z};
            nb[dir] += side ? 1 : -1;
            const int outside = nb[dir] < 0 || nb[dir] >= pb->n[dir];
            if (outside && pb->bc[dir][side] == 1) continue; /* outflow: exterior = interior */
            nb[dir] = ((nb[dir] % pb->n[dir]) + pb->n[dir]) % pb->n[dir];
            const long cn = ((long)nb[2] * pb->n[1] + nb[1]) * pb->n[0] + nb[0];
            for (int t = 0; t < nt; ++t) {
              const int s_in = (dir * 2 + side) * nt + t;
              const int s_out = (dir * 2 + (1 - side)) * nt + t;
              double um[5], up[5];
              for (int v = 0; v < nv; ++v) {
                um[v] = faces[((long)s_in * nv + v) * nc + c];
                up[v] = faces[((long)s_out * nv + v) * nc + cn];
              }
              const double qm = entropy_q(um, dim, pb->gamma), qp = entropy_q(up, dim, pb->gamma);
              const double j = (isinf(qm) || isinf(qp)) ? INFINITY : fabs(qp - qm);
              if (j > jmax) jmax = j;
            }
          }
        const double r = isinf(Q) ? INFINITY : jmax / Q;
        if (ratio) ratio[c] = r;
        if (mask) mask[c] = r < thresh ? 1 : 0;
      }
  free(faces);
  return KFO_OK;
}

int kfo_rhs(const kfo_problem* pb, const double* U, double* dUdt) {
  const long nc = ncell_of(pb);
  double* faces = (double*)malloc(sizeof(double) * (size_t)pb->nface * pb->nv * nc);
  if (!faces) return KFO_ERR_NOMEM;
  int s1 = kfo_reconstruct(pb, U, faces, NULL);
  if (pb->positivity) s1 = kfo_limit(pb, U, faces);
  int s2 = kfo_flux(pb, faces, dUdt);
  free(faces);
  return s1 ? s1 : s2;
}

/* One SSP-RK3 step (Shu-Osher form) of the semi-discrete system dU/dt = L(U). */
int kfo_step(const kfo_problem* pb, double* U, double cfl, double t_rem, double* dt_out) {
  const long nn = (long)pb->nv * ncell_of(pb);
  double rate = kfo_max_rate(pb, U);
  if (!(rate > 0) || !isfinite(rate)) return KFO_ERR_NONPHYSICAL;
  double dt = cfl / rate;
  if (dt > t_rem) dt = t_rem;
  if (dt_out) *dt_out = dt;
  double* Un = (double*)malloc(sizeof(double) * nn);
  double* L = (double*)malloc(sizeof(double) * nn);
  double* Us = (double*)malloc(sizeof(double) * nn);
  if (!Un || !L || !Us) { free(Un); free(L); free(Us); return KFO_ERR_NOMEM; }
  memcpy(Un, U, sizeof(double) * nn);
  int st = kfo_rhs(pb, Un, L);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < nn; ++i) Us[i] = Un[i] + dt * L[i];
  st |= kfo_rhs(pb, Us, L);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < nn; ++i) Us[i] = 0.75 * Un[i] + 0.25 * (Us[i] + dt * L[i]);
  st |= kfo_rhs(pb, Us, L);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < nn; ++i) U[i] = (1.0 / 3.0) * Un[i] + (2.0 / 3.0) * (Us[i] + dt * L[i]);
  free(Un);
  free(L);
  free(Us);
  return st ? KFO_ERR_NONPHYSICAL : KFO_OK;
}
