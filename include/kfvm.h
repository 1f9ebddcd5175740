/*
 * kfvm.h -- C ABI of the GB300 (sm_103a) KFVM-WENO hot path.
 *
 * The library computes the semi-discrete right-hand side and the SSP-RK3
 * update of the compressible Euler equations (Eq. 1 and the Euler system of
 * Sec. 1) with the kernel-based, fully multidimensional WENO-AO finite volume
 * method of May & Lee, "KFVM-WENO: a high-order accurate kernel-based finite
 * volume method for compressible hydrodynamics" (arXiv 2401.16543).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Pointers named U, dUdt, faces are DEVICE pointers owned by the caller; the
 * library never frees or keeps them beyond the call.  The library owns its
 * weight tables, its scratch buffers and the gate network, all allocated by
 * kfvm_init / kfvm_build_weights / kfvm_gate_* and released by kfvm_destroy.
 * A `stream` argument is a cudaStream_t passed as void* (NULL = the legacy
 * default stream); every call is asynchronous on it unless stated otherwise.
 *
 * State layout: float64, structure of arrays [var][z][y][x], x fastest,
 * interior cells only (ghost cells are never stored).  Variables are
 * (rho, rho*u, rho*v, [rho*w,] E): nv = dims + 2.
 *
 * Face (Riemann) state layout: point index
 * s = (dir*2 + side)*R^(dims-1) + t, side 0 the low face (x_dir = -1/2),
 * t = t0 + R*t1 over the transverse axes in increasing order and the
 * Gauss-Legendre nodes (R per face dimension, Sec. 5.1) ascending.  In the
 * FP64 precision mode the values are float64 conservative variables laid out
 * [point][var][cell].  In the FP32 mode they are float32 PRIMITIVE variables:
 * [point][cell] float4 (rho, u, v, p) and, in 3D, a following plane
 * [point][cell] of w (F*nv*ncell floats in all).
 *
 * Errors: every call returns a kfvm_status; nothing throws across the ABI.
 * Device-side failures (a non-admissible state, a NaN) raise a device flag
 * that kfvm_sync_status reads (and kfvm_step reads when dt_out is given).
 * A context is not thread-safe; use one per host thread or serialise.
 * There is no CPU fallback: without a CUDA device every compute call returns
 * KFVM_ERR_CUDA.
 */
#ifndef KFVM_H
#define KFVM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KFVM_OK = 0,
  KFVM_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, unsupported option) */
  KFVM_ERR_CUDA = 2,         /* a CUDA runtime call failed (no device, launch failure)         */
  KFVM_ERR_SINGULAR = 3,     /* a weight system could not be factored                           */
  KFVM_ERR_NONPHYSICAL = 4,  /* rho <= 0, p <= 0 or NaN met in a cell average or Riemann state */
  KFVM_ERR_STATE = 5,        /* call out of order (e.g. a step before kfvm_build_weights)      */
  KFVM_ERR_TIMEOUT = 6,      /* a bounded device wait gave up                                   */
  KFVM_ERR_NOMEM = 7,        /* device or host allocation failed                                */
  KFVM_ERR_TOO_LARGE = 8     /* the problem exceeds a fixed-size buffer (kfvm_flux_static)      */
} kfvm_status;

typedef enum { KFVM_BC_PERIODIC = 0, KFVM_BC_OUTFLOW = 1 } kfvm_bc;

/* Uniform Cartesian grid.  n[2] = 1 and lo/hi[2] unused in 2D.  bc[a][0] is
 * the low side of axis a, bc[a][1] the high side; periodic must be set on
 * both sides of an axis.  Ghost cells (Sec. 5.3 step 1): periodic wraps,
 * outflow copies the nearest interior cell. */
typedef struct {
  int n[3];
  double lo[3];
  double hi[3];
  int bc[3][2];
} kfvm_grid;

typedef struct kfvm_ctx kfvm_ctx;

/* ------------------------------------------------------------------------- */
/* Set-up (Sec. 5.1, stage (i) of the method)                                 */
/* ------------------------------------------------------------------------- */

/* Create a context for a dims-D grid (dims = 2 or 3) with stencil radius R
 * (2 or 3; Sec. 3.1), kernel length scale ell/Delta (the paper uses 5,
 * Sec. 5.1) and ratio of specific heats gamma.  Enumerates S0 and its 2*dims+1
 * substencils (Sec. 3.1), picks each polynomial degree as the largest that
 * keeps the cell-average monomial matrix unisolvent (Sec. 2.1, exact rank over
 * the integers mod two 61-bit primes), and allocates the device buffers (the
 * Riemann-state buffer holds the whole grid's float64 states, in 3D at most
 * 24 GiB: larger grids are stepped in z-slabs, see "slab_planes").
 * Requires an exactly uniform spacing per axis; cells may be non-square.
 * Errors: KFVM_ERR_ARG (null out/grid, dims/R outside {2,3}, n < 1,
 * hi <= lo, ell <= 0, gamma <= 1, mixed periodic sides), KFVM_ERR_CUDA,
 * KFVM_ERR_NOMEM.  On error *out is NULL. */
kfvm_status kfvm_init(kfvm_ctx** out, const kfvm_grid* grid, int dims, int radius, double ell_over_dx, double gamma);

/* Build every reconstruction vector r (face Gauss points; Eqs. 14-18) and
 * derivative vector (Eq. 23, multi-indices 0 < |alpha| <= R) of every
 * (sub)stencil on the GPU: one CTA per (sub)stencil assembles the saddle-point
 * system [[Q^T, P], [P^T, 0]] [r; w] = [T; S] in double-double arithmetic
 * (kernel integrals through series for erf and exp written for this library)
 * and solves it by Gaussian elimination with partial pivoting, then rounds to
 * float64.  Must precede every compute call.  Synchronises the stream.
 * Errors: KFVM_ERR_SINGULAR, KFVM_ERR_CUDA. */
kfvm_status kfvm_build_weights(kfvm_ctx* ctx, void* stream);

/* Copy the weight tables to host memory (synchronous).  Layout: for
 * q = 0..N_S, the F x N_q face rows, then the M x N_q derivative rows.
 * count must equal kfvm_weights_count(ctx).  Errors: KFVM_ERR_ARG,
 * KFVM_ERR_STATE (weights not built). */
kfvm_status kfvm_get_weights(kfvm_ctx* ctx, double* host, size_t count);
size_t kfvm_weights_count(const kfvm_ctx* ctx);

/* Options (key, value):
 *   "precision"   64 (default) or 32: arithmetic of the reconstruction,
 *                 Riemann solve and flux divergence.  The state and its RK
 *                 accumulation stay float64 in both modes.
 *   "recon"       0 WENO-AO in linearized primitive variables on every cell
 *                 (default; Sec. 3, Sec. 5.3), 1 unlimited linear S0
 *                 reconstruction of the conservative variables on every cell
 *                 (Sec. 5.3 step 2a), 2 gated: cells the gate network marks
 *                 smooth take the linear reconstruction, the others WENO-AO,
 *                 4 KXRCF: the paper's troubled-cell indicator (Sec. 3.5,
 *                 evaluated as in Sec. 5.3 step 2 items 1-2; kfvm_kxrcf_mask)
 *                 picks each cell's reconstruction from every stage's own
 *                 state, cells it does not flag take the linear one.
 *   "variables"   WENO-AO variables: 0 linearized primitive (default,
 *                 Sec. 3.4.2: one set of nonlinear weights per cell serves
 *                 every face), 1 characteristic (Sec. 3.4.1: per direction,
 *                 Phi = L and Phi^{-1} = R from the eigenvectors of that
 *                 direction's flux Jacobian at the central cell average, and
 *                 the weights recomputed per direction for its two faces).
 *                 Characteristic variables run on the FP64 path and on the
 *                 FP32 path in 2D and in 3D at radius 2; with dims = 3,
 *                 radius 3 in the FP32 mode the hot-path calls return
 *                 KFVM_ERR_STATE.
 *   "riemann"     0 HLLC (default), 1 HLL; Batten wave speeds (Sec. 5.4).
 *   "positivity"  1 (default) apply the positivity-preserving limiter of
 *                 Sec. 4 to the Riemann states; 0 off.
 *   "kappa", "eta"  bound relaxation and flattener of Sec. 4.1 (0.1, 0).
 *   "eps"         epsilon of the nonlinear weights, Eq. 24 (1e-40).
 *                 (3 is set by kfvm_set_smooth_mask: gated by a caller mask.)
 *   "gate_threshold"  probability above which a cell is treated as smooth (0.5).
 *   "kxrcf_m"     power m of the KXRCF threshold Delta^m (Sec. 3.5: 3/2),
 *                 0 < m <= 16.
 *   "tensor_cores" 1 (default) / 0: in the FP32 mode with dims = 3, radius 3,
 *                 run the stencil contraction on the tcgen05 tensor cores (FP16
 *                 hi/lo split operands, FP32 accumulation in tensor memory) or
 *                 on the FP32 pipe.  Ignored elsewhere.
 *   "slab_planes" 3D only: process kfvm_step / kfvm_rhs in z-slabs of this many
 *                 planes.  The Riemann-state buffer holds the whole grid's
 *                 float64 states up to 24 GiB; above that the library picks
 *                 the slabs itself (as few as the buffer holds, the float32
 *                 mode's half-size states taking twice the planes), and a
 *                 slab of S planes needs S + 2 planes of states: a larger
 *                 value is lowered to fit.  Results do not depend on the slab
 *                 size.
 *   "timeout_probe" 1: test hook of the bounded device waits: the next
 *                 tensor-core launch waits on a barrier phase nothing completes,
 *                 gives up after a short limit, raises the timeout flag (read by
 *                 kfvm_sync_status as KFVM_ERR_TIMEOUT) and does no work; the
 *                 option resets itself and the context stays usable.
 *   "profile"     1: time every hot-path launch with CUDA events (see
 *                 kfvm_profile_get); 0 (default) off.
 * Errors: KFVM_ERR_ARG for an unknown key or value out of range. */
kfvm_status kfvm_set_option(kfvm_ctx* ctx, const char* key, double value);

/* ------------------------------------------------------------------------- */
/* The hot path (Sec. 5.3, stage (iii) of the method)                         */
/* ------------------------------------------------------------------------- */

/* Riemann states at every face Gauss point of every cell (Sec. 5.3 steps 1-3):
 * ghost-cell map, linearized primitive transform (Eq. 33, appendix A with the
 * exact inverse; or the characteristic transform of each direction, option
 * "variables"), contraction with the weight tables, smoothness indicators
 * (Eq. 22), nonlinear weights (Eqs. 24-25), WENO-AO blend (Eq. 19), back
 * transform (Eq. 28), then the positivity limiter (Sec. 4) when enabled.
 * U: device, float64 state.  faces: device, F*nv*ncell values in the layout
 * and type described above.  Errors: KFVM_ERR_ARG, KFVM_ERR_STATE (weights
 * not built, no network loaded in the gated mode, characteristic variables in
 * the FP32 mode), KFVM_ERR_CUDA (launch); non-admissible states raise the
 * device flag. */
kfvm_status kfvm_reconstruct(kfvm_ctx* ctx, const double* U, void* faces, void* stream);

/* Flux divergence from Riemann states (Sec. 5.3 steps 4-6): exterior states at
 * physical boundaries (periodic: the neighbour's; outflow: a copy of the
 * interior state), HLLC/HLL at every face Gauss point, Gauss-Legendre face
 * average, dUdt = -sum_d (F_{d,+} - F_{d,-}) / Delta_d.
 * faces: device, as written by kfvm_reconstruct in the same precision mode.
 * dUdt: device, float64 [var][cell]. */
kfvm_status kfvm_flux(kfvm_ctx* ctx, const void* faces, double* dUdt, void* stream);

/* Allocation-free variant of kfvm_flux, for callers that must not allocate
 * device memory at all: plug-ins whose host application owns the whole
 * device-memory budget through its own pool, and latency-sensitive loops in
 * which cudaMalloc / cudaFree (which may synchronise the device) are not
 * allowed.  It needs no context: the caller passes the grid, dims (2 or 3),
 * radius (2 or 3), gamma, the Riemann solver (0 HLLC, 1 HLL), float64
 * conservative Riemann states `faces` (device, the layout of kfvm_reconstruct
 * in the FP64 mode) and the output dUdt (device, float64 [var][cell]).  The
 * paper has no counterpart of this entry point.
 *
 * Scratch: the face-averaged fluxes live in one fixed device array of
 * 16 MiB (plus a 256-byte status word) that every GPU loading the library
 * holds until the process exits.  Problems whose fluxes need more,
 * (dims+2) * sum_d (n_d+1) * prod_{e != d} n_e * 8 bytes > 16 MiB
 * (in 2D up to 511 x 511 cells, in 3D up to 51^3), are rejected with
 * KFVM_ERR_TOO_LARGE before any device work.  Nothing is allocated: no
 * cudaMalloc, no cudaFree, no allocating library routine.  The first call
 * made with a given device current looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  Every call shares the one array and overwrites it, so
 * calls that overlap on the GPU (on different streams, or from different
 * threads) race and must be serialised by the caller.  The status word is
 * cleared at the start of each call; if status_out (device int*) is non-NULL
 * it receives the call's device status bits (1 = non-admissible state).
 * Errors: KFVM_ERR_ARG, KFVM_ERR_TOO_LARGE, KFVM_ERR_CUDA. */
kfvm_status kfvm_flux_static(const kfvm_grid* grid, int dims, int radius, double gamma, int riemann,
                             const double* faces, double* dUdt, int* status_out, void* stream);

/* dUdt = L(U): kfvm_reconstruct followed by kfvm_flux through the library's
 * own face buffer. */
kfvm_status kfvm_rhs(kfvm_ctx* ctx, const double* U, double* dUdt, void* stream);

/* One SSP-RK3 (Shu-Osher) step of U in place:
 *   U1 = U + dt L(U);  U2 = 3/4 U + 1/4 (U1 + dt L(U1));  U = 1/3 U + 2/3 (U2 + dt L(U2)),
 * with dt = cfl / max_cells sum_d (|u_d| + c)/Delta_d computed on the device
 * from U and clipped to t_remaining.  The step never leaves the device: dt
 * stays in device memory.  If dt_out is non-NULL the call synchronises the
 * stream, writes dt to *dt_out and returns the device status flag.  U must
 * not alias the library's scratch.  Errors: as kfvm_reconstruct. */
kfvm_status kfvm_step(kfvm_ctx* ctx, double* U, double cfl, double t_remaining, double* dt_out, void* stream);

/* Synchronise the stream and return (and clear) the device status flag. */
kfvm_status kfvm_sync_status(kfvm_ctx* ctx, void* stream);

/* ------------------------------------------------------------------------- */
/* Troubled-cell indicator (Sec. 3.5): which cells need WENO-AO               */
/* ------------------------------------------------------------------------- */

/* The KXRCF troubled-cell indicator of Sec. 3.5, adapted there from
 * discontinuous Galerkin methods, evaluated as in Sec. 5.3 step 2 items 1-2.
 * Every cell of U gets its unlimited linear S0 reconstruction of the
 * conservative variables at its face Gauss points; at each point s of the
 * cell's faces the entropy q = p / rho^gamma of that state and of the state
 * the cell across the face reconstructs at the same point are compared, and
 * the cell is smooth when  max_s |q+ - q-| / <Q>  <  Delta^m  with
 * <Q> = p / rho^gamma of the cell average, Delta the largest cell width and m
 * the "kxrcf_m" option.  Faces on an outflow boundary carry no jump (the
 * exterior state copies the interior one, Sec. 5.3 step 4), periodic faces
 * compare with the wrapped neighbour; a non-admissible state (rho <= 0,
 * p <= 0, not finite) at a point or in the average flags the cell.
 * mask_out: device, one byte per cell in the state's cell order, 1 = smooth
 * (linear reconstruction), 0 = flagged (WENO-AO).  In the FP32 mode the
 * reconstruction and the comparison run in float32 on the float32 copy of U,
 * as the "recon" 4 step does; in the FP64 mode in float64 on U.  The
 * library's scratch (the float32 copy) is overwritten; nothing is allocated.
 * Errors: KFVM_ERR_ARG (null pointer), KFVM_ERR_STATE (weights not built),
 * KFVM_ERR_CUDA (launch). */
kfvm_status kfvm_kxrcf_mask(kfvm_ctx* ctx, const double* U, unsigned char* mask_out, void* stream);

/* ------------------------------------------------------------------------- */
/* Learned gate (an extension, no counterpart in the paper; it plays the role  */
/* of the troubled-cell indicator of Sec. 3.5: cells it marks smooth skip     */
/* WENO, exactly as the indicator's unflagged cells do, Sec. 5.3 step 2).    */
/* ------------------------------------------------------------------------- */

/* Network: in -> 32 -> 32 -> 1, ReLU hidden layers, sigmoid output; the input
 * is the radius-2 full stencil of rho and p (cell-average pressure), each as
 * deviations from the central value divided by d = max(max |deviation|,
 * 1e-4 |central value|): 2*|S0(R=2)| values (26 in 2D, 66 in 3D).  In 3D two
 * more inputs, m/(m + d) with m = max |deviation| over the shell
 * 4 < |o|^2 <= 9 of rho and of p, let the network see what a radius-3
 * reconstruction reads (zero when the radius is 2): in = 68 in 3D.
 * Parameters are float32 masters; inference and training run in BF16 with
 * FP32 accumulation.  Packed parameter order: W1 [32][in], b1 [32],
 * W2 [32][32], b2 [32], W3 [1][32], b3 [1]. */
size_t kfvm_gate_param_count(const kfvm_ctx* ctx);
kfvm_status kfvm_gate_set_params(kfvm_ctx* ctx, const float* host_params, size_t count);
kfvm_status kfvm_gate_get_params(kfvm_ctx* ctx, float* host_params, size_t count);

/* Gate inputs and WENO-AO training labels of every cell of U:
 * X (device, float32 [ncell][in]) and y (device, float32 [ncell]) with
 * y = 1 when the density and the pressure components of the linearized
 * primitive variables each either have omega_0/gamma_0 >= 1 - tau (the cell's
 * own WENO-AO weights at the context's radius say it is smooth) or vary over
 * S0 by at most 1e-4 of their scale, else 0.  The deltas are formed in float64. */
kfvm_status kfvm_gate_features(kfvm_ctx* ctx, const double* U, float* X, float* y, double tau, void* stream);

/* The smooth mask the gated step computes from U with the loaded network
 * (device, one byte per cell, 1 = the network's probability exceeds
 * "gate_threshold"), written to mask_out (device).  In the FP32 mode the
 * features come from the float32 copy of U, as in the step. */
kfvm_status kfvm_gate_mask(kfvm_ctx* ctx, const double* U, unsigned char* mask_out, void* stream);

/* Use a caller-supplied smooth mask (device, one byte per cell, 1 = linear
 * reconstruction, 0 = WENO-AO) instead of the network: sets the gated mode
 * ("recon" 3) with this mask until "recon" is set again.  Lets another
 * troubled-cell indicator drive the gated path, and tests compare the gated
 * path with the oracle on one mask.  The mask is copied on the stream. */
kfvm_status kfvm_set_smooth_mask(kfvm_ctx* ctx, const unsigned char* mask, void* stream);

/* Smooth-cell probabilities prob (device, float32 [n]) for inputs X. */
kfvm_status kfvm_gate_forward(kfvm_ctx* ctx, const float* X, float* prob, size_t n, void* stream);

/* One Adam step (lr, beta1 0.9, beta2 0.999, eps 1e-8) on the mean binary
 * cross-entropy of the batch (X, y) of n samples; the batch loss is written
 * to *loss_dev (device float32) when non-NULL.  grads_out (device float32,
 * kfvm_gate_param_count values) receives the batch gradient when non-NULL. */
kfvm_status kfvm_gate_train_step(kfvm_ctx* ctx, const float* X, const float* y, size_t n, float lr,
                                 float* loss_dev, float* grads_out, void* stream);

/* Load the network from host memory: the packed parameters of
 * kfvm_gate_set_params as float32 (bytes = 4 * kfvm_gate_param_count) or as
 * bfloat16 (bytes = 2 * count, widened exactly to the float32 masters).
 * Errors: KFVM_ERR_ARG for any other size. */
kfvm_status kfvm_gate_load(kfvm_ctx* ctx, const void* host_weights, size_t bytes);

/* `epochs` passes of Adam steps (kfvm_gate_train_step) over the n samples
 * (X: device float32 [n][in], y: device float32 [n]) in consecutive
 * mini-batches of 2048, in order (shuffle X, y beforehand if wanted).
 * Errors: KFVM_ERR_ARG, KFVM_ERR_STATE (no network loaded), KFVM_ERR_CUDA. */
kfvm_status kfvm_gate_train(kfvm_ctx* ctx, const float* X, const float* y, size_t n, int epochs, float lr,
                            void* stream);

/* ------------------------------------------------------------------------- */
/* Introspection and lifetime                                                  */
/* ------------------------------------------------------------------------- */

/* Host-only stencil description (no GPU needed): sizes[q] = N_q and
 * degrees[q] = p_q for q = 0..N_S (arrays of at least 8), *nface = F,
 * *nderiv = M; returns the number of (sub)stencils N_S + 1, or -1 for an
 * unsupported (dims, radius). */
int kfvm_stencil_info(int dims, int radius, int* sizes, int* degrees, int* nface, int* nderiv);

/* Number of kernels the library launched on this context since creation
 * (for launch accounting). */
long long kfvm_launch_count(const kfvm_ctx* ctx);

/* Per-kernel device timing (tracing).  With the option "profile" = 1 every
 * hot-path launch is bracketed by CUDA events on its stream.  After the
 * caller has synchronised that stream, kfvm_profile_get(ctx, i, ...) returns
 * for kernel family i (0 <= i < kfvm_profile_count()) its name, the number of
 * launches and their summed device time in milliseconds since the last
 * kfvm_profile_reset.  Errors: KFVM_ERR_ARG (bad index), KFVM_ERR_CUDA (an
 * event not yet complete: synchronise first). */
int kfvm_profile_count(void);
kfvm_status kfvm_profile_get(kfvm_ctx* ctx, int index, const char** name, long long* launches, double* ms);
kfvm_status kfvm_profile_reset(kfvm_ctx* ctx);

/* Measure the device's FP64 (bits = 64) or FP32 (bits = 32) FMA throughput
 * with a register-only multiply-add loop on every SM; writes flop/s to
 * *flops.  Synchronous. */
kfvm_status kfvm_measure_fma_peak(int bits, double* flops);

void kfvm_destroy(kfvm_ctx* ctx);
const char* kfvm_status_string(kfvm_status s);

#ifdef __cplusplus
}
#endif

#endif /* KFVM_H */
