/*
 * rsv.h - C ABI of the GB300 resolvent time-march library (librsv.so).
 *
 * The library computes the action of the resolvent of a stable linear system
 *     du/dt = A u + f(t),   y = u                       (B = C = I)
 * on Fourier coefficients for many frequencies at once by time marching,
 * and the resolvent gains and modes from it (Martini, Rodriguez, Towne &
 * Cavalieri, "Efficient computation of global resolvent modes", Sec. 2).
 *
 * Conventions shared by every entry point
 *   - Sign convention: forcing f(t) = sum_j fhat_j exp(+i w_j t); the result is
 *     yhat_j = R(w_j) fhat_j with R(w) = (i w I - A)^{-1} up to the RK4
 *     discretisation.  The paper writes du/dt + A_p u = B f with signals
 *     exp(-i w t) (Sec. 2.1, Eqs. (system), (fourier)); A = -A_p.
 *   - Coefficient blocks (fhat, yhat, what, test vectors, modes) are DEVICE
 *     buffers owned by the caller, complex numbers stored (re, im)
 *     interleaved, row-major [n_omega][k][n]: frequency slowest, state index
 *     fastest.  Element type: complex128 when the operator was created with
 *     RSV_PREC_FP64, complex64 with RSV_PREC_FP32.
 *   - All device work runs on the CUDA stream given at creation.  Every call
 *     returns after its work has completed (it synchronises that stream).
 *   - Errors: every function returns an rsv_status; nothing throws across the
 *     ABI.  rsv_last_error() gives a message for the calling thread's last
 *     failing call.  A failed call leaves caller buffers unspecified.
 *   - Workspace (state, forcing tiles, accumulators, glue buffers) is owned
 *     by the operator object and freed by rsv_destroy_operator.
 */
#ifndef RSV_H
#define RSV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rsv_operator_s* rsv_operator;

typedef enum {
  RSV_OK = 0,
  RSV_ERR_INVALID_ARG = 1,       /* a null pointer, size or enum out of range     */
  RSV_ERR_UNSTABLE = 2,          /* RK4 amplification or decay probe says unstable */
  RSV_ERR_NOT_COMMENSURATE = 3,  /* frequencies not on one grid (m_j + phi) dw    */
  RSV_ERR_DIVERGED = 4,          /* state norm became NaN/Inf during a march       */
  RSV_ERR_TIMEOUT = 5,           /* a bounded device wait gave up                  */
  RSV_ERR_OOM = 6,               /* device allocation failed                       */
  RSV_ERR_CUDA = 7,              /* any other CUDA runtime error                   */
  RSV_ERR_STATE = 8              /* call order: e.g. march before frequencies      */
} rsv_status;

typedef enum {
  RSV_OP_GL1D = 0,   /* batched linearised complex Ginzburg-Landau, 3-point FD     */
  RSV_OP_DENSE = 1,  /* caller-supplied dense complex matrix A                     */
  RSV_OP_ADR2D = 2,  /* 2-D scalar advection-diffusion-reaction, 5-point (real)    */
  RSV_OP_ADV3D = 3   /* 3-D 3-component advection-diffusion, 7-point (real)        */
} rsv_op_kind;

typedef enum {
  RSV_PREC_FP64 = 0, /* everything in FP64; parity path                             */
  RSV_PREC_FP32 = 1  /* state, operator and products in FP32; DFT accumulators and
                        the per-frequency QR/SVD glue in FP64                        */
} rsv_precision;

typedef enum {
  RSV_SSRM = 0,      /* steady-state response: periodic forcing (Sec. 2.3)          */
  RSV_TRM = 1        /* transient response: one forcing window + decay tail (Sec. 2.2) */
} rsv_variant;

/* System description.  Only the fields of the chosen kind are read.
 * Grids are interior points with homogeneous Dirichlet boundaries. */
typedef struct {
  int32_t kind;              /* rsv_op_kind                                          */
  int32_t precision;         /* rsv_precision                                        */
  double dt;                 /* target step; the march uses h = T / ceil(T / dt)     */

  /* RSV_OP_GL1D: du/dt = -nu u_x + gamma u_xx + mu(x) u, mu = mu0 + mu_shift + mu2 x^2,
   * on x in (x0, x1); instance i has gl_n[i] points and its own mu0 (Sec. 3,
   * Eq. (GL_timeDomain) family).  Instances are independent diagonal blocks. */
  int32_t n_instances;
  const int32_t* gl_n;       /* host [n_instances]                                   */
  const double* gl_mu0;      /* host [n_instances]                                   */
  double x0, x1;
  double nu_re, nu_im, gamma_re, gamma_im;
  double mu_shift, mu2;

  /* RSV_OP_DENSE: A given as host complex128, row-major [dense_n][dense_n]. */
  int32_t dense_n;
  const double* dense_a;

  /* RSV_OP_ADR2D: du/dt = -U(y) u_x + visc lap u + (r(y) - sigma) u,
   *   U = 0.5 (1 + tanh((0.5 - |y|) / jet_delta)), r = -kappa dU/dy,
   *   sigma = sponge_amp ((S - d) / S)^2 within S = sponge_cells cells of a wall
   *   (d = cell distance to the nearest wall), grid nx x ny on (0,lx) x (-ly/2, ly/2),
   *   state index iy * nx + ix.
   * RSV_OP_ADV3D: du/dt = -(U.grad)u - (u.grad)U + visc lap u, U = (erf(r/delta(x)),0,0),
   *   r = sqrt(y^2 + z^2), delta = delta0 + (delta1 - delta0) x / lx, grid
   *   nx x ny x nz on (0,lx) x (-ly/2,ly/2) x (-lz/2,lz/2), state index
   *   ((c * nz + iz) * ny + iy) * nx + ix for component c. */
  int32_t nx, ny, nz;
  double lx, ly, lz;
  double visc;
  double kappa, jet_delta, sponge_amp;
  int32_t sponge_cells;
  double delta0, delta1;
} rsv_operator_desc;

typedef struct {
  int32_t variant;              /* rsv_variant                                      */
  int32_t n_transient_windows;  /* SSRM: forced windows before the analysed one     */
  int64_t tail_steps;           /* TRM: unforced steps after the forcing window
                                   (the cap on the tail when tail_tol > 0)          */
  int32_t tile_steps;           /* steps per time tile S (0 = library default)      */
  int32_t reserved;             /* must be 0                                        */
  double tail_tol;              /* TRM: 0 = march the whole tail; > 0 = truncate the
                                   record by the state norm (Sec. 2.2; Sec. 3 marches
                                   until the norm is below 1e-9, Sec. 4 until it is
                                   1e-3 of its maximum).  At the end of every time
                                   tile the library takes each vector's 2-norm over
                                   the whole state; the march ends at the first tile
                                   end at or after the end of the forcing window
                                   where every vector of the group is at most
                                   tail_tol times the largest norm it had at any tile
                                   end so far.  Check points are therefore the tile
                                   ends: multiples of the tile length reported by
                                   rsv_describe ("tile="), and the last step.  SSRM
                                   ignores it.  Negative or NaN: INVALID_ARG.       */
} rsv_march_opts;

/* Create an operator.  desc: system description (read during the call only).
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * out: receives the handle.  Builds the operator's coefficient arrays on the
 * device.  Errors: INVALID_ARG (bad kind/sizes), OOM, CUDA. */
rsv_status rsv_create_operator(const rsv_operator_desc* desc, void* cuda_stream, rsv_operator* out);

/* Release the operator and all of its device workspace. NULL is ignored. */
void rsv_destroy_operator(rsv_operator op);

/* State size n (points x components, all instances) and instance count. */
rsv_status rsv_operator_info(rsv_operator op, int64_t* n, int32_t* n_instances, int32_t* real_state);

/* Instance i's offset and length in the state vector. */
rsv_status rsv_instance_range(rsv_operator op, int32_t i, int64_t* offset, int64_t* length);

/* Frequencies w_j (host [n_omega]).  They must lie on one grid w_j = (m_j + phi) dw,
 * integer m_j, common phi in {0, 1/2} (Sec. 2.3: Delta omega = 2 pi / T).  dw: grid
 * spacing, or 0 to take the smallest gap.  Fixes T = 2 pi / dw, N_T = ceil(T / dt),
 * h = T / N_T and the exact twiddle table exp(i pi q / (2 N_T)), q < 4 N_T.
 * Outputs (nullable): n_steps_per_window, h.  Errors: INVALID_ARG,
 * NOT_COMMENSURATE (off-grid or aliasing frequencies), OOM, CUDA.  An unstable
 * system is caught by the march's norm monitor (RSV_ERR_DIVERGED). */
rsv_status rsv_set_frequencies(rsv_operator op, const double* omega, int32_t n_omega, double dw,
                               int64_t* n_steps_per_window, double* h);

/* Direct run (Sec. 2.1 Eq. (system), methods of Sec. 2.2 / 2.3): march
 * du/dt = A u + f(t) from u = 0 with f synthesised from f_hat, and return the
 * response's Fourier coefficients y_hat = R_h(w_j) f_hat_j, where R_h is the
 * resolvent of the RK4-discretised system.  f_hat, y_hat: device
 * [n_omega][k][n] (may not alias).  For real-state kinds the w = 0 row of
 * f_hat must be real (its imaginary part is ignored).  k >= 1. */
rsv_status rsv_march_direct(rsv_operator op, const void* f_hat, int32_t k, const rsv_march_opts* opts,
                            void* y_hat);

/* Adjoint run (Sec. 2.1 Eqs. (adsystem), (adsystemFreqDomain)): the backward
 * march of -dz/dt + A^H z = y, run forward in reversed time as
 * dz/dt = A^H z + y with every w_j negated.  Returns w_hat_j = R_h(w_j)^H y_hat_j. */
rsv_status rsv_march_adjoint(rsv_operator op, const void* y_hat, int32_t k, const rsv_march_opts* opts,
                             void* w_hat);

/* Size in bytes of the fixed device array rsv_march_direct_static works in. */
#define RSV_STATIC_SCRATCH_BYTES (32u << 20)

/* rsv_march_direct without any device allocation.  The paper has no
 * counterpart: this is a service to callers that cannot allocate device
 * memory once running - a host solver that gives the library a fixed memory
 * budget at start-up, a thread recording into a CUDA stream capture, a
 * real-time loop that must not wait on the allocator.  rsv_march_direct
 * grows the operator's workspace on demand; this entry point instead keeps
 * the march's scratch (state, forcing and snapshot tiles, FP64
 * accumulators) in one static device array of RSV_STATIC_SCRATCH_BYTES that
 * every GPU loading the library holds until the process exits.  Arguments
 * and result are those of rsv_march_direct (same y_hat to rounding).  The
 * tile length is halved until the scratch fits; if it cannot fit,
 * RSV_ERR_INVALID_ARG names the bytes needed.  All calls share the array and
 * each clears what must start at zero; calls whose device work overlaps
 * race on it.  The first call on a device takes the array's device address
 * (cudaGetSymbolAddress) with that device current: make it before any stream
 * capture begins.  The operator and its frequencies must already exist
 * (rsv_create_operator / rsv_set_frequencies allocate). */
rsv_status rsv_march_direct_static(rsv_operator op, const void* f_hat, int32_t k, const rsv_march_opts* opts,
                                   void* y_hat);

/* Randomized SVD of R_h(w_j) for every frequency (Sec. 1 cites it; App. A for
 * the power iteration it generalises): Y = R Omega, n_power_iter times
 * {Q = qr(Y), Z = R^H Q, Q = qr(Z), Y = R Q}, Q = qr(Y), W = R^H Q, and the
 * eigen-decomposition of W^H W = B B^H (B = Q^H R) per frequency and instance.
 * omega_block: device [n_omega][k][n] test vectors (for real-state kinds the
 * w = 0 row must be real).  gains: HOST [n_instances][n_omega][n_modes] doubles,
 * descending.  forcing_modes / response_modes: DEVICE [n_omega][n_modes][n]
 * (nullable), unit norm per instance, defined up to a phase.
 * n_modes <= k <= 32 and k <= every instance's length. */
rsv_status rsv_gains_modes(rsv_operator op, const void* omega_block, int32_t k, int32_t n_power_iter,
                           int32_t n_modes, const rsv_march_opts* opts, double* gains, void* forcing_modes,
                           void* response_modes);

/* y = A x (adjoint = 0) or y = A^H x (adjoint = 1) for a device block x, y [k][n]
 * of the operator's element type (complex for every kind; real-state kinds
 * act on real and imaginary parts alike).  For testing the operator kernels. */
rsv_status rsv_apply_operator(rsv_operator op, const void* x, int32_t k, int32_t adjoint, void* y);

/* Kernel-time accounting.  With enable = 1 the operator brackets each group
 * of device launches of one kind with CUDA events on its stream, grouped by
 * category: 0 synthesis, 1 march (operator stages of one time tile),
 * 2 analysis, 3 glue (Gram / combine / coefficient transforms).
 * rsv_profile_read returns, for one category since the last reset, the number
 * of bracketed groups, the number of kernels they launched, and their summed
 * event time in ms (it synchronises the stream).  enable = 0 stops recording;
 * rsv_profile_reset clears the totals. */
rsv_status rsv_profile_enable(rsv_operator op, int32_t enable);
rsv_status rsv_profile_reset(rsv_operator op);
rsv_status rsv_profile_read(rsv_operator op, int32_t category, int64_t* groups, int64_t* kernels, double* ms);

/* One-line description of the operator's execution path (kernels chosen for
 * this GPU, e.g. the dense step's tensor-core variant and resident-CTA
 * capacity) and of the latest march: "tile=" steps per time tile, "group="
 * vectors marched together, "steps=" steps marched by its last vector group
 * (smaller than the schedule when the TRM record was truncated by tail_tol).
 * Written NUL-terminated into buf (host, buflen bytes); a longer description
 * is cut at buflen - 1 characters.  Errors: INVALID_ARG. */
rsv_status rsv_describe(rsv_operator op, char* buf, int32_t buflen);

/* Message of the calling thread's last failing call ("" if none). */
const char* rsv_last_error(void);

/* Library version string. */
const char* rsv_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RSV_H */
