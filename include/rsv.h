/*
 * rsv.h - C ABI of the GB300 resolvent time-march library (librsv.so).
 *
 * The library computes the action of the resolvent of a stable linear system
 *     du/dt = A u + B f(t),   y = C u      (B, C diagonal; B = C = I by default)
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
  RSV_PREC_FP32 = 1, /* state, operator and products in FP32; DFT accumulators and
                        the per-frequency QR/SVD glue in FP64                        */
  RSV_PREC_BF16_STATE = 2 /* as RSV_PREC_FP32 (complex64 blocks), with the march state and
                        stage inputs stored in BF16 (arithmetic, RK4 accumulator,
                        forcing and snapshot tiles in FP32); ADV3D with nx a multiple
                        of 4.  BF16 storage rounds to 2^-8 relative per step: use the
                        FP64 refinement pass (rsv_refine_gains) for accurate gains    */
} rsv_precision;

typedef enum {
  RSV_SCHEME_RK4 = 0, /* classical 4-stage Runge-Kutta, forcing at t_n, t_n + h/2, t_n + h      */
  RSV_SCHEME_CN = 1   /* Crank-Nicolson (I - hA/2) u' = (I + hA/2) u + h/2 (f(t_n) + f(t_n + h)),
                         second order, GL1D only (Sec. 3)                                   */
} rsv_scheme;

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

  /* RSV_OP_GL1D: du/dt = -nu u_x + gamma u_xx + mu(x) u, mu = mu0 + mu_shift + mu1 x + mu2 x^2,
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

  /* RSV_OP_GL1D: linear term of mu(x) (the paper's Sec. 3 case has mu linear in x). */
  double mu1;
  /* Time scheme (rsv_scheme): classical RK4 for every kind, or Crank-Nicolson
   * for RSV_OP_GL1D (the scheme of the paper's Sec. 3 validation case). */
  int32_t scheme;
} rsv_operator_desc;

typedef struct {
  int32_t variant;              /* rsv_variant                                      */
  int32_t n_transient_windows;  /* SSRM: forced windows before the analysed one;
                                   -1 = as many as the decay run of rsv_decay_probe
                                   needs (Sec. 2.3): ceil(decay steps / N_T), with
                                   decay_tol / decay_max_steps / decay_seed below,
                                   check points every tile_steps steps; the run is
                                   made once per operator, direction and setting and
                                   remembered until the frequencies change.  A probe
                                   that grows or does not decay: RSV_ERR_UNSTABLE.  */
  int64_t tail_steps;           /* TRM: unforced steps after the forcing window
                                   (the cap on the tail when tail_tol > 0)          */
  int32_t tile_steps;           /* steps per time tile S (0 = library default)      */
  int32_t group_vectors;        /* most test vectors marched together (0 = the
                                   library's choice: all k, halved until the march
                                   workspace fits, or rsv_autotune's choice)        */
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
  double decay_tol;             /* n_transient_windows = -1: the probe's norm ratio
                                   target (0 = 1e-8)                                 */
  int64_t decay_max_steps;      /* n_transient_windows = -1: cap on the probe's steps
                                   (0 = 1000 windows of N_T steps)                   */
  uint64_t decay_seed;          /* n_transient_windows = -1: SplitMix64 stream of the
                                   probe's random initial state                     */
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

/* Forcing matrix B, observation matrix C and the metrics of the forcing and
 * observation spaces (Sec. 2.1: y = C u, the inner products <a, b>_W = a^H W b
 * and the adjoints B^dag = W_f^{-1} B^H W_u, C^dag = W_y^{-1} C^H W_u), all
 * diagonal over the state: host arrays of n doubles (read during the call),
 * NULL = identity; all four NULL clears them.  b, c >= 0 (masks or weights in
 * space), w_f, w_y > 0 (e.g. quadrature weights).  Afterwards
 *   rsv_march_direct  returns y_hat = C R_h B f_hat,
 *   rsv_march_adjoint returns w_hat = R_y^dag y_hat = W_f^{-1} B^H R_h^H C^H W_y y_hat
 *                     (the state metric W_u cancels from the adjoint run's output),
 *   rsv_gains_modes / rsv_refine_gains work on W_y^{1/2} C R_h B W_f^{-1/2}: gains
 *   ||y||_{W_y} / ||f||_{W_f}, forcing modes unit in W_f, response modes unit in
 *   W_y (the refinement basis is W_f-orthonormalised);
 * rsv_orthonormalize stays Euclidean.  Errors: INVALID_ARG (negative,
 * non-finite or zero metric entries), OOM, CUDA. */
rsv_status rsv_set_weights(rsv_operator op, const double* b, const double* c, const double* w_f, const double* w_y);

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
 * memory once running - a host solver that reserves the whole device-memory
 * budget for its own pool at start-up and forbids any later cudaMalloc, or a
 * real-time loop that must never stall on the allocator (cudaMalloc and
 * cudaFree can synchronise the device).  rsv_march_direct grows the
 * operator's workspace on demand; this entry point instead keeps the march's
 * scratch (state, forcing and snapshot tiles, FP64 accumulators) in one
 * static device array of RSV_STATIC_SCRATCH_BYTES that every GPU loading the
 * library holds until the process exits.  Arguments and result are those of
 * rsv_march_direct (same y_hat to rounding) for the GL1D kind; TRM runs its
 * whole tail (tail_tol must be 0).  The tile length is halved until the
 * scratch fits; if it cannot fit, RSV_ERR_INVALID_ARG names the bytes
 * needed.  All calls share the array and each clears what must start at
 * zero; calls whose device work overlaps race on it.  Like every other
 * entry point the call ends by synchronising the operator's stream.  The
 * first call on a device takes the array's device address
 * (cudaGetSymbolAddress) with that device current: make it before any
 * stream capture begins.  The operator and its frequencies must already
 * exist (rsv_create_operator / rsv_set_frequencies allocate). */
rsv_status rsv_march_direct_static(rsv_operator op, const void* f_hat, int32_t k, const rsv_march_opts* opts,
                                   void* y_hat);

/* Decay run (Sec. 2.3: the transient length of the steady-state method is
 * estimated from a prior run in which the norm of a random initial condition
 * falls to a prescribed small value).  Marches the unforced system
 * du/dt = A u (adjoint = 1: A^H) with the operator's step h from the random
 * state u_0 whose entries are uniform in [-1, 1): value i of the SplitMix64
 * stream `seed` (Steele, Lea & Flood 2014; increment 0x9E3779B97F4A7C15),
 * top 53 bits as 2 (z >> 11) 2^-53 - 1; a complex state takes values 2p and
 * 2p + 1 as the real and imaginary parts of entry p, a real state value p.
 * Every check_every steps (0 = the default tile length) it takes, per
 * instance, ||u_i|| / ||u_0,i|| and stops at the first check point where the
 * largest of them is <= tol.  Outputs (host, nullable): *steps marched and
 * *ratio (largest instance ratio) there.  Errors: RSV_ERR_UNSTABLE when a
 * ratio exceeds 1e6 or turns non-finite at a check point (the system grows),
 * or when max_steps pass without decay (outputs still written);
 * INVALID_ARG (tol not in (0, 1), max_steps < 1); STATE (no frequencies:
 * h is set by rsv_set_frequencies). */
rsv_status rsv_decay_probe(rsv_operator op, int32_t adjoint, double tol, int64_t max_steps, uint64_t seed,
                           int32_t check_every, int64_t* steps, double* ratio);

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

/* rsv_gains_modes with the test block drawn by the library from a seed: entry
 * e of the [n_omega][k][n] block (row-major) takes the values 2e and 2e + 1 of
 * the SplitMix64 stream `seed` (Steele, Lea & Flood 2014; top 53 bits:
 * u1 = (x + 1) 2^-53, u2 = x 2^-53) through the Box-Muller transform, giving
 * (z0 + i z1) / sqrt(2) with z0 + i z1 = sqrt(-2 ln u1) exp(2 pi i u2); for a
 * real-state operator the w = 0 row holds the real N(0, 1) values z0.  The
 * block lives in a library workspace.  Other arguments and errors as for
 * rsv_gains_modes. */
rsv_status rsv_gains_modes_seeded(rsv_operator op, int32_t k, int32_t n_power_iter, int32_t n_modes, uint64_t seed,
                                  const rsv_march_opts* opts, double* gains, void* forcing_modes,
                                  void* response_modes);

/* Rayleigh-Ritz refinement on a given forcing basis (App. A: gains and modes
 * estimated from the eigen-decomposition of R^H R projected onto a subspace).
 * With Q the orthonormalised basis (CholeskyQR2 per frequency and instance),
 * one direct run gives Y = R Q, and the eigen-decomposition of
 * Y^H Y = Q^H R^H R Q = W S^2 W^H yields gains S (descending), forcing modes
 * Q W and response modes Y W S^{-1}.  Made on an RSV_PREC_FP64 operator with
 * the basis of a lower-precision randomized SVD (its forcing modes, n_modes
 * = k), this is the FP64 refinement pass: the gain error becomes quadratic in
 * the basis error.  basis: device [n_omega][k][n] of the operator's element
 * type (read only; for real-state kinds the w = 0 row must be real, its
 * imaginary part is ignored).  gains: HOST [n_instances][n_omega][n_modes];
 * forcing_modes / response_modes: DEVICE [n_omega][n_modes][n] (nullable).
 * n_modes <= k <= 32, k <= every instance's length.  Errors: INVALID_ARG,
 * STATE, DIVERGED (basis loses rank), and those of the march. */
rsv_status rsv_refine_gains(rsv_operator op, const void* basis, int32_t k, int32_t n_modes,
                            const rsv_march_opts* opts, double* gains, void* forcing_modes, void* response_modes);

/* Optimal and suboptimal gains by the Arnoldi algorithm (App. A: the runs give
 * w = R^H R f; each new forcing f_{n+1} is the part of w_n orthogonal to
 * f_0 .. f_n, Eq. (freqOrt); the projection H = F^H W of R^H R on the
 * orthonormal Krylov basis F is Hermitian tridiagonal, and H psi = gamma^2 psi
 * gives gains gamma, forcing modes F psi and response modes R F psi / gamma).
 * One vector per frequency and instance, m iterations = m direct + m adjoint
 * runs; classical Gram-Schmidt with one reorthogonalisation.  f0: device
 * [n_omega][1][n] start vectors of the operator's element type (for real-state
 * kinds the w = 0 row must be real).  gains: HOST [n_instances][n_omega][n_modes]
 * descending; forcing_modes / response_modes: DEVICE [n_omega][n_modes][n]
 * (nullable), unit norm (in W_f / W_y with rsv_set_weights).  1 <= n_modes <= m
 * <= 31, m <= every instance's length.  Errors: INVALID_ARG, STATE, DIVERGED
 * (the Krylov space stopped growing), and those of the march. */
rsv_status rsv_arnoldi_gains(rsv_operator op, const void* f0, int32_t m, int32_t n_modes,
                             const rsv_march_opts* opts, double* gains, void* forcing_modes, void* response_modes);

/* Orthonormalise a block in place, per frequency and instance (CholeskyQR2:
 * the QR factorisation with a positive real diagonal in R; the per-frequency
 * normalisation and orthogonalisation of Fourier blocks of Sec. 2.3).
 * block: device [n_omega][k][n] of the operator's element type.  r_factor:
 * HOST [n_omega][n_instances][k][k] complex128 (re, im) row-major, upper
 * triangular, block = Q R (nullable).  Errors: INVALID_ARG, STATE, DIVERGED
 * (a block is rank deficient). */
rsv_status rsv_orthonormalize(rsv_operator op, void* block, int32_t k, double* r_factor);

/* y = A x (adjoint = 0) or y = A^H x (adjoint = 1) for a device block x, y [k][n]
 * of the operator's element type (complex for every kind; real-state kinds
 * act on real and imaginary parts alike).  For testing the operator kernels. */
rsv_status rsv_apply_operator(rsv_operator op, const void* x, int32_t k, int32_t adjoint, void* y);

/* rsv_march_direct / rsv_march_adjoint with the input block in HOST memory
 * (f_hat_host / y_hat_host: [n_omega][k][n] of the operator's element type;
 * pinned memory lets the copies run asynchronously).  The march processes the
 * vectors in groups (see rsv_march_opts.group_vectors); each group's slice of
 * the block is copied to a device staging buffer on a second stream while the
 * previous group marches (two staging buffers), so the host-to-device transfer
 * overlaps the march.  Output as for the device versions (device y_hat /
 * w_hat).  Returns when the march is done.  Errors: those of the device
 * versions, OOM (staging buffers). */
rsv_status rsv_march_direct_host(rsv_operator op, const void* f_hat_host, int32_t k, const rsv_march_opts* opts,
                                 void* y_hat);
rsv_status rsv_march_adjoint_host(rsv_operator op, const void* y_hat_host, int32_t k, const rsv_march_opts* opts,
                                  void* w_hat);

/* Measured choice of the march's time-tile length and vector-group size for
 * marches of k vectors with these options.  Candidates: the default tile and
 * half of it, times groups of k, k/2, k/4 and 1 vectors that fit in device
 * memory next to what is allocated; each is timed on one synthesised, marched
 * and analysed tile of the first vector group of f_hat (device [n_omega][k][n],
 * the block a following march will use; nothing is written to it), and the
 * configuration with the least time per vector-step is kept in the operator
 * for later marches of k vectors whose opts->tile_steps is 0.  tile, group:
 * host (nullable), the chosen values.  Errors: INVALID_ARG, STATE, OOM (no
 * candidate fits), and those of the march. */
rsv_status rsv_autotune(rsv_operator op, const void* f_hat, int32_t k, const rsv_march_opts* opts, int32_t* tile,
                        int32_t* group);

/* ---------------------------------------------------------------------------
 * Transient-response method in time-series form (Sec. 2.2 with App. B and C).
 *
 * A run is driven by a sampled series instead of Fourier coefficients: its
 * forcing at the stage times of each step (RK4: t_n, t_n + h/2, t_n + h;
 * Crank-Nicolson: t_n, t_n + h) is the App. C interpolant of the input series,
 * whose samples lie every `every` steps from t = 0, and is zero after the last
 * sample; the state is recorded every `every` steps.  Series are device arrays
 * [n_snap][k][n] of the state's element type: complex (re, im) for complex-
 * state kinds, real for real-state kinds, FP64 or FP32 by the operator's
 * precision.  The time step is the operator's h (rsv_set_frequencies must come
 * first).  Kinds: GL1D (RK4 or Crank-Nicolson), ADR2D and ADV3D (RK4); not the
 * dense kind, BF16 state or operators with rsv_set_weights.
 * ------------------------------------------------------------------------- */
typedef enum { RSV_INTERP_C0 = 0, RSV_INTERP_C1 = 1, RSV_INTERP_C2 = 2 } rsv_interp;

typedef struct {
  int32_t every;      /* steps between input samples and between recorded snapshots (>= 1) */
  int32_t interp;     /* rsv_interp: C0 linear, C1 cubic Hermite, C2 quintic Hermite (App. C) */
  double tail_tol;    /* truncation (Sec. 2.2): vector v's record ends at the first snapshot at or
                         after the end of its forcing whose norm is <= tail_tol x the largest norm of
                         its snapshots so far; later snapshots are zero.  0: no truncation. */
} rsv_series_opts;

/* One series-driven run.  u(0) = init (device [k][n], nullable: zero), forcing
 * from `forcing` (device [n_in][k][n], nullable; sample i is read from row
 * n_in - 1 - i when reverse_in = 1, the time reversal that turns a direct
 * run's output into its adjoint run's forcing, Sec. 2.1).  adjoint = 1 marches
 * with A^H.  out (device [n_out_max][k][n], must not alias forcing): snapshot j
 * = u(j every h), j = 0 the initial state.  The run ends when every vector has
 * stopped (tail_tol) or after n_out_max snapshots.  *n_out (host): snapshots
 * written, rows >= *n_out untouched.  stops (host [k], nullable): the
 * snapshot at which each vector stopped, -1 if it did not.  Errors:
 * INVALID_ARG, STATE, DIVERGED, CUDA, OOM. */
rsv_status rsv_series_march(rsv_operator op, int32_t adjoint, int32_t k, const void* init, const void* forcing,
                            int64_t n_in, int32_t reverse_in, const rsv_series_opts* opts, void* out,
                            int64_t n_out_max, int64_t* n_out, int64_t* stops);

/* Fourier transform of a series at arbitrary frequencies by the rectangle rule
 * (Sec. 2.1 Eq. (fourier), the sign of du/dt = A u + f):
 *   out[j][v][p] = d sum_i x[i][v][p] exp(-i omega_j (t0 + i d)).
 * series: device [n_snap][k][n] (state element type); omega: host
 * [n_omega]; out: device [n_omega][k][n] complex of the operator's precision.
 * Accumulated in FP64.  Errors: INVALID_ARG, CUDA, OOM. */
rsv_status rsv_series_fourier(rsv_operator op, const void* series, int64_t n_snap, int32_t k, double d,
                              double t0, const double* omega, int32_t n_omega, void* out);

/* FIR filtering of a series (App. B), the whole convolution:
 *   out[m][v][p] = sum_j phi_v[j] x[m - j][v][p],  0 <= m < n_in + order,
 * phi_v = taps[v] (reverse_taps = 0) or taps[v] reversed (phi_v[j] =
 * taps[v][order - j]; filtering a time-reversed series: reverse(phi * x) =
 * reversed(phi) * reverse(x)).  taps: host [k][order + 1] complex128 (re, im);
 * for real-state operators the taps must be real.  in: device [n_in][k][n];
 * out: device [n_in + order][k][n], must not alias in.  Errors: INVALID_ARG,
 * CUDA, OOM. */
rsv_status rsv_series_filter(rsv_operator op, const void* in, int64_t n_in, int32_t k, const double* taps,
                             int32_t order, int32_t reverse_taps, void* out);

/* Linear-phase FIR filter by frequency sampling with a Hamming window (App. B):
 * the amplitude A(w) is given at n_pts ascending frequencies w_pts (host),
 * linear in between and constant beyond; if every w_pts >= 0 it is mirrored
 * to negative frequencies (real taps), otherwise it is taken over signed
 * frequencies (complex taps, for complex signals).  The spectrum
 * A(w) exp(-i w order d / 2) on the 8 (order + 1)-point grid of spacing
 * 2 pi / (8 (order + 1) d) is transformed back and its first order + 1 points
 * are windowed.  order even; taps: host [order + 1] complex128 (re, im).
 * Host computation, no device use.  Errors: INVALID_ARG. */
rsv_status rsv_fir_design(int32_t order, double d, const double* w_pts, const double* amp, int32_t n_pts,
                          double* taps);

typedef struct {
  rsv_series_opts series;
  int32_t n_iter;        /* power iterations (>= 1) */
  int32_t filter_order;  /* order of the flattening filter, even; 0: no filter, scalar normalisation */
  int64_t n_snap_max;    /* snapshot capacity of each run's record */
} rsv_trm_opts;

/* Power iteration on R^H R by the transient-response method (Sec. 2.2, App. A
 * Eqs. (iteration), (tildeSig)), each of the k vectors independently.
 * Iteration 0 starts from the impulse f0 delta(t), applied as u(0) = f0
 * (device [k][n], state element type).  Each iteration: a direct run, an
 * adjoint run forced by the direct output reversed in time, w = the adjoint
 * output reversed back; the gain estimate sigma(w)^2 = |w_hat(w)| / |f_hat(w)|
 * at the n_omega frequencies omega (host); the next forcing is w filtered by
 * the FIR filter of amplitude 1 / |w_hat(w)| at those frequencies (App. B),
 * or, with filter_order = 0, w / max_w |w_hat(w)|.  gains: host
 * [n_iter][n_omega][k]; w_hat (device [n_omega][k][n] complex, nullable): the
 * last iteration's w_hat, the direction of the leading forcing mode, with w
 * on the time axis t_i = i d (d = every h).  Errors: those of the runs, and
 * INVALID_ARG when a record fills n_snap_max before it is negligible. */
rsv_status rsv_trm_power_iteration(rsv_operator op, const void* f0, int32_t k, const double* omega,
                                   int32_t n_omega, const rsv_trm_opts* opts, double* gains, void* w_hat);

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
