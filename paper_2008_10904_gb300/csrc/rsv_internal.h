// Internal declarations of librsv: complex helpers, the operator object,
// and the kernel launchers each .cu file provides.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rsv.h"

namespace rsv {

// ---------------------------------------------------------------------------
// Complex numbers stored (re, im) interleaved, as at the ABI.
// ---------------------------------------------------------------------------
template <typename R>
struct alignas(2 * sizeof(R)) cpx {
  R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cpx<R> mk(R a, R b) {
  cpx<R> c;
  c.re = a;
  c.im = b;
  return c;
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) {
  return mk<R>(a.re + b.re, a.im + b.im);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) {
  return mk<R>(a.re - b.re, a.im - b.im);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
  return mk<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) {
  return mk<R>(s * a.re, s * a.im);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> conjg(cpx<R> a) {
  return mk<R>(a.re, -a.im);
}
// acc += a * b
template <typename R>
__host__ __device__ __forceinline__ void cfma(cpx<R>& acc, cpx<R> a, cpx<R> b) {
  acc.re = fma(a.re, b.re, fma(-a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(a.im, b.re, acc.im));
}
// acc += conj(a) * b
template <typename R>
__host__ __device__ __forceinline__ void cfma_conj(cpx<R>& acc, cpx<R> a, cpx<R> b) {
  acc.re = fma(a.re, b.re, fma(a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(-a.im, b.re, acc.im));
}

// Phase index of exp(i w_j t) at t = (2 n + sigma) h / 2: q = sgn p_j (2n + sigma) mod 4 N_T,
// with p_j = 2 (m_j + phi) an integer; table[q] = exp(i pi q / (2 N_T)).
__host__ __device__ __forceinline__ int64_t phase_index(int64_t pj, int64_t half_steps, int64_t m4) {
  int64_t q = (pj * half_steps) % m4;
  return q < 0 ? q + m4 : q;
}

// ---------------------------------------------------------------------------
// Operator object
// ---------------------------------------------------------------------------
struct Workspace {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// Per-category CUDA-event accounting of kernel launches (rsv_profile_*).
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<int> cat;  // category of each recorded pair (events 2i, 2i+1)
  size_t used = 0;
  std::vector<int> nk;   // kernels launched inside each recorded pair
  int64_t launches[4] = {0, 0, 0, 0};
  int64_t kernels[4] = {0, 0, 0, 0};
  double ms[4] = {0, 0, 0, 0};
};

}  // namespace rsv

namespace rsv {
// Launch sequence of one time tile, relative to its first step (ops.cu, CUDA graphs).
struct TileGraphKey {
  size_t elem;
  int steps, forced, y_first, kg;
  bool adjoint;
  const void *state, *F, *Y, *norms;
  bool operator==(const TileGraphKey& o) const {
    return elem == o.elem && steps == o.steps && forced == o.forced && y_first == o.y_first && kg == o.kg &&
           adjoint == o.adjoint && state == o.state && F == o.F && Y == o.Y && norms == o.norms;
  }
};
struct TileGraph {
  TileGraphKey key;
  cudaGraphExec_t exec;
  int seen;
  bool failed;
};
}  // namespace rsv

struct rsv_operator_s {
  int kind = 0;
  int prec = 0;                          // RSV_PREC_FP64 or RSV_PREC_FP32 (also for BF16 state)
  bool bf16_state = false;               // RSV_PREC_BF16_STATE: march state stored in BF16
  bool real_state = false;
  double dt = 0.0;
  int64_t n = 0;                        // state length (all instances, all components)
  int n_inst = 1;
  std::vector<int64_t> inst_off, inst_len;
  cudaStream_t stream = nullptr;
  int sm_count = 0;

  // frequencies
  bool have_freq = false;
  int n_omega = 0;
  std::vector<double> omega;
  std::vector<int64_t> pj;              // 2 (m_j + phi)
  double dw = 0.0, phi = 0.0, period = 0.0, h = 0.0;
  int64_t n_t = 0;
  void* d_tw = nullptr;                 // twiddle table [4 N_T], cpx<double> or cpx<float>
  int64_t* d_pj = nullptr;              // [n_omega]
  float* d_cw = nullptr;                // real-state synthesis weights c_j (1 at w = 0, else 2)

  // device arrays of the operator (kind specific)
  std::vector<void*> dev;               // freed at destroy
  void* d_inst_off = nullptr;           // int64 [n_inst + 1]
  void* d_inst_of_point = nullptr;      // int32 [n]
  // GL1D: tridiagonal coefficients, direct then adjoint: lo, di, up
  void* tri[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int gl_max_n = 0;
  // packed launch of uneven GL1D batches (built per vector-group size): slot map, CTA count, threads
  // and slots per thread of a CTA, CTAs per wave (SMs x CTAs resident per SM)
  void* pack_map = nullptr;
  int pack_kg = 0, pack_count = 0, pack_threads = 0, pack_ppt = 0, pack_wave = 0;
  // FP64 RK4 GL1D marches: CTAs per (instance, vector) cluster of the last tile (0: one CTA)
  int gl_cluster = 0;
  // Crank-Nicolson (scheme = RSV_SCHEME_CN): host copies of the tridiagonal coefficients (FP64,
  // direct then adjoint: lo, di, up) and, per step h, the cyclic-reduction factors of
  // I - h/2 A on the device: [dir][level][n] for both neighbours, then [dir][n] inverse pivots
  int scheme = RSV_SCHEME_RK4;
  std::vector<double> tri_host;           // [6][n] complex (re, im)
  void* pcr = nullptr;
  int pcr_levels = 0;
  // DENSE: A (FP64), A and A^H in the element type, and the RK4 propagator
  // blocks D, P1, P2, D^H, P1^H, P2^H (element type) for the step dense_h
  void* dense64[1] = {nullptr};
  void* dense[2] = {nullptr, nullptr};
  void* prop[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double dense_h = 0.0;
  // tensor-core operand tiles of D and D^H (FP32 mode), and the switch that turns them off
  void* tc_tiles[2] = {nullptr, nullptr};
  bool tc_disabled = false;
  bool tc_persistent = false;   // all clusters of the tile kernel fit on the GPU at once
  uint64_t wait_limit_ns = 2000000000ull;  // limit of each cross-CTA wait (RSV_WAIT_LIMIT_NS)
  bool test_stall_wait = false;  // test hook (RSV_TEST_STALL_WAIT=1): a wait on a count nobody reaches
  int tc_max_clusters = 0;      // resident CTAs of the persistent tile kernel on this GPU
  void* d_ready = nullptr;      // per-block step counters and arrival counters of the persistent tile kernel
  void* tc_acc = nullptr;       // its FP32 partial-sum accumulators
  // stencil kinds: base-flow fields
  void* fld[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double c_dx = 0, c_dy = 0, c_dz = 0;
  int nx = 0, ny = 0, nz = 0;
  double visc = 0;
  int sponge_cells = 0;
  double sponge_amp = 0;

  // march workspace (grown on demand)
  rsv::Workspace ws_state, ws_ftile, ws_ysnap, ws_acc, ws_norm, ws_glue_a, ws_glue_b, ws_gram, ws_small;
  rsv::Workspace ws_coef, ws_coef2, ws_tcb;
  // time-series runs (series.cu): Fourier table, filter taps, the TRM power iteration's records
  // (direct output, adjoint output, next forcing), its FP64 Fourier block and norms
  rsv::Workspace ws_ser_e, ws_ser_t, ws_ser_y, ws_ser_z, ws_ser_g, ws_ser_f, ws_ser_n;
  bool tc_contract_disabled = false;   // keep the synthesis / analysis on the CUDA cores
  int* d_flag = nullptr;
  rsv::Profiler prof;
  // diagonal forcing / observation matrices and metrics (rsv_set_weights): per-point FP64 factors
  // [b, c, c w_y, b / w_f, b / sqrt(w_f), c sqrt(w_y), 1 / sqrt(w_f), 1 / sqrt(w_y), sqrt(w_f)]
  bool have_weights = false;
  double* d_wt = nullptr;               // [9][n]
  rsv::Workspace ws_scaled;             // scaled input coefficients of one vector group
  // decay-probe results (n_transient_windows = -1), valid for the current frequency grid
  struct ProbeMemo {
    int adjoint;
    double tol;
    int64_t max_steps;
    uint64_t seed;
    int every;
    int64_t steps;
  };
  std::vector<ProbeMemo> probe_memo;
  int last_tile = 0, last_group = 0;   // tile length and vector-group size of the latest march
  // CUDA graphs of tile launch sequences (ops.cu), the private capture stream, replays so far
  std::vector<rsv::TileGraph> tile_graphs;
  cudaStream_t cap_stream = nullptr;
  int64_t graph_replays = 0;
  // host-input marches: two device staging buffers of one vector group's coefficients, the copy
  // stream, and events (copy done / buffer free) per staging buffer
  rsv::Workspace ws_stage[2];
  rsv::Workspace ws_omega;               // the seeded randomized SVD's test block
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
  // autotuned tile length and vector group (rsv_autotune) for marches of tuned_k vectors
  int tuned_k = 0, tuned_tile = 0, tuned_group = 0;
  int64_t last_steps = 0;              // steps marched by the latest march's last vector group

  ~rsv_operator_s();
};

namespace rsv {

// Thread-local error message; returns the status for convenience.
rsv_status fail(rsv_status s, const std::string& msg);
rsv_status cuda_fail(cudaError_t e, const char* where);
rsv_status ensure(Workspace& w, size_t bytes);

// Brackets one kernel launch with profiling events when profiling is on.
struct ProfScope {
  rsv_operator op;
  int cat;
  ProfScope(rsv_operator o, int c, int nkernels = 1);
  ~ProfScope();
};
enum { PROF_SYNTH = 0, PROF_MARCH = 1, PROF_ANALYSIS = 2, PROF_GLUE = 3 };
// scalings of a march by the weights of rsv_set_weights: none, the plain runs of R_y and R_y^dag,
// or the runs of W_y^{1/2} C R B W_f^{-1/2} and its conjugate transpose
enum { SCALE_NONE = 0, SCALE_PLAIN = 1, SCALE_TILDE = 2 };
rsv_status march_any(rsv_operator op, const void* in, int k, const rsv_march_opts* opts, void* out, bool adjoint,
                     int scaling, bool host_in = false);

// ----- launchers (contract_kernels.cu) -------------------------------------
struct TileGeom {
  int64_t rows;        // rows in this vector group = kg * n
  int64_t coef_stride; // stride between frequencies in the coefficient block
  int n_omega;
  int64_t n0;          // first step of the tile
  int steps;           // steps in the tile
  int sgn;             // +1 direct, -1 adjoint (frequencies negated)
  int64_t m4;          // 4 N_T
  int n_tau = 0;       // synthesis points (0: 2 * steps + 1, the RK4 stage times)
  int tau_stride = 1;  // half steps between synthesis points
};

// F[tau][r] = sum_j c_j x(table[q_j(2 n0 + tau * tau_stride)] * fhat[j][r]), tau < n_tau
template <typename R>
cudaError_t launch_synth(const TileGeom& g, const void* fhat, const void* tw, const int64_t* pj,
                         const float* cw, bool real_state, void* F, cudaStream_t st);
// acc[j][r] += sum_{s in [s0, s1)} conj(table[q_j(2 (n0 + s))]) Y[s][r]
template <typename R>
cudaError_t launch_analysis(const TileGeom& g, const void* Y, int s0, int s1, const void* tw,
                            const int64_t* pj, bool real_state, cpx<double>* acc, int64_t acc_stride,
                            cudaStream_t st);
// out[j][r] = acc[j][r] * scale (* pscale[r mod n] when given), converted to the element type R
template <typename R>
cudaError_t launch_finish(const cpx<double>* acc, int64_t acc_stride, int n_omega, int64_t rows,
                          double scale, void* out, int64_t out_stride, cudaStream_t st,
                          const double* pscale = nullptr, int64_t n = 0);
// out[j][r] = in[j][r] * s[r mod n] for j < n_omega, r < rows (in and out may alias)
template <typename R>
cudaError_t launch_scale_block(const void* in, int64_t in_stride, void* out, int64_t out_stride, int n_omega,
                               int64_t rows, int64_t n, const double* s, cudaStream_t st);
cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st);

// ----- tensor-core contractions (tc_contract.cu), FP32 mode -----------------
bool tc_contract_supported(rsv_operator op, bool synth);
cudaError_t tc_synth(rsv_operator op, const TileGeom& g, const void* fhat, void* F);
cudaError_t tc_analysis(rsv_operator op, const TileGeom& g, const void* Y, int s0, int s1, cpx<double>* acc,
                        int64_t acc_stride);

// ----- GL1D (gl1d_kernels.cu) ---------------------------------------------
struct Gl1dTile {
  const void* lo;
  const void* di;
  const void* up;
  // Crank-Nicolson: cyclic-reduction factors of I - h/2 A ([levels][n] each) and inverse pivots [n]
  const void* cr_lo;
  const void* cr_up;
  const void* cr_inv;
  int cr_levels;
  const int64_t* inst_off;  // [n_inst + 1]
  int n_inst, max_n;
  int64_t n;                // points per vector
  int kg;                   // vectors in the group
  double h;
  int64_t n0;
  int steps;
  int64_t n_forced;         // forcing active for steps < n_forced
  int y_first;              // store the state of tile steps s >= y_first into Y
  bool real_state;
};
template <typename R>
cudaError_t launch_gl1d_tile(const Gl1dTile& t, void* u, const void* F, void* Y, double* norms,
                             int* flag, cudaStream_t st);
// Cluster size the FP64 RK4 tile launch takes for this tile (0: one CTA per (instance, vector)).
int gl1d_cluster_size(const Gl1dTile& t);
template <typename R>
cudaError_t launch_gl1d_apply(const Gl1dTile& t, const int32_t* inst_of_point, const void* x, void* y,
                              cudaStream_t st);
// Batches of uneven instances: CTAs of gl1d_pack_threads<R>() threads x ppt slots (ppt 1 to 4) holding
// several (instance, vector) segments each (map [n_packs][threads * ppt] of rows, -1 for separators and
// unused slots).  FP32 takes 1024 threads, FP64 512 (twice the registers per slot).
template <typename R>
constexpr int gl1d_pack_threads() { return sizeof(R) == 4 ? 1024 : 512; }
// CTAs of the packed kernel with ppt slots per thread that one SM holds at once.
template <typename R>
cudaError_t gl1d_pack_occupancy(int ppt, int* ctas_per_sm);
template <typename R>
cudaError_t launch_gl1d_pack(const Gl1dTile& t, const int32_t* map, int n_packs, int ppt, void* u, const void* F,
                             void* Y, int* flag, cudaStream_t st);

// ----- glue (glue_kernels.cu) ----------------------------------------------
// G[j][i][a][b] = sum_{p in instance i} conj(X[j][a][p]) X[j][b][p]
template <typename R>
cudaError_t launch_gram(const void* X, int n_omega, int k, int64_t n, const int64_t* inst_off, int n_inst,
                        int64_t max_len, cpx<double>* G, cudaStream_t st);
// Out[j][b][p] = sum_a In[j][a][p] * M[j][inst(p)][a][b] * colscale[j][inst][b]
template <typename R>
cudaError_t launch_combine(const void* In, int n_omega, int ka, int kb, int64_t n, const int32_t* inst_of_point,
                           int n_inst, const void* M, void* Out, int64_t out_k, cudaStream_t st);   // M: cpx<R>

}  // namespace rsv
