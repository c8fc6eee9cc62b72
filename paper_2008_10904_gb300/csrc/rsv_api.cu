// C ABI of librsv: operator objects, the frequency grid and twiddle table,
// and the tile-by-tile driver of the direct and adjoint marches.
//
// Method (Sec. 2 of the paper): the action of the resolvent on Fourier
// coefficients for all frequencies at once, by marching the linear system
// with a forcing synthesised from the coefficients and Fourier-analysing the
// response.  The march is cut into time tiles of S steps; per tile the
// driver launches
//   synthesis  F[0..2S] = forcing at the tile's step starts and midpoints
//              (only while the forcing is on),
//   march      S RK4 steps of the operator's fused stage kernel, storing the
//              state of analysed steps in Y,
//   analysis   acc[j] += sum_s Y[s] exp(-i w_j t_s) (only in the analysis window).
// Schedules: SSRM (Sec. 2.3) forces n_trans + 1 windows of N_T steps and
// analyses the last; TRM (Sec. 2.2) forces one window, then marches an
// unforced tail, and analyses the whole record.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "rsv_internal.h"
#include "rsv_ops.h"

namespace rsv {

static thread_local std::string g_err;

rsv_status fail(rsv_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

rsv_status cuda_fail(cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(e == cudaErrorMemoryAllocation ? RSV_ERR_OOM : RSV_ERR_CUDA, m);
}

rsv_status ensure(Workspace& w, size_t bytes) {
  if (w.bytes >= bytes && w.ptr != nullptr) return RSV_OK;
  if (w.ptr) cudaFree(w.ptr);
  w.ptr = nullptr;
  w.bytes = 0;
  cudaError_t e = cudaMalloc(&w.ptr, bytes < 256 ? 256 : bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    w.ptr = nullptr;
    return cuda_fail(e, "workspace allocation");
  }
  w.bytes = bytes;
  return RSV_OK;
}

rsv_status upload(rsv_operator op, const void* host, size_t bytes, void** dst) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes < 16 ? 16 : bytes);
  if (e != cudaSuccess) return cuda_fail(e, "operator allocation");
  op->dev.push_back(p);
  e = cudaMemcpy(p, host, bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "operator upload");
  *dst = p;
  return RSV_OK;
}

static void prof_flush(rsv_operator op) {
  Profiler& p = op->prof;
  if (p.used == 0) return;
  cudaStreamSynchronize(op->stream);
  for (size_t i = 0; i < p.used; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p.pool[2 * i], p.pool[2 * i + 1]) == cudaSuccess) {
      p.ms[p.cat[i]] += t;
      p.launches[p.cat[i]] += 1;
      p.kernels[p.cat[i]] += p.nk[i];
    }
  }
  p.used = 0;
}

ProfScope::ProfScope(rsv_operator o, int c, int nkernels) : op(o), cat(c) {
  Profiler& p = op->prof;
  if (!p.on) return;
  if (p.used >= 4096) prof_flush(op);
  if (2 * p.used + 2 > p.pool.size()) {
    for (int i = 0; i < 2; ++i) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      p.pool.push_back(e);
    }
    p.cat.push_back(0);
    p.nk.push_back(0);
  }
  p.cat[p.used] = c;
  p.nk[p.used] = nkernels;
  cudaEventRecord(p.pool[2 * p.used], op->stream);
}

ProfScope::~ProfScope() {
  Profiler& p = op->prof;
  if (!p.on) return;
  cudaEventRecord(p.pool[2 * p.used + 1], op->stream);
  p.used += 1;
}

size_t elem_bytes(rsv_operator op) { return op->prec == RSV_PREC_FP64 ? 8 : 4; }
size_t coef_bytes(rsv_operator op) { return 2 * elem_bytes(op); }
size_t state_elem_bytes(rsv_operator op) { return op->real_state ? elem_bytes(op) : coef_bytes(op); }

}  // namespace rsv

using namespace rsv;

rsv_operator_s::~rsv_operator_s() {
  for (void* p : dev) cudaFree(p);
  Workspace* ws[] = {&ws_state, &ws_ftile, &ws_ysnap, &ws_acc,   &ws_norm,  &ws_glue_a, &ws_glue_b,
                     &ws_gram,  &ws_small, &ws_coef,  &ws_coef2, &ws_tcb,   &ws_ser_e, &ws_ser_t,
                     &ws_ser_y, &ws_ser_z, &ws_ser_g, &ws_ser_f, &ws_ser_n};
  for (Workspace* w : ws)
    if (w->ptr) cudaFree(w->ptr);
  if (d_tw) cudaFree(d_tw);
  if (d_pj) cudaFree(d_pj);
  if (d_cw) cudaFree(d_cw);
  if (d_flag) cudaFree(d_flag);
  if (d_wt) cudaFree(d_wt);
  if (pcr) cudaFree(pcr);
  if (pack_map) cudaFree(pack_map);
  for (rsv::TileGraph& g : tile_graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (cap_stream) cudaStreamDestroy(cap_stream);
  if (ws_omega.ptr) cudaFree(ws_omega.ptr);
  for (int i = 0; i < 2; ++i) {
    if (ws_stage[i].ptr) cudaFree(ws_stage[i].ptr);
    if (ev_copied[i]) cudaEventDestroy(ev_copied[i]);
    if (ev_free[i]) cudaEventDestroy(ev_free[i]);
  }
  if (copy_stream) cudaStreamDestroy(copy_stream);
  if (ws_scaled.ptr) cudaFree(ws_scaled.ptr);
  for (cudaEvent_t e : prof.pool) cudaEventDestroy(e);
}

extern "C" rsv_status rsv_profile_enable(rsv_operator op, int32_t enable) {
  if (!op) return fail(RSV_ERR_INVALID_ARG, "null operator");
  if (!enable) prof_flush(op);
  op->prof.on = enable != 0;
  return RSV_OK;
}

extern "C" rsv_status rsv_profile_reset(rsv_operator op) {
  if (!op) return fail(RSV_ERR_INVALID_ARG, "null operator");
  prof_flush(op);
  for (int c = 0; c < 4; ++c) {
    op->prof.launches[c] = 0;
    op->prof.kernels[c] = 0;
    op->prof.ms[c] = 0.0;
  }
  return RSV_OK;
}

extern "C" rsv_status rsv_profile_read(rsv_operator op, int32_t category, int64_t* groups, int64_t* kernels,
                                       double* ms) {
  if (!op || category < 0 || category > 3) return fail(RSV_ERR_INVALID_ARG, "bad profile query");
  prof_flush(op);
  if (groups) *groups = op->prof.launches[category];
  if (kernels) *kernels = op->prof.kernels[category];
  if (ms) *ms = op->prof.ms[category];
  return RSV_OK;
}

extern "C" const char* rsv_last_error(void) { return g_err.c_str(); }
extern "C" const char* rsv_version(void) { return "rsv 0.2 (sm_103a)"; }

extern "C" rsv_status rsv_create_operator(const rsv_operator_desc* d, void* stream, rsv_operator* out) {
  if (!d || !out) return fail(RSV_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (d->precision != RSV_PREC_FP64 && d->precision != RSV_PREC_FP32 && d->precision != RSV_PREC_BF16_STATE)
    return fail(RSV_ERR_INVALID_ARG, "unknown precision");
  if (d->precision == RSV_PREC_BF16_STATE && !(d->kind == RSV_OP_ADV3D && d->nx % 4 == 0))
    return fail(RSV_ERR_INVALID_ARG, "BF16 state is built for the ADV3D kind with nx a multiple of 4");
  if (!(d->dt > 0.0)) return fail(RSV_ERR_INVALID_ARG, "dt must be positive");
  if (d->scheme != RSV_SCHEME_RK4 && d->scheme != RSV_SCHEME_CN) return fail(RSV_ERR_INVALID_ARG, "unknown scheme");
  if (d->scheme == RSV_SCHEME_CN && d->kind != RSV_OP_GL1D)
    return fail(RSV_ERR_INVALID_ARG, "the Crank-Nicolson scheme is built for the GL1D kind only");
  rsv_operator op = new rsv_operator_s();
  op->kind = d->kind;
  op->scheme = d->scheme;
  op->prec = d->precision == RSV_PREC_FP64 ? RSV_PREC_FP64 : RSV_PREC_FP32;
  op->bf16_state = d->precision == RSV_PREC_BF16_STATE;
  op->dt = d->dt;
  op->stream = (cudaStream_t)stream;
  {
    // RSV_DENSE_TENSOR=0 keeps dense FP32 operators on the CUDA-core step (for comparisons)
    const char* env = getenv("RSV_DENSE_TENSOR");
    op->tc_disabled = env != nullptr && env[0] == '0';
    // RSV_CONTRACT_TENSOR=0 keeps FP32 synthesis / analysis on the CUDA cores (for comparisons)
    const char* env2 = getenv("RSV_CONTRACT_TENSOR");
    op->tc_contract_disabled = env2 != nullptr && env2[0] == '0';
    // RSV_WAIT_LIMIT_NS shortens the limit of the persistent kernels' waits on other CTAs; with
    // RSV_TEST_STALL_WAIT=1 the dense persistent kernel's first wait targets a count nobody
    // reaches, so a test can make a bounded wait run out and check RSV_ERR_TIMEOUT
    const char* env3 = getenv("RSV_WAIT_LIMIT_NS");
    if (env3 != nullptr) {
      const long long v = atoll(env3);
      if (v > 0) op->wait_limit_ns = (uint64_t)v;
    }
    const char* env4 = getenv("RSV_TEST_STALL_WAIT");
    op->test_stall_wait = env4 != nullptr && env4[0] == '1';
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&op->sm_count, cudaDevAttrMultiProcessorCount, dev);
  rsv_status s;
  switch (d->kind) {
    case RSV_OP_GL1D: s = build_gl1d(op, d); break;
    case RSV_OP_DENSE: s = build_dense(op, d); break;
    case RSV_OP_ADR2D: s = build_adr2d(op, d); break;
    case RSV_OP_ADV3D: s = build_adv3d(op, d); break;
    default: s = fail(RSV_ERR_INVALID_ARG, "unknown operator kind");
  }
  if (s == RSV_OK) {
    // instance tables shared by every kind
    std::vector<int64_t> off(op->n_inst + 1);
    std::vector<int32_t> iop(op->n);
    for (int i = 0; i < op->n_inst; ++i) {
      off[i] = op->inst_off[i];
      for (int64_t p = op->inst_off[i]; p < op->inst_off[i] + op->inst_len[i]; ++p) iop[p] = i;
    }
    off[op->n_inst] = op->n;
    s = upload(op, off.data(), off.size() * sizeof(int64_t), &op->d_inst_off);
    if (s == RSV_OK) s = upload(op, iop.data(), iop.size() * sizeof(int32_t), &op->d_inst_of_point);
    if (s == RSV_OK) {
      cudaError_t e = cudaMalloc(&op->d_flag, sizeof(int));
      if (e != cudaSuccess) s = cuda_fail(e, "flag allocation");
    }
  }
  if (s != RSV_OK) {
    delete op;
    return s;
  }
  *out = op;
  return RSV_OK;
}

extern "C" void rsv_destroy_operator(rsv_operator op) {
  if (!op) return;
  cudaStreamSynchronize(op->stream);
  delete op;
}

extern "C" rsv_status rsv_describe(rsv_operator op, char* buf, int32_t buflen) {
  if (!op || !buf || buflen < 1) return fail(RSV_ERR_INVALID_ARG, "bad describe arguments");
  static const char* kinds[] = {"gl1d", "dense", "adr2d", "adv3d"};
  const char* path = "cuda-core stages";
  if (op->kind == RSV_OP_GL1D)
    path = op->scheme == RSV_SCHEME_CN ? "cuda-core crank-nicolson tile kernel" : "cuda-core tile kernel";
  if (op->kind == RSV_OP_ADV3D && op->prec == RSV_PREC_FP32) {
    const char* e = getenv("RSV_STENCIL3D_STAGED");
    const bool pairs = !(e != nullptr && e[0] == '1') && !op->bf16_state && op->nx % 4 == 0 &&
                       op->n < ((int64_t)1 << 31);
    path = pairs ? "cuda-core 3-D stage-pair kernels" : (op->bf16_state ? "cuda-core stages, bf16 state" : "cuda-core stages");
  }
  if (op->kind == RSV_OP_ADR2D) {
    const char* e = getenv("RSV_STENCIL_FUSED");
    if (e != nullptr && e[0] == '1')
      path = "cuda-core whole-step kernel";
    else if (op->prec == RSV_PREC_FP32 && adr2d_pairs_enabled() && op->nx % 4 == 0 && op->n < ((int64_t)1 << 31))
      path = "cuda-core 2-D stage-pair kernels";
  }
  if (op->kind == RSV_OP_DENSE) {
    if (op->prec == RSV_PREC_FP32 && op->tc_tiles[0] && !op->tc_disabled)
      path = op->tc_persistent ? "tcgen05 3xTF32 persistent tile kernel" : "tcgen05 3xTF32 one launch per step";
    else
      path = "cuda-core propagator step";
  }
  const char* contract = (op->prec == RSV_PREC_FP32 && !op->tc_contract_disabled) ? "tcgen05" : "cuda-core";
  char packs[96] = "";
  if (op->kind == RSV_OP_GL1D && op->pack_kg > 0)
    snprintf(packs, sizeof(packs), " packed=%d ctas of %d slots (%dx%d, %d per wave)", op->pack_count,
             op->pack_threads * op->pack_ppt, op->pack_threads, op->pack_ppt, op->pack_wave);
  else if (op->kind == RSV_OP_GL1D && op->gl_cluster > 0)
    snprintf(packs, sizeof(packs), " cluster=%d ctas per march", op->gl_cluster);
  char tuned[64] = "";
  if (op->tuned_k > 0) snprintf(tuned, sizeof(tuned), " tuned=%d/%d for k=%d", op->tuned_tile, op->tuned_group, op->tuned_k);
  snprintf(buf, (size_t)buflen,
           "kind=%s precision=%s n=%lld instances=%d path=%s%s contractions=%s resident_ctas=%d sms=%d tile=%d "
           "group=%d steps=%lld graphs=%d%s",
           (op->kind >= 0 && op->kind < 4) ? kinds[op->kind] : "?",
           op->prec == RSV_PREC_FP64 ? "fp64" : (op->bf16_state ? "bf16-state" : "fp32"),
           (long long)op->n, op->n_inst, path, packs, contract, op->tc_max_clusters, op->sm_count, op->last_tile,
           op->last_group, (long long)op->last_steps, (int)op->graph_replays, tuned);
  return RSV_OK;
}

extern "C" rsv_status rsv_operator_info(rsv_operator op, int64_t* n, int32_t* n_instances, int32_t* real_state) {
  if (!op) return fail(RSV_ERR_INVALID_ARG, "null operator");
  if (n) *n = op->n;
  if (n_instances) *n_instances = op->n_inst;
  if (real_state) *real_state = op->real_state ? 1 : 0;
  return RSV_OK;
}

extern "C" rsv_status rsv_instance_range(rsv_operator op, int32_t i, int64_t* offset, int64_t* length) {
  if (!op || i < 0 || i >= op->n_inst) return fail(RSV_ERR_INVALID_ARG, "bad instance index");
  if (offset) *offset = op->inst_off[i];
  if (length) *length = op->inst_len[i];
  return RSV_OK;
}

// Frequencies: w_j = (m_j + phi) dw with integer m_j and common phi in {0, 1/2}
// (Sec. 2.3, Delta omega = 2 pi / T).  The twiddle table holds exp(i pi q / (2 N_T))
// for q < 4 N_T, so exp(i w_j (2n + sigma) h / 2) = table[p_j (2n + sigma) mod 4 N_T]
// with p_j = 2 (m_j + phi), exact in the integer index for any t.
extern "C" rsv_status rsv_set_frequencies(rsv_operator op, const double* omega, int32_t n_omega, double dw,
                                          int64_t* n_steps_per_window, double* h_out) {
  if (!op || !omega || n_omega < 1) return fail(RSV_ERR_INVALID_ARG, "bad frequency arguments");
  if (dw <= 0.0) {
    if (n_omega < 2) return fail(RSV_ERR_INVALID_ARG, "a single frequency needs an explicit dw");
    std::vector<double> srt(omega, omega + n_omega);
    std::sort(srt.begin(), srt.end());
    dw = 0.0;
    for (int i = 1; i < n_omega; ++i) {
      const double g = srt[i] - srt[i - 1];
      if (g <= 0.0) return fail(RSV_ERR_INVALID_ARG, "repeated frequency");
      if (dw == 0.0 || g < dw) dw = g;
    }
  }
  const double r0 = omega[0] / dw;
  const double frac = r0 - std::floor(r0);
  const double phi = std::fabs(frac - 0.5) < 1e-6 ? 0.5 : 0.0;
  std::vector<int64_t> pj(n_omega);
  for (int j = 0; j < n_omega; ++j) {
    const double r = omega[j] / dw - phi;
    const double m = std::nearbyint(r);
    if (std::fabs(r - m) > 1e-6)
      return fail(RSV_ERR_NOT_COMMENSURATE, "frequency " + std::to_string(j) + " is not on the grid (m + phi) dw");
    pj[j] = (int64_t)(2.0 * m + 2.0 * phi);
  }
  const double period = 2.0 * M_PI / dw;
  const int64_t n_t = (int64_t)std::ceil(period / op->dt - 1e-9);
  if (n_t < 1 || n_t > (int64_t)1 << 40) return fail(RSV_ERR_INVALID_ARG, "window length out of range");
  for (int j = 0; j < n_omega; ++j) {
    for (int l = 0; l < j; ++l) {
      const int64_t dm = (pj[j] - pj[l]) / 2;
      if (dm % n_t == 0) return fail(RSV_ERR_NOT_COMMENSURATE, "two frequencies alias on the window");
    }
  }
  const int64_t m4 = 4 * n_t;
  std::vector<cpx<double>> tab(m4);
  for (int64_t q = 0; q < m4; ++q) {
    // reduce to the first octant by symmetry so that every entry is correctly rounded
    const int64_t quad = q / n_t, rr = q % n_t;  // angle = (quad + rr / n_t) * pi/2
    double c, s;
    if (2 * rr <= n_t) {
      const double a = M_PI_2 * (double)rr / (double)n_t;
      c = std::cos(a);
      s = std::sin(a);
    } else {
      const double a = M_PI_2 * (double)(n_t - rr) / (double)n_t;
      c = std::sin(a);
      s = std::cos(a);
    }
    double re, im;
    switch (quad) {
      case 0: re = c; im = s; break;
      case 1: re = -s; im = c; break;
      case 2: re = -c; im = -s; break;
      default: re = s; im = -c; break;
    }
    tab[q] = mk<double>(re, im);
  }
  if (op->d_tw) cudaFree(op->d_tw);
  if (op->d_pj) cudaFree(op->d_pj);
  if (op->d_cw) cudaFree(op->d_cw);
  op->d_tw = nullptr;
  op->d_pj = nullptr;
  op->d_cw = nullptr;
  cudaError_t e;
  if (op->prec == RSV_PREC_FP64) {
    e = cudaMalloc(&op->d_tw, m4 * sizeof(cpx<double>));
    if (e == cudaSuccess) e = cudaMemcpy(op->d_tw, tab.data(), m4 * sizeof(cpx<double>), cudaMemcpyHostToDevice);
  } else {
    std::vector<cpx<float>> t32(m4);
    for (int64_t q = 0; q < m4; ++q) t32[q] = mk<float>((float)tab[q].re, (float)tab[q].im);
    e = cudaMalloc(&op->d_tw, m4 * sizeof(cpx<float>));
    if (e == cudaSuccess) e = cudaMemcpy(op->d_tw, t32.data(), m4 * sizeof(cpx<float>), cudaMemcpyHostToDevice);
  }
  std::vector<float> cw(n_omega);
  for (int j = 0; j < n_omega; ++j) cw[j] = (pj[j] == 0) ? 1.0f : 2.0f;
  if (e == cudaSuccess) e = cudaMalloc(&op->d_pj, n_omega * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMemcpy(op->d_pj, pj.data(), n_omega * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&op->d_cw, n_omega * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(op->d_cw, cw.data(), n_omega * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "twiddle table");
  op->omega.assign(omega, omega + n_omega);
  op->pj = pj;
  op->n_omega = n_omega;
  op->dw = dw;
  op->phi = phi;
  op->period = period;
  op->n_t = n_t;
  op->h = period / (double)n_t;
  op->have_freq = true;
  op->probe_memo.clear();
  rsv_status ks = on_frequencies(op);
  if (ks != RSV_OK) {
    op->have_freq = false;
    return ks;
  }
  if (n_steps_per_window) *n_steps_per_window = n_t;
  if (h_out) *h_out = op->h;
  return RSV_OK;
}

namespace rsv {

// Decay run (Sec. 2.3): unforced march of one random state in tiles of `every` steps; per-instance
// norm ratios at the tile ends.  Returns OK with the steps at the first check point where every
// ratio is <= tol, UNSTABLE when a ratio passes 1e6 / turns non-finite or max_steps pass first.
template <typename R>
static rsv_status probe_impl(rsv_operator op, bool adjoint, double tol, int64_t max_steps, uint64_t seed, int every,
                             int64_t* steps_out, double* ratio_out) {
  const size_t se = state_elem_bytes(op);
  const int ni = op->n_inst;
  rsv_status st;
  if ((st = ensure(op->ws_state, (size_t)op->n * se + stage_scratch_bytes(op, 1))) != RSV_OK) return st;
  if ((st = ensure(op->ws_norm, (size_t)2 * ni * sizeof(double))) != RSV_OK) return st;
  double* d_tile_norms = (double*)op->ws_norm.ptr;   // written by the 1-D tile kernel
  double* d_inst = d_tile_norms + ni;
  const cudaStream_t stream = op->stream;
  cudaError_t e = cudaMemsetAsync(op->ws_state.ptr, 0, (size_t)op->n * se + stage_scratch_bytes(op, 1), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(op->d_flag, 0, sizeof(int), stream);
  if (e == cudaSuccess) e = probe_initial_state(op, seed);
  std::vector<double> n0(ni), nn(ni);
  if (e == cudaSuccess) e = instance_sq_norms(op, 0, d_inst);
  if (e == cudaSuccess) e = cudaMemcpyAsync(n0.data(), d_inst, sizeof(double) * ni, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "decay probe set-up");
  int64_t done = 0;
  double ratio = 1.0;
  while (done < max_steps) {
    MarchTile mt;
    mt.n0 = done;
    mt.steps = (int)std::min<int64_t>(every, max_steps - done);
    mt.n_forced = 0;
    mt.y_first = mt.steps;
    mt.kg = 1;
    mt.adjoint = adjoint;
    {
      ProfScope ps(op, PROF_MARCH, march_tile_kernels(op, mt.steps, 1));
      e = march_tile<R>(op, mt, op->ws_state.ptr, nullptr, nullptr, d_tile_norms);
    }
    done += mt.steps;
    int flag = 0;
    if (e == cudaSuccess) e = instance_sq_norms(op, done, d_inst);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nn.data(), d_inst, sizeof(double) * ni, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, op->d_flag, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "decay probe");
    ratio = 0.0;
    bool finite = flag == 0;
    for (int i = 0; i < ni; ++i) {
      const double r = std::sqrt(nn[i] / n0[i]);
      if (!std::isfinite(r)) finite = false;
      ratio = std::max(ratio, r);
    }
    if (steps_out) *steps_out = done;
    if (ratio_out) *ratio_out = finite ? ratio : INFINITY;
    if (!finite || ratio > 1e6)
      return fail(RSV_ERR_UNSTABLE, "decay probe: the state norm grew (ratio " + std::to_string(ratio) + " after " +
                                        std::to_string(done) + " steps): the system is not stable");
    if (ratio <= tol) return RSV_OK;
  }
  return fail(RSV_ERR_UNSTABLE, "decay probe: the state norm did not fall to tol within " +
                                    std::to_string(max_steps) + " steps (ratio " + std::to_string(ratio) + ")");
}

static rsv_status probe_any(rsv_operator op, bool adjoint, double tol, int64_t max_steps, uint64_t seed, int every,
                            int64_t* steps, double* ratio) {
  if (!(tol > 0.0 && tol < 1.0)) return fail(RSV_ERR_INVALID_ARG, "decay tol must be in (0, 1)");
  if (max_steps < 1) return fail(RSV_ERR_INVALID_ARG, "decay max_steps must be >= 1");
  if (every <= 0) every = default_tile_steps(op);
  return op->prec == RSV_PREC_FP64 ? probe_impl<double>(op, adjoint, tol, max_steps, seed, every, steps, ratio)
                                   : probe_impl<float>(op, adjoint, tol, max_steps, seed, every, steps, ratio);
}

struct Schedule {
  int64_t total, first, forced;
};

// Transient windows for n_transient_windows = -1: the decay run's length in windows, remembered per
// direction and setting until the frequencies change.
static rsv_status auto_windows(rsv_operator op, const rsv_march_opts* o, bool adjoint, int64_t* windows) {
  const double tol = o->decay_tol > 0.0 ? o->decay_tol : 1e-8;
  const int64_t cap = o->decay_max_steps > 0 ? o->decay_max_steps : 1000 * op->n_t;
  const int every = o->tile_steps > 0 ? o->tile_steps : default_tile_steps(op);
  for (const auto& m : op->probe_memo) {
    if (m.adjoint == (int)adjoint && m.tol == tol && m.max_steps == cap && m.seed == o->decay_seed && m.every == every) {
      *windows = (m.steps + op->n_t - 1) / op->n_t;
      return RSV_OK;
    }
  }
  int64_t steps = 0;
  rsv_status st = probe_any(op, adjoint, tol, cap, o->decay_seed, every, &steps, nullptr);
  if (st != RSV_OK) return st;
  op->probe_memo.push_back({(int)adjoint, tol, cap, o->decay_seed, every, steps});
  *windows = (steps + op->n_t - 1) / op->n_t;
  return RSV_OK;
}

static rsv_status make_schedule(rsv_operator op, const rsv_march_opts* o, bool adjoint, Schedule* s) {
  rsv_march_opts def{};
  if (!o) o = &def;
  if (o->variant == RSV_SSRM) {
    int64_t nw = o->n_transient_windows;
    if (nw == -1) {
      rsv_status st = auto_windows(op, o, adjoint, &nw);
      if (st != RSV_OK) return st;
    } else if (nw < 0) {
      return fail(RSV_ERR_INVALID_ARG, "n_transient_windows must be >= 0, or -1 for the decay probe");
    }
    s->total = (nw + 1) * op->n_t;
    s->first = nw * op->n_t;
    s->forced = s->total;
  } else if (o->variant == RSV_TRM) {
    if (o->tail_steps < 0) return fail(RSV_ERR_INVALID_ARG, "tail_steps < 0");
    if (!(o->tail_tol >= 0.0)) return fail(RSV_ERR_INVALID_ARG, "tail_tol must be >= 0");
    s->total = op->n_t + o->tail_steps;
    s->first = 0;
    s->forced = op->n_t;
  } else {
    return fail(RSV_ERR_INVALID_ARG, "unknown variant");
  }
  return RSV_OK;
}

// Per-point factors of the weighted runs (rsv_set_weights), rows of op->d_wt.
enum { WT_B = 0, WT_C, WT_CWY, WT_B_WF, WT_B_SWF, WT_C_SWY, WT_ISWF, WT_ISWY, WT_SWF };

// Input and output scalings of one march: SCALE_PLAIN gives yhat = C R B fhat (direct) and
// what = W_f^{-1} B^H R^H C^H W_y yhat (adjoint); SCALE_TILDE gives the runs of
// W_y^{1/2} C R B W_f^{-1/2} and its conjugate transpose (the randomized SVD's operator).
static void march_scalings(rsv_operator op, int scaling, bool adjoint, const double** sin, const double** sout) {
  *sin = *sout = nullptr;
  if (!op->have_weights || scaling == SCALE_NONE) return;
  const int64_t n = op->n;
  auto row = [&](int r) { return op->d_wt + (size_t)r * n; };
  if (scaling == SCALE_PLAIN) {
    *sin = adjoint ? row(WT_CWY) : row(WT_B);
    *sout = adjoint ? row(WT_B_WF) : row(WT_C);
  } else {
    *sin = adjoint ? row(WT_C_SWY) : row(WT_B_SWF);
    *sout = adjoint ? row(WT_B_SWF) : row(WT_C_SWY);
  }
}

// A timed trial of one tile configuration for rsv_autotune: the first vector group of kg vectors,
// one forced and analysed time tile of S steps, accumulators in the workspace, nothing written to
// the caller; *ms receives the device time of the tile's launches.
struct TileTrial {
  int S, kg;
  float* ms;
  int* steps;   // steps of the timed tile
};

template <typename R>
static rsv_status march_impl(rsv_operator op, const void* in, int k, const rsv_march_opts* opts, void* out,
                             bool adjoint, int scaling, const TileTrial* trial = nullptr, bool host_in = false) {
  const double *s_in = nullptr, *s_out = nullptr;
  march_scalings(op, scaling, adjoint, &s_in, &s_out);
  Schedule sc;
  rsv_status st = make_schedule(op, opts, adjoint, &sc);
  if (st != RSV_OK) return st;
  const int64_t n = op->n;
  const size_t se = state_elem_bytes(op);
  // Tile length S and vector-group size kg: the requested / default tile and all k vectors, shrunk
  // (kg halved, then S down to 16) until the march workspace fits in 90% of the device memory not
  // held by others.
  int S = (opts && opts->tile_steps > 0) ? opts->tile_steps
                                         : (op->tuned_k == k ? op->tuned_tile : default_tile_steps(op));
  int kg = (op->tuned_k == k && !(opts && opts->tile_steps > 0)) ? op->tuned_group : k;
  if (opts && opts->group_vectors > 0) kg = std::min(kg, (int)opts->group_vectors);
  if (trial) {
    S = trial->S;
    kg = trial->kg;
  }
  {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      free_b = (size_t)1 << 62;
    }
    const size_t held = op->ws_state.bytes + op->ws_ftile.bytes + op->ws_ysnap.bytes + op->ws_acc.bytes +
                        op->ws_coef.bytes + op->ws_coef2.bytes;
    const double budget = 0.9 * (double)(free_b + held);
    auto need = [&](int s_, int kg_) {
      const double rows_ = (double)kg_ * n;
      double b = rows_ * se + (double)stage_scratch_bytes(op, kg_) + (2.0 * s_ + 1) * rows_ * se + s_ * rows_ * se;
      if (op->prec != RSV_PREC_FP64) b += (double)op->n_omega * rows_ * sizeof(cpx<double>);
      if (s_in) b += (double)op->n_omega * rows_ * coef_bytes(op);
      if (op->kind == RSV_OP_DENSE) b += 2.0 * op->n_omega * rows_ * 2 * sizeof(R);
      if (host_in) b += 2.0 * op->n_omega * rows_ * coef_bytes(op);   // staging buffers
      return b;
    };
    // per-tile traffic (coefficients, FP64 accumulators) is amortised over S, while the vector
    // group only sets how much is resident: shrink the group first, then the tile
    if (trial && need(S, kg) > budget) return fail(RSV_ERR_OOM, "trial configuration does not fit");
    while (need(S, kg) > budget && (S > 16 || kg > 1)) {
      if (kg > 1)
        kg = (kg + 1) / 2;
      else
        S = std::max(16, S / 2);
    }
  }
  const cudaStream_t stream = op->stream;
  cudaError_t e;
  op->last_tile = S;
  op->last_group = kg;
  const int64_t rows_max = (int64_t)kg * n;
  if ((st = ensure(op->ws_state, rows_max * se + stage_scratch_bytes(op, kg))) != RSV_OK) return st;
  if ((st = ensure(op->ws_ftile, (size_t)(2 * S + 1) * rows_max * se)) != RSV_OK) return st;
  if ((st = ensure(op->ws_ysnap, (size_t)S * rows_max * se)) != RSV_OK) return st;
  if ((st = ensure(op->ws_norm, (size_t)kg * op->n_inst * sizeof(double))) != RSV_OK) return st;
  const bool acc_in_out = (op->prec == RSV_PREC_FP64) && trial == nullptr;
  if (!acc_in_out && (st = ensure(op->ws_acc, (size_t)op->n_omega * rows_max * sizeof(cpx<double>))) != RSV_OK)
    return st;
  if ((e = cudaMemsetAsync(op->d_flag, 0, sizeof(int), stream)) != cudaSuccess) return cuda_fail(e, "flag reset");
  const size_t ce = coef_bytes(op);
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (trial) {
    if ((e = cudaEventCreate(&ev0)) != cudaSuccess || (e = cudaEventCreate(&ev1)) != cudaSuccess) {
      if (ev0) cudaEventDestroy(ev0);
      return cuda_fail(e, "trial events");
    }
  }
  struct EventGuard {
    cudaEvent_t a, b;
    ~EventGuard() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev_guard{ev0, ev1};
  // host input: each group's [n_omega][kv][n] slice is copied into a staging buffer on the copy stream
  // while the previous group marches; a buffer is refilled once the group that used it two groups
  // earlier has finished with it
  if (host_in) {
    const size_t sb = (size_t)op->n_omega * kg * n * ce;
    for (int i = 0; i < 2; ++i) {
      if ((st = ensure(op->ws_stage[i], sb)) != RSV_OK) return st;
      if (!op->ev_copied[i] && (e = cudaEventCreateWithFlags(&op->ev_copied[i], cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "staging events");
      if (!op->ev_free[i] && (e = cudaEventCreateWithFlags(&op->ev_free[i], cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "staging events");
    }
    if (!op->copy_stream && (e = cudaStreamCreateWithFlags(&op->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e, "copy stream");
  }
  // whatever path the march leaves by, no copy from the caller's host block is left in flight
  struct CopyDrain {
    cudaStream_t s;
    ~CopyDrain() {
      if (s) cudaStreamSynchronize(s);
    }
  } copy_drain{host_in ? op->copy_stream : nullptr};
  auto stage_copy = [&](int gi) -> cudaError_t {   // group gi into staging buffer gi % 2
    const int a0 = gi * kg;
    const int kv = std::min(kg, k - a0);
    const int b = gi & 1;
    cudaError_t ee = cudaSuccess;
    if (gi >= 2) ee = cudaStreamWaitEvent(op->copy_stream, op->ev_free[b], 0);
    if (ee == cudaSuccess)
      ee = cudaMemcpy2DAsync(op->ws_stage[b].ptr, (size_t)kv * n * ce, static_cast<const char*>(in) + (size_t)a0 * n * ce,
                             (size_t)k * n * ce, (size_t)kv * n * ce, op->n_omega, cudaMemcpyHostToDevice,
                             op->copy_stream);
    if (ee == cudaSuccess) ee = cudaEventRecord(op->ev_copied[b], op->copy_stream);
    return ee;
  };
  if (host_in && (e = stage_copy(0)) != cudaSuccess) return cuda_fail(e, "staging copy");
  for (int v0 = 0; v0 < (trial ? std::min(kg, k) : k); v0 += kg) {
    const int kv = std::min(kg, k - v0);
    const int64_t rows = (int64_t)kv * n;
    cpx<double>* acc;
    int64_t acc_stride;
    if (acc_in_out) {
      acc = reinterpret_cast<cpx<double>*>(out) + (int64_t)v0 * n;
      acc_stride = (int64_t)k * n;
      e = cudaMemset2DAsync(acc, acc_stride * sizeof(cpx<double>), 0, rows * sizeof(cpx<double>), op->n_omega,
                            stream);
    } else {
      acc = reinterpret_cast<cpx<double>*>(op->ws_acc.ptr);
      acc_stride = rows;
      e = cudaMemsetAsync(acc, 0, (size_t)op->n_omega * rows * sizeof(cpx<double>), stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(op->ws_state.ptr, 0, rows * se + stage_scratch_bytes(op, kv), stream);
    if (e != cudaSuccess) return cuda_fail(e, "march reset");
    TileGeom g;
    g.rows = rows;
    g.coef_stride = (int64_t)k * n;
    g.n_omega = op->n_omega;
    g.sgn = adjoint ? -1 : 1;
    g.m4 = 4 * op->n_t;
    const void* fh = nullptr;
    int synth_stride = 1;
    const void* gin = static_cast<const char*>(in) + (size_t)v0 * n * ce;
    int64_t gin_stride = (int64_t)k * n;
    const int gi = v0 / kg;
    if (host_in) {   // next group's copy first, then wait for this group's
      if (v0 + kg < k && (e = stage_copy(gi + 1)) != cudaSuccess) return cuda_fail(e, "staging copy");
      if ((e = cudaStreamWaitEvent(stream, op->ev_copied[gi & 1], 0)) != cudaSuccess) return cuda_fail(e, "staging wait");
      gin = op->ws_stage[gi & 1].ptr;
      gin_stride = rows;
    }
    if (s_in) {   // the group's coefficients times the input scaling (B, or C W_y for the adjoint)
      if ((st = ensure(op->ws_scaled, (size_t)op->n_omega * rows * ce)) != RSV_OK) return st;
      ProfScope ps(op, PROF_GLUE);
      e = launch_scale_block<R>(gin, gin_stride, op->ws_scaled.ptr, rows, op->n_omega, rows, n, s_in, stream);
      if (e != cudaSuccess) return cuda_fail(e, "input scaling");
      gin = op->ws_scaled.ptr;
      gin_stride = rows;
    }
    {
      ProfScope ps(op, PROF_GLUE, op->kind == RSV_OP_DENSE ? (kv == k ? 3 : 2 * op->n_omega + 1) : 0);
      st = prepare_coefficients<R>(op, gin, gin_stride, kv, adjoint, &fh, &g.coef_stride, &synth_stride);
    }
    if (st != RSV_OK) return st;
    g.tau_stride = synth_stride;
    // TRM truncation by the state norm: per-vector peak over the tile ends so far
    const bool truncate = opts != nullptr && opts->variant == RSV_TRM && opts->tail_tol > 0.0;
    std::vector<double> peak(truncate ? kv : 0, 0.0), nrm(truncate ? kv : 0, 0.0);
    if (trial && (e = cudaEventRecord(ev0, stream)) != cudaSuccess) return cuda_fail(e, "trial event");
    for (int64_t n0 = 0; n0 < (trial ? std::min<int64_t>(S, sc.total) : sc.total); n0 += S) {
      g.n0 = n0;
      g.steps = (int)std::min<int64_t>(S, sc.total - n0);
      g.n_tau = synth_stride == 2 ? g.steps : 0;
      const bool forced = trial ? true : n0 < sc.forced;
      const bool analysed = trial ? true : n0 + g.steps > sc.first;
      if (forced) {
        if (sizeof(R) == 4 && tc_contract_supported(op, true)) {
          const int nt = g.n_tau > 0 ? g.n_tau : 2 * g.steps + 1;
          const int calls = (nt + (op->real_state ? 511 : 255)) / (op->real_state ? 512 : 256);
          ProfScope ps(op, PROF_SYNTH, 2 * calls);
          e = tc_synth(op, g, fh, op->ws_ftile.ptr);
        } else {
          ProfScope ps(op, PROF_SYNTH);
          e = launch_synth<R>(g, fh, op->d_tw, op->d_pj, op->d_cw, op->real_state, op->ws_ftile.ptr, stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "synthesis");
      }
      const int y_first = trial ? 0 : (analysed ? (int)std::max<int64_t>(0, sc.first - n0) : g.steps);
      MarchTile mt;
      mt.n0 = n0;
      mt.steps = g.steps;
      mt.n_forced = trial ? n0 + g.steps : sc.forced;
      mt.y_first = y_first;
      mt.kg = kv;
      mt.adjoint = adjoint;
      {
        ProfScope ps(op, PROF_MARCH, march_tile_kernels(op, g.steps, kv));
        e = march_tile<R>(op, mt, op->ws_state.ptr, forced ? op->ws_ftile.ptr : nullptr,
                          analysed ? op->ws_ysnap.ptr : nullptr, (double*)op->ws_norm.ptr);
      }
      if (e != cudaSuccess) return cuda_fail(e, "march tile");
      if (analysed) {
        if (sizeof(R) == 4 && tc_contract_supported(op, false)) {
          ProfScope ps(op, PROF_ANALYSIS, 2);
          e = tc_analysis(op, g, op->ws_ysnap.ptr, y_first, g.steps, acc, acc_stride);
        } else {
          ProfScope ps(op, PROF_ANALYSIS);
          e = launch_analysis<R>(g, op->ws_ysnap.ptr, y_first, g.steps, op->d_tw, op->d_pj, op->real_state, acc,
                                 acc_stride, stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "analysis");
      }
      if (truncate) {
        const int64_t n_end = n0 + g.steps;
        e = state_sq_norms(op, kv, n_end, (double*)op->ws_norm.ptr);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(nrm.data(), op->ws_norm.ptr, sizeof(double) * kv, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_fail(e, "tail norm");
        bool small = true;
        for (int v = 0; v < kv; ++v) {
          const double r = std::sqrt(nrm[v]);
          peak[v] = std::max(peak[v], r);
          if (!(r <= opts->tail_tol * peak[v])) small = false;
        }
        op->last_steps = n_end;
        if (n_end >= sc.forced && small) break;
      }
    }
    if (host_in && (e = cudaEventRecord(op->ev_free[gi & 1], stream)) != cudaSuccess)
      return cuda_fail(e, "staging event");
    if (trial) {
      float ms = 0.f;
      e = cudaEventRecord(ev1, stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
      if (e != cudaSuccess) return cuda_fail(e, "trial timing");
      *trial->ms = ms;
      *trial->steps = g.steps;
      break;
    }
    if (!truncate) op->last_steps = sc.total;
    void* o = static_cast<char*>(out) + (size_t)v0 * n * ce;
    e = launch_finish<R>(acc, acc_stride, op->n_omega, rows, 1.0 / (double)op->n_t, o, (int64_t)k * n, stream,
                         s_out, n);
    if (e != cudaSuccess) return cuda_fail(e, "finish");
  }
  int flag = 0;
  e = cudaMemcpyAsync(&flag, op->d_flag, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "march");
  if (flag == 2) return fail(RSV_ERR_TIMEOUT, "a bounded device wait expired in the tensor-core step");
  if (flag) return fail(RSV_ERR_DIVERGED, "state norm became non-finite during the march");
  return RSV_OK;
}

// Measured choice of the tile length and vector group (rsv_autotune): candidates S in {D, D/2}
// (D the default tile) and kg in {k, k/2, k/4, 1}, each timed on one forced and analysed tile of
// the first vector group (run twice, the second timing kept), compared by time per vector-step.
template <typename R>
static rsv_status autotune_impl(rsv_operator op, const void* in, int k, const rsv_march_opts* opts, int32_t* tile,
                                int32_t* group) {
  const int d = default_tile_steps(op);
  std::vector<int> ss = {d};
  if (d / 2 >= 16) ss.push_back(d / 2);
  std::vector<int> gs;
  for (int c : {k, (k + 1) / 2, (k + 3) / 4, 1})
    if (std::find(gs.begin(), gs.end(), c) == gs.end()) gs.push_back(c);
  double best = 1e300;
  int bs = 0, bg = 0;
  for (int S : ss)
    for (int kg : gs) {
      float ms = 0.f;
      int steps = 0;
      TileTrial tr{S, kg, &ms, &steps};
      rsv_status st = RSV_OK;
      for (int rep = 0; rep < 2 && st == RSV_OK; ++rep)
        st = march_impl<R>(op, in, k, opts, nullptr, false, SCALE_NONE, &tr);
      if (st == RSV_ERR_OOM) continue;   // does not fit next to the caller's blocks
      if (st != RSV_OK) return st;
      const double per = (double)ms / ((double)std::max(steps, 1) * std::min(kg, k));
      if (per < best) {
        best = per;
        bs = S;
        bg = kg;
      }
    }
  if (bs == 0) return fail(RSV_ERR_OOM, "no tile configuration fits in device memory");
  op->tuned_k = k;
  op->tuned_tile = bs;
  op->tuned_group = bg;
  if (tile) *tile = bs;
  if (group) *group = bg;
  return RSV_OK;
}

rsv_status march_any(rsv_operator op, const void* in, int k, const rsv_march_opts* opts, void* out, bool adjoint,
                     int scaling, bool host_in) {
  if (!op || !in || !out || k < 1) return fail(RSV_ERR_INVALID_ARG, "bad march arguments");
  if (!op->have_freq) return fail(RSV_ERR_STATE, "rsv_set_frequencies must come first");
  if (in == out) return fail(RSV_ERR_INVALID_ARG, "input and output blocks must not alias");
  if (opts && opts->group_vectors < 0) return fail(RSV_ERR_INVALID_ARG, "group_vectors must be >= 0");
  return op->prec == RSV_PREC_FP64 ? march_impl<double>(op, in, k, opts, out, adjoint, scaling, nullptr, host_in)
                                   : march_impl<float>(op, in, k, opts, out, adjoint, scaling, nullptr, host_in);
}

}  // namespace rsv

extern "C" rsv_status rsv_march_direct(rsv_operator op, const void* f_hat, int32_t k, const rsv_march_opts* opts,
                                       void* y_hat) {
  return march_any(op, f_hat, k, opts, y_hat, false, SCALE_PLAIN);
}

extern "C" rsv_status rsv_march_adjoint(rsv_operator op, const void* y_hat, int32_t k, const rsv_march_opts* opts,
                                        void* w_hat) {
  return march_any(op, y_hat, k, opts, w_hat, true, SCALE_PLAIN);
}

extern "C" rsv_status rsv_march_direct_host(rsv_operator op, const void* f_hat_host, int32_t k,
                                            const rsv_march_opts* opts, void* y_hat) {
  return march_any(op, f_hat_host, k, opts, y_hat, false, SCALE_PLAIN, true);
}

extern "C" rsv_status rsv_march_adjoint_host(rsv_operator op, const void* y_hat_host, int32_t k,
                                             const rsv_march_opts* opts, void* w_hat) {
  return march_any(op, y_hat_host, k, opts, w_hat, true, SCALE_PLAIN, true);
}

// Diagonal B, C, W_f, W_y (Sec. 2.1).  The per-point factors the runs use are formed here in FP64.
extern "C" rsv_status rsv_autotune(rsv_operator op, const void* f_hat, int32_t k, const rsv_march_opts* opts,
                                   int32_t* tile, int32_t* group) {
  if (!op || !f_hat || k < 1) return fail(RSV_ERR_INVALID_ARG, "bad autotune arguments");
  if (!op->have_freq) return fail(RSV_ERR_STATE, "rsv_set_frequencies must come first");
  return op->prec == RSV_PREC_FP64 ? autotune_impl<double>(op, f_hat, k, opts, tile, group)
                                   : autotune_impl<float>(op, f_hat, k, opts, tile, group);
}

extern "C" rsv_status rsv_set_weights(rsv_operator op, const double* b, const double* c, const double* w_f,
                                      const double* w_y) {
  if (!op) return fail(RSV_ERR_INVALID_ARG, "null operator");
  if (op->d_wt) cudaFree(op->d_wt);
  op->d_wt = nullptr;
  op->have_weights = false;
  if (!b && !c && !w_f && !w_y) return RSV_OK;
  const int64_t n = op->n;
  std::vector<double> t((size_t)9 * n);
  for (int64_t p = 0; p < n; ++p) {
    const double bp = b ? b[p] : 1.0, cp = c ? c[p] : 1.0, wf = w_f ? w_f[p] : 1.0, wy = w_y ? w_y[p] : 1.0;
    if (!(bp >= 0.0 && std::isfinite(bp)) || !(cp >= 0.0 && std::isfinite(cp)))
      return fail(RSV_ERR_INVALID_ARG, "forcing and observation entries must be finite and >= 0");
    if (!(wf > 0.0 && std::isfinite(wf)) || !(wy > 0.0 && std::isfinite(wy)))
      return fail(RSV_ERR_INVALID_ARG, "metric entries must be finite and > 0");
    const double v[9] = {bp, cp, cp * wy, bp / wf, bp / std::sqrt(wf), cp * std::sqrt(wy), 1.0 / std::sqrt(wf),
                         1.0 / std::sqrt(wy), std::sqrt(wf)};
    for (int r = 0; r < 9; ++r) t[(size_t)r * n + p] = v[r];
  }
  cudaError_t e = cudaMalloc(&op->d_wt, t.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(op->d_wt, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (op->d_wt) cudaFree(op->d_wt);
    op->d_wt = nullptr;
    return cuda_fail(e, "weights upload");
  }
  op->have_weights = true;
  return RSV_OK;
}

extern "C" rsv_status rsv_decay_probe(rsv_operator op, int32_t adjoint, double tol, int64_t max_steps, uint64_t seed,
                                      int32_t check_every, int64_t* steps, double* ratio) {
  if (!op) return fail(RSV_ERR_INVALID_ARG, "null operator");
  if (!op->have_freq) return fail(RSV_ERR_STATE, "rsv_set_frequencies must come first (it sets the step)");
  return probe_any(op, adjoint != 0, tol, max_steps, seed, check_every, steps, ratio);
}

extern "C" rsv_status rsv_apply_operator(rsv_operator op, const void* x, int32_t k, int32_t adjoint, void* y) {
  if (!op || !x || !y || k < 1) return fail(RSV_ERR_INVALID_ARG, "bad apply arguments");
  cudaError_t e = op->prec == RSV_PREC_FP64 ? apply_op<double>(op, x, k, adjoint != 0, y)
                                            : apply_op<float>(op, x, k, adjoint != 0, y);
  if (e == cudaSuccess) e = cudaStreamSynchronize(op->stream);
  if (e != cudaSuccess) return cuda_fail(e, "apply");
  return RSV_OK;
}
