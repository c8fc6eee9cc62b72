// Direct march that allocates nothing: rsv_march_direct_static.
//
// Some callers cannot call cudaMalloc once they are running: a solver that
// reserves the device memory for its own pool at start-up and forbids any
// later allocation, or a real-time loop that must never stall on the
// allocator (cudaMalloc / cudaFree may synchronise the whole device).
// rsv_march_direct grows its workspace lazily and therefore may allocate on
// any call.  This variant keeps all of the march's scratch (state, forcing
// tile, snapshot tile, FP64 accumulators) in one file-scope device array of
// fixed size instead.  The call still ends by synchronising the operator's
// stream, as every entry point of the library does.
//
// The array exists once per GPU that loads the library and stays allocated
// until the process exits.  Every call shares it and it keeps the contents
// of the last call, so each call clears the parts that must start at zero;
// two calls whose device work overlaps (different streams, no ordering
// between them) race on it.  Host code must not pass the array's name to a
// kernel: in host code that name is only a host-side stand-in for the
// symbol.  The device address comes from cudaGetSymbolAddress, taken once
// per device with that device current, on the first call made there; make
// that first call before any stream capture begins.
#include <mutex>

#include "rsv_ops.h"

namespace rsv {
rsv_status fail(rsv_status s, const std::string& msg);
size_t state_elem_bytes(rsv_operator op);
size_t coef_bytes(rsv_operator op);
}  // namespace rsv

namespace {

constexpr size_t kStaticScratchBytes = (size_t)RSV_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_march_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the static array on the current device (set-up on first use).
rsv_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rsv::cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return rsv::fail(RSV_ERR_INVALID_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_march_scratch);
    if (e != cudaSuccess || p == nullptr) return rsv::cuda_fail(e, "cudaGetSymbolAddress(static march scratch)");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return RSV_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename R>
rsv_status march_static_impl(rsv_operator op, const void* in, int k, const rsv_march_opts* o, void* out) {
  using namespace rsv;
  rsv_march_opts def{};
  if (!o) o = &def;
  int64_t total, first, forced;
  if (o->variant == RSV_SSRM) {
    if (o->n_transient_windows < 0) return fail(RSV_ERR_INVALID_ARG, "n_transient_windows < 0");
    total = (int64_t)(o->n_transient_windows + 1) * op->n_t;
    first = (int64_t)o->n_transient_windows * op->n_t;
    forced = total;
  } else if (o->variant == RSV_TRM) {
    if (o->tail_steps < 0) return fail(RSV_ERR_INVALID_ARG, "tail_steps < 0");
    if (o->tail_tol != 0.0)
      return fail(RSV_ERR_INVALID_ARG, "the allocation-free march runs the whole TRM tail: tail_tol must be 0");
    total = op->n_t + o->tail_steps;
    first = 0;
    forced = op->n_t;
  } else {
    return fail(RSV_ERR_INVALID_ARG, "unknown variant");
  }
  const int64_t n = op->n;
  const int64_t rows = (int64_t)k * n;
  const size_t se = state_elem_bytes(op);
  const bool acc_in_out = (op->prec == RSV_PREC_FP64);
  // Layout of the static array: state | forcing tile | snapshot tile | accumulators | norms.
  // The tile length shrinks (halving) until the layout fits.
  int S = o->tile_steps > 0 ? o->tile_steps : default_tile_steps(op);
  size_t b_state = 0, b_f = 0, b_y = 0, b_acc = 0, b_norm = 0;
  for (;;) {
    b_state = align256(rows * se + stage_scratch_bytes(op, k));
    b_f = align256((size_t)(2 * S + 1) * rows * se);
    b_y = align256((size_t)S * rows * se);
    b_acc = acc_in_out ? 0 : align256((size_t)op->n_omega * rows * sizeof(cpx<double>));
    b_norm = align256((size_t)k * op->n_inst * sizeof(double));
    if (b_state + b_f + b_y + b_acc + b_norm <= kStaticScratchBytes || S <= 8) break;
    S /= 2;
  }
  const size_t need = b_state + b_f + b_y + b_acc + b_norm;
  if (need > kStaticScratchBytes)
    return fail(RSV_ERR_INVALID_ARG, "rsv_march_direct_static needs " + std::to_string(need) +
                                         " bytes of scratch for this operator, k and frequency count; its static "
                                         "array holds " + std::to_string(kStaticScratchBytes) + " bytes");
  void* base = nullptr;
  rsv_status st = scratch_address(&base);
  if (st != RSV_OK) return st;
  char* p = static_cast<char*>(base);
  void* d_state = p;
  void* d_f = p + b_state;
  void* d_y = p + b_state + b_f;
  cpx<double>* d_acc = reinterpret_cast<cpx<double>*>(p + b_state + b_f + b_y);
  double* d_norm = reinterpret_cast<double*>(p + b_state + b_f + b_y + b_acc);
  const cudaStream_t stream = op->stream;
  cudaError_t e;
  cpx<double>* acc;
  int64_t acc_stride;
  if (acc_in_out) {
    acc = reinterpret_cast<cpx<double>*>(out);
    acc_stride = rows;
  } else {
    acc = d_acc;
    acc_stride = rows;
  }
  // the array holds the previous call's data: clear state, accumulators and the divergence flag
  e = cudaMemsetAsync(acc, 0, (size_t)op->n_omega * rows * sizeof(cpx<double>), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_state, 0, rows * se, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(op->d_flag, 0, sizeof(int), stream);
  if (e != cudaSuccess) return cuda_fail(e, "static march reset");
  TileGeom g;
  g.rows = rows;
  g.coef_stride = rows;
  g.n_omega = op->n_omega;
  g.sgn = 1;
  g.m4 = 4 * op->n_t;
  for (int64_t n0 = 0; n0 < total; n0 += S) {
    g.n0 = n0;
    g.steps = (int)std::min<int64_t>(S, total - n0);
    const bool is_forced = n0 < forced;
    const bool analysed = n0 + g.steps > first;
    if (is_forced) {
      e = launch_synth<R>(g, in, op->d_tw, op->d_pj, op->d_cw, op->real_state, d_f, stream);
      if (e != cudaSuccess) return cuda_fail(e, "synthesis");
    }
    const int y_first = analysed ? (int)std::max<int64_t>(0, first - n0) : g.steps;
    MarchTile mt;
    mt.n0 = n0;
    mt.steps = g.steps;
    mt.n_forced = forced;
    mt.y_first = y_first;
    mt.kg = k;
    mt.adjoint = false;
    e = march_tile<R>(op, mt, d_state, is_forced ? d_f : nullptr, analysed ? d_y : nullptr, d_norm);
    if (e != cudaSuccess) return cuda_fail(e, "march tile");
    if (analysed) {
      e = launch_analysis<R>(g, d_y, y_first, g.steps, op->d_tw, op->d_pj, op->real_state, acc, acc_stride, stream);
      if (e != cudaSuccess) return cuda_fail(e, "analysis");
    }
  }
  e = launch_finish<R>(acc, acc_stride, op->n_omega, rows, 1.0 / (double)op->n_t, out, rows, stream);
  if (e != cudaSuccess) return cuda_fail(e, "finish");
  int flag = 0;
  e = cudaMemcpyAsync(&flag, op->d_flag, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "static march");
  if (flag) return fail(RSV_ERR_DIVERGED, "state norm became non-finite during the march");
  return RSV_OK;
}

}  // namespace

extern "C" rsv_status rsv_march_direct_static(rsv_operator op, const void* f_hat, int32_t k,
                                              const rsv_march_opts* opts, void* y_hat) {
  using namespace rsv;
  if (!op || !f_hat || !y_hat || k < 1) return fail(RSV_ERR_INVALID_ARG, "bad march arguments");
  if (!op->have_freq) return fail(RSV_ERR_STATE, "rsv_set_frequencies must come first");
  if (op->kind != RSV_OP_GL1D)
    return fail(RSV_ERR_INVALID_ARG, "rsv_march_direct_static supports the three-point (GL1D) operator kind only");
  if (f_hat == y_hat) return fail(RSV_ERR_INVALID_ARG, "input and output blocks must not alias");
  if (op->have_weights)
    return fail(RSV_ERR_INVALID_ARG, "rsv_march_direct_static applies no forcing / observation weights: clear them "
                                     "with rsv_set_weights(op, NULL, NULL, NULL, NULL)");
  return op->prec == RSV_PREC_FP64 ? march_static_impl<double>(op, f_hat, k, opts, y_hat)
                                   : march_static_impl<float>(op, f_hat, k, opts, y_hat);
}
