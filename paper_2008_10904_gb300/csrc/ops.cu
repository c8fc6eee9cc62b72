// Operator kinds: construction of the device coefficient arrays and the
// dispatch of one march tile / one operator application to each kind's
// kernels.
#include <cuda_bf16.h>

#include <cstdlib>
#include <algorithm>
#include <cmath>
#include <complex>
#include <functional>
#include <queue>
#include <type_traits>
#include <vector>

#include "rsv_ops.h"

namespace rsv {

namespace {

template <typename R>
std::vector<cpx<R>> narrow(const std::vector<std::complex<double>>& v) {
  std::vector<cpx<R>> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = mk<R>((R)v[i].real(), (R)v[i].imag());
  return o;
}

rsv_status upload_cvec(rsv_operator op, const std::vector<std::complex<double>>& v, void** dst) {
  if (op->prec == RSV_PREC_FP64) {
    auto o = narrow<double>(v);
    return upload(op, o.data(), o.size() * sizeof(cpx<double>), dst);
  }
  auto o = narrow<float>(v);
  return upload(op, o.data(), o.size() * sizeof(cpx<float>), dst);
}

}  // namespace

// Linearised GL (Sec. 3, Eq. (GL_timeDomain) family) with central differences:
//   (A u)_i = lo_i u_{i-1} + di_i u_i + up_i u_{i+1},
//   lo = nu/(2dx) + gamma/dx^2, up = -nu/(2dx) + gamma/dx^2,
//   di = -2 gamma/dx^2 + mu(x_i),  mu = mu0 + mu_shift + mu2 x^2,
// Dirichlet zeros beyond each instance.  The adjoint (A^H) coefficients are
//   lo^H_i = conj(up_{i-1}), di^H_i = conj(di_i), up^H_i = conj(lo_{i+1}).
rsv_status build_gl1d(rsv_operator op, const rsv_operator_desc* d) {
  if (d->n_instances < 1 || !d->gl_n || !d->gl_mu0) return fail(RSV_ERR_INVALID_ARG, "GL1D needs instances");
  if (!(d->x1 > d->x0)) return fail(RSV_ERR_INVALID_ARG, "GL1D needs x1 > x0");
  op->n_inst = d->n_instances;
  int64_t tot = 0;
  int maxn = 0;
  for (int i = 0; i < d->n_instances; ++i) {
    if (d->gl_n[i] < 2 || d->gl_n[i] > 4096) return fail(RSV_ERR_INVALID_ARG, "GL1D instance size must be 2..4096");
    op->inst_off.push_back(tot);
    op->inst_len.push_back(d->gl_n[i]);
    tot += d->gl_n[i];
    maxn = std::max(maxn, (int)d->gl_n[i]);
  }
  op->n = tot;
  op->gl_max_n = maxn;
  op->real_state = false;
  const std::complex<double> nu(d->nu_re, d->nu_im), ga(d->gamma_re, d->gamma_im);
  std::vector<std::complex<double>> lo(tot), di(tot), up(tot), alo(tot), adi(tot), aup(tot);
  for (int i = 0; i < d->n_instances; ++i) {
    const int64_t off = op->inst_off[i];
    const int n = d->gl_n[i];
    const double dx = (d->x1 - d->x0) / (double)(n + 1);
    for (int p = 0; p < n; ++p) {
      const double x = d->x0 + (p + 1) * dx;
      const double mu = d->gl_mu0[i] + d->mu_shift + d->mu1 * x + d->mu2 * x * x;
      lo[off + p] = (p > 0) ? nu / (2.0 * dx) + ga / (dx * dx) : 0.0;
      up[off + p] = (p < n - 1) ? -nu / (2.0 * dx) + ga / (dx * dx) : 0.0;
      di[off + p] = -2.0 * ga / (dx * dx) + mu;
    }
    for (int p = 0; p < n; ++p) {
      alo[off + p] = (p > 0) ? std::conj(up[off + p - 1]) : 0.0;
      adi[off + p] = std::conj(di[off + p]);
      aup[off + p] = (p < n - 1) ? std::conj(lo[off + p + 1]) : 0.0;
    }
  }
  const std::vector<std::complex<double>>* arrs[6] = {&lo, &di, &up, &alo, &adi, &aup};
  op->tri_host.assign((size_t)12 * tot, 0.0);
  for (int a = 0; a < 6; ++a) {
    rsv_status s = upload_cvec(op, *arrs[a], &op->tri[a]);
    if (s != RSV_OK) return s;
    for (int64_t p = 0; p < tot; ++p) {
      op->tri_host[(size_t)2 * (a * tot + p)] = (*arrs[a])[p].real();
      op->tri_host[(size_t)2 * (a * tot + p) + 1] = (*arrs[a])[p].imag();
    }
  }
  return RSV_OK;
}

// Cyclic-reduction factors of I - h/2 A (Crank-Nicolson), direct and adjoint, per instance, in FP64:
// with b, a, c the diagonal and the couplings to i - s and i + s, level l (s = 2^l) eliminates
// both neighbours, k1 = a_i / b_{i-s}, k2 = c_i / b_{i+s}; a_i <- -k1 a_{i-s}, c_i <- -k2 c_{i+s},
// b_i <- b_i - k1 c_{i-s} - k2 a_{i+s}.  Stored: k1, k2 per level, then 1 / b after the last level.
static rsv_status gl1d_cn_factors(rsv_operator op) {
  using cdd = std::complex<double>;
  const int64_t n = op->n;
  int L = 0;
  while ((1 << L) < op->gl_max_n) ++L;
  const double hh = 0.5 * op->h;
  std::vector<cdd> out((size_t)2 * (2 * L + 1) * n);
  auto coef = [&](int a, int64_t p) {
    return cdd(op->tri_host[(size_t)2 * (a * n + p)], op->tri_host[(size_t)2 * (a * n + p) + 1]);
  };
  for (int dir = 0; dir < 2; ++dir) {
    cdd* K1 = out.data() + (size_t)dir * (2 * L + 1) * n;
    cdd* K2 = K1 + (size_t)L * n;
    cdd* INV = K2 + (size_t)L * n;
    for (int i = 0; i < op->n_inst; ++i) {
      const int64_t off = op->inst_off[i];
      const int len = (int)op->inst_len[i];
      std::vector<cdd> a(len), b(len), c(len), na(len), nb(len), nc(len);
      for (int p = 0; p < len; ++p) {
        b[p] = 1.0 - hh * coef(3 * dir + 1, off + p);
        a[p] = p > 0 ? -hh * coef(3 * dir, off + p) : 0.0;
        c[p] = p + 1 < len ? -hh * coef(3 * dir + 2, off + p) : 0.0;
      }
      for (int l = 0; l < L; ++l) {
        const int sd = 1 << l;
        for (int p = 0; p < len; ++p) {
          const cdd k1 = p - sd >= 0 ? a[p] / b[p - sd] : 0.0;
          const cdd k2 = p + sd < len ? c[p] / b[p + sd] : 0.0;
          na[p] = p - sd >= 0 ? -k1 * a[p - sd] : 0.0;
          nc[p] = p + sd < len ? -k2 * c[p + sd] : 0.0;
          nb[p] = b[p] - (p - sd >= 0 ? k1 * c[p - sd] : 0.0) - (p + sd < len ? k2 * a[p + sd] : 0.0);
          K1[(size_t)l * n + off + p] = k1;
          K2[(size_t)l * n + off + p] = k2;
        }
        a.swap(na);
        b.swap(nb);
        c.swap(nc);
      }
      for (int p = 0; p < len; ++p) {
        if (!(std::abs(b[p]) > 0.0)) return fail(RSV_ERR_INVALID_ARG, "Crank-Nicolson matrix is singular");
        INV[off + p] = 1.0 / b[p];
      }
    }
  }
  if (op->pcr) cudaFree(op->pcr);
  op->pcr = nullptr;
  const size_t cnt = out.size();
  cudaError_t e;
  if (op->prec == RSV_PREC_FP64) {
    std::vector<cpx<double>> o(cnt);
    for (size_t i = 0; i < cnt; ++i) o[i] = mk<double>(out[i].real(), out[i].imag());
    e = cudaMalloc(&op->pcr, cnt * sizeof(cpx<double>));
    if (e == cudaSuccess) e = cudaMemcpy(op->pcr, o.data(), cnt * sizeof(cpx<double>), cudaMemcpyHostToDevice);
  } else {
    std::vector<cpx<float>> o(cnt);
    for (size_t i = 0; i < cnt; ++i) o[i] = mk<float>((float)out[i].real(), (float)out[i].imag());
    e = cudaMalloc(&op->pcr, cnt * sizeof(cpx<float>));
    if (e == cudaSuccess) e = cudaMemcpy(op->pcr, o.data(), cnt * sizeof(cpx<float>), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return cuda_fail(e, "Crank-Nicolson factors");
  op->pcr_levels = L;
  return RSV_OK;
}


// Default time-tile length: 256 steps, trimmed in FP32 so one tile's stage times fit the
// tensor-core synthesis accumulator (<= 512 columns): 2S + 1 <= 512 real, 2 (2S + 1) <= 512 complex.
int default_tile_steps(rsv_operator op) {
  if (op->prec != RSV_PREC_FP32 || op->kind == RSV_OP_DENSE) return 256;
  return op->real_state ? 255 : 127;
}

static size_t elem_size(rsv_operator op) { return op->prec == RSV_PREC_FP64 ? 8 : 4; }

// Extra march scratch that lives behind the state vector in the state workspace.
size_t stage_scratch_bytes(rsv_operator op, int kg) {
  if (op->kind == RSV_OP_DENSE)  // second state buffer, then the tensor-core operand buffers
    return (size_t)kg * op->n * 2 * elem_size(op) +
           (dense_tc_supported(op, kg) ? std::max(dense_tc_scratch_bytes(op), dense_tc_chain_x_bytes(op)) : 0);
  if (op->kind == RSV_OP_ADR2D || op->kind == RSV_OP_ADV3D) return stencil_scratch_bytes(op, kg);
  return 0;
}

int march_tile_kernels(rsv_operator op, int steps, int kg) {
  switch (op->kind) {
    case RSV_OP_GL1D:
      return 1;
    case RSV_OP_DENSE:
      if (op->prec == RSV_PREC_FP32 && dense_tc_supported(op, kg)) return op->tc_persistent ? 2 : steps + 1;
      return steps + 1;
    case RSV_OP_ADR2D: {
      const char* e = getenv("RSV_STENCIL_FUSED");
      if (e != nullptr && e[0] == '1') return steps + 1;
      const bool pairs = op->prec == RSV_PREC_FP32 && adr2d_pairs_enabled() && op->nx % 4 == 0 &&
                         op->n < ((int64_t)1 << 31);
      return pairs ? 2 * steps + 1 : 4 * steps + 1;   // two stage-pair kernels per step, or four stages
    }
    case RSV_OP_ADV3D: {
      const bool pairs = op->prec == RSV_PREC_FP32 && !op->bf16_state && adv3d_pairs_enabled() &&
                         op->nx % 4 == 0 && op->n < ((int64_t)1 << 31);
      return pairs ? 2 * steps + 1 : 4 * steps + 1;   // two stage-pair kernels per step, or four stages
    }
    default:
      return 4 * steps + 1;
  }
}

rsv_status on_frequencies(rsv_operator op) {
  if (op->kind == RSV_OP_DENSE) return dense_on_frequencies(op);
  if (op->kind == RSV_OP_GL1D && op->scheme == RSV_SCHEME_CN) return gl1d_cn_factors(op);
  return RSV_OK;
}

template <typename R>
rsv_status prepare_coefficients(rsv_operator op, const void* fhat, int64_t f_stride, int kg, bool adjoint,
                                const void** coef, int64_t* coef_stride, int* synth_stride) {
  if (op->kind != RSV_OP_DENSE) {
    *coef = fhat;
    *coef_stride = f_stride;
    *synth_stride = 1;
    return RSV_OK;
  }
  const size_t bytes = (size_t)op->n_omega * kg * op->n * sizeof(cpx<R>);
  rsv_status s = ensure(op->ws_coef, bytes);
  if (s == RSV_OK) s = ensure(op->ws_coef2, bytes);
  if (s != RSV_OK) return s;
  cudaError_t e = dense_prepare<R>(op, fhat, f_stride, kg, adjoint, op->ws_coef.ptr, op->ws_coef2.ptr);
  if (e != cudaSuccess) return cuda_fail(e, "dense coefficient transform");
  *coef = op->ws_coef.ptr;
  *coef_stride = (int64_t)kg * op->n;
  *synth_stride = 2;
  return RSV_OK;
}

namespace {
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return (double)x; }
__device__ __forceinline__ double to_d(__nv_bfloat16 x) { return (double)__bfloat162float(x); }

template <typename T>
__global__ void finite_kernel(const T* __restrict__ x, int64_t count, int* flag) {
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = to_d(x[e]);
    if (!(fabs(v) < 1e300)) bad = true;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(flag, 1);
}

// out[v] += sum of squares of vector v's values (FP64 sums; out zeroed by the caller).
template <typename T>
__global__ void vec_sumsq_kernel(const T* __restrict__ x, int64_t vals_per_vec, double* __restrict__ out) {
  const T* xv = x + (int64_t)blockIdx.y * vals_per_vec;
  double acc = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < vals_per_vec; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = to_d(xv[e]);
    acc += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    atomicAdd(out + blockIdx.y, t);
  }
}
// out[i] += sum of squares of the values of instance i of one vector (FP64 sums; out zeroed by the caller).
template <typename T>
__global__ void inst_sumsq_kernel(const T* __restrict__ x, const int64_t* __restrict__ inst_off, int vals_per_point,
                                  double* __restrict__ out) {
  const int inst = blockIdx.y;
  const int64_t a = inst_off[inst] * vals_per_point, b = inst_off[inst + 1] * vals_per_point;
  double acc = 0.0;
  for (int64_t e = a + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < b; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = to_d(x[e]);
    acc += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    atomicAdd(out + inst, t);
  }
}

// SplitMix64 (Steele, Lea & Flood 2014): value i of stream `seed`.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// x[e] = 2 (z_e >> 11) 2^-53 - 1 for the interleaved values e of the state (exact in FP64).
template <typename T>
__global__ void probe_init_kernel(T* __restrict__ x, int64_t vals, uint64_t seed) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < vals; e += (int64_t)gridDim.x * blockDim.x) {
    const double u = 2.0 * (double)(splitmix64_at(seed, (uint64_t)e) >> 11) * 0x1.0p-53 - 1.0;
    if constexpr (std::is_same<T, __nv_bfloat16>::value)
      x[e] = __float2bfloat16((float)u);
    else
      x[e] = (T)u;
  }
}
}  // namespace

// Per-instance squared 2-norms of vector 0 of the march state after step n_end (kg = 1 layout).
cudaError_t instance_sq_norms(rsv_operator op, int64_t n_end, double* d_out) {
  const size_t elem = op->prec == RSV_PREC_FP64 ? 8 : 4;
  const int vpp = op->real_state ? 1 : 2;
  const char* st = static_cast<const char*>(op->ws_state.ptr);
  if (op->kind == RSV_OP_DENSE) st += (size_t)(n_end & 1) * (size_t)op->n * vpp * elem;
  cudaError_t e = cudaMemsetAsync(d_out, 0, sizeof(double) * op->n_inst, op->stream);
  if (e != cudaSuccess) return e;
  int64_t max_len = 1;
  for (int i = 0; i < op->n_inst; ++i) max_len = std::max(max_len, op->inst_len[i]);
  const unsigned bx = (unsigned)std::min<int64_t>((max_len * vpp + 255) / 256, 2 * std::max(op->sm_count, 1));
  dim3 grid(std::max(bx, 1u), (unsigned)op->n_inst);
  const int64_t* off = (const int64_t*)op->d_inst_off;
  if (op->prec == RSV_PREC_FP64)
    inst_sumsq_kernel<double><<<grid, 256, 0, op->stream>>>((const double*)st, off, vpp, d_out);
  else if (op->bf16_state)
    inst_sumsq_kernel<__nv_bfloat16><<<grid, 256, 0, op->stream>>>((const __nv_bfloat16*)st, off, vpp, d_out);
  else
    inst_sumsq_kernel<float><<<grid, 256, 0, op->stream>>>((const float*)st, off, vpp, d_out);
  return cudaGetLastError();
}

// The decay probe's random initial state in vector 0 of the march state (step 0 layout).
cudaError_t probe_initial_state(rsv_operator op, uint64_t seed) {
  const int64_t vals = (op->real_state ? 1 : 2) * op->n;
  const unsigned blocks = (unsigned)std::min<int64_t>((vals + 255) / 256, 8 * std::max(op->sm_count, 1));
  if (op->prec == RSV_PREC_FP64)
    probe_init_kernel<double><<<blocks, 256, 0, op->stream>>>((double*)op->ws_state.ptr, vals, seed);
  else if (op->bf16_state)
    probe_init_kernel<__nv_bfloat16><<<blocks, 256, 0, op->stream>>>((__nv_bfloat16*)op->ws_state.ptr, vals, seed);
  else
    probe_init_kernel<float><<<blocks, 256, 0, op->stream>>>((float*)op->ws_state.ptr, vals, seed);
  return cudaGetLastError();
}

// Squared 2-norm of each of the kg vectors of the march state after step n_end
// (the dense path keeps two step-parity copies of the state).
cudaError_t state_sq_norms(rsv_operator op, int kg, int64_t n_end, double* d_out) {
  const size_t elem = op->prec == RSV_PREC_FP64 ? 8 : 4;
  const int64_t vals = (op->real_state ? 1 : 2) * op->n;
  const char* st = static_cast<const char*>(op->ws_state.ptr);
  if (op->kind == RSV_OP_DENSE) st += (size_t)(n_end & 1) * (size_t)kg * vals * elem;
  cudaError_t e = cudaMemsetAsync(d_out, 0, sizeof(double) * kg, op->stream);
  if (e != cudaSuccess) return e;
  const unsigned bx = (unsigned)std::min<int64_t>((vals + 255) / 256, std::max(1, 2 * op->sm_count / std::max(kg, 1)));
  dim3 grid(std::max(bx, 1u), (unsigned)kg);
  if (op->prec == RSV_PREC_FP64)
    vec_sumsq_kernel<double><<<grid, 256, 0, op->stream>>>((const double*)st, vals, d_out);
  else if (op->bf16_state)   // BF16 state: vector v's values at v * vals BF16 elements
    vec_sumsq_kernel<__nv_bfloat16><<<grid, 256, 0, op->stream>>>((const __nv_bfloat16*)st, vals, d_out);
  else
    vec_sumsq_kernel<float><<<grid, 256, 0, op->stream>>>((const float*)st, vals, d_out);
  return cudaGetLastError();
}

cudaError_t check_finite(rsv_operator op, const void* state, int64_t count, bool real_state) {
  const int64_t vals = real_state ? count : 2 * count;
  const unsigned blocks = (unsigned)std::min<int64_t>((vals + 255) / 256, 4 * std::max(op->sm_count, 1));
  if (op->prec == RSV_PREC_FP64)
    finite_kernel<double><<<blocks, 256, 0, op->stream>>>((const double*)state, vals, op->d_flag);
  else if (op->bf16_state)
    finite_kernel<__nv_bfloat16><<<blocks, 256, 0, op->stream>>>((const __nv_bfloat16*)state, vals, op->d_flag);
  else
    finite_kernel<float><<<blocks, 256, 0, op->stream>>>((const float*)state, vals, op->d_flag);
  return cudaGetLastError();
}

static Gl1dTile gl1d_geom(rsv_operator op, bool adjoint, int kg) {
  Gl1dTile g;
  const int b = adjoint ? 3 : 0;
  g.lo = op->tri[b];
  g.di = op->tri[b + 1];
  g.up = op->tri[b + 2];
  g.inst_off = (const int64_t*)op->d_inst_off;
  g.n_inst = op->n_inst;
  g.max_n = op->gl_max_n;
  g.n = op->n;
  g.kg = kg;
  g.h = op->h;
  g.n0 = 0;
  g.steps = 0;
  g.n_forced = 0;
  g.y_first = 0;
  g.real_state = false;
  g.cr_lo = g.cr_up = g.cr_inv = nullptr;
  g.cr_levels = 0;
  if (op->scheme == RSV_SCHEME_CN && op->pcr) {
    const size_t es = op->prec == RSV_PREC_FP64 ? sizeof(cpx<double>) : sizeof(cpx<float>);
    const int L = op->pcr_levels;
    const char* base = static_cast<const char*>(op->pcr) + (size_t)(adjoint ? 1 : 0) * (2 * L + 1) * op->n * es;
    g.cr_lo = base;
    g.cr_up = base + (size_t)L * op->n * es;
    g.cr_inv = base + (size_t)2 * L * op->n * es;
    g.cr_levels = L;                // >= 1: every instance has at least two points
  }
  return g;
}

// Packing of uneven GL1D batches: when the one-CTA-per-(instance, vector) launch needs more CTAs than
// there are SMs, the (instance, vector) segments are packed into CTAs of gl1d_pack_threads<R>() threads
// x ppt slots (each segment followed by a zero separator slot), so that short instances do not hold a
// CTA sized for the longest one.  RSV_GL1D_PACK=0 keeps the one-per-pair launch.
template <typename R>
static bool gl1d_pack_wanted(rsv_operator op, int kg) {
  static const bool env = [] {
    const char* e = getenv("RSV_GL1D_PACK");
    return !(e != nullptr && e[0] == '0');
  }();
  return env && op->scheme == RSV_SCHEME_RK4 && op->n_inst > 1 && op->gl_max_n <= 4 * gl1d_pack_threads<R>() &&
         (int64_t)op->n_inst * kg > op->sm_count && (int64_t)kg * op->n < ((int64_t)1 << 31);
}

namespace {
struct PackItem {
  int64_t len;
  int inst, v;
};
// Longest processing time first: the segments, longest first, each go to the least loaded of n_bins
// packs of cap slots (a separator slot before every segment but a pack's first).  The packs of one wave
// then carry nearly equal loads, which set the time of the wave.  Returns false when a segment finds no
// pack with room (the least loaded has none), so the caller can add a wave.
bool pack_lpt(const std::vector<PackItem>& items, int64_t cap, int n_bins, std::vector<std::vector<PackItem>>& packs) {
  using Load = std::pair<int64_t, int>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  packs.assign((size_t)n_bins, {});
  for (int b = 0; b < n_bins; ++b) heap.push({0, b});
  for (const PackItem& it : items) {
    Load top = heap.top();
    const int64_t need = (top.first > 0 ? 1 : 0) + it.len;
    if (top.first + need > cap) return false;
    heap.pop();
    packs[(size_t)top.second].push_back(it);
    heap.push({top.first + need, top.second});
  }
  packs.erase(std::remove_if(packs.begin(), packs.end(), [](const std::vector<PackItem>& p) { return p.empty(); }),
              packs.end());
  return true;
}
}  // namespace

// Slots per thread (ppt, 1 to 4, at least enough for the longest instance): the one whose packs fill
// the fewest waves (SMs x resident CTAs), the smaller on a tie.  Each wave costs about the time of its
// fullest pack, so one wave of CTAs holding ~2400 of 3072 slots beats two of ~1200 of 2048 (0.29
// against 0.38 ms per 127-step tile on the 64-instance batch, where the fixed per-warp work of a step
// is spread over fewer slots).  For each ppt the fill takes as many waves as the slots need, one more
// while the longest-first fill leaves a segment without room.  RSV_GL1D_PPT forces a ppt.
template <typename R>
static cudaError_t gl1d_build_packs(rsv_operator op, int kg) {
  if (op->pack_map != nullptr && op->pack_kg == kg) return cudaSuccess;
  const int nt = gl1d_pack_threads<R>();
  std::vector<PackItem> items;
  int64_t slots = 0;
  for (int v = 0; v < kg; ++v)
    for (int i = 0; i < op->n_inst; ++i) {
      items.push_back({op->inst_len[i], i, v});
      slots += op->inst_len[i] + 1;
    }
  std::stable_sort(items.begin(), items.end(), [](const PackItem& a, const PackItem& b) { return a.len > b.len; });
  const int ppt_min = (int)((op->gl_max_n + nt - 1) / nt);
  const char* env = getenv("RSV_GL1D_PPT");
  const int forced = env ? atoi(env) : 0;
  const bool force = forced >= ppt_min && forced <= 4;
  int ppt = 0, wave = 0;
  int64_t best_waves = 0;
  std::vector<std::vector<PackItem>> packs;
  for (int q = force ? forced : ppt_min; q <= (force ? forced : 4); ++q) {
    const int64_t cap_q = (int64_t)nt * q;
    int per_sm = 0;
    cudaError_t e = gl1d_pack_occupancy<R>(q, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) continue;
    const int wave_q = op->sm_count * per_sm;
    std::vector<std::vector<PackItem>> packs_q;
    int64_t waves = std::max<int64_t>(1, (slots + wave_q * cap_q - 1) / (wave_q * cap_q));
    while (!pack_lpt(items, cap_q, (int)(waves * wave_q), packs_q)) ++waves;   // ends: one segment per pack fits
    if (ppt == 0 || waves < best_waves) {
      ppt = q;
      wave = wave_q;
      best_waves = waves;
      packs.swap(packs_q);
    }
  }
  if (ppt == 0) return cudaErrorInvalidConfiguration;
  const int64_t cap = (int64_t)nt * ppt;
  std::vector<int32_t> map(packs.size() * (size_t)cap, -1);
  for (size_t b = 0; b < packs.size(); ++b) {
    int64_t pos = 0;
    for (const PackItem& it : packs[b]) {
      const int64_t r0 = (int64_t)it.v * op->n + op->inst_off[it.inst];
      for (int64_t j = 0; j < it.len; ++j) map[b * cap + pos + j] = (int32_t)(r0 + j);
      pos += it.len + 1;
    }
  }
  if (op->pack_map) cudaFree(op->pack_map);
  op->pack_map = nullptr;
  op->pack_kg = 0;
  cudaError_t e = cudaMalloc(&op->pack_map, map.size() * sizeof(int32_t));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(op->pack_map, map.data(), map.size() * sizeof(int32_t), cudaMemcpyHostToDevice, op->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(op->stream);
  if (e != cudaSuccess) return e;
  op->pack_kg = kg;
  op->pack_count = (int)packs.size();
  op->pack_threads = nt;
  op->pack_ppt = ppt;
  op->pack_wave = wave;
  return cudaSuccess;
}

template <typename R>
static cudaError_t march_tile_direct(rsv_operator op, const MarchTile& t, void* state, const void* F, void* Y,
                                     double* norms) {
  switch (op->kind) {
    case RSV_OP_GL1D: {
      Gl1dTile g = gl1d_geom(op, t.adjoint, t.kg);
      g.n0 = t.n0;
      g.steps = t.steps;
      g.n_forced = t.n_forced;
      g.y_first = t.y_first;
      if (gl1d_pack_wanted<R>(op, t.kg)) {
        cudaError_t e = gl1d_build_packs<R>(op, t.kg);
        if (e != cudaSuccess) return e;
        return launch_gl1d_pack<R>(g, (const int32_t*)op->pack_map, op->pack_count, op->pack_ppt, state, F, Y,
                                   op->d_flag, op->stream);
      }
      if (sizeof(R) == 8) op->gl_cluster = gl1d_cluster_size(g);
      return launch_gl1d_tile<R>(g, state, F, Y, norms, op->d_flag, op->stream);
    }
    case RSV_OP_DENSE: {
      const size_t half = (size_t)t.kg * op->n * sizeof(cpx<R>);
      char* buf = static_cast<char*>(state);
      cudaError_t e = cudaSuccess;
      if (sizeof(R) == 4 && dense_tc_supported(op, t.kg) && op->tc_persistent) {
        e = dense_tc_march_tile(op, t.kg, t.adjoint, t.n0, t.steps, t.n_forced, t.y_first, buf, F, Y, buf + 2 * half);
        if (e == cudaSuccess)
          e = check_finite(op, buf + (size_t)((t.n0 + t.steps) & 1) * half, (int64_t)t.kg * op->n, false);
        return e;
      }
      for (int s = 0; s < t.steps && e == cudaSuccess; ++s) {
        const int64_t n = t.n0 + s;
        const bool forced = F != nullptr && n < t.n_forced;
        void* uin = buf + (size_t)(n & 1) * half;
        void* uout = buf + (size_t)((n + 1) & 1) * half;
        const void* f = forced ? static_cast<const char*>(F) + (size_t)s * half : nullptr;
        void* y = (Y != nullptr && s >= t.y_first) ? static_cast<char*>(Y) + (size_t)s * half : nullptr;
        if (sizeof(R) == 4 && dense_tc_supported(op, t.kg))
          e = dense_tc_step(op, t.kg, t.adjoint, n, uin, uout, f, y, buf + 2 * half);
        else
          e = dense_step<R>(op, t.kg, t.adjoint, uin, uout, f, y);
      }
      if (e == cudaSuccess) e = check_finite(op, buf + (size_t)((t.n0 + t.steps) & 1) * half, (int64_t)t.kg * op->n, false);
      return e;
    }
    case RSV_OP_ADR2D:
    case RSV_OP_ADV3D:
      return stencil_march_tile<R>(op, t, state, F, Y);
    default:
      return cudaErrorNotSupported;
  }
}

// ---------------------------------------------------------------------------
// CUDA graphs of a time tile's launch sequence (structured-grid kinds: two to four launches per
// step).  What a tile launches depends on the tile only through tile-relative quantities: the step
// count, how many of its steps are forced, which steps store snapshots, the vector group and the
// workspace pointers.  So the tile is described relative to its first step (n0 = 0, n_forced = the
// forced steps of the tile), and a sequence met a second time is captured once into a graph on a
// private stream and replayed on the operator's stream from then on.  The first meeting runs the
// launches directly (one-time set-up such as shared-memory opt-ins stays outside any capture).  A
// capture that fails falls back to direct launches for that sequence.  RSV_TILE_GRAPHS=0 disables.
// ---------------------------------------------------------------------------
static bool tile_graphs_enabled(rsv_operator op) {
  static const bool env = [] {
    const char* e = getenv("RSV_TILE_GRAPHS");
    return !(e != nullptr && e[0] == '0');
  }();
  return env && (op->kind == RSV_OP_ADR2D || op->kind == RSV_OP_ADV3D);
}

template <typename R>
cudaError_t march_tile(rsv_operator op, const MarchTile& t, void* state, const void* F, void* Y, double* norms) {
  if (!tile_graphs_enabled(op)) return march_tile_direct<R>(op, t, state, F, Y, norms);
  MarchTile rel = t;
  rel.n0 = 0;
  rel.n_forced = F != nullptr ? std::max<int64_t>(0, std::min<int64_t>(t.steps, t.n_forced - t.n0)) : 0;
  const void* Fk = rel.n_forced > 0 ? F : nullptr;
  TileGraphKey key{sizeof(R), rel.steps, (int)rel.n_forced, Y != nullptr ? rel.y_first : -1, rel.kg,
                   rel.adjoint, state, Fk, Y, norms};
  TileGraph* hit = nullptr;
  for (TileGraph& g : op->tile_graphs)
    if (g.key == key) hit = &g;
  if (hit == nullptr) {
    if (op->tile_graphs.size() >= 8) {   // bounded cache: drop the oldest sequence
      if (op->tile_graphs.front().exec) cudaGraphExecDestroy(op->tile_graphs.front().exec);
      op->tile_graphs.erase(op->tile_graphs.begin());
    }
    op->tile_graphs.push_back(TileGraph{key, nullptr, 1, false});
    return march_tile_direct<R>(op, rel, state, Fk, Y, norms);
  }
  if (hit->exec == nullptr && !hit->failed) {
    if (op->cap_stream == nullptr && cudaStreamCreateWithFlags(&op->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      hit->failed = true;
    } else {
      const cudaStream_t orig = op->stream;
      op->stream = op->cap_stream;
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamBeginCapture(op->cap_stream, cudaStreamCaptureModeRelaxed);
      if (e == cudaSuccess) {
        const cudaError_t el = march_tile_direct<R>(op, rel, state, Fk, Y, norms);
        e = cudaStreamEndCapture(op->cap_stream, &graph);
        if (e == cudaSuccess) e = el;
      }
      op->stream = orig;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&hit->exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        cudaGetLastError();
        hit->exec = nullptr;
        hit->failed = true;
      }
    }
  }
  if (hit->exec == nullptr) return march_tile_direct<R>(op, rel, state, Fk, Y, norms);
  op->graph_replays += 1;
  return cudaGraphLaunch(hit->exec, op->stream);
}

template <typename R>
cudaError_t apply_op(rsv_operator op, const void* x, int k, bool adjoint, void* y) {
  switch (op->kind) {
    case RSV_OP_GL1D: {
      Gl1dTile g = gl1d_geom(op, adjoint, k);
      return launch_gl1d_apply<R>(g, (const int32_t*)op->d_inst_of_point, x, y, op->stream);
    }
    case RSV_OP_DENSE:
      return dense_apply<R>(op, x, k, adjoint, y);
    case RSV_OP_ADR2D:
    case RSV_OP_ADV3D:
      return stencil_apply<R>(op, x, k, adjoint, y);
    default:
      return cudaErrorNotSupported;
  }
}

template cudaError_t march_tile<double>(rsv_operator, const MarchTile&, void*, const void*, void*, double*);
template cudaError_t march_tile<float>(rsv_operator, const MarchTile&, void*, const void*, void*, double*);
template rsv_status prepare_coefficients<double>(rsv_operator, const void*, int64_t, int, bool, const void**,
                                                 int64_t*, int*);
template rsv_status prepare_coefficients<float>(rsv_operator, const void*, int64_t, int, bool, const void**,
                                                int64_t*, int*);
template cudaError_t apply_op<double>(rsv_operator, const void*, int, bool, void*);
template cudaError_t apply_op<float>(rsv_operator, const void*, int, bool, void*);

}  // namespace rsv
