// Transient-response method in time-series form (Sec. 2.2 with App. B and C):
// runs driven by a sampled series, Fourier transforms of series at arbitrary
// frequencies, FIR filtering, the FIR design, and the TRM power iteration.
//
// A series-driven run reuses the march's tile machinery: per time tile of S
// steps, series_forcing_kernel fills the forcing tile F[2S + 1][rows] at the
// half steps of the tile from the App. C interpolant of the input series, the
// operator's march kernels advance the state and store every step's starting
// state in the snapshot tile, and series_record_kernel copies every `every`-th
// of them into the output series together with its squared norm per vector.
// The host reads those norms once per tile to apply the truncation rule.
#include <algorithm>
#include <cmath>
#include <vector>

#include "rsv_ops.h"

namespace rsv {

size_t state_elem_bytes(rsv_operator op);

namespace {

template <typename R>
__device__ __forceinline__ double sq(R x) {
  return (double)x * (double)x;
}
template <typename R>
__device__ __forceinline__ double sq(cpx<R> x) {
  return (double)x.re * (double)x.re + (double)x.im * (double)x.im;
}
template <typename T>
__device__ __forceinline__ T zero_of();
template <>
__device__ __forceinline__ float zero_of<float>() { return 0.f; }
template <>
__device__ __forceinline__ double zero_of<double>() { return 0.0; }
template <>
__device__ __forceinline__ cpx<float> zero_of<cpx<float>>() { return mk<float>(0.f, 0.f); }
template <>
__device__ __forceinline__ cpx<double> zero_of<cpx<double>>() { return mk<double>(0.0, 0.0); }

template <typename R>
__device__ __forceinline__ R add(R a, R b) { return a + b; }
template <typename R>
__device__ __forceinline__ cpx<R> add(cpx<R> a, cpx<R> b) { return a + b; }
template <typename R>
__device__ __forceinline__ R scl(R s, R a) { return s * a; }
template <typename R>
__device__ __forceinline__ cpx<R> scl(R s, cpx<R> a) { return s * a; }

// ---------------------------------------------------------------------------
// Forcing tile from a sampled series (App. C)
// ---------------------------------------------------------------------------
// Sample i of the series in run order (reversed storage when rev).
template <typename T>
__device__ __forceinline__ T sample(const T* src, int64_t stride, int64_t n_in, int rev, int64_t i, int64_t r) {
  const int64_t p = rev ? n_in - 1 - i : i;
  return src[p * stride + r];
}

// Unit-spacing first (v) and second (a) derivative estimates at sample i (App. C):
// C1  second-order central differences, first-order one-sided at the two ends;
// C2  5-point centred differences; next to the ends second-order central ones;
//     at the ends first-order one-sided first derivative and zero second derivative.
template <typename T, typename R>
__device__ void derivs(const T* src, int64_t stride, int64_t n_in, int rev, int64_t i, int64_t r, int kind, T* v,
                       T* a) {
  const T z = zero_of<T>();
  *a = z;
  if (i == 0 || i == n_in - 1) {
    const T x0 = sample(src, stride, n_in, rev, i == 0 ? 0 : n_in - 2, r);
    const T x1 = sample(src, stride, n_in, rev, i == 0 ? 1 : n_in - 1, r);
    *v = add(x1, scl(R(-1), x0));
    return;
  }
  const T xm = sample(src, stride, n_in, rev, i - 1, r);
  const T xp = sample(src, stride, n_in, rev, i + 1, r);
  if (kind == 1 || i == 1 || i == n_in - 2) {
    *v = scl(R(0.5), add(xp, scl(R(-1), xm)));
    if (kind == 2) {
      const T x0 = sample(src, stride, n_in, rev, i, r);
      *a = add(add(xp, xm), scl(R(-2), x0));
    }
    return;
  }
  const T xmm = sample(src, stride, n_in, rev, i - 2, r);
  const T xpp = sample(src, stride, n_in, rev, i + 2, r);
  const T x0 = sample(src, stride, n_in, rev, i, r);
  const R c12 = R(1) / R(12);
  *v = scl(c12, add(add(xmm, scl(R(-8), xm)), add(scl(R(8), xp), scl(R(-1), xpp))));
  *a = scl(c12, add(add(scl(R(-1), xmm), scl(R(16), xm)), add(add(scl(R(-30), x0), scl(R(16), xp)), scl(R(-1), xpp))));
}

// F[tau][r] = g(t) at t = (q0 + tau) h / 2: the interpolant on the interval of the sample
// spacing d = every h that holds t, the last sample at its own time, zero after it.
template <typename T, typename R>
__global__ void series_forcing_kernel(const T* __restrict__ src, int64_t stride, int64_t n_in, int rev, int every,
                                      int kind, int64_t q0, int n_tau, int64_t rows, T* __restrict__ F) {
  const int64_t total = (int64_t)n_tau * rows;
  const int64_t span = 2 * (int64_t)every;
  const int64_t q_end = span * (n_in - 1);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t tau = idx / rows;
    const int64_t r = idx - tau * rows;
    const int64_t q = q0 + tau;
    T out = zero_of<T>();
    if (q < q_end) {
      const int64_t i = q / span;
      const R s = R(q - i * span) / R(span);
      const T x0 = sample(src, stride, n_in, rev, i, r);
      const T x1 = sample(src, stride, n_in, rev, i + 1, r);
      if (kind == 0) {
        out = add(scl(R(1) - s, x0), scl(s, x1));
      } else {
        T v0, v1, a0, a1;
        derivs<T, R>(src, stride, n_in, rev, i, r, kind, &v0, &a0);
        derivs<T, R>(src, stride, n_in, rev, i + 1, r, kind, &v1, &a1);
        const R s2 = s * s, s3 = s2 * s;
        if (kind == 1) {   // cubic Hermite: values and first derivatives at both ends
          const R h00 = R(2) * s3 - R(3) * s2 + R(1), h10 = s3 - R(2) * s2 + s;
          const R h01 = R(-2) * s3 + R(3) * s2, h11 = s3 - s2;
          out = add(add(scl(h00, x0), scl(h10, v0)), add(scl(h01, x1), scl(h11, v1)));
        } else {           // quintic Hermite: values, first and second derivatives at both ends
          const R s4 = s3 * s, s5 = s4 * s;
          const R b0 = R(1) - R(10) * s3 + R(15) * s4 - R(6) * s5;
          const R b1 = s - R(6) * s3 + R(8) * s4 - R(3) * s5;
          const R b2 = R(0.5) * s2 - R(1.5) * s3 + R(1.5) * s4 - R(0.5) * s5;
          const R b5 = R(10) * s3 - R(15) * s4 + R(6) * s5;
          const R b4 = R(-4) * s3 + R(7) * s4 - R(3) * s5;
          const R b3 = R(0.5) * s3 - s4 + R(0.5) * s5;
          out = add(add(add(scl(b0, x0), scl(b1, v0)), scl(b2, a0)), add(add(scl(b5, x1), scl(b4, v1)), scl(b3, a1)));
        }
      }
    } else if (q == q_end) {
      out = sample(src, stride, n_in, rev, n_in - 1, r);
    }
    F[idx] = out;
  }
}

// ---------------------------------------------------------------------------
// Recording snapshots: out[j][v][p] = Y[j every - n0][v][p] for j in [j0, j0 + n_j), with
// nrm[(j - j0) kv + v] += |.|^2 (nrm zeroed by the caller).  Block (x: points, y: (j, v)).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void series_record_kernel(const T* __restrict__ Y, int64_t rows, int64_t n, int kv, int64_t j0,
                                     int every, int64_t n0, T* __restrict__ out, int64_t out_stride,
                                     double* __restrict__ nrm) {
  const int64_t jj = blockIdx.y / kv;
  const int v = blockIdx.y - (int)jj * kv;
  const int64_t j = j0 + jj;
  const T* src = Y + (j * every - n0) * rows + (int64_t)v * n;
  T* dst = out + j * out_stride + (int64_t)v * n;
  double acc = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const T x = src[p];
    dst[p] = x;
    acc += sq(x);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    atomicAdd(nrm + jj * kv + v, t);
  }
}

// ---------------------------------------------------------------------------
// Fourier transform at arbitrary frequencies: out[j][c] = d sum_i E[i][j] x[i][c], E from the host
// (exp(-i w_j (t0 + i d)) in FP64).  Thread per column c, 8 frequencies per block row.
// ---------------------------------------------------------------------------
constexpr int kFw = 8;     // frequencies per block
constexpr int kFi = 64;    // snapshots per shared-memory chunk of E

template <typename R>
__device__ __forceinline__ cpx<double> to_c64(R x) { return mk<double>((double)x, 0.0); }
template <typename R>
__device__ __forceinline__ cpx<double> to_c64(cpx<R> x) { return mk<double>((double)x.re, (double)x.im); }

template <typename T, typename O>
__global__ void series_fourier_kernel(const T* __restrict__ x, int64_t n_snap, int64_t cols,
                                      const cpx<double>* __restrict__ E, int n_omega, double d, O* __restrict__ out) {
  __shared__ cpx<double> e_s[kFi][kFw];
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int j0 = blockIdx.y * kFw;
  const int nj = min(kFw, n_omega - j0);
  cpx<double> acc[kFw];
#pragma unroll
  for (int q = 0; q < kFw; ++q) acc[q] = mk<double>(0.0, 0.0);
  for (int64_t i0 = 0; i0 < n_snap; i0 += kFi) {
    const int ni = (int)(n_snap - i0 < kFi ? n_snap - i0 : kFi);
    __syncthreads();
    for (int t = threadIdx.x; t < kFi * kFw; t += blockDim.x) {
      const int ii = t / kFw, q = t - (t / kFw) * kFw;
      e_s[ii][q] = (ii < ni && q < nj) ? E[(i0 + ii) * n_omega + j0 + q] : mk<double>(0.0, 0.0);
    }
    __syncthreads();
    if (c < cols) {
      for (int ii = 0; ii < ni; ++ii) {
        const cpx<double> xv = to_c64(x[(i0 + ii) * cols + c]);
#pragma unroll
        for (int q = 0; q < kFw; ++q) cfma(acc[q], e_s[ii][q], xv);
      }
    }
  }
  if (c < cols) {
    for (int q = 0; q < nj; ++q) {
      O o;
      o.re = (decltype(o.re))(d * acc[q].re);
      o.im = (decltype(o.im))(d * acc[q].im);
      out[(int64_t)(j0 + q) * cols + c] = o;
    }
  }
}

// ---------------------------------------------------------------------------
// FIR filter, whole convolution: out[m][v][p] = sum_j phi_v[j] x[m - j][v][p].  Each thread owns
// kFm consecutive outputs of one point and reads each input it needs once.
// ---------------------------------------------------------------------------
constexpr int kFm = 16;

template <typename R>
__device__ __forceinline__ void mac(R& acc, R c, R x) { acc = fma(c, x, acc); }
template <typename R>
__device__ __forceinline__ void mac(cpx<R>& acc, cpx<R> c, cpx<R> x) { cfma(acc, c, x); }

template <typename T>
__global__ void series_fir_kernel(const T* __restrict__ x, int64_t n_in, int64_t cols, int64_t n, int64_t p_blocks,
                                  const T* __restrict__ taps, int order, int rev_taps, T* __restrict__ out) {
  const int64_t mb = blockIdx.x / p_blocks;
  const int64_t p = (blockIdx.x - mb * p_blocks) * (int64_t)blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  const int64_t m0 = mb * kFm;
  const int64_t n_out = n_in + order;
  if (p >= n) return;
  const int64_t c = (int64_t)v * n + p;
  const T* tv = taps + (int64_t)v * (order + 1);
  T acc[kFm];
#pragma unroll
  for (int u = 0; u < kFm; ++u) acc[u] = zero_of<T>();
  const int64_t i_lo = m0 - order > 0 ? m0 - order : 0;
  const int64_t i_hi = (n_in - 1 < m0 + kFm - 1) ? n_in - 1 : m0 + kFm - 1;
  for (int64_t i = i_lo; i <= i_hi; ++i) {
    const T xi = x[i * cols + c];
#pragma unroll
    for (int u = 0; u < kFm; ++u) {
      const int64_t j = m0 + u - i;
      if (j >= 0 && j <= order) mac(acc[u], tv[rev_taps ? order - j : j], xi);
    }
  }
#pragma unroll
  for (int u = 0; u < kFm; ++u)
    if (m0 + u < n_out) out[(m0 + u) * cols + c] = acc[u];
}

// Squared norms of rows of a complex FP64 block: out[row] = sum_p |X[row][p]|^2.
__global__ void row_sq_norms_kernel(const cpx<double>* __restrict__ X, int64_t len, double* __restrict__ out) {
  const cpx<double>* x = X + blockIdx.x * len;
  double acc = 0.0;
  for (int64_t p = threadIdx.x; p < len; p += blockDim.x) acc += x[p].re * x[p].re + x[p].im * x[p].im;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    out[blockIdx.x] = t;
  }
}

// x[i][v][p] *= s[v] for the n_snap snapshots of a series (out of place).
template <typename T, typename R>
__global__ void scale_vectors_kernel(const T* __restrict__ x, int64_t total, int64_t n, int k,
                                     const double* __restrict__ s, T* __restrict__ y) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int v = (int)((idx / n) % k);
    y[idx] = scl((R)s[v], x[idx]);
  }
}

// Records snapshots [j0, j0 + nj) (see series_record_kernel), in launches of at most 65535 (j, v) rows.
template <typename T>
cudaError_t launch_record(const T* Y, int64_t rows, int64_t n, int kv, int64_t j0, int64_t nj, int every, int64_t n0,
                          T* out, int64_t out_stride, double* nrm, cudaStream_t st) {
  const int thr = 256;
  const int gx = std::max(1, std::min<int>((int)((n + thr - 1) / thr), 64));
  const int64_t per = std::max<int64_t>(1, 65535 / kv);
  for (int64_t a = 0; a < nj; a += per) {
    const int64_t c = std::min(per, nj - a);
    dim3 grid(gx, (unsigned)(c * kv));
    series_record_kernel<T><<<grid, thr, 0, st>>>(Y, rows, n, kv, j0 + a, every, n0, out, out_stride, nrm + a * kv);
  }
  return cudaGetLastError();
}

int grid_for(int64_t work, int threads, int sms) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, (int64_t)sms * 16));
}

// ---------------------------------------------------------------------------
// host parts
// ---------------------------------------------------------------------------
rsv_status series_check(rsv_operator op) {
  if (!op) return fail(RSV_ERR_INVALID_ARG, "null operator");
  if (!op->have_freq) return fail(RSV_ERR_STATE, "rsv_set_frequencies must come first (it sets the step h)");
  if (op->kind == RSV_OP_DENSE)
    return fail(RSV_ERR_INVALID_ARG, "series-driven runs serve the GL1D, ADR2D and ADV3D kinds, not the dense kind");
  if (op->bf16_state) return fail(RSV_ERR_INVALID_ARG, "series-driven runs need FP32 or FP64 state");
  if (op->have_weights) return fail(RSV_ERR_INVALID_ARG, "series-driven runs take no weights (B = C = W = I)");
  return RSV_OK;
}

template <typename R, typename T>
rsv_status series_march_impl(rsv_operator op, bool adjoint, int k, const void* init, const void* forcing,
                             int64_t n_in, bool reverse_in, const rsv_series_opts& o, void* out, int64_t n_out_max,
                             int64_t* n_out, int64_t* stops) {
  const int64_t n = op->n;
  const size_t se = sizeof(T);
  const cudaStream_t st = op->stream;
  const int every = o.every;
  cudaError_t e;
  rsv_status s;
  // tile and group: the march's default tile, vectors halved until the tiles fit in 90% of free memory
  int S = default_tile_steps(op);
  int kg = k;
  {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      free_b = (size_t)1 << 62;
    }
    const size_t held = op->ws_state.bytes + op->ws_ftile.bytes + op->ws_ysnap.bytes;
    const double budget = 0.9 * (double)(free_b + held);
    auto need = [&](int s_, int kg_) {
      const double rows_ = (double)kg_ * n;
      return rows_ * se + (double)stage_scratch_bytes(op, kg_) + (3.0 * s_ + 1) * rows_ * se;
    };
    while (need(S, kg) > budget && (S > 16 || kg > 1)) {
      if (kg > 1)
        kg = (kg + 1) / 2;
      else
        S = std::max(16, S / 2);
    }
  }
  const int64_t rows_max = (int64_t)kg * n;
  const int64_t snaps_per_tile = S / every + 2;
  if ((s = ensure(op->ws_state, rows_max * se + stage_scratch_bytes(op, kg))) != RSV_OK) return s;
  if ((s = ensure(op->ws_ftile, (size_t)(2 * S + 1) * rows_max * se)) != RSV_OK) return s;
  if ((s = ensure(op->ws_ysnap, (size_t)S * rows_max * se)) != RSV_OK) return s;
  // norms: the recorded snapshots' [snaps_per_tile][kg], then the march kernels' own [kg][n_inst]
  if ((s = ensure(op->ws_norm, ((size_t)snaps_per_tile * kg + (size_t)kg * op->n_inst) * sizeof(double))) != RSV_OK)
    return s;
  if ((e = cudaMemsetAsync(op->d_flag, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(e, "flag reset");
  const bool truncate = o.tail_tol > 0.0;
  const int64_t j_end = std::max<int64_t>(n_in - 1, 0);   // first snapshot at or after the end of the forcing
  const int64_t q_end = forcing ? 2 * (int64_t)every * (n_in - 1) : -1;
  const int64_t out_stride = (int64_t)k * n;
  int64_t n_total = 0;
  std::vector<int64_t> stop_all(k, -1);
  std::vector<double> h_nrm;
  double* d_nrm = static_cast<double*>(op->ws_norm.ptr);
  T* outp = static_cast<T*>(out);
  const int thr = 256;
  for (int v0 = 0; v0 < k; v0 += kg) {
    const int kv = std::min(kg, k - v0);
    const int64_t rows = (int64_t)kv * n;
    T* out_g = outp + (int64_t)v0 * n;
    e = cudaMemsetAsync(op->ws_state.ptr, 0, rows * se + stage_scratch_bytes(op, kv), st);
    if (e == cudaSuccess && init)
      e = cudaMemcpyAsync(op->ws_state.ptr, static_cast<const T*>(init) + (int64_t)v0 * n, rows * se,
                          cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "series run reset");
    std::vector<double> peak(kv, 0.0);
    std::vector<int64_t> stop(kv, -1);
    int n_stopped = 0;
    int64_t recorded = 0;   // snapshots written so far
    // decides on snapshots [j0, j0 + nj) whose squared norms are in h_nrm
    auto decide = [&](int64_t j0, int64_t nj) {
      for (int64_t jj = 0; jj < nj && !(truncate && n_stopped == kv); ++jj) {
        const int64_t j = j0 + jj;
        recorded = j + 1;
        for (int v = 0; v < kv; ++v) {
          if (stop[v] >= 0) continue;
          const double r = std::sqrt(h_nrm[jj * kv + v]);
          peak[v] = std::max(peak[v], r);
          if (truncate && j >= j_end && r <= o.tail_tol * peak[v]) {
            stop[v] = j;
            ++n_stopped;
          }
        }
      }
    };
    auto read_norms = [&](int64_t count) -> rsv_status {
      h_nrm.assign(count, 0.0);
      cudaError_t ee = cudaMemcpyAsync(h_nrm.data(), d_nrm, count * sizeof(double), cudaMemcpyDeviceToHost, st);
      if (ee == cudaSuccess) ee = cudaStreamSynchronize(st);
      return ee == cudaSuccess ? RSV_OK : cuda_fail(ee, "series norms");
    };
    // snapshot 0: the initial state
    {
      if ((e = cudaMemsetAsync(d_nrm, 0, kv * sizeof(double), st)) != cudaSuccess) return cuda_fail(e, "norms");
      e = launch_record<T>(static_cast<const T*>(op->ws_state.ptr), rows, n, kv, 0, 1, 1, 0, out_g, out_stride, d_nrm,
                           st);
      if (e != cudaSuccess) return cuda_fail(e, "series record");
      if ((s = read_norms(kv)) != RSV_OK) return s;
      decide(0, 1);
    }
    for (int64_t n0 = 0; recorded < n_out_max && !(truncate && n_stopped == kv); n0 += S) {
      // steps of this tile: up to the one that records the last allowed snapshot
      const int64_t last_step = (n_out_max - 1) * (int64_t)every;   // step index of snapshot n_out_max - 1
      const int steps = (int)std::min<int64_t>(S, last_step - n0);
      if (steps <= 0) break;
      const bool forced = forcing != nullptr && 2 * n0 <= q_end;
      if (forced) {
        ProfScope ps(op, PROF_SYNTH);
        const int n_tau = 2 * steps + 1;
        series_forcing_kernel<T, R><<<grid_for((int64_t)n_tau * rows, thr, op->sm_count), thr, 0, st>>>(
            static_cast<const T*>(forcing) + (int64_t)v0 * n, out_stride, n_in, reverse_in ? 1 : 0, every, o.interp,
            2 * n0, n_tau, rows, static_cast<T*>(op->ws_ftile.ptr));
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "series forcing");
      }
      MarchTile mt;
      mt.n0 = n0;
      mt.steps = steps;
      mt.n_forced = forced ? n0 + steps : 0;
      mt.y_first = 0;
      mt.kg = kv;
      mt.adjoint = adjoint;
      {
        ProfScope ps(op, PROF_MARCH, march_tile_kernels(op, steps, kv));
        e = march_tile<R>(op, mt, op->ws_state.ptr, forced ? op->ws_ftile.ptr : nullptr, op->ws_ysnap.ptr,
                          static_cast<double*>(op->ws_norm.ptr) + snaps_per_tile * kg);
      }
      if (e != cudaSuccess) return cuda_fail(e, "series march tile");
      // snapshots whose step lies in (n0, n0 + steps]: steps n0 + 1 .. n0 + steps - 1 are in the tile's
      // snapshot store; step n0 + steps is the state after the tile
      const int64_t j_lo = n0 / every + 1;
      const int64_t j_hi = std::min<int64_t>((n0 + steps) / every, n_out_max - 1);   // inclusive
      if (j_hi < j_lo) continue;
      const int64_t nj = j_hi - j_lo + 1;
      if ((e = cudaMemsetAsync(d_nrm, 0, nj * kv * sizeof(double), st)) != cudaSuccess) return cuda_fail(e, "norms");
      const bool last_is_end = j_hi * every == n0 + steps;
      const int64_t nj_in = last_is_end ? nj - 1 : nj;
      e = cudaSuccess;
      if (nj_in > 0)
        e = launch_record<T>(static_cast<const T*>(op->ws_ysnap.ptr), rows, n, kv, j_lo, nj_in, every, n0, out_g,
                             out_stride, d_nrm, st);
      if (e == cudaSuccess && last_is_end)
        e = launch_record<T>(static_cast<const T*>(op->ws_state.ptr), rows, n, kv, 0, 1, 1, 0,
                             out_g + j_hi * out_stride, out_stride, d_nrm + (nj - 1) * kv, st);
      if (e != cudaSuccess) return cuda_fail(e, "series record");
      if ((s = read_norms(nj * kv)) != RSV_OK) return s;
      decide(j_lo, nj);
    }
    // this group's record length, and each stopped vector's later snapshots zeroed up to it
    for (int v = 0; v < kv; ++v) stop_all[v0 + v] = stop[v];
    n_total = std::max(n_total, (truncate && n_stopped == kv) ? recorded : std::min<int64_t>(recorded, n_out_max));
  }
  // common length: the longest group; zero what lies beyond each vector's stop (or its group's end)
  for (int v = 0; v < k; ++v) {
    const int64_t first_zero = stop_all[v] >= 0 ? stop_all[v] + 1 : n_total;
    if (first_zero < n_total) {
      e = cudaMemset2DAsync(outp + first_zero * out_stride + (int64_t)v * n, out_stride * se, 0, n * se,
                            n_total - first_zero, st);
      if (e != cudaSuccess) return cuda_fail(e, "series zero fill");
    }
  }
  int flag = 0;
  e = cudaMemcpyAsync(&flag, op->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "series run");
  if (flag) return fail(RSV_ERR_DIVERGED, "state norm became non-finite during the series-driven run");
  *n_out = n_total;
  if (stops)
    for (int v = 0; v < k; ++v) stops[v] = stop_all[v];
  op->last_tile = S;
  op->last_group = kg;
  return RSV_OK;
}

rsv_status series_march_any(rsv_operator op, bool adjoint, int k, const void* init, const void* forcing,
                            int64_t n_in, bool reverse_in, const rsv_series_opts& o, void* out, int64_t n_out_max,
                            int64_t* n_out, int64_t* stops) {
  rsv_status s = series_check(op);
  if (s != RSV_OK) return s;
  if (k < 1 || k > 65535 || !out || !n_out || n_out_max < 1 || o.every < 1 || o.interp < 0 || o.interp > 2 ||
      !(o.tail_tol >= 0.0))
    return fail(RSV_ERR_INVALID_ARG, "bad series run arguments");
  if (forcing && n_in < 1) return fail(RSV_ERR_INVALID_ARG, "a forcing series needs at least one sample");
  if (forcing && forcing == out) return fail(RSV_ERR_INVALID_ARG, "forcing and output series must not alias");
  if (!forcing) n_in = 0;
  if (op->scheme == RSV_SCHEME_CN && op->kind != RSV_OP_GL1D)
    return fail(RSV_ERR_INVALID_ARG, "Crank-Nicolson serves the GL1D kind only");
  if (op->prec == RSV_PREC_FP64)
    return op->real_state ? series_march_impl<double, double>(op, adjoint, k, init, forcing, n_in, reverse_in, o, out,
                                                              n_out_max, n_out, stops)
                          : series_march_impl<double, cpx<double>>(op, adjoint, k, init, forcing, n_in, reverse_in,
                                                                   o, out, n_out_max, n_out, stops);
  return op->real_state ? series_march_impl<float, float>(op, adjoint, k, init, forcing, n_in, reverse_in, o, out,
                                                          n_out_max, n_out, stops)
                        : series_march_impl<float, cpx<float>>(op, adjoint, k, init, forcing, n_in, reverse_in, o,
                                                               out, n_out_max, n_out, stops);
}

// Fourier transform into an FP64 (internal) or element-type (ABI) complex block.
template <typename T, typename O>
rsv_status fourier_impl(rsv_operator op, const void* series, int64_t n_snap, int k, double d, double t0,
                        const double* omega, int n_omega, O* out) {
  const int64_t cols = (int64_t)k * op->n;
  std::vector<cpx<double>> e_host((size_t)n_snap * n_omega);
  for (int64_t i = 0; i < n_snap; ++i)
    for (int j = 0; j < n_omega; ++j) {
      const double ph = -omega[j] * (t0 + (double)i * d);
      e_host[(size_t)i * n_omega + j] = mk<double>(std::cos(ph), std::sin(ph));
    }
  rsv_status s = ensure(op->ws_ser_e, e_host.size() * sizeof(cpx<double>));
  if (s != RSV_OK) return s;
  cudaError_t e = cudaMemcpyAsync(op->ws_ser_e.ptr, e_host.data(), e_host.size() * sizeof(cpx<double>),
                                  cudaMemcpyHostToDevice, op->stream);
  if (e != cudaSuccess) return cuda_fail(e, "series Fourier table");
  {
    ProfScope ps(op, PROF_ANALYSIS);
    const int thr = 128;
    dim3 grid((unsigned)((cols + thr - 1) / thr), (unsigned)((n_omega + kFw - 1) / kFw));
    series_fourier_kernel<T, O><<<grid, thr, 0, op->stream>>>(static_cast<const T*>(series), n_snap, cols,
                                                              static_cast<const cpx<double>*>(op->ws_ser_e.ptr),
                                                              n_omega, d, out);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "series Fourier");
  }
  // the host table must outlive the copy
  if ((e = cudaStreamSynchronize(op->stream)) != cudaSuccess) return cuda_fail(e, "series Fourier");
  return RSV_OK;
}

template <typename T>
rsv_status filter_impl(rsv_operator op, const void* in, int64_t n_in, int k, const std::vector<T>& taps, int order,
                       bool rev_taps, void* out) {
  const size_t bytes = taps.size() * sizeof(T);
  rsv_status s = ensure(op->ws_ser_t, bytes);
  if (s != RSV_OK) return s;
  cudaError_t e = cudaMemcpyAsync(op->ws_ser_t.ptr, taps.data(), bytes, cudaMemcpyHostToDevice, op->stream);
  if (e != cudaSuccess) return cuda_fail(e, "filter taps");
  {
    ProfScope ps(op, PROF_GLUE);
    const int thr = 128;
    const int64_t n_out = n_in + order;
    const int64_t pb = (op->n + thr - 1) / thr, mbk = (n_out + kFm - 1) / kFm;
    if (pb * mbk > 0x7fffffffLL) return fail(RSV_ERR_INVALID_ARG, "series too long for one filter launch");
    dim3 grid((unsigned)(pb * mbk), (unsigned)k);
    series_fir_kernel<T><<<grid, thr, 0, op->stream>>>(static_cast<const T*>(in), n_in, (int64_t)k * op->n, op->n, pb,
                                                       static_cast<const T*>(op->ws_ser_t.ptr), order,
                                                       rev_taps ? 1 : 0, static_cast<T*>(out));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "series filter");
  }
  if ((e = cudaStreamSynchronize(op->stream)) != cudaSuccess) return cuda_fail(e, "series filter");
  return RSV_OK;
}

template <typename R>
void taps_to(const double* taps, int k, int order, std::vector<R>* v) {
  v->resize((size_t)k * (order + 1));
  for (size_t i = 0; i < v->size(); ++i) (*v)[i] = (R)taps[2 * i];
}
template <typename R>
void taps_to(const double* taps, int k, int order, std::vector<cpx<R>>* v) {
  v->resize((size_t)k * (order + 1));
  for (size_t i = 0; i < v->size(); ++i) (*v)[i] = mk<R>((R)taps[2 * i], (R)taps[2 * i + 1]);
}

rsv_status filter_any(rsv_operator op, const void* in, int64_t n_in, int k, const double* taps, int order,
                      bool rev_taps, void* out) {
  if (!op || !in || !out || !taps || k < 1 || n_in < 1 || order < 0 || in == out)
    return fail(RSV_ERR_INVALID_ARG, "bad filter arguments");
  if ((int64_t)k > 65535) return fail(RSV_ERR_INVALID_ARG, "at most 65535 vectors per filter call");
  if (op->real_state)
    for (int64_t i = 0; i < (int64_t)k * (order + 1); ++i)
      if (taps[2 * i + 1] != 0.0) return fail(RSV_ERR_INVALID_ARG, "a real-state series takes real taps");
  if (op->prec == RSV_PREC_FP64) {
    if (op->real_state) {
      std::vector<double> t;
      taps_to(taps, k, order, &t);
      return filter_impl<double>(op, in, n_in, k, t, order, rev_taps, out);
    }
    std::vector<cpx<double>> t;
    taps_to(taps, k, order, &t);
    return filter_impl<cpx<double>>(op, in, n_in, k, t, order, rev_taps, out);
  }
  if (op->real_state) {
    std::vector<float> t;
    taps_to(taps, k, order, &t);
    return filter_impl<float>(op, in, n_in, k, t, order, rev_taps, out);
  }
  std::vector<cpx<float>> t;
  taps_to(taps, k, order, &t);
  return filter_impl<cpx<float>>(op, in, n_in, k, t, order, rev_taps, out);
}

// Fourier transform of a series (state element type by the operator) into cpx<double> or cpx<R>.
template <typename O>
rsv_status fourier_any(rsv_operator op, const void* series, int64_t n_snap, int k, double d, double t0,
                       const double* omega, int n_omega, O* out) {
  if (op->prec == RSV_PREC_FP64)
    return op->real_state ? fourier_impl<double, O>(op, series, n_snap, k, d, t0, omega, n_omega, out)
                          : fourier_impl<cpx<double>, O>(op, series, n_snap, k, d, t0, omega, n_omega, out);
  return op->real_state ? fourier_impl<float, O>(op, series, n_snap, k, d, t0, omega, n_omega, out)
                        : fourier_impl<cpx<float>, O>(op, series, n_snap, k, d, t0, omega, n_omega, out);
}

// Linear interpolation with constant extension, on ascending points.
double interp_amp(double w, const double* xp, const double* fp, int n) {
  if (w <= xp[0]) return fp[0];
  if (w >= xp[n - 1]) return fp[n - 1];
  int lo = 0, hi = n - 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (xp[mid] <= w)
      lo = mid;
    else
      hi = mid;
  }
  const double t = (w - xp[lo]) / (xp[hi] - xp[lo]);
  return fp[lo] + t * (fp[hi] - fp[lo]);
}

}  // namespace

// Frequency-sampling design (host): taps[m] = hamming(m) (1/N) sum_q spec_q exp(2 pi i q m / N).
rsv_status fir_design_host(int order, double d, const double* w_pts, const double* amp, int n_pts, double* taps) {
  if (order < 0 || order % 2 || !(d > 0.0) || !w_pts || !amp || n_pts < 1 || !taps)
    return fail(RSV_ERR_INVALID_ARG, "bad filter design arguments (order must be even)");
  for (int i = 1; i < n_pts; ++i)
    if (!(w_pts[i] > w_pts[i - 1])) return fail(RSV_ERR_INVALID_ARG, "design frequencies must ascend");
  bool two_sided = false;
  for (int i = 0; i < n_pts; ++i) two_sided = two_sided || w_pts[i] < 0.0;
  const int ntap = order + 1;
  const int64_t nfft = 8 * (int64_t)ntap;
  const double pi = 3.14159265358979323846;
  const double dw = 2.0 * pi / ((double)nfft * d);
  std::vector<double> cs(nfft), sn(nfft);
  for (int64_t q = 0; q < nfft; ++q) {
    const double a = 2.0 * pi * (double)q / (double)nfft;
    cs[q] = std::cos(a);
    sn[q] = std::sin(a);
  }
  // spectrum on the signed grid: w_q = q dw (q <= N/2), (q - N) dw above; linear phase of order/2 samples
  std::vector<double> sr(nfft), si(nfft);
  for (int64_t q = 0; q < nfft; ++q) {
    const double w = (double)(q <= nfft / 2 ? q : q - nfft) * dw;
    const double a = interp_amp(two_sided ? w : std::fabs(w), w_pts, amp, n_pts);
    // exp(-i w order d / 2) = exp(-2 pi i q (order/2) / N): an exact table index
    const int64_t qq = (q * (order / 2)) % nfft;
    sr[q] = a * cs[qq];
    si[q] = -a * sn[qq];
  }
  for (int m = 0; m < ntap; ++m) {
    double re = 0.0, im = 0.0;
    for (int64_t q = 0; q < nfft; ++q) {
      const int64_t idx = (q * m) % nfft;
      re += sr[q] * cs[idx] - si[q] * sn[idx];
      im += sr[q] * sn[idx] + si[q] * cs[idx];
    }
    const double win = ntap > 1 ? 0.54 - 0.46 * std::cos(2.0 * pi * (double)m / (double)(ntap - 1)) : 1.0;
    taps[2 * m] = win * re / (double)nfft;
    taps[2 * m + 1] = two_sided ? win * im / (double)nfft : 0.0;
  }
  return RSV_OK;
}

namespace {

// TRM power iteration (see rsv_trm_power_iteration).
template <typename R, typename T>
rsv_status trm_impl(rsv_operator op, const void* f0, int k, const double* omega, int n_omega, const rsv_trm_opts& o,
                    double* gains, void* w_hat) {
  const int64_t n = op->n;
  const int64_t cols = (int64_t)k * n;
  const size_t se = sizeof(T);
  const double d = o.series.every * op->h;
  const int order = o.filter_order;
  const int64_t cap = o.n_snap_max;
  rsv_status s;
  if ((s = ensure(op->ws_ser_y, (size_t)cap * cols * se)) != RSV_OK) return s;
  if ((s = ensure(op->ws_ser_z, (size_t)cap * cols * se)) != RSV_OK) return s;
  if ((s = ensure(op->ws_ser_g, (size_t)(cap + order) * cols * se)) != RSV_OK) return s;
  if ((s = ensure(op->ws_ser_f, (size_t)n_omega * cols * sizeof(cpx<double>))) != RSV_OK) return s;
  if ((s = ensure(op->ws_ser_n, (size_t)n_omega * k * sizeof(double))) != RSV_OK) return s;
  T* y = static_cast<T*>(op->ws_ser_y.ptr);
  T* z = static_cast<T*>(op->ws_ser_z.ptr);
  T* g = static_cast<T*>(op->ws_ser_g.ptr);   // the next direct run's forcing, stored reversed in time
  cpx<double>* fh = static_cast<cpx<double>*>(op->ws_ser_f.ptr);
  const cudaStream_t st = op->stream;
  std::vector<double> nf((size_t)n_omega * k), nw((size_t)n_omega * k);
  // squared norms per (frequency, vector) of the FP64 block in fh
  auto norms = [&](std::vector<double>* dst) -> rsv_status {
    row_sq_norms_kernel<<<(unsigned)(n_omega * k), 256, 0, st>>>(fh, n, static_cast<double*>(op->ws_ser_n.ptr));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dst->data(), op->ws_ser_n.ptr, dst->size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? RSV_OK : cuda_fail(e, "TRM norms");
  };
  int64_t n_g = 0;   // samples of the stored (reversed) next forcing
  for (int it = 0; it < o.n_iter; ++it) {
    int64_t n_y = 0, n_z = 0;
    std::vector<int64_t> stops(k);
    if ((s = series_march_any(op, false, k, it == 0 ? f0 : nullptr, it == 0 ? nullptr : g, n_g, true, o.series, y,
                              cap, &n_y, stops.data())) != RSV_OK)
      return s;
    for (int v = 0; v < k; ++v)
      if (stops[v] < 0) return fail(RSV_ERR_INVALID_ARG, "a direct-run record filled n_snap_max before it was negligible");
    if ((s = series_march_any(op, true, k, nullptr, y, n_y, true, o.series, z, cap, &n_z, stops.data())) != RSV_OK)
      return s;
    for (int v = 0; v < k; ++v)
      if (stops[v] < 0)
        return fail(RSV_ERR_INVALID_ARG, "an adjoint-run record filled n_snap_max before it was negligible");
    // w[i] = z[n_z - 1 - i] at t_i = i d: w_hat(w) = d sum_m z[m] exp(+i w (m - n_z + 1) d)
    std::vector<double> neg(n_omega);
    for (int j = 0; j < n_omega; ++j) neg[j] = -omega[j];
    if ((s = fourier_any(op, z, n_z, k, d, -(double)(n_z - 1) * d, neg.data(), n_omega, fh)) != RSV_OK) return s;
    if ((s = norms(&nw)) != RSV_OK) return s;
    if (it == 0) {
      // the impulse's transform is f0 itself at every frequency
      std::vector<T> hf((size_t)cols);
      cudaError_t e = cudaMemcpyAsync(hf.data(), f0, cols * se, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "TRM start vector");
      for (int v = 0; v < k; ++v) {
        double acc = 0.0;
        for (int64_t p = 0; p < n; ++p) {
          const T x = hf[(size_t)v * n + p];
          if constexpr (sizeof(T) == sizeof(R))
            acc += (double)x * (double)x;
          else
            acc += (double)x.re * (double)x.re + (double)x.im * (double)x.im;
        }
        for (int j = 0; j < n_omega; ++j) nf[(size_t)j * k + v] = acc;
      }
    }
    for (int j = 0; j < n_omega; ++j)
      for (int v = 0; v < k; ++v)
        gains[((size_t)it * n_omega + j) * k + v] =
            std::sqrt(std::sqrt(nw[(size_t)j * k + v]) / std::sqrt(nf[(size_t)j * k + v]));
    if (it == o.n_iter - 1) {
      if (w_hat) {
        cudaError_t e = cudaSuccess;
        if (op->prec == RSV_PREC_FP64)
          e = cudaMemcpyAsync(w_hat, fh, (size_t)n_omega * cols * sizeof(cpx<double>), cudaMemcpyDeviceToDevice, st);
        else
          s = fourier_any(op, z, n_z, k, d, -(double)(n_z - 1) * d, neg.data(), n_omega, static_cast<cpx<float>*>(w_hat));
        if (e != cudaSuccess) return cuda_fail(e, "TRM w_hat");
        if (s != RSV_OK) return s;
      }
      break;
    }
    // next forcing g = filter(w) (or w scaled), stored reversed: reverse(phi * w) = reversed(phi) * z
    if (order > 0) {
      std::vector<int> idx(n_omega);
      for (int j = 0; j < n_omega; ++j) idx[j] = j;
      std::sort(idx.begin(), idx.end(), [&](int a, int b) { return omega[a] < omega[b]; });
      std::vector<double> wp(n_omega), ap(n_omega), taps((size_t)k * (order + 1) * 2);
      for (int v = 0; v < k; ++v) {
        for (int j = 0; j < n_omega; ++j) {
          wp[j] = omega[idx[j]];
          ap[j] = 1.0 / std::sqrt(nw[(size_t)idx[j] * k + v]);
        }
        if ((s = fir_design_host(order, d, wp.data(), ap.data(), n_omega, taps.data() + (size_t)v * (order + 1) * 2)) !=
            RSV_OK)
          return s;
      }
      if (op->real_state)
        for (size_t i = 0; i < taps.size() / 2; ++i) taps[2 * i + 1] = 0.0;
      if ((s = filter_any(op, z, n_z, k, taps.data(), order, true, g)) != RSV_OK) return s;
      n_g = n_z + order;
    } else {
      std::vector<double> sc(k, 0.0);
      for (int v = 0; v < k; ++v) {
        double mx = 0.0;
        for (int j = 0; j < n_omega; ++j) mx = std::max(mx, std::sqrt(nw[(size_t)j * k + v]));
        sc[v] = 1.0 / mx;
      }
      if ((s = ensure(op->ws_ser_n, std::max<size_t>((size_t)n_omega * k, (size_t)k) * sizeof(double))) != RSV_OK)
        return s;
      cudaError_t e = cudaMemcpyAsync(op->ws_ser_n.ptr, sc.data(), k * sizeof(double), cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "TRM scale");
      const int64_t total = n_z * cols;
      scale_vectors_kernel<T, R><<<grid_for(total, 256, op->sm_count), 256, 0, st>>>(
          z, total, n, k, static_cast<const double*>(op->ws_ser_n.ptr), g);
      if ((e = cudaGetLastError()) == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "TRM scale");
      n_g = n_z;
    }
    // |f_hat| of the next forcing g (stored reversed, n_g samples; g[i] at t_i = i d)
    if ((s = fourier_any(op, g, n_g, k, d, -(double)(n_g - 1) * d, neg.data(), n_omega, fh)) != RSV_OK) return s;
    if ((s = norms(&nf)) != RSV_OK) return s;
  }
  return RSV_OK;
}

}  // namespace
}  // namespace rsv

using namespace rsv;

extern "C" rsv_status rsv_series_march(rsv_operator op, int32_t adjoint, int32_t k, const void* init,
                                       const void* forcing, int64_t n_in, int32_t reverse_in,
                                       const rsv_series_opts* opts, void* out, int64_t n_out_max, int64_t* n_out,
                                       int64_t* stops) {
  if (!opts) return fail(RSV_ERR_INVALID_ARG, "series options required");
  return series_march_any(op, adjoint != 0, k, init, forcing, n_in, reverse_in != 0, *opts, out, n_out_max, n_out,
                          stops);
}

extern "C" rsv_status rsv_series_fourier(rsv_operator op, const void* series, int64_t n_snap, int32_t k, double d,
                                         double t0, const double* omega, int32_t n_omega, void* out) {
  if (!op || !series || !omega || !out || n_snap < 1 || k < 1 || n_omega < 1 || !(d > 0.0))
    return fail(RSV_ERR_INVALID_ARG, "bad Fourier arguments");
  if (op->bf16_state) return fail(RSV_ERR_INVALID_ARG, "series need FP32 or FP64 state");
  if (op->prec == RSV_PREC_FP64)
    return fourier_any(op, series, n_snap, k, d, t0, omega, n_omega, static_cast<cpx<double>*>(out));
  return fourier_any(op, series, n_snap, k, d, t0, omega, n_omega, static_cast<cpx<float>*>(out));
}

extern "C" rsv_status rsv_series_filter(rsv_operator op, const void* in, int64_t n_in, int32_t k, const double* taps,
                                        int32_t order, int32_t reverse_taps, void* out) {
  if (op && op->bf16_state) return fail(RSV_ERR_INVALID_ARG, "series need FP32 or FP64 state");
  return filter_any(op, in, n_in, k, taps, order, reverse_taps != 0, out);
}

extern "C" rsv_status rsv_fir_design(int32_t order, double d, const double* w_pts, const double* amp, int32_t n_pts,
                                     double* taps) {
  return fir_design_host(order, d, w_pts, amp, n_pts, taps);
}

extern "C" rsv_status rsv_trm_power_iteration(rsv_operator op, const void* f0, int32_t k, const double* omega,
                                              int32_t n_omega, const rsv_trm_opts* opts, double* gains,
                                              void* w_hat) {
  rsv_status s = series_check(op);
  if (s != RSV_OK) return s;
  if (!f0 || k < 1 || !omega || n_omega < 1 || !opts || !gains || opts->n_iter < 1 || opts->n_snap_max < 2 ||
      opts->filter_order < 0 || opts->filter_order % 2 || !(opts->series.tail_tol > 0.0))
    return fail(RSV_ERR_INVALID_ARG, "bad TRM arguments (tail_tol > 0, even filter order, n_iter >= 1)");
  if (op->real_state)
    for (int j = 0; j < n_omega; ++j)
      if (omega[j] < 0.0) return fail(RSV_ERR_INVALID_ARG, "a real-state operator takes frequencies >= 0");
  if (op->prec == RSV_PREC_FP64)
    return op->real_state ? trm_impl<double, double>(op, f0, k, omega, n_omega, *opts, gains, w_hat)
                          : trm_impl<double, cpx<double>>(op, f0, k, omega, n_omega, *opts, gains, w_hat);
  return op->real_state ? trm_impl<float, float>(op, f0, k, omega, n_omega, *opts, gains, w_hat)
                        : trm_impl<float, cpx<float>>(op, f0, k, omega, n_omega, *opts, gains, w_hat);
}
