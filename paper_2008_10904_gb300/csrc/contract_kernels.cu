// Forcing synthesis and response analysis over one time tile.
//
// Synthesis (Sec. 2.3, Eq. (forceFseries), sign flipped to exp(+i w t)):
//   F[tau][r] = sum_j fhat[j][r] exp(i sgn w_j t_tau),  t_tau = (2 n0 + tau) h / 2,
// for the tile's 2 S + 1 stage times (step starts and midpoints).  For a real
// state the forcing is sum_j c_j Re(fhat_j exp(i w_j t)), c_j = 1 at w = 0, else 2.
//
// Analysis (Sec. 2.1, Eq. (fourier), rectangle rule over the window):
//   acc[j][r] += sum_s Y[s][r] exp(-i sgn w_j t_s),  t_s = (n0 + s) h.
//
// Both are contractions over a short dimension (frequencies or tile steps)
// that stream one long dimension r (state rows): each thread owns a few rows
// and keeps a chunk of outputs in registers; the exact twiddles exp(i pi q / 2N_T)
// (integer phase index q) are staged in shared memory per block.  Products
// and in-tile sums run in the element precision R; in-tile partial sums are
// folded into FP64 registers every 64 steps and then added to the FP64
// accumulator array once per tile.
#include "rsv_internal.h"

namespace rsv {
namespace {

constexpr int kTPB = 128;
constexpr int kTauChunk = 8;
constexpr int kOmChunk = 8;
constexpr int kSChunk = 64;

// Register blocking: each thread owns RB rows (RB = 4 in FP32, 2 in FP64) and a
// chunk of 8 output columns (synthesis: stage times, analysis: frequencies), so
// every twiddle read from shared memory feeds RB complex multiply-adds.
template <typename R>
struct Blk {
  static constexpr int RB = sizeof(R) == 4 ? 4 : 2;
};

template <typename R, bool REAL>
__global__ void __launch_bounds__(kTPB) synth_kernel(TileGeom g, const cpx<R>* __restrict__ fhat,
                                                     const cpx<R>* __restrict__ tw,
                                                     const int64_t* __restrict__ pj,
                                                     const float* __restrict__ cw, void* __restrict__ Fout) {
  constexpr int RB = Blk<R>::RB;
  extern __shared__ unsigned char smem_raw[];
  cpx<R>* stw = reinterpret_cast<cpx<R>*>(smem_raw);  // [n_omega][kTauChunk]
  const int n_tau = g.n_tau > 0 ? g.n_tau : 2 * g.steps + 1;
  // blocks of the same rows are adjacent in launch order (chunk index fastest), so the
  // coefficient rows they all read stay in L2
  const int n_chunks = (n_tau + kTauChunk - 1) / kTauChunk;
  const int tau0 = (int)(blockIdx.x % n_chunks) * kTauChunk;
  const int64_t row_block = blockIdx.x / n_chunks;
  const int nt = min(kTauChunk, n_tau - tau0);
  for (int e = threadIdx.x; e < kTauChunk * g.n_omega; e += blockDim.x) {
    const int j = e / kTauChunk, t = e - j * kTauChunk;
    cpx<R> v = mk<R>(0, 0);
    if (t < nt) {
      const int64_t q = phase_index(g.sgn * pj[j], 2 * g.n0 + (int64_t)(tau0 + t) * g.tau_stride, g.m4);
      v = tw[q];
      if (REAL) v = R(cw[j]) * v;
    }
    stw[j * kTauChunk + t] = v;
  }
  __syncthreads();
  const int64_t r0 = row_block * (kTPB * RB) + threadIdx.x;
  bool ok[RB];
#pragma unroll
  for (int b = 0; b < RB; ++b) ok[b] = r0 + b * kTPB < g.rows;
  cpx<R> acc[RB][kTauChunk];
#pragma unroll
  for (int b = 0; b < RB; ++b)
#pragma unroll
    for (int t = 0; t < kTauChunk; ++t) acc[b][t] = mk<R>(0, 0);
  for (int j = 0; j < g.n_omega; ++j) {
    cpx<R> x[RB];
#pragma unroll
    for (int b = 0; b < RB; ++b) x[b] = ok[b] ? fhat[(int64_t)j * g.coef_stride + r0 + b * kTPB] : mk<R>(0, 0);
#pragma unroll
    for (int t = 0; t < kTauChunk; ++t) {
      const cpx<R> w = stw[j * kTauChunk + t];
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        if (REAL)
          acc[b][t].re = fma(w.re, x[b].re, fma(-w.im, x[b].im, acc[b][t].re));
        else
          cfma(acc[b][t], w, x[b]);
      }
    }
  }
#pragma unroll
  for (int b = 0; b < RB; ++b) {
    if (!ok[b]) continue;
    const int64_t r = r0 + b * kTPB;
    if (REAL) {
      R* F = reinterpret_cast<R*>(Fout);
      for (int t = 0; t < nt; ++t) F[(int64_t)(tau0 + t) * g.rows + r] = acc[b][t].re;
    } else {
      cpx<R>* F = reinterpret_cast<cpx<R>*>(Fout);
      for (int t = 0; t < nt; ++t) F[(int64_t)(tau0 + t) * g.rows + r] = acc[b][t];
    }
  }
}

template <typename R, bool REAL>
__global__ void __launch_bounds__(kTPB) analysis_kernel(TileGeom g, const void* __restrict__ Yin, int s0, int s1,
                                                        const cpx<R>* __restrict__ tw,
                                                        const int64_t* __restrict__ pj,
                                                        cpx<double>* __restrict__ acc, int64_t acc_stride) {
  constexpr int RB = REAL ? 2 : 1;  // complex state: fewer registers, more resident blocks
  __shared__ cpx<R> stw[kSChunk][kOmChunk];
  // frequency chunk fastest in launch order: the blocks sharing a row block reuse its snapshots in L2
  const int n_chunks = (g.n_omega + kOmChunk - 1) / kOmChunk;
  const int j0 = (int)(blockIdx.x % n_chunks) * kOmChunk;
  const int64_t row_block = blockIdx.x / n_chunks;
  const int nj = min(kOmChunk, g.n_omega - j0);
  const int64_t r0 = row_block * (kTPB * RB) + threadIdx.x;
  bool ok[RB];
#pragma unroll
  for (int b = 0; b < RB; ++b) ok[b] = r0 + b * kTPB < g.rows;
  cpx<double> a64[RB][kOmChunk];
#pragma unroll
  for (int b = 0; b < RB; ++b)
#pragma unroll
    for (int jj = 0; jj < kOmChunk; ++jj) a64[b][jj] = mk<double>(0, 0);
  for (int sc = s0; sc < s1; sc += kSChunk) {
    const int ns = min(kSChunk, s1 - sc);
    __syncthreads();
    for (int e = threadIdx.x; e < ns * kOmChunk; e += blockDim.x) {
      const int s = e / kOmChunk, jj = e - s * kOmChunk;
      cpx<R> v = mk<R>(0, 0);
      if (jj < nj) v = tw[phase_index(g.sgn * pj[j0 + jj], 2 * (g.n0 + sc + s), g.m4)];
      stw[s][jj] = v;
    }
    __syncthreads();
    cpx<R> a[RB][kOmChunk];
#pragma unroll
    for (int b = 0; b < RB; ++b)
#pragma unroll
      for (int jj = 0; jj < kOmChunk; ++jj) a[b][jj] = mk<R>(0, 0);
    for (int s = 0; s < ns; ++s) {
      cpx<R> y[RB];
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        const int64_t off = (int64_t)(sc + s) * g.rows + r0 + b * kTPB;
        if (!ok[b])
          y[b] = mk<R>(0, 0);
        else if (REAL)
          y[b] = mk<R>(reinterpret_cast<const R*>(Yin)[off], R(0));
        else
          y[b] = reinterpret_cast<const cpx<R>*>(Yin)[off];
      }
#pragma unroll
      for (int jj = 0; jj < kOmChunk; ++jj) {
        const cpx<R> w = stw[s][jj];
#pragma unroll
        for (int b = 0; b < RB; ++b) {
          if (REAL) {
            a[b][jj].re = fma(w.re, y[b].re, a[b][jj].re);
            a[b][jj].im = fma(-w.im, y[b].re, a[b][jj].im);
          } else {
            cfma_conj(a[b][jj], w, y[b]);
          }
        }
      }
    }
#pragma unroll
    for (int b = 0; b < RB; ++b)
#pragma unroll
      for (int jj = 0; jj < kOmChunk; ++jj) {
        a64[b][jj].re += (double)a[b][jj].re;
        a64[b][jj].im += (double)a[b][jj].im;
      }
  }
#pragma unroll
  for (int b = 0; b < RB; ++b) {
    if (!ok[b]) continue;
    const int64_t r = r0 + b * kTPB;
    for (int jj = 0; jj < nj; ++jj) {
      cpx<double>* p = acc + (int64_t)(j0 + jj) * acc_stride + r;
      cpx<double> v = *p;
      v.re += a64[b][jj].re;
      v.im += a64[b][jj].im;
      *p = v;
    }
  }
}

template <typename R>
__global__ void finish_kernel(const cpx<double>* __restrict__ acc, int64_t acc_stride, int n_omega, int64_t rows,
                              double scale, const double* __restrict__ pscale, int64_t n, cpx<R>* __restrict__ out,
                              int64_t out_stride) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (r >= rows || j >= n_omega) return;
  const cpx<double> v = acc[(int64_t)j * acc_stride + r];
  const double f = pscale ? scale * pscale[r % n] : scale;
  out[(int64_t)j * out_stride + r] = mk<R>(R(v.re * f), R(v.im * f));
}

// out[j][r] = in[j][r] * s[r mod n] (products in FP64, rounded to the element type)
template <typename R>
__global__ void scale_block_kernel(const cpx<R>* in, int64_t in_stride, cpx<R>* out, int64_t out_stride,
                                   int64_t rows, int64_t n, const double* __restrict__ s) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (r >= rows) return;
  const double f = s[r % n];
  const cpx<R> v = in[(int64_t)j * in_stride + r];
  out[(int64_t)j * out_stride + r] = mk<R>(R((double)v.re * f), R((double)v.im * f));
}

}  // namespace

template <typename R>
cudaError_t launch_synth(const TileGeom& g, const void* fhat, const void* tw, const int64_t* pj, const float* cw,
                         bool real_state, void* F, cudaStream_t st) {
  const int n_tau = g.n_tau > 0 ? g.n_tau : 2 * g.steps + 1;
  const int64_t per_block = (int64_t)kTPB * Blk<R>::RB;
  const int64_t blocks = ((g.rows + per_block - 1) / per_block) * ((n_tau + kTauChunk - 1) / kTauChunk);
  dim3 grid((unsigned)blocks);
  const size_t smem = sizeof(cpx<R>) * kTauChunk * g.n_omega;
  if (real_state) {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(synth_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    synth_kernel<R, true><<<grid, kTPB, smem, st>>>(g, (const cpx<R>*)fhat, (const cpx<R>*)tw, pj, cw, F);
  } else {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(synth_kernel<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    synth_kernel<R, false><<<grid, kTPB, smem, st>>>(g, (const cpx<R>*)fhat, (const cpx<R>*)tw, pj, cw, F);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_analysis(const TileGeom& g, const void* Y, int s0, int s1, const void* tw, const int64_t* pj,
                            bool real_state, cpx<double>* acc, int64_t acc_stride, cudaStream_t st) {
  if (s1 <= s0) return cudaSuccess;
  const int rb = real_state ? 2 : 1;
  const int64_t blocks = ((g.rows + rb * kTPB - 1) / (rb * kTPB)) * ((g.n_omega + kOmChunk - 1) / kOmChunk);
  dim3 grid((unsigned)blocks);
  if (real_state)
    analysis_kernel<R, true><<<grid, kTPB, 0, st>>>(g, Y, s0, s1, (const cpx<R>*)tw, pj, acc, acc_stride);
  else
    analysis_kernel<R, false><<<grid, kTPB, 0, st>>>(g, Y, s0, s1, (const cpx<R>*)tw, pj, acc, acc_stride);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_finish(const cpx<double>* acc, int64_t acc_stride, int n_omega, int64_t rows, double scale,
                          void* out, int64_t out_stride, cudaStream_t st, const double* pscale, int64_t n) {
  dim3 grid((unsigned)((rows + 255) / 256), (unsigned)n_omega);
  finish_kernel<R><<<grid, 256, 0, st>>>(acc, acc_stride, n_omega, rows, scale, pscale, n > 0 ? n : rows,
                                         (cpx<R>*)out, out_stride);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_scale_block(const void* in, int64_t in_stride, void* out, int64_t out_stride, int n_omega,
                               int64_t rows, int64_t n, const double* s, cudaStream_t st) {
  dim3 grid((unsigned)((rows + 255) / 256), (unsigned)n_omega);
  scale_block_kernel<R><<<grid, 256, 0, st>>>((const cpx<R>*)in, in_stride, (cpx<R>*)out, out_stride, rows, n, s);
  return cudaGetLastError();
}

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st) { return cudaMemsetAsync(p, 0, bytes, st); }

template cudaError_t launch_synth<double>(const TileGeom&, const void*, const void*, const int64_t*, const float*,
                                         bool, void*, cudaStream_t);
template cudaError_t launch_synth<float>(const TileGeom&, const void*, const void*, const int64_t*, const float*,
                                        bool, void*, cudaStream_t);
template cudaError_t launch_analysis<double>(const TileGeom&, const void*, int, int, const void*, const int64_t*,
                                            bool, cpx<double>*, int64_t, cudaStream_t);
template cudaError_t launch_analysis<float>(const TileGeom&, const void*, int, int, const void*, const int64_t*,
                                           bool, cpx<double>*, int64_t, cudaStream_t);
template cudaError_t launch_finish<double>(const cpx<double>*, int64_t, int, int64_t, double, void*, int64_t,
                                          cudaStream_t, const double*, int64_t);
template cudaError_t launch_finish<float>(const cpx<double>*, int64_t, int, int64_t, double, void*, int64_t,
                                         cudaStream_t, const double*, int64_t);
template cudaError_t launch_scale_block<double>(const void*, int64_t, void*, int64_t, int, int64_t, int64_t,
                                               const double*, cudaStream_t);
template cudaError_t launch_scale_block<float>(const void*, int64_t, void*, int64_t, int, int64_t, int64_t,
                                              const double*, cudaStream_t);

}  // namespace rsv
