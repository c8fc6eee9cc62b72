// Per-frequency block algebra of the randomized SVD: Gram matrices of the
// k-vector blocks and recombination of a block by a small matrix.  Both run
// with FP64 arithmetic whatever the storage type of the blocks.
//
//   gram:    G[j][i][a][b] = sum_{p in instance i} conj(X[j][a][p]) X[j][b][p]
//   combine: Out[j][b][p]  = sum_a In[j][a][p] M[j][inst(p)][a][b]
//
// gram gives the CholeskyQR factor (Q = X R^{-1}, R^H R = G) and the small
// Hermitian eigenproblem W^H W = B B^H of the final SVD step.
#include "rsv_internal.h"

namespace rsv {
namespace {

constexpr int kMaxK = 32;

// One CTA per (a, instance, frequency); threads stride over the instance's
// points and keep the k products with row a in registers.
template <typename R>
__global__ void __launch_bounds__(256) gram_kernel(const cpx<R>* __restrict__ X, int k, int64_t n,
                                                   const int64_t* __restrict__ inst_off, int n_inst,
                                                   cpx<double>* __restrict__ G) {
  const int a = blockIdx.x;
  const int inst = blockIdx.y;
  const int j = blockIdx.z;
  const int64_t p0 = inst_off[inst], p1 = inst_off[inst + 1];
  const cpx<R>* Xj = X + (int64_t)j * k * n;
  cpx<double> acc[kMaxK];
#pragma unroll
  for (int b = 0; b < kMaxK; ++b) acc[b] = mk<double>(0, 0);
  for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const cpx<R> xa = Xj[(int64_t)a * n + p];
    const cpx<double> xa64 = mk<double>(xa.re, xa.im);
#pragma unroll
    for (int b = 0; b < kMaxK; ++b) {
      if (b < k) {
        const cpx<R> xb = Xj[(int64_t)b * n + p];
        cfma_conj(acc[b], xa64, mk<double>(xb.re, xb.im));
      }
    }
  }
  __shared__ cpx<double> red[8][kMaxK];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int b = 0; b < kMaxK; ++b) {
    double re = acc[b].re, im = acc[b].im;
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) red[warp][b] = mk<double>(re, im);
  }
  __syncthreads();
  if (threadIdx.x < k) {
    const int b = threadIdx.x;
    cpx<double> s = mk<double>(0, 0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = s + red[w][b];
    G[(((int64_t)j * n_inst + inst) * k + a) * k + b] = s;
  }
}

template <typename R>
__global__ void __launch_bounds__(256) combine_kernel(const cpx<R>* In, int ka, int kb, int64_t n,
                                                     const int32_t* __restrict__ inst_of_point, int n_inst,
                                                     const cpx<double>* __restrict__ M, cpx<R>* Out,
                                                     int64_t out_k) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (p >= n) return;
  const int inst = inst_of_point[p];
  const cpx<double>* Mj = M + ((int64_t)j * n_inst + inst) * ka * kb;
  cpx<double> x[kMaxK];
#pragma unroll
  for (int a = 0; a < kMaxK; ++a) {
    x[a] = mk<double>(0, 0);
    if (a < ka) {
      const cpx<R> v = In[((int64_t)j * ka + a) * n + p];
      x[a] = mk<double>(v.re, v.im);
    }
  }
  // In and Out may alias: every input of this point is in registers now.
  for (int b = 0; b < kb; ++b) {
    cpx<double> s = mk<double>(0, 0);
#pragma unroll
    for (int a = 0; a < kMaxK; ++a)
      if (a < ka) cfma(s, x[a], Mj[a * kb + b]);
    Out[((int64_t)j * out_k + b) * n + p] = mk<R>(R(s.re), R(s.im));
  }
}

}  // namespace

template <typename R>
cudaError_t launch_gram(const void* X, int n_omega, int k, int64_t n, const int64_t* inst_off, int n_inst,
                        cpx<double>* G, cudaStream_t st) {
  if (k > kMaxK) return cudaErrorInvalidValue;
  dim3 grid((unsigned)k, (unsigned)n_inst, (unsigned)n_omega);
  gram_kernel<R><<<grid, 256, 0, st>>>((const cpx<R>*)X, k, n, inst_off, n_inst, G);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_combine(const void* In, int n_omega, int ka, int kb, int64_t n, const int32_t* inst_of_point,
                           int n_inst, const cpx<double>* M, void* Out, int64_t out_k, cudaStream_t st) {
  if (ka > kMaxK || kb > kMaxK) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)n_omega);
  combine_kernel<R><<<grid, 256, 0, st>>>((const cpx<R>*)In, ka, kb, n, inst_of_point, n_inst, M, (cpx<R>*)Out,
                                          out_k);
  return cudaGetLastError();
}

template cudaError_t launch_gram<double>(const void*, int, int, int64_t, const int64_t*, int, cpx<double>*,
                                        cudaStream_t);
template cudaError_t launch_gram<float>(const void*, int, int, int64_t, const int64_t*, int, cpx<double>*,
                                       cudaStream_t);
template cudaError_t launch_combine<double>(const void*, int, int, int, int64_t, const int32_t*, int,
                                           const cpx<double>*, void*, int64_t, cudaStream_t);
template cudaError_t launch_combine<float>(const void*, int, int, int, int64_t, const int32_t*, int,
                                          const cpx<double>*, void*, int64_t, cudaStream_t);

}  // namespace rsv
