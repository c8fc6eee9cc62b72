// Per-frequency block algebra of the randomized SVD: Gram matrices of the
// k-vector blocks and recombination of a block by a small matrix.  Products
// are formed in the storage precision of the blocks; the Gram sums across
// 256-point slabs are FP64, and the small matrices are formed in FP64 on the
// host and applied in the block's precision.
//
//   gram:    G[j][i][a][b] = sum_{p in instance i} conj(X[j][a][p]) X[j][b][p]
//   combine: Out[j][b][p]  = sum_a In[j][a][p] M[j][inst(p)][a][b]   (M in the block's precision)
//
// gram gives the CholeskyQR factor (Q = X R^{-1}, R^H R = G) and the small
// Hermitian eigenproblem W^H W = B B^H of the final SVD step.
#include "rsv_internal.h"

namespace rsv {
namespace {

constexpr int kMaxK = 32;

// One CTA per (frequency, instance, chunk of points).  The CTA stages the k
// vectors of 256 points at a time in shared memory (each value read once from
// HBM); thread t accumulates the pairs (a, b) = t, t + 256, ... of the k x k
// Gram over its chunk, in the element precision per 256-point slab and in FP64
// across slabs, and adds its FP64 partial into G with one atomic per pair.
constexpr int kSlab = 256;
constexpr int kSlabLd = kSlab + 1;   // padded row: the k rows of a slab fall in different banks
constexpr int kSlabsPerCta = 16;

template <typename R>
__global__ void __launch_bounds__(256) gram_kernel(const cpx<R>* __restrict__ X, int k, int64_t n,
                                                   const int64_t* __restrict__ inst_off, int n_inst,
                                                   cpx<double>* __restrict__ G) {
  extern __shared__ unsigned char smem_raw[];
  cpx<R>* xs = reinterpret_cast<cpx<R>*>(smem_raw);  // [k][kSlabLd]
  const int inst = blockIdx.y;
  const int j = blockIdx.z;
  const int64_t p0 = inst_off[inst], p1 = inst_off[inst + 1];
  const int64_t c0 = p0 + (int64_t)blockIdx.x * kSlab * kSlabsPerCta;
  if (c0 >= p1) return;
  const cpx<R>* Xj = X + (int64_t)j * k * n;
  const int npairs = k * k;
  cpx<double> acc[kMaxK * kMaxK / 256];
#pragma unroll
  for (int q = 0; q < kMaxK * kMaxK / 256; ++q) acc[q] = mk<double>(0, 0);
  for (int sl = 0; sl < kSlabsPerCta; ++sl) {
    const int64_t s0 = c0 + (int64_t)sl * kSlab;
    if (s0 >= p1) break;
    const int cnt = (int)min((int64_t)kSlab, p1 - s0);
    __syncthreads();
    for (int e = threadIdx.x; e < k * kSlab; e += blockDim.x) {
      const int a = e / kSlab, pp = e % kSlab;
      xs[a * kSlabLd + pp] = pp < cnt ? Xj[(int64_t)a * n + s0 + pp] : mk<R>(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kMaxK * kMaxK / 256; ++q) {
      const int pair = threadIdx.x + 256 * q;
      if (pair < npairs) {
        const int a = pair / k, b = pair % k;
        cpx<R> part = mk<R>(0, 0);
        for (int pp = 0; pp < cnt; ++pp) cfma_conj(part, xs[a * kSlabLd + pp], xs[b * kSlabLd + pp]);
        acc[q].re += (double)part.re;
        acc[q].im += (double)part.im;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kMaxK * kMaxK / 256; ++q) {
    const int pair = threadIdx.x + 256 * q;
    if (pair < npairs) {
      double* g = reinterpret_cast<double*>(G + (((int64_t)j * n_inst + inst) * k) * k + pair);
      atomicAdd(g, acc[q].re);
      atomicAdd(g + 1, acc[q].im);
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(256) combine_kernel(const cpx<R>* In, int ka, int kb, int64_t n,
                                                     const int32_t* __restrict__ inst_of_point, int n_inst,
                                                     const cpx<R>* __restrict__ M, cpx<R>* Out,
                                                     int64_t out_k) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (p >= n) return;
  const int inst = inst_of_point[p];
  const cpx<R>* Mj = M + ((int64_t)j * n_inst + inst) * ka * kb;
  // arithmetic in the element precision R (FP64 blocks: FP64; FP32 blocks: FP32)
  cpx<R> x[kMaxK];
#pragma unroll
  for (int a = 0; a < kMaxK; ++a) x[a] = a < ka ? In[((int64_t)j * ka + a) * n + p] : mk<R>(0, 0);
  // In and Out may alias: every input of this point is in registers now.
  for (int b = 0; b < kb; ++b) {
    cpx<R> s = mk<R>(0, 0);
#pragma unroll
    for (int a = 0; a < kMaxK; ++a) {
      if (a < ka) cfma(s, x[a], Mj[a * kb + b]);
    }
    Out[((int64_t)j * out_k + b) * n + p] = s;
  }
}

}  // namespace

template <typename R>
cudaError_t launch_gram(const void* X, int n_omega, int k, int64_t n, const int64_t* inst_off, int n_inst,
                        int64_t max_len, cpx<double>* G, cudaStream_t st) {
  if (k > kMaxK) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(G, 0, sizeof(cpx<double>) * (size_t)n_omega * n_inst * k * k, st);
  if (e != cudaSuccess) return e;
  // chunks per instance: enough for the longest instance (short instances return early)
  const int64_t per_cta = (int64_t)kSlab * kSlabsPerCta;
  dim3 grid((unsigned)((max_len + per_cta - 1) / per_cta), (unsigned)n_inst, (unsigned)n_omega);
  const size_t smem = sizeof(cpx<R>) * (size_t)k * kSlabLd;
  if (smem > 48 * 1024) cudaFuncSetAttribute(gram_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  gram_kernel<R><<<grid, 256, smem, st>>>((const cpx<R>*)X, k, n, inst_off, n_inst, G);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_combine(const void* In, int n_omega, int ka, int kb, int64_t n, const int32_t* inst_of_point,
                           int n_inst, const void* M, void* Out, int64_t out_k, cudaStream_t st) {
  if (ka > kMaxK || kb > kMaxK) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)n_omega);
  combine_kernel<R><<<grid, 256, 0, st>>>((const cpx<R>*)In, ka, kb, n, inst_of_point, n_inst, (const cpx<R>*)M,
                                          (cpx<R>*)Out, out_k);
  return cudaGetLastError();
}

template cudaError_t launch_gram<double>(const void*, int, int, int64_t, const int64_t*, int, int64_t,
                                        cpx<double>*, cudaStream_t);
template cudaError_t launch_gram<float>(const void*, int, int, int64_t, const int64_t*, int, int64_t, cpx<double>*,
                                       cudaStream_t);
template cudaError_t launch_combine<double>(const void*, int, int, int, int64_t, const int32_t*, int, const void*,
                                           void*, int64_t, cudaStream_t);
template cudaError_t launch_combine<float>(const void*, int, int, int, int64_t, const int32_t*, int, const void*,
                                          void*, int64_t, cudaStream_t);

}  // namespace rsv
