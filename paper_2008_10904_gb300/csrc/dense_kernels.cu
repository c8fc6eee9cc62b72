// Dense operators (caller-supplied complex A): the RK4 step as one dense
// product.
//
// For a linear time-invariant system the classical RK4 step with forcing
// sampled at t_n, t_n + h/2, t_n + h is exactly
//     u_{n+1} = u_n + D u_n + (h/6) [P1 f(t_n) + P2 f(t_n + h/2) + f(t_n + h)],
//     B = h A,  D = B + B^2/2 + B^3/6 + B^4/24,
//     P1 = I + B + B^2/2 + B^3/4,  P2 = 4I + 2B + B^2/2.
// With f(t) = sum_j fhat_j e^{i w_j t} the forcing term of step n is
//     sum_j c_j e^{i w_j t_n},   c_j = (h/6) (P1 + s_j P2 + z_j I) fhat_j,
// s_j = e^{i w_j h/2}, z_j = s_j^2.  So the march needs one dense product per
// step (D u_n) instead of four dependent operator applications, and one
// synthesis point per step.  D, P1, P2 (and their conjugate transposes for
// the adjoint run, whose frequencies are negated) are built once per
// frequency grid in FP64 on the device; c_j once per march.
#include <cmath>
#include <vector>

#include "rsv_ops.h"

namespace rsv {
namespace {

// ---------------------------------------------------------------------------
// General complex GEMM on CUDA cores:
//   C[i][j] = alpha * sum_l A(i, l) B(j, l) + beta * C[i][j]
// A(i, l) = A[i * lda + l];  B(j, l) = B[j * sbj + l * sbl] (any layout).
// 64 x 64 output tile per CTA, 256 threads, 4 x 4 outputs per thread.
// ---------------------------------------------------------------------------
constexpr int GBM = 64, GBN = 64, GBK = 16;

template <typename R>
__global__ void __launch_bounds__(256) cgemm_kernel(int M, int N, int K, const cpx<R>* __restrict__ A, int64_t lda,
                                                    const cpx<R>* __restrict__ B, int64_t sbj, int64_t sbl,
                                                    cpx<R>* __restrict__ C, int64_t ldc, cpx<R> alpha, cpx<R> beta) {
  __shared__ cpx<R> As[GBK][GBM + 1];
  __shared__ cpx<R> Bs[GBK][GBN + 1];
  const int i0 = blockIdx.y * GBM, j0 = blockIdx.x * GBN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  cpx<R> acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = mk<R>(0, 0);
  for (int l0 = 0; l0 < K; l0 += GBK) {
    for (int e = threadIdx.x; e < GBM * GBK; e += 256) {
      const int ii = e / GBK, ll = e % GBK;
      const int gi = i0 + ii, gl = l0 + ll;
      As[ll][ii] = (gi < M && gl < K) ? A[(int64_t)gi * lda + gl] : mk<R>(0, 0);
    }
    for (int e = threadIdx.x; e < GBN * GBK; e += 256) {
      const int jj = e / GBK, ll = e % GBK;
      const int gj = j0 + jj, gl = l0 + ll;
      Bs[ll][jj] = (gj < N && gl < K) ? B[(int64_t)gj * sbj + (int64_t)gl * sbl] : mk<R>(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int ll = 0; ll < GBK; ++ll) {
      cpx<R> av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[ll][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[ll][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) cfma(acc[a][b], av[a], bv[b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gi = i0 + ty + 16 * a, gj = j0 + tx + 16 * b;
      if (gi < M && gj < N) {
        cpx<R>* c = C + (int64_t)gi * ldc + gj;
        cpx<R> v = alpha * acc[a][b];
        if (beta.re != R(0) || beta.im != R(0)) v = v + beta * (*c);
        *c = v;
      }
    }
  }
}

template <typename R>
cudaError_t cgemm(int M, int N, int K, const void* A, int64_t lda, const void* B, int64_t sbj, int64_t sbl, void* C,
                  int64_t ldc, cpx<R> alpha, cpx<R> beta, cudaStream_t st) {
  dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
  cgemm_kernel<R><<<grid, 256, 0, st>>>(M, N, K, (const cpx<R>*)A, lda, (const cpx<R>*)B, sbj, sbl, (cpx<R>*)C, ldc,
                                        alpha, beta);
  return cudaGetLastError();
}

// out = a*X + b*Y + c*Z + d*I (n x n, FP64), any argument pointer may be null (treated as 0).
__global__ void combo_kernel(int n, double a, const cpx<double>* X, double b, const cpx<double>* Y, double c,
                             const cpx<double>* Z, double d, cpx<double>* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  cpx<double> v = mk<double>(0, 0);
  if (X) v = v + a * X[e];
  if (Y) v = v + b * Y[e];
  if (Z) v = v + c * Z[e];
  if (e / n == e % n) v.re += d;
  out[e] = v;
}

// out (precision R) = conj-transpose or copy of an FP64 n x n matrix.
template <typename R>
__global__ void narrow_kernel(int n, const cpx<double>* __restrict__ X, bool conj_transpose, cpx<R>* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  cpx<double> v = conj_transpose ? conjg(X[(int64_t)j * n + i]) : X[e];
  out[e] = mk<R>((R)v.re, (R)v.im);
}

// c[j][r] = (h/6) (G1[j][r] + s_j G2[j][r] + z_j fhat[j][r]),  s_j = tw(sgn p_j * 1), z_j = tw(sgn p_j * 2)
template <typename R>
__global__ void coef_combine_kernel(int n_omega, int64_t rows, const cpx<R>* __restrict__ fhat, int64_t f_stride,
                                    const cpx<R>* __restrict__ G1, const cpx<R>* __restrict__ G2,
                                    const cpx<R>* __restrict__ tw, const int64_t* __restrict__ pj, int sgn,
                                    int64_t m4, R h6, cpx<R>* __restrict__ out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (r >= rows) return;
  const cpx<R> s = tw[phase_index(sgn * pj[j], 1, m4)];
  const cpx<R> z = tw[phase_index(sgn * pj[j], 2, m4)];
  const int64_t e = (int64_t)j * rows + r;
  cpx<R> v = G1[e];
  cfma(v, s, G2[e]);
  cfma(v, z, fhat[(int64_t)j * f_stride + r]);
  out[e] = h6 * v;
}

// ---------------------------------------------------------------------------
// One RK4 step of the dense propagator on CUDA cores:
//   u_out[v][i] = u_in[v][i] + sum_l D[i][l] u_in[v][l] + F[v][i]
// CTA = 8 rows (one warp each) x 32 vectors (one lane each), K in chunks of 128.
// ---------------------------------------------------------------------------
constexpr int SROWS = 8, SVEC = 32, SK = 128;

template <typename R>
__global__ void __launch_bounds__(256) dense_step_kernel(int n, int kg, const cpx<R>* __restrict__ D,
                                                         const cpx<R>* __restrict__ uin, cpx<R>* __restrict__ uout,
                                                         const cpx<R>* __restrict__ F, cpx<R>* __restrict__ Y) {
  extern __shared__ unsigned char smem_raw[];
  cpx<R>* Ds = reinterpret_cast<cpx<R>*>(smem_raw);  // [SROWS][SK]
  cpx<R>* Us = Ds + SROWS * SK;                         // [SK][SVEC + 1]
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int i = blockIdx.x * SROWS + w;
  const int v = blockIdx.y * SVEC + lane;
  cpx<R> acc = mk<R>(0, 0);
  for (int l0 = 0; l0 < n; l0 += SK) {
    for (int e = threadIdx.x; e < SROWS * SK; e += blockDim.x) {
      const int rr = e / SK, ll = e % SK;
      const int gi = blockIdx.x * SROWS + rr, gl = l0 + ll;
      Ds[e] = (gi < n && gl < n) ? D[(int64_t)gi * n + gl] : mk<R>(0, 0);
    }
    for (int e = threadIdx.x; e < SVEC * SK; e += blockDim.x) {
      const int vv = e / SK, ll = e % SK;
      const int gv = blockIdx.y * SVEC + vv, gl = l0 + ll;
      Us[ll * (SVEC + 1) + vv] = (gv < kg && gl < n) ? uin[(int64_t)gv * n + gl] : mk<R>(0, 0);
    }
    __syncthreads();
#pragma unroll 8
    for (int ll = 0; ll < SK; ++ll) cfma(acc, Ds[w * SK + ll], Us[ll * (SVEC + 1) + lane]);
    __syncthreads();
  }
  if (i < n && v < kg) {
    const int64_t e = (int64_t)v * n + i;
    const cpx<R> u0 = uin[e];
    if (Y) Y[e] = u0;
    cpx<R> u1 = u0 + acc;
    if (F) u1 = u1 + F[e];
    uout[e] = u1;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Operator construction and per-grid / per-march preparation
// ---------------------------------------------------------------------------
rsv_status build_dense(rsv_operator op, const rsv_operator_desc* d) {
  if (d->dense_n < 2 || !d->dense_a) return fail(RSV_ERR_INVALID_ARG, "DENSE needs dense_n >= 2 and dense_a");
  const int n = d->dense_n;
  op->n = n;
  op->n_inst = 1;
  op->inst_off.assign(1, 0);
  op->inst_len.assign(1, n);
  op->real_state = false;
  const size_t nn = (size_t)n * n;
  rsv_status s = upload(op, d->dense_a, nn * sizeof(cpx<double>), &op->dense64[0]);
  if (s != RSV_OK) return s;
  const size_t eb = (op->prec == RSV_PREC_FP64 ? sizeof(cpx<double>) : sizeof(cpx<float>));
  for (int m = 0; m < 2; ++m) {
    cudaError_t e = cudaMalloc(&op->dense[m], nn * eb);
    if (e != cudaSuccess) return cuda_fail(e, "dense allocation");
    op->dev.push_back(op->dense[m]);
  }
  for (int m = 0; m < 6; ++m) {
    cudaError_t e = cudaMalloc(&op->prop[m], nn * eb);
    if (e != cudaSuccess) return cuda_fail(e, "dense allocation");
    op->dev.push_back(op->prop[m]);
  }
  const unsigned blocks = (unsigned)((nn + 255) / 256);
  if (op->prec == RSV_PREC_FP64) {
    narrow_kernel<double><<<blocks, 256, 0, op->stream>>>(n, (const cpx<double>*)op->dense64[0], false,
                                                          (cpx<double>*)op->dense[0]);
    narrow_kernel<double><<<blocks, 256, 0, op->stream>>>(n, (const cpx<double>*)op->dense64[0], true,
                                                          (cpx<double>*)op->dense[1]);
  } else {
    narrow_kernel<float><<<blocks, 256, 0, op->stream>>>(n, (const cpx<double>*)op->dense64[0], false,
                                                         (cpx<float>*)op->dense[0]);
    narrow_kernel<float><<<blocks, 256, 0, op->stream>>>(n, (const cpx<double>*)op->dense64[0], true,
                                                         (cpx<float>*)op->dense[1]);
  }
  cudaError_t e = cudaStreamSynchronize(op->stream);
  if (e != cudaSuccess) return cuda_fail(e, "dense build");
  return RSV_OK;
}

// D, P1, P2 and their conjugate transposes for the step h (FP64 build, stored in precision R).
rsv_status dense_on_frequencies(rsv_operator op) {
  const int n = (int)op->n;
  const size_t nn = (size_t)n * n;
  std::vector<void*> tmp(6, nullptr);
  for (auto& p : tmp) {
    cudaError_t e = cudaMalloc(&p, nn * sizeof(cpx<double>));
    if (e != cudaSuccess) {
      for (auto q : tmp)
        if (q) cudaFree(q);
      return cuda_fail(e, "propagator temporaries");
    }
  }
  cpx<double>*B = (cpx<double>*)tmp[0], *B2 = (cpx<double>*)tmp[1], *B3 = (cpx<double>*)tmp[2],
  *B4 = (cpx<double>*)tmp[3], *Dm = (cpx<double>*)tmp[4], *T = (cpx<double>*)tmp[5];
  const cudaStream_t st = op->stream;
  const unsigned blocks = (unsigned)((nn + 255) / 256);
  const cpx<double> one = mk<double>(1, 0), zero = mk<double>(0, 0);
  cudaError_t e;
  combo_kernel<<<blocks, 256, 0, st>>>(n, op->h, (const cpx<double>*)op->dense64[0], 0, nullptr, 0, nullptr, 0, B);
  // B^(p+1) = B^p B: element (i, j) = sum_l B^p[i][l] B[l][j]  -> B(j, l) = B[l * n + j]
  e = cgemm<double>(n, n, n, B, n, B, 1, n, B2, n, one, zero, st);
  if (e == cudaSuccess) e = cgemm<double>(n, n, n, B2, n, B, 1, n, B3, n, one, zero, st);
  if (e == cudaSuccess) e = cgemm<double>(n, n, n, B3, n, B, 1, n, B4, n, one, zero, st);
  if (e != cudaSuccess) return cuda_fail(e, "propagator powers");
  auto store = [&](const cpx<double>* src, int slot_direct) {
    if (op->prec == RSV_PREC_FP64) {
      narrow_kernel<double><<<blocks, 256, 0, st>>>(n, src, false, (cpx<double>*)op->prop[slot_direct]);
      narrow_kernel<double><<<blocks, 256, 0, st>>>(n, src, true, (cpx<double>*)op->prop[slot_direct + 3]);
    } else {
      narrow_kernel<float><<<blocks, 256, 0, st>>>(n, src, false, (cpx<float>*)op->prop[slot_direct]);
      narrow_kernel<float><<<blocks, 256, 0, st>>>(n, src, true, (cpx<float>*)op->prop[slot_direct + 3]);
    }
  };
  // D = B + B^2/2 + B^3/6 + B^4/24 : B + B^2/2 into T, then add B^3/6 + B^4/24
  combo_kernel<<<blocks, 256, 0, st>>>(n, 1.0, B, 0.5, B2, 1.0 / 6.0, B3, 0.0, T);
  combo_kernel<<<blocks, 256, 0, st>>>(n, 1.0, T, 1.0 / 24.0, B4, 0, nullptr, 0.0, Dm);
  store(Dm, 0);
  // P1 = I + B + B^2/2 + B^3/4
  combo_kernel<<<blocks, 256, 0, st>>>(n, 1.0, B, 0.5, B2, 0.25, B3, 1.0, T);
  store(T, 1);
  e = cudaStreamSynchronize(st);  // T is rewritten next
  // P2 = 4I + 2B + B^2/2
  combo_kernel<<<blocks, 256, 0, st>>>(n, 2.0, B, 0.5, B2, 0, nullptr, 4.0, T);
  store(T, 2);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    for (auto q : tmp) cudaFree(q);
    return cuda_fail(e, "propagator build");
  }
  rsv_status ts = dense_tc_prepare(op, Dm);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  for (auto q : tmp) cudaFree(q);
  if (ts != RSV_OK) return ts;
  if (e != cudaSuccess) return cuda_fail(e, "propagator build");
  op->dense_h = op->h;
  return RSV_OK;
}

// c_j = (h/6)(P1 + s_j P2 + z_j I) fhat_j for the kg vectors of one group.
template <typename R>
cudaError_t dense_prepare(rsv_operator op, const void* fhat, int64_t f_stride, int kg, bool adjoint, void* out,
                          void* tmp) {
  const int n = (int)op->n;
  const int64_t rows = (int64_t)kg * n;
  const int M = op->n_omega * kg;  // GEMM rows: (j, v) pairs; the group is strided by f_stride per j
  const void* P1 = op->prop[adjoint ? 4 : 1];
  const void* P2 = op->prop[adjoint ? 5 : 2];
  const cpx<R> one = mk<R>(1, 0), zero = mk<R>(0, 0);
  cudaError_t e = cudaSuccess;
  // G[j][v][i] = sum_p fhat[j][v][p] P[i][p]  (A rows (j, v): (j * f_stride + v * n); B(j=i, l=p) = P[i * n + p])
  // The (j, v) rows of a group are not uniformly strided when kg < k, so run one GEMM per frequency.
  char* g1 = static_cast<char*>(out);
  char* g2 = static_cast<char*>(tmp);
  if (f_stride == rows) {  // the whole block: rows (j, v) are uniformly strided by n
    e = cgemm<R>(M, n, n, fhat, n, P1, n, 1, g1, n, one, zero, op->stream);
    if (e == cudaSuccess) e = cgemm<R>(M, n, n, fhat, n, P2, n, 1, g2, n, one, zero, op->stream);
  }
  for (int j = 0; f_stride != rows && j < op->n_omega && e == cudaSuccess; ++j) {
    const void* a = static_cast<const char*>(fhat) + (size_t)j * f_stride * sizeof(cpx<R>);
    e = cgemm<R>(kg, n, n, a, n, P1, n, 1, g1 + (size_t)j * rows * sizeof(cpx<R>), n, one, zero, op->stream);
    if (e == cudaSuccess)
      e = cgemm<R>(kg, n, n, a, n, P2, n, 1, g2 + (size_t)j * rows * sizeof(cpx<R>), n, one, zero, op->stream);
  }
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((rows + 255) / 256), (unsigned)op->n_omega);
  coef_combine_kernel<R><<<grid, 256, 0, op->stream>>>(op->n_omega, rows, (const cpx<R>*)fhat, f_stride,
                                                       (const cpx<R>*)g1, (const cpx<R>*)g2, (const cpx<R>*)op->d_tw,
                                                       op->d_pj, adjoint ? -1 : 1, 4 * op->n_t, R(op->h / 6.0),
                                                       (cpx<R>*)out);
  return cudaGetLastError();
}

template <typename R>
cudaError_t dense_step(rsv_operator op, int kg, bool adjoint, const void* uin, void* uout, const void* F, void* Y) {
  const int n = (int)op->n;
  dim3 grid((unsigned)((n + SROWS - 1) / SROWS), (unsigned)((kg + SVEC - 1) / SVEC));
  const size_t smem = sizeof(cpx<R>) * (SROWS * SK + SK * (SVEC + 1));
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(dense_step_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dense_step_kernel<R><<<grid, 256, smem, op->stream>>>(n, kg, (const cpx<R>*)op->prop[adjoint ? 3 : 0],
                                                        (const cpx<R>*)uin, (cpx<R>*)uout, (const cpx<R>*)F,
                                                        (cpx<R>*)Y);
  return cudaGetLastError();
}

template <typename R>
cudaError_t dense_apply(rsv_operator op, const void* x, int k, bool adjoint, void* y) {
  const int n = (int)op->n;
  return cgemm<R>(k, n, n, x, n, op->dense[adjoint ? 1 : 0], n, 1, y, n, mk<R>(1, 0), mk<R>(0, 0), op->stream);
}

template cudaError_t dense_prepare<double>(rsv_operator, const void*, int64_t, int, bool, void*, void*);
template cudaError_t dense_prepare<float>(rsv_operator, const void*, int64_t, int, bool, void*, void*);
template cudaError_t dense_step<double>(rsv_operator, int, bool, const void*, void*, const void*, void*);
template cudaError_t dense_step<float>(rsv_operator, int, bool, const void*, void*, const void*, void*);
template cudaError_t dense_apply<double>(rsv_operator, const void*, int, bool, void*);
template cudaError_t dense_apply<float>(rsv_operator, const void*, int, bool, void*);

}  // namespace rsv
