// Randomized SVD of the resolvent for all frequencies at once (the block
// generalisation of the power iteration of App. A, Eqs. (iteration) and
// (powerMethod); the randomized SVD is the algorithm the paper cites in
// Sec. 1).  Device work: the marches and the k x k Gram / recombination
// kernels.  Host work: k x k Cholesky and Hermitian Jacobi eigensolves in FP64.
//
//   Y = R Omega
//   repeat q times:  Q = qr(Y);  Z = R^H Q;  Q = qr(Z);  Y = R Q
//   Q = qr(Y);  W = R^H Q                       (W = B^H, B = Q^H R)
//   W^H W = U_s S^2 U_s^H  ->  gains S, response modes Q U_s, forcing modes W U_s S^{-1}
//
// qr is CholeskyQR2: G = X^H X = R^H R, X <- X R^{-1}, applied twice, which
// gives the unique Q with a positive real diagonal in R.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "rsv_ops.h"

namespace rsv {

rsv_status march_any(rsv_operator op, const void* in, int k, const rsv_march_opts* opts, void* out, bool adjoint);

namespace {

using cd = std::complex<double>;

// G (k x k Hermitian positive definite) = R^H R, R upper triangular, real positive diagonal.
bool cholesky_upper(const cd* G, int k, cd* R) {
  std::fill(R, R + k * k, cd(0));
  for (int j = 0; j < k; ++j) {
    double d = G[j * k + j].real();
    for (int i = 0; i < j; ++i) d -= std::norm(R[i * k + j]);
    if (!(d > 0.0)) return false;
    const double rjj = std::sqrt(d);
    R[j * k + j] = rjj;
    for (int l = j + 1; l < k; ++l) {
      cd s = G[j * k + l];
      for (int i = 0; i < j; ++i) s -= std::conj(R[i * k + j]) * R[i * k + l];
      R[j * k + l] = s / rjj;
    }
  }
  return true;
}

// Inverse of an upper triangular matrix (back substitution, column by column).
void invert_upper(const cd* R, int k, cd* X) {
  std::fill(X, X + k * k, cd(0));
  for (int c = 0; c < k; ++c) {
    X[c * k + c] = 1.0 / R[c * k + c];
    for (int r = c - 1; r >= 0; --r) {
      cd s = 0;
      for (int l = r + 1; l <= c; ++l) s += R[r * k + l] * X[l * k + c];
      X[r * k + c] = -s / R[r * k + r];
    }
  }
}

// Cyclic Jacobi for a Hermitian matrix H (k x k, overwritten).  Returns the
// eigenvalues in descending order and the eigenvectors as columns of V.
void jacobi_eig(cd* H, int k, double* lam, cd* V) {
  std::vector<cd> A(H, H + k * k), U(k * k, cd(0));
  for (int i = 0; i < k; ++i) U[i * k + i] = 1.0;
  double fro = 0.0;
  for (int i = 0; i < k * k; ++i) fro += std::norm(A[i]);
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) off += std::norm(A[p * k + q]);
    if (off <= 1e-32 * fro) break;
    for (int p = 0; p < k; ++p) {
      for (int q = p + 1; q < k; ++q) {
        const cd apq = A[p * k + q];
        const double mag = std::abs(apq);
        if (mag == 0.0) continue;
        const cd ph = apq / mag;  // e^{i phi}
        const double tau = (A[q * k + q].real() - A[p * k + p].real()) / (2.0 * mag);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        // J restricted to (p, q): [[c, s], [-s e^{-i phi}, c e^{-i phi}]]
        const cd jpp = c, jpq = s, jqp = -s * std::conj(ph), jqq = c * std::conj(ph);
        for (int i = 0; i < k; ++i) {  // columns: A <- A J
          const cd aip = A[i * k + p], aiq = A[i * k + q];
          A[i * k + p] = aip * jpp + aiq * jqp;
          A[i * k + q] = aip * jpq + aiq * jqq;
          const cd uip = U[i * k + p], uiq = U[i * k + q];
          U[i * k + p] = uip * jpp + uiq * jqp;
          U[i * k + q] = uip * jpq + uiq * jqq;
        }
        for (int i = 0; i < k; ++i) {  // rows: A <- J^H A
          const cd api = A[p * k + i], aqi = A[q * k + i];
          A[p * k + i] = std::conj(jpp) * api + std::conj(jqp) * aqi;
          A[q * k + i] = std::conj(jpq) * api + std::conj(jqq) * aqi;
        }
        A[p * k + q] = 0.0;
        A[q * k + p] = 0.0;
      }
    }
  }
  std::vector<int> idx(k);
  for (int i = 0; i < k; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return A[a * k + a].real() > A[b * k + b].real(); });
  for (int c = 0; c < k; ++c) {
    lam[c] = A[idx[c] * k + idx[c]].real();
    for (int r = 0; r < k; ++r) V[r * k + c] = U[r * k + idx[c]];
  }
}

template <typename R>
cudaError_t gram_to_host(rsv_operator op, const void* X, int k, std::vector<cd>& G) {
  const size_t cnt = (size_t)op->n_omega * op->n_inst * k * k;
  if (ensure(op->ws_gram, cnt * sizeof(cpx<double>)) != RSV_OK) return cudaErrorMemoryAllocation;
  cudaError_t e;
  {
    ProfScope ps(op, PROF_GLUE);
    int64_t max_len = 0;
    for (int i = 0; i < op->n_inst; ++i) max_len = std::max(max_len, op->inst_len[i]);
    e = launch_gram<R>(X, op->n_omega, k, op->n, (const int64_t*)op->d_inst_off, op->n_inst, max_len,
                       (cpx<double>*)op->ws_gram.ptr, op->stream);
  }
  if (e != cudaSuccess) return e;
  G.resize(cnt);
  e = cudaMemcpyAsync(G.data(), op->ws_gram.ptr, cnt * sizeof(cpx<double>), cudaMemcpyDeviceToHost, op->stream);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(op->stream);
}

template <typename R>
cudaError_t combine_from_host(rsv_operator op, const void* in, int ka, int kb, const std::vector<cd>& M, void* out,
                              int out_k) {
  // the small matrices go to the device in the block's precision (the kernel computes in it)
  std::vector<cpx<R>> Mr(M.size());
  for (size_t i = 0; i < M.size(); ++i) Mr[i] = mk<R>((R)M[i].real(), (R)M[i].imag());
  const size_t bytes = Mr.size() * sizeof(cpx<R>);
  if (ensure(op->ws_small, bytes) != RSV_OK) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMemcpyAsync(op->ws_small.ptr, Mr.data(), bytes, cudaMemcpyHostToDevice, op->stream);
  if (e == cudaSuccess) {
    ProfScope ps(op, PROF_GLUE);
    e = launch_combine<R>(in, op->n_omega, ka, kb, op->n, (const int32_t*)op->d_inst_of_point, op->n_inst,
                          op->ws_small.ptr, out, out_k, op->stream);
  }
  // Mr is host memory of this frame: the copy must be done before it goes away
  const cudaError_t es = cudaStreamSynchronize(op->stream);
  return e != cudaSuccess ? e : es;
}

// CholeskyQR2 of every (frequency, instance) block of X, in place.
template <typename R>
rsv_status orthonormalize(rsv_operator op, void* X, int k) {
  std::vector<cd> G, M((size_t)op->n_omega * op->n_inst * k * k), Rf(k * k);
  for (int pass = 0; pass < 2; ++pass) {
    cudaError_t e = gram_to_host<R>(op, X, k, G);
    if (e != cudaSuccess) return cuda_fail(e, "gram");
    for (size_t b = 0; b < (size_t)op->n_omega * op->n_inst; ++b) {
      if (!cholesky_upper(&G[b * k * k], k, Rf.data()))
        return fail(RSV_ERR_DIVERGED, "block lost rank in CholeskyQR (frequency " +
                                          std::to_string(b / op->n_inst) + ")");
      invert_upper(Rf.data(), k, &M[b * k * k]);
    }
    e = combine_from_host<R>(op, X, k, k, M, X, k);
    if (e != cudaSuccess) return cuda_fail(e, "qr combine");
  }
  return RSV_OK;
}

template <typename R>
rsv_status gains_impl(rsv_operator op, const void* omega_block, int k, int q, int n_modes,
                      const rsv_march_opts* opts, double* gains, void* fmodes, void* rmodes) {
  const size_t blk = (size_t)op->n_omega * k * op->n * 2 * sizeof(R);
  rsv_status s;
  if ((s = ensure(op->ws_glue_a, blk)) != RSV_OK) return s;
  if ((s = ensure(op->ws_glue_b, blk)) != RSV_OK) return s;
  void* A = op->ws_glue_a.ptr;
  void* B = op->ws_glue_b.ptr;
  if ((s = march_any(op, omega_block, k, opts, A, false)) != RSV_OK) return s;
  for (int it = 0; it < q; ++it) {
    if ((s = orthonormalize<R>(op, A, k)) != RSV_OK) return s;
    if ((s = march_any(op, A, k, opts, B, true)) != RSV_OK) return s;
    if ((s = orthonormalize<R>(op, B, k)) != RSV_OK) return s;
    if ((s = march_any(op, B, k, opts, A, false)) != RSV_OK) return s;
  }
  if ((s = orthonormalize<R>(op, A, k)) != RSV_OK) return s;
  if ((s = march_any(op, A, k, opts, B, true)) != RSV_OK) return s;
  std::vector<cd> G;
  cudaError_t e = gram_to_host<R>(op, B, k, G);
  if (e != cudaSuccess) return cuda_fail(e, "gram");
  const size_t nb = (size_t)op->n_omega * op->n_inst;
  std::vector<cd> Mu(nb * k * n_modes), Mv(nb * k * n_modes), V(k * k);
  std::vector<double> lam(k);
  for (int j = 0; j < op->n_omega; ++j) {
    for (int i = 0; i < op->n_inst; ++i) {
      const size_t b = (size_t)j * op->n_inst + i;
      jacobi_eig(&G[b * k * k], k, lam.data(), V.data());
      for (int m = 0; m < n_modes; ++m) {
        const double sg = std::sqrt(std::max(lam[m], 0.0));
        gains[((size_t)i * op->n_omega + j) * n_modes + m] = sg;
        for (int a = 0; a < k; ++a) {
          Mu[(b * k + a) * n_modes + m] = V[a * k + m];
          Mv[(b * k + a) * n_modes + m] = sg > 0 ? V[a * k + m] / sg : cd(0);
        }
      }
    }
  }
  if (rmodes) {
    e = combine_from_host<R>(op, A, k, n_modes, Mu, rmodes, n_modes);
    if (e != cudaSuccess) return cuda_fail(e, "response modes");
  }
  if (fmodes) {
    e = combine_from_host<R>(op, B, k, n_modes, Mv, fmodes, n_modes);
    if (e != cudaSuccess) return cuda_fail(e, "forcing modes");
  }
  return RSV_OK;
}

}  // namespace
}  // namespace rsv

using namespace rsv;

extern "C" rsv_status rsv_gains_modes(rsv_operator op, const void* omega_block, int32_t k, int32_t n_power_iter,
                                      int32_t n_modes, const rsv_march_opts* opts, double* gains, void* fmodes,
                                      void* rmodes) {
  if (!op || !omega_block || !gains) return fail(RSV_ERR_INVALID_ARG, "null argument");
  if (!op->have_freq) return fail(RSV_ERR_STATE, "rsv_set_frequencies must come first");
  if (k < 1 || k > 32) return fail(RSV_ERR_INVALID_ARG, "k must be 1..32");
  if (n_modes < 1 || n_modes > k) return fail(RSV_ERR_INVALID_ARG, "n_modes must be 1..k");
  if (n_power_iter < 0) return fail(RSV_ERR_INVALID_ARG, "n_power_iter < 0");
  for (int i = 0; i < op->n_inst; ++i)
    if (op->inst_len[i] < k) return fail(RSV_ERR_INVALID_ARG, "k exceeds an instance's length");
  return op->prec == RSV_PREC_FP64
             ? gains_impl<double>(op, omega_block, k, n_power_iter, n_modes, opts, gains, fmodes, rmodes)
             : gains_impl<float>(op, omega_block, k, n_power_iter, n_modes, opts, gains, fmodes, rmodes);
}
