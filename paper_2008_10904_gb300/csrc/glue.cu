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

// CholeskyQR2 of every (frequency, instance) block of X, in place.  With r_out (host,
// [n_omega][n_inst][k][k]) the combined triangular factor X = Q R, R = R2 R1, is returned too.
template <typename R>
rsv_status orthonormalize(rsv_operator op, void* X, int k, cd* r_out = nullptr) {
  const size_t nb = (size_t)op->n_omega * op->n_inst;
  std::vector<cd> G, M(nb * k * k), Rf(k * k), R1;
  if (r_out) R1.assign(nb * k * k, cd(0));
  for (int pass = 0; pass < 2; ++pass) {
    cudaError_t e = gram_to_host<R>(op, X, k, G);
    if (e != cudaSuccess) return cuda_fail(e, "gram");
    for (size_t b = 0; b < nb; ++b) {
      if (!cholesky_upper(&G[b * k * k], k, Rf.data()))
        return fail(RSV_ERR_DIVERGED, "block lost rank in CholeskyQR (frequency " +
                                          std::to_string(b / op->n_inst) + ")");
      invert_upper(Rf.data(), k, &M[b * k * k]);
      if (r_out && pass == 0) std::copy(Rf.begin(), Rf.end(), R1.begin() + b * k * k);
      if (r_out && pass == 1) {
        cd* Rt = r_out + b * k * k;   // R2 R1 (both upper triangular)
        for (int i = 0; i < k; ++i)
          for (int j = 0; j < k; ++j) {
            cd acc = 0;
            for (int l = i; l <= j; ++l) acc += Rf[i * k + l] * R1[b * k * k + l * k + j];
            Rt[i * k + j] = acc;
          }
      }
    }
    e = combine_from_host<R>(op, X, k, k, M, X, k);
    if (e != cudaSuccess) return cuda_fail(e, "qr combine");
  }
  return RSV_OK;
}

// Modes of the weighted problem back to the forcing / response spaces: x <- x * row (per point).
template <typename R>
cudaError_t unweight_modes(rsv_operator op, void* modes, int n_modes, int row) {
  if (!op->have_weights || modes == nullptr) return cudaSuccess;
  const int64_t rows = (int64_t)n_modes * op->n;
  return launch_scale_block<R>(modes, rows, modes, rows, op->n_omega, rows, op->n, op->d_wt + (size_t)row * op->n,
                               op->stream);
}

// Imaginary parts of the w = 0 rows of a block of a real-state operator are dropped (the march
// ignores them as input: the forcing of a real system at w = 0 is real).
template <typename R>
cudaError_t zero_rows_imag(rsv_operator op, void* X, int k) {
  if (!op->real_state) return cudaSuccess;
  for (int j = 0; j < op->n_omega; ++j) {
    if (op->pj[j] != 0) continue;
    char* row = static_cast<char*>(X) + (size_t)j * k * op->n * 2 * sizeof(R) + sizeof(R);
    cudaError_t e = cudaMemset2DAsync(row, 2 * sizeof(R), 0, sizeof(R), (size_t)k * op->n, op->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Rayleigh-Ritz step on a basis (App. A): Q = qr(basis), Y = R Q, Y^H Y = W S^2 W^H; gains S,
// forcing modes Q W, response modes Y W S^{-1}.
template <typename R>
rsv_status refine_impl(rsv_operator op, const void* basis, int k, int n_modes, const rsv_march_opts* opts,
                       double* gains, void* fmodes, void* rmodes) {
  const size_t blk = (size_t)op->n_omega * k * op->n * 2 * sizeof(R);
  rsv_status s;
  if ((s = ensure(op->ws_glue_a, blk)) != RSV_OK) return s;
  if ((s = ensure(op->ws_glue_b, blk)) != RSV_OK) return s;
  void* Q = op->ws_glue_a.ptr;
  void* Y = op->ws_glue_b.ptr;
  cudaError_t e = cudaMemcpyAsync(Q, basis, blk, cudaMemcpyDeviceToDevice, op->stream);
  if (e == cudaSuccess) e = zero_rows_imag<R>(op, Q, k);
  // with metrics: W_f-orthonormalising the basis is orthonormalising W_f^{1/2} basis
  if (e == cudaSuccess && op->have_weights)
    e = launch_scale_block<R>(Q, (int64_t)k * op->n, Q, (int64_t)k * op->n, op->n_omega, (int64_t)k * op->n, op->n,
                              op->d_wt + (size_t)8 * op->n, op->stream);
  if (e != cudaSuccess) return cuda_fail(e, "refinement basis");
  if ((s = orthonormalize<R>(op, Q, k)) != RSV_OK) return s;
  if ((s = march_any(op, Q, k, opts, Y, false, SCALE_TILDE)) != RSV_OK) return s;
  std::vector<cd> G;
  e = gram_to_host<R>(op, Y, k, G);
  if (e != cudaSuccess) return cuda_fail(e, "gram");
  const size_t nb = (size_t)op->n_omega * op->n_inst;
  std::vector<cd> Mf(nb * k * n_modes), Mr(nb * k * n_modes), V(k * k);
  std::vector<double> lam(k);
  for (int j = 0; j < op->n_omega; ++j) {
    for (int i = 0; i < op->n_inst; ++i) {
      const size_t b = (size_t)j * op->n_inst + i;
      jacobi_eig(&G[b * k * k], k, lam.data(), V.data());
      for (int m = 0; m < n_modes; ++m) {
        const double sg = std::sqrt(std::max(lam[m], 0.0));
        gains[((size_t)i * op->n_omega + j) * n_modes + m] = sg;
        for (int a = 0; a < k; ++a) {
          Mf[(b * k + a) * n_modes + m] = V[a * k + m];
          Mr[(b * k + a) * n_modes + m] = sg > 0 ? V[a * k + m] / sg : cd(0);
        }
      }
    }
  }
  if (fmodes) {
    e = combine_from_host<R>(op, Q, k, n_modes, Mf, fmodes, n_modes);
    if (e == cudaSuccess) e = unweight_modes<R>(op, fmodes, n_modes, 6);
    if (e != cudaSuccess) return cuda_fail(e, "forcing modes");
  }
  if (rmodes) {
    e = combine_from_host<R>(op, Y, k, n_modes, Mr, rmodes, n_modes);
    if (e == cudaSuccess) e = unweight_modes<R>(op, rmodes, n_modes, 7);
    if (e != cudaSuccess) return cuda_fail(e, "response modes");
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
  if ((s = march_any(op, omega_block, k, opts, A, false, SCALE_TILDE)) != RSV_OK) return s;
  for (int it = 0; it < q; ++it) {
    if ((s = orthonormalize<R>(op, A, k)) != RSV_OK) return s;
    if ((s = march_any(op, A, k, opts, B, true, SCALE_TILDE)) != RSV_OK) return s;
    if ((s = orthonormalize<R>(op, B, k)) != RSV_OK) return s;
    if ((s = march_any(op, B, k, opts, A, false, SCALE_TILDE)) != RSV_OK) return s;
  }
  if ((s = orthonormalize<R>(op, A, k)) != RSV_OK) return s;
  if ((s = march_any(op, A, k, opts, B, true, SCALE_TILDE)) != RSV_OK) return s;
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
    if (e == cudaSuccess) e = unweight_modes<R>(op, rmodes, n_modes, 7);
    if (e != cudaSuccess) return cuda_fail(e, "response modes");
  }
  if (fmodes) {
    e = combine_from_host<R>(op, B, k, n_modes, Mv, fmodes, n_modes);
    if (e == cudaSuccess) e = unweight_modes<R>(op, fmodes, n_modes, 6);
    if (e != cudaSuccess) return cuda_fail(e, "forcing modes");
  }
  return RSV_OK;
}

// Arnoldi (App. A, Eq. (freqOrt)) per frequency and instance, one vector each: f_0 normalised;
// for it = 0 .. m - 1: y_it = R f_it, w_it = R^H y_it; column it of H holds <f_i, w_it> (i <= it,
// classical Gram-Schmidt done twice) and the norm beta of the remainder (H[it+1][it]);
// f_{it+1} = remainder / beta.  Then H psi = gamma^2 psi: gains gamma, forcing modes F psi,
// response modes Y psi / gamma (F is orthonormal, so R_F = I).
template <typename R>
rsv_status arnoldi_impl(rsv_operator op, const void* f0, int m, int n_modes, const rsv_march_opts* opts,
                        double* gains, void* fmodes, void* rmodes) {
  const int64_t n = op->n;
  const int nw = op->n_omega, ni = op->n_inst;
  const size_t nb = (size_t)nw * ni;
  const size_t vec = (size_t)nw * n * 2 * sizeof(R);          // one vector per frequency, [n_omega][1][n]
  rsv_status s;
  if ((s = ensure(op->ws_glue_a, 2 * (size_t)m * vec)) != RSV_OK) return s;
  if ((s = ensure(op->ws_glue_b, (size_t)(m + 1) * vec + 3 * vec)) != RSV_OK) return s;
  char* Fb = static_cast<char*>(op->ws_glue_a.ptr);             // [n_omega][m][n]
  char* Yb = Fb + (size_t)m * vec;                              // [n_omega][m][n]
  char* X = static_cast<char*>(op->ws_glue_b.ptr);              // [n_omega][it + 2][n], compact
  char* cur = X + (size_t)(m + 1) * vec;
  char* yt = cur + vec;
  char* wt = yt + vec;
  const size_t el = 2 * sizeof(R), row = (size_t)n * el;
  const cudaStream_t st = op->stream;
  // columns [rows of H][it] per (frequency, instance)
  std::vector<cd> H(nb * m * m, cd(0)), rfac(nb);
  cudaError_t e = cudaMemcpyAsync(cur, f0, vec, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = zero_rows_imag<R>(op, cur, 1);
  if (e != cudaSuccess) return cuda_fail(e, "arnoldi start");
  if ((s = orthonormalize<R>(op, cur, 1)) != RSV_OK) return s;
  std::vector<cd> G, M;
  for (int it = 0; it < m; ++it) {
    // f_it into the basis (column it of every frequency's block)
    e = cudaMemcpy2DAsync(Fb + it * row, (size_t)m * row, cur, row, row, nw, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "arnoldi basis");
    if ((s = march_any(op, cur, 1, opts, yt, false, SCALE_TILDE)) != RSV_OK) return s;
    if ((s = march_any(op, yt, 1, opts, wt, true, SCALE_TILDE)) != RSV_OK) return s;
    e = cudaMemcpy2DAsync(Yb + it * row, (size_t)m * row, yt, row, row, nw, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "arnoldi responses");
    const int kk = it + 2;                                      // f_0 .. f_it and the vector being reduced
    const char* src = wt;
    for (int pass = 0; pass < 2; ++pass) {
      e = cudaMemcpy2DAsync(X, (size_t)kk * row, Fb, (size_t)m * row, (size_t)(it + 1) * row, nw,
                            cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(X + (size_t)(it + 1) * row, (size_t)kk * row, src, row, row, nw, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess) e = gram_to_host<R>(op, X, kk, G);
      if (e != cudaSuccess) return cuda_fail(e, "arnoldi projection");
      M.assign(nb * kk, cd(0));
      for (size_t b = 0; b < nb; ++b) {
        for (int i = 0; i <= it; ++i) {
          const cd th = G[(b * kk + i) * kk + it + 1];            // <f_i, w>
          H[(b * m + i) * m + it] += th;
          M[b * kk + i] = -th;
        }
        M[b * kk + it + 1] = 1.0;
      }
      e = combine_from_host<R>(op, X, kk, 1, M, cur, 1);       // w - F theta
      if (e != cudaSuccess) return cuda_fail(e, "arnoldi orthogonalisation");
      src = cur;
    }
    if (it + 1 < m) {
      std::vector<cd> rr(nb);
      if ((s = orthonormalize<R>(op, cur, 1, rr.data())) != RSV_OK)
        return fail(RSV_ERR_DIVERGED, "Arnoldi: the Krylov space stopped growing (a frequency's remainder vanished)");
      for (size_t b = 0; b < nb; ++b) H[(b * m + it + 1) * m + it] = rr[b];
    }
  }
  // eigen-decomposition of the Hermitian part of H per (frequency, instance)
  std::vector<cd> Mf(nb * m * n_modes), Mr(nb * m * n_modes), Hs(m * m), V(m * m);
  std::vector<double> lam(m);
  for (int j = 0; j < nw; ++j) {
    for (int i = 0; i < ni; ++i) {
      const size_t b = (size_t)j * ni + i;
      for (int r = 0; r < m; ++r)
        for (int c = 0; c < m; ++c) Hs[r * m + c] = 0.5 * (H[(b * m + r) * m + c] + std::conj(H[(b * m + c) * m + r]));
      if (op->real_state && op->pj[j] == 0)
        for (auto& x : Hs) x = x.real();
      jacobi_eig(Hs.data(), m, lam.data(), V.data());
      for (int q = 0; q < n_modes; ++q) {
        const double g = std::sqrt(std::max(lam[q], 0.0));
        gains[((size_t)i * nw + j) * n_modes + q] = g;
        for (int a = 0; a < m; ++a) {
          Mf[(b * m + a) * n_modes + q] = V[a * m + q];
          Mr[(b * m + a) * n_modes + q] = g > 0 ? V[a * m + q] / g : cd(0);
        }
      }
    }
  }
  if (fmodes) {
    e = combine_from_host<R>(op, Fb, m, n_modes, Mf, fmodes, n_modes);
    if (e == cudaSuccess) e = unweight_modes<R>(op, fmodes, n_modes, 6);
    if (e != cudaSuccess) return cuda_fail(e, "forcing modes");
  }
  if (rmodes) {
    e = combine_from_host<R>(op, Yb, m, n_modes, Mr, rmodes, n_modes);
    if (e == cudaSuccess) e = unweight_modes<R>(op, rmodes, n_modes, 7);
    if (e != cudaSuccess) return cuda_fail(e, "response modes");
  }
  return RSV_OK;
}

}  // namespace
}  // namespace rsv

using namespace rsv;

extern "C" rsv_status rsv_arnoldi_gains(rsv_operator op, const void* f0, int32_t m, int32_t n_modes,
                                        const rsv_march_opts* opts, double* gains, void* fmodes, void* rmodes) {
  if (!op || !f0 || !gains) return fail(RSV_ERR_INVALID_ARG, "null argument");
  if (!op->have_freq) return fail(RSV_ERR_STATE, "rsv_set_frequencies must come first");
  if (m < 1 || m > 31) return fail(RSV_ERR_INVALID_ARG, "m must be 1..31");
  if (n_modes < 1 || n_modes > m) return fail(RSV_ERR_INVALID_ARG, "n_modes must be 1..m");
  for (int i = 0; i < op->n_inst; ++i)
    if (op->inst_len[i] < m) return fail(RSV_ERR_INVALID_ARG, "m exceeds an instance's length");
  return op->prec == RSV_PREC_FP64 ? arnoldi_impl<double>(op, f0, m, n_modes, opts, gains, fmodes, rmodes)
                                   : arnoldi_impl<float>(op, f0, m, n_modes, opts, gains, fmodes, rmodes);
}

namespace {
rsv_status check_block_args(rsv_operator op, int k) {
  if (!op->have_freq) return fail(RSV_ERR_STATE, "rsv_set_frequencies must come first");
  if (k < 1 || k > 32) return fail(RSV_ERR_INVALID_ARG, "k must be 1..32");
  for (int i = 0; i < op->n_inst; ++i)
    if (op->inst_len[i] < k) return fail(RSV_ERR_INVALID_ARG, "k exceeds an instance's length");
  return RSV_OK;
}
}  // namespace

extern "C" rsv_status rsv_refine_gains(rsv_operator op, const void* basis, int32_t k, int32_t n_modes,
                                       const rsv_march_opts* opts, double* gains, void* fmodes, void* rmodes) {
  if (!op || !basis || !gains) return fail(RSV_ERR_INVALID_ARG, "null argument");
  rsv_status s = check_block_args(op, k);
  if (s != RSV_OK) return s;
  if (n_modes < 1 || n_modes > k) return fail(RSV_ERR_INVALID_ARG, "n_modes must be 1..k");
  return op->prec == RSV_PREC_FP64 ? refine_impl<double>(op, basis, k, n_modes, opts, gains, fmodes, rmodes)
                                   : refine_impl<float>(op, basis, k, n_modes, opts, gains, fmodes, rmodes);
}

extern "C" rsv_status rsv_orthonormalize(rsv_operator op, void* block, int32_t k, double* r_factor) {
  if (!op || !block) return fail(RSV_ERR_INVALID_ARG, "null argument");
  rsv_status s = check_block_args(op, k);
  if (s != RSV_OK) return s;
  cd* r = reinterpret_cast<cd*>(r_factor);
  return op->prec == RSV_PREC_FP64 ? orthonormalize<double>(op, block, k, r) : orthonormalize<float>(op, block, k, r);
}

namespace rsv {
namespace {
__device__ __forceinline__ uint64_t splitmix64_value(uint64_t seed, uint64_t i) {   // value i of stream seed
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Entry e of the seeded test block: SplitMix64 values 2e, 2e + 1 through the Box-Muller transform,
// (z0 + i z1) / sqrt 2, or z0 in the w = 0 row of a real-state operator (row_real).
template <typename R>
__global__ void gaussian_block_kernel(cpx<R>* __restrict__ out, int64_t count, int64_t row_len, int row_real,
                                      uint64_t seed) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const double u1 = (double)((splitmix64_value(seed, 2 * (uint64_t)e) >> 11) + 1ull) * 0x1.0p-53;
    const double u2 = (double)(splitmix64_value(seed, 2 * (uint64_t)e + 1) >> 11) * 0x1.0p-53;
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    const bool real_row = row_real >= 0 && e / row_len == row_real;
    const double s = real_row ? 1.0 : 0.70710678118654752440;
    out[e] = mk<R>((R)(s * r * cs), real_row ? R(0) : (R)(s * r * sn));
  }
}
}  // namespace
}  // namespace rsv

extern "C" rsv_status rsv_gains_modes_seeded(rsv_operator op, int32_t k, int32_t n_power_iter, int32_t n_modes,
                                             uint64_t seed, const rsv_march_opts* opts, double* gains, void* fmodes,
                                             void* rmodes) {
  if (!op || !gains) return fail(RSV_ERR_INVALID_ARG, "null argument");
  if (!op->have_freq) return fail(RSV_ERR_STATE, "rsv_set_frequencies must come first");
  if (k < 1 || k > 32) return fail(RSV_ERR_INVALID_ARG, "k must be 1..32");
  const int64_t count = (int64_t)op->n_omega * k * op->n;
  const size_t eb = op->prec == RSV_PREC_FP64 ? sizeof(cpx<double>) : sizeof(cpx<float>);
  rsv_status s = ensure(op->ws_omega, (size_t)count * eb);
  if (s != RSV_OK) return s;
  int row_real = -1;   // the w = 0 row of a real-state operator carries real test vectors
  if (op->real_state)
    for (int j = 0; j < op->n_omega; ++j)
      if (op->pj[j] == 0) row_real = j;
  const unsigned blocks = (unsigned)std::min<int64_t>((count + 255) / 256, 16 * std::max(op->sm_count, 1));
  if (op->prec == RSV_PREC_FP64)
    gaussian_block_kernel<double><<<blocks, 256, 0, op->stream>>>((cpx<double>*)op->ws_omega.ptr, count,
                                                                  (int64_t)k * op->n, row_real, seed);
  else
    gaussian_block_kernel<float><<<blocks, 256, 0, op->stream>>>((cpx<float>*)op->ws_omega.ptr, count,
                                                                 (int64_t)k * op->n, row_real, seed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "seeded test block");
  return rsv_gains_modes(op, op->ws_omega.ptr, k, n_power_iter, n_modes, opts, gains, fmodes, rmodes);
}

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
