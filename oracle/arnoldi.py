"""Krylov subspace and Arnoldi estimates of optimal and suboptimal gains (oracle).

App. A of the paper.  The runs give w_n = R^H R f_n (one direct run y_n = R f_n,
one adjoint run w_n = R^H y_n; Eq. (iteration)).  With F = [f_0 .. f_{m-1}] and
W = [w_0 .. w_{m-1}], R^H R F = W (Eq. (RRFi), with the typo R R^H read as R^H R),
and after F = Q_F R_F the projection of R^H R on span F is
H = Q_F^H W R_F^{-1} (Eq. (arDec)); its eigen-decomposition H psi = gamma^2 psi
gives gains gamma_i, forcing modes Q_F psi_i and response modes
gamma_i^{-1} R Q_F psi_i (the response of the direct run, so the runs' y_n are kept).

* Krylov variant: f_{n+1} = w_n (the power-iteration sequence, normalised),
  and H from the QR of F; ill-conditioned once the sequence has converged.
* Arnoldi variant (Eq. (freqOrt)): f_{n+1} is the part of w_n orthogonal to
  f_0 .. f_n in the forcing metric W_f (here W_f = I), normalised; F is then
  orthonormal, R_F is diagonal and H is Hessenberg and Hermitian, i.e.
  tridiagonal (Lanczos on R^H R).  The orthogonalisation is done twice
  (classical Gram-Schmidt with one reorthogonalisation) so that F stays
  orthonormal to rounding.

Each frequency is its own problem; the runs act on [n_omega][1][n] blocks.
"""
from __future__ import annotations

import numpy as np


def _normalise(b):
    nrm = np.linalg.norm(b, axis=(1, 2), keepdims=True)
    return b / nrm, nrm[:, 0, 0]


def arnoldi(march_direct, march_adjoint, f0, m, n_modes, real_rows=(), krylov=False):
    """m iterations from f0 [n_omega][1][n]; returns (gains [n_omega][n_modes], V, U, H).

    V, U: [n_omega][n_modes][n] forcing and response modes (unit 2-norm); H: [n_omega][m][m].
    """
    nom, _, n = f0.shape
    f, _ = _normalise(np.array(f0, dtype=np.complex128))
    for j in real_rows:
        f[j] = f[j].real
        f[j] /= np.linalg.norm(f[j])
    F = np.zeros((nom, m, n), dtype=np.complex128)
    Y = np.zeros((nom, m, n), dtype=np.complex128)
    Wb = np.zeros((nom, m, n), dtype=np.complex128)
    for it in range(m):
        F[:, it] = f[:, 0]
        y = march_direct(f)
        w = march_adjoint(y)
        Y[:, it] = y[:, 0]
        Wb[:, it] = w[:, 0]
        nxt = w.copy()
        if not krylov:
            for _ in range(2):          # Eq. (freqOrt), Gram-Schmidt against f_0 .. f_it, twice
                for j in range(nom):
                    theta = F[j, :it + 1].conj() @ nxt[j, 0]
                    nxt[j, 0] -= theta @ F[j, :it + 1]
        f, _ = _normalise(nxt)
    gains = np.zeros((nom, n_modes))
    V = np.zeros((nom, n_modes, n), dtype=np.complex128)
    U = np.zeros((nom, n_modes, n), dtype=np.complex128)
    H = np.zeros((nom, m, m), dtype=np.complex128)
    for j in range(nom):
        Fj = F[j].T                                   # n x m
        q, r = np.linalg.qr(Fj)
        h = q.conj().T @ Wb[j].T @ np.linalg.inv(r)   # Eq. (arDec): H = Q_F^H W R_F^{-1}
        if j in real_rows:
            h = h.real
        H[j] = h
        lam, psi = np.linalg.eigh(0.5 * (h + h.conj().T))
        order = np.argsort(lam)[::-1][:n_modes]
        g = np.sqrt(np.maximum(lam[order], 0.0))
        gains[j] = g
        vq = q @ psi[:, order]                        # forcing modes Q_F psi
        V[j] = vq.T
        # response: R Q_F psi = Y R_F^{-1} psi (the direct runs are linear in f)
        U[j] = ((Y[j].T @ np.linalg.inv(r) @ psi[:, order]) / np.where(g > 0, g, 1.0)).T
    return gains, V, U, H
