"""Algorithms on top of the march: power iteration and block randomized SVD (oracle).

App. A: the action w = R_y^H R_y f (App. A Eq. (iteration)) comes from one
direct and one adjoint run.  With f_n = w_{n-1} the iterate converges to the
leading forcing mode (App. A Eq. (powerMethod)) and the gain is estimated by
sigma_n = sqrt(||f_n|| / ||f_{n-1}||) (App. A Eq. (tildeSig)); the error falls
by (sigma_2 / sigma_1)^2 per iteration.  Normalising per frequency on the
Fourier coefficients replaces a temporal filter (Sec. 2.3).

The block form runs k test vectors per frequency at once (the randomized SVD
the paper cites in Sec. 1): Y = R Omega; q times {Q = qr(Y); Z = R^H Q;
Q = qr(Z); Y = R Q}; Q = qr(Y); W = R^H Q; then B = W^H = Q^H R and its SVD
B = U_s S V^H give gains S, response modes Q U_s and forcing modes V
(Sec. 2.1: R_y = U Sigma V^H).

`march_direct(block)` / `march_adjoint(block)` map [n_omega][k][n] blocks to
[n_omega][k][n] blocks.

Refinement (a higher-precision pass after a lower-precision rSVD): given the
forcing basis Q of span V, one direct run gives R Q, and the SVD of R Q is the
Rayleigh-Ritz step for R^H R on span(Q): the Ritz values are the gains of
R restricted to that subspace, exact when span(Q) holds the leading right
singular vectors and in error by O(eps^2) when the basis is off by eps.  `instances` lists (offset, size) of independent
diagonal blocks of a batched operator; each gets its own QR and SVD.
"""
from __future__ import annotations

import numpy as np

from .decay import splitmix64


def gaussian_test_block(seed: int, n_omega: int, k: int, n: int, real_rows=()) -> np.ndarray:
    """Seeded Gaussian test block Omega [n_omega][k][n] complex128 that the seeded randomized SVD
    draws: entry e (row-major over the block) takes the SplitMix64 values 2e and 2e + 1 of stream
    `seed` (top 53 bits: u1 = (x + 1) 2^-53 in (0, 1], u2 = x 2^-53 in [0, 1)) through the Box-Muller
    transform (Box & Muller 1958), z0 + i z1 = sqrt(-2 ln u1) exp(2 pi i u2); the entry is
    (z0 + i z1) / sqrt(2), and in the rows listed in `real_rows` (the w = 0 row of a real system)
    the real N(0, 1) value z0."""
    count = n_omega * k * n
    x = splitmix64(seed, 2 * count) >> np.uint64(11)
    u1 = (x[0::2].astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = x[1::2].astype(np.float64) * 2.0 ** -53
    r = np.sqrt(-2.0 * np.log(u1))
    z0 = r * np.cos(2.0 * np.pi * u2)
    z1 = r * np.sin(2.0 * np.pi * u2)
    out = ((z0 + 1j * z1) / np.sqrt(2.0)).reshape(n_omega, k, n)
    for j in real_rows:
        out[j] = z0.reshape(n_omega, k, n)[j]
    return out


def qr_positive(y):
    """Thin QR of y (n x k) with a positive real diagonal in R (unique form)."""
    q, r = np.linalg.qr(y)
    d = np.diag(r)
    ph = np.where(np.abs(d) > 0, d / np.abs(d), 1.0)
    return q * ph[None, :], ph.conj()[:, None] * r


def orthonormalize(block, instances, real_rows=()):
    out = np.empty_like(block)
    for j in range(block.shape[0]):
        for off, size in instances:
            y = block[j, :, off:off + size].T
            if j in real_rows:
                y = y.real
            q, _ = qr_positive(y)
            out[j, :, off:off + size] = q.T
    return out


def power_iteration(march_direct, march_adjoint, f0, n_iter):
    """Power iteration per frequency with per-frequency normalisation (k = 1 block).

    Returns (gain estimates [n_iter][n_omega], last forcing f_n [n_omega][1][n]).
    """
    f = f0 / np.linalg.norm(f0, axis=(1, 2), keepdims=True)
    hist = []
    for _ in range(n_iter):
        w = march_adjoint(march_direct(f))
        nw = np.linalg.norm(w, axis=(1, 2))              # ||f_{n+1}|| with ||f_n|| = 1
        hist.append(np.sqrt(nw))
        f = w / nw[:, None, None]
    return np.array(hist), f


def block_rsvd(march_direct, march_adjoint, omega_block, n_power_iter, n_modes,
               instances=None, real_rows=()):
    """Randomized SVD of R(w_j) for every frequency; returns (gains, V, U).

    gains [n_inst][n_omega][n_modes]; V, U [n_inst][n_omega][n_modes][n_i] lists.
    """
    nom, kk, n = omega_block.shape
    inst = instances or [(0, n)]
    y = march_direct(omega_block)
    for _ in range(n_power_iter):
        q = orthonormalize(y, inst, real_rows)
        z = march_adjoint(q)
        q = orthonormalize(z, inst, real_rows)
        y = march_direct(q)
    q = orthonormalize(y, inst, real_rows)
    w = march_adjoint(q)
    gains = np.zeros((len(inst), nom, n_modes))
    vmodes, umodes = [], []
    for i, (off, size) in enumerate(inst):
        vi, ui = [], []
        for j in range(nom):
            qj = q[j, :, off:off + size].T                # n x k
            bj = w[j, :, off:off + size].conj()           # k x n  = Q^H R
            if j in real_rows:
                bj = bj.real
            us, s, vh = np.linalg.svd(bj, full_matrices=False)
            gains[i, j] = s[:n_modes]
            vi.append(vh[:n_modes].conj())                # forcing modes, rows
            ui.append((qj @ us[:, :n_modes]).T)           # response modes, rows
        vmodes.append(np.array(vi))
        umodes.append(np.array(ui))
    return gains, vmodes, umodes


def rayleigh_ritz_refine(march_direct, basis, n_modes, instances=None, real_rows=()):
    """One direct run on an orthonormalised basis [n_omega][k][n] and the SVD of R Q.

    Returns (gains [n_inst][n_omega][n_modes], forcing modes V, response modes U) as in
    block_rsvd.  The adjoint run is not needed: R^H R restricted to span(Q) is
    (R Q)^H (R Q), whose eigen-pairs are the singular pairs of R Q.
    """
    nom, kk, n = basis.shape
    inst = instances or [(0, n)]
    q = orthonormalize(basis, inst, real_rows)
    y = march_direct(q)
    gains = np.zeros((len(inst), nom, n_modes))
    vmodes, umodes = [], []
    for i, (off, size) in enumerate(inst):
        vi, ui = [], []
        for j in range(nom):
            qj = q[j, :, off:off + size].T                # n x k
            yj = y[j, :, off:off + size].T                # n x k = R Q
            if j in real_rows:
                yj = yj.real
            us, s, wh = np.linalg.svd(yj, full_matrices=False)
            gains[i, j] = s[:n_modes]
            vi.append((qj @ wh.conj().T[:, :n_modes]).T)  # forcing modes Q W, rows
            ui.append(us[:, :n_modes].T)                  # response modes, rows
        vmodes.append(np.array(vi))
        umodes.append(np.array(ui))
    return gains, vmodes, umodes
