"""RK4 time march with Fourier-series forcing and DFT of the response (oracle).

Follows Sec. 2.1-2.3 of the paper in the sign convention du/dt = A u + f:

* forcing synthesis from Fourier coefficients (Sec. 2.3 Eq. (forceFseries), with the
  exponent sign flipped for this convention):
      complex state  f(t) = sum_j fhat_j exp(+i w_j t)
      real state     f(t) = sum_j c_j Re(fhat_j exp(+i w_j t)),  c_j = 1 at w_j = 0, else 2
* the classical 4-stage Runge-Kutta step with the forcing taken at t_n,
  t_n + h/2 and t_n + h;
* the response's Fourier coefficient over a window of N_T steps by the
  rectangle rule, yhat_j = (1/N_T) sum_n u_n exp(-i w_j t_n) (Sec. 2.1 Eq. (fourier));
* schedules:
      SSRM (Sec. 2.3): force for n_trans + 1 windows, analyse the last one;
      TRM  (Sec. 2.2): force for one window only (compact forcing), keep
           marching the unforced response for `tail_steps` more steps and
           analyse the whole record.  Sec. 2.2 truncates the record once the
           state norm has become negligible (Sec. 3: below 1e-9; Sec. 4: 1e-3 of
           its maximum over the run).  With tail_tol > 0 the tail ends at the
           first check point at or after the end of the forcing window where
           every vector's norm is at most tail_tol times the largest norm that
           vector had at any check point so far; check points are every
           `check_every` steps from the start (default: every step, the plain
           reading of "until the norm is negligible") and the last step, and
           `tail_steps` caps the tail.
* adjoint run (Sec. 2.1 Eq. (adsystem)): -dz/dt + A^H z = y backward in time is,
  after t -> -t, a forward march of dz/dt = A^H z + y(-t); the Fourier
  coefficient at w of y(-t) is the coefficient at -w of y.  So the adjoint
  run is the same march with A^H and every w_j negated, and returns
  R(w_j)^H yhat_j (Sec. 2.1 Eq. (adsystemFreqDomain)).

Arrays of Fourier coefficients are [n_omega][k][n] complex128.  The state is
kept as [n][k] so that sparse matrix products apply to all k vectors at once.
"""
from __future__ import annotations

import numpy as np


def _apply(a, x):
    return a @ x


def synthesize(fhat2, omegas, t, real_state, weights):
    """Forcing at time t for all k vectors: returns [n][k]."""
    tw = np.exp(1j * omegas * t)                         # e^{+i w_j t}
    nom, kk, n = fhat2.shape
    if real_state:
        f = ((weights * tw) @ fhat2.reshape(nom, kk * n)).real
    else:
        f = tw @ fhat2.reshape(nom, kk * n)
    return f.reshape(kk, n).T


def rk4_step(a, u, h, f0, fh, f1):
    """One classical RK4 step of du/dt = A u + f(t)."""
    k1 = _apply(a, u) + f0
    k2 = _apply(a, u + 0.5 * h * k1) + fh
    k3 = _apply(a, u + 0.5 * h * k2) + fh
    k4 = _apply(a, u + h * k3) + f1
    return u + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def cn_factor(a, h):
    """Crank-Nicolson matrices of du/dt = A u + f: the LU factors of (I - h/2 A) and (I + h/2 A)."""
    import scipy.sparse as sps
    import scipy.sparse.linalg as spla
    n = a.shape[0]
    eye = sps.identity(n, dtype=np.complex128, format="csc")
    asp = sps.csc_matrix(a, dtype=np.complex128)
    return spla.splu((eye - 0.5 * h * asp).tocsc()), (eye + 0.5 * h * asp).tocsr()


def cn_step(lu_rhs, u, h, f0, f1):
    """One Crank-Nicolson step: (I - h/2 A) u' = (I + h/2 A) u + h/2 (f(t_n) + f(t_n + h)) (Sec. 3)."""
    lu, rhs_m = lu_rhs
    return lu.solve(rhs_m @ u + 0.5 * h * (f0 + f1))


def schedule(grid, variant, n_trans=0, tail_steps=0):
    """(total steps, first analysed step, steps with forcing)."""
    if variant == "ssrm":
        total = (n_trans + 1) * grid.n_t
        return total, n_trans * grid.n_t, total
    if variant == "trm":
        return grid.n_t + tail_steps, 0, grid.n_t
    raise ValueError(variant)


def march(a, grid, fhat, *, variant="ssrm", n_trans=0, tail_steps=0, adjoint=False,
          real_state=False, return_state=False, stop_after=None, tail_tol=0.0, check_every=None,
          return_steps=False, scheme="rk4"):
    """Direct (adjoint=False) or adjoint run; returns yhat [n_omega][k][n].

    `a` is the system matrix (sparse or dense); the adjoint run uses a^H.
    `scheme`: "rk4" (classical RK4) or "cn" (Crank-Nicolson, forcing at the step ends).
    `stop_after` ends the march early (for timing a bounded sample only).
    `tail_tol`, `check_every`: TRM truncation by the state norm (see the module
    docstring).  `return_steps` also returns the number of steps marched.
    """
    op = a.conj().T.tocsr() if (adjoint and hasattr(a, "tocsr")) else (a.conj().T if adjoint else a)
    om = -grid.omegas if adjoint else grid.omegas
    nom, kk, n = fhat.shape
    weights = np.where(grid.omegas == 0.0, 1.0, 2.0)
    h = grid.h
    total, first, forced = schedule(grid, variant, n_trans, tail_steps)
    dtype = np.float64 if real_state else np.complex128
    u = np.zeros((n, kk), dtype=dtype)
    acc = np.zeros((nom, kk, n), dtype=np.complex128)
    zero = np.zeros((n, kk), dtype=dtype)
    adaptive = variant == "trm" and tail_tol > 0.0
    if adaptive and not check_every:
        check_every = 1
    peak = np.zeros(kk)
    last = total if stop_after is None else min(total, stop_after)
    marched = 0
    cn = cn_factor(op, h) if scheme == "cn" else None
    for step in range(last):
        t = step * h
        if step >= first:
            acc += np.exp(-1j * om * t)[:, None, None] * u.T[None, :, :]
        if step < forced:
            f0 = synthesize(fhat, om, t, real_state, weights)
            fh = synthesize(fhat, om, t + 0.5 * h, real_state, weights) if cn is None else None
            f1 = synthesize(fhat, om, t + h, real_state, weights)
        else:
            f0 = fh = f1 = zero
        u = rk4_step(op, u, h, f0, fh, f1) if cn is None else cn_step(cn, u, h, f0, f1)
        marched = step + 1
        if adaptive and (marched % check_every == 0 or marched == total):
            norms = np.sqrt(np.sum(np.abs(u) ** 2, axis=0))
            peak = np.maximum(peak, norms)
            if marched >= forced and np.all(norms <= tail_tol * peak):
                break
    out = acc / grid.n_t
    res = (out, u.T.copy()) if return_state else (out,)
    if return_steps:
        res = res + (marched,)
    return res if len(res) > 1 else res[0]
