"""Closed-form resolvents (oracle, small dense systems).

* continuous: R(w) = (i w I - A)^{-1}, the map fhat -> uhat of Sec. 2.1
  Eq. (systemFreqDomain) in the convention du/dt = A u + f;
* discrete: the exact steady-state map of the classical RK4 scheme with
  forcing a e^{i w t} sampled at t_n, t_n + h/2, t_n + h.  Writing B = hA,
  s = e^{i w h/2}, z = s^2, one RK4 step is
      u_{n+1} = M u_n + (h/6) G a_n,
      M = I + B + B^2/2 + B^3/6 + B^4/24,
      G = (I + B + B^2/2 + B^3/4) + s (4I + 2B + B^2/2) + z I,
  and a periodic steady state u_n = uhat e^{i w t_n} gives
      R_h(w) = (z I - M)^{-1} (h/6) G.
  The TRM record (one forcing window, full decay, rectangle rule, 1/N_T)
  reaches the same map, since the window's DFT of the forcing extracts
  exactly one frequency of the grid.
* singular values of R and R_h give the gains of Sec. 2.1 (gain definition).
"""
from __future__ import annotations

import numpy as np


def continuous(a, omega):
    a = np.asarray(a.todense() if hasattr(a, "todense") else a, dtype=np.complex128)
    n = a.shape[0]
    return np.linalg.inv(1j * omega * np.eye(n) - a)


def rk4_discrete(a, omega, h):
    a = np.asarray(a.todense() if hasattr(a, "todense") else a, dtype=np.complex128)
    n = a.shape[0]
    eye = np.eye(n)
    b = h * a
    b2 = b @ b
    b3 = b2 @ b
    b4 = b3 @ b
    m = eye + b + b2 / 2 + b3 / 6 + b4 / 24
    s = np.exp(0.5j * omega * h)
    z = s * s
    g = (eye + b + b2 / 2 + b3 / 4) + s * (4 * eye + 2 * b + b2 / 2) + z * eye
    return np.linalg.solve(z * eye - m, (h / 6.0) * g)


def cn_discrete(a, omega, h):
    """Exact steady-state map of the Crank-Nicolson scheme with forcing a e^{i w t} at the step ends:
    u_{n+1} = M u_n + (h/2) L^{-1} (a_n + a_{n+1}), L = I - hA/2, M = L^{-1}(I + hA/2), and
    u_n = uhat e^{i w t_n} gives R_h^CN(w) = (z I - M)^{-1} L^{-1} (h/2)(1 + z), z = e^{i w h}."""
    a = np.asarray(a.todense() if hasattr(a, "todense") else a, dtype=np.complex128)
    n = a.shape[0]
    eye = np.eye(n)
    lmat = eye - 0.5 * h * a
    m = np.linalg.solve(lmat, eye + 0.5 * h * a)
    z = np.exp(1j * omega * h)
    return np.linalg.solve(z * eye - m, np.linalg.solve(lmat, 0.5 * h * (1 + z) * eye))


def gains(r, n_modes=None):
    sv = np.linalg.svd(r, compute_uv=False)
    return sv if n_modes is None else sv[:n_modes]
