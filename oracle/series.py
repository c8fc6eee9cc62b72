"""Time-series form of the transient-response method (oracle): snapshots, their
interpolation (App. C), temporal FIR filtering (App. B) and Fourier transforms
at arbitrary frequencies (Sec. 2.1 Eq. (fourier)).

Sec. 2.2: a compactly supported forcing (an impulse, f(t) = f0 delta(t),
applied as the initial condition u(0) = f0 in the paper's Sec. 3) gives a
response that decays in time; its snapshots y(t_i), saved every `every`
steps, are Fourier-transformed at any frequency, filtered in time to flatten
their spectrum, and, reversed in time and interpolated between snapshots,
drive the adjoint run.

* Interpolation (App. C), between snapshots spaced by d:
    C0  linear;
    C1  cubic Hermite, derivatives by second-order central differences
        (first-order one-sided at the two ends);
    C2  quintic Hermite matching value, first and second derivative at both
        ends of the interval, derivatives from 5-point centred differences;
        at the first and last snapshot the first derivative is one-sided
        first order and the second derivative is zero; at the second and the
        last-but-one snapshot, second-order central differences.
* FIR filter (App. B): x' = phi * x (discrete convolution) with an order-n
  filter phi (n + 1 taps).  Designed by frequency sampling: the desired
  amplitude A(w) on a uniform grid of [0, pi/dt] is given a linear phase
  exp(-i w n dt / 2), inverse-transformed to n + 1 real taps and shaped by a
  Hamming window; its delay of n dt / 2 is compensated by shifting the
  output back by n / 2 samples (n even).
* Fourier transform: xhat(w) = sum_i x(t_i) exp(-i w t_i) dt (rectangle rule
  on the sample grid; the sign is that of the build's convention).
"""
from __future__ import annotations

import numpy as np

from . import march as _march


# ---------------------------------------------------------------------------
# impulse response series
# ---------------------------------------------------------------------------
def impulse_response(a, h, f0, n_steps, every=1, adjoint=False):
    """Unforced RK4 march from u(0) = f0 (an impulse at t = 0); snapshots every `every` steps.

    Returns (times [n_snap], snapshots [n_snap][k][n]), the first at t = 0.
    """
    op = a.conj().T if adjoint else a
    u = np.array(f0, dtype=np.complex128).T          # [n][k]
    zero = np.zeros_like(u)
    snaps, times = [u.T.copy()], [0.0]
    for s in range(1, n_steps + 1):
        u = _march.rk4_step(op, u, h, zero, zero, zero)
        if s % every == 0:
            snaps.append(u.T.copy())
            times.append(s * h)
    return np.array(times), np.array(snaps)


def fourier(series, times, omegas):
    """xhat(w_j) = sum_i x(t_i) exp(-i w_j t_i) dt, for series [n_t][...] on a uniform grid."""
    dt = times[1] - times[0]
    ph = np.exp(-1j * np.outer(omegas, times))          # [n_omega][n_t]
    return np.tensordot(ph, series, axes=(1, 0)) * dt


def discrete_impulse_transform(a, h, omega, every=1):
    """Closed form of fourier(impulse_response(...)) for the full (infinite) record:
    sum_i M^(every i) exp(-i w every h i) every h = every h (I - M^every z^-every)^-1, z = e^{i w h}."""
    a = np.asarray(a.todense() if hasattr(a, "todense") else a, dtype=np.complex128)
    n = a.shape[0]
    b = h * a
    m = np.eye(n) + b + b @ b / 2 + b @ b @ b / 6 + b @ b @ b @ b / 24
    me = np.linalg.matrix_power(m, every)
    return every * h * np.linalg.inv(np.eye(n) - me * np.exp(-1j * omega * every * h))


# ---------------------------------------------------------------------------
# interpolation between snapshots (App. C)
# ---------------------------------------------------------------------------
def _derivatives(x, d, order):
    """First (and second) derivatives at the samples, with the App. C stencils and edge rules."""
    n = x.shape[0]
    d1 = np.zeros_like(x)
    d2 = np.zeros_like(x)
    if order == 1:
        d1[1:-1] = (x[2:] - x[:-2]) / (2 * d)
        d1[0] = (x[1] - x[0]) / d
        d1[-1] = (x[-1] - x[-2]) / d
        return d1, d2
    # 5-point centred first and second derivatives (fourth order)
    d1[2:-2] = (x[:-4] - 8 * x[1:-3] + 8 * x[3:-1] - x[4:]) / (12 * d)
    d2[2:-2] = (-x[:-4] + 16 * x[1:-3] - 30 * x[2:-2] + 16 * x[3:-1] - x[4:]) / (12 * d * d)
    if n >= 3:   # next to the edges: second-order central differences
        d1[1] = (x[2] - x[0]) / (2 * d)
        d2[1] = (x[2] - 2 * x[1] + x[0]) / (d * d)
        d1[-2] = (x[-1] - x[-3]) / (2 * d)
        d2[-2] = (x[-1] - 2 * x[-2] + x[-3]) / (d * d)
    d1[0] = (x[1] - x[0]) / d      # edges: one-sided first order, zero second derivative
    d1[-1] = (x[-1] - x[-2]) / d
    d2[0] = 0.0
    d2[-1] = 0.0
    return d1, d2


def interpolate(series, d, t, kind="c2"):
    """Value at times t (array, 0 <= t <= (n-1) d) of a series sampled every d (App. C: c0, c1, c2)."""
    x = np.asarray(series)
    n = x.shape[0]
    t = np.asarray(t, dtype=np.float64)
    i = np.clip(np.floor(t / d).astype(int), 0, n - 2)
    s = (t - i * d) / d                                   # in [0, 1]
    sh = (slice(None),) + (None,) * (x.ndim - 1)
    s = s[sh]
    x0, x1 = x[i], x[i + 1]
    if kind == "c0":
        return (1 - s) * x0 + s * x1
    if kind == "c1":
        d1, _ = _derivatives(x, d, 1)
        m0, m1 = d1[i] * d, d1[i + 1] * d
        h00 = 2 * s ** 3 - 3 * s ** 2 + 1
        h10 = s ** 3 - 2 * s ** 2 + s
        h01 = -2 * s ** 3 + 3 * s ** 2
        h11 = s ** 3 - s ** 2
        return h00 * x0 + h10 * m0 + h01 * x1 + h11 * m1
    d1, d2 = _derivatives(x, d, 2)
    v0, v1 = d1[i] * d, d1[i + 1] * d
    a0, a1 = d2[i] * d * d, d2[i + 1] * d * d
    # quintic Hermite basis on [0, 1]: value, first and second derivative at both ends
    s2, s3, s4, s5 = s * s, s ** 3, s ** 4, s ** 5
    h0 = 1 - 10 * s3 + 15 * s4 - 6 * s5
    h1 = s - 6 * s3 + 8 * s4 - 3 * s5
    h2 = 0.5 * s2 - 1.5 * s3 + 1.5 * s4 - 0.5 * s5
    h5 = 10 * s3 - 15 * s4 + 6 * s5
    h4 = -4 * s3 + 7 * s4 - 3 * s5
    h3 = 0.5 * s3 - s4 + 0.5 * s5
    return h0 * x0 + h1 * v0 + h2 * a0 + h5 * x1 + h4 * v1 + h3 * a1


# ---------------------------------------------------------------------------
# FIR filtering (App. B)
# ---------------------------------------------------------------------------
def fir_design(order, dt, amp_fn):
    """Order-`order` (even) linear-phase FIR filter with amplitude response amp_fn(w), w in [0, pi/dt],
    by frequency sampling with a Hamming window.  Returns the order + 1 real taps."""
    if order % 2:
        raise ValueError("order must be even (integer delay order / 2)")
    ntap = order + 1
    nfft = 8 * ntap
    w = np.arange(nfft // 2 + 1) * (2 * np.pi / (nfft * dt))
    spec = amp_fn(w) * np.exp(-1j * w * (order / 2) * dt)           # linear phase: delay order/2 samples
    taps = np.fft.irfft(spec, nfft)[:ntap]
    return taps * np.hamming(ntap)


def fir_apply(taps, series):
    """x' = phi * x along the first axis, the delay of order/2 samples removed (same length as x)."""
    order = len(taps) - 1
    x = np.asarray(series)
    out = np.zeros(x.shape, dtype=np.result_type(x, taps))
    n = x.shape[0]
    for i in range(n):
        acc = 0.0
        for j, c in enumerate(taps):
            src = i + order // 2 - j
            if 0 <= src < n:
                acc = acc + c * x[src]
        out[i] = acc
    return out


def fir_response(taps, dt, omegas):
    """Frequency response of the delay-compensated filter at w: sum_j phi_j exp(-i w (j - order/2) dt)."""
    order = len(taps) - 1
    j = np.arange(len(taps)) - order / 2
    return np.exp(-1j * np.outer(omegas, j * dt)) @ taps
