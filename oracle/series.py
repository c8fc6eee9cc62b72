"""Time-series form of the transient-response method (oracle): snapshots, their
interpolation (App. C), temporal FIR filtering (App. B), Fourier transforms
at arbitrary frequencies (Sec. 2.1 Eq. (fourier)), runs driven by a sampled
series, and the TRM power iteration built from them (Sec. 2.2, App. A).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this module; the library never does.

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
* Series-driven run: the forcing at the RK4 (or Crank-Nicolson) stage times is
  the interpolant of the input series, zero after its last sample; the state
  is recorded every `every` steps; the record is truncated per vector once its
  norm is negligible against its running peak (Sec. 2.2).
* Readings where the paper is silent: the amplitude of the flattening filter
  is 1 / |w_hat(w)| at the frequencies of interest, linear in between and
  constant beyond; for a complex state the amplitude is specified over signed
  frequencies (complex taps), since a complex signal's spectrum is not
  symmetric; the whole convolution is kept (length n + order), so that the
  filtered series decays at both ends instead of being cut off.
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


def hermite_data(series, d, kind="c2"):
    """Values and the App. C derivative estimates, scaled to unit spacing (v = d x', a = d^2 x'')."""
    x = np.asarray(series)
    if kind == "c0":
        return x, None, None
    d1, d2 = _derivatives(x, d, 1 if kind == "c1" else 2)
    return x, d1 * d, (d2 * d * d if kind == "c2" else None)


def hermite_eval(data, i, s, kind="c2"):
    """Interpolant on interval [t_i, t_{i+1}] at local coordinate s in [0, 1] (arrays i, s broadcast
    against the series' trailing axes)."""
    x, v, a = data
    sh = (slice(None),) + (None,) * (x.ndim - 1)
    i = np.asarray(i)
    s = np.asarray(s, dtype=np.float64)[sh]
    x0, x1 = x[i], x[i + 1]
    if kind == "c0":
        return (1 - s) * x0 + s * x1
    if kind == "c1":
        h00 = 2 * s ** 3 - 3 * s ** 2 + 1
        h10 = s ** 3 - 2 * s ** 2 + s
        h01 = -2 * s ** 3 + 3 * s ** 2
        h11 = s ** 3 - s ** 2
        return h00 * x0 + h10 * v[i] + h01 * x1 + h11 * v[i + 1]
    # quintic Hermite basis on [0, 1]: value, first and second derivative at both ends
    s2, s3, s4, s5 = s * s, s ** 3, s ** 4, s ** 5
    h0 = 1 - 10 * s3 + 15 * s4 - 6 * s5
    h1 = s - 6 * s3 + 8 * s4 - 3 * s5
    h2 = 0.5 * s2 - 1.5 * s3 + 1.5 * s4 - 0.5 * s5
    h5 = 10 * s3 - 15 * s4 + 6 * s5
    h4 = -4 * s3 + 7 * s4 - 3 * s5
    h3 = 0.5 * s3 - s4 + 0.5 * s5
    return h0 * x0 + h1 * v[i] + h2 * a[i] + h5 * x1 + h4 * v[i + 1] + h3 * a[i + 1]


def interpolate(series, d, t, kind="c2"):
    """Value at times t (array, 0 <= t <= (n-1) d) of a series sampled every d (App. C: c0, c1, c2)."""
    x = np.asarray(series)
    n = x.shape[0]
    t = np.asarray(t, dtype=np.float64)
    i = np.clip(np.floor(t / d).astype(int), 0, n - 2)
    s = (t - i * d) / d                                   # in [0, 1]
    return hermite_eval(hermite_data(x, d, kind), i, s, kind)


# ---------------------------------------------------------------------------
# FIR filtering (App. B)
# ---------------------------------------------------------------------------
def fir_design(order, dt, amp_fn, two_sided=False):
    """Order-`order` (even) linear-phase FIR filter with amplitude response amp_fn(w), by frequency
    sampling with a Hamming window.  One-sided (default): amp_fn on w in [0, pi/dt], mirrored to
    negative w, real taps.  Two-sided: amp_fn on signed w in (-pi/dt, pi/dt], complex taps (a complex
    signal's spectrum need not be symmetric in w).  Returns the order + 1 taps."""
    if order % 2:
        raise ValueError("order must be even (integer delay order / 2)")
    ntap = order + 1
    nfft = 8 * ntap
    if not two_sided:
        w = np.arange(nfft // 2 + 1) * (2 * np.pi / (nfft * dt))
        spec = amp_fn(w) * np.exp(-1j * w * (order / 2) * dt)       # linear phase: delay order/2 samples
        taps = np.fft.irfft(spec, nfft)[:ntap]
        return taps * np.hamming(ntap)
    m = np.arange(nfft)
    w = np.where(m <= nfft // 2, m, m - nfft) * (2 * np.pi / (nfft * dt))   # signed grid frequencies
    spec = amp_fn(w) * np.exp(-1j * w * (order / 2) * dt)
    taps = np.fft.ifft(spec)[:ntap]
    return taps * np.hamming(ntap)


def fir_design_points(order, dt, w_pts, amp_pts):
    """fir_design with the amplitude given at points (ascending w_pts), linearly interpolated between
    them and held constant beyond the first and last; two-sided when any point is negative."""
    w_pts = np.asarray(w_pts, dtype=np.float64)
    amp_pts = np.asarray(amp_pts, dtype=np.float64)
    two = bool((w_pts < 0).any())
    return fir_design(order, dt, lambda w: np.interp(w, w_pts, amp_pts), two_sided=two)


def fir_apply(taps, series, full=False):
    """x' = phi * x along the first axis (App. B).  Default: the delay of order/2 samples removed and
    the output cut to the input's length.  full=True: the whole convolution, n + order samples,
    out[m] = sum_j phi_j x[m - j]; sample m belongs to time (m - order/2) d once the delay is
    compensated, and the output decays at both ends as the input does (nothing is cut off)."""
    order = len(taps) - 1
    x = np.asarray(series)
    n = x.shape[0]
    base = 0 if full else order // 2
    m_out = n + order if full else n
    out = np.zeros((m_out,) + x.shape[1:], dtype=np.result_type(x, taps))
    for j, c in enumerate(taps):                 # out[i] += c_j x[i + base - j] where in range
        shift = base - j
        lo, hi = max(0, -shift), min(m_out, n - shift)
        if lo < hi:
            out[lo:hi] += c * x[lo + shift:hi + shift]
    return out


def fir_response(taps, dt, omegas):
    """Frequency response of the delay-compensated filter at w: sum_j phi_j exp(-i w (j - order/2) dt)."""
    order = len(taps) - 1
    j = np.arange(len(taps)) - order / 2
    return np.exp(-1j * np.outer(omegas, j * dt)) @ taps


# ---------------------------------------------------------------------------
# runs driven by a sampled series (Sec. 2.2 with App. C)
# ---------------------------------------------------------------------------
def series_forcing(series, every, kind="c2"):
    """Forcing at every half step q = 0 .. 2 every (n_in - 1) (t = q h / 2) from a series sampled every
    `every` steps: the App. C interpolant between samples and the last sample at its own time; zero
    after it (not returned).  Returns [2 every (n_in - 1) + 1][k][n]."""
    x = np.asarray(series, dtype=np.complex128)
    n_in = x.shape[0]
    span = 2 * every
    if n_in == 1:
        return x[:1].copy()
    q = np.arange(span * (n_in - 1))
    i, r = np.divmod(q, span)
    body = hermite_eval(hermite_data(x, 1.0, kind), i, r / span, kind)
    return np.concatenate([body, x[-1:]], axis=0)


def series_march(a, h, every, n_snap_max, *, init=None, forcing=None, kind="c2", adjoint=False,
                 tail_tol=0.0, scheme="rk4"):
    """March du/dt = A u + g(t) (A^H for the adjoint run) from u(0) = init (zero if None), g from the
    sampled series `forcing` [n_in][k][n] (samples every `every` steps, first at t = 0; zero after the
    last).  Records u every `every` steps: snapshot j is u(j every h), snapshot 0 the initial state.

    Truncation (Sec. 2.2, "until the norm is negligible"): with tail_tol > 0 vector v stops at the
    first snapshot j at or after the end of its forcing (j >= n_in - 1) whose norm is at most
    tail_tol times the largest norm of its snapshots 0..j; its later snapshots are zero.  The record
    ends when every vector has stopped (length max stop + 1) or at n_snap_max snapshots.

    Returns the snapshots [n_out][k][n] complex128.
    """
    from . import march as _m
    op = a.conj().T if adjoint else a
    if init is not None:
        k, n = np.asarray(init).shape
    else:
        _, k, n = np.asarray(forcing).shape
    u = np.zeros((n, k), dtype=np.complex128) if init is None else np.array(init, dtype=np.complex128).T
    n_in = 0 if forcing is None else forcing.shape[0]
    gq = series_forcing(forcing, every, kind) if n_in else np.zeros((0, k, n), dtype=np.complex128)
    zero = np.zeros((n, k), dtype=np.complex128)

    def g(q):
        return gq[q].T if q < len(gq) else zero

    lu = _m.cn_factor(op, h) if scheme == "cn" else None
    snaps = [u.T.copy()]
    nrm = np.linalg.norm(u, axis=0)
    peak = nrm.copy()
    stop = [None] * k
    j_end = max(n_in - 1, 0)
    if tail_tol > 0:
        for v in range(k):
            if j_end == 0 and nrm[v] <= tail_tol * peak[v]:
                stop[v] = 0
    s = 0
    while len(snaps) < n_snap_max and not (tail_tol > 0 and all(x is not None for x in stop)):
        if scheme == "cn":
            u = _m.cn_step(lu, u, h, g(2 * s), g(2 * s + 2))
        else:
            u = _m.rk4_step(op, u, h, g(2 * s), g(2 * s + 1), g(2 * s + 2))
        s += 1
        if s % every:
            continue
        j = s // every
        snaps.append(u.T.copy())
        nrm = np.linalg.norm(u, axis=0)
        peak = np.maximum(peak, nrm)
        if tail_tol > 0 and j >= j_end:
            for v in range(k):
                if stop[v] is None and nrm[v] <= tail_tol * peak[v]:
                    stop[v] = j
    out = np.array(snaps)
    if tail_tol > 0 and all(x is not None for x in stop):
        out = out[:max(stop) + 1]
        for v in range(k):
            out[stop[v] + 1:, v] = 0.0
    return out


def trm_power_iteration(a, h, f0, every, n_iter, omegas, *, kind="c2", scheme="rk4", tail_tol=1e-9,
                        n_snap_max=100000, filter_order=0):
    """Power iteration on R^H R with the transient-response method (Sec. 2.2, App. A Eq. (iteration)).

    Iteration n, for each of the k test vectors independently:
      direct run   forcing f_n(t): the impulse f0 delta(t) as the initial condition u(0) = f0 (n = 0),
                   else the series g_n; output y_n(t) sampled every `every` steps until negligible;
      adjoint run  forced by y_n reversed in time (the adjoint equation runs backward in time);
                   its output reversed back is w_n(t), with w_hat_n = R^H R f_hat_n;
      gains        sigma_n(w)^2 = |w_hat_n(w)| / |f_hat_n(w)| (Eq. (tildeSig)), Fourier transforms
                   at the requested w by the rectangle rule on the samples (f_hat_0 = f0);
      next forcing g_{n+1} = w_n filtered by the order-`filter_order` FIR filter whose amplitude is
                   1 / |w_hat_n(w)| at the requested w (App. B: flattens the spectrum, Sec. 2.2), the
                   whole convolution kept so that g_{n+1} decays at both ends as w_n does; or, with
                   filter_order = 0, w_n scaled by 1 / max_w |w_hat_n(w)| (no flattening).
    Returns (sigma [n_iter][n_omega][k], w_hat of the last iteration [n_omega][k][n]).
    """
    d = every * h
    f0 = np.asarray(f0, dtype=np.complex128)
    k = f0.shape[0]
    omegas = np.asarray(omegas, dtype=np.float64)
    sig = np.zeros((n_iter, len(omegas), k))
    g = None
    f_hat = np.broadcast_to(f0, (len(omegas),) + f0.shape)
    w_hat = None
    for it in range(n_iter):
        y = series_march(a, h, every, n_snap_max, init=f0 if g is None else None, forcing=g, kind=kind,
                         tail_tol=tail_tol, scheme=scheme)
        z = series_march(a, h, every, n_snap_max, forcing=y[::-1], kind=kind, adjoint=True,
                         tail_tol=tail_tol, scheme=scheme)
        w = z[::-1]
        w_hat = fourier(w, np.arange(len(w)) * d, omegas)
        nw = np.linalg.norm(w_hat, axis=2)
        nf = np.linalg.norm(f_hat, axis=2)
        sig[it] = np.sqrt(nw / nf)
        if filter_order:
            g = np.zeros((len(w) + filter_order,) + w.shape[1:], dtype=np.complex128)
            order = np.argsort(omegas)
            for v in range(k):
                taps = fir_design_points(filter_order, d, omegas[order], 1.0 / nw[order, v])
                g[:, v] = fir_apply(taps, w[:, v], full=True)
        else:
            g = w / nw.max(axis=0)[None, :, None]
        f_hat = fourier(g, np.arange(len(g)) * d, omegas)
    return sig, w_hat
