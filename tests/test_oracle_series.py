"""Pins of the oracle's time-series tools: snapshot interpolation (App. C), FIR filtering (App. B),
and Fourier transforms of an impulse response (Sec. 2.1, 2.2).

* Interpolation reproduces polynomials exactly up to the degree its
  derivative stencils are exact for: C0 linear, C1 quadratic, C2 quartic
  (away from the edges, where the App. C edge rules lower the order).
* The paper's own statements about a sinusoid: with C2 about 4.5 points per
  cycle give errors of the order 1e-2, and n points per cycle put the first
  spurious spectral peak at n - 1 times the signal frequency.
* FIR: the taps of a linear-phase filter are symmetric, its delay-compensated
  response is real and follows the design amplitude; filtering a sinusoid
  scales it by the amplitude at its frequency.
* The Fourier transform of the sampled impulse response equals its closed
  form every h (I - M^every e^{-i w every h})^{-1} f0.
"""
import numpy as np
import pytest

import workloads as W
from oracle import frequencies, operators, series


@pytest.mark.parametrize("kind,deg", [("c0", 1), ("c1", 2), ("c2", 4)])
def test_interpolation_exact_for_low_degree(kind, deg):
    d = 0.3
    t_s = np.arange(20) * d
    coef = np.array([0.7, -1.1, 0.4, 0.25, -0.05][:deg + 1])
    x = np.polyval(coef, t_s)
    t = np.linspace(3 * d, 16 * d, 101)                   # interior intervals (edges two samples away)
    got = series.interpolate(x, d, t, kind)
    assert np.abs(got - np.polyval(coef, t)).max() < 1e-11
    if kind != "c0":                                      # one degree more is no longer exact
        coef2 = np.concatenate([[0.3], coef])
        x2 = np.polyval(coef2, t_s)
        assert np.abs(series.interpolate(x2, d, t, kind) - np.polyval(coef2, t)).max() > 1e-8


def _sine_error(ppc, kind, cycles=40):
    om = 1.0
    d = 2 * np.pi / (om * ppc)
    t_s = np.arange(int(cycles * ppc) + 1) * d
    x = np.sin(om * t_s)
    t = np.linspace(5 * d, t_s[-6], 4001)
    err = series.interpolate(x, d, t, kind) - np.sin(om * t)
    return np.sqrt(np.mean(err ** 2)) / np.sqrt(0.5)


def test_paper_interpolation_accuracy_statement():
    """App. C: to obtain errors of the order 1e-2 about 4.5 points per cycle should be used (C2)."""
    e = _sine_error(4.5, "c2")
    assert 3e-3 < e < 3e-2, e
    assert _sine_error(4.5, "c0") > 5 * e              # the smoother interpolants do better
    assert _sine_error(9.0, "c2") < 0.1 * e            # and the error falls quickly with resolution


@pytest.mark.parametrize("ppc", [3, 4, 5])
def test_first_spurious_peak_at_n_minus_one(ppc):
    """App. C: a signal interpolated from n points per cycle shows its first spurious peak at (n - 1) f."""
    om = 1.0
    d = 2 * np.pi / (om * ppc)
    cycles = 64
    t_s = np.arange(cycles * ppc + 6) * d
    x = np.cos(om * t_s)
    fine = 32
    t = np.arange(cycles * ppc * fine) * (d / fine) + 2 * d
    y = series.interpolate(x, d, t, "c2")
    spec = np.abs(np.fft.rfft(y * np.hanning(len(y))))
    freqs = np.fft.rfftfreq(len(y), d / fine) * 2 * np.pi
    base = np.argmin(np.abs(freqs - om))
    spec[max(0, base - 8):base + 9] = 0.0                 # remove the signal's own peak
    peak = freqs[np.argmax(spec)]
    assert abs(peak / om - (ppc - 1)) < 0.1, (peak, ppc)


def test_fir_linear_phase_and_amplitude():
    dt = 0.05
    amp = lambda w: 1.0 / (1.0 + (w / 10.0) ** 2)          # a smooth flattening target
    taps = series.fir_design(200, dt, amp)
    assert np.allclose(taps, taps[::-1], atol=1e-15)         # symmetric: linear phase
    w = np.linspace(0.0, 0.8 * np.pi / dt, 50)
    r = series.fir_response(taps, dt, w)
    assert np.abs(r.imag).max() < 1e-12                       # delay removed: real response
    assert np.abs(r.real - amp(w)).max() < 2e-2
    # a sinusoid comes out scaled by the amplitude at its frequency (away from the edges)
    om = 7.0
    t = np.arange(4000) * dt
    y = series.fir_apply(taps, np.cos(om * t))
    mid = slice(300, 3700)
    scale = series.fir_response(taps, dt, np.array([om]))[0].real
    assert np.abs(y[mid] - scale * np.cos(om * t[mid])).max() < 1e-12 + 1e-10


def test_impulse_response_transform_closed_form():
    w = W.small_gl(n=16, k=2, mu0=-0.3)
    a = operators.gl1d(w.system).toarray()
    h = 0.05
    f0 = W.gaussian_block(4, 1, 2, 16)[0]
    for every in (1, 3):
        times, snaps = series.impulse_response(a, h, f0, 6000, every)
        om = np.array([-0.7, 0.0, 0.4, 1.3])
        got = series.fourier(snaps, times, om)               # [n_omega][k][n]
        for j, o in enumerate(om):
            ref = (series.discrete_impulse_transform(a, h, o, every) @ f0.T).T
            assert np.abs(got[j] - ref).max() < 1e-10 * np.abs(ref).max(), (every, o)


# ---------------------------------------------------------------------------
# runs driven by sampled series, and the TRM power iteration (Sec. 2.2, App. A-C)
# ---------------------------------------------------------------------------
def _gl(n=60):
    w = W.gl_paper(n=n)
    return operators.gl1d(w.system)


@pytest.mark.parametrize("scheme", ["rk4", "cn"])
@pytest.mark.parametrize("kind", ["c0", "c1", "c2"])
def test_series_march_linear_forcing_is_exact(scheme, kind):
    """A forcing linear in time is reproduced exactly by every interpolant (edge rules included), so
    the series-driven march equals the march with the analytic forcing, zero after the last sample."""
    from oracle import march
    a = _gl()
    n, k, h, every, n_in = a.shape[0], 2, 0.01, 3, 9
    rng = np.random.default_rng(3)
    al = rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))
    be = rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))
    t_end = (n_in - 1) * every * h
    samples = np.array([al + be * (i * every * h) for i in range(n_in)])
    got = series.series_march(a, h, every, 14, forcing=samples, kind=kind, scheme=scheme)
    f = lambda t: ((al + be * t).T if t <= t_end + 1e-12 else np.zeros((n, k)))
    u = np.zeros((n, k), dtype=np.complex128)
    ref = [u.T.copy()]
    lu = march.cn_factor(a, h) if scheme == "cn" else None
    for s in range(13 * every):
        t = s * h
        u = (march.cn_step(lu, u, h, f(t), f(t + h)) if scheme == "cn"
             else march.rk4_step(a, u, h, f(t), f(t + 0.5 * h), f(t + h)))
        if (s + 1) % every == 0:
            ref.append(u.T.copy())
    ref = np.array(ref)
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_series_march_impulse_and_truncation():
    """u(0) = f0 and no forcing: snapshot j is M^(j every) f0 (M the RK4 step polynomial of hA); the
    record stops per vector at the first snapshot whose norm is at most tol times its running peak."""
    a = _gl()
    n, h, every = a.shape[0], 0.01, 4
    f0 = W.gaussian_block(5, 1, 2, n)[0]
    f0[1] *= 1e-3                                          # a second vector with another scale
    tol = 1e-6
    got = series.series_march(a, h, every, 100000, init=f0, tail_tol=tol)
    b = h * a.toarray()
    m = np.eye(n) + b + b @ b / 2 + b @ b @ b / 6 + b @ b @ b @ b / 24
    me = np.linalg.matrix_power(m, every)
    snaps = [f0.T]
    for _ in range(len(got) - 1):
        snaps.append(me @ snaps[-1])
    ref = np.array(snaps).transpose(0, 2, 1)
    nrm = np.linalg.norm(ref, axis=2)
    peak = np.maximum.accumulate(nrm, axis=0)
    stops = [int(np.argmax(nrm[:, v] <= tol * peak[:, v])) for v in range(2)]
    assert len(got) == max(stops) + 1
    for v in range(2):
        assert nrm[stops[v], v] <= tol * peak[stops[v], v] and (nrm[:stops[v], v] > tol * peak[:stops[v], v]).all()
        assert np.abs(got[:stops[v] + 1, v] - ref[:stops[v] + 1, v]).max() < 1e-12 * np.abs(ref[:, v]).max()
        assert not got[stops[v] + 1:, v].any()


def test_reversed_adjoint_run_gives_rhr():
    """Sec. 2.1/2.2: the adjoint run forced by the direct output reversed in time, reversed back, has
    the Fourier transform R(w)^H R(w) f_hat(w), R(w) = (i w I - A)^-1, for a smooth compact forcing."""
    from oracle import resolvent
    a = _gl(60)
    n, h, every = a.shape[0], 0.01, 5
    d = every * h
    sp = W.gaussian_block(8, 1, 1, n)[0, 0]
    t = np.arange(int(6.0 / d) + 1) * d
    g = (np.exp(-((t - 3.0) / 0.7) ** 2) * np.exp(2j * t))[:, None, None] * sp[None, None, :]
    y = series.series_march(a, h, every, 100000, forcing=g, tail_tol=1e-13)
    z = series.series_march(a, h, every, 100000, forcing=y[::-1], adjoint=True, tail_tol=1e-13)
    w = z[::-1]
    # the adjoint run's time tau = T_y - t, T_y = (len(y) - 1) d: w[i] lies at t = (i - len(z) + len(y)) d
    om = np.array([0.0, 2.0, 5.0, -2.0])
    gh = series.fourier(g, t, om)
    wh = series.fourier(w, (np.arange(len(w)) - len(z) + len(y)) * d, om)
    ad = a.toarray()
    for j, o in enumerate(om):
        r = resolvent.continuous(ad, o)
        ref = r.conj().T @ (r @ gh[j, 0])
        assert np.linalg.norm(wh[j, 0] - ref) < 1e-5 * np.linalg.norm(ref), o


def test_fir_two_sided_design_and_full_convolution():
    dt, order = 0.05, 120
    sym = lambda w: 1.0 / (1.0 + (w / 8.0) ** 2)
    real = series.fir_design(order, dt, sym)
    two = series.fir_design(order, dt, sym, two_sided=True)
    assert np.abs(two - real).max() < 1e-14 and np.abs(two.imag).max() < 1e-14
    skew = lambda w: np.interp(w, [-60.0, -10.0, 0.0, 10.0, 60.0], [0.2, 0.4, 1.0, 2.0, 2.5])
    taps = series.fir_design(order, dt, skew, two_sided=True)
    w = np.linspace(-50.0, 50.0, 41)
    r = series.fir_response(taps, dt, w)
    assert np.abs(r.imag).max() < 2e-2 and np.abs(r.real - skew(w)).max() < 6e-2
    pts = series.fir_design_points(order, dt, [-10.0, 0.0, 10.0], [0.4, 1.0, 2.0])
    assert np.abs(pts - series.fir_design(order, dt, lambda x: np.interp(x, [-10.0, 0.0, 10.0], [0.4, 1.0, 2.0]),
                                          two_sided=True)).max() == 0.0
    x = np.random.default_rng(1).standard_normal((300, 2)) + 0j
    full = series.fir_apply(taps, x, full=True)
    assert full.shape == (300 + order, 2)
    for c in range(2):
        assert np.abs(full[:, c] - np.convolve(x[:, c], taps)).max() < 1e-12


def test_trm_power_iteration_paper_gl_filter():
    """Sec. 3 (Figs. of the gains with and without normalisation): on the paper's Ginzburg-Landau case
    the TRM power iteration without spectral flattening converges at low frequencies but the weak
    high-frequency components are swamped by the strong ones within a few iterations (their
    estimates drift towards the largest gain); with the FIR flattening filter every frequency
    converges, at the power-iteration rate (sigma_2 / sigma_1)^4 per iteration (App. A), and the
    final w_hat is the leading force mode."""
    from oracle import resolvent
    w = W.gl_paper(n=100)
    a = operators.gl1d(w.system)
    ad = a.toarray()
    om = np.array([0.0, 3.0, 6.0, 9.0, 12.0, 15.0])
    svd = [np.linalg.svd(resolvent.continuous(ad, o)) for o in om]
    s1 = np.array([x[1][0] for x in svd])
    s2 = np.array([x[1][1] for x in svd])
    f0 = W.gaussian_block(11, 1, 1, a.shape[0])[0]
    kw = dict(tail_tol=1e-9, n_snap_max=20000)
    raw, _ = series.trm_power_iteration(a, 0.01, f0, 5, 4, om, filter_order=0, **kw)
    flt, wh = series.trm_power_iteration(a, 0.01, f0, 5, 5, om, filter_order=600, **kw)
    e_raw = np.abs(raw[:, :, 0] / s1 - 1)
    e_flt = np.abs(flt[:, :, 0] / s1 - 1)
    assert e_raw[-1, 0] < 1e-8 and e_flt[-1, 0] < 1e-8              # the dominant frequency either way
    assert e_raw[-1, -1] > 10.0                                      # w = 15 swamped without the filter
    assert (e_flt[-1] < 3e-2).all()                                  # every frequency with it
    rate = e_flt[-1, -1] / e_flt[-2, -1]
    assert abs(rate / (s2[-1] / s1[-1]) ** 4 - 1) < 0.3, rate
    for j in range(4):                                               # converged frequencies: modes
        v1 = svd[j][2][0].conj()
        c = abs(np.vdot(v1, wh[j, 0])) / np.linalg.norm(wh[j, 0])
        assert 1 - c < 1e-6, (om[j], 1 - c)
