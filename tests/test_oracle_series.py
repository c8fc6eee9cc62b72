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
