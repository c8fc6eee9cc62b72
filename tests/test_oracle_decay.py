"""Pins of the oracle's decay run (Sec. 2.3: transient length from the decay of a random state).

The probe's step count is checked against the closed form of the RK4
amplification |P(h lambda)|^s, P(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, for
diagonal and normal systems; growth and the step cap are checked on systems
that do not decay; the SplitMix64 generator against its published test
vector; and the SSRM schedule the probe sets against the closed-form RK4
resolvent.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import decay, frequencies, march, operators, resolvent


def _p4(z):
    return 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24


def _closed_form_steps(lam, c, h, tol, check_every, cap=10 ** 6):
    """First multiple of check_every with sqrt(sum |P(h lam_i)|^(2s) |c_i|^2) <= tol ||c||."""
    amp2 = np.abs(_p4(h * lam)) ** 2
    n0 = np.linalg.norm(c)
    for s in range(check_every, cap, check_every):
        if math.sqrt(float(np.sum(amp2 ** s * np.abs(c) ** 2))) <= tol * n0:
            return s
    raise AssertionError("no decay")


def test_splitmix64_published_vector():
    # reference output of SplitMix64 seeded with 1234567 (first five values)
    assert [int(v) for v in decay.splitmix64(1234567, 5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
        16408922859458223821]


def test_initial_state_layout_and_range():
    u = decay.uniform_pm1(99, 10000)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.05
    # exact in binary64: 2 (z >> 11) 2^-53 - 1 is a multiple of 2^-52
    assert np.all(np.ldexp(u + 1.0, 52) == np.round(np.ldexp(u + 1.0, 52)))
    c = decay.initial_state(7, 5, True)
    v = decay.uniform_pm1(5, 14)
    assert np.array_equal(c.real, v[0::2]) and np.array_equal(c.imag, v[1::2])
    assert np.array_equal(decay.initial_state(7, 5, False), decay.uniform_pm1(5, 7))


@pytest.mark.parametrize("check_every", [1, 7, 50])
def test_decay_steps_diagonal_closed_form(check_every):
    lam = np.array([-0.05 + 0.3j, -0.2, -0.02 - 1.0j, -1.5 + 0.2j])
    h, tol = 0.05, 1e-6
    u0 = decay.initial_state(4, 11, True)
    steps, ratio, status = decay.decay_probe(np.diag(lam), h, u0, tol, 10 ** 6, check_every)
    assert status == "decayed" and ratio <= tol
    assert steps == _closed_form_steps(lam, u0, h, tol, check_every)


def test_decay_steps_normal_matrix_closed_form():
    """A = Q diag(lam) Q^H: the norm decays as that of the coefficients Q^H u0."""
    rng = np.random.default_rng(2)
    q, _ = np.linalg.qr(rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6)))
    lam = -np.linspace(0.03, 0.8, 6) + 1j * np.linspace(-1, 1, 6)
    a = q @ np.diag(lam) @ q.conj().T
    u0 = decay.initial_state(6, 3, True)
    h, tol = 0.1, 1e-8
    steps, _, status = decay.decay_probe(a, h, u0, tol, 10 ** 6, 4)
    assert status == "decayed"
    assert steps == _closed_form_steps(lam, q.conj().T @ u0, h, tol, 4)


def test_decay_steps_per_instance_closed_form():
    """A batched system decays only when every block has: the slowest block sets the length, even
    when its share of the total norm is small."""
    lam_a = np.array([-0.5 + 0.2j, -0.8])          # fast block
    lam_b = np.array([-0.03 + 0.1j])               # slow block
    a = np.diag(np.concatenate([lam_a, lam_b]))
    u0 = np.array([1.0, 1.0, 1e-3])                 # the slow block starts small
    h, tol = 0.1, 1e-6
    steps, _, status = decay.decay_probe(a, h, u0, tol, 10 ** 6, 5, instances=[(0, 2), (2, 1)])
    assert status == "decayed"
    assert steps == max(_closed_form_steps(lam_a, u0[:2], h, tol, 5), _closed_form_steps(lam_b, u0[2:], h, tol, 5))
    whole, _, _ = decay.decay_probe(a, h, u0, tol, 10 ** 6, 5)
    assert whole < steps                            # the whole-vector ratio would stop too early


def test_decay_probe_reports_growth_and_cap():
    grow = np.diag([0.05, -0.3])
    steps, ratio, status = decay.decay_probe(grow, 0.1, np.array([1.0, 1.0]), 1e-6, 10 ** 6, 10)
    assert status == "grew" and ratio > 1e6 and steps % 10 == 0
    # closed form: the ratio first exceeds 1e6 between the previous check point and this one
    amp = np.abs(_p4(0.1 * np.array([0.05, -0.3])))
    closed = lambda s: math.sqrt(float(np.sum(amp ** (2 * s)))) / math.sqrt(2.0)
    assert closed(steps - 10) <= 1e6 < closed(steps)
    assert abs(closed(steps) / ratio - 1.0) < 1e-12
    slow = np.diag([-1e-4])
    steps, ratio, status = decay.decay_probe(slow, 0.1, np.array([1.0]), 1e-6, 500, 10)
    assert status == "cap" and steps == 500 and 0.99 < ratio < 1.0


def test_probe_sets_ssrm_transient_length():
    """With the windows the probe sets, SSRM's leakage against R_h fhat is of the order of tol;
    with one window fewer it is not (the probe is not overly generous either)."""
    w = W.small_gl(n=24, k=2, mu0=0.1)
    a = operators.gl1d(w.system)
    g = frequencies.make_grid(w.omegas, w.dt)
    tol = 1e-6
    steps, _, status = decay.decay_probe(a, g.h, decay.initial_state(w.n, 2008, True), tol, 10 ** 6, 1)
    assert status == "decayed"
    n_trans = decay.transient_windows(steps, g.n_t)
    assert (n_trans - 1) * g.n_t < steps <= n_trans * g.n_t
    fh = W.test_block(w)
    ref = np.stack([(resolvent.rk4_discrete(a, om, g.h) @ fh[j].T).T for j, om in enumerate(g.omegas)])
    err = lambda nt: np.abs(march.march(a, g, fh, variant="ssrm", n_trans=nt) - ref).max() / np.abs(ref).max()
    assert err(n_trans) < 50 * tol
    assert err(n_trans - 1) > err(n_trans)


def test_transient_windows_rounds_up():
    assert decay.transient_windows(1, 100) == 1
    assert decay.transient_windows(100, 100) == 1
    assert decay.transient_windows(101, 100) == 2
    assert decay.transient_windows(0, 100) == 0
