"""Pins of the oracle's forcing / observation matrices and metrics (Sec. 2.1).

* The direct run returns C R_h B fhat (closed-form RK4 resolvent).
* The adjoint run is the adjoint of the direct run in the weighted inner
  products <a, b>_W = a^H W b of Sec. 2.1: <yhat, R_y fhat>_{W_y} =
  <R_y^dag yhat, fhat>_{W_f} for arbitrary blocks.
* The weighted randomized SVD with a full-rank sketch returns the singular
  values of W_y^{1/2} C R_h B W_f^{-1/2}; its leading forcing mode attains the
  gain ||R_y v||_{W_y} / ||v||_{W_f} = sigma_1, which no random forcing exceeds.
* With B = C = W = I everything reduces to the unweighted runs.
"""
import numpy as np
import pytest

import workloads as W
from oracle import frequencies, march, operators, resolvent, rsvd, weighted


def _system(n=10):
    w = W.small_gl(n=n, k=n, n_omega=4, mu0=-0.3)
    a = operators.gl1d(w.system)
    g = frequencies.make_grid(w.omegas, w.dt)
    rng = np.random.default_rng(8)
    b = np.where(rng.random(n) < 0.3, 0.0, rng.uniform(0.5, 2.0, n))    # forcing mask / weights
    c = np.where(rng.random(n) < 0.3, 0.0, rng.uniform(0.5, 2.0, n))    # observation mask / weights
    w_f = rng.uniform(0.2, 3.0, n)
    w_y = rng.uniform(0.2, 3.0, n)
    return w, a, g, b, c, w_f, w_y


def _rh(a, g):
    return [resolvent.rk4_discrete(a, om, g.h) for om in g.omegas]


def test_direct_and_adjoint_closed_forms():
    w, a, g, b, c, w_f, w_y = _system()
    fh = W.test_block(w)
    y = weighted.march_direct(a, g, fh, b, c, variant="ssrm", n_trans=12)
    yy = weighted.march_adjoint(a, g, fh, b, c, w_f, w_y, variant="ssrm", n_trans=12)
    for j, r in enumerate(_rh(a, g)):
        ry = np.diag(c) @ r @ np.diag(b)
        ref = (ry @ fh[j].T).T
        assert np.abs(y[j] - ref).max() < 1e-12 * np.abs(ref).max()
        refa = (np.diag(1 / w_f) @ ry.conj().T @ np.diag(w_y) @ fh[j].T).T
        assert np.abs(yy[j] - refa).max() < 1e-12 * np.abs(refa).max()


def test_adjoint_identity_in_weighted_inner_products():
    w, a, g, b, c, w_f, w_y = _system()
    f = W.gaussian_block(1, 4, 3, w.n)
    q = W.gaussian_block(2, 4, 3, w.n)
    kw = dict(variant="ssrm", n_trans=12)
    rf = weighted.march_direct(a, g, f, b, c, **kw)
    rq = weighted.march_adjoint(a, g, q, b, c, w_f, w_y, **kw)
    for j in range(4):
        for m in range(3):
            lhs = np.vdot(q[j, m], w_y * rf[j, m])        # <q, R_y f>_{W_y}
            rhs = np.vdot(rq[j, m], w_f * f[j, m])        # <R_y^dag q, f>_{W_f}
            assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)


def test_weighted_rsvd_equals_svd_of_scaled_resolvent():
    w, a, g, b, c, w_f, w_y = _system()
    b = np.abs(b) + 0.3       # full-rank forcing and observation for this pin
    c = np.abs(c) + 0.3
    kw = dict(variant="ssrm", n_trans=12)
    gains, v, u = weighted.weighted_rsvd(a, g, W.test_block(w), b, c, w_f, w_y, 0, 3, **kw)
    for j, r in enumerate(_rh(a, g)):
        rt = np.diag(np.sqrt(w_y) * c) @ r @ np.diag(b / np.sqrt(w_f))
        s = np.linalg.svd(rt, compute_uv=False)
        assert np.allclose(gains[0, j], s[:3], rtol=1e-10)
        ry = np.diag(c) @ r @ np.diag(b)
        v1, u1 = v[0][j][0], u[0][j][0]
        assert abs(np.vdot(v1, w_f * v1).real - 1.0) < 1e-10          # unit in the W_f norm
        assert abs(np.vdot(u1, w_y * u1).real - 1.0) < 1e-10          # unit in the W_y norm
        r1 = ry @ v1
        gain = np.sqrt(np.vdot(r1, w_y * r1).real / np.vdot(v1, w_f * v1).real)
        assert abs(gain - s[0]) < 1e-10 * s[0]
        assert np.abs(r1 - s[0] * u1).max() < 1e-9 * np.abs(r1).max()    # R_y v = sigma u
        rng = np.random.default_rng(j)
        for _ in range(20):                                              # optimality of v1
            f = rng.standard_normal(w.n) + 1j * rng.standard_normal(w.n)
            rf = ry @ f
            assert np.sqrt(np.vdot(rf, w_y * rf).real / np.vdot(f, w_f * f).real) <= s[0] * (1 + 1e-12)


def test_masked_forcing_limits_the_rank():
    """A forcing mask with m active points leaves at most m non-zero gains."""
    w, a, g, b, c, w_f, w_y = _system()
    b = np.zeros(w.n)
    b[[1, 4]] = 1.0
    gains, _, _ = weighted.weighted_rsvd(a, g, W.test_block(w), b, c + 0.3, w_f, w_y, 0, 4,
                                         variant="ssrm", n_trans=12)
    assert np.all(gains[0, :, 2:] < 1e-12 * gains[0, :, :1])
    assert np.all(gains[0, :, 1] > 1e-6 * gains[0, :, 0])


def test_identity_weights_reduce_to_plain_runs():
    w, a, g, b, c, w_f, w_y = _system()
    one = np.ones(w.n)
    fh = W.test_block(w)
    kw = dict(variant="ssrm", n_trans=12)
    assert np.array_equal(weighted.march_direct(a, g, fh, one, one, **kw), march.march(a, g, fh, **kw))
    assert np.array_equal(weighted.march_adjoint(a, g, fh, one, one, one, one, **kw),
                          march.march(a, g, fh, adjoint=True, **kw))
    g1, _, _ = weighted.weighted_rsvd(a, g, fh, one, one, one, one, 1, 3, **kw)
    g0, _, _ = rsvd.block_rsvd(lambda x: march.march(a, g, x, **kw),
                               lambda x: march.march(a, g, x, adjoint=True, **kw), fh, 1, 3)
    assert np.allclose(g1, g0, rtol=1e-12)
