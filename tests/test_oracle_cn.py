"""Pins of the oracle's Crank-Nicolson march (the time scheme of the paper's Ginzburg-Landau case, Sec. 3).

* The SSRM and TRM marches return the exact discrete resolvent of the CN
  scheme, R_h(w) = (z I - M)^{-1} (I - hA/2)^{-1} (h/2)(1 + z) with
  M = (I - hA/2)^{-1}(I + hA/2), z = e^{i w h} (adjoint: its conjugate transpose).
* CN is second order: halving h cuts the error against R(w) about fourfold.
* The paper's case (U = 6, gamma = 1, mu = beta mu_c (1 - x/20), x in (0, 40))
  is stable and its operator matches the model's finite differences.
"""
import numpy as np
import pytest

import workloads as W
from oracle import frequencies, march, operators, resolvent


def _small(n=100, dt=0.05, **kw):
    w = W.gl_paper(n=n, n_omega=8, dt=dt)
    w = W.Workload(w.name, w.system, np.linspace(0.0, 3.5, 8), dt, 3, "ssrm", n_transient_windows=2,
                   seed=w.seed)
    return w, operators.gl1d(w.system), frequencies.make_grid(w.omegas, dt)


@pytest.mark.parametrize("variant,extra", [("ssrm", dict(n_trans=2)), ("trm", dict(tail_steps=3000))])
@pytest.mark.parametrize("adjoint", [False, True])
def test_cn_march_equals_discrete_resolvent(variant, extra, adjoint):
    w, a, g = _small()
    fh = W.test_block(w)
    y = march.march(a, g, fh, variant=variant, adjoint=adjoint, scheme="cn", **extra)
    for j, om in enumerate(g.omegas):
        r = resolvent.cn_discrete(a, om, g.h)
        if adjoint:
            r = resolvent.cn_discrete(a.conj().T, -om, g.h)
            # the adjoint run with A^H at -w is R_h(w)^H
            assert np.allclose(r, resolvent.cn_discrete(a, om, g.h).conj().T, atol=1e-13)
        ref = (r @ fh[j].T).T
        assert np.abs(y[j] - ref).max() < 1e-12 * np.abs(ref).max(), (j, variant)


def test_cn_second_order():
    errs = []
    for dt in (0.02, 0.01):
        w, a, g = _small(dt=dt)
        fh = W.test_block(w)
        y = march.march(a, g, fh, variant="ssrm", n_trans=2, scheme="cn")
        ref = np.stack([(resolvent.continuous(a, om) @ fh[j].T).T for j, om in enumerate(g.omegas)])
        errs.append(np.abs(y - ref).max() / np.abs(ref).max())
    assert 3.5 < errs[0] / errs[1] < 4.5, errs


def test_paper_case_operator():
    w = W.gl_paper()
    a = operators.gl1d(w.system).toarray()
    n = w.n
    dx = 40.0 / (n + 1)
    x = (np.arange(n) + 1) * dx
    mu = 0.1 * 36.0 * (1 - x / 20.0)
    assert np.allclose(np.diag(a).real, -2.0 / dx ** 2 + mu)
    assert np.allclose(np.diag(a, -1), 6.0 / (2 * dx) + 1.0 / dx ** 2)     # -U u_x + u_xx, upwind side
    assert np.allclose(np.diag(a, 1), -6.0 / (2 * dx) + 1.0 / dx ** 2)
    assert np.linalg.eigvals(a).real.max() < 0                               # globally stable at beta = 0.1
