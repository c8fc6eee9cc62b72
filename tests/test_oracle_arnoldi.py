"""Pins of the oracle's Krylov / Arnoldi gains (App. A) against direct SVDs and the power iteration.

* With as many iterations as unknowns the Krylov space is everything: the
  Arnoldi gains are svd(R_h) exactly.
* The Arnoldi projection H is Hermitian and Hessenberg, hence tridiagonal.
* The Krylov (plain power sequence + QR) and Arnoldi (orthogonalised)
  variants span the same space: the same Ritz values while F is well
  conditioned.
* For a few iterations the leading Arnoldi gain is at least as accurate as
  the power iteration's after the same number of runs, and it also gives
  suboptimal gains; its modes satisfy R v = sigma u.
"""
import numpy as np
import pytest

import workloads as W
from oracle import arnoldi, frequencies, march, operators, resolvent, rsvd


def _case(n=12, mu0=-0.3):
    w = W.small_gl(n=n, k=1, n_omega=4, mu0=mu0)
    a = operators.gl1d(w.system)
    g = frequencies.make_grid(w.omegas, w.dt)
    md = lambda b: march.march(a, g, b, variant="ssrm", n_trans=12)
    ma = lambda b: march.march(a, g, b, variant="ssrm", n_trans=12, adjoint=True)
    svs = [np.linalg.svd(resolvent.rk4_discrete(a, om, g.h)) for om in g.omegas]
    return w, md, ma, svs


def test_full_krylov_space_gives_exact_gains():
    w, md, ma, svs = _case(n=10)
    gains, v, u, _ = arnoldi.arnoldi(md, ma, W.test_block(w), 10, 4)
    for j, (uu, s, vh) in enumerate(svs):
        assert np.allclose(gains[j], s[:4], rtol=1e-9), (j, gains[j], s[:4])
        for m in range(4):
            assert abs(abs(np.vdot(v[j, m], vh[m].conj())) - 1) < 1e-7
            assert abs(abs(np.vdot(u[j, m], uu[:, m])) - 1) < 1e-7


def test_arnoldi_projection_is_hermitian_tridiagonal():
    w, md, ma, _ = _case()
    _, _, _, H = arnoldi.arnoldi(md, ma, W.test_block(w), 6, 2)
    for h in H:
        scale = np.abs(h).max()
        assert np.abs(h - h.conj().T).max() < 1e-10 * scale
        assert np.abs(np.triu(h, 2)).max() < 1e-10 * scale and np.abs(np.tril(h, -2)).max() < 1e-10 * scale


def test_krylov_and_arnoldi_share_ritz_values():
    w, md, ma, _ = _case()
    ga, _, _, _ = arnoldi.arnoldi(md, ma, W.test_block(w), 3, 3)
    gk, _, _, _ = arnoldi.arnoldi(md, ma, W.test_block(w), 3, 3, krylov=True)
    assert np.allclose(ga, gk, rtol=1e-8)


def test_arnoldi_beats_power_iteration_and_gives_suboptimals():
    w, md, ma, svs = _case(n=16, mu0=-0.2)
    f0 = W.test_block(w)
    ga, v, u, _ = arnoldi.arnoldi(md, ma, f0, 5, 2)
    gb, vb, ub, _ = arnoldi.arnoldi(md, ma, f0, 9, 2)
    hist, _ = rsvd.power_iteration(md, ma, f0, 5)
    for j, (_, s, _) in enumerate(svs):
        e_arn = abs(ga[j, 0] - s[0]) / s[0]
        e_pow = abs(hist[-1, j] - s[0]) / s[0]
        assert e_arn <= e_pow * 1.0001 + 1e-13, (j, e_arn, e_pow)
        # the suboptimal gain converges with the iterations
        assert abs(gb[j, 1] - s[1]) < abs(ga[j, 1] - s[1]) or abs(gb[j, 1] - s[1]) < 1e-10 * s[0]
        # modes: R v_1 = gamma_1 u_1 holds by the formula of u (the direct runs are kept), and the Ritz
        # residual ||R^H R v_1 - gamma_1^2 v_1|| shrinks with the iterations
        res = []
        for vv, uu, gg in ((v, u, ga), (vb, ub, gb)):
            blk = np.zeros((w.n_omega, 1, w.n), dtype=np.complex128)
            blk[j, 0] = vv[j, 0]
            ry = md(blk)
            assert np.linalg.norm(ry[j, 0] - gg[j, 0] * uu[j, 0]) < 1e-10 * gg[j, 0]
            rr = ma(ry)[j, 0]
            res.append(np.linalg.norm(rr - gg[j, 0] ** 2 * vv[j, 0]) / gg[j, 0] ** 2)
        assert res[1] < res[0] or res[1] < 1e-12, res
    assert np.allclose(np.linalg.norm(u, axis=2), 1.0, atol=1e-10)
