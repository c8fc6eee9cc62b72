"""Pins of the oracle against what the paper and the mathematics fix.

Each test checks the oracle's time march against something other than
itself: the closed-form RK4 discrete resolvent, the continuous resolvent of
Sec. 2.1 Eq. (systemFreqDomain) with the RK4 error order, the exponential
decay of transients (Sec. 2.2/2.3), orthogonality of the Fourier series
(Sec. 2.3), realness for real systems, and brute-force SVDs (Sec. 2.1).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import frequencies, march, operators, resolvent, rsvd


def _small(**kw):
    w = W.small_gl(**kw)
    return w, operators.gl1d(w.system), frequencies.make_grid(w.omegas, w.dt)


def _apply_r(rmats, fh):
    return np.stack([(r @ fh[j].T).T for j, r in enumerate(rmats)])


@pytest.mark.parametrize("variant,extra", [("ssrm", dict(n_trans=12)), ("trm", dict(tail_steps=5280))])
@pytest.mark.parametrize("adjoint", [False, True])
def test_march_equals_discrete_resolvent(variant, extra, adjoint):
    """P1/P2: SSRM and TRM both return R_h(w) fhat (adjoint: R_h(w)^H fhat) exactly."""
    w, a, g = _small()
    fh = W.test_block(w)
    y = march.march(a, g, fh, variant=variant, adjoint=adjoint, **extra)
    rm = [resolvent.rk4_discrete(a, om, g.h) for om in g.omegas]
    if adjoint:
        rm = [r.conj().T for r in rm]
    ref = _apply_r(rm, fh)
    assert np.abs(y - ref).max() / np.abs(ref).max() < 1e-12


def test_rk4_order_to_continuous_resolvent():
    """P3: uhat = R(w) fhat (Sec. 2.1) is reached with the 4th-order error of RK4."""
    errs = []
    for dt in (0.2, 0.1):
        w, a, g = _small(dt=dt)
        fh = W.test_block(w)
        y = march.march(a, g, fh, variant="ssrm", n_trans=12)
        ref = _apply_r([resolvent.continuous(a, om) for om in g.omegas], fh)
        errs.append(np.abs(y - ref).max() / np.abs(ref).max())
    ratio = errs[0] / errs[1]
    assert errs[1] < 1e-4
    assert 12.0 < ratio < 20.0, (errs, ratio)


def test_transient_error_decays_at_spectral_abscissa():
    """P4: SSRM leakage shrinks by about exp(alpha T) per added transient window."""
    w, a, g = _small()
    fh = W.test_block(w)
    alpha = np.linalg.eigvals(a.toarray()).real.max()
    ref = _apply_r([resolvent.rk4_discrete(a, om, g.h) for om in g.omegas], fh)
    e = []
    for nt in (1, 2, 3):
        y = march.march(a, g, fh, variant="ssrm", n_trans=nt)
        e.append(np.abs(y - ref).max())
    expected = math.exp(alpha * g.period)
    for r in (e[1] / e[0], e[2] / e[1]):
        assert 0.2 * expected < r < 5.0 * expected, (e, expected)


def test_trm_tail_leakage_decays():
    """Sec. 2.2: truncation leakage decreases exponentially with the record length."""
    w, a, g = _small()
    fh = W.test_block(w)
    ref = _apply_r([resolvent.rk4_discrete(a, om, g.h) for om in g.omegas], fh)
    errs = [np.abs(march.march(a, g, fh, variant="trm", tail_steps=t) - ref).max()
            for t in (g.n_t, 2 * g.n_t, 3 * g.n_t)]
    alpha = np.linalg.eigvals(a.toarray()).real.max()
    expected = math.exp(alpha * g.period)
    assert errs[0] > errs[1] > errs[2]
    for r in (errs[1] / errs[0], errs[2] / errs[1]):
        assert 0.2 * expected < r < 5.0 * expected, (errs, expected)


def test_trm_norm_truncation():
    """Sec. 2.2 / Sec. 3: ending the TRM record once the state norm has fallen to tol times its
    peak leaves a leakage error of the order of tol against the closed-form R_h fhat, and a
    tighter tol marches longer."""
    w, a, g = _small()
    fh = W.test_block(w)
    ref = _apply_r([resolvent.rk4_discrete(a, om, g.h) for om in g.omegas], fh)
    prev = 0
    for tol in (1e-3, 1e-6, 1e-9):
        y, steps = march.march(a, g, fh, variant="trm", tail_steps=20 * g.n_t, tail_tol=tol, check_every=50,
                               return_steps=True)
        err = np.abs(y - ref).max() / np.abs(ref).max()
        assert 1e-3 * tol < err < tol, (tol, err)
        assert steps % 50 == 0 and steps >= g.n_t and steps > prev
        prev = steps
        # the first check point that meets the rule: at the one before, some vector was above it
        _, u_before = march.march(a, g, fh, variant="trm", tail_steps=20 * g.n_t, stop_after=steps - 50,
                                  return_state=True)
        _, u_stop = march.march(a, g, fh, variant="trm", tail_steps=20 * g.n_t, stop_after=steps,
                                return_state=True)
        assert np.linalg.norm(u_before, axis=1).max() > np.linalg.norm(u_stop, axis=1).max()


def test_frequency_orthogonality():
    """P8: forcing one grid frequency gives no response at the others (Sec. 2.3)."""
    w, a, g = _small()
    fh = W.test_block(w)
    only = np.zeros_like(fh)
    only[3] = fh[3]
    y = march.march(a, g, only, variant="ssrm", n_trans=12)
    others = np.delete(y, 3, axis=0)
    assert np.abs(others).max() < 1e-13 * np.abs(y[3]).max()


def test_diagonal_system_gains():
    """P6: for a diagonal A the gains are |1/(i w - lambda)| up to O(h^4)."""
    lam = np.array([-0.3 + 0.5j, -0.1 - 0.2j, -0.6, -0.05 + 1.0j])
    a = np.diag(lam)
    g = frequencies.make_grid(np.linspace(-1.0, 1.0, 8), 0.01)
    fh = W.gaussian_block(7, 8, 4, 4)
    y = march.march(a, g, fh, variant="ssrm", n_trans=40)
    # uhat_i = fhat_i / (i w - lambda_i) componentwise
    ref = fh / (1j * g.omegas[:, None, None] - lam[None, None, :])
    assert np.abs(y - ref).max() / np.abs(ref).max() < 1e-8


def test_real_state_symmetries():
    """P9: a real system answers real at w = 0 and with R(-w) = conj R(w)."""
    lam = np.array([[-0.3, 0.8, 0.0], [-0.8, -0.3, 0.2], [0.0, 0.1, -0.5]])
    g = frequencies.make_grid(np.array([0.0, 0.25, 0.5, 0.75]), 0.05)
    fh = W.gaussian_block(3, 4, 2, 3, real_rows=[0])
    y = march.march(lam, g, fh, variant="ssrm", n_trans=25, real_state=True)
    assert np.abs(y[0].imag).max() == 0.0
    rm = [resolvent.rk4_discrete(lam, om, g.h) for om in g.omegas]
    ref = _apply_r(rm, fh)
    assert np.abs(y - ref).max() / np.abs(ref).max() < 1e-12
    # the real march equals a complex march forced at +w and -w with conjugate coefficients
    r_neg = resolvent.rk4_discrete(lam, -0.5, g.h)
    assert np.allclose(r_neg, rm[2].conj(), atol=1e-14)


def test_rsvd_full_rank_equals_direct_svd():
    """P5: with k = n the sketch spans everything and the gains are svd(R_h)."""
    w, a, g = _small(n=10, k=10, n_omega=4, mu0=-0.3)
    om_block = W.test_block(w)
    md = lambda b: march.march(a, g, b, variant="ssrm", n_trans=12)
    ma = lambda b: march.march(a, g, b, variant="ssrm", n_trans=12, adjoint=True)
    gains, vm, um = rsvd.block_rsvd(md, ma, om_block, 0, 3)
    for j, om in enumerate(g.omegas):
        rh = resolvent.rk4_discrete(a, om, g.h)
        u, s, vh = np.linalg.svd(rh)
        assert np.allclose(gains[0, j], s[:3], rtol=1e-11)
        # leading forcing/response modes up to a phase
        assert abs(abs(np.vdot(vm[0][j][0], vh[0].conj())) - 1) < 1e-9
        assert abs(abs(np.vdot(um[0][j][0], u[:, 0])) - 1) < 1e-9


def test_gains_approach_continuous_svd():
    """P5: the discrete gains differ from svd((i w I - A)^{-1}) by O(h^4)."""
    w, a, g = _small(n=12, k=12, n_omega=4, dt=0.05, mu0=-0.3)
    md = lambda b: march.march(a, g, b, variant="ssrm", n_trans=12)
    ma = lambda b: march.march(a, g, b, variant="ssrm", n_trans=12, adjoint=True)
    gains, _, _ = rsvd.block_rsvd(md, ma, W.test_block(w), 0, 2)
    for j, om in enumerate(g.omegas):
        s = np.linalg.svd(resolvent.continuous(a, om), compute_uv=False)
        assert np.allclose(gains[0, j], s[:2], rtol=1e-4)


def test_rayleigh_ritz_refinement():
    """A refinement pass (one direct run on the basis, SVD of R Q) returns the exact leading gains
    when the basis spans the leading right singular vectors, and its error is quadratic in the
    basis error (Rayleigh quotient), against the direct SVD of R_h."""
    w, a, g = _small()
    rm = [resolvent.rk4_discrete(a, om, g.h) for om in g.omegas]
    svs = [np.linalg.svd(r) for r in rm]
    k, n_modes = 4, 3
    exact = np.array([s[:n_modes] for _, s, _ in svs])
    vlead = np.stack([vh[:k].conj() for _, _, vh in svs])          # [n_omega][k][n]
    direct = lambda b: _apply_r(rm, b)
    g0, v0, u0 = rsvd.rayleigh_ritz_refine(direct, vlead, n_modes)
    assert np.abs(g0[0] - exact).max() / exact.max() < 1e-12
    # forcing modes: the right singular vectors up to phase
    for j, (_, _, vh) in enumerate(svs):
        for m in range(n_modes):
            assert abs(abs(np.vdot(vh[m].conj(), v0[0][j][m])) - 1.0) < 1e-10
    rng = np.random.default_rng(3)
    errs = []
    for eps in (1e-3, 1e-4):
        noise = rng.standard_normal(vlead.shape) + 1j * rng.standard_normal(vlead.shape)
        ge, _, _ = rsvd.rayleigh_ritz_refine(direct, vlead + eps * noise, n_modes)
        errs.append(np.abs(ge[0] - exact).max() / exact.max())
    assert errs[0] < 1e-3 and 50.0 < errs[0] / errs[1] < 200.0, errs   # tenfold eps -> hundredfold error
    # through the oracle's march: the same numbers
    gm, _, _ = rsvd.rayleigh_ritz_refine(lambda b: march.march(a, g, b, variant="ssrm", n_trans=12), vlead, n_modes)
    assert np.abs(gm[0] - exact).max() / exact.max() < 1e-11


def test_power_iteration_rate():
    """P7 / App. A: the gain estimate converges with error ratio (sigma2/sigma1)^2."""
    w, a, g = _small(n=16, n_omega=4, k=1, mu0=-0.3)
    md = lambda b: march.march(a, g, b, variant="ssrm", n_trans=12)
    ma = lambda b: march.march(a, g, b, variant="ssrm", n_trans=12, adjoint=True)
    hist, _ = rsvd.power_iteration(md, ma, W.test_block(w), 6)
    for j, om in enumerate(g.omegas):
        s = np.linalg.svd(resolvent.rk4_discrete(a, om, g.h), compute_uv=False)
        err = np.abs(hist[:, j] ** 2 - s[0] ** 2)
        rate = (s[1] / s[0]) ** 2
        assert err[-1] < err[0]
        measured = err[4] / err[3]
        if err[4] > 1e-11 * s[0] ** 2:
            assert 0.3 * rate < measured < 3.0 * rate, (measured, rate)


def test_frequency_grid():
    g = frequencies.make_grid(W.gl_fd_c1().omegas, 0.02)
    assert g.phi == 0.5
    assert g.n_t == 3247
    assert abs(g.n_t * g.h - g.period) < 1e-12
    assert np.allclose((g.m + g.phi) * g.dw, g.omegas, atol=1e-13)
    g2 = frequencies.make_grid(W.dense_hermite_c2().omegas, 0.005)
    assert g2.n_t == 80111 and g2.phi == 0.5
    with pytest.raises(ValueError):
        frequencies.make_grid(np.array([0.0, 0.1, 0.25]), 0.01)


def _block_diag_rh(blocks, om, h):
    """R_h(w) of each diagonal block of a block-diagonal system."""
    return [resolvent.rk4_discrete(b, om, h) for b in blocks]


def test_rsvd_instances_equal_blockwise_direct_svd():
    """A batched (block-diagonal) system: with `instances`, each block gets its own QR and SVD,
    so full-rank sketches (k = block size) give svd(R_h) of each block, modes up to phase."""
    sysm = W.GL1D(n=(5, 5, 5), mu0=(-0.1, -0.3, 0.05), x0=-6.0, x1=6.0)
    a = operators.gl1d(sysm)
    blocks = [operators.gl1d(W.GL1D(n=(5,), mu0=(m,), x0=-6.0, x1=6.0)).toarray() for m in sysm.mu0]
    g = frequencies.make_grid(np.linspace(-1.0, 1.0, 4), 0.05)
    om_block = W.gaussian_block(17, 4, 5, 15)
    md = lambda b: march.march(a, g, b, variant="ssrm", n_trans=30)
    ma = lambda b: march.march(a, g, b, variant="ssrm", n_trans=30, adjoint=True)
    inst = [(0, 5), (5, 5), (10, 5)]
    gains, vm, um = rsvd.block_rsvd(md, ma, om_block, 1, 3, instances=inst)
    for j, om in enumerate(g.omegas):
        for i, rh in enumerate(_block_diag_rh(blocks, om, g.h)):
            u, s, vh = np.linalg.svd(rh)
            assert np.allclose(gains[i, j], s[:3], rtol=1e-10), (i, j)
            for m in range(3):
                assert abs(abs(np.vdot(vm[i][j][m], vh[m].conj())) - 1) < 1e-8
                assert abs(abs(np.vdot(um[i][j][m], u[:, m])) - 1) < 1e-8
    # the orthonormalised block is orthonormal within each instance and zero across
    q = rsvd.orthonormalize(om_block, inst)
    for j in range(4):
        for off, size in inst:
            blk = q[j, :, off:off + size]
            assert np.allclose(blk @ blk.conj().T, np.eye(5), atol=1e-13)
    # refinement on the same batch: per-block SVD of R Q
    gr, _, _ = rsvd.rayleigh_ritz_refine(md, om_block, 3, instances=inst)
    for j, om in enumerate(g.omegas):
        for i, rh in enumerate(_block_diag_rh(blocks, om, g.h)):
            assert np.allclose(gr[i, j], np.linalg.svd(rh, compute_uv=False)[:3], rtol=1e-10)


def test_rsvd_real_rows_equal_real_zero_frequency_svd():
    """A real system forced at w = 0: R_h(0) is a real matrix; with `real_rows` the rSVD of that
    row works on real blocks and returns svd(R_h(0)) with real modes; the other rows are the
    complex svd(R_h(w))."""
    sysm = W.ADR2D(nx=4, ny=3, lx=4.0, ly=2.0, jet_delta=0.3, sponge_cells=1, visc=0.05)
    a = operators.adr2d(sysm)
    n = a.shape[0]
    g = frequencies.make_grid(np.array([0.0, 0.5, 1.0, 1.5]), 0.05)
    om_block = W.gaussian_block(23, 4, n, n, real_rows=[0])
    kw = dict(variant="ssrm", n_trans=40, real_state=True)
    md = lambda b: march.march(a, g, b, **kw)
    ma = lambda b: march.march(a, g, b, adjoint=True, **kw)
    gains, vm, um = rsvd.block_rsvd(md, ma, om_block, 0, 3, real_rows=[0])
    for j, om in enumerate(g.omegas):
        rh = resolvent.rk4_discrete(a, om, g.h)
        if j == 0:
            assert np.abs(rh.imag).max() < 1e-13 * np.abs(rh).max()
            rh = rh.real
        u, s, vh = np.linalg.svd(rh)
        assert np.allclose(gains[0, j], s[:3], rtol=1e-10), j
        for m in range(3):
            assert abs(abs(np.vdot(vm[0][j][m], vh[m].conj())) - 1) < 1e-8
            assert abs(abs(np.vdot(um[0][j][m], u[:, m])) - 1) < 1e-8
    assert np.abs(np.asarray(vm[0][0]).imag).max() == 0.0 and np.abs(np.asarray(um[0][0]).imag).max() == 0.0
    q = rsvd.orthonormalize(om_block, [(0, n)], real_rows=[0])
    assert np.abs(q[0].imag).max() == 0.0 and np.allclose(q[0] @ q[0].T, np.eye(n), atol=1e-13)


def test_trm_check_points_every_step_by_default():
    """Sec. 2.2 ends the record once the norm is negligible and fixes no check cadence: the oracle
    checks every step unless told otherwise.  A coarser cadence (the library checks at tile ends)
    stops at or after the per-step stop, and both records are within tol of R_h fhat."""
    w, a, g = _small()
    fh = W.test_block(w)
    ref = _apply_r([resolvent.rk4_discrete(a, om, g.h) for om in g.omegas], fh)
    tol = 1e-6
    y1, s1 = march.march(a, g, fh, variant="trm", tail_steps=20 * g.n_t, tail_tol=tol, return_steps=True)
    y64, s64 = march.march(a, g, fh, variant="trm", tail_steps=20 * g.n_t, tail_tol=tol, check_every=64,
                           return_steps=True)
    assert g.n_t <= s1 <= s64 and s64 % 64 == 0 and s64 - s1 < 64 * 4
    for y in (y1, y64):
        assert np.abs(y - ref).max() / np.abs(ref).max() < tol
    assert np.abs(y64 - y1).max() / np.abs(ref).max() < tol


def test_seeded_gaussian_block_distribution():
    """The seeded test block is standard complex Gaussian ((N(0,1) + i N(0,1)) / sqrt 2 per entry;
    N(0,1) in real rows): moments, independence of the two parts and a Kolmogorov-Smirnov test
    against the normal distribution; the same seed gives the same block, another seed another."""
    from scipy import stats
    from oracle import rsvd
    b = rsvd.gaussian_test_block(77, 3, 4, 5000, real_rows=(0,))
    assert b.shape == (3, 4, 5000)
    c = b[1:].ravel()
    m = c.size
    assert abs(c.real.mean()) < 5 * np.sqrt(0.5 / m) and abs(c.imag.mean()) < 5 * np.sqrt(0.5 / m)
    assert abs(c.real.var() - 0.5) < 0.02 and abs(c.imag.var() - 0.5) < 0.02
    assert abs(np.corrcoef(c.real, c.imag)[0, 1]) < 5 / np.sqrt(m)
    assert stats.kstest(c.real * np.sqrt(2.0), "norm").pvalue > 1e-3
    assert stats.kstest(c.imag * np.sqrt(2.0), "norm").pvalue > 1e-3
    r = b[0].ravel()
    assert not r.imag.any() and abs(r.real.var() - 1.0) < 0.05
    assert stats.kstest(r.real, "norm").pvalue > 1e-3
    assert np.array_equal(b, rsvd.gaussian_test_block(77, 3, 4, 5000, real_rows=(0,)))
    assert not np.allclose(b, rsvd.gaussian_test_block(78, 3, 4, 5000, real_rows=(0,)))
