"""GPU parity of the forcing / observation matrices and metrics (Sec. 2.1) against the oracle.

With diagonal B, C, W_f, W_y set by rsv_set_weights, the direct run returns
C R_h B fhat, the adjoint run W_f^{-1} B^H R_h^H C^H W_y yhat, and the
randomized SVD and the refinement work in the W_f / W_y norms; each is
compared with oracle.weighted on the same inputs (FP64 1e-10, FP32 2e-5 per
frequency row; gains 1e-10 / 1e-4 each).
"""
import numpy as np
import pytest

import workloads as W
from oracle import frequencies, operators, weighted
from parity import gain_rel, rel_rows

pytestmark = pytest.mark.gpu


def _dev(x, prec):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda",
                                                        dtype=torch.complex128 if prec == 0 else torch.complex64)


def _case(kind):
    rng = np.random.default_rng(12)
    if kind == "gl1d":
        w = W.small_gl(n=48, n_omega=8, k=4, n_trans=4, mu0=-0.1)
        a, dense = operators.gl1d(w.system), None
    else:
        sysm = W.ADR2D(nx=40, ny=24, lx=40.0, ly=10.0, sponge_cells=4, visc=0.05)
        dx = sysm.lx / (sysm.nx + 1)
        w = W.Workload("adr_w", sysm, np.linspace(0.0, 4.0, 8), 0.5 * dx, 4, "ssrm", n_transient_windows=2,
                       real_state=True, seed=W.SEED_BASE + 37)
        a, dense = operators.adr2d(sysm), None
    n = w.n
    b = np.where(rng.random(n) < 0.25, 0.0, rng.uniform(0.5, 2.0, n))
    c = np.where(rng.random(n) < 0.25, 0.0, rng.uniform(0.5, 2.0, n))
    return w, a, dense, b, c, rng.uniform(0.3, 3.0, n), rng.uniform(0.3, 3.0, n)


@pytest.mark.parametrize("kind", ["gl1d", "adr2d"])
@pytest.mark.parametrize("prec", [0, 1])
def test_weighted_runs_match_oracle(rsv, kind, prec):
    import torch
    w, a, dense, b, c, wf, wy = _case(kind)
    g = frequencies.make_grid(w.omegas, w.dt)
    op = rsv.create_for_workload(w, prec, dense_matrix=dense)
    try:
        rsv.rsv_set_weights(op, b, c, wf, wy)
        fh = W.test_block(w)
        if prec == 1:
            fh = fh.astype(np.complex64).astype(np.complex128)
        x = _dev(fh, prec)
        y, z = torch.empty_like(x), torch.empty_like(x)
        opts = rsv.march_opts_for(w, 32)
        rsv.rsv_march_direct(op, x, w.k, y, **opts)
        rsv.rsv_march_adjoint(op, x, w.k, z, **opts)
        kw = dict(variant=w.variant, n_trans=w.n_transient_windows, real_state=w.real_state)
        tol = 1e-10 if prec == 0 else 2e-5
        assert rel_rows(y.cpu().numpy().astype(np.complex128), weighted.march_direct(a, g, fh, b, c, **kw)) < tol
        assert rel_rows(z.cpu().numpy().astype(np.complex128),
                        weighted.march_adjoint(a, g, fh, b, c, wf, wy, **kw)) < tol
        # clearing the weights restores the plain runs
        rsv.rsv_set_weights(op)
        y2 = torch.empty_like(x)
        rsv.rsv_march_direct(op, x, w.k, y2, **opts)
        from oracle import march
        assert rel_rows(y2.cpu().numpy().astype(np.complex128), march.march(a, g, fh, **kw)) < tol
    finally:
        rsv.rsv_destroy_operator(op)


@pytest.mark.parametrize("kind", ["gl1d", "adr2d"])
def test_weighted_gains_match_oracle(rsv, kind):
    import torch
    w, a, dense, b, c, wf, wy = _case(kind)
    g = frequencies.make_grid(w.omegas, w.dt)
    op = rsv.create_for_workload(w, 0, dense_matrix=dense)
    try:
        rsv.rsv_set_weights(op, b, c, wf, wy)
        fh = W.test_block(w)
        gains = np.zeros((1, w.n_omega, 3))
        fm = torch.empty((w.n_omega, 3, w.n), dtype=torch.complex128, device="cuda")
        rm = torch.empty_like(fm)
        rsv.rsv_gains_modes(op, _dev(fh, 0), w.k, 1, 3, gains, fm, rm, **rsv.march_opts_for(w, 32))
        real_rows = [j for j, om in enumerate(w.omegas) if w.real_state and om == 0.0]
        rg, rv, ru = weighted.weighted_rsvd(a, g, fh, b, c, wf, wy, 1, 3, real_rows=real_rows,
                                            variant=w.variant, n_trans=w.n_transient_windows,
                                            real_state=w.real_state)
        assert gain_rel(gains, rg) < 1e-10
        fmh, rmh = fm.cpu().numpy(), rm.cpu().numpy()
        for j in range(w.n_omega):
            for m in range(3):
                assert abs(np.vdot(fmh[j, m], wf * fmh[j, m]).real - 1.0) < 1e-9    # unit in W_f
                assert abs(abs(np.vdot(fmh[j, m], wf * rv[0][j][m])) - 1.0) < 1e-8
                assert abs(abs(np.vdot(rmh[j, m], wy * ru[0][j][m])) - 1.0) < 1e-8
    finally:
        rsv.rsv_destroy_operator(op)


def test_weighted_refinement_full_rank(rsv):
    """A full-rank basis (k = n): the refined gains are the singular values of
    W_y^{1/2} C R_h B W_f^{-1/2} from the closed-form RK4 resolvent."""
    from oracle import resolvent
    w = W.small_gl(n=12, n_omega=4, k=12, n_trans=12, mu0=-0.3)
    a = operators.gl1d(w.system)
    g = frequencies.make_grid(w.omegas, w.dt)
    rng = np.random.default_rng(4)
    b, c = rng.uniform(0.5, 2.0, w.n), rng.uniform(0.5, 2.0, w.n)
    wf, wy = rng.uniform(0.3, 3.0, w.n), rng.uniform(0.3, 3.0, w.n)
    op = rsv.create_for_workload(w, 0)
    try:
        rsv.rsv_set_weights(op, b, c, wf, wy)
        gr = np.zeros((1, w.n_omega, 3))
        rsv.rsv_refine_gains(op, _dev(W.test_block(w), 0), w.k, 3, gr, **rsv.march_opts_for(w, 32))
        for j, om in enumerate(g.omegas):
            rt = np.diag(np.sqrt(wy) * c) @ resolvent.rk4_discrete(a, om, g.h) @ np.diag(b / np.sqrt(wf))
            s = np.linalg.svd(rt, compute_uv=False)[:3]
            assert np.abs(gr[0, j] - s).max() < 1e-10 * s[0]
    finally:
        rsv.rsv_destroy_operator(op)
