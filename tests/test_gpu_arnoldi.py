"""GPU parity of the Arnoldi gains (App. A, Eq. (freqOrt)) against the oracle.

rsv_arnoldi_gains runs m direct + m adjoint marches of one vector per
frequency, orthogonalising each new forcing against the previous ones; the
gains, forcing and response modes must match oracle.arnoldi on the same start
vectors: FP64 1e-10 (gains), modes up to phase; FP32 gains within 1e-4.
"""
import numpy as np
import pytest

import workloads as W
from oracle import arnoldi, frequencies, march, operators, resolvent
from parity import gain_rel

pytestmark = pytest.mark.gpu


def _dev(x, prec):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda",
                                                        dtype=torch.complex128 if prec == 0 else torch.complex64)


def _case(kind):
    if kind == "gl1d":
        w = W.small_gl(n=40, n_omega=8, k=1, n_trans=6, mu0=-0.15)
        return w, operators.gl1d(w.system), None, []
    sysm = W.ADR2D(nx=40, ny=24, lx=40.0, ly=10.0, sponge_cells=4, visc=0.05)
    dx = sysm.lx / (sysm.nx + 1)
    # 45 transient windows: the decay run of this system needs about 42 (to 1e-6) before the direct and
    # adjoint runs are the exact adjoints R_h and R_h^H that make the Arnoldi projection Hermitian
    w = W.Workload("adr_a", sysm, np.linspace(0.0, 4.0, 8), 0.5 * dx, 1, "ssrm", n_transient_windows=45,
                   real_state=True, seed=W.SEED_BASE + 38)
    return w, operators.adr2d(sysm), None, [0]


@pytest.mark.parametrize("kind", ["gl1d", "adr2d"])
@pytest.mark.parametrize("prec", [0, 1])
def test_arnoldi_matches_oracle(rsv, kind, prec):
    import torch
    w, a, dense, real_rows = _case(kind)
    g = frequencies.make_grid(w.omegas, w.dt)
    m, nm = 6, 3
    op = rsv.create_for_workload(w, prec, dense_matrix=dense)
    try:
        f0 = W.test_block(w)
        if prec == 1:
            f0 = f0.astype(np.complex64).astype(np.complex128)
        gains = np.zeros((1, w.n_omega, nm))
        cdt = torch.complex128 if prec == 0 else torch.complex64
        fm = torch.empty((w.n_omega, nm, w.n), dtype=cdt, device="cuda")
        rm = torch.empty_like(fm)
        rsv.rsv_arnoldi_gains(op, _dev(f0, prec), m, nm, gains, fm, rm, **rsv.march_opts_for(w, 32))
        kw = dict(variant=w.variant, n_trans=w.n_transient_windows, real_state=w.real_state)
        rg, rv, ru, _ = arnoldi.arnoldi(lambda b: march.march(a, g, b, **kw),
                                        lambda b: march.march(a, g, b, adjoint=True, **kw), f0, m, nm,
                                        real_rows=real_rows)
        err = gain_rel(gains[0], rg)
        assert err < (1e-10 if prec == 0 else 1e-4), err
        if prec == 0:
            fmh, rmh = fm.cpu().numpy(), rm.cpu().numpy()
            cosang = lambda x, y: abs(np.vdot(x, y)) / (np.linalg.norm(x) * np.linalg.norm(y))
            for j in range(w.n_omega):
                for q in range(nm):
                    assert abs(cosang(fmh[j, q], rv[j, q]) - 1) < 1e-8
                    assert abs(cosang(rmh[j, q], ru[j, q]) - 1) < 1e-8
                    assert abs(np.linalg.norm(rmh[j, q]) / np.linalg.norm(ru[j, q]) - 1) < 1e-8
    finally:
        rsv.rsv_destroy_operator(op)


def test_arnoldi_full_space_is_exact(rsv):
    """m = n: the Krylov space is the whole state space and the gains are svd(R_h)."""
    w = W.small_gl(n=12, n_omega=4, k=1, n_trans=12, mu0=-0.3)
    a = operators.gl1d(w.system)
    g = frequencies.make_grid(w.omegas, w.dt)
    op = rsv.create_for_workload(w, 0)
    try:
        gains = np.zeros((1, w.n_omega, 4))
        rsv.rsv_arnoldi_gains(op, _dev(W.test_block(w), 0), 12, 4, gains, **rsv.march_opts_for(w, 32))
        for j, om in enumerate(g.omegas):
            s = np.linalg.svd(resolvent.rk4_discrete(a, om, g.h), compute_uv=False)[:4]
            assert np.abs(gains[0, j] - s).max() < 1e-9 * s[0]
    finally:
        rsv.rsv_destroy_operator(op)
