"""GPU parity of the Crank-Nicolson march (the scheme of the paper's Ginzburg-Landau case, Sec. 3).

The 1-D kind with scheme = RSV_SCHEME_CN solves (I - h/2 A) u' = (I + h/2 A) u
+ h/2 (f(t_n) + f(t_n + h)) per step by cyclic reduction; it must match the
oracle's sparse-LU Crank-Nicolson march element by element (FP64 1e-10, FP32
2e-5 per frequency row) for single and batched instances, direct and adjoint,
SSRM and TRM with ragged tiles, and its randomized-SVD gains the oracle's.
"""
import numpy as np
import pytest

import workloads as W
from oracle import frequencies, march, operators, resolvent, rsvd
from parity import gain_rel, rel_rows

pytestmark = pytest.mark.gpu


def _dev(x, prec):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda",
                                                        dtype=torch.complex128 if prec == 0 else torch.complex64)


def _paper_small(variant="ssrm", n=100, k=3):
    w = W.gl_paper(n=n, n_omega=8, dt=0.05)
    return W.Workload(w.name, w.system, np.linspace(0.0, 3.5, 8), 0.05, k, variant, n_transient_windows=2,
                      tail_steps=400, n_power_iter=1, seed=w.seed)


def _batch(variant="ssrm"):
    p = W.gl_paper().system
    sysm = W.GL1D(n=(100, 77, 300, 2), mu0=(3.6, 3.0, 3.6, -1.0), x0=0.0, x1=40.0, nu=p.nu, gamma=p.gamma,
                  mu_shift=0.0, mu2=0.0, mu1=p.mu1)
    return W.Workload("paper_batch", sysm, np.linspace(0.0, 3.5, 8), 0.05, 2, variant, n_transient_windows=2,
                      tail_steps=400, seed=W.SEED_BASE + 71)


@pytest.mark.parametrize("make", [_paper_small, _batch])
@pytest.mark.parametrize("variant,tile", [("ssrm", 64), ("trm", 7)])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
def test_cn_march_matches_oracle(rsv, make, variant, tile, prec, adjoint):
    import torch
    w = make(variant)
    op = rsv.create_for_workload(w, prec, scheme=rsv.RSV_SCHEME_CN)
    try:
        assert "crank-nicolson" in rsv.rsv_describe(op)
        fh = W.test_block(w)
        if prec == 1:
            fh = fh.astype(np.complex64).astype(np.complex128)
        x = _dev(fh, prec)
        y = torch.empty_like(x)
        (rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct)(op, x, w.k, y, **rsv.march_opts_for(w, tile))
        g = frequencies.make_grid(w.omegas, w.dt)
        ref = march.march(operators.gl1d(w.system), g, fh, variant=variant, n_trans=w.n_transient_windows,
                          tail_steps=w.tail_steps, adjoint=adjoint, scheme="cn")
        err = rel_rows(y.cpu().numpy().astype(np.complex128), ref)
        assert err < (1e-10 if prec == 0 else 2e-5), err
    finally:
        rsv.rsv_destroy_operator(op)


def test_cn_gains_match_oracle_and_closed_form(rsv):
    w = _paper_small(k=4)
    a = operators.gl1d(w.system)
    g = frequencies.make_grid(w.omegas, w.dt)
    op = rsv.create_for_workload(w, 0, scheme=rsv.RSV_SCHEME_CN)
    try:
        fh = W.test_block(w)
        gains = np.zeros((1, w.n_omega, 3))
        rsv.rsv_gains_modes(op, _dev(fh, 0), w.k, 1, 3, gains, **rsv.march_opts_for(w, 64))
        kw = dict(variant="ssrm", n_trans=w.n_transient_windows, scheme="cn")
        rg, _, _ = rsvd.block_rsvd(lambda b: march.march(a, g, b, **kw),
                                   lambda b: march.march(a, g, b, adjoint=True, **kw), fh, 1, 3)
        assert gain_rel(gains, rg) < 1e-10
        # the leading gain approaches svd of the Crank-Nicolson resolvent (the rSVD sketch is not full rank)
        lead = np.array([np.linalg.svd(resolvent.cn_discrete(a, om, g.h), compute_uv=False)[0] for om in g.omegas])
        assert np.abs(gains[0, :, 0] - lead).max() / lead.max() < 1e-3
    finally:
        rsv.rsv_destroy_operator(op)


def test_cn_rejected_for_other_kinds(rsv):
    sysm = W.ADR2D(nx=40, ny=24, lx=40.0, ly=10.0, sponge_cells=4)
    d, keep = rsv.desc_for(sysm, 0.5, rsv.RSV_PREC_FP64, rsv.RSV_SCHEME_CN)
    with pytest.raises(rsv.RsvError) as e:
        rsv.rsv_create_operator(d, keep=keep)
    assert e.value.status == 1
