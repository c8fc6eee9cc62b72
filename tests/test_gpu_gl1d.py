"""GPU parity of the 1-D (Ginzburg-Landau) path against the FP64 oracle.

Element-by-element comparison of the CUDA marches (through the C ABI) with
the oracle's march on the same seeded inputs, each frequency row against its
own largest entry: FP64 path within 1e-10; FP32 path within 2e-5 (FP32 rounding of
~6e-8 per operation, amplified by gains of order 10-30 and by the 64-step
FP32 partial sums of the DFT, stays at a few 1e-6).  Sizes span several
time tiles with ragged last tiles.
"""
import numpy as np
import pytest

import workloads as W
from parity import gain_rel, rel_rows
from oracle import frequencies, march, operators, rsvd

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32_MARCH = 2e-5     # element-wise, relative to each frequency row's largest entry
TOL32_GAIN = 1e-4      # leading gains


def _torch():
    import torch
    return torch


def _dev(x, prec, rsv):
    t = _torch()
    dt = t.complex128 if prec == rsv.RSV_PREC_FP64 else t.complex64
    return t.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dt)




def _oracle_pair(w, fh, adjoint=False, **kw):
    a = operators.gl1d(w.system)
    g = frequencies.make_grid(w.omegas, w.dt)
    opts = dict(variant=w.variant, n_trans=w.n_transient_windows, tail_steps=w.tail_steps)
    opts.update(kw)
    return march.march(a, g, fh, adjoint=adjoint, **opts)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
def test_apply_operator_matches_oracle_matrix(rsv, prec, adjoint):
    w = W.small_gl(n=300, k=3)
    op = rsv.create_for_workload(w, prec)
    try:
        x = W.gaussian_block(11, 1, 3, 300)[0]
        xd = _dev(x, prec, rsv)
        yd = _torch().empty_like(xd)
        rsv.rsv_apply_operator(op, xd, 3, adjoint, yd)
        a = operators.gl1d(w.system)
        if adjoint:
            a = a.conj().T
        ref = (a @ x.T).T
        err = rel_rows(yd.cpu().numpy(), ref)
        assert err < (1e-14 if prec == 0 else 1e-6), err
    finally:
        rsv.rsv_destroy_operator(op)


@pytest.mark.parametrize("variant,tile", [("ssrm", 64), ("ssrm", 37), ("trm", 100), ("ssrm", 10000), ("trm", 1)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_march_fp64_matches_oracle(rsv, variant, tile, adjoint):
    w = W.small_gl(n=40, n_omega=8, k=3, variant=variant, n_trans=3, tail_steps=700, mu0=-0.1)
    op = rsv.create_for_workload(w, rsv.RSV_PREC_FP64)
    try:
        fh = W.test_block(w)
        xd = _dev(fh, 0, rsv)
        yd = _torch().empty_like(xd)
        f = rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct
        f(op, xd, w.k, yd, **rsv.march_opts_for(w, tile_steps=tile))
        ref = _oracle_pair(w, fh, adjoint=adjoint)
        assert rel_rows(yd.cpu().numpy(), ref) < TOL64
    finally:
        rsv.rsv_destroy_operator(op)


@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("contract", ["tensor", "cuda_cores"])
def test_march_fp32_matches_oracle(rsv, adjoint, contract, monkeypatch):
    monkeypatch.setenv("RSV_CONTRACT_TENSOR", "1" if contract == "tensor" else "0")
    w = W.small_gl(n=200, n_omega=16, k=4, n_trans=3, mu0=-0.1, dt=0.005, x_half=40.0)
    op = rsv.create_for_workload(w, rsv.RSV_PREC_FP32)
    try:
        fh = W.test_block(w)
        xd = _dev(fh, 1, rsv)
        yd = _torch().empty_like(xd)
        f = rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct
        f(op, xd, w.k, yd, **rsv.march_opts_for(w, tile_steps=128))
        ref = _oracle_pair(w, fh.astype(np.complex64).astype(np.complex128), adjoint=adjoint)
        assert rel_rows(yd.cpu().numpy().astype(np.complex128), ref) < TOL32_MARCH
    finally:
        rsv.rsv_destroy_operator(op)


def test_batched_instances_match_oracle(rsv):
    sysm = W.GL1D(n=(33, 70, 130, 17), mu0=(0.0, -0.1, 0.05, -0.2), x0=-20.0, x1=20.0)
    w = W.Workload("batch", sysm, np.linspace(-1.0, 1.0, 6), 0.02, 2, "ssrm", n_transient_windows=3)
    op = rsv.create_for_workload(w, rsv.RSV_PREC_FP64)
    try:
        fh = W.test_block(w)
        xd = _dev(fh, 0, rsv)
        yd = _torch().empty_like(xd)
        rsv.rsv_march_direct(op, xd, w.k, yd, **rsv.march_opts_for(w, tile_steps=50))
        ref = _oracle_pair(w, fh)
        assert rel_rows(yd.cpu().numpy(), ref) < TOL64
        assert rsv.rsv_operator_info(op) == (250, 4, False)
        assert rsv.rsv_instance_range(op, 2) == (103, 130)
    finally:
        rsv.rsv_destroy_operator(op)


def _oracle_rsvd(w, fh, instances=None):
    a = operators.gl1d(w.system)
    g = frequencies.make_grid(w.omegas, w.dt)
    kw = dict(variant=w.variant, n_trans=w.n_transient_windows, tail_steps=w.tail_steps)
    md = lambda b: march.march(a, g, b, **kw)
    ma = lambda b: march.march(a, g, b, adjoint=True, **kw)
    return rsvd.block_rsvd(md, ma, fh, w.n_power_iter, w.n_modes, instances=instances)


@pytest.mark.parametrize("variant", ["ssrm", "trm"])
def test_rsvd_fp64_matches_oracle(rsv, variant):
    w = W.small_gl(n=60, n_omega=8, k=4, variant=variant, n_trans=3, tail_steps=900, q=2, mu0=-0.1)
    w = W.Workload(w.name, w.system, w.omegas, w.dt, 4, variant, n_transient_windows=3, tail_steps=900,
                   n_power_iter=2, n_modes=3, seed=w.seed)
    op = rsv.create_for_workload(w, rsv.RSV_PREC_FP64)
    try:
        fh = W.test_block(w)
        xd = _dev(fh, 0, rsv)
        t = _torch()
        fm = t.empty((w.n_omega, 3, w.n), dtype=t.complex128, device="cuda")
        rm = t.empty_like(fm)
        gains = np.zeros((1, w.n_omega, 3))
        rsv.rsv_gains_modes(op, xd, w.k, w.n_power_iter, 3, gains, fm, rm, **rsv.march_opts_for(w, 64))
        rg, rv, ru = _oracle_rsvd(w, fh)
        assert gain_rel(gains, rg) < TOL64
        fmh, rmh = fm.cpu().numpy(), rm.cpu().numpy()
        for j in range(w.n_omega):
            for m in range(3):
                assert abs(abs(np.vdot(fmh[j, m], rv[0][j][m])) - 1) < 1e-8
                assert abs(abs(np.vdot(rmh[j, m], ru[0][j][m])) - 1) < 1e-8
    finally:
        rsv.rsv_destroy_operator(op)


def test_rsvd_batched_instances(rsv):
    sysm = W.GL1D(n=(40, 64, 50), mu0=(-0.1, -0.05, -0.2), x0=-20.0, x1=20.0)
    w = W.Workload("batch", sysm, np.linspace(-1.0, 1.0, 4), 0.05, 3, "ssrm", n_transient_windows=3,
                   n_power_iter=1, n_modes=2)
    op = rsv.create_for_workload(w, rsv.RSV_PREC_FP64)
    try:
        fh = W.test_block(w)
        gains = np.zeros((3, w.n_omega, 2))
        rsv.rsv_gains_modes(op, _dev(fh, 0, rsv), w.k, 1, 2, gains, **rsv.march_opts_for(w, 50))
        rg, _, _ = _oracle_rsvd(w, fh, instances=[(0, 40), (40, 64), (104, 50)])
        assert gain_rel(gains, rg) < TOL64
    finally:
        rsv.rsv_destroy_operator(op)


def test_errors_are_reported(rsv):
    w = W.small_gl(n=20)
    d, keep = rsv.desc_for(w.system, w.dt, rsv.RSV_PREC_FP64)
    op = rsv.rsv_create_operator(d, keep=keep)
    try:
        x = _dev(W.test_block(w), 0, rsv)
        y = _torch().empty_like(x)
        with pytest.raises(rsv.RsvError) as e:
            rsv.rsv_march_direct(op, x, w.k, y)
        assert e.value.status == 8
        with pytest.raises(rsv.RsvError) as e:
            rsv.rsv_set_frequencies(op, [0.0, 0.1, 0.25])
        assert e.value.status == 3
        rsv.rsv_set_frequencies(op, w.omegas)
        with pytest.raises(rsv.RsvError) as e:
            rsv.rsv_gains_modes(op, x, 40, 1, 3, np.zeros((1, 8, 3)))
        assert e.value.status == 1
    finally:
        rsv.rsv_destroy_operator(op)


def test_unstable_system_reports_divergence(rsv):
    """A strongly growing system overflows; the march returns DIVERGED instead of garbage."""
    sysm = W.GL1D(n=(32,), mu0=(400.0,), x0=-5.0, x1=5.0)
    w = W.Workload("grow", sysm, np.linspace(-1.0, 1.0, 4), 0.05, 1, "ssrm", n_transient_windows=30)
    op = rsv.create_for_workload(w, rsv.RSV_PREC_FP32)
    try:
        x = _dev(W.test_block(w), 1, rsv)
        y = _torch().empty_like(x)
        with pytest.raises(rsv.RsvError) as e:
            rsv.rsv_march_direct(op, x, 1, y, **rsv.march_opts_for(w))
        assert e.value.status == 4
    finally:
        rsv.rsv_destroy_operator(op)
