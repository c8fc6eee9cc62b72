"""GPU parity of the structured-grid paths (2-D jet ADR, 3-D advection-diffusion) against the oracle.

Real state: the forcing is synthesised as sum_j c_j Re(fhat_j e^{i w_j t}) and
the w = 0 row of the test block is real.  Down-scaled grids with the
workloads' physics; element-wise parity of direct and adjoint marches (FP64
1e-10, FP32 2e-5) and of the randomized-SVD gains.  At full grid size the
FP32 march is checked against the FP64 GPU march (itself oracle-parity
tested here) on a short schedule with few frequencies.
"""
import numpy as np
import pytest

import workloads as W
from parity import gain_rel, rel_rows
from oracle import frequencies, march, operators, rsvd

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 2e-5


def _dev(x, prec):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda",
                                                        dtype=torch.complex128 if prec == 0 else torch.complex64)




def _adr_small(variant="ssrm", omegas=None, k=3):
    sysm = W.ADR2D(nx=40, ny=24, lx=40.0, ly=10.0, sponge_cells=4)
    om = np.linspace(0.0, 4.0, 8) if omegas is None else omegas
    dx = sysm.lx / (sysm.nx + 1)
    return W.Workload("adr_small", sysm, om, 0.5 * dx, k, variant, n_transient_windows=2, tail_steps=60,
                      n_power_iter=1, real_state=True, seed=W.SEED_BASE + 33)


def _adr_odd(variant="ssrm", omegas=None, k=3):
    """nx not a multiple of 4: the scalar stage kernels."""
    sysm = W.ADR2D(nx=42, ny=22, lx=40.0, ly=10.0, sponge_cells=4)
    om = np.linspace(0.0, 4.0, 8) if omegas is None else omegas
    dx = sysm.lx / (sysm.nx + 1)
    return W.Workload("adr_odd", sysm, om, 0.5 * dx, k, variant, n_transient_windows=2, tail_steps=60,
                      n_power_iter=1, real_state=True, seed=W.SEED_BASE + 34)


def _adr_multi(variant="ssrm", omegas=None, k=2):
    """Several fused-kernel tiles (64 x 32) in each direction, ragged at the far edges."""
    sysm = W.ADR2D(nx=150, ny=70, lx=40.0, ly=10.0, sponge_cells=6)
    om = np.linspace(0.0, 4.0, 8) if omegas is None else omegas
    dx = sysm.lx / (sysm.nx + 1)
    return W.Workload("adr_multi", sysm, om, 0.5 * dx, k, variant, n_transient_windows=1, tail_steps=60,
                      n_power_iter=1, real_state=True, seed=W.SEED_BASE + 35)


def _adv_small(variant="ssrm", k=2):
    sysm = W.ADV3D(nx=12, ny=8, nz=6, lx=20.0, ly=10.0, lz=10.0, visc=0.02)
    om = np.array([0.04 * np.pi * 5 * j for j in range(6)])
    dx = sysm.lx / (sysm.nx + 1)
    return W.Workload("adv_small", sysm, om, 0.5 * dx, k, variant, n_transient_windows=2, tail_steps=40,
                      n_power_iter=1, real_state=True, seed=W.SEED_BASE + 44)


def _matrix(w):
    return operators.adr2d(w.system) if type(w.system).__name__ == "ADR2D" else operators.adv3d(w.system)


def _oracle(w, a, fh, adjoint=False):
    g = frequencies.make_grid(w.omegas, w.dt)
    return march.march(a, g, fh, variant=w.variant, n_trans=w.n_transient_windows, tail_steps=w.tail_steps,
                       adjoint=adjoint, real_state=True)


@pytest.mark.parametrize("make", [_adr_small, _adv_small])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
def test_stencil_apply(rsv, make, prec, adjoint):
    w = make()
    op = rsv.create_for_workload(w, prec)
    try:
        x = W.gaussian_block(9, 1, 3, w.n)[0]
        y = _dev(x, prec) * 0
        rsv.rsv_apply_operator(op, _dev(x, prec), 3, adjoint, y)
        a = _matrix(w)
        ref = ((a.T if adjoint else a) @ x.T).T
        assert rel_rows(y.cpu().numpy(), ref) < (1e-13 if prec == 0 else 1e-5)
    finally:
        rsv.rsv_destroy_operator(op)


@pytest.mark.parametrize("make", [_adr_small, _adv_small])
@pytest.mark.parametrize("variant,tile", [("ssrm", 16), ("ssrm", 7), ("trm", 32)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_stencil_march_fp64(rsv, make, variant, tile, adjoint):
    w = make(variant)
    op = rsv.create_for_workload(w, 0)
    try:
        fh = W.test_block(w)
        x = _dev(fh, 0)
        y = x * 0
        f = rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct
        f(op, x, w.k, y, **rsv.march_opts_for(w, tile_steps=tile))
        ref = _oracle(w, _matrix(w), fh, adjoint)
        got = y.cpu().numpy()
        assert rel_rows(got, ref) < TOL64
        assert np.abs(got[0].imag).max() == 0.0   # w = 0 response of a real system is real
    finally:
        rsv.rsv_destroy_operator(op)


@pytest.mark.parametrize("make", [_adr_small, _adr_odd, _adv_small])
@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("contract", ["tensor", "cuda_cores"])
def test_stencil_march_fp32(rsv, make, adjoint, contract, monkeypatch):
    """FP32 march with the synthesis / analysis on the tensor cores and on the CUDA cores."""
    monkeypatch.setenv("RSV_CONTRACT_TENSOR", "1" if contract == "tensor" else "0")
    w = make("trm")
    op = rsv.create_for_workload(w, 1)
    try:
        fh = W.test_block(w).astype(np.complex64).astype(np.complex128)
        x = _dev(fh, 1)
        y = x * 0
        f = rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct
        f(op, x, w.k, y, **rsv.march_opts_for(w, tile_steps=16))
        ref = _oracle(w, _matrix(w), fh, adjoint)
        assert rel_rows(y.cpu().numpy().astype(np.complex128), ref) < TOL32
    finally:
        rsv.rsv_destroy_operator(op)


@pytest.mark.parametrize("make", [_adr_small, _adv_small])
def test_stencil_rsvd_fp64(rsv, make):
    w = make("ssrm", k=3)
    op = rsv.create_for_workload(w, 0)
    try:
        fh = W.test_block(w)
        gains = np.zeros((1, w.n_omega, 2))
        rsv.rsv_gains_modes(op, _dev(fh, 0), w.k, 1, 2, gains, **rsv.march_opts_for(w, 16))
        a = _matrix(w)
        g = frequencies.make_grid(w.omegas, w.dt)
        kw = dict(variant=w.variant, n_trans=w.n_transient_windows, tail_steps=w.tail_steps, real_state=True)
        rg, _, _ = rsvd.block_rsvd(lambda b: march.march(a, g, b, **kw),
                                   lambda b: march.march(a, g, b, adjoint=True, **kw), fh, 1, 2,
                                   real_rows=[j for j, om in enumerate(w.omegas) if om == 0.0])
        assert gain_rel(gains, rg) < TOL64
    finally:
        rsv.rsv_destroy_operator(op)


@pytest.mark.slow
@pytest.mark.parametrize("make", [W.adr2d_c3, W.adv3d_c4])
def test_stencil_full_grid_fp32_vs_fp64(rsv, make):
    """Full workload grid, 4 frequencies, one forced window: FP32 march vs the FP64 march."""
    import torch
    full = make()
    om = full.omegas[:4]
    w = W.Workload(full.name, full.system, om, full.dt, 2, "ssrm", n_transient_windows=0, real_state=True,
                   seed=full.seed)
    fh = W.test_block(w)
    outs = []
    for prec in (0, 1):
        op = rsv.create_for_workload(w, prec)
        try:
            x = _dev(fh.astype(np.complex64).astype(np.complex128), prec)
            y = x * 0
            rsv.rsv_march_direct(op, x, w.k, y, **rsv.march_opts_for(w, tile_steps=64))
            outs.append(y.cpu().numpy().astype(np.complex128))
            del x, y
            torch.cuda.empty_cache()
        finally:
            rsv.rsv_destroy_operator(op)
    assert rel_rows(outs[1], outs[0]) < 1e-4


@pytest.mark.parametrize("make", [_adr_small, _adr_multi])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("path", ["fused", "staged"])
def test_adr2d_step_paths(rsv, make, prec, adjoint, path, monkeypatch):
    """2-D march with the whole-step kernel (four stages in shared memory) and with the per-stage
    kernels, vs the oracle."""
    monkeypatch.setenv("RSV_STENCIL_FUSED", "1" if path == "fused" else "0")
    w = make("trm")
    op = rsv.create_for_workload(w, prec)
    try:
        fh = W.test_block(w)
        if prec == 1:
            fh = fh.astype(np.complex64).astype(np.complex128)
        x = _dev(fh, prec)
        y = x * 0
        f = rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct
        f(op, x, w.k, y, **rsv.march_opts_for(w, tile_steps=15))
        ref = _oracle(w, _matrix(w), fh, adjoint)
        assert rel_rows(y.cpu().numpy().astype(np.complex128), ref) < (TOL64 if prec == 0 else TOL32)
    finally:
        rsv.rsv_destroy_operator(op)


def _adv_multi(variant="trm", k=2):
    """Two fused-pair tiles in x (64 + 8 cells) and y (8 + 3), and two z chunks (16 + 4 planes); nx a multiple of 4."""
    sysm = W.ADV3D(nx=72, ny=11, nz=20, lx=20.0, ly=10.0, lz=10.0, visc=0.02)
    om = np.array([0.04 * np.pi * 5 * j for j in range(6)])
    dx = sysm.lx / (sysm.nx + 1)
    return W.Workload("adv_multi", sysm, om, 0.5 * dx, k, variant, n_transient_windows=1, tail_steps=30,
                      n_power_iter=1, real_state=True, seed=W.SEED_BASE + 45)


@pytest.mark.parametrize("make", [_adv_small, _adv_multi])
@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("path", ["pairs", "staged"])
def test_adv3d_step_paths(rsv, make, adjoint, path, monkeypatch):
    """FP32 3-D march with the two fused stage-pair kernels per step (z-streaming, shared-memory
    rings) and with the four single-stage kernels, vs the oracle, on grids with ragged tiles."""
    monkeypatch.setenv("RSV_STENCIL3D_STAGED", "1" if path == "staged" else "0")
    w = make("trm")
    op = rsv.create_for_workload(w, 1)
    try:
        fh = W.test_block(w).astype(np.complex64).astype(np.complex128)
        x = _dev(fh, 1)
        y = x * 0
        f = rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct
        f(op, x, w.k, y, **rsv.march_opts_for(w, tile_steps=15))
        ref = _oracle(w, _matrix(w), fh, adjoint)
        assert rel_rows(y.cpu().numpy().astype(np.complex128), ref) < TOL32
    finally:
        rsv.rsv_destroy_operator(op)


def _adr_pair_tiles(variant="ssrm", k=2):
    """nx a multiple of 4 over several 64 x 32 pair-kernel tiles, ragged at the far edges."""
    sysm = W.ADR2D(nx=200, ny=70, lx=40.0, ly=10.0, sponge_cells=6)
    om = np.linspace(0.0, 4.0, 8)
    dx = sysm.lx / (sysm.nx + 1)
    return W.Workload("adr_pair_tiles", sysm, om, 0.5 * dx, k, variant, n_transient_windows=1, tail_steps=60,
                      n_power_iter=1, real_state=True, seed=W.SEED_BASE + 36)


@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("variant", ["ssrm", "trm"])
def test_adr2d_stage_pairs_multi_tile(rsv, adjoint, variant):
    """FP32 2-D march through the stage-pair kernels on a grid of 4 x 3 ragged tiles."""
    w = _adr_pair_tiles(variant)
    op = rsv.create_for_workload(w, 1)
    try:
        assert "2-D stage-pair" in rsv.rsv_describe(op)
        fh = W.test_block(w).astype(np.complex64).astype(np.complex128)
        x = _dev(fh, 1)
        y = x * 0
        (rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct)(op, x, w.k, y, **rsv.march_opts_for(w, tile_steps=37))
        ref = _oracle(w, _matrix(w), fh, adjoint)
        assert rel_rows(y.cpu().numpy().astype(np.complex128), ref) < TOL32
    finally:
        rsv.rsv_destroy_operator(op)
