"""GPU parity on the kernel variants the full-size workloads run, and of FP32 gains, against the oracle.

* 1-D kernel with two and four points per thread (instances longer than 1024
  points, as in the batched Ginzburg-Landau workload), in one batch with short
  instances: FP64 (1e-10) and FP32 (2e-5), per frequency row.
* Dense persistent tcgen05 march at n = 512 and n = 1024 with 32 vectors (two
  vector chains), on a short transient run: FP32 within 2e-5.
* FP32 randomized SVD of every operator kind against the oracle's FP64 block
  randomized SVD on the same inputs: leading-3 gains within 1e-4 each (the
  accuracy target) and the response-mode spans within a small principal angle.
"""
import numpy as np
import pytest

import workloads as W
from oracle import frequencies, march, operators, rsvd
from parity import gain_rel, rel_rows, subspace_cos

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 2e-5
# The long 1-D batch marches 8378 steps whose slowest mode decays over about 3400 steps (h = 0.0015,
# spectral abscissa -0.197): FP32 rounding (6e-8 per operation, about eight roundings per step
# reaching the state) accumulates like a random walk over that time, 6e-8 x 8 x sqrt(3400) = 2.8e-5,
# above the short cases' 2e-5; the tolerance for this case is 5e-5.
TOL32_LONG = 5e-5
TOL_GAIN = 1e-4
ANGLE = 1e-3          # radians, largest principal angle between leading-3 response-mode spans


def _dev(x, prec):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda",
                                                        dtype=torch.complex128 if prec == 0 else torch.complex64)


def _long_batch():
    """Instances of 1500, 2048 and 3000 points (two and four points per thread) next to short ones."""
    sysm = W.GL1D(n=(1500, 200, 2048, 64, 3000), mu0=(0.2, 0.1, 0.25, 0.0, 0.15))
    om = np.array([-1.5, -0.5, 0.5, 1.5])
    return W.Workload("gl_long", sysm, om, 0.0015, 2, "ssrm", n_transient_windows=1, seed=W.SEED_BASE + 61)


@pytest.mark.slow
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
def test_gl1d_long_instances_match_oracle(rsv, prec, adjoint):
    import torch
    w = _long_batch()
    op = rsv.create_for_workload(w, prec)
    try:
        fh = W.test_block(w)
        if prec == 1:
            fh = fh.astype(np.complex64).astype(np.complex128)
        x = _dev(fh, prec)
        y = torch.empty_like(x)
        (rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct)(op, x, w.k, y, **rsv.march_opts_for(w))
        g = frequencies.make_grid(w.omegas, w.dt)
        ref = march.march(operators.gl1d(w.system), g, fh, variant="ssrm", n_trans=1, adjoint=adjoint)
        err = rel_rows(y.cpu().numpy().astype(np.complex128), ref)
        assert err < (TOL64 if prec == 0 else TOL32_LONG), err
    finally:
        rsv.rsv_destroy_operator(op)


@pytest.mark.slow
@pytest.mark.parametrize("n", [512, 1024])
@pytest.mark.parametrize("adjoint", [False, True])
def test_dense_tensor_core_full_width(rsv, n, adjoint):
    """k = 32 in two chains of 16, the persistent kernel's full-size configuration; 4 frequencies on
    a 400-step window, 600-step unforced tail."""
    import torch
    sysm = W.Dense(n=n, x_half_width=110.0)
    om = np.pi * np.array([-1.5, -0.5, 0.5, 1.5])
    w = W.Workload("dense_wide", sysm, om, 0.005, 32, "trm", tail_steps=600, seed=W.SEED_BASE + 62)
    a = W.hermite_gl_matrix(sysm)
    op = rsv.create_for_workload(w, rsv.RSV_PREC_FP32, dense_matrix=a)
    try:
        assert "tcgen05 3xTF32 persistent" in rsv.rsv_describe(op)
        fh = W.test_block(w).astype(np.complex64).astype(np.complex128)
        x = _dev(fh, 1)
        y = torch.empty_like(x)
        (rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct)(op, x, w.k, y, **rsv.march_opts_for(w))
        assert "group=32" in rsv.rsv_describe(op)
        g = frequencies.make_grid(w.omegas, w.dt)
        ref = march.march(a, g, fh, variant="trm", tail_steps=w.tail_steps, adjoint=adjoint)
        err = rel_rows(y.cpu().numpy().astype(np.complex128), ref)
        assert err < TOL32, err
    finally:
        rsv.rsv_destroy_operator(op)


def _gain_case(kind):
    if kind == "gl1d":
        w = W.small_gl(n=60, n_omega=8, k=4, n_trans=4, mu0=-0.1)
        return w, operators.gl1d(w.system), None, None
    if kind == "gl_batch":
        sysm = W.GL1D(n=(40, 64, 50), mu0=(-0.1, -0.05, -0.2), x0=-20.0, x1=20.0)
        w = W.Workload("batch", sysm, np.linspace(-1.0, 1.0, 4), 0.05, 4, "ssrm", n_transient_windows=3)
        return w, operators.gl1d(sysm), None, [(0, 40), (40, 64), (104, 50)]
    if kind == "dense":
        sysm = W.Dense(n=48, x_half_width=20.0)
        w = W.Workload("dense_small", sysm, np.linspace(-1.0, 1.0, 8), 0.02, 4, "trm", tail_steps=2200)
        a = W.hermite_gl_matrix(sysm)
        return w, a, a, None
    if kind == "adr2d":
        sysm = W.ADR2D(nx=40, ny=24, lx=40.0, ly=10.0, sponge_cells=4, visc=0.05)
        dx = sysm.lx / (sysm.nx + 1)
        w = W.Workload("adr_small", sysm, np.linspace(0.0, 4.0, 8), 0.5 * dx, 4, "ssrm", n_transient_windows=2,
                       real_state=True, seed=W.SEED_BASE + 33)
        return w, operators.adr2d(sysm), None, None
    sysm = W.ADV3D(nx=12, ny=8, nz=6, lx=20.0, ly=10.0, lz=10.0, visc=0.1)
    dx = sysm.lx / (sysm.nx + 1)
    w = W.Workload("adv_small", sysm, np.array([0.04 * np.pi * 5 * j for j in range(6)]), 0.5 * dx, 4, "ssrm",
                   n_transient_windows=2, real_state=True, seed=W.SEED_BASE + 44)
    return w, operators.adv3d(sysm), None, None


@pytest.mark.parametrize("kind", ["gl1d", "gl_batch", "dense", "adr2d", "adv3d"])
def test_fp32_gains_match_oracle(rsv, kind):
    import torch
    w, a, dense, inst = _gain_case(kind)
    op = rsv.create_for_workload(w, rsv.RSV_PREC_FP32, dense_matrix=dense)
    try:
        fh = W.test_block(w).astype(np.complex64).astype(np.complex128)
        nm, q = 3, 1
        ni = len(inst) if inst else 1
        gains = np.zeros((ni, w.n_omega, nm))
        rm = torch.empty((w.n_omega, nm, w.n), dtype=torch.complex64, device="cuda")
        rsv.rsv_gains_modes(op, _dev(fh, 1), w.k, q, nm, gains, response_modes=rm, **rsv.march_opts_for(w, 64))
        g = frequencies.make_grid(w.omegas, w.dt)
        kw = dict(variant=w.variant, n_trans=w.n_transient_windows, tail_steps=w.tail_steps,
                  real_state=w.real_state)
        real_rows = [j for j, om in enumerate(w.omegas) if w.real_state and om == 0.0]
        rg, _, ru = rsvd.block_rsvd(lambda b: march.march(a, g, b, **kw),
                                    lambda b: march.march(a, g, b, adjoint=True, **kw), fh, q, nm,
                                    instances=inst, real_rows=real_rows)
        err = gain_rel(gains, rg)
        assert err < TOL_GAIN, err
        rmh = rm.cpu().numpy()
        segs = inst or [(0, w.n)]
        worst = 0.0
        for i, (off, size) in enumerate(segs):
            for j in range(w.n_omega):
                c = subspace_cos(rmh[j, :, off:off + size], ru[i][j])
                worst = max(worst, float(np.arccos(min(1.0, c))))
        assert worst < ANGLE, worst
    finally:
        rsv.rsv_destroy_operator(op)
