"""GPU parity of the dense-operator path (spectral Ginzburg-Landau) against the FP64 oracle.

The CUDA path steps the exact RK4 map as one dense propagator product per
step; the oracle runs the four RK4 stages.  Both are the same discrete map,
so the FP64 path must agree to 1e-10.  At the full workload size
(n = 1024, 256 frequencies, k = 32, TRM over 120111 steps) the oracle's
march is out of reach, so sampled frequencies are checked against the
closed-form RK4 resolvent R_h(w) (which the oracle march reaches, pinned in
tests/test_oracle_pins.py) one frequency at a time.
"""
import numpy as np
import pytest

import workloads as W
from parity import gain_rel, rel_rows
from oracle import frequencies, march, resolvent, rsvd

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32_MARCH = 2e-5
TOL32_GAIN = 1e-4


def _small(variant="ssrm", k=3, n_omega=8, q=1):
    sysm = W.Dense(n=48, x_half_width=20.0)
    return W.Workload("dense_small", sysm, np.linspace(-1.0, 1.0, n_omega), 0.02, k, variant,
                      n_transient_windows=4, tail_steps=2200, n_power_iter=q, n_modes=3)


def _dev(x, prec):
    import torch
    dt = torch.complex128 if prec == 0 else torch.complex64
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dt)




def _oracle(w, a, fh, adjoint=False):
    g = frequencies.make_grid(w.omegas, w.dt)
    return march.march(a, g, fh, variant=w.variant, n_trans=w.n_transient_windows, tail_steps=w.tail_steps,
                       adjoint=adjoint)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
def test_dense_apply(rsv, prec, adjoint):
    w = _small()
    a = W.hermite_gl_matrix(w.system)
    op = rsv.create_for_workload(w, prec, dense_matrix=a)
    try:
        x = W.gaussian_block(5, 1, 5, 48)[0]
        y = _dev(x, prec) * 0
        rsv.rsv_apply_operator(op, _dev(x, prec), 5, adjoint, y)
        ref = ((a.conj().T if adjoint else a) @ x.T).T
        assert rel_rows(y.cpu().numpy(), ref) < (1e-13 if prec == 0 else 1e-6)
    finally:
        rsv.rsv_destroy_operator(op)


@pytest.mark.parametrize("variant,tile", [("ssrm", 64), ("ssrm", 100), ("trm", 256), ("trm", 7)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_dense_march_fp64(rsv, variant, tile, adjoint):
    w = _small(variant)
    a = W.hermite_gl_matrix(w.system)
    op = rsv.create_for_workload(w, 0, dense_matrix=a)
    try:
        fh = W.test_block(w)
        x = _dev(fh, 0)
        y = x * 0
        f = rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct
        f(op, x, w.k, y, **rsv.march_opts_for(w, tile_steps=tile))
        assert rel_rows(y.cpu().numpy(), _oracle(w, a, fh, adjoint)) < TOL64
    finally:
        rsv.rsv_destroy_operator(op)


@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("contract", ["tensor", "cuda_cores"])
def test_dense_march_fp32(rsv, adjoint, contract, monkeypatch):
    monkeypatch.setenv("RSV_CONTRACT_TENSOR", "1" if contract == "tensor" else "0")
    w = _small("trm", k=4)
    a = W.hermite_gl_matrix(w.system)
    op = rsv.create_for_workload(w, 1, dense_matrix=a)
    try:
        fh = W.test_block(w).astype(np.complex64).astype(np.complex128)
        x = _dev(fh, 1)
        y = x * 0
        f = rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct
        f(op, x, w.k, y, **rsv.march_opts_for(w, tile_steps=128))
        assert rel_rows(y.cpu().numpy().astype(np.complex128), _oracle(w, a, fh, adjoint)) < TOL32_MARCH
    finally:
        rsv.rsv_destroy_operator(op)


def test_dense_rsvd_fp64(rsv):
    w = _small("ssrm", k=4, q=2)
    a = W.hermite_gl_matrix(w.system)
    op = rsv.create_for_workload(w, 0, dense_matrix=a)
    try:
        fh = W.test_block(w)
        gains = np.zeros((1, w.n_omega, 3))
        rsv.rsv_gains_modes(op, _dev(fh, 0), w.k, w.n_power_iter, 3, gains, **rsv.march_opts_for(w, 128))
        g = frequencies.make_grid(w.omegas, w.dt)
        kw = dict(variant=w.variant, n_trans=w.n_transient_windows, tail_steps=w.tail_steps)
        rg, _, _ = rsvd.block_rsvd(lambda b: march.march(a, g, b, **kw),
                                   lambda b: march.march(a, g, b, adjoint=True, **kw), fh, w.n_power_iter, 3)
        assert gain_rel(gains, rg) < TOL64
    finally:
        rsv.rsv_destroy_operator(op)


def _closed_form_rsvd(a, h, om, omega_j, q, n_modes):
    """The randomized SVD of one frequency with the action R_h(w) applied in closed form."""
    rh = resolvent.rk4_discrete(a, om, h)
    block = omega_j[None]
    md = lambda b: (rh @ b[0].T).T[None]
    ma = lambda b: (rh.conj().T @ b[0].T).T[None]
    gains, _, _ = rsvd.block_rsvd(md, ma, block, q, n_modes)
    return gains[0, 0], rh


@pytest.mark.slow
def test_dense_full_size_sampled(rsv):
    """Full spectral-GL workload: FP32 march and rSVD gains at sampled frequencies vs closed form."""
    import torch
    w = W.dense_hermite_c2()
    a = W.hermite_gl_matrix(w.system)
    op = rsv.create_for_workload(w, 1, dense_matrix=a)
    try:
        h = frequencies.make_grid(w.omegas, w.dt).h
        fh = W.test_block(w)
        x = _dev(fh, 1)
        gains = np.zeros((1, w.n_omega, 3))
        rsv.rsv_gains_modes(op, x, w.k, w.n_power_iter, 3, gains, **rsv.march_opts_for(w))
        for j in (0, 77, 128, 255):
            ref, rh = _closed_form_rsvd(a, h, w.omegas[j], fh[j].astype(np.complex64).astype(np.complex128),
                                        w.n_power_iter, 3)
            err = np.abs(gains[0, j] - ref) / ref
            assert err.max() < TOL32_GAIN, (j, gains[0, j], ref)
        # one direct march, element-wise at a sampled frequency
        y = torch.empty_like(x)
        rsv.rsv_march_direct(op, x, w.k, y, **rsv.march_opts_for(w))
        j = 100
        rh = resolvent.rk4_discrete(a, w.omegas[j], h)
        ref = (rh @ fh[j].astype(np.complex64).astype(np.complex128).T).T
        assert rel_rows(y[j].cpu().numpy().astype(np.complex128), ref) < 1e-4
    finally:
        rsv.rsv_destroy_operator(op)


@pytest.mark.parametrize("n,x_half", [(128, 30.0), (256, 40.0)])
@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("path,k", [("persistent", 5), ("persistent", 20), ("per_step", 5), ("cuda_cores", 5)])
def test_dense_tensor_core_step(rsv, n, x_half, adjoint, path, k, monkeypatch):
    """FP32 dense march on the tcgen05 paths (persistent tile kernel with one or two vector
    chains, one launch per step) and on the CUDA-core step, vs the oracle."""
    monkeypatch.setenv("RSV_DENSE_TENSOR", "0" if path == "cuda_cores" else "1")
    monkeypatch.setenv("RSV_DENSE_PERSISTENT", "0" if path == "per_step" else "1")
    sysm = W.Dense(n=n, x_half_width=x_half)
    w = W.Workload("dense_tc", sysm, np.linspace(-1.0, 1.0, 8), 0.01, k, "trm", tail_steps=2200)
    a = W.hermite_gl_matrix(sysm)
    op = rsv.create_for_workload(w, 1, dense_matrix=a)
    try:
        fh = W.test_block(w).astype(np.complex64).astype(np.complex128)
        x = _dev(fh, 1)
        y = x * 0
        f = rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct
        f(op, x, w.k, y, **rsv.march_opts_for(w, tile_steps=200))
        assert rel_rows(y.cpu().numpy().astype(np.complex128), _oracle(w, a, fh, adjoint)) < TOL32_MARCH
    finally:
        rsv.rsv_destroy_operator(op)


def test_dense_fp32_size_outside_tensor_tiles(rsv):
    """n = 384: three 128-column K slices do not split a 64-row block evenly, so the FP32 path
    takes the CUDA-core propagator step; it still matches the oracle."""
    sysm = W.Dense(n=384, x_half_width=60.0)          # RK4 stable at dt = 0.01 (max |M| = 0.998)
    w = W.Workload("dense_384", sysm, np.linspace(-1.0, 1.0, 8), 0.01, 3, "trm", tail_steps=2200)
    a = W.hermite_gl_matrix(sysm)
    op = rsv.create_for_workload(w, 1, dense_matrix=a)
    try:
        assert "cuda-core propagator step" in rsv.rsv_describe(op)
        fh = W.test_block(w).astype(np.complex64).astype(np.complex128)
        x = _dev(fh, 1)
        y = x * 0
        rsv.rsv_march_direct(op, x, w.k, y, **rsv.march_opts_for(w, tile_steps=200))
        assert rel_rows(y.cpu().numpy().astype(np.complex128), _oracle(w, a, fh)) < TOL32_MARCH
    finally:
        rsv.rsv_destroy_operator(op)


def test_bounded_wait_runs_out(rsv, monkeypatch):
    """Failure detection without a GPU fault: with the test hook RSV_TEST_STALL_WAIT=1 the dense
    persistent kernel's first wait targets a step count that nothing reaches; with the limit
    RSV_WAIT_LIMIT_NS = 200 us the wait gives up, the kernel finishes every step without issuing
    copies or products, frees its tensor memory and returns, and the march reports RSV_ERR_TIMEOUT.
    An operator created afterwards marches correctly (the context stays usable)."""
    import time
    import torch
    sysm = W.Dense(n=128, x_half_width=30.0)
    w = W.Workload("dense_stall", sysm, np.linspace(-1.0, 1.0, 8), 0.01, 5, "trm", tail_steps=300)
    a = W.hermite_gl_matrix(sysm)
    fh = W.test_block(w).astype(np.complex64).astype(np.complex128)
    monkeypatch.setenv("RSV_TEST_STALL_WAIT", "1")
    monkeypatch.setenv("RSV_WAIT_LIMIT_NS", "200000")
    op = rsv.create_for_workload(w, 1, dense_matrix=a)
    try:
        assert "tcgen05 3xTF32 persistent" in rsv.rsv_describe(op)
        x = _dev(fh, 1)
        y = torch.empty_like(x)
        t0 = time.perf_counter()
        with pytest.raises(rsv.RsvError) as e:
            rsv.rsv_march_direct(op, x, w.k, y, **rsv.march_opts_for(w, tile_steps=256))
        assert e.value.status == 5, e.value
        assert time.perf_counter() - t0 < 20.0
    finally:
        rsv.rsv_destroy_operator(op)
    monkeypatch.delenv("RSV_TEST_STALL_WAIT")
    monkeypatch.delenv("RSV_WAIT_LIMIT_NS")
    op = rsv.create_for_workload(w, 1, dense_matrix=a)
    try:
        x = _dev(fh, 1)
        y = torch.empty_like(x)
        rsv.rsv_march_direct(op, x, w.k, y, **rsv.march_opts_for(w, tile_steps=256))
        assert rel_rows(y.cpu().numpy().astype(np.complex128), _oracle(w, a, fh)) < TOL32_MARCH
    finally:
        rsv.rsv_destroy_operator(op)
