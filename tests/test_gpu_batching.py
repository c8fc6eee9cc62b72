"""GPU checks of the batching machinery against the oracle: packed launches of uneven 1-D batches,
CUDA-graph replay of the per-tile launch sequence, and the measured tile / vector-group choice.

Tolerances are those of the march parity tests: 1e-10 per frequency row in FP64, 2e-5 in FP32.
"""
import functools

import numpy as np
import pytest

import workloads as W
from oracle import frequencies, march, operators
from parity import rel_rows

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 2e-5


def _dev(x, prec):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda",
                                                        dtype=torch.complex128 if prec == 0 else torch.complex64)


def _uneven_batch(max_len):
    """Instances of the uneven 1-D batch (N log-uniform in [128, 2048], checked decaying): its 25
    shortest and, with max_len = 2048, its 3 longest, 6 test vectors: more (instance, vector) pairs
    than the GPU has SMs, so the launch packs several per CTA (FP32 CTAs of 1024 threads, FP64 of 512,
    with the fewest slots per thread that hold the longest instance)."""
    c5 = W.gl_batch_c5().system
    order = sorted(range(len(c5.n)), key=lambda i: c5.n[i])
    keep = order[:25] + (order[-3:] if max_len > 1024 else order[25:28])
    sysm = W.GL1D(n=tuple(c5.n[i] for i in keep), mu0=tuple(c5.mu0[i] for i in keep))
    om = np.array([-2.0, 0.0, 2.0])
    return W.Workload("gl_uneven", sysm, om, 0.003, 6, "ssrm", n_transient_windows=0, seed=W.SEED_BASE + 71)


@functools.lru_cache(maxsize=None)
def _uneven_case(max_len, adjoint):
    """Inputs (FP32-representable, so that both precisions march the same numbers) and the oracle."""
    w = _uneven_batch(max_len)
    fh = W.test_block(w).astype(np.complex64).astype(np.complex128)
    g = frequencies.make_grid(w.omegas, w.dt)
    ref = march.march(operators.gl1d(w.system), g, fh, variant="ssrm", n_trans=0, adjoint=adjoint)
    return w, fh, ref


@pytest.mark.parametrize("max_len", [1024, 2048])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
def test_packed_uneven_batch_matches_oracle(rsv, max_len, prec, adjoint):
    import torch
    w, fh, ref = _uneven_case(max_len, adjoint)
    assert len(w.system.n) * w.k > 152
    op = rsv.create_for_workload(w, prec)
    try:
        x = _dev(fh, prec)
        y = torch.empty_like(x)
        (rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct)(op, x, w.k, y, **rsv.march_opts_for(w))
        desc = rsv.rsv_describe(op)
        threads = 1024 if prec == 1 else 512
        slots = threads * -(-max(w.system.n) // threads)   # the fewest slots per thread holding the longest
        assert f"of {slots} slots" in desc, desc
        err = rel_rows(y.cpu().numpy().astype(np.complex128), ref)
        assert err < (TOL64 if prec == 0 else TOL32), err
    finally:
        rsv.rsv_destroy_operator(op)


@pytest.mark.parametrize("ppt", ["3", "4"])
@pytest.mark.parametrize("prec", [0, 1])
def test_packed_more_slots_per_thread(rsv, ppt, prec, monkeypatch):
    """Three or four slots per thread forced on the same batch (FP64's 512 threads need four slots for
    its longest instance, so a forced three is ignored there)."""
    import torch
    monkeypatch.setenv("RSV_GL1D_PPT", ppt)
    w, fh, ref = _uneven_case(2048, False)
    op = rsv.create_for_workload(w, prec)
    try:
        x = _dev(fh, prec)
        y = torch.empty_like(x)
        rsv.rsv_march_direct(op, x, w.k, y, **rsv.march_opts_for(w))
        slots = 1024 * int(ppt) if prec == 1 else 2048
        assert f"of {slots} slots" in rsv.rsv_describe(op)
        err = rel_rows(y.cpu().numpy().astype(np.complex128), ref)
        assert err < (TOL64 if prec == 0 else TOL32), err
    finally:
        rsv.rsv_destroy_operator(op)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
def test_packed_uneven_batch_trm_tail(rsv, prec, adjoint):
    """TRM on the packed batch in tiles of 37 steps: one tile straddles the end of the forcing window and
    the tail's tiles are unforced (no forcing copies, zero forcing reads)."""
    import torch
    w = _uneven_batch(1024)
    fh = W.test_block(w).astype(np.complex64).astype(np.complex128)
    g = frequencies.make_grid(w.omegas, w.dt)
    tail = 150
    assert g.n_t % 37 != 0
    ref = march.march(operators.gl1d(w.system), g, fh, variant="trm", tail_steps=tail, adjoint=adjoint)
    op = rsv.create_for_workload(w, prec)
    try:
        x = _dev(fh, prec)
        y = torch.empty_like(x)
        (rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct)(op, x, w.k, y, variant="trm",
                                                                      tail_steps=tail, tile_steps=37)
        assert "packed=" in rsv.rsv_describe(op)
        err = rel_rows(y.cpu().numpy().astype(np.complex128), ref)
        assert err < (TOL64 if prec == 0 else TOL32), err
    finally:
        rsv.rsv_destroy_operator(op)


def _fp32_tolerance(a, h):
    """FP32 march tolerance of one instance: rounding (6e-8 per operation, about eight roundings per
    step reaching the state) accumulates like a random walk over the slowest mode's decay time,
    1 / (|spectral abscissa| h) steps; twice that estimate, and no less than the short cases' 2e-5."""
    import scipy.sparse as sp
    dense = a.toarray() if sp.issparse(a) else np.asarray(a)
    decay_steps = 1.0 / (abs(np.linalg.eigvals(dense).real.max()) * h)
    return max(TOL32, 2 * 6e-8 * 8 * np.sqrt(decay_steps))


@pytest.mark.slow
def test_packed_full_batch_in_bench_launch_sampled(rsv):
    """The full 64-instance batch with its 8 test vectors in one group, in the bench's launch
    configuration (one wave of 152 CTAs x 3072 slots, three per thread), on the first 4 frequencies of
    its grid over one window (the window and the step are those of the full grid; the packing depends
    only on the instances and the vector group).  The shortest, the median and the longest instance,
    vectors 0 and 7, against the oracle marching each instance alone (the batch's operator is block
    diagonal), per frequency row, FP32."""
    import torch
    c5 = W.gl_batch_c5()
    w = W.Workload("gl_batch_sample", c5.system, c5.omegas[:4], c5.dt, c5.k, "ssrm", n_transient_windows=0,
                   seed=W.SEED_BASE + 75)
    fh = W.test_block(w).astype(np.complex64).astype(np.complex128)
    op = rsv.create_for_workload(w, 1)
    try:
        x = _dev(fh, 1)
        y = torch.empty_like(x)
        rsv.rsv_march_direct(op, x, w.k, y, **rsv.march_opts_for(w))
        desc = rsv.rsv_describe(op)
        assert "packed=152 ctas of 3072 slots (1024x3" in desc and "group=8" in desc, desc
        got = y.cpu().numpy().astype(np.complex128)
    finally:
        rsv.rsv_destroy_operator(op)
    g = frequencies.make_grid(w.omegas, w.dt)
    n = list(w.system.n)
    off = np.concatenate([[0], np.cumsum(n)])
    order = sorted(range(len(n)), key=lambda i: n[i])
    vecs = [0, w.k - 1]
    for i in (order[0], order[len(order) // 2], order[-1]):
        a = operators.gl1d(W.GL1D(n=(n[i],), mu0=(w.system.mu0[i],)))
        seg = slice(off[i], off[i + 1])
        ref = march.march(a, g, fh[:, vecs, seg], variant="ssrm", n_trans=0)
        err = rel_rows(got[:, vecs, seg], ref)
        tol = _fp32_tolerance(a, g.h)
        assert err < tol, (i, n[i], err, tol)


def _adr(k=3):
    sysm = W.ADR2D(nx=40, ny=24, lx=40.0, ly=10.0, sponge_cells=4)
    dx = sysm.lx / (sysm.nx + 1)
    return W.Workload("adr_graphs", sysm, np.linspace(0.0, 4.0, 8), 0.5 * dx, k, "ssrm", n_transient_windows=2,
                      real_state=True, seed=W.SEED_BASE + 72)


def _adv(k=2):
    sysm = W.ADV3D(nx=12, ny=8, nz=6, lx=20.0, ly=10.0, lz=10.0, visc=0.02)
    dx = sysm.lx / (sysm.nx + 1)
    return W.Workload("adv_graphs", sysm, np.array([0.04 * np.pi * 5 * j for j in range(6)]), 0.5 * dx, k,
                      "ssrm", n_transient_windows=2, real_state=True, seed=W.SEED_BASE + 73)


def _matrix(w):
    return operators.adr2d(w.system) if type(w.system).__name__ == "ADR2D" else operators.adv3d(w.system)


def _graphs(desc):
    return int(desc.split("graphs=")[1].split()[0])


@pytest.mark.parametrize("make", [_adr, _adv])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
def test_tile_graph_replay_matches_oracle(rsv, make, prec, adjoint):
    """Many short tiles (13 steps): the repeated tile sequences are captured once and replayed; two
    marches in a row reuse the graphs and give the same result bit for bit."""
    import torch
    w = make()
    op = rsv.create_for_workload(w, prec)
    try:
        fh = W.test_block(w)
        if prec == 1:
            fh = fh.astype(np.complex64).astype(np.complex128)
        x = _dev(fh, prec)
        y1 = torch.empty_like(x)
        y2 = torch.empty_like(x)
        f = rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct
        f(op, x, w.k, y1, **rsv.march_opts_for(w, tile_steps=13))
        first = _graphs(rsv.rsv_describe(op))
        f(op, x, w.k, y2, **rsv.march_opts_for(w, tile_steps=13))
        assert _graphs(rsv.rsv_describe(op)) > first > 0
        assert torch.equal(y1, y2)
        g = frequencies.make_grid(w.omegas, w.dt)
        ref = march.march(_matrix(w), g, fh, variant="ssrm", n_trans=2, adjoint=adjoint, real_state=True)
        err = rel_rows(y1.cpu().numpy().astype(np.complex128), ref)
        assert err < (TOL64 if prec == 0 else TOL32), err
    finally:
        rsv.rsv_destroy_operator(op)


@pytest.mark.parametrize("make,prec", [(_adr, 0), (_adr, 1), (_adv, 1)])
def test_autotune_choice_is_used_and_exact(rsv, make, prec):
    """The tuned (tile, group) is one of the candidates, later marches of k vectors use it, and their
    result still matches the oracle."""
    import torch
    w = make(k=4)
    op = rsv.create_for_workload(w, prec)
    try:
        fh = W.test_block(w)
        if prec == 1:
            fh = fh.astype(np.complex64).astype(np.complex128)
        x = _dev(fh, prec)
        opts = rsv.march_opts_for(w)
        tile, group = rsv.rsv_autotune(op, x, w.k, **opts)
        d = 256 if prec == 0 else 255
        assert tile in (d, d // 2) and group in (4, 2, 1)
        y = torch.empty_like(x)
        rsv.rsv_march_direct(op, x, w.k, y, **opts)
        desc = rsv.rsv_describe(op)
        assert f"tile={tile} group={group}" in desc and f"tuned={tile}/{group} for k=4" in desc, desc
        g = frequencies.make_grid(w.omegas, w.dt)
        ref = march.march(_matrix(w), g, fh, variant="ssrm", n_trans=2, real_state=True)
        err = rel_rows(y.cpu().numpy().astype(np.complex128), ref)
        assert err < (TOL64 if prec == 0 else TOL32), err
    finally:
        rsv.rsv_destroy_operator(op)


def _gl_small_k5():
    sysm = W.GL1D(n=(96,), mu0=(-0.1,))
    return W.Workload("gl_host", sysm, np.linspace(-1.0, 1.0, 6), 0.02, 5, "ssrm", n_transient_windows=1,
                      seed=W.SEED_BASE + 74)


@pytest.mark.parametrize("make,prec", [(_gl_small_k5, 0), (_gl_small_k5, 1), (lambda: _adr(k=5), 1),
                                       (lambda: _adv(k=5), 1)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_host_input_march_overlaps_and_matches(rsv, make, prec, adjoint):
    """Host-input march in groups of 2 vectors (groups 2, 2, 1: the staging buffers are refilled) =
    the device-input march, bit for bit, for pinned and pageable input; grouping does not change
    any vector's result; and the result matches the oracle."""
    import torch
    w = make()
    real = w.real_state
    op = rsv.create_for_workload(w, prec)
    try:
        fh = W.test_block(w)
        if prec == 1:
            fh = fh.astype(np.complex64).astype(np.complex128)
        x = _dev(fh, prec)
        y_dev = torch.empty_like(x)
        y_grp = torch.empty_like(x)
        y_pin = torch.empty_like(x)
        y_pag = torch.empty_like(x)
        opts = rsv.march_opts_for(w)
        f_dev = rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct
        f_host = rsv.rsv_march_adjoint_host if adjoint else rsv.rsv_march_direct_host
        f_dev(op, x, w.k, y_dev, **opts)
        f_dev(op, x, w.k, y_grp, group_vectors=2, **opts)
        assert "group=2" in rsv.rsv_describe(op)
        pinned = x.cpu().pin_memory()
        f_host(op, pinned, w.k, y_pin, group_vectors=2, **opts)
        f_host(op, x.cpu().numpy(), w.k, y_pag, group_vectors=2, **opts)
        assert torch.equal(y_dev, y_grp) and torch.equal(y_dev, y_pin) and torch.equal(y_dev, y_pag)
        g = frequencies.make_grid(w.omegas, w.dt)
        a = operators.gl1d(w.system) if not real else _matrix(w)
        ref = march.march(a, g, fh, variant="ssrm", n_trans=w.n_transient_windows, adjoint=adjoint, real_state=real)
        err = rel_rows(y_dev.cpu().numpy().astype(np.complex128), ref)
        assert err < (TOL64 if prec == 0 else TOL32), err
    finally:
        rsv.rsv_destroy_operator(op)
