"""GPU parity of the decay run, the automatic SSRM transient length, the FP64
refinement pass and the block orthonormalisation, against the oracle.

* rsv_decay_probe (Sec. 2.3: transient length from the decay of a random
  state) must stop after exactly the oracle's step count in FP64 (same
  SplitMix64 initial state, same check points, per-instance ratios); in FP32
  within one check interval.  A growing system is reported as UNSTABLE.
* n_transient_windows = -1 must march the windows the probe sets.
* rsv_refine_gains (App. A, Rayleigh-Ritz on a basis) must match the
  oracle's refinement to 1e-10 in FP64, and on the basis of an FP32
  randomized SVD it must cut the FP32 gain error to about its square.
* rsv_orthonormalize must return the unique QR with a positive diagonal.
"""
import numpy as np
import pytest

import workloads as W
from oracle import decay, frequencies, march, operators, resolvent, rsvd
from parity import gain_rel, rel_rows

pytestmark = pytest.mark.gpu


def _dev(x, prec):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda",
                                                        dtype=torch.complex128 if prec == 0 else torch.complex64)


def _probe_case(kind):
    """(workload, system matrix, dense matrix or None, instances) of a small system of each kind."""
    if kind == "gl1d":
        sysm = W.GL1D(n=(40, 64, 25), mu0=(-0.1, 0.05, -0.2), x0=-20.0, x1=20.0)
        w = W.Workload("probe_gl", sysm, np.linspace(-1.0, 1.0, 4), 0.05, 1, "ssrm")
        return w, operators.gl1d(sysm), None, [(0, 40), (40, 64), (104, 25)]
    if kind == "dense":
        sysm = W.Dense(n=48, x_half_width=20.0)
        w = W.Workload("probe_dense", sysm, np.linspace(-1.0, 1.0, 4), 0.02, 1, "ssrm")
        a = W.hermite_gl_matrix(sysm)
        return w, a, a, None
    if kind == "adr2d":
        sysm = W.ADR2D(nx=40, ny=24, lx=40.0, ly=10.0, sponge_cells=4, visc=0.05)
        dx = sysm.lx / (sysm.nx + 1)
        w = W.Workload("probe_adr", sysm, np.linspace(0.0, 4.0, 8), 0.5 * dx, 1, "ssrm", real_state=True)
        return w, operators.adr2d(sysm), None, None
    sysm = W.ADV3D(nx=12, ny=8, nz=6, lx=20.0, ly=10.0, lz=10.0, visc=0.3)
    dx = sysm.lx / (sysm.nx + 1)
    w = W.Workload("probe_adv", sysm, np.array([0.04 * np.pi * 5 * j for j in range(6)]), 0.5 * dx, 1, "ssrm",
                   real_state=True)
    return w, operators.adv3d(sysm), None, None


@pytest.mark.parametrize("kind", ["gl1d", "dense", "adr2d", "adv3d"])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
def test_decay_probe_matches_oracle(rsv, kind, prec, adjoint):
    w, a, dense, inst = _probe_case(kind)
    g = frequencies.make_grid(w.omegas, w.dt)
    tol, seed, every = 1e-6, 77, 25
    op = rsv.create_for_workload(w, prec, dense_matrix=dense)
    try:
        steps, ratio = rsv.rsv_decay_probe(op, tol, 10 ** 6, seed=seed, check_every=every, adjoint=adjoint)
        u0 = decay.initial_state(w.n, seed, not w.real_state)
        if prec == 1:
            u0 = u0.astype(np.complex64 if not w.real_state else np.float32).astype(u0.dtype)
        aa = a.conj().T if adjoint else a
        ref_steps, ref_ratio, status = decay.decay_probe(aa, g.h, u0, tol, 10 ** 6, every, instances=inst)
        assert status == "decayed" and ratio <= tol
        if prec == 0:
            assert steps == ref_steps, (steps, ref_steps)
            assert abs(ratio / ref_ratio - 1.0) < 1e-9
        else:
            assert abs(steps - ref_steps) <= every, (steps, ref_steps)
    finally:
        rsv.rsv_destroy_operator(op)


def test_decay_probe_reports_unstable(rsv):
    sysm = W.GL1D(n=(32,), mu0=(2.0,), x0=-5.0, x1=5.0)
    w = W.Workload("grow", sysm, np.linspace(-1.0, 1.0, 4), 0.05, 1, "ssrm")
    op = rsv.create_for_workload(w, rsv.RSV_PREC_FP64)
    try:
        with pytest.raises(rsv.RsvError) as e:
            rsv.rsv_decay_probe(op, 1e-6, 10 ** 6, check_every=50)
        assert e.value.status == 2 and "grew" in str(e.value)
        x = _dev(W.test_block(w), 0)
        with pytest.raises(rsv.RsvError) as e:
            rsv.rsv_march_direct(op, x, 1, x * 0, variant="ssrm", n_transient_windows=-1)
        assert e.value.status == 2
    finally:
        rsv.rsv_destroy_operator(op)
    # a stable system that has not decayed within the cap is reported too
    w = W.small_gl(n=24, mu0=-0.05)
    op = rsv.create_for_workload(w, rsv.RSV_PREC_FP64)
    try:
        with pytest.raises(rsv.RsvError) as e:
            rsv.rsv_decay_probe(op, 1e-12, 100, check_every=50)
        assert e.value.status == 2 and "did not fall" in str(e.value)
    finally:
        rsv.rsv_destroy_operator(op)


@pytest.mark.parametrize("prec", [0, 1])
def test_auto_transient_windows(rsv, prec):
    """n_transient_windows = -1 marches ceil(probe steps / N_T) transient windows (decay_tol,
    decay_seed, check points every tile), the same as giving that number explicitly, and the
    oracle on that schedule."""
    import torch
    w = W.small_gl(n=40, n_omega=8, k=2, mu0=-0.1)
    g = frequencies.make_grid(w.omegas, w.dt)
    op = rsv.create_for_workload(w, prec)
    try:
        tile, tol, seed = 64, 1e-8, 5
        steps, _ = rsv.rsv_decay_probe(op, tol, 1000 * g.n_t, seed=seed, check_every=tile)
        nt = decay.transient_windows(steps, g.n_t)
        fh = W.test_block(w)
        if prec == 1:
            fh = fh.astype(np.complex64).astype(np.complex128)
        x = _dev(fh, prec)
        y_auto, y_expl = torch.empty_like(x), torch.empty_like(x)
        rsv.rsv_march_direct(op, x, w.k, y_auto, variant="ssrm", n_transient_windows=-1, tile_steps=tile,
                             decay_tol=tol, decay_seed=seed)
        rsv.rsv_march_direct(op, x, w.k, y_expl, variant="ssrm", n_transient_windows=nt, tile_steps=tile)
        assert torch.equal(y_auto, y_expl)
        desc = dict(kv.split("=", 1) for kv in rsv.rsv_describe(op).split() if "=" in kv)
        assert int(desc["steps"]) == (nt + 1) * g.n_t
        ref = march.march(operators.gl1d(w.system), g, fh, variant="ssrm", n_trans=nt)
        assert rel_rows(y_auto.cpu().numpy().astype(np.complex128), ref) < (1e-10 if prec == 0 else 2e-5)
        # the probe's own oracle count
        u0 = decay.initial_state(w.n, seed, True)
        ref_steps, _, _ = decay.decay_probe(operators.gl1d(w.system), g.h, u0, tol, 1000 * g.n_t, tile)
        if prec == 0:
            assert steps == ref_steps
    finally:
        rsv.rsv_destroy_operator(op)


def test_orthonormalize_is_unique_qr(rsv):
    sysm = W.GL1D(n=(40, 64, 50), mu0=(-0.1, -0.05, -0.2), x0=-20.0, x1=20.0)
    w = W.Workload("batch", sysm, np.linspace(-1.0, 1.0, 4), 0.05, 5, "ssrm")
    op = rsv.create_for_workload(w, rsv.RSV_PREC_FP64)
    try:
        x = W.test_block(w)
        xd = _dev(x, 0)
        r = np.zeros((w.n_omega, 3, w.k, w.k), dtype=np.complex128)
        rsv.rsv_orthonormalize(op, xd, w.k, r)
        q = xd.cpu().numpy()
        inst = [(0, 40), (40, 64), (104, 50)]
        ref = rsvd.orthonormalize(x, inst)
        assert np.abs(q - ref).max() < 1e-12
        for j in range(w.n_omega):
            for i, (off, size) in enumerate(inst):
                rr = r[j, i]
                assert np.allclose(np.tril(rr, -1), 0) and np.all(np.diag(rr).real > 0)
                assert np.allclose(np.diag(rr).imag, 0, atol=1e-13)
                assert np.abs(rr.T @ q[j, :, off:off + size] - x[j, :, off:off + size]).max() < 1e-12
    finally:
        rsv.rsv_destroy_operator(op)


def _refine_case(k=6, q=4):
    w = W.small_gl(n=40, n_omega=8, k=k, n_trans=12, mu0=-0.1, q=q)
    return W.Workload(w.name, w.system, w.omegas, w.dt, k, "ssrm", n_transient_windows=12, n_power_iter=q,
                      n_modes=3, seed=w.seed)


def test_refine_fp64_matches_oracle(rsv):
    import torch
    w = _refine_case()
    a = operators.gl1d(w.system)
    g = frequencies.make_grid(w.omegas, w.dt)
    op = rsv.create_for_workload(w, rsv.RSV_PREC_FP64)
    try:
        basis = W.test_block(w)
        gains = np.zeros((1, w.n_omega, 3))
        fm = torch.empty((w.n_omega, 3, w.n), dtype=torch.complex128, device="cuda")
        rm = torch.empty_like(fm)
        rsv.rsv_refine_gains(op, _dev(basis, 0), w.k, 3, gains, fm, rm, **rsv.march_opts_for(w, 64))
        md = lambda b: march.march(a, g, b, variant="ssrm", n_trans=w.n_transient_windows)
        rg, rv, ru = rsvd.rayleigh_ritz_refine(md, basis, 3)
        assert gain_rel(gains, rg) < 1e-10
        fmh, rmh = fm.cpu().numpy(), rm.cpu().numpy()
        for j in range(w.n_omega):
            for m in range(3):
                assert abs(abs(np.vdot(fmh[j, m], rv[0][j][m])) - 1) < 1e-8
                assert abs(abs(np.vdot(rmh[j, m], ru[0][j][m])) - 1) < 1e-8
    finally:
        rsv.rsv_destroy_operator(op)


def test_fp64_refinement_of_fp32_rsvd(rsv):
    """FP32 randomized SVD, then the FP64 refinement pass on its forcing modes: the refined gains equal
    the oracle's refinement of that basis (1e-10), and their error against svd(R_h) falls to about the
    square of the FP32 gain error.  Twelve test vectors and eight power iterations converge the
    subspace (algorithmic error 5e-11 in FP64), so the FP32 error is the precision's."""
    import torch
    w = _refine_case(k=12, q=8)
    a = operators.gl1d(w.system)
    g = frequencies.make_grid(w.omegas, w.dt)
    op32 = rsv.create_for_workload(w, rsv.RSV_PREC_FP32)
    op64 = rsv.create_for_workload(w, rsv.RSV_PREC_FP64)
    try:
        opts = rsv.march_opts_for(w, 64)
        x = W.test_block(w)
        g32 = np.zeros((1, w.n_omega, w.k))
        v32 = torch.empty((w.n_omega, w.k, w.n), dtype=torch.complex64, device="cuda")
        rsv.rsv_gains_modes(op32, _dev(x, 1), w.k, w.n_power_iter, w.k, g32, forcing_modes=v32, **opts)
        basis = v32.to(torch.complex128).contiguous()
        gref = np.zeros((1, w.n_omega, 3))
        rsv.rsv_refine_gains(op64, basis, w.k, 3, gref, **opts)
        md = lambda b: march.march(a, g, b, variant="ssrm", n_trans=w.n_transient_windows)
        og, _, _ = rsvd.rayleigh_ritz_refine(md, basis.cpu().numpy(), 3)
        assert gain_rel(gref, og) < 1e-10
        exact = np.array([np.linalg.svd(resolvent.rk4_discrete(a, om, g.h), compute_uv=False)[:3]
                          for om in g.omegas])[None]
        e32 = gain_rel(g32[:, :, :3], exact)
        eref = gain_rel(gref, exact)
        print(f"FP32 rSVD gain error {e32:.2e}, after FP64 refinement {eref:.2e}")
        assert e32 < 1e-4
        assert eref < max(10 * e32 ** 2, 1e-9) and eref < 1e-2 * e32, (e32, eref)
    finally:
        rsv.rsv_destroy_operator(op32)
        rsv.rsv_destroy_operator(op64)
