"""GPU parity of the FP64 1-D march on thread-block clusters against the oracle.

FP64 RK4 marches of few (instance, vector) pairs spread each pair over a cluster of 2 to 16 CTAs, each
owning a contiguous chunk of points and reading the points beyond its ends (4 per step between
exchanges) from the CTAs that own them.  These tests take that path (the describe line names the
cluster size) and compare with the oracle element by element, each frequency row against its own
largest entry, within 1e-10:

* the 256-point single-instance case: with 4 test vectors clusters of 16 CTAs of 16 points exchanging
  every 2 steps (where the device takes 16-CTA clusters, else 8), with 10 vectors (16-CTA clusters
  would not fit in one wave) clusters of 8 CTAs of 32 points exchanging every step; SSRM and TRM,
  direct and adjoint, ragged tiles (odd tile lengths end tiles between two exchanges);
* an uneven batch with a 5-point instance (CTAs of its cluster that own no point still take part in
  every cluster barrier) and a 70-point one (a short last chunk);
* the norm-truncated TRM tail: the state each clustered tile leaves decides where the tail stops.
"""
import numpy as np
import pytest

import workloads as W
from oracle import frequencies, march, operators
from parity import rel_rows

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=torch.complex128)


def _cluster(desc):
    return int(desc.split("cluster=")[1].split()[0]) if "cluster=" in desc else 0


@pytest.mark.parametrize("k,clusters", [(4, (16, 8)), (10, (8,))])
@pytest.mark.parametrize("variant,tile", [("ssrm", 37), ("trm", 100)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_single_instance_on_clusters(rsv, k, clusters, variant, tile, adjoint):
    import torch
    w = W.small_gl(n=256, n_omega=8, k=k, variant=variant, n_trans=1, tail_steps=300, mu0=-0.1, dt=0.02,
                   x_half=40.0)
    op = rsv.create_for_workload(w, rsv.RSV_PREC_FP64)
    try:
        fh = W.test_block(w)
        x = _dev(fh)
        y = torch.empty_like(x)
        (rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct)(op, x, w.k, y,
                                                                      **rsv.march_opts_for(w, tile_steps=tile))
        assert _cluster(rsv.rsv_describe(op)) in clusters, rsv.rsv_describe(op)
        g = frequencies.make_grid(w.omegas, w.dt)
        ref = march.march(operators.gl1d(w.system), g, fh, variant=variant, n_trans=1, tail_steps=300,
                          adjoint=adjoint)
        assert rel_rows(y.cpu().numpy(), ref) < TOL64
    finally:
        rsv.rsv_destroy_operator(op)


def _uneven():
    sysm = W.GL1D(n=(5, 256, 70), mu0=(-0.2, -0.1, 0.0), x0=-40.0, x1=40.0)
    return W.Workload("gl_cluster_uneven", sysm, np.linspace(-1.0, 1.0, 6), 0.02, 3, "ssrm",
                      n_transient_windows=1, seed=W.SEED_BASE + 76)


@pytest.mark.parametrize("adjoint", [False, True])
def test_uneven_batch_on_clusters(rsv, adjoint):
    import torch
    w = _uneven()
    op = rsv.create_for_workload(w, rsv.RSV_PREC_FP64)
    try:
        fh = W.test_block(w)
        x = _dev(fh)
        y = torch.empty_like(x)
        (rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct)(op, x, w.k, y,
                                                                      **rsv.march_opts_for(w, tile_steps=50))
        assert _cluster(rsv.rsv_describe(op)) in (16, 8), rsv.rsv_describe(op)
        g = frequencies.make_grid(w.omegas, w.dt)
        ref = march.march(operators.gl1d(w.system), g, fh, variant="ssrm", n_trans=1, adjoint=adjoint)
        assert rel_rows(y.cpu().numpy(), ref) < TOL64
    finally:
        rsv.rsv_destroy_operator(op)


@pytest.mark.parametrize("adjoint", [False, True])
def test_norm_truncated_tail_on_clusters(rsv, adjoint):
    """TRM with tail_tol: the library stops at the first tile end where every vector's norm (of the
    state the clustered tiles leave) is at most tail_tol times its largest so far; the oracle applies
    the same rule at the same check points, so the step counts and the coefficients agree."""
    import torch
    w = _uneven()
    g = frequencies.make_grid(w.omegas, w.dt)
    cap, tol, tile = 200 * g.n_t, 1e-6, 64
    op = rsv.create_for_workload(w, rsv.RSV_PREC_FP64)
    try:
        fh = W.test_block(w)
        x = _dev(fh)
        y = torch.empty_like(x)
        (rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct)(op, x, w.k, y, variant="trm", tail_steps=cap,
                                                                      tile_steps=tile, tail_tol=tol)
        desc = rsv.rsv_describe(op)
        assert _cluster(desc) in (16, 8), desc
        ref, steps = march.march(operators.gl1d(w.system), g, fh, variant="trm", tail_steps=cap, adjoint=adjoint,
                                 tail_tol=tol, check_every=tile, return_steps=True)
        assert g.n_t <= steps < g.n_t + cap
        assert int(desc.split("steps=")[1].split()[0]) == steps
        assert rel_rows(y.cpu().numpy(), ref) < TOL64
    finally:
        rsv.rsv_destroy_operator(op)
