"""The k-split randomized SVD driver with the library's march and orthonormalisation, on one GPU.

distributed.library_callables backs distributed_rsvd with rsv_march_direct /
rsv_march_adjoint (an operator holding every frequency) and rsv_orthonormalize
(an operator holding this rank's frequencies, set with the full grid's
spacing).  A one-rank NCCL group runs it on the single GPU: its gains must
equal rsv_gains_modes' (FP64, 1e-10), and rsv_set_frequencies on a frequency
subset with the full grid's spacing must keep the window and step.
"""
import os
import socket

import numpy as np
import pytest

import workloads as W
from parity import gain_rel

pytestmark = pytest.mark.gpu


def test_distributed_rsvd_one_rank_equals_gains_modes(rsv):
    import torch
    import torch.distributed as dist
    from paper_2008_10904_gb300 import distributed as D
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    w = W.small_gl(n=40, n_omega=8, k=4, n_trans=6, mu0=-0.1)
    op_all = rsv.create_for_workload(w, rsv.RSV_PREC_FP64)
    d, keep = rsv.desc_for(w.system, w.dt, rsv.RSV_PREC_FP64)
    op_chunk = rsv.rsv_create_operator(d, keep=keep)
    try:
        n_t, h = rsv.rsv_set_frequencies(op_all, w.omegas)
        dw = w.omegas[1] - w.omegas[0]
        n_t2, h2 = rsv.rsv_set_frequencies(op_chunk, w.omegas[2:5], dw)   # a subset keeps the grid
        assert n_t2 == n_t and abs(h2 - h) < 1e-15
        rsv.rsv_set_frequencies(op_chunk, w.omegas, dw)
        opts = rsv.march_opts_for(w, 64)
        march, orth = D.library_callables(op_all, op_chunk, opts)
        x = torch.from_numpy(W.test_block(w)).cuda()
        gains = D.distributed_rsvd(march, orth, x, [w.k], [w.n_omega], 1, 3)
        ref = np.zeros((1, w.n_omega, 3))
        rsv.rsv_gains_modes(op_all, x, w.k, 1, 3, ref, **opts)
        assert gain_rel(gains, ref) < 1e-10
    finally:
        rsv.rsv_destroy_operator(op_all)
        rsv.rsv_destroy_operator(op_chunk)
        dist.destroy_process_group()
