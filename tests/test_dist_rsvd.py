"""The k-split randomized SVD across ranks, on CPU: world size 2 over gloo.

Each rank marches its share of the test vectors for every frequency; between
marches two all-to-alls regroup the Fourier blocks by frequency for the
per-frequency QR and back.  Here the marches and QRs are the FP64 oracle's, so
the distributed result must equal the single-process oracle randomized SVD;
the regroup itself must be an exact round trip for uneven splits.
"""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _block(seed, nw, k, n):
    return W.gaussian_block(seed, nw, k, n)


def _worker(rank, world, port, results):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2008_10904_gb300 import distributed as D
    from oracle import frequencies, march, operators, rsvd

    # 1. regroup round trip with uneven splits
    k_counts, f_counts, n = [3, 1], [3, 2], 7
    mine = torch.from_numpy(_block(100 + rank, 5, k_counts[rank], n))
    full = np.concatenate([_block(100 + s, 5, k_counts[s], n) for s in range(world)], axis=1)
    bf = D.regroup_to_frequencies(mine, k_counts, f_counts)
    fo = np.concatenate([[0], np.cumsum(f_counts)])
    ok_f = np.array_equal(bf.numpy(), full[fo[rank]:fo[rank + 1]])
    back = D.regroup_to_vectors(bf, k_counts, f_counts)
    ok_b = np.array_equal(back.numpy(), mine.numpy())

    # 2. the distributed randomized SVD with oracle marches and QRs = the oracle's own
    w = W.small_gl(n=30, n_omega=6, k=4, n_trans=6, mu0=-0.1)
    a = operators.gl1d(w.system)
    g = frequencies.make_grid(w.omegas, w.dt)
    kc = D.split_counts(w.k, world)
    fc = D.split_counts(w.n_omega, world)
    ko = np.concatenate([[0], np.cumsum(kc)])
    omega_all = W.test_block(w)

    def mrch(block, adjoint):
        out = march.march(a, g, block.numpy(), variant="ssrm", n_trans=w.n_transient_windows, adjoint=adjoint)
        return torch.from_numpy(out)

    def orth(block_f):
        b = block_f.numpy()
        q = np.empty_like(b)
        r = np.empty((b.shape[0], 1, b.shape[1], b.shape[1]), dtype=np.complex128)
        for j in range(b.shape[0]):
            qq, rr = rsvd.qr_positive(b[j].T)
            q[j] = qq.T
            r[j, 0] = rr
        return torch.from_numpy(q), torch.from_numpy(r)

    gains = D.distributed_rsvd(mrch, orth, torch.from_numpy(omega_all[:, ko[rank]:ko[rank + 1]].copy()), kc, fc,
                               1, 3)
    results[rank] = (ok_f, ok_b, gains)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_k_split_rsvd_equals_oracle():
    from oracle import frequencies, march, operators, rsvd
    world, port = 2, _free_port()
    mgr = mp.Manager()
    results = mgr.dict()
    mp.spawn(_worker, args=(world, port, results), nprocs=world, join=True)
    for r in range(world):
        assert results[r][0] and results[r][1]           # regroup and its inverse are exact
    w = W.small_gl(n=30, n_omega=6, k=4, n_trans=6, mu0=-0.1)
    a = operators.gl1d(w.system)
    g = frequencies.make_grid(w.omegas, w.dt)
    kw = dict(variant="ssrm", n_trans=w.n_transient_windows)
    ref, _, _ = rsvd.block_rsvd(lambda b: march.march(a, g, b, **kw), lambda b: march.march(a, g, b, adjoint=True, **kw),
                                W.test_block(w), 1, 3)
    got = np.concatenate([results[0][2], results[1][2]], axis=1)   # [inst][n_omega][modes]
    assert np.allclose(got, ref, rtol=1e-12), np.abs(got - ref).max()


def test_split_counts():
    from paper_2008_10904_gb300 import distributed as D
    assert D.split_counts(8, 3) == [3, 3, 2]
    assert D.split_counts(4, 4) == [1, 1, 1, 1]
    assert sum(D.split_counts(64, 5)) == 64
