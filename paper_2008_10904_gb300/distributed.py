"""Randomized SVD with the test vectors split across ranks (one GPU per rank).

The marches of different test vectors are independent, so each rank marches
its own share k_r of the k vectors for every frequency, with no communication.
The per-frequency block algebra (the CholeskyQR2 orthonormalisation and the
final small SVD, Sec. 2.3's normalisation and orthogonalisation on Fourier
coefficients) needs all k vectors of a frequency together: between marches one
all-to-all regroups the Fourier blocks from [n_omega][k_r][n] (all
frequencies, this rank's vectors) to [n_omega_r][k][n] (this rank's
frequencies, all vectors), and a second all-to-all sends them back.  These
two exchanges are the only data-path collectives.

The numerical work is passed in as callables, so the same driver runs the
library (march through rsv_march_direct / rsv_march_adjoint of an operator
holding all frequencies; orthonormalisation through rsv_orthonormalize of an
operator holding this rank's frequencies) or any other implementation of the
same steps:

    march(block, adjoint) -> block            [n_omega][k_r][n] -> [n_omega][k_r][n]
    orthonormalize(block_f) -> (q_f, r)       [n_omega_r][k][n] -> same, r [n_omega_r][n_inst][k][k]
                                              (block = Q R per frequency and instance)

Blocks are torch tensors (CPU for gloo, CUDA for NCCL); the all-to-all is
torch.distributed.all_to_all_single on contiguous buffers.
"""
from __future__ import annotations

import numpy as np


def split_counts(total: int, world: int) -> list[int]:
    """Balanced split of `total` items over `world` ranks (the first ranks take one more)."""
    base, extra = divmod(total, world)
    return [base + (1 if r < extra else 0) for r in range(world)]


def _offsets(counts):
    return np.concatenate([[0], np.cumsum(counts)]).astype(int)


def regroup_to_frequencies(block, k_counts, f_counts, group=None):
    """[n_omega][k_r][n] on every rank -> [n_omega_r][k][n]: this rank's frequencies, all vectors."""
    import torch
    import torch.distributed as dist
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    n = block.shape[2]
    kr = k_counts[rank]
    foff = _offsets(f_counts)
    send = torch.cat([block[foff[s]:foff[s + 1]].reshape(-1) for s in range(world)]).contiguous()
    in_sizes = [f_counts[s] * kr * n for s in range(world)]
    out_sizes = [f_counts[rank] * k_counts[s] * n for s in range(world)]
    recv = torch.empty(sum(out_sizes), dtype=block.dtype, device=block.device)
    dist.all_to_all_single(recv, send, out_sizes, in_sizes, group=group)
    parts = list(recv.split(out_sizes))
    return torch.cat([parts[s].reshape(f_counts[rank], k_counts[s], n) for s in range(world)], dim=1).contiguous()


def regroup_to_vectors(block_f, k_counts, f_counts, group=None):
    """[n_omega_r][k][n] -> [n_omega][k_r][n]: the inverse of regroup_to_frequencies."""
    import torch
    import torch.distributed as dist
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    n = block_f.shape[2]
    koff = _offsets(k_counts)
    send = torch.cat([block_f[:, koff[s]:koff[s + 1]].reshape(-1) for s in range(world)]).contiguous()
    in_sizes = [f_counts[rank] * k_counts[s] * n for s in range(world)]
    out_sizes = [f_counts[s] * k_counts[rank] * n for s in range(world)]
    recv = torch.empty(sum(out_sizes), dtype=block_f.dtype, device=block_f.device)
    dist.all_to_all_single(recv, send, out_sizes, in_sizes, group=group)
    parts = list(recv.split(out_sizes))
    return torch.cat([parts[s].reshape(f_counts[s], k_counts[rank], n) for s in range(world)], dim=0).contiguous()


def distributed_rsvd(march, orthonormalize, omega_local, k_counts, f_counts, n_power_iter, n_modes, group=None):
    """Block randomized SVD with the vectors split across ranks.

    Y = R Omega; q times {Q = qr(Y); Z = R^H Q; Q = qr(Z); Y = R Q}; Q = qr(Y); W = R^H Q; and per
    frequency the singular values of W (= those of its triangular factor R_W, W = Q_W R_W), which
    are the gains (B = Q^H R = W^H).  Each qr regroups by frequency and back.  Returns this rank's
    gains [n_inst][n_omega_r][n_modes] (descending) for its frequency chunk.
    """
    def qr(block):
        q_f, _ = orthonormalize(regroup_to_frequencies(block, k_counts, f_counts, group))
        return regroup_to_vectors(q_f, k_counts, f_counts, group)

    y = march(omega_local, False)
    for _ in range(n_power_iter):
        q = qr(y)
        z = march(q, True)
        q = qr(z)
        y = march(q, False)
    q = qr(y)
    w = march(q, True)
    _, r = orthonormalize(regroup_to_frequencies(w, k_counts, f_counts, group))
    r = r.cpu().numpy() if hasattr(r, "cpu") else np.asarray(r)
    gains = np.zeros((r.shape[1], r.shape[0], n_modes))
    for j in range(r.shape[0]):
        for i in range(r.shape[1]):
            gains[i, j] = np.linalg.svd(r[j, i], compute_uv=False)[:n_modes]
    return gains


def library_callables(op_all, op_chunk, opts):
    """march / orthonormalize callables backed by librsv for distributed_rsvd.

    op_all: operator with every frequency (marches this rank's k_r vectors); op_chunk: operator of
    the same system with this rank's frequencies (set with the full grid's spacing dw), used for the
    per-frequency orthonormalisation of [n_omega_r][k][n] blocks.
    """
    import torch
    from . import rsv

    def march(block, adjoint):
        out = torch.empty_like(block)
        (rsv.rsv_march_adjoint if adjoint else rsv.rsv_march_direct)(op_all, block, block.shape[1], out, **opts)
        return out

    def orthonormalize(block_f):
        q = block_f.clone()
        nw, k = q.shape[0], q.shape[1]
        _, ni, _ = rsv.rsv_operator_info(op_chunk)
        r = np.zeros((nw, ni, k, k), dtype=np.complex128)
        rsv.rsv_orthonormalize(op_chunk, q, k, r)
        return q, torch.from_numpy(r)

    return march, orthonormalize
