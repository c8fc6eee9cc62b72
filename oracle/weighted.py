"""Forcing and observation matrices and metrics: R_y = C R B with weighted adjoints (oracle).

Sec. 2.1 of the paper: the direct system du/dt = A u + B f, y = C u gives
yhat = C R B fhat = R_y fhat (Eq. (systemFreqDomain)); the adjoint system of
Eq. (adsystem) uses the adjoints in the metrics W_u, W_f, W_y,
    A^dag = W_u^{-1} A^H W_u,  B^dag = W_f^{-1} B^H W_u,  C^dag = W_y^{-1} C^H W_u,
and returns what = B^dag R^dag C^dag yhat = R_y^dag yhat (Eq. (adsystemFreqDomain)).
Written out, R_y^dag = W_f^{-1} B^H R^H C^H W_y: W_u cancels, and the gain
||yhat||_{W_y} / ||fhat||_{W_f} is maximised by the SVD of
W_y^{1/2} R_y W_f^{-1/2}.

Here B, C and the metrics are diagonal (real, non-negative B and C entries:
masks or weights in space; positive metric entries, e.g. quadrature
weights of a non-uniform mesh), given as vectors over the state.  The runs are
the march module's, with the diagonal factors applied to its input and
output blocks exactly as the formulas above compose them.
"""
from __future__ import annotations

import numpy as np

from . import march as _march
from . import rsvd as _rsvd


def march_direct(a, grid, fhat, b, c, **kw):
    """yhat = C R B fhat: the direct run (Sec. 2.1) forced by B fhat, observed through C."""
    return c[None, None, :] * _march.march(a, grid, b[None, None, :] * fhat, **kw)


def march_adjoint(a, grid, yhat, b, c, w_f, w_y, **kw):
    """what = R_y^dag yhat = W_f^{-1} B^H R^H C^H W_y yhat (Sec. 2.1, adjoint run)."""
    z = _march.march(a, grid, (c * w_y)[None, None, :] * yhat, adjoint=True, **kw)
    return (b / w_f)[None, None, :] * z


def weighted_rsvd(a, grid, omega_block, b, c, w_f, w_y, n_power_iter, n_modes, real_rows=(), **kw):
    """Gains and modes of R_y in the W_f (forcing) and W_y (response) norms.

    Randomized SVD of Rt = W_y^{1/2} C R B W_f^{-1/2} (block_rsvd of the rsvd module with the two
    runs scaled accordingly); forcing modes W_f^{-1/2} vt and response modes W_y^{-1/2} ut are
    unit vectors in their metrics.  Returns (gains, forcing modes, response modes) as block_rsvd.
    """
    sf = b / np.sqrt(w_f)                # B W_f^{-1/2}
    sy = c * np.sqrt(w_y)                # W_y^{1/2} C
    md = lambda blk: sy[None, None, :] * _march.march(a, grid, sf[None, None, :] * blk, **kw)
    ma = lambda blk: sf[None, None, :] * _march.march(a, grid, sy[None, None, :] * blk, adjoint=True, **kw)
    gains, vt, ut = _rsvd.block_rsvd(md, ma, omega_block, n_power_iter, n_modes, real_rows=real_rows)
    v = [[vm / np.sqrt(w_f)[None, :] for vm in vt[0]]]
    u = [[um / np.sqrt(w_y)[None, :] for um in ut[0]]]
    return gains, v, u
