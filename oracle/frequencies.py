"""Commensurate frequency grid and the analysis window (oracle).

Sec. 2.3: the periodic forcing has period T and resolves the frequencies
w_k = 2 pi k / T, i.e. Delta omega = 2 pi / T.  Here every frequency must be
w_j = (m_j + phi) * dw with integer m_j and a common offset phi in {0, 1/2};
phi = 1/2 gives an anti-periodic forcing whose DFT over any window of length
T is still exact.  The window holds N_T = ceil(T / dt) steps and the step is
shrunk to h = T / N_T so the window is an integer number of steps.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Grid:
    omegas: np.ndarray
    dw: float
    phi: float          # 0 or 0.5
    m: np.ndarray       # integers, omegas = (m + phi) * dw
    period: float       # T = 2 pi / dw
    n_t: int            # steps per window
    h: float            # step, period / n_t


def make_grid(omegas, dt: float, dw: float | None = None) -> Grid:
    om = np.asarray(omegas, dtype=np.float64)
    if dw is None:
        if om.size < 2:
            raise ValueError("a single frequency needs an explicit dw")
        dw = float(np.min(np.diff(np.sort(om))))
    ratio = om / dw
    base = ratio - np.floor(ratio)
    phi = 0.5 if abs(base[0] - 0.5) < 1e-6 else 0.0
    m = np.rint(ratio - phi).astype(np.int64)
    if np.max(np.abs(ratio - phi - m)) > 1e-6:
        raise ValueError("frequencies are not on a common grid (m + phi) * dw")
    period = 2.0 * math.pi / dw
    n_t = int(math.ceil(period / dt - 1e-9))
    return Grid(om, dw, phi, m, period, n_t, period / n_t)
