"""Seeded synthetic workloads shared by the oracle and the CUDA path.

This module holds the *inputs* of the resolvent computation and nothing of
the method itself: physical parameters of the five benchmark systems, their
frequency lists, the seeded Gaussian test-vector blocks that the randomized
SVD starts from, and the dense spectral Ginzburg-Landau matrix that the
dense-operator workload hands to both sides as a given system matrix A
(the paper treats the discretised operator as given, Sec. 2.1, Eq. (system)).

No time marching, synthesis, Fourier analysis, QR or SVD lives here.

Sign convention (both sides): du/dt = A u + f(t), forcing synthesised as
f(t) = sum_j fhat_j exp(+i w_j t), resolvent R(w) = (i w I - A)^{-1}.  The
paper writes du/dt + A_p u = B f with signals exp(-i w t) (Sec. 2.1,
Eqs. (system), (systemFreqDomain), (fourier)); A = -A_p and the paper's gain at w is the gain here at -w.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2008109040


# ---------------------------------------------------------------------------
# System definitions
# ---------------------------------------------------------------------------
@dataclass(frozen=True)
class GL1D:
    """Linearised complex Ginzburg-Landau, du/dt = -nu u_x + gamma u_xx + mu(x) u.

    mu(x) = mu0 + mu_shift + mu1 * x + mu2 * x**2 on x in (x0, x1), n interior points
    per instance, homogeneous Dirichlet ends, 2nd-order central differences
    (Sec. 3, Eq. (GL_timeDomain) gives the model family).  A batch of instances with
    their own n and mu0 forms one block-diagonal operator.
    """
    n: tuple = (256,)
    mu0: tuple = (0.23,)
    x0: float = -85.0
    x1: float = 85.0
    nu: complex = 2.0 + 0.4j
    gamma: complex = 1.0 - 1.0j
    mu_shift: float = -0.04
    mu2: float = -0.005
    mu1: float = 0.0

    @property
    def n_total(self) -> int:
        return int(sum(self.n))


@dataclass(frozen=True)
class Dense:
    """Caller-supplied dense complex operator A (n x n)."""
    n: int = 1024
    x_half_width: float = 110.0
    nu: complex = 2.0 + 0.4j
    gamma: complex = 1.0 - 1.0j
    mu_c: float = 0.19
    mu2: float = -0.005

    @property
    def n_total(self) -> int:
        return self.n


@dataclass(frozen=True)
class ADR2D:
    """2-D scalar linearised advection-diffusion-reaction on a jet base flow.

    du/dt = -U(y) u_x + visc (u_xx + u_yy) + r(y) u - sigma(x, y) u,
    U(y) = 0.5 (1 + tanh((0.5 - |y|) / jet_delta)), r = -kappa dU/dy,
    sigma a quadratic sponge over `sponge_cells` cells next to every wall.
    Interior grid nx x ny on x in (0, lx), y in (-ly/2, ly/2), Dirichlet.
    Real state, 5-point central stencil.
    """
    nx: int = 1024
    ny: int = 512
    lx: float = 40.0
    ly: float = 10.0
    visc: float = 1e-3
    kappa: float = 0.01
    jet_delta: float = 0.05
    sponge_cells: int = 32
    sponge_amp: float = 1.0

    @property
    def n_total(self) -> int:
        return self.nx * self.ny


@dataclass(frozen=True)
class ADV3D:
    """3-D, 3-component linearised advection-diffusion (no pressure).

    du/dt = -(U.grad)u - (u.grad)U + visc lap(u), U = (erf(r / delta(x)), 0, 0),
    r = sqrt(y^2 + z^2), delta(x) = delta0 + (delta1 - delta0) x / lx.
    Interior grid nx x ny x nz on (0, lx) x (-ly/2, ly/2) x (-lz/2, lz/2),
    Dirichlet, 7-point central stencil; state ordered [component][z][y][x].
    """
    nx: int = 256
    ny: int = 128
    nz: int = 128
    lx: float = 20.0
    ly: float = 10.0
    lz: float = 10.0
    visc: float = 5e-4
    delta0: float = 0.2
    delta1: float = 1.0

    @property
    def n_total(self) -> int:
        return 3 * self.nx * self.ny * self.nz


@dataclass(frozen=True)
class Workload:
    name: str
    system: object
    omegas: np.ndarray = field(repr=False)
    dt: float
    k: int
    variant: str            # "ssrm" | "trm"
    n_transient_windows: int = 0
    tail_steps: int = 0
    n_power_iter: int = 1
    n_modes: int = 3
    real_state: bool = False
    seed: int = SEED_BASE

    @property
    def n(self) -> int:
        return self.system.n_total

    @property
    def n_omega(self) -> int:
        return len(self.omegas)


def _lin(a, b, m):
    return np.array([a + (b - a) * j / (m - 1) for j in range(m)], dtype=np.float64)


def gl_fd_c1() -> Workload:
    """Plain FP64 GL (N = 256, k = 4, 32 frequencies in [-1.5, 1.5], dt = 0.02, SSRM, q = 3)."""
    return Workload("gl_fd_n256_k4_w32_ssrm", GL1D(), _lin(-1.5, 1.5, 32), 0.02, 4, "ssrm",
                    n_transient_windows=4, n_power_iter=3, seed=SEED_BASE + 1)


def dense_hermite_c2() -> Workload:
    """Dense spectral GL (N = 1024, k = 32, 256 frequencies in [-2, 2], dt = 0.005, TRM)."""
    return Workload("dense_hermite_gl_n1024_k32_w256_trm", Dense(), _lin(-2.0, 2.0, 256), 0.005, 32,
                    "trm", tail_steps=40000, n_power_iter=1, seed=SEED_BASE + 2)


def adr2d_c3() -> Workload:
    """2-D jet ADR (1024 x 512, k = 16, 128 frequencies in [0, 4], SSRM)."""
    sysm = ADR2D()
    dx = sysm.lx / (sysm.nx + 1)
    return Workload("adr2d_1024x512_k16_w128_ssrm", sysm, _lin(0.0, 4.0, 128), 0.5 * dx, 16, "ssrm",
                    n_transient_windows=2, n_power_iter=1, real_state=True, seed=SEED_BASE + 3)


def adv3d_c4() -> Workload:
    """3-D boundary-layer advection-diffusion (256 x 128 x 128 x 3, k = 8, 64 frequencies, SSRM)."""
    sysm = ADV3D()
    dx = sysm.lx / (sysm.nx + 1)
    om = np.array([0.04 * math.pi * j for j in range(64)])
    return Workload("adv3d_256x128x128x3_k8_w64_ssrm", sysm, om, 0.5 * dx, 8, "ssrm",
                    n_transient_windows=3, n_power_iter=2, real_state=True, seed=SEED_BASE + 4)


def _gl_abscissa(n: int, mu0: float, sysm: GL1D) -> float:
    """Largest real part of the spectrum of one finite-difference GL instance (input validation)."""
    dx = (sysm.x1 - sysm.x0) / (n + 1)
    x = sysm.x0 + (np.arange(n) + 1) * dx
    a = np.diag(-2.0 * sysm.gamma / dx ** 2 + mu0 + sysm.mu_shift + sysm.mu2 * x * x)
    a += np.diag(np.full(n - 1, sysm.nu / (2 * dx) + sysm.gamma / dx ** 2), -1)
    a += np.diag(np.full(n - 1, -sysm.nu / (2 * dx) + sysm.gamma / dx ** 2), 1)
    return float(np.linalg.eigvals(a).real.max())


def gl_batch_c5(seed: int = SEED_BASE + 5) -> Workload:
    """64 GL instances, N log-uniform in [128, 2048], mu0 uniform in [0.1, 0.3], k = 8, 64 frequencies.

    Instances whose discrete spectral abscissa is >= -0.02 (coarse grids with
    strong growth; only N <= 400 is at risk) get a new mu0 from the same
    stream until they decay fast enough for two transient windows.
    """
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(math.log(128), math.log(2048), size=64)).round().astype(int)
    mu0 = rng.uniform(0.1, 0.3, size=64)
    proto = GL1D()
    for i in range(64):
        while n[i] <= 400 and _gl_abscissa(int(n[i]), float(mu0[i]), proto) >= -0.02:
            mu0[i] = rng.uniform(0.1, 0.3)
    sysm = GL1D(n=tuple(int(v) for v in n), mu0=tuple(float(v) for v in mu0))
    return Workload("gl_batch64_k8_w64_ssrm", sysm, _lin(-1.5, 1.5, 64), 0.003, 8, "ssrm",
                    n_transient_windows=2, n_power_iter=4, seed=seed)


def gl_paper(n: int = 400, beta: float = 0.1, n_omega: int = 61, dt: float = 0.01) -> Workload:
    """The paper's Ginzburg-Landau validation case (Sec. 3): advection speed U = 6, gamma = 1 (real),
    mu(x) = beta mu_c (1 - x/20) with mu_c = U^2 Re(gamma) / |gamma|^2 = 36, x in (0, 40), Dirichlet,
    Crank-Nicolson with dt = 0.01, frequencies up to 15.  The paper's operator A_p = U d/dx - mu - gamma
    d^2/dx^2 is -A here.  The paper gives no grid size: n = 400 interior points (dx = 40/401); the
    frequency grid is 0, 0.25, ..., 15 for the steady-state method."""
    mu_c = 36.0
    sysm = GL1D(n=(n,), mu0=(beta * mu_c,), x0=0.0, x1=40.0, nu=6.0 + 0.0j, gamma=1.0 + 0.0j, mu_shift=0.0,
                mu2=0.0, mu1=-beta * mu_c / 20.0)
    return Workload(f"gl_paper_n{n}_cn", sysm, _lin(0.0, 15.0, n_omega), dt, 4, "ssrm", n_transient_windows=2,
                    n_power_iter=2, seed=SEED_BASE + 7)


def small_gl(n: int = 24, n_omega: int = 8, k: int = 2, dt: float = 0.05, x_half: float = 20.0,
             mu0: float = 0.1, variant: str = "ssrm", n_trans: int = 6, tail_steps: int = 0,
             q: int = 1, seed: int = SEED_BASE + 100, omega_max: float = 1.0) -> Workload:
    """Small GL case the oracle finishes in well under a second."""
    sysm = GL1D(n=(n,), mu0=(mu0,), x0=-x_half, x1=x_half)
    return Workload(f"gl_fd_n{n}_small", sysm, _lin(-omega_max, omega_max, n_omega), dt, k, variant,
                    n_transient_windows=n_trans, tail_steps=tail_steps, n_power_iter=q, seed=seed)


# ---------------------------------------------------------------------------
# Seeded inputs
# ---------------------------------------------------------------------------
def gaussian_block(seed: int, n_omega: int, k: int, n: int, real_rows=()) -> np.ndarray:
    """Test-vector block [n_omega][k][n], complex128, entries (N(0,1) + i N(0,1))/sqrt(2).

    Rows listed in `real_rows` (frequency indices) are drawn real N(0,1): a
    real-state system forced at w = 0 responds to the real part only.
    """
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((n_omega, k, n))
    im = rng.standard_normal((n_omega, k, n))
    out = (re + 1j * im) / math.sqrt(2.0)
    for j in real_rows:
        out[j] = re[j]
    return out


def test_block(w: Workload, k: int | None = None, seed_offset: int = 0) -> np.ndarray:
    kk = w.k if k is None else k
    real_rows = [j for j, om in enumerate(w.omegas) if w.real_state and om == 0.0]
    return gaussian_block(w.seed + seed_offset, w.n_omega, kk, w.n, real_rows)


def test_block_row(w: Workload, j: int, k: int | None = None, seed_offset: int = 0) -> np.ndarray:
    """Row j ([k][n], complex64) of a test block drawn one frequency at a time.

    For blocks too large to draw at once on the host (tens of GB): each row has
    its own stream, numpy.random.default_rng((seed, j)); same distribution as
    `gaussian_block` (not the same numbers).
    """
    kk = w.k if k is None else k
    rng = np.random.default_rng((w.seed + seed_offset, j))
    re = rng.standard_normal((kk, w.n), dtype=np.float32)
    if w.real_state and w.omegas[j] == 0.0:
        return re.astype(np.complex64)
    im = rng.standard_normal((kk, w.n), dtype=np.float32)
    return ((re + 1j * im) / np.float32(math.sqrt(2.0))).astype(np.complex64)


def hermite_gl_matrix(sysm: Dense) -> np.ndarray:
    """Dense GL operator on Hermite-function collocation nodes (input data).

    Nodes: roots of the degree-n Hermite polynomial, scaled so the outermost
    node sits at +-x_half_width.  D1 differentiates the weighted interpolant
    exp(-x^2/2) * (polynomial of degree < n) exactly; its entries come from
    the barycentric formula evaluated in the log domain to avoid overflow.
    A = -nu D1 + gamma D1 @ D1 + diag(mu_c + mu2 x^2).  Returns complex128
    [n][n] row-major.
    """
    import scipy.special as sp

    nn = sysm.n
    x, _ = sp.roots_hermite(nn)
    x = np.sort(x)
    b = sysm.x_half_width / x[-1]
    diff = x[:, None] - x[None, :]
    np.fill_diagonal(diff, 1.0)
    logabs = np.log(np.abs(diff))
    np.fill_diagonal(logabs, 0.0)
    logw = -logabs.sum(axis=1)
    sgnw = (-1.0) ** (nn - 1 - np.arange(nn))
    loga = -x ** 2 / 2
    expo = (loga[:, None] - loga[None, :]) + (logw[None, :] - logw[:, None]) - logabs
    d1 = np.exp(expo) * (sgnw[None, :] / sgnw[:, None]) * np.sign(diff)
    inv = 1.0 / diff
    np.fill_diagonal(inv, 0.0)
    np.fill_diagonal(d1, -x + inv.sum(axis=1))
    d1 = d1 / b
    xi = x * b
    a = -sysm.nu * d1 + sysm.gamma * (d1 @ d1) + np.diag(sysm.mu_c + sysm.mu2 * xi ** 2)
    return np.ascontiguousarray(a.astype(np.complex128))


def hermite_nodes(sysm: Dense) -> np.ndarray:
    import scipy.special as sp
    x = np.sort(sp.roots_hermite(sysm.n)[0])
    return x * (sysm.x_half_width / x[-1])


ALL = {"c1": gl_fd_c1, "c2": dense_hermite_c2, "c3": adr2d_c3, "c4": adv3d_c4, "c5": gl_batch_c5}
