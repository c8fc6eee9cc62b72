"""Pins of the oracle's system matrices against analytic derivatives.

Each discretised operator is applied to smooth fields that vanish on the
boundary; the result must approach the continuous operator of the workload
with the 2nd-order error of central differences (halving the spacing cuts
the error about 4x).  The dense Hermite operator must differentiate
Hermite functions exactly.
"""
import math

import numpy as np
from scipy.special import erf

import workloads as W
from oracle import operators


def test_gl1d_second_order():
    errs = []
    for n in (199, 399):
        sysm = W.GL1D(n=(n,), mu0=(0.23,), x0=-10.0, x1=10.0)
        a = operators.gl1d(sysm)
        dx = 20.0 / (n + 1)
        x = -10.0 + (np.arange(n) + 1) * dx
        u = np.exp(-x ** 2) * (1 + 0.5j * x)
        ux = np.exp(-x ** 2) * (-2 * x * (1 + 0.5j * x) + 0.5j)
        uxx = np.exp(-x ** 2) * ((4 * x ** 2 - 2) * (1 + 0.5j * x) - 2 * x * 0.5j * 2)
        mu = 0.23 - 0.04 - 0.005 * x ** 2
        exact = -sysm.nu * ux + sysm.gamma * uxx + mu * u
        errs.append(np.abs(a @ u - exact).max())
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_gl1d_batch_is_block_diagonal():
    sysm = W.GL1D(n=(5, 7), mu0=(0.1, 0.3))
    a = operators.gl1d(sysm).toarray()
    assert a.shape == (12, 12)
    assert np.all(a[:5, 5:] == 0) and np.all(a[5:, :5] == 0)


def test_adr2d_second_order():
    errs = []
    for nx, ny in ((63, 31), (127, 63)):
        sysm = W.ADR2D(nx=nx, ny=ny, lx=4.0, ly=2.0, jet_delta=0.3, sponge_cells=4)
        a = operators.adr2d(sysm)
        dx, dy, uy, react, sigma = operators.adr2d_fields(sysm)
        x = (np.arange(nx) + 1) * dx
        y = -1.0 + (np.arange(ny) + 1) * dy
        yy, xx = np.meshgrid(y, x, indexing="ij")
        f = np.sin(math.pi * xx / 4.0) * np.cos(math.pi * yy / 2.0)
        fx = math.pi / 4.0 * np.cos(math.pi * xx / 4.0) * np.cos(math.pi * yy / 2.0)
        lap = -((math.pi / 4.0) ** 2 + (math.pi / 2.0) ** 2) * f
        exact = -uy[:, None] * fx + sysm.visc * lap + (react[:, None] - sigma) * f
        errs.append(np.abs(a @ f.ravel() - exact.ravel()).max())
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_adr2d_fields():
    sysm = W.ADR2D(nx=64, ny=64, lx=4.0, ly=10.0, sponge_cells=8)
    dx, dy, u, react, sigma = operators.adr2d_fields(sysm)
    assert np.all((u >= 0) & (u <= 1)) and u.max() > 0.99
    assert sigma[0, 30] == 1.0 and sigma[20, 20] == 0.0
    # r = -kappa dU/dy against a centered difference of U
    y = -5.0 + (np.arange(64) + 1) * dy
    fd = (0.5 * (1 + np.tanh((0.5 - np.abs(y + 1e-6)) / 0.05)) -
          0.5 * (1 + np.tanh((0.5 - np.abs(y - 1e-6)) / 0.05))) / 2e-6
    assert np.allclose(react, -sysm.kappa * fd, atol=1e-5)


def test_adv3d_second_order_and_coupling():
    errs = []
    for n in (16, 32):
        sysm = W.ADV3D(nx=n, ny=n, nz=n, lx=2.0, ly=2.0, lz=2.0, delta0=0.5, delta1=1.0, visc=0.01)
        a = operators.adv3d(sysm)
        (dx, dy, dz), ux, dudx, dudy, dudz = operators.adv3d_fields(sysm)
        c = (np.arange(n) + 1) * dx
        yc = -1.0 + (np.arange(n) + 1) * dy
        zc = -1.0 + (np.arange(n) + 1) * dz
        zz, yy, xx = np.meshgrid(zc, yc, c, indexing="ij")
        s = np.sin(math.pi * xx / 2) * np.cos(math.pi * yy / 2) * np.cos(math.pi * zz / 2)
        sx = math.pi / 2 * np.cos(math.pi * xx / 2) * np.cos(math.pi * yy / 2) * np.cos(math.pi * zz / 2)
        lap = -3 * (math.pi / 2) ** 2 * s
        comps = [s, 2 * s, -s]
        u = np.concatenate([q.ravel() for q in comps])
        out = (a @ u).reshape(3, n, n, n)
        exact = []
        for ci, q in enumerate(comps):
            fac = (1, 2, -1)[ci]
            e = -ux * fac * sx + sysm.visc * fac * lap
            if ci == 0:
                e = e - (comps[0] * dudx + comps[1] * dudy + comps[2] * dudz)
            exact.append(e)
        errs.append(np.abs(out - np.array(exact)).max())
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_adv3d_base_flow_gradient():
    sysm = W.ADV3D(nx=8, ny=8, nz=8, lx=2.0, ly=2.0, lz=2.0)
    (dx, dy, dz), ux, dudx, dudy, dudz = operators.adv3d_fields(sysm)
    x, y, z, e = 0.3, 0.4, -0.2, 1e-6
    def f(x, y, z):
        d = sysm.delta0 + (sysm.delta1 - sysm.delta0) * x / sysm.lx
        return erf(math.hypot(y, z) / d)
    g = [(f(x + e, y, z) - f(x - e, y, z)) / (2 * e), (f(x, y + e, z) - f(x, y - e, z)) / (2 * e),
         (f(x, y, z + e) - f(x, y, z - e)) / (2 * e)]
    d = sysm.delta0 + (sysm.delta1 - sysm.delta0) * x / sysm.lx
    r = math.hypot(y, z)
    gg = 2 / math.sqrt(math.pi) * math.exp(-(r / d) ** 2)
    ana = [gg * (-r * (sysm.delta1 - sysm.delta0) / sysm.lx / d ** 2), gg * y / (r * d), gg * z / (r * d)]
    assert np.allclose(g, ana, rtol=1e-6)


def test_hermite_matrix_differentiates_hermite_functions():
    """The dense operator's D1 is exact on exp(-x^2/2) p(x), deg p < n."""
    sysm = W.Dense(n=48, x_half_width=10.0, nu=1.0, gamma=0.0, mu_c=0.0, mu2=0.0)
    a = W.hermite_gl_matrix(sysm)           # A = -D1 here
    xi = W.hermite_nodes(sysm)
    import scipy.special as sp
    b = sysm.x_half_width / np.sort(sp.roots_hermite(48)[0])[-1]
    x = xi / b
    p = x ** 5 - 3 * x ** 2 + 1
    dp = 5 * x ** 4 - 6 * x
    u = np.exp(-x ** 2 / 2) * p
    du = np.exp(-x ** 2 / 2) * (dp - x * p) / b
    assert np.abs(-a @ u - du).max() < 1e-9 * np.abs(du).max()


def test_hermite_workload_is_rk4_stable():
    """The dense workload (half-width 110, dt = 0.005) keeps every RK4 amplification below 1."""
    w = W.dense_hermite_c2()
    a = W.hermite_gl_matrix(w.system)
    ev = np.linalg.eigvals(a)
    z = w.dt * ev
    amp = np.abs(1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24)
    assert ev.real.max() < -0.1
    assert amp.max() < 1.0
