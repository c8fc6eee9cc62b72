"""Explicit system matrices A of the workloads (oracle).

Each builder writes the discretised operator of Sec. 2.1 Eq. (system) (here in
the form du/dt = A u + f) as a scipy sparse matrix, straight from the
difference formulas: one array of entries per stencil direction.  The adjoint system of
Sec. 2.1 Eq. (adsystem) with identity metrics uses A^H (discrete adjoints with W = I).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sps
from scipy.special import erf


def gl1d(sysm) -> sps.csr_matrix:
    """Linearised GL (Sec. 3 Eq. (GL_timeDomain) family): -nu u_x + gamma u_xx + mu(x) u,
    mu(x) = mu0 + mu_shift + mu1 x + mu2 x^2.

    Central differences u_x ~ (u[i+1] - u[i-1]) / (2 dx),
    u_xx ~ (u[i+1] - 2 u[i] + u[i-1]) / dx^2, Dirichlet zero outside the
    n interior points; instances of a batch form a block-diagonal matrix.
    """
    blocks = []
    for n, mu0 in zip(sysm.n, sysm.mu0):
        dx = (sysm.x1 - sysm.x0) / (n + 1)
        rows, cols, vals = [], [], []
        for i in range(n):
            x = sysm.x0 + (i + 1) * dx
            mu = mu0 + sysm.mu_shift + getattr(sysm, "mu1", 0.0) * x + sysm.mu2 * x * x
            rows.append(i); cols.append(i); vals.append(-2.0 * sysm.gamma / dx ** 2 + mu)
            if i > 0:
                rows.append(i); cols.append(i - 1)
                vals.append(sysm.nu / (2.0 * dx) + sysm.gamma / dx ** 2)
            if i < n - 1:
                rows.append(i); cols.append(i + 1)
                vals.append(-sysm.nu / (2.0 * dx) + sysm.gamma / dx ** 2)
        blocks.append(sps.csr_matrix((np.array(vals, dtype=np.complex128), (rows, cols)), shape=(n, n)))
    return sps.block_diag(blocks, format="csr")


def adr2d_fields(sysm):
    """Base-flow fields of the 2-D jet: U(y), r(y) = -kappa dU/dy, sponge sigma(x, y)."""
    dx = sysm.lx / (sysm.nx + 1)
    dy = sysm.ly / (sysm.ny + 1)
    y = -0.5 * sysm.ly + (np.arange(sysm.ny) + 1) * dy
    arg = (0.5 - np.abs(y)) / sysm.jet_delta
    u = 0.5 * (1.0 + np.tanh(arg))
    dudy = 0.5 / np.cosh(arg) ** 2 * (-np.sign(y) / sysm.jet_delta)
    react = -sysm.kappa * dudy
    ix = np.arange(sysm.nx)
    iy = np.arange(sysm.ny)
    dxw = np.minimum(ix, sysm.nx - 1 - ix)
    dyw = np.minimum(iy, sysm.ny - 1 - iy)
    d = np.minimum(dyw[:, None], dxw[None, :])
    s = float(sysm.sponge_cells)
    sigma = np.where(d < s, sysm.sponge_amp * ((s - d) / s) ** 2, 0.0)
    return dx, dy, u, react, sigma


def _couple(rows, cols, vals, p, q, v, mask):
    rows.append(p[mask]); cols.append(q[mask]); vals.append(np.broadcast_to(v, p.shape)[mask])


def adr2d(sysm) -> sps.csr_matrix:
    """2-D ADR: -U(y) u_x + visc lap(u) + (r(y) - sigma) u, index p = iy * nx + ix.

    Entries (central differences, Dirichlet zeros outside the grid):
      diagonal  -2 visc/dx^2 - 2 visc/dy^2 + r(y) - sigma(x, y)
      (ix -/+ 1)  +/- U(y)/(2 dx) + visc/dx^2,   (iy -/+ 1)  visc/dy^2.
    """
    dx, dy, u, react, sigma = adr2d_fields(sysm)
    nx, ny, nu = sysm.nx, sysm.ny, sysm.visc
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    p = (jj * nx + ii).ravel()
    jf, i_f = jj.ravel(), ii.ravel()
    uy = u[jf]
    rows, cols, vals = [], [], []
    _couple(rows, cols, vals, p, p, -2.0 * nu / dx ** 2 - 2.0 * nu / dy ** 2 + react[jf] - sigma.ravel(),
            np.ones_like(p, bool))
    _couple(rows, cols, vals, p, p - 1, uy / (2 * dx) + nu / dx ** 2, i_f > 0)
    _couple(rows, cols, vals, p, p + 1, -uy / (2 * dx) + nu / dx ** 2, i_f < nx - 1)
    _couple(rows, cols, vals, p, p - nx, nu / dy ** 2, jf > 0)
    _couple(rows, cols, vals, p, p + nx, nu / dy ** 2, jf < ny - 1)
    return sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(nx * ny, nx * ny))


def adv3d_fields(sysm):
    """Base flow U_x = erf(r / delta(x)) and its exact gradient on the grid [z][y][x]."""
    dx = sysm.lx / (sysm.nx + 1)
    dy = sysm.ly / (sysm.ny + 1)
    dz = sysm.lz / (sysm.nz + 1)
    x = (np.arange(sysm.nx) + 1) * dx
    y = -0.5 * sysm.ly + (np.arange(sysm.ny) + 1) * dy
    z = -0.5 * sysm.lz + (np.arange(sysm.nz) + 1) * dz
    zz, yy, xx = np.meshgrid(z, y, x, indexing="ij")
    delta = sysm.delta0 + (sysm.delta1 - sysm.delta0) * xx / sysm.lx
    ddelta = (sysm.delta1 - sysm.delta0) / sysm.lx
    r = np.sqrt(yy ** 2 + zz ** 2)
    ux = erf(r / delta)
    g = 2.0 / math.sqrt(math.pi) * np.exp(-(r / delta) ** 2)
    dudx = g * (-r * ddelta / delta ** 2)
    rs = np.where(r > 0, r, 1.0)
    dudy = np.where(r > 0, g * (yy / (rs * delta)), 0.0)   # the cone tip r = 0 takes 0
    dudz = np.where(r > 0, g * (zz / (rs * delta)), 0.0)
    return (dx, dy, dz), ux, dudx, dudy, dudz


def adv3d(sysm) -> sps.csr_matrix:
    """3-D, 3 components: -(U.grad)u_c + visc lap(u_c) - delta_{c,x} (u.grad)U_x.

    Index p = ((c * nz + kz) * ny + jy) * nx + ix.  Entries per component c:
      diagonal  -2 visc (1/dx^2 + 1/dy^2 + 1/dz^2),
      (ix -/+ 1)  +/- U(x,y,z)/(2 dx) + visc/dx^2,  (jy -/+ 1) visc/dy^2,  (kz -/+ 1) visc/dz^2;
    component x also couples to every component cc at the same cell with -dU_x/dx_cc.
    """
    (dx, dy, dz), ux, dudx, dudy, dudz = adv3d_fields(sysm)
    nx, ny, nz, nu = sysm.nx, sysm.ny, sysm.nz, sysm.visc
    ncell = nx * ny * nz
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cell = ((kk * ny + jj) * nx + ii).ravel()
    i_f, j_f, k_f = ii.ravel(), jj.ravel(), kk.ravel()
    u = ux.ravel()
    grads = (dudx.ravel(), dudy.ravel(), dudz.ravel())
    diag = -2.0 * nu * (1 / dx ** 2 + 1 / dy ** 2 + 1 / dz ** 2)
    rows, cols, vals = [], [], []
    allm = np.ones_like(cell, bool)
    for c in range(3):
        p = c * ncell + cell
        _couple(rows, cols, vals, p, p, np.full(p.shape, diag), allm)
        _couple(rows, cols, vals, p, p - 1, u / (2 * dx) + nu / dx ** 2, i_f > 0)
        _couple(rows, cols, vals, p, p + 1, -u / (2 * dx) + nu / dx ** 2, i_f < nx - 1)
        _couple(rows, cols, vals, p, p - nx, np.full(p.shape, nu / dy ** 2), j_f > 0)
        _couple(rows, cols, vals, p, p + nx, np.full(p.shape, nu / dy ** 2), j_f < ny - 1)
        _couple(rows, cols, vals, p, p - nx * ny, np.full(p.shape, nu / dz ** 2), k_f > 0)
        _couple(rows, cols, vals, p, p + nx * ny, np.full(p.shape, nu / dz ** 2), k_f < nz - 1)
    for cc in range(3):
        _couple(rows, cols, vals, cell, cc * ncell + cell, -grads[cc], allm)
    return sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(3 * ncell, 3 * ncell))


def dense(a) -> np.ndarray:
    """A caller-supplied dense operator is used as given."""
    return np.asarray(a, dtype=np.complex128)
