"""Explicit system matrices A of the workloads (oracle).

Each builder writes the discretised operator of Sec. 2.1 Eq. (system) (here in
the form du/dt = A u + f) as a scipy sparse matrix, straight from the
difference formulas, one stencil entry at a time.  The adjoint system of
Sec. 2.1 Eq. (adsystem) with identity metrics uses A^H (discrete adjoints with W = I).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sps
from scipy.special import erf


def gl1d(sysm) -> sps.csr_matrix:
    """Linearised GL (Sec. 3 Eq. (GL_timeDomain) family): -nu u_x + gamma u_xx + mu(x) u.

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
            mu = mu0 + sysm.mu_shift + sysm.mu2 * x * x
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


def adr2d(sysm) -> sps.csr_matrix:
    """2-D ADR: -U(y) u_x + visc lap(u) + (r(y) - sigma) u, index p = iy * nx + ix."""
    dx, dy, u, react, sigma = adr2d_fields(sysm)
    nx, ny, nu = sysm.nx, sysm.ny, sysm.visc
    rows, cols, vals = [], [], []
    for j in range(ny):
        for i in range(nx):
            p = j * nx + i
            rows.append(p); cols.append(p)
            vals.append(-2.0 * nu / dx ** 2 - 2.0 * nu / dy ** 2 + react[j] - sigma[j, i])
            if i > 0:
                rows.append(p); cols.append(p - 1); vals.append(u[j] / (2 * dx) + nu / dx ** 2)
            if i < nx - 1:
                rows.append(p); cols.append(p + 1); vals.append(-u[j] / (2 * dx) + nu / dx ** 2)
            if j > 0:
                rows.append(p); cols.append(p - nx); vals.append(nu / dy ** 2)
            if j < ny - 1:
                rows.append(p); cols.append(p + nx); vals.append(nu / dy ** 2)
    return sps.csr_matrix((np.array(vals), (rows, cols)), shape=(nx * ny, nx * ny))


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

    Index p = ((c * nz + kz) * ny + jy) * nx + ix.
    """
    (dx, dy, dz), ux, dudx, dudy, dudz = adv3d_fields(sysm)
    nx, ny, nz, nu = sysm.nx, sysm.ny, sysm.nz, sysm.visc
    ncell = nx * ny * nz
    rows, cols, vals = [], [], []
    grads = (dudx, dudy, dudz)
    for c in range(3):
        for kz in range(nz):
            for jy in range(ny):
                for ix in range(nx):
                    cell = (kz * ny + jy) * nx + ix
                    p = c * ncell + cell
                    u = ux[kz, jy, ix]
                    diag = -2.0 * nu * (1 / dx ** 2 + 1 / dy ** 2 + 1 / dz ** 2)
                    rows.append(p); cols.append(p); vals.append(diag)
                    if ix > 0:
                        rows.append(p); cols.append(p - 1); vals.append(u / (2 * dx) + nu / dx ** 2)
                    if ix < nx - 1:
                        rows.append(p); cols.append(p + 1); vals.append(-u / (2 * dx) + nu / dx ** 2)
                    if jy > 0:
                        rows.append(p); cols.append(p - nx); vals.append(nu / dy ** 2)
                    if jy < ny - 1:
                        rows.append(p); cols.append(p + nx); vals.append(nu / dy ** 2)
                    if kz > 0:
                        rows.append(p); cols.append(p - nx * ny); vals.append(nu / dz ** 2)
                    if kz < nz - 1:
                        rows.append(p); cols.append(p + nx * ny); vals.append(nu / dz ** 2)
                    if c == 0:
                        for cc in range(3):
                            rows.append(p); cols.append(cc * ncell + cell)
                            vals.append(-grads[cc][kz, jy, ix])
    return sps.csr_matrix((np.array(vals), (rows, cols)), shape=(3 * ncell, 3 * ncell))


def dense(a) -> np.ndarray:
    """A caller-supplied dense operator is used as given."""
    return np.asarray(a, dtype=np.complex128)
