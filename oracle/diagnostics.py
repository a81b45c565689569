"""Flow statistics of Sec. 4.3 for the oracle: the viscous dissipation rate and the energy
spectrum of a DG velocity field.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain FP64 NumPy.

* dissipation rate eps = (1 / |Omega|) int nu grad v : grad v dOmega (the paper writes
  nu / (8 pi^3) for its box [-pi, pi]^3 and constant nu).  Reading: the gradient is the
  element-local (broken) gradient of the DG field, integrated by the GLL quadrature of the
  velocity nodes.
* energy spectrum E(k), k = 0, 1, 2, ...: the velocity interpolated to a regular grid of
  M points per direction (x_j = lo + j L / M, each point evaluated by the interpolant of the
  element containing it, the right end of an element belonging to its right neighbour), its
  discrete Fourier coefficients v^(n) = M^-d sum_j v(x_j) exp(-2 pi i n . j / M), and
  E(k) = |Omega| / 2 sum over the integer wave vectors n with k - 1/2 <= |n| < k + 1/2 of
  sum_c |v^_c(n)|^2, so that sum_k E(k) = |Omega| / 2 mean_j |v(x_j)|^2 ~ 1/2 int |v|^2.
  The signed index of n along a direction is j for j < M / 2 and j - M otherwise.
"""
import numpy as np

from . import dg, gll


def dissipation(mesh, v, nu):
    """eps of the velocity v ([d][ne * N^d]) with nodal (or constant) viscosity nu: the
    dissipation rate of Sec. 4.3 (broken gradient, GLL quadrature)."""
    d, N = mesh.d, mesh.P + 1
    D = gll.lagrange_eval(gll.gll_nodes_weights(N)[0], gll.gll_nodes_weights(N)[0], deriv=1)
    I = np.eye(N)
    W = dg.volume_weights(mesh, N)                  # (ne, N^d) quadrature weights
    nu = np.broadcast_to(np.asarray(nu, dtype=np.float64), (mesh.ne * N ** d,)).reshape(mesh.ne, -1)
    v = np.asarray(v).reshape(d, mesh.ne, -1)
    total = 0.0
    for k in range(d):
        Dk = dg.kron_dims([(2.0 / mesh.h[k]) * D if j == k else I for j in range(d)])
        for c in range(d):
            g = v[c] @ Dk.T                         # element-local derivative at the nodes
            total += np.sum(W * nu * g * g)
    vol = np.prod([mesh.hi[k] - mesh.lo[k] for k in range(d)])
    return total / vol


def regular_grid(mesh, v, M):
    """v interpolated to the M^d regular grid, shape (d, M, ..., M) with x the last axis (the
    grid of the energy spectrum of Sec. 4.3)."""
    d, N = mesh.d, mesh.P + 1
    xg, _ = gll.gll_nodes_weights(N)
    v = np.asarray(v).reshape(d, mesh.ne, *([N] * d))      # [c][e][z][y][x] (x fastest)
    # per direction: element index and interpolation row of every grid coordinate
    elem, rows = [], []
    for k in range(d):
        L = mesh.hi[k] - mesh.lo[k]
        xs = mesh.lo[k] + np.arange(M) * L / M
        ek = np.minimum(((xs - mesh.lo[k]) / mesh.h[k]).astype(int), mesh.n[k] - 1)
        xi = 2.0 * (xs - (mesh.lo[k] + ek * mesh.h[k])) / mesh.h[k] - 1.0
        elem.append(ek)
        rows.append(gll.lagrange_eval(xg, xi))
    out = np.zeros((d,) + (M,) * d)
    for idx in np.ndindex(*((M,) * d)):                    # idx = (iz, iy, ix) / (iy, ix)
        kk = idx[::-1]                                     # kk[0] = x index
        ec = [elem[k][kk[k]] for k in range(d)]
        e = mesh.eindex(ec)
        tile = v[:, e]
        for k in range(d):                                 # contract x first (last axis)
            tile = tile @ rows[k][kk[k]]
        out[(slice(None),) + idx] = tile
    return out


def energy_spectrum(mesh, v, M, kmax):
    """E(0..kmax-1) of the velocity v on an M^d regular grid: the energy spectrum of Sec. 4.3
    (shells k - 1/2 <= |n| < k + 1/2)."""
    d = mesh.d
    grid = regular_grid(mesh, v, M)
    vol = np.prod([mesh.hi[k] - mesh.lo[k] for k in range(d)])
    E = np.zeros(kmax)
    n1 = np.where(np.arange(M) < M // 2, np.arange(M), np.arange(M) - M).astype(float)
    mag = np.sqrt(sum(np.meshgrid(*([n1] * d), indexing="ij")[k] ** 2 for k in range(d)))
    shell = np.floor(mag + 0.5).astype(int)
    power = np.zeros((M,) * d)
    for c in range(d):
        power += np.abs(np.fft.fftn(grid[c]) / M ** d) ** 2
    for k in range(kmax):
        E[k] = 0.5 * vol * power[shell == k].sum()
    return E
