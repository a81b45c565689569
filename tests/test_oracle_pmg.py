"""Pins of the oracle's p-multigrid preconditioner (oracle/pmg.py), checked against what the
mathematics fixes, independently of the CUDA path:

* the level degrees halve down to degree 1;
* the 1D transfer interpolates polynomials of the coarse degree exactly, and the
  prolongation maps every element-wise polynomial of the coarse degree to itself;
* the Chebyshev recurrence multiplies an eigenvector of D^{-1} A with eigenvalue lam by the
  closed-form factor T_k((theta - lam) / delta) / T_k(theta / delta) (numpy's Chebyshev
  series as the independent evaluation of T_k);
* the V-cycle is a symmetric operator, positive on the mean-free vectors (what CG needs of a
  preconditioner);
* CG preconditioned by it reaches the solution of the bordered sparse LU of the oracle's
  Poisson problem, in far fewer iterations than Jacobi and in a count that does not grow
  with the mesh.
"""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

from oracle import dg, flows, gll, ns, pmg

TWO_PI = 2 * np.pi


def rng(seed):
    return np.random.default_rng(seed)


def test_level_points():
    assert pmg.level_points(7) == [7, 4, 2]      # degrees 6, 3, 1
    assert pmg.level_points(8) == [8, 4, 2]      # 7, 3, 1
    assert pmg.level_points(6) == [6, 3, 2]      # 5, 2, 1
    assert pmg.level_points(4) == [4, 2]
    assert pmg.level_points(3) == [3, 2]
    assert pmg.level_points(2) == [2]


@pytest.mark.parametrize("Nc,Nf", [(2, 4), (4, 7), (3, 5), (4, 8), (5, 5)])
def test_interp_exact_for_coarse_polynomials(Nc, Nf):
    I = pmg.interp_1d(Nc, Nf)
    xc, _ = gll.gll_nodes_weights(Nc)
    xf, _ = gll.gll_nodes_weights(Nf)
    for deg in range(Nc):
        c = rng(deg).standard_normal(deg + 1)
        assert np.abs(I @ np.polyval(c, xc) - np.polyval(c, xf)).max() < 1e-13
    if Nc == Nf:
        assert np.abs(I - np.eye(Nc)).max() < 1e-13


def test_prolongation_of_elementwise_polynomials():
    mesh = dg.Mesh(3, 5, (2, 3, 2), [0.1, 0.0, -0.2], [1.3, 0.9, 0.8], (True, False, True))
    Nc, Nf = 3, 5
    Pr = pmg.prolongation(mesh, Nc, Nf)
    Xc, Xf = mesh.node_coords(Nc), mesh.node_coords(Nf)
    # a different polynomial of degree Nc - 1 per direction in every element
    for e in range(mesh.ne):
        a = rng(e).standard_normal(3)
        fc = np.zeros_like(Xc[..., 0])
        fc[e] = (1 + a[0] * Xc[e, :, 0] ** 2) * (a[1] - Xc[e, :, 1]) * (2 + a[2] * Xc[e, :, 2] + Xc[e, :, 2] ** 2)
        ff = (Pr @ fc.ravel()).reshape(mesh.ne, -1)
        ref = (1 + a[0] * Xf[e, :, 0] ** 2) * (a[1] - Xf[e, :, 1]) * (2 + a[2] * Xf[e, :, 2] + Xf[e, :, 2] ** 2)
        assert np.abs(ff[e] - ref).max() < 1e-13
        others = np.delete(ff, e, axis=0)
        assert np.abs(others).max() == 0.0
    assert np.abs(Pr @ np.ones(Pr.shape[1]) - 1.0).max() < 1e-14


@pytest.mark.parametrize("steps,ratio", [(1, 10.0), (3, 10.0), (5, 30.0), (10, 100.0)])
def test_chebyshev_closed_form_factor(steps, ratio):
    mesh = dg.Mesh(2, 3, (3, 2), [0, 0], [1.0, 0.7], (True, False))
    A = dg.sipg_matrix(mesh, 3, 1.0, dirichlet=False).toarray()
    dinv = 1.0 / np.diag(A)
    s = np.sqrt(dinv)
    lam, W = np.linalg.eigh(s[:, None] * A * s[None, :])
    V = s[:, None] * W                       # A v = lam D v
    lmax = 1.05 * lam[-1]
    lmin = lmax / ratio
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    Tk = npcheb.Chebyshev.basis(steps)
    for j in (0, 3, len(lam) // 2, len(lam) - 1):
        v = V[:, j]
        got = pmg.chebyshev(A, dinv, np.zeros_like(v), v, steps, lmax, ratio)   # error e_0 = v
        factor = Tk((theta - lam[j]) / delta) / Tk(theta / delta)
        assert np.abs(got - factor * v).max() < 1e-12 * max(1.0, np.abs(v).max())
        assert abs(factor) <= 1.0 + 1e-12        # (1 at the null-space eigenvalue 0)


@pytest.fixture(scope="module")
def small3d():
    mesh = dg.Mesh(3, 5, (3, 2, 3), [0, 0, 0], [1.5, 1.0, 1.2], (True, False, True))
    return mesh, pmg.PMG(mesh, 5)


def test_vcycle_symmetric_positive(small3d):
    _, M = small3d
    n = M.A[0].shape[0]
    for seed in range(3):
        a = rng(10 + seed).standard_normal(n)
        b = rng(20 + seed).standard_normal(n)
        a -= a.mean()
        b -= b.mean()
        Va, Vb = M.vcycle(a), M.vcycle(b)
        assert abs(Va @ b - a @ Vb) < 1e-12 * np.linalg.norm(Va) * np.linalg.norm(b)
        assert Va @ a > 0.0


def test_pcg_solution_equals_bordered_lu(small3d):
    mesh, M = small3d
    disc = ns.Discretization(mesh, flows.Flow("tgtravel", 0.01))
    b = rng(5).standard_normal(disc.npr)
    ref = disc.poisson(b.copy())
    x, its = pmg.pcg(M.A[0], b, M.vcycle, 1e-13, weights=disc.Mp)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-11
    _, its_j = pmg.pcg(M.A[0], b, lambda r: M.dinv[0] * r, 1e-13, maxit=5000)
    assert its <= 20 and its_j > 4 * its


def test_iterations_flat_in_mesh_size():
    counts = []
    for n in (4, 8, 16):
        mesh = dg.Mesh(2, 6, (n, n), [0, 0], [TWO_PI, TWO_PI], (True, True))
        M = pmg.PMG(mesh, 6)
        b = rng(n).standard_normal(M.A[0].shape[0])
        counts.append(pmg.pcg(M.A[0], b, M.vcycle, 1e-10)[1])
    assert max(counts) <= 20 and counts[-1] - counts[0] <= 6, counts


def test_largest_eig_matches_dense():
    mesh = dg.Mesh(2, 5, (5, 4), [0, 0], [1, 1], (False, True))
    A = dg.sipg_matrix(mesh, 5, 1.0, dirichlet=False)
    dinv = 1.0 / A.diagonal()
    s = np.sqrt(dinv)
    dense = np.linalg.eigvalsh(s[:, None] * A.toarray() * s[None, :])[-1]
    assert abs(pmg.largest_eig(A, dinv) - dense) < 1e-9 * dense
