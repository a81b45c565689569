"""The one-dimensional tables the CUDA kernels read (csrc/basis.cpp: GLL points by Newton's
method and closed-form differentiation matrices, barycentric Lagrange evaluation), compiled
for the host and compared with the oracle's independent construction (numpy's Legendre
roots and product-form Lagrange polynomials, oracle/gll.py) for every supported N = 2..9:
GLL points and weights, differentiation matrices, the pressure basis (N-1 GLL points)
and its derivative at the velocity points, the Gauss over-integration points' weights,
interpolation and derivative matrices (Q = ceil(3N/2) points), the FP32 copies, the
p-multigrid prolongation factors between GLL sets, and the one-dimensional SIPG line
operators (own blocks and neighbour couplings of interior, Dirichlet and Neumann faces)
against the direction-x factor of the oracle's assembled 2D SIPG matrix."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import dg, gll

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2112_04167_gb300", "csrc")


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("basis") / "basis_tables_dump")
    # basis.cpp includes the CUDA header of the tables, so both files compile as CUDA (host
    # code only runs)
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, "-x", "cu", os.path.join(HERE, "native", "basis_tables_dump.cu"),
                    os.path.join(CSRC, "basis.cpp"), "-o", exe], check=True, capture_output=True, timeout=300)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120, check=True)
    out = {}
    for line in r.stdout.splitlines():
        f = line.split()
        if f[0] in ("E", "LDN"):
            out[(f[0], int(f[1]), int(f[2]))] = np.array([float(v) for v in f[3:]])
        elif f[0] == "LA":
            out[("LA", int(f[1]), int(f[2]), int(f[3]))] = np.array([float(v) for v in f[4:]])
        elif f[0] == "LC":
            out[("LC",) + tuple(int(v) for v in f[1:5])] = np.array([float(v) for v in f[5:]])
        elif f[0] == "Q":
            out[("Q", int(f[1]))] = int(f[2])
        else:
            out[(f[0], int(f[1]))] = np.array([float(v) for v in f[2:]])
    return out


def close(a, b, tol):
    a, b = np.ravel(a), np.ravel(b)
    return a.shape == b.shape and np.abs(a - b).max() <= tol * max(1.0, np.abs(b).max())


@pytest.mark.parametrize("N", range(2, 10))
def test_gll_points_weights_derivative(tables, N):
    x, w = gll.gll_nodes_weights(N)
    # numpy's companion-matrix roots (the oracle) carry errors of a few units in the last
    # place (residuals of L_P' up to ~1.5e-13 at N = 8, 9); the library's Newton roots leave
    # residuals below 1e-14, checked directly
    assert close(tables[("x", N)], x, 4e-15)
    if N > 2:
        dLP = np.polynomial.legendre.Legendre.basis(N - 1).deriv()
        assert np.abs(dLP(tables[("x", N)][1:-1])).max() < 1e-14 * N * N
    assert close(tables[("w", N)], w, 1e-14)
    assert close(tables[("D", N)].reshape(N, N), gll.lagrange_eval(x, x, 1), 1e-12)
    # the FP32 tables are the library's own FP64 tables rounded
    assert np.array_equal(tables[("x32", N)], tables[("x", N)].astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("N", range(3, 10))
def test_pressure_basis_at_velocity_points(tables, N):
    x, _ = gll.gll_nodes_weights(N)
    xp, _ = gll.gll_nodes_weights(N - 1)
    assert close(tables[("Ipv", N)].reshape(N, N - 1), gll.lagrange_eval(xp, x, 0), 1e-13)
    assert close(tables[("Gpv", N)].reshape(N, N - 1), gll.lagrange_eval(xp, x, 1), 1e-12)


@pytest.mark.parametrize("N", range(2, 10))
def test_over_integration_tables(tables, N):
    Q = tables[("Q", N)]
    assert Q == gll.over_integration_points(N - 1)
    x, _ = gll.gll_nodes_weights(N)
    xg, wg = gll.gauss_nodes_weights(Q)
    assert close(tables[("gw", N)], wg, 1e-14)
    assert close(tables[("IG", N)].reshape(Q, N), gll.lagrange_eval(x, xg, 0), 1e-13)
    assert close(tables[("DG", N)].reshape(Q, N), gll.lagrange_eval(x, xg, 1), 1e-12)


def test_prolongation_factors(tables):
    for Nf in range(3, 10):
        for Nc in range(2, Nf):
            xc, _ = gll.gll_nodes_weights(Nc)
            xf, _ = gll.gll_nodes_weights(Nf)
            assert close(tables[("E", Nc, Nf)].reshape(Nf, Nc), gll.lagrange_eval(xc, xf, 0), 1e-13), (Nc, Nf)


def line_matrix(tables, N, n, periodic, dirichlet):
    """The 1D SIPG matrix of n unit elements assembled from the library's line operators the
    way the line kernels apply them: the own block for the element's two face kinds, and for
    an interior face the neighbour's trace (its end node) and normal derivative (a row of its
    line) times the side's coefficients."""
    A = np.zeros((n * N, n * N))
    bkind = 2 if dirichlet else 0
    for e in range(n):
        kl = 1 if (periodic or e > 0) else bkind
        kr = 1 if (periodic or e < n - 1) else bkind
        A[e * N:(e + 1) * N, e * N:(e + 1) * N] += tables[("LA", N, kl, kr)].reshape(N, N)
        for side, nb, end in ((0, (e - 1) % n, N - 1), (1, (e + 1) % n, 0)):
            if (kl, kr)[side] != 1:
                continue
            tr = np.zeros(N)
            tr[end] = 1.0
            blk = np.outer(tables[("LC", N, side, 1, 0)], tr) + np.outer(tables[("LC", N, side, 1, 1)],
                                                                         tables[("LDN", N, side)])
            A[e * N:(e + 1) * N, nb * N:(nb + 1) * N] += blk
    return A


def oracle_line_matrix(N, n, periodic, dirichlet):
    """The direction-x factor of the oracle's 2D SIPG matrix (unit viscosity) on n unit
    elements in x and one periodic element in y: for a field constant in y the y-direction
    terms vanish and the 2D operator is (A_x u) times the y mass weights (h_y / 2) w_j."""
    hy = 0.7
    mesh = dg.Mesh(2, N - 1, (n, 1), [0.0, 0.0], [float(n), hy], (periodic, True))
    A2 = dg.sipg_matrix(mesh, N, 1.0, dirichlet=dirichlet)
    A2 = A2.toarray() if hasattr(A2, "toarray") else np.asarray(A2)
    _, w = gll.gll_nodes_weights(N)
    out = np.zeros((n * N, n * N))
    for col in range(n * N):
        U = np.zeros(n * N * N)
        e, i = divmod(col, N)
        for j in range(N):
            U[e * N * N + j * N + i] = 1.0
        Y = (A2 @ U).reshape(n, N, N)                    # [element, y node, x node]
        cols = Y / (0.5 * hy * w)[None, :, None]
        assert np.abs(cols - cols[:, :1, :]).max() <= 1e-11 * max(1.0, np.abs(cols).max())
        out[:, col] = cols[:, 0, :].reshape(-1)
    return out


@pytest.mark.parametrize("N", range(2, 10))
@pytest.mark.parametrize("periodic,dirichlet", [(True, True), (False, True), (False, False)])
def test_line_operators_against_assembled_sipg(tables, N, periodic, dirichlet):
    n = 3
    got = line_matrix(tables, N, n, periodic, dirichlet)
    ref = oracle_line_matrix(N, n, periodic, dirichlet)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), np.abs(got - ref).max()
