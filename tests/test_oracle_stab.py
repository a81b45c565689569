"""Pins of the oracle's divergence / mass-flux stabilisation (oracle/stab.py):

* the penalty matrix is symmetric and positive semi-definite, the stabilised system positive
  definite, and zero penalty factors give back the input;
* a continuous, divergence-free polynomial velocity (no broken divergence, no normal jumps)
  is left unchanged;
* the stabilised velocity minimises  ||w - v||_M^2 + w^T A w  over all w (compared with random
  perturbations), so its penalised divergence and jumps are below those of the input.
"""
import numpy as np
import pytest

from oracle import dg, stab

TWO_PI = 2 * np.pi


def field(mesh, seed):
    n = mesh.ne * (mesh.P + 1) ** mesh.d
    return np.random.default_rng(seed).standard_normal((mesh.d, n)) + 0.5


@pytest.mark.parametrize("d,P,n,per", [(2, 3, (3, 2), (True, False)), (3, 2, (2, 2, 2), (True, True, False))])
def test_penalty_symmetric_semidefinite(d, P, n, per):
    mesh = dg.Mesh(d, P, n, [0.0] * d, [1.0, 1.3, 0.8][:d], per)
    v = field(mesh, 1)
    A = stab.penalty_matrix(mesh, v, 0.05, 1.0, 1.0).toarray()
    assert np.abs(A - A.T).max() < 1e-14 * np.abs(A).max()
    lam = np.linalg.eigvalsh(A)
    assert lam.min() > -1e-12 * lam.max() and lam.max() > 0
    assert np.abs(stab.stabilize(mesh, v, 0.05, 0.0, 0.0) - v).max() < 1e-14


@pytest.mark.parametrize("d", [2, 3])
def test_divergence_free_polynomial_unchanged(d):
    mesh = dg.Mesh(d, 3, (3,) * d, [0.0] * d, [1.0] * d, (False,) * d)
    X = mesh.node_coords(4)
    x, y = X[..., 0].ravel(), X[..., 1].ravel()
    if d == 2:
        v = np.stack([y ** 2, x ** 2 + 1.0])
    else:
        z = X[..., 2].ravel()
        v = np.stack([y ** 2 + z, z ** 2 - x, x ** 2 + 2.0])
    assert np.abs(stab.stabilize(mesh, v, 0.1, 2.0, 2.0) - v).max() < 1e-11 * np.abs(v).max()


def test_minimiser_of_the_penalised_distance():
    mesh = dg.Mesh(2, 4, (3, 3), [0, 0], [TWO_PI, TWO_PI], (True, True))
    v = field(mesh, 2)
    dt, zd, zc = 0.1, 1.0, 1.0
    A = stab.penalty_matrix(mesh, v, dt, zd, zc)
    M = np.tile(dg.mass_diag(mesh, 5), 2)
    vt = stab.stabilize(mesh, v, dt, zd, zc).ravel()
    vr = v.ravel()

    def J(w):
        return (w - vr) @ (M * (w - vr)) + w @ (A @ w)

    rng = np.random.default_rng(3)
    for _ in range(5):
        assert J(vt) <= J(vt + 1e-3 * rng.standard_normal(vt.size))
    assert vt @ (A @ vt) < vr @ (A @ vr)


@pytest.mark.parametrize("d", [2, 3])
def test_mean_speed_closed_forms(d):
    """|u_K| of a constant field is its length on every element; the mass-weighted mean of an
    affine field over an element is its value at the element's centre (GLL quadrature is
    exact for degree 1), so |u_K| is the speed there."""
    mesh = dg.Mesh(d, 3, (3, 2, 2)[:d], [0.0] * d, [1.0, 1.3, 0.8][:d], (False,) * d)
    n = mesh.ne * (mesh.P + 1) ** d
    c = np.array([0.3, -1.2, 0.7][:d])
    v = np.repeat(c[:, None], n, axis=1)
    assert np.abs(stab.mean_speed(mesh, v) - np.linalg.norm(c)).max() < 1e-14
    X = mesh.node_coords(mesh.P + 1)                       # (ne, N^d, d)
    A = np.random.default_rng(4).standard_normal((d, d))
    b = np.random.default_rng(5).standard_normal(d)
    v = (np.einsum("ck,enk->cen", A, X) + b[:, None, None]).reshape(d, -1)
    centre = X.mean(axis=1)                                # symmetric nodes: the mean is the centre
    exact = np.linalg.norm(np.einsum("ck,ek->ce", A, centre) + b[:, None], axis=0)
    assert np.abs(stab.mean_speed(mesh, v) - exact).max() < 1e-13
