"""Pins of the flow statistics of Sec. 4.3 (oracle/diagnostics.py) against closed forms:

* the dissipation rate of the 3D Taylor-Green initial field, (1 / |Omega|) int nu |grad v|^2 =
  3 nu / 4 (each of its six nonzero derivatives squared averages to 1/8), reached by the DG
  interpolant to its interpolation error; and exact for a field inside the polynomial space;
* the energy spectrum of the Taylor-Green field: all of the energy 1/2 int |v|^2 = pi^3 in the
  shell k = 2 (its wave vectors (+-1, +-1, +-1) have length sqrt 3), and of a single Fourier
  mode sin(3 x) in the shell k = 3 with energy 2 pi^3; the shells add up to the grid energy.
"""
import numpy as np
import pytest

from oracle import dg, diagnostics, flows

TWO_PI = 2 * np.pi


@pytest.fixture(scope="module")
def tg3d():
    mesh = dg.Mesh(3, 7, (4, 4, 4), [0, 0, 0], [TWO_PI] * 3, (True, True, True))
    X = mesh.node_coords(8)
    return mesh, flows.tg3d_velocity(X).reshape(3, -1)


def test_dissipation_taylor_green(tg3d):
    mesh, v = tg3d
    nu = 1.0 / 1600
    assert abs(diagnostics.dissipation(mesh, v, nu) - 0.75 * nu) < 1e-5 * 0.75 * nu


def test_dissipation_exact_for_polynomials():
    mesh = dg.Mesh(2, 4, (3, 2), [0.0, -1.0], [1.5, 1.0], (False, False))
    X = mesh.node_coords(5)
    x, y = X[..., 0].ravel(), X[..., 1].ravel()
    v = np.stack([x ** 2 * y, x - 3 * y ** 2])          # grad: (2xy, x^2; 1, -6y)
    # int over [0, 1.5] x [-1, 1] of (4 x^2 y^2 + x^4 + 1 + 36 y^2), divided by the area 3
    ref = (4 * (1.5 ** 3 / 3) * (2 / 3) + (1.5 ** 5 / 5) * 2 + 3 + 36 * 1.5 * (2 / 3)) / 3.0
    assert abs(diagnostics.dissipation(mesh, v, 1.0) - ref) < 1e-12 * ref


def test_spectrum_taylor_green(tg3d):
    mesh, v = tg3d
    E = diagnostics.energy_spectrum(mesh, v, 32, 8)
    assert abs(E[2] - np.pi ** 3) < 1e-5 * np.pi ** 3
    assert np.abs(np.delete(E, 2)).max() < 1e-5 * np.pi ** 3


def test_spectrum_single_mode():
    mesh = dg.Mesh(3, 6, (8, 2, 2), [0, 0, 0], [TWO_PI] * 3, (True, True, True))
    X = mesh.node_coords(7)
    v = np.zeros((3, X.shape[0] * X.shape[1]))
    v[0] = np.sin(3 * X[..., 0]).ravel()
    E = diagnostics.energy_spectrum(mesh, v, 16, 6)
    assert abs(E[3] - 2 * np.pi ** 3) < 1e-5 * 2 * np.pi ** 3
    assert np.abs(np.delete(E, 3)).max() < 1e-5 * 2 * np.pi ** 3
    grid = diagnostics.regular_grid(mesh, v, 16)
    assert abs(E.sum() - 0.5 * TWO_PI ** 3 * np.mean(np.sum(grid ** 2, axis=0))) < 1e-10
