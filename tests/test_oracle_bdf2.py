"""Pins of the oracle's IMEX BDF2 (Sec. 2.2 Eq. (bdf2:constant-nu) for the scalar model,
Sec. 3.2.1 for the incompressible flow), against closed forms:

* on the linear model problem du/dt = lambda_c u + lambda_d u the scalar scheme, started with
  one IMEX Euler step, converges to exp((lambda_c + lambda_d) t) at order 2;
* the four-substep flow scheme converges at order 2 in time to the closed-form decaying
  Taylor-Green vortex (periodic) and to the manufactured traveling vortex with time-dependent
  Dirichlet data, variable viscosity and forcing (spatial error far below the temporal one);
* it conserves the mean velocity on a periodic mesh.
"""
import numpy as np
import pytest

from oracle import dg, flows, ns, scalar

TWO_PI = 2 * np.pi


def eoc(errs):
    return [np.log2(a / b) for a, b in zip(errs, errs[1:])]


@pytest.mark.parametrize("lc,ld", [(2.0j, -0.5), (-1.0 + 3.0j, -2.0), (0.5j, 0.0)])
def test_scalar_bdf2_order_two(lc, ld):
    errs = []
    for n in (20, 40, 80, 160):
        us = scalar.bdf2_run(1.0 + 0j, 1.0 / n, n, lambda u: lc * u, lambda r, g: r / (1 - g * ld))
        errs.append(abs(us[-1] - np.exp(lc + ld)))
    assert all(1.9 < e < 2.1 for e in eoc(errs)), errs


def run(disc, fl, n, T):
    dt = T / n
    v, prev, t = fl.initial(disc.X).reshape(disc.d, -1), None, 0.0
    for _ in range(n):
        v, prev, _ = ns.bdf2_step(disc, v, t, dt, prev)
        t += dt
    return v, t


def test_tg2d_order_two():
    mesh = dg.Mesh(2, 8, (4, 4), [0, 0], [TWO_PI, TWO_PI], (True, True))
    fl = flows.Flow("tg2d", 0.05)
    disc = ns.Discretization(mesh, fl)
    errs = []
    for n in (8, 16, 32):
        v, t = run(disc, fl, n, 0.8)
        ex = fl.exact(disc.X, t).reshape(2, -1)
        errs.append(np.linalg.norm(v - ex) / np.linalg.norm(ex))
    assert all(1.9 < e < 2.1 for e in eoc(errs)), errs


@pytest.mark.slow
def test_manufactured_dirichlet_variable_viscosity_order_two():
    mesh = dg.Mesh(2, 8, (4, 4), [0, 0], [1, 1], (False, False))
    fl = flows.Flow("tgtravel", 0.01, nu_kind="varxyt")
    disc = ns.Discretization(mesh, fl)
    errs = []
    for n in (4, 8, 16):
        v, t = run(disc, fl, n, 0.04)
        ex = fl.exact(disc.X, t).reshape(2, -1)
        errs.append(np.linalg.norm(v - ex) / np.linalg.norm(ex))
    assert errs[-1] > 1e-5                       # temporal error above the spatial floor (6e-7)
    assert all(1.8 < e < 2.2 for e in eoc(errs)), errs


def test_mean_velocity_conserved():
    mesh = dg.Mesh(2, 5, (3, 3), [0, 0], [TWO_PI, TWO_PI], (True, True))
    fl = flows.Flow("tg2d", 0.02)
    disc = ns.Discretization(mesh, fl)
    rng = np.random.default_rng(3)
    v = fl.initial(disc.X).reshape(2, -1) + 0.1 * rng.standard_normal((2, disc.nv)) + np.array([[0.3], [-0.2]])
    m0 = (v * disc.Mv).sum(axis=1)
    prev, t = None, 0.0
    for _ in range(3):
        v, prev, _ = ns.bdf2_step(disc, v, t, 0.02, prev)
        t += 0.02
    assert np.abs((v * disc.Mv).sum(axis=1) - m0).max() < 1e-12 * disc.Mv.sum()
