"""Pins of the oracle's closed-form flows (oracle/flows.py) against what the paper and the
mathematics fix, independently of the CUDA path.

* tg3d_velocity: the initial field of the Taylor-Green transition, Eq. (transition:v0) of
  Sec. 4.3, v0 = (cos x sin y sin z, -sin x cos y sin z, 0) on [-pi, pi]^3, is written on
  [0, 2 pi]^3 as (sin x cos y cos z, -cos x sin y cos z, 0): the paper's field at the point
  shifted by -pi/2 in x and +pi/2 in y and z.  It is solenoidal, 2 pi-periodic and its
  largest velocity is v_{0,max} = 1 (the reference velocity of Sec. 4.3).
* tg2d_velocity / tg2d_pressure: the decaying Taylor-Green vortex is an exact solution of
  the incompressible Navier-Stokes equations, d_t v + (v . grad) v + grad p = nu lap v,
  div v = 0 -- checked by finite differences at random points (a wrong sign, factor or
  decay rate in either field fails it).
"""
import numpy as np

from oracle import flows

PI = np.pi


def paper_v0(X):
    """Eq. (transition:v0) as printed in Sec. 4.3 (domain [-pi, pi]^3)."""
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    return np.stack([np.cos(x) * np.sin(y) * np.sin(z), -np.sin(x) * np.cos(y) * np.sin(z), np.zeros_like(x)])


def points(n, d, seed, lo=0.0, hi=2 * PI):
    return np.random.default_rng(seed).uniform(lo, hi, size=(n, d))


def fd_grad(f, X, h=1e-5):
    """G[c, k, i] = d f_c / d x_k at the points X (central differences)."""
    d = X.shape[-1]
    cols = []
    for k in range(d):
        e = np.zeros(d)
        e[k] = h
        cols.append((f(X + e) - f(X - e)) / (2 * h))
    return np.stack(cols, axis=1)


def test_tg3d_is_the_papers_field_shifted():
    X = points(2000, 3, 1)
    shift = np.array([-PI / 2, PI / 2, PI / 2])
    assert np.abs(flows.tg3d_velocity(X) - paper_v0(X + shift)).max() < 1e-14


def test_tg3d_solenoidal_periodic_unit_maximum():
    X = points(2000, 3, 2)
    G = fd_grad(flows.tg3d_velocity, X)
    assert np.abs(G[0, 0] + G[1, 1] + G[2, 2]).max() < 1e-9
    # not trivially solenoidal: the in-plane strain is order one
    assert np.abs(G[0, 0]).max() > 0.5
    for k in range(3):
        e = np.zeros(3)
        e[k] = 2 * PI
        assert np.abs(flows.tg3d_velocity(X + e) - flows.tg3d_velocity(X)).max() < 1e-13
    g = np.linspace(0, 2 * PI, 33)
    Xg = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1)
    assert abs(np.abs(flows.tg3d_velocity(Xg)).max() - 1.0) < 1e-14


def test_tg2d_exact_navier_stokes_solution():
    nu, h = 0.037, 1e-4
    X = points(500, 2, 3)
    for t in (0.0, 0.7, 3.1):
        v = flows.tg2d_velocity(X, t, nu)
        dvdt = (flows.tg2d_velocity(X, t + h, nu) - flows.tg2d_velocity(X, t - h, nu)) / (2 * h)
        G = fd_grad(lambda Y: flows.tg2d_velocity(Y, t, nu), X, h)
        gp = fd_grad(lambda Y: flows.tg2d_pressure(Y, t, nu)[None], X, h)[0]
        lap = np.zeros_like(v)
        for k in range(2):
            e = np.zeros(2)
            e[k] = h
            lap += (flows.tg2d_velocity(X + e, t, nu) - 2 * v + flows.tg2d_velocity(X - e, t, nu)) / h ** 2
        adv = np.stack([v[0] * G[c, 0] + v[1] * G[c, 1] for c in range(2)])
        res = dvdt + adv + gp - nu * lap
        assert np.abs(res).max() < 1e-6, t
        assert np.abs(G[0, 0] + G[1, 1]).max() < 1e-9


def vv_flux_divergence_fd(X, t, nu0, nu1, vmax, h=1e-4):
    """div(v v) - div[nu(v) (grad v + grad v^T)] at X by central differences of the fluxes,
    each flux built from the closed-form velocity and a finite-difference gradient."""
    def flux(Y):
        v = flows.vv_velocity(Y, t)
        G = fd_grad(lambda Z: flows.vv_velocity(Z, t), Y, 1e-5)
        nu = nu0 + nu1 * np.sum(v ** 2, axis=0) / vmax ** 2
        return np.stack([np.stack([v[c] * v[k] - nu * (G[c, k] + G[k, c]) for k in range(3)]) for c in range(3)])
    out = np.zeros((3,) + X.shape[:-1])
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        out += (flux(X + e)[:, k] - flux(X - e)[:, k]) / (2 * h)
    return out


def test_vv_exact_solution_of_the_forced_problem():
    """Eq. (var-visc-test): solenoidal, period 1, maximum speed 2, and the forcing of Eq.
    (var-visc-test:rhs) equals d_t v + div(v v) - div[nu(v)(grad v + grad v^T)] + grad p
    evaluated by finite differences of the closed forms."""
    nu0, nu1, vmax, t = 0.01, 0.03, 2.0, 0.37
    X = points(200, 3, 5, -0.5, 0.5)
    G = fd_grad(lambda Y: flows.vv_velocity(Y, t), X)
    assert np.abs(G[0, 0] + G[1, 1] + G[2, 2]).max() < 1e-8
    assert np.abs(G - flows.vv_grad(X, t)).max() < 1e-7
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        assert np.abs(flows.vv_velocity(X + e, t) - flows.vv_velocity(X, t)).max() < 1e-12
    g = np.linspace(-0.5, 0.5, 41)
    Xg = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1)
    assert abs(np.sqrt(np.sum(flows.vv_velocity(Xg, 0.0) ** 2, axis=0)).max() - 2.0) < 1e-12
    h = 1e-5
    dvdt = (flows.vv_velocity(X, t + h) - flows.vv_velocity(X, t - h)) / (2 * h)
    gp = fd_grad(lambda Y: flows.vv_pressure(Y, t)[None], X)[0]
    ref = dvdt + vv_flux_divergence_fd(X, t, nu0, nu1, vmax) + gp
    f = flows.forcing_vv(X, t, nu0, nu1, vmax)
    assert np.abs(f - ref).max() < 1e-4 * np.abs(ref).max()


def tgtravel_pressure(X, t, nu0):
    """Pressure of the traveling Taylor-Green vortex (the uniform translation (1, 1) carries
    the classical field p = (cos 2a + cos 2b) / 4 decaying with the square of the velocity's
    factor), written out here so that the pin below does not rest on the oracle's fields."""
    a = 2 * PI * (X[..., 0] - t)
    b = 2 * PI * (X[..., 1] - 0.125 - t)
    return 0.25 * (np.cos(2 * a) + np.cos(2 * b)) * np.exp(-16 * PI ** 2 * nu0 * t)


def test_tgtravel_gradients_are_the_derivatives():
    """The closed-form gradients of the traveling vortex and of the viscosity nu(x, y, t) used
    by the manufactured forcing equal central differences of the fields themselves."""
    nu0, t = 0.01, 0.41
    X = points(400, 2, 7, 0.0, 1.0)
    G = fd_grad(lambda Y: flows.tgtravel_velocity(Y, t, nu0), X)
    assert np.abs(G - flows.tgtravel_grad(X, t, nu0)).max() < 1e-8
    gn = fd_grad(lambda Y: flows.nu_varxyt(Y, t, nu0)[None], X)[0]
    assert np.abs(gn - flows.nu_varxyt_grad(X, t, nu0)).max() < 1e-10
    # the viscosity law: nu0 (1 + sin(2 pi x) sin(2 pi y) cos(t) / 2) stays within nu0 [1/2, 3/2]
    nu = flows.nu_varxyt(points(4000, 2, 8, 0.0, 1.0), 0.0, nu0)
    assert nu.min() >= 0.5 * nu0 - 1e-15 and nu.max() <= 1.5 * nu0 + 1e-15
    assert nu.max() - nu.min() > 0.9 * nu0


def test_tgtravel_constant_viscosity_is_exact():
    """With nu = nu0 the traveling vortex solves the unforced Navier-Stokes equations with the
    pressure above and is solenoidal (so the forcing below carries only the viscosity's
    variation)."""
    nu0, h = 0.01, 1e-4
    X = points(400, 2, 9, 0.0, 1.0)
    for t in (0.0, 0.23, 0.9):
        v = flows.tgtravel_velocity(X, t, nu0)
        dvdt = (flows.tgtravel_velocity(X, t + h, nu0) - flows.tgtravel_velocity(X, t - h, nu0)) / (2 * h)
        G = fd_grad(lambda Y: flows.tgtravel_velocity(Y, t, nu0), X, h)
        gp = fd_grad(lambda Y: tgtravel_pressure(Y, t, nu0)[None], X, h)[0]
        lap = np.zeros_like(v)
        for k in range(2):
            e = np.zeros(2)
            e[k] = h
            lap += (flows.tgtravel_velocity(X + e, t, nu0) - 2 * v + flows.tgtravel_velocity(X - e, t, nu0)) / h ** 2
        adv = np.stack([v[0] * G[c, 0] + v[1] * G[c, 1] for c in range(2)])
        res = dvdt + adv + gp - nu0 * lap
        assert np.abs(res).max() < 1e-5 * np.abs(dvdt).max(), t
        assert np.abs(G[0, 0] + G[1, 1]).max() < 1e-8
        assert np.abs(flows.forcing_tgtravel_varnu(X, t, nu0) - 0.0).max() > 1e-3  # nu varies: f != 0


def test_tgtravel_varnu_forcing_closes_the_equations():
    """The manufactured forcing of the variable-viscosity traveling vortex equals
    d_t v + div(v v) + grad p - div[nu(x, y, t) (grad v + grad v^T)] evaluated by finite
    differences of the closed forms (a dropped term, a wrong sign or a transposed gradient
    in the forcing fails this)."""
    nu0, t, h = 0.01, 0.37, 1e-4
    X = points(300, 2, 11, 0.0, 1.0)

    def flux(Y):
        v = flows.tgtravel_velocity(Y, t, nu0)
        G = fd_grad(lambda Z: flows.tgtravel_velocity(Z, t, nu0), Y, 1e-5)
        nu = flows.nu_varxyt(Y, t, nu0)
        return np.stack([np.stack([v[c] * v[k] - nu * (G[c, k] + G[k, c]) for k in range(2)]) for c in range(2)])

    div = np.zeros((2, X.shape[0]))
    for k in range(2):
        e = np.zeros(2)
        e[k] = h
        div += (flux(X + e)[:, k] - flux(X - e)[:, k]) / (2 * h)
    dvdt = (flows.tgtravel_velocity(X, t + 1e-5, nu0) - flows.tgtravel_velocity(X, t - 1e-5, nu0)) / 2e-5
    gp = fd_grad(lambda Y: tgtravel_pressure(Y, t, nu0)[None], X)[0]
    ref = dvdt + div + gp
    f = flows.forcing_tgtravel_varnu(X, t, nu0)
    assert np.abs(ref).max() > 0.05
    assert np.abs(f - ref).max() < 1e-4 * np.abs(ref).max()
