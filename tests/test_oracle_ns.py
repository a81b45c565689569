"""Pins of the oracle's Navier-Stokes steps (Alg. 3, Alg. 4) against closed-form flows,
invariants and the design orders of the tableaux (Sec. 3.2, Sec. 4.1)."""
import numpy as np
import pytest

from oracle import dg, flows, ns

TWO_PI = 2 * np.pi


def _tg2d(P=4, n=4, mode="sipg"):
    m = dg.Mesh(2, P, (n, n), [0, 0], [TWO_PI, TWO_PI], (True, True))
    fl = flows.Flow("tg2d", 0.01)
    return ns.Discretization(m, fl, poisson=mode), fl


def test_tg2d_closed_form_and_invariants():
    disc, fl = _tg2d(P=6)
    v = fl.initial(disc.X).reshape(2, -1)
    t, dt = 0.0, 0.01
    for _ in range(20):
        v, _ = ns.rk_step(disc, "CB3e", v, t, dt)
        t += dt
    ex = fl.exact(disc.X, t).reshape(2, -1)
    assert ns.relative_l2(v, ex) < 2e-4                     # spatial floor at P=6
    M = disc.Mv
    assert np.abs((M[None] * v).sum(axis=1)).max() < 1e-13  # mean momentum conserved


def test_tg2d_spectral_in_p():
    errs = []
    for P in (4, 6, 8):
        disc, fl = _tg2d(P=P)
        v = fl.initial(disc.X).reshape(2, -1)
        t = 0.0
        for _ in range(5):
            v, _ = ns.rk_step(disc, "ARS3", v, t, 0.02)
            t += 0.02
        errs.append(ns.relative_l2(v, fl.exact(disc.X, t).reshape(2, -1)))
    assert errs[0] > 20 * errs[1] > 400 * errs[2]


def test_consistent_projection_is_divergence_free():
    """In the consistent mode v'' = v' - G psi satisfies B v'' = int (n . v_b) q to round-off."""
    m = dg.Mesh(2, 4, (3, 2), [0, 0], [1, 1], (False, True))
    fl = flows.Flow("tgtravel", 0.01)
    disc = ns.Discretization(m, fl, poisson="consistent")
    rng = np.random.default_rng(5)
    vp = rng.standard_normal((2, disc.nv))
    vb = disc.vb(0.1)
    b0 = disc.div_rhs(vp, vb, "data")
    psi = disc.poisson(b0)
    vpp = vp - disc.grad_p(psi)
    b1 = disc.div_rhs(vpp, vb, "data")
    assert np.linalg.norm(b1 - b1.mean()) < 1e-12 * np.linalg.norm(b0)


def test_sipg_projection_reduces_divergence():
    disc, fl = _tg2d(P=5)
    v = fl.initial(disc.X).reshape(2, -1)
    X = disc.X.reshape(-1, 2)
    gp = np.stack([-0.5 * np.sin(2 * X[:, 0]), -0.5 * np.sin(2 * X[:, 1])])
    vp = v + 0.3 * gp
    psi = disc.poisson(disc.div_rhs(vp, None, "data"))
    vpp = vp - disc.grad_p(psi)
    assert ns.relative_l2(vpp, v) < 2e-2
    assert ns.divergence_norm(disc, vpp, None, 0) < 0.05 * ns.divergence_norm(disc, vp, None, 0)


@pytest.mark.parametrize("periodic", [(True, True), (False, True)])
def test_fd2_plus_fd3_vanishes_for_constant_nu(periodic):
    m = dg.Mesh(2, 3, (3, 2), [0, 0], [1, 1.5], periodic)
    disc = ns.Discretization(m, flows.Flow("tgtravel", 0.01))
    v = np.random.default_rng(2).standard_normal((2, disc.nv))
    nu = np.full(disc.nv, 0.37)
    s = disc.Fd2(v, nu) + disc.Fd3(v, nu)
    assert np.abs(s).max() < 1e-10 * np.abs(disc.Fd3(v, nu)).max()


def test_mms_forcing_consistency():
    """With the exact traveling vortex, F_c + F_d + F_s - grad p = d_t v up to the spatial error
    (checks the derived forcing of the variable-viscosity case)."""
    errs = []
    for P in (6, 8):
        m = dg.Mesh(2, P, (4, 4), [0, 0], [1, 1], (False, False))
        fl = flows.Flow("tgtravel", 0.01, nu_kind="varxyt")
        disc = ns.Discretization(m, fl)
        t = 0.3
        X = disc.X.reshape(-1, 2)
        v = fl.exact(disc.X, t).reshape(2, -1)
        nu = disc.nu_field(t, v)
        vb = disc.vb(t)
        F = disc.Fc(v, vb) + disc.Fd1(v, nu, vb) + disc.Fd2(v, nu) + disc.Fd3(v, nu) + disc.fs(t)
        x, y = X.T
        a, b = TWO_PI * (x - t), TWO_PI * (y - 0.125 - t)
        E2 = np.exp(-16 * np.pi ** 2 * 0.01 * t)
        gp = np.stack([-np.pi * np.sin(2 * a) * E2, -np.pi * np.sin(2 * b) * E2])
        h = 1e-6
        dvdt = (fl.exact(disc.X, t + h) - fl.exact(disc.X, t - h)).reshape(2, -1) / (2 * h)
        errs.append(np.abs(F - gp - dvdt).max() / np.abs(dvdt).max())
    assert errs[1] < 0.05 * errs[0] and errs[1] < 1e-3, errs


def _travel_periodic(P=7, n=3):
    m = dg.Mesh(2, P, (n, n), [0, 0], [1, 1], (True, True))
    fl = flows.Flow("tgtravel", 0.02)
    return ns.Discretization(m, fl, poisson="consistent"), fl


def _time_eoc(stepper, T, dts, dt_ref):
    """EOC against a fine-step run of the same spatial discretisation.  At low P the DG
    divergence / Helmholtz commutator adds a first-order splitting term of size
    O(dt nu eps_h); at P = 7 it is below the measured range."""
    disc, fl = _travel_periodic()
    v0 = fl.initial(disc.X).reshape(2, -1)

    def run(dt):
        v, t = v0, 0.0
        for _ in range(int(round(T / dt))):
            v = stepper(disc, v, t, dt)
            t += dt
        return v
    ref = run(dt_ref)
    e = [ns.rms(run(dt) - ref) for dt in dts]
    return np.log(e[0] / e[1]) / np.log(dts[0] / dts[1])


@pytest.mark.parametrize("tab,order", [("ARS3", 3), ("CB2", 2), ("CB3e", 3)])
def test_alg3_temporal_order_periodic(tab, order):
    """TGP-like periodic traveling vortex: the semi-discrete system shows the design order."""
    eoc = _time_eoc(lambda d, v, t, dt: ns.rk_step(d, tab, v, t, dt)[0], 0.1, (0.01, 0.005), 0.00125)
    assert eoc == pytest.approx(order, abs=0.35)


def test_alg4_temporal_order_periodic():
    """SDC-Eu(2,2): order min(K+1, 2M) = 3 on the periodic traveling vortex."""
    eoc = _time_eoc(lambda d, v, t, dt: ns.sdc_step(d, 2, 2, "EULER", v, t, dt), 0.1, (0.05, 0.025),
                    0.0025)
    assert eoc == pytest.approx(3.0, abs=0.4)


def test_dirichlet_variable_nu_step_accuracy():
    """Config-3-type step (Dirichlet data, variable nu, forcing, final projection) stays close
    to the manufactured solution."""
    m = dg.Mesh(2, 6, (3, 3), [0, 0], [1, 1], (False, False))
    fl = flows.Flow("tgtravel", 0.01, nu_kind="varxyt")
    disc = ns.Discretization(m, fl)
    v = fl.initial(disc.X).reshape(2, -1)
    t, dt = 0.0, 2e-3
    for _ in range(5):
        v, _ = ns.rk_step(disc, "ARS3", v, t, dt)
        t += dt
    assert ns.relative_l2(v, fl.exact(disc.X, t).reshape(2, -1)) < 5e-4
