"""GPU parity of whole steps of Alg. 3 (IMEX RK) and Alg. 4 (SISDC) against the oracle.

Each step starts both sides from the same state; the FP64 GPU step must match the
oracle's step to 1e-11 relative L2 (solves converged to 1e-14 on both sides: the
oracle by sparse LU, the GPU by CG).  The mixed form (FP32 inner solves, FP64
refinement to 1e-12) must agree to 1e-9."""
import numpy as np
import pytest

from oracle import dg, flows, ns

pytestmark = pytest.mark.gpu

imex = pytest.importorskip("paper_2112_04167_gb300.imex")
TWO_PI = 2 * np.pi


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2112_04167_gb300 import build
    build.build()
    imex.load()


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def tg2d_pair(P=4, n=4, precision=imex.FP64, poisson=imex.POISSON_SIPG, tol=1e-14):
    ctx = imex.Context(2, P, (n, n), [0, 0], [TWO_PI, TWO_PI], (1, 1), precision=precision, poisson=poisson,
                       tol=tol, maxit=50000)
    ctx.set_viscosity_const(0.01)
    mesh = dg.Mesh(2, P, (n, n), [0, 0], [TWO_PI, TWO_PI], (True, True))
    fl = flows.Flow("tg2d", 0.01)
    disc = ns.Discretization(mesh, fl, poisson="sipg" if poisson == imex.POISSON_SIPG else "consistent")
    return ctx, disc, fl


def mms_pair(P=5, n=3, precision=imex.FP64, tol=1e-14):
    ctx = imex.Context(2, P, (n, n), [0, 0], [1, 1], (0, 0), precision=precision, tol=tol, maxit=50000)
    ctx.set_viscosity_model(imex.NU_VARXYT, [0.01])
    ctx.set_boundary(imex.FLOW_TGTRAVEL, [0.01])
    ctx.set_forcing(imex.FORCE_TGTRAVEL_VARNU, [0.01])
    mesh = dg.Mesh(2, P, (n, n), [0, 0], [1, 1], (False, False))
    fl = flows.Flow("tgtravel", 0.01, nu_kind="varxyt")
    return ctx, ns.Discretization(mesh, fl), fl


def run_steps(ctx, disc, stepper, v0, t0, dt, nsteps, tol):
    v, t = v0, t0
    for _ in range(nsteps):
        ctx.set_state(t, v)
        ctx.step(dt, 1)
        got = ctx.get_velocity()
        v = stepper(v, t, dt)
        t += dt
        assert rel(got, v) < tol, rel(got, v)
    return v


@pytest.mark.parametrize("tab", ["CB3e", "ARS3", "CB2", "TR", "CB4", "CB3c"])
def test_rk_step_tg2d(tab):
    ctx, disc, fl = tg2d_pair()
    ctx.set_tableau_named(tab)
    v0 = fl.initial(disc.X).reshape(2, -1)
    run_steps(ctx, disc, lambda v, t, dt: ns.rk_step(disc, tab, v, t, dt)[0], v0, 0.0, 0.01, 3, 1e-11)


@pytest.mark.parametrize("precision,tol", [(imex.FP64, 1e-11), (imex.MIXED, 1e-9)])
def test_rk_step_jacobi_pressure(precision, tol):
    """Alg. 3 with Jacobi-preconditioned pressure solves (the default is p-multigrid)."""
    ctx, disc, fl = tg2d_pair(precision=precision, tol=1e-14 if precision == imex.FP64 else 1e-12)
    ctx.set_pressure_precond(imex.PRECOND_JACOBI)
    v0 = fl.initial(disc.X).reshape(2, -1)
    run_steps(ctx, disc, lambda v, t, dt: ns.rk_step(disc, "CB3e", v, t, dt)[0], v0, 0.0, 0.01, 2, tol)


def test_rk_step_tg2d_consistent_projection():
    ctx, disc, fl = tg2d_pair(poisson=imex.POISSON_CONSISTENT)
    v0 = fl.initial(disc.X).reshape(2, -1)
    run_steps(ctx, disc, lambda v, t, dt: ns.rk_step(disc, "CB3e", v, t, dt)[0], v0, 0.0, 0.01, 2, 1e-11)


def test_rk_step_tg3d():
    P, n = 3, (3, 2, 2)
    ctx = imex.Context(3, P, n, [0, 0, 0], [TWO_PI] * 3, (1, 1, 1), tol=1e-14, maxit=50000)
    ctx.set_viscosity_const(1.0 / 1600)
    mesh = dg.Mesh(3, P, n, [0, 0, 0], [TWO_PI] * 3, (True, True, True))
    fl = flows.Flow("tg3d", 1.0 / 1600)
    disc = ns.Discretization(mesh, fl)
    ctx.init_flow(imex.FLOW_TG3D, [0.0])
    v0 = fl.initial(disc.X).reshape(3, -1)
    assert rel(ctx.get_velocity(), v0) < 1e-14
    run_steps(ctx, disc, lambda v, t, dt: ns.rk_step(disc, "CB3e", v, t, dt)[0], v0, 0.0, 0.05, 2, 1e-11)


@pytest.mark.parametrize("tab", ["ARS3", "CB3e"])
def test_rk_step_mms_dirichlet_varnu(tab):
    ctx, disc, fl = mms_pair()
    ctx.set_tableau_named(tab)
    v0 = fl.initial(disc.X).reshape(2, -1)
    run_steps(ctx, disc, lambda v, t, dt: ns.rk_step(disc, tab, v, t, dt)[0], v0, 0.0, 2e-3, 2, 1e-11)


@pytest.mark.parametrize("case", ["tg2d", "mms"])
def test_pressure_is_last_stage_potential(case):
    """get_pressure returns the potential psi'' of the last stage projection of Alg. 3
    (mass-weighted mean removed), also when a final projection follows (variable viscosity);
    each stage solve starts from the previous potential scaled to its own time scale, which
    must leave every result unchanged."""
    ctx, disc, fl = tg2d_pair() if case == "tg2d" else mms_pair()
    dt = 0.01 if case == "tg2d" else 2e-3
    v, t = fl.initial(disc.X).reshape(2, -1), 0.0
    for _ in range(2):
        ctx.set_state(t, v)
        ctx.step(dt, 1)
        v, info = ns.rk_step(disc, "CB3e", v, t, dt)
        t += dt
        assert rel(ctx.get_velocity(), v) < 1e-11
        assert rel(ctx.get_pressure(), info["psi"]) < 1e-9


def test_sdc_step_tg2d():
    ctx, disc, fl = tg2d_pair(P=3, n=3)
    ctx.set_sdc(3, 2, "CB3e")
    v0 = fl.initial(disc.X).reshape(2, -1)
    run_steps(ctx, disc, lambda v, t, dt: ns.sdc_step(disc, 3, 2, "CB3e", v, t, dt), v0, 0.0, 0.05, 1, 1e-11)


def test_sdc_euler_step_mms():
    ctx, disc, fl = mms_pair(P=4, n=2)
    ctx.set_sdc(2, 2, "EULER")
    v0 = fl.initial(disc.X).reshape(2, -1)
    run_steps(ctx, disc, lambda v, t, dt: ns.sdc_step(disc, 2, 2, "EULER", v, t, dt), v0, 0.0, 5e-3, 1, 1e-11)


def test_mixed_precision_step():
    ctx, disc, fl = tg2d_pair(precision=imex.MIXED, tol=1e-12)
    v0 = fl.initial(disc.X).reshape(2, -1)
    run_steps(ctx, disc, lambda v, t, dt: ns.rk_step(disc, "CB3e", v, t, dt)[0], v0, 0.0, 0.01, 2, 1e-9)
    assert ctx.stats()["refinements"] > 0


def test_mixed_precision_mms():
    ctx, disc, fl = mms_pair(precision=imex.MIXED, tol=1e-12)
    v0 = fl.initial(disc.X).reshape(2, -1)
    run_steps(ctx, disc, lambda v, t, dt: ns.rk_step(disc, "CB3e", v, t, dt)[0], v0, 0.0, 2e-3, 1, 1e-9)


def test_closed_form_accuracy_config1():
    """2D decaying Taylor-Green on 4x4 quads, P = 4, RK-CB3e, dt = 0.01 to t = 0.2: same
    error against the closed form as the oracle's run."""
    ctx, disc, fl = tg2d_pair(tol=1e-12)
    ctx.init_flow(imex.FLOW_TG2D, [0.01])
    ctx.step(0.01, 20)
    ex = fl.exact(disc.X, ctx.time()).reshape(2, -1)
    err = rel(ctx.get_velocity(), ex)
    assert 1e-4 < err < 5e-3


# ---- failure states (host-side, no GPU fault) ------------------------------------
def test_nan_state_is_unstable():
    ctx, disc, fl = tg2d_pair(P=3, n=2)
    v = fl.initial(disc.X).reshape(2, -1).copy()
    v[0, 3] = np.nan
    ctx.set_state(0.0, v)
    with pytest.raises(imex.ImexError) as e:
        ctx.step(0.01, 1)
    assert e.value.status in (imex.EUNSTABLE, imex.ENOTCONV)


def test_maxit_is_notconv():
    ctx = imex.Context(2, 4, (4, 4), [0, 0], [TWO_PI, TWO_PI], (1, 1), tol=1e-14, maxit=2)
    ctx.set_viscosity_const(0.01)
    ctx.init_flow(imex.FLOW_TG2D, [0.01])
    with pytest.raises(imex.ImexError) as e:
        ctx.step(0.01, 1)
    assert e.value.status == imex.ENOTCONV


def test_invalid_inputs():
    with pytest.raises(imex.ImexError):
        imex.Context(4, 4, (2, 2), [0, 0], [1, 1], (1, 1))
    with pytest.raises(imex.ImexError):
        imex.Context(2, 12, (2, 2), [0, 0], [1, 1], (1, 1))
    ctx = imex.Context(2, 3, (2, 2), [0, 0], [1, 1], (1, 1))
    with pytest.raises(imex.ImexError):                  # a^IM_11 != 0: not CK form
        ctx.set_tableau([0, 1], [[0.5, 0], [0, 1]], [0, 1], [[0, 0], [1, 0]], [1, 0])
    with pytest.raises(imex.ImexError):
        ctx.set_tableau_named("NOPE")
    d = imex.Context(2, 3, (2, 2), [0, 0], [1, 1], (0, 1))
    d.init_flow(imex.FLOW_TGTRAVEL, [0.01])
    with pytest.raises(imex.ImexError):                  # Dirichlet sides need boundary data
        d.step(0.01, 1)


@pytest.mark.parametrize("P,n", [(3, (3, 2, 2)), (5, (2, 3, 2)), (7, (2, 2, 2))])
def test_mixed_precision_tg3d(P, n):
    # 3D periodic: the inner FP32 iterations of the pressure solves run in one persistent launch
    ctx = imex.Context(3, P, n, [0, 0, 0], [TWO_PI] * 3, (1, 1, 1), precision=imex.MIXED, tol=1e-12, maxit=50000)
    ctx.set_viscosity_const(1.0 / 1600)
    mesh = dg.Mesh(3, P, n, [0, 0, 0], [TWO_PI] * 3, (True, True, True))
    fl = flows.Flow("tg3d", 1.0 / 1600)
    disc = ns.Discretization(mesh, fl)
    v0 = fl.initial(disc.X).reshape(3, -1)
    run_steps(ctx, disc, lambda v, t, dt: ns.rk_step(disc, "CB3e", v, t, dt)[0], v0, 0.0, 0.05, 2, 1e-9)
    assert ctx.stats()["refinements"] > 0


@pytest.mark.parametrize("P,n", [(3, (3, 2, 2)), (7, (2, 2, 2))])
def test_mixed_fast_tg3d(P, n):
    # IMEX_MIXED_FAST adds FP32 explicit operators: their rounding (about eps32 times the
    # convective and viscous terms, times dt) measured at 2e-8 .. 5e-8 relative per step here
    ctx = imex.Context(3, P, n, [0, 0, 0], [TWO_PI] * 3, (1, 1, 1), precision=imex.MIXED_FAST, tol=1e-12,
                       maxit=50000)
    ctx.set_viscosity_const(1.0 / 1600)
    mesh = dg.Mesh(3, P, n, [0, 0, 0], [TWO_PI] * 3, (True, True, True))
    fl = flows.Flow("tg3d", 1.0 / 1600)
    disc = ns.Discretization(mesh, fl)
    v0 = fl.initial(disc.X).reshape(3, -1)
    run_steps(ctx, disc, lambda v, t, dt: ns.rk_step(disc, "CB3e", v, t, dt)[0], v0, 0.0, 0.05, 2, 2e-7)


def test_mixed_fast_mms():
    # Dirichlet faces: the penalty terms of A v and of the boundary data cancel in FP32
    # (about 1e-8 relative after one step of 2e-3 here)
    ctx, disc, fl = mms_pair(precision=imex.MIXED_FAST, tol=1e-12)
    v0 = fl.initial(disc.X).reshape(2, -1)
    run_steps(ctx, disc, lambda v, t, dt: ns.rk_step(disc, "CB3e", v, t, dt)[0], v0, 0.0, 2e-3, 1, 2e-7)


def test_persistent_pressure_cg(monkeypatch):
    # the opt-in persistent FP32 pressure CG (one cooperative launch per refinement cycle)
    monkeypatch.setenv("IMEX_PERSIST", "1")
    P, n = 5, (2, 3, 2)
    ctx = imex.Context(3, P, n, [0, 0, 0], [TWO_PI] * 3, (1, 1, 1), precision=imex.MIXED, tol=1e-12, maxit=50000)
    ctx.set_viscosity_const(1.0 / 1600)
    mesh = dg.Mesh(3, P, n, [0, 0, 0], [TWO_PI] * 3, (True, True, True))
    fl = flows.Flow("tg3d", 1.0 / 1600)
    disc = ns.Discretization(mesh, fl)
    v0 = fl.initial(disc.X).reshape(3, -1)
    run_steps(ctx, disc, lambda v, t, dt: ns.rk_step(disc, "CB3e", v, t, dt)[0], v0, 0.0, 0.05, 2, 1e-9)


@pytest.mark.parametrize("case", ["tg3d", "mms"])
def test_mixed_matches_fp64(case):
    # IMEX_MIXED (FP32 inner CG with FP64 refinement, float-float convection) against
    # IMEX_FP64 from the same state: equal to the solver tolerance
    def make(prec):
        if case == "tg3d":
            c = imex.Context(3, 5, (2, 3, 2), [0, 0, 0], [TWO_PI] * 3, (1, 1, 1), precision=prec, tol=1e-13,
                             maxit=50000)
            c.set_viscosity_const(1.0 / 1600)
            c.init_flow(imex.FLOW_TG3D, [0.0])
            return c, 0.05
        c = mms_pair(P=5, n=3, precision=prec, tol=1e-13)[0]
        c.init_flow(imex.FLOW_TGTRAVEL, [0.01], 0.0)
        return c, 2e-3
    (a, dt), (b, _) = make(imex.MIXED), make(imex.FP64)
    a.step(dt, 2)
    b.step(dt, 2)
    assert rel(a.get_velocity(), b.get_velocity()) < 1e-11


@pytest.mark.parametrize("precision", [imex.FP64, imex.MIXED])
def test_viscosity_change_between_steps(precision):
    # the Helmholtz diagonal of a constant viscosity is kept between solves: a context whose
    # viscosity changes between steps must step exactly like a new context with the new one
    def make(nu):
        c = imex.Context(3, 4, (2, 2, 3), [0, 0, 0], [TWO_PI] * 3, (1, 1, 1), precision=precision, tol=1e-13,
                         maxit=50000)
        c.set_viscosity_const(nu)
        c.init_flow(imex.FLOW_TG3D, [0.0])
        return c
    a = make(0.05)
    a.step(0.02, 1)
    v1 = a.get_velocity()
    a.set_viscosity_const(0.2)
    a.set_state(a.time(), v1)
    a.step(0.02, 1)
    b = make(0.2)
    b.set_state(a.time() - 0.02, v1)
    b.step(0.02, 1)
    assert rel(a.get_velocity(), b.get_velocity()) < 1e-11


def test_sdc_cb3e_33_tg3d():
    """SDC-CB3e(3,3) on 4 GLL nodes (Alg. 4 with the RK-CB3e predictor: the SDC method of the
    3D Taylor-Green workload) on a 3D periodic mesh."""
    P, n = 3, (3, 2, 2)
    ctx = imex.Context(3, P, n, [0, 0, 0], [TWO_PI] * 3, (1, 1, 1), tol=1e-14, maxit=50000)
    ctx.set_viscosity_const(1.0 / 1600)
    ctx.set_sdc(3, 3, "CB3e")
    mesh = dg.Mesh(3, P, n, [0, 0, 0], [TWO_PI] * 3, (True, True, True))
    fl = flows.Flow("tg3d", 1.0 / 1600)
    disc = ns.Discretization(mesh, fl)
    v0 = fl.initial(disc.X).reshape(3, -1)
    run_steps(ctx, disc, lambda v, t, dt: ns.sdc_step(disc, 3, 3, "CB3e", v, t, dt), v0, 0.0, 0.05, 1, 1e-11)
    assert ctx.stats()["stages"] == 18


@pytest.mark.parametrize("tab", ["CB3e", "ARS3"])
def test_rk_step_velocity_dependent_viscosity(tab):
    """Alg. 3 with nu = nu_0 + nu_1 (|v| / v_max)^2 (the law of Sec. 4.2): the viscosity of
    each stage follows from the projected velocity, and the final projection applies."""
    nu0, nu1, vmax = 0.01, 0.05, 1.0
    ctx = imex.Context(2, 4, (4, 4), [0, 0], [TWO_PI, TWO_PI], (1, 1), tol=1e-14, maxit=50000)
    ctx.set_viscosity_model(imex.NU_VELOCITY, [nu0, nu1, vmax])
    ctx.set_tableau_named(tab)
    mesh = dg.Mesh(2, 4, (4, 4), [0, 0], [TWO_PI, TWO_PI], (True, True))
    fl = flows.Flow("tg2d", nu0, nu_kind="velocity", nu1=nu1, vmax=vmax)
    disc = ns.Discretization(mesh, fl)
    v0 = fl.initial(disc.X).reshape(2, -1)
    run_steps(ctx, disc, lambda v, t, dt: ns.rk_step(disc, tab, v, t, dt)[0], v0, 0.0, 0.02, 2, 1e-11)


def test_sdc_velocity_dependent_viscosity_3d():
    """Alg. 4 (SDC-Eu(2,2)) with the velocity-dependent viscosity law in 3D."""
    nu0, nu1, vmax = 1e-3, 4e-3, 1.0
    P, n = 3, (2, 2, 3)
    ctx = imex.Context(3, P, n, [0, 0, 0], [TWO_PI] * 3, (1, 1, 1), tol=1e-14, maxit=50000)
    ctx.set_viscosity_model(imex.NU_VELOCITY, [nu0, nu1, vmax])
    ctx.set_sdc(2, 2, "EULER")
    mesh = dg.Mesh(3, P, n, [0, 0, 0], [TWO_PI] * 3, (True, True, True))
    fl = flows.Flow("tg3d", nu0, nu_kind="velocity", nu1=nu1, vmax=vmax)
    disc = ns.Discretization(mesh, fl)
    v0 = fl.initial(disc.X).reshape(3, -1)
    run_steps(ctx, disc, lambda v, t, dt: ns.sdc_step(disc, 2, 2, "EULER", v, t, dt), v0, 0.0, 0.03, 1, 1e-11)


def test_pressure_closed_form_tg2d():
    """imex_get_pressure against the closed-form pressure of the decaying Taylor-Green vortex,
    p = (cos 2x + cos 2y) e^{-4 nu t} / 4: the last stage potential of Alg. 3, divided by the
    stage's time scale c_s dt, approximates p at the stage time to first order in dt (the
    splitting error of the projection), once the spatial error is below it (P = 6, 8^2)."""
    from oracle import tableaux
    P, n, nu = 6, 8, 0.01
    cs = float(tableaux.get("CB3e").as_float()[0][-1])
    mesh = dg.Mesh(2, P, (n, n), [0, 0], [TWO_PI, TWO_PI], (True, True))
    Xp = mesh.node_coords(P)
    Mp = dg.mass_diag(mesh, P)
    errs = []
    for dt in (0.02, 0.01, 0.005):
        ctx = imex.Context(2, P, (n, n), [0, 0], [TWO_PI, TWO_PI], (1, 1), tol=1e-13, maxit=50000)
        ctx.set_viscosity_const(nu)
        ctx.init_flow(imex.FLOW_TG2D, [nu])
        ctx.step(dt, 1)
        q = ctx.get_pressure() / (cs * dt)
        pex = flows.tg2d_pressure(Xp, cs * dt, nu).ravel()
        pex -= np.dot(Mp, pex) / Mp.sum()
        assert abs(np.dot(Mp, q)) < 1e-12 * np.abs(q).max() * Mp.sum()     # mass-weighted mean-free
        errs.append(rel(q, pex))
    assert errs[0] < 1e-3
    for a, b in zip(errs, errs[1:]):
        assert 1.6 < a / b < 2.4, errs
