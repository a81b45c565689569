"""GPU parity of the batched form: many uneven instances advanced together (one union mesh
per (d, P, ...) group, per-instance viscosity, time step and time) give the same fields as
each instance stepped alone, and an instance inside a batch matches the oracle's steps.

Alone and batched runs differ only in the order of the CG reductions (a fused operator dot
alone, per-segment dots in a batch), so with solves converged to 1e-13 the fields agree to
1e-10 relative in FP64; in the mixed form (FP32 inner iterations, FP64 refinement to 1e-10)
to 1e-7."""
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


def tg2d(P, n, nu, precision=imex.FP64, tol=1e-13):
    ctx = imex.Context(2, P, (n, n), [0, 0], [TWO_PI, TWO_PI], (1, 1), precision=precision, tol=tol, maxit=50000)
    ctx.set_viscosity_const(nu)
    ctx.init_flow(imex.FLOW_TG2D, [nu], 0.0)
    return ctx


def tg3d(P, n, nu, precision=imex.FP64, tol=1e-13):
    ctx = imex.Context(3, P, (n, n, n), [0, 0, 0], [TWO_PI] * 3, (1, 1, 1), precision=precision, tol=tol,
                       maxit=50000)
    ctx.set_viscosity_const(nu)
    ctx.init_flow(imex.FLOW_TG3D, [0.0], 0.0)
    return ctx


def mms(P, n, nu0, precision=imex.FP64, tol=1e-13):
    ctx = imex.Context(2, P, (n, n), [0, 0], [1, 1], (0, 0), precision=precision, tol=tol, maxit=50000)
    ctx.set_viscosity_model(imex.NU_VARXYT, [nu0])
    ctx.set_boundary(imex.FLOW_TGTRAVEL, [nu0])
    ctx.set_forcing(imex.FORCE_TGTRAVEL_VARNU, [nu0])
    ctx.init_flow(imex.FLOW_TGTRAVEL, [nu0], 0.0)
    return ctx


def alone_vs_batch(make, specs, dts, nsteps, tol):
    alone = [make(*s) for s in specs]
    for c, dt in zip(alone, dts):
        c.step(dt, nsteps)
    batch = imex.Batch([make(*s) for s in specs])
    batch.step(dts, nsteps)
    for i, c in enumerate(alone):
        assert batch.time(i) == pytest.approx(c.time(), rel=1e-15)
        r = rel(batch.get_velocity(i), c.get_velocity())
        assert r < tol, (i, r)
    return batch


def test_batch_tg2d_uneven_fp64():
    # different element counts, viscosities and steps; one P (one group)
    specs = [(4, 3, 0.01), (4, 5, 0.05), (4, 2, 0.002), (4, 7, 0.02)]
    dts = [0.02, 0.011, 0.03, 0.005]
    b = alone_vs_batch(tg2d, specs, dts, 3, 1e-10)
    assert b.groups == 1


def test_batch_mixed_degrees_groups():
    # P differs: one union mesh per degree, groups stepped concurrently
    specs = [(3, 4, 0.01), (5, 3, 0.03), (3, 6, 0.004), (6, 2, 0.02), (5, 5, 0.01)]
    dts = [0.01, 0.02, 0.015, 0.01, 0.005]
    b = alone_vs_batch(tg2d, specs, dts, 2, 1e-10)
    assert b.groups == 3


def test_batch_tg3d_periodic():
    specs = [(3, 2, 1e-3), (3, 3, 2e-3)]
    alone_vs_batch(tg3d, specs, [0.02, 0.01], 2, 1e-10)


def test_batch_dirichlet_variable_viscosity():
    # analytic boundary data, viscosity and forcing evaluated at each instance's own time
    specs = [(4, 3, 0.01), (4, 4, 0.02), (4, 2, 0.005)]
    alone_vs_batch(mms, specs, [0.01, 0.004, 0.02], 3, 1e-10)


def test_batch_mixed_precision():
    specs = [(5, 4, 0.01), (5, 6, 0.002), (5, 3, 0.05)]
    mk = lambda P, n, nu: tg2d(P, n, nu, precision=imex.MIXED, tol=1e-10)   # noqa: E731
    alone_vs_batch(mk, specs, [0.01, 0.02, 0.005], 3, 1e-7)


def test_batch_instance_matches_oracle():
    # the second instance of a batch against the oracle's CB3e steps
    P, n, nu, dt = 4, 4, 0.01, 0.01
    others = [tg2d(4, 3, 0.02), tg2d(4, 5, 0.03)]
    b = imex.Batch([others[0], tg2d(P, n, nu), others[1]])
    mesh = dg.Mesh(2, P, (n, n), [0, 0], [TWO_PI, TWO_PI], (True, True))
    fl = flows.Flow("tg2d", nu)
    disc = ns.Discretization(mesh, fl)
    v = fl.initial(disc.X).reshape(2, -1)
    t = 0.0
    for _ in range(2):
        b.step([0.02, dt, 0.005], 1)
        v = ns.rk_step(disc, "CB3e", v, t, dt)[0]
        t += dt
        assert rel(b.get_velocity(1), v) < 1e-11


def test_batch_rejects_bad_arguments():
    c = tg2d(3, 2, 0.01)
    b = imex.Batch([c])
    with pytest.raises(imex.ImexError):
        b.step([-1.0], 1)
    s = imex.Context(2, 3, (2, 2), [0, 0], [1, 1], (1, 1))
    s.set_sdc(3, 2)
    with pytest.raises(imex.ImexError):
        imex.Batch([s])


def test_batch_edge_cases():
    # one instance alone in a batch equals the context stepped alone; a one-element instance
    # (the element is its own neighbour in both directions) joins a group of larger ones
    a = tg2d(4, 3, 0.01)
    a.step(0.01, 2)
    b = imex.Batch([tg2d(4, 3, 0.01)])
    b.step([0.01], 2)
    assert rel(b.get_velocity(0), a.get_velocity()) < 1e-10
    specs = [(4, 1, 0.01), (4, 4, 0.02)]
    alone_vs_batch(tg2d, specs, [0.01, 0.02], 2, 1e-10)
    # zero steps leave the state unchanged
    c = imex.Batch([tg2d(3, 2, 0.01)])
    v0 = c.get_velocity(0)
    c.step([0.01], 0)
    assert np.array_equal(c.get_velocity(0), v0) and c.time(0) == 0.0
    with pytest.raises(IndexError):
        c.get_velocity(1)
