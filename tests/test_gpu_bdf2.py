"""GPU parity of IMEX BDF2 (Sec. 3.2.1) against the oracle's step (oracle/ns.py bdf2_step):
consecutive steps from the same initial field -- the first an IMEX Euler step, then the
two-step formula with the extrapolated viscosity -- compared after every step, FP64 to
1e-11 relative L2 (solves to 1e-14), the mixed form to 1e-9; periodic and Dirichlet, constant,
space-time and velocity-dependent viscosity, with forcing, 2D and 3D; a change of the step
size restarts the formula with an Euler step."""
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


def compare(ctx, disc, fl, dts, bar):
    v = fl.initial(disc.X).reshape(disc.d, -1)
    ctx.set_state(0.0, v)
    ctx.set_bdf2()
    prev, t, last_dt = None, 0.0, None
    for dt in dts:
        if dt != last_dt:
            prev = None                   # a new step size restarts with IMEX Euler
        ctx.step(dt, 1)
        v, prev, info = ns.bdf2_step(disc, v, t, dt, prev)
        t += dt
        last_dt = dt
        assert rel(ctx.get_velocity(), v) < bar
    assert ctx.time() == pytest.approx(t, rel=1e-14)
    return info


@pytest.mark.parametrize("precision,tol,bar", [(imex.FP64, 1e-14, 1e-11), (imex.MIXED, 1e-12, 1e-9)])
def test_bdf2_tg2d(precision, tol, bar):
    ctx = imex.Context(2, 5, (3, 4), [0, 0], [TWO_PI, TWO_PI], (1, 1), precision=precision, tol=tol, maxit=50000)
    ctx.set_viscosity_const(0.02)
    mesh = dg.Mesh(2, 5, (3, 4), [0, 0], [TWO_PI, TWO_PI], (True, True))
    fl = flows.Flow("tg2d", 0.02)
    disc = ns.Discretization(mesh, fl)
    info = compare(ctx, disc, fl, [0.02] * 4, bar)
    # the potential of the last projection, (dt / gamma_0) p''
    assert rel(ctx.get_pressure(), info["psi"]) < 1e3 * bar


def test_bdf2_mms_dirichlet_varnu_forcing():
    P, n = 4, 3
    ctx = imex.Context(2, P, (n, n), [0, 0], [1, 1], (0, 0), tol=1e-14, maxit=50000)
    ctx.set_viscosity_model(imex.NU_VARXYT, [0.01])
    ctx.set_boundary(imex.FLOW_TGTRAVEL, [0.01])
    ctx.set_forcing(imex.FORCE_TGTRAVEL_VARNU, [0.01])
    mesh = dg.Mesh(2, P, (n, n), [0, 0], [1, 1], (False, False))
    fl = flows.Flow("tgtravel", 0.01, nu_kind="varxyt")
    compare(ctx, ns.Discretization(mesh, fl), fl, [2e-3] * 3, 1e-11)


def test_bdf2_velocity_viscosity_3d_and_step_change():
    nu0, nu1, vmax = 1e-3, 4e-3, 1.0
    P, n = 3, (2, 3, 2)
    ctx = imex.Context(3, P, n, [0, 0, 0], [TWO_PI] * 3, (1, 1, 1), tol=1e-14, maxit=50000)
    ctx.set_viscosity_model(imex.NU_VELOCITY, [nu0, nu1, vmax])
    mesh = dg.Mesh(3, P, n, [0, 0, 0], [TWO_PI] * 3, (True, True, True))
    fl = flows.Flow("tg3d", nu0, nu_kind="velocity", nu1=nu1, vmax=vmax)
    compare(ctx, ns.Discretization(mesh, fl), fl, [0.03, 0.03, 0.02, 0.02], 1e-11)


def test_bdf2_rejected_by_batches():
    c = imex.Context(2, 3, (2, 2), [0, 0], [TWO_PI, TWO_PI], (1, 1))
    c.set_viscosity_const(0.01)
    c.set_bdf2()
    with pytest.raises(imex.ImexError):
        imex.Batch([c])
