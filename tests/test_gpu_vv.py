"""GPU parity of the 3D vortex-array flows of Sec. 4.2 (VVP periodic, VVD with time-dependent
Dirichlet data v_b = v_ex) with the velocity-dependent viscosity nu = nu_0 + nu_1 (|v| / v_max)^2
and the forcing of Eq. (var-visc-test:rhs): the closed-form fields evaluated on the device
against the oracle, and whole steps of Alg. 3 and of IMEX BDF2 (final projection every step,
as the viscosity varies) against the oracle's steps, FP64 to 1e-11 relative L2."""
import numpy as np
import pytest

from oracle import dg, flows, ns

pytestmark = pytest.mark.gpu

imex = pytest.importorskip("paper_2112_04167_gb300.imex")
NU0, NU1, VMAX = 0.01, 0.01, 2.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2112_04167_gb300 import build
    build.build()
    imex.load()


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def pair(periodic, P=3, n=(2, 2, 2), precision=imex.FP64, tol=1e-14):
    per = (1, 1, 1) if periodic else (0, 0, 0)
    ctx = imex.Context(3, P, n, [-0.5] * 3, [0.5] * 3, per, precision=precision, tol=tol, maxit=50000)
    ctx.set_viscosity_model(imex.NU_VELOCITY, [NU0, NU1, VMAX])
    ctx.set_forcing(imex.FORCE_VV, [NU0, NU1, VMAX])
    if not periodic:
        ctx.set_boundary(imex.FLOW_VV)
    mesh = dg.Mesh(3, P, n, [-0.5] * 3, [0.5] * 3, (bool(periodic),) * 3)
    fl = flows.Flow("vv", NU0, nu_kind="velocity", nu1=NU1, vmax=VMAX)
    return ctx, ns.Discretization(mesh, fl), fl


def test_vv_fields():
    ctx, disc, fl = pair(True, P=4, n=(2, 3, 2))
    X = disc.X
    got = ctx.eval_field(0, imex.FLOW_VV, (), t=0.3)
    assert np.abs(got - flows.vv_velocity(X, 0.3).reshape(3, -1)).max() < 1e-14
    got = ctx.eval_field(2, imex.FORCE_VV, [NU0, NU1, VMAX], t=0.3)
    ref = flows.forcing_vv(X, 0.3, NU0, NU1, VMAX).reshape(3, -1)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("periodic", [True, False])
def test_vv_rk_steps(periodic):
    ctx, disc, fl = pair(periodic)
    ctx.set_tableau_named("ARS3")
    v, t = fl.initial(disc.X).reshape(3, -1), 0.0
    ctx.set_state(0.0, v)
    for _ in range(2):
        ctx.step(0.01, 1)
        v, _ = ns.rk_step(disc, "ARS3", v, t, 0.01)
        t += 0.01
        assert rel(ctx.get_velocity(), v) < 1e-11
    # the discrete solution follows the exact vortex array (spatial error of the 2^3 mesh)
    assert rel(v, fl.exact(disc.X, t).reshape(3, -1)) < 0.2


def test_vv_bdf2_dirichlet():
    ctx, disc, fl = pair(False)
    v, t, prev = fl.initial(disc.X).reshape(3, -1), 0.0, None
    ctx.set_state(0.0, v)
    ctx.set_bdf2()
    for _ in range(3):
        ctx.step(0.01, 1)
        v, prev, _ = ns.bdf2_step(disc, v, t, 0.01, prev)
        t += 0.01
        assert rel(ctx.get_velocity(), v) < 1e-11
