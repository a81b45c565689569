"""GPU parity of the divergence / mass-flux stabilisation (imex_set_stabilization) against the
oracle (oracle/stab.py): the stabilised projection of random velocities, 2D and 3D, periodic
and bounded (solves to 1e-14: 1e-11 relative), and whole Alg. 3, Alg. 4 and BDF2 steps with
the stabilisation after every stage projection against the oracle's steps (1e-11)."""
import numpy as np
import pytest

from oracle import dg, flows, ns, stab
from tests import inputs

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


@pytest.mark.parametrize("case", [(2, 4, (3, 5), (True, False)), (3, 3, (2, 3, 2), (True, True, False)),
                                  (2, 6, (1, 3), (True, True)), (3, 5, (2, 2, 2), (False, False, False))])
def test_stabilized_projection(case):
    d, P, n, per = case
    lo, hi = [0.1, -0.3, 0.0][:d], [1.3, 0.9, 2.0][:d]
    ctx = imex.Context(d, P, n, lo, hi, per, tol=1e-14, maxit=5000)
    ctx.set_stabilization(1.5, 0.7)
    mesh = dg.Mesh(d, P, n, lo, hi, per)
    v = inputs.field(d * ctx.nvel, seed=81).reshape(d, -1) + 0.4
    got = ctx.stabilize(v, 0.05)
    ref = stab.stabilize(mesh, v, 0.05, 1.5, 0.7)
    assert rel(got, ref) < 1e-11
    assert rel(got, v) > 1e-4                  # the penalty did act


@pytest.mark.parametrize("method", ["rk", "sdc", "bdf2"])
def test_steps_with_stabilization(method):
    P, n = 4, (3, 3)
    ctx = imex.Context(2, P, n, [0, 0], [1, 1], (0, 0), tol=1e-14, maxit=50000)
    ctx.set_viscosity_model(imex.NU_VARXYT, [0.01])
    ctx.set_boundary(imex.FLOW_TGTRAVEL, [0.01])
    ctx.set_forcing(imex.FORCE_TGTRAVEL_VARNU, [0.01])
    ctx.set_stabilization(1.0, 1.0)
    mesh = dg.Mesh(2, P, n, [0, 0], [1, 1], (False, False))
    fl = flows.Flow("tgtravel", 0.01, nu_kind="varxyt")
    disc = ns.Discretization(mesh, fl, stab=(1.0, 1.0))
    v, t, prev, dt = fl.initial(disc.X).reshape(2, -1), 0.0, None, 4e-3
    ctx.set_state(0.0, v)
    if method == "sdc":
        ctx.set_sdc(2, 1, "EULER")
    if method == "bdf2":
        ctx.set_bdf2()
    for _ in range(2):
        ctx.step(dt, 1)
        if method == "rk":
            v, _ = ns.rk_step(disc, "CB3e", v, t, dt)
        elif method == "sdc":
            v = ns.sdc_step(disc, 2, 1, "EULER", v, t, dt)
        else:
            v, prev, _ = ns.bdf2_step(disc, v, t, dt, prev)
        t += dt
        assert rel(ctx.get_velocity(), v) < 1e-11


def test_stabilization_rejected_by_batches():
    c = imex.Context(2, 3, (2, 2), [0, 0], [TWO_PI, TWO_PI], (1, 1))
    c.set_viscosity_const(0.01)
    c.set_stabilization(1.0, 1.0)
    with pytest.raises(imex.ImexError):
        imex.Batch([c])
