"""Element-by-element parity of the float-float kernels (FP64 fields, float-float arithmetic on
the FP32 pipes: the FP64-class operators of the IMEX_MIXED form) and of the FP32 convection
(IMEX_MIXED_FAST) against the oracle's assembled matrices and per-element definitions.

Float-float carries about 48 significant bits, so each float-float operator must match the
oracle to 1e-12 relative, the bar of the FP64 kernels; the FP32 convection to 1e-5.  Meshes
span several blocks with a ragged tail, in 2D and 3D, periodic and Dirichlet; the SIPG
float-float kernel exists for the periodic 3D constant-viscosity operator (both spaces)."""
import numpy as np
import pytest

from oracle import dg
from tests import inputs

pytestmark = pytest.mark.gpu

imex = pytest.importorskip("paper_2112_04167_gb300.imex")

CASES = [
    (2, 4, (3, 5), (True, False)),
    (2, 7, (4, 3), (False, False)),
    (3, 3, (3, 2, 3), (True, False, True)),
    (3, 5, (2, 3, 2), (False, True, False)),
    (3, 7, (2, 2, 3), (True, True, True)),
    (2, 8, (7, 5), (True, True)),
]
LO = [0.1, -0.3, 0.0]
HI = [1.3, 0.9, 2.0]
FF = imex.ARITH_FF


def rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def make(case):
    d, P, n, per = case
    return imex.Context(d, P, n, LO[:d], HI[:d], per), dg.Mesh(d, P, n, LO[:d], HI[:d], per)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2112_04167_gb300 import build
    build.build()
    imex.load()


@pytest.mark.parametrize("case", CASES)
def test_convection_ff_and_fp32(case):
    ctx, mesh = make(case)
    d = case[0]
    v = inputs.field(d * ctx.nvel, seed=41)
    vb = inputs.field(d * ctx.nvel, seed=42) if not all(case[3]) else None
    ref = dg.Convection(mesh)(v, vb)
    assert rel(ctx.op_conv(v, vb, arith=FF), ref) < 1e-12
    assert rel(ctx.op_conv(v, vb, arith=imex.ARITH_FP32), ref) < 1e-5


@pytest.mark.parametrize("case", CASES)
def test_div_grad_ff(case):
    ctx, mesh = make(case)
    d, P = case[0], case[1]
    B = dg.div_matrix(mesh, P + 1, P)
    v = inputs.field(d * ctx.nvel, seed=43)
    assert rel(ctx.op_div(v, mode=0, arith=FF), B @ v) < 1e-12
    if not all(case[3]):
        w = inputs.field(d * ctx.nvel, seed=44)
        assert rel(ctx.op_div(v, w=w, mode=1, arith=FF), B @ v - dg.div_boundary_vector(mesh, P + 1, P, w)) < 1e-12
        assert rel(ctx.op_div(v, mode=2, arith=FF), B @ v - dg.div_boundary_vector(mesh, P + 1, P, v)) < 1e-12
    psi = inputs.field(ctx.npres, seed=45)
    ref = (B.T @ psi).reshape(d, -1) / dg.mass_diag(mesh, P + 1)[None, :]
    assert rel(ctx.op_grad(psi, arith=FF), ref) < 1e-12


@pytest.mark.parametrize("case", CASES)
def test_graddiv_ff(case):
    ctx, mesh = make(case)
    d, P = case[0], case[1]
    D = [dg.dg_derivative_matrix(mesh, P + 1, k) for k in range(d)]
    v = inputs.field(d * ctx.nvel, seed=46).reshape(d, -1)
    nu = inputs.positive_field(ctx.nvel, seed=47)
    phi = nu * sum(D[k] @ v[k] for k in range(d))
    fd3_ref = np.stack([-(D[c] @ phi) for c in range(d)])
    fd2_ref = np.zeros_like(fd3_ref)
    for c in range(d):
        for k in range(d):
            fd2_ref[c] += D[k] @ (nu * (D[c] @ v[k]))
    fd3, fd2 = ctx.op_graddiv(v, nu=nu, with_fd2=True, arith=FF)
    assert rel(fd3, fd3_ref) < 1e-12
    assert rel(fd2, fd2_ref) < 1e-12


@pytest.mark.parametrize("case", [(3, 7, (2, 2, 3), (True, True, True)), (3, 3, (3, 2, 3), (True, True, True)),
                                  (3, 5, (2, 3, 2), (True, True, True))])
def test_sipg_ff_periodic_3d(case):
    """Both spaces of the periodic 3D constant-viscosity float-float apply: the residual
    checks of the mixed solves (pressure N = P, velocity N = P + 1 with alpha M + beta A)."""
    ctx, mesh = make(case)
    P = case[1]
    xp = inputs.field(ctx.npres, seed=48)
    L = dg.sipg_matrix(mesh, P, 1.0, dirichlet=False)
    assert rel(ctx.op_sipg(xp, space=imex.SPACE_PRESSURE, precision=FF), L @ xp) < 1e-12
    ctx.set_viscosity_const(0.013)
    n = ctx.nvel
    xv = inputs.field(3 * n, seed=49)
    A = dg.sipg_matrix(mesh, P + 1, 0.013, dirichlet=True)
    M = dg.mass_diag(mesh, P + 1)
    y = ctx.op_sipg(xv, nsys=3, alpha=1.0, beta=0.03, precision=FF)
    for s in range(3):
        xs = xv[s * n:(s + 1) * n]
        assert rel(y[s * n:(s + 1) * n], M * xs + 0.03 * (A @ xs)) < 1e-12
    y = ctx.op_sipg(xv[:n], alpha=0.0, beta=-1.0, minv=1, precision=FF)
    assert rel(y, -(A @ xv[:n]) / M) < 1e-12


def test_sipg_ff_rejects_unsupported():
    ctx, _ = make(CASES[0])
    with pytest.raises(imex.ImexError):
        ctx.op_sipg(np.zeros(ctx.nvel), precision=FF)
    with pytest.raises(imex.ImexError):
        ctx.op_div(np.zeros(2 * ctx.nvel), arith=7)
