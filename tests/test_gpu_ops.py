"""GPU parity of every operator of the CUDA path against the oracle's assembled
matrices and per-element definitions, element by element (FP64 to 1e-12 relative;
FP32 kernels to 1e-5), on meshes that span several thread blocks and end in a
ragged tail, in 2D and 3D, periodic and Dirichlet."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import dg, flows, ns
from tests import inputs

pytestmark = pytest.mark.gpu

imex = pytest.importorskip("paper_2112_04167_gb300.imex")

CASES = [
    # d, P, nelem, periodic
    (2, 4, (3, 5), (True, False)),
    (2, 7, (4, 3), (False, False)),
    (2, 3, (2, 2), (True, True)),
    (3, 3, (3, 2, 3), (True, False, True)),
    (3, 5, (2, 3, 2), (False, True, False)),
    (3, 7, (2, 2, 3), (True, True, True)),
    (2, 8, (7, 5), (True, True)),      # 2D periodic line-owner path: several blocks and a ragged tail
]
LO = [0.1, -0.3, 0.0]
HI = [1.3, 0.9, 2.0]


def rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def make(case, **kw):
    d, P, n, per = case
    ctx = imex.Context(d, P, n, LO[:d], HI[:d], per, **kw)
    mesh = dg.Mesh(d, P, n, LO[:d], HI[:d], per)
    return ctx, mesh


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2112_04167_gb300 import build
    build.build()
    imex.load()


@pytest.mark.parametrize("case", CASES)
def test_sipg_velocity(case):
    ctx, mesh = make(case)
    d, P = case[0], case[1]
    N = P + 1
    n = ctx.nvel
    x = inputs.field(2 * n, seed=1)
    nu = inputs.positive_field(n, seed=2)
    g = inputs.field(2 * n, seed=3)
    A = dg.sipg_matrix(mesh, N, nu, dirichlet=True)
    M = dg.mass_diag(mesh, N)
    # alpha M x + beta (A x - r_b(g)) for two systems sharing nu
    y = ctx.op_sipg(x, nsys=2, alpha=0.7, beta=1.3, nu=nu, g=g)
    for s in range(2):
        xs, gs = x[s * n:(s + 1) * n], g[s * n:(s + 1) * n]
        ref = 0.7 * M * xs + 1.3 * (A @ xs - dg.sipg_dirichlet_rhs(mesh, N, nu, gs))
        assert rel(y[s * n:(s + 1) * n], ref) < 1e-12
    # constant viscosity of the context, M^{-1} scaling, homogeneous data
    ctx.set_viscosity_const(0.37)
    y = ctx.op_sipg(x[:n], alpha=0.0, beta=-1.0, minv=1)
    ref = -(dg.sipg_matrix(mesh, N, 0.37, dirichlet=True) @ x[:n]) / M
    assert rel(y, ref) < 1e-12


@pytest.mark.parametrize("case", CASES)
def test_sipg_pressure_and_diag(case):
    ctx, mesh = make(case)
    P = case[1]
    x = inputs.field(ctx.npres, seed=4)
    L = dg.sipg_matrix(mesh, P, 1.0, dirichlet=False)
    assert rel(ctx.op_sipg(x, space=imex.SPACE_PRESSURE), L @ x) < 1e-12
    assert rel(ctx.op_sipg_diag(space=imex.SPACE_PRESSURE), L.diagonal()) < 1e-12
    nu = inputs.positive_field(ctx.nvel, seed=5)
    A = dg.sipg_matrix(mesh, P + 1, nu, dirichlet=True)
    M = dg.mass_diag(mesh, P + 1)
    if min(case[2]) >= 2:
        got = ctx.op_sipg_diag(alpha=2.0, beta=0.5, nu=nu)
        assert rel(got, 2.0 * M + 0.5 * A.diagonal()) < 1e-12


def test_sipg_brute_force_columns():
    """GPU apply on unit vectors reproduces every column of the oracle's matrix (2 elements)."""
    case = (2, 3, (2, 1), (False, True))
    ctx, mesh = make(case)
    N = 4
    nu = inputs.positive_field(ctx.nvel, seed=6)
    A = dg.sipg_matrix(mesh, N, nu, dirichlet=True).toarray()
    for j in range(ctx.nvel):
        e = np.zeros(ctx.nvel)
        e[j] = 1.0
        col = ctx.op_sipg(e, nu=nu)
        assert np.abs(col - A[:, j]).max() < 1e-12 * np.abs(A).max()


@pytest.mark.parametrize("case", CASES)
def test_sipg_fp32(case):
    ctx, mesh = make(case)
    N = case[1] + 1
    n = ctx.nvel
    x = inputs.field(n, seed=7)
    nu = inputs.positive_field(n, seed=8)
    A = dg.sipg_matrix(mesh, N, nu, dirichlet=True)
    M = dg.mass_diag(mesh, N)
    y = ctx.op_sipg(x, alpha=1.0, beta=0.01, nu=nu, precision=imex.MIXED)
    assert rel(y, M * x + 0.01 * (A @ x)) < 1e-5


@pytest.mark.parametrize("case", CASES)
def test_div_grad(case):
    ctx, mesh = make(case)
    d, P = case[0], case[1]
    Nv, Np = P + 1, P
    B = dg.div_matrix(mesh, Nv, Np)
    v = inputs.field(d * ctx.nvel, seed=9)
    w = inputs.field(d * ctx.nvel, seed=10)
    assert rel(ctx.op_div(v, mode=0), B @ v) < 1e-12
    if not all(case[3]):
        ref1 = B @ v - dg.div_boundary_vector(mesh, Nv, Np, w)
        assert rel(ctx.op_div(v, w=w, mode=1), ref1) < 1e-12
        ref2 = B @ v - dg.div_boundary_vector(mesh, Nv, Np, v)
        assert rel(ctx.op_div(v, mode=2), ref2) < 1e-12
    psi = inputs.field(ctx.npres, seed=11)
    Mv = dg.mass_diag(mesh, Nv)
    ref = (B.T @ psi).reshape(d, -1) / Mv[None, :]
    assert rel(ctx.op_grad(psi), ref) < 1e-12


@pytest.mark.parametrize("case", CASES)
def test_convection(case):
    ctx, mesh = make(case)
    d = case[0]
    v = inputs.field(d * ctx.nvel, seed=12)
    vb = inputs.field(d * ctx.nvel, seed=13)
    ref = dg.Convection(mesh)(v, vb)
    assert rel(ctx.op_conv(v, vb if not all(case[3]) else None), ref) < 1e-12


@pytest.mark.parametrize("case", CASES)
def test_graddiv(case):
    ctx, mesh = make(case)
    d, P = case[0], case[1]
    fl = flows.Flow("tgtravel", 0.01)
    disc_D = [dg.dg_derivative_matrix(mesh, P + 1, k) for k in range(d)]
    v = inputs.field(d * ctx.nvel, seed=14).reshape(d, -1)
    nu = inputs.positive_field(ctx.nvel, seed=15)
    phi = nu * sum(disc_D[k] @ v[k] for k in range(d))
    fd3_ref = np.stack([-(disc_D[c] @ phi) for c in range(d)])
    fd2_ref = np.zeros_like(fd3_ref)
    for c in range(d):
        for k in range(d):
            fd2_ref[c] += disc_D[k] @ (nu * (disc_D[c] @ v[k]))
    fd3, fd2 = ctx.op_graddiv(v, nu=nu, with_fd2=True)
    assert rel(fd3, fd3_ref) < 1e-12
    assert rel(fd2, fd2_ref) < 1e-12
    del fl


@pytest.mark.parametrize("precond", [imex.PRECOND_JACOBI, imex.PRECOND_PMG])
@pytest.mark.parametrize("mode", [imex.POISSON_SIPG, imex.POISSON_CONSISTENT])
@pytest.mark.parametrize("case", [CASES[0], CASES[3], CASES[2]])
def test_poisson_solve(case, mode, precond):
    ctx, mesh = make(case, poisson=mode, tol=1e-14, maxit=20000)
    ctx.set_pressure_precond(precond)
    d, P = case[0], case[1]
    fl = flows.Flow("tgtravel", 0.01)
    disc = ns.Discretization(mesh, fl, poisson="sipg" if mode == imex.POISSON_SIPG else "consistent")
    b = inputs.field(ctx.npres, seed=16)
    psi = ctx.solve_poisson(b)
    ref = disc.poisson(b.copy())
    assert rel(psi, ref) < 1e-10


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[4]])
def test_helmholtz_solve(case):
    ctx, mesh = make(case, tol=1e-14, maxit=20000)
    d, P = case[0], case[1]
    fl = flows.Flow("tgtravel", 0.01, nu_kind="varxyt")
    disc = ns.Discretization(mesh, fl)
    g = inputs.field(d * ctx.nvel, seed=17).reshape(d, -1)
    nu = inputs.positive_field(ctx.nvel, seed=18, lo=0.005, hi=0.02)
    vb = inputs.field(d * ctx.nvel, seed=19).reshape(d, -1)
    gamma = 0.05
    got = ctx.solve_helmholtz(g, gamma, nu=nu, vb=vb)
    ref = disc.helmholtz(g, nu, gamma, vb if disc.has_boundary else None)
    assert rel(got, ref) < 1e-11


@pytest.mark.parametrize("case", [CASES[0], CASES[3]])
def test_fields(case):
    ctx, mesh = make(case)
    d = case[0]
    X = mesh.node_coords(case[1] + 1)
    if d == 2:
        got = ctx.eval_field(0, imex.FLOW_TGTRAVEL, [0.02], t=0.3)
        ref = flows.tgtravel_velocity(X, 0.3, 0.02).reshape(d, -1)
        assert np.abs(got - ref).max() < 1e-13
        got = ctx.eval_field(1, imex.NU_VARXYT, [0.01], t=0.7)
        ref = flows.nu_varxyt(X, 0.7, 0.01).ravel()
        assert np.abs(got.ravel() - ref).max() < 1e-15
        got = ctx.eval_field(2, imex.FORCE_TGTRAVEL_VARNU, [0.01], t=0.4)
        ref = flows.forcing_tgtravel_varnu(X, 0.4, 0.01).reshape(d, -1)
        assert np.abs(got - ref).max() < 1e-11
    else:
        got = ctx.eval_field(0, imex.FLOW_TG3D, [0.0], t=0.0)
        ref = flows.tg3d_velocity(X).reshape(d, -1)
        assert np.abs(got - ref).max() < 1e-14
    v = inputs.field(d * ctx.nvel, seed=20)
    got = ctx.eval_field(1, imex.NU_VELOCITY, [0.01, 0.02, 2.0], v=v)
    ref = 0.01 + 0.02 * np.sum(v.reshape(d, -1) ** 2, axis=0) / 4.0
    assert np.abs(got.ravel() - ref).max() < 1e-15


def test_reductions():
    ctx, mesh = make(CASES[3])
    n = ctx.dim * ctx.nvel
    x = inputs.field(n, seed=21)
    y = inputs.field(n, seed=22)
    assert ctx.reduce(imex.REDUCE_DOT, x, y) == pytest.approx(float(np.dot(x, y)), rel=1e-13)
    assert ctx.reduce(imex.REDUCE_SUM, x) == pytest.approx(float(np.sum(x)), rel=1e-12, abs=1e-12)
    assert ctx.reduce(imex.REDUCE_MAXABS, x) == float(np.abs(x).max())
    x[17] = np.nan
    assert np.isnan(ctx.reduce(imex.REDUCE_MAXABS, x))
    with pytest.raises(imex.ImexError):
        ctx.reduce(imex.REDUCE_SUM, np.zeros(n + 1))


@pytest.mark.parametrize("case", [CASES[5], (3, 3, (3, 2, 3), (True, True, True)), (3, 8, (2, 3, 2), (True, True, True))])
def test_sipg_pressure_periodic_fp32(case):
    """The periodic constant-coefficient FP32 kernel (line-owner passes) on the pressure space."""
    ctx, mesh = make(case)
    P = case[1]
    x = inputs.field(ctx.npres, seed=23)
    L = dg.sipg_matrix(mesh, P, 1.0, dirichlet=False)
    M = dg.mass_diag(mesh, P)
    assert rel(ctx.op_sipg(x, space=imex.SPACE_PRESSURE, precision=imex.MIXED), L @ x) < 1e-5
    y = ctx.op_sipg(x, space=imex.SPACE_PRESSURE, alpha=0.3, beta=1.7, minv=1, precision=imex.MIXED)
    assert rel(y, (0.3 * M * x + 1.7 * (L @ x)) / M) < 1e-5


@pytest.mark.parametrize("case", [(3, 2, (3, 2, 2), (True, False, False)), (3, 2, (2, 3, 2), (False, True, True)),
                                  (3, 2, (2, 2, 3), (False, False, False))])
def test_sipg_pressure_two_points_3d(case):
    """P = 2 (pressure degree 1, N = 2 points: four threads per element in the constant-
    viscosity 3D kernel, fewer than the element's six neighbours) with non-periodic sides."""
    ctx, mesh = make(case)
    x = inputs.field(ctx.npres, seed=24)
    L = dg.sipg_matrix(mesh, 2, 1.0, dirichlet=False)
    assert rel(ctx.op_sipg(x, space=imex.SPACE_PRESSURE), L @ x) < 1e-12
    assert rel(ctx.op_sipg(x, space=imex.SPACE_PRESSURE, precision=imex.MIXED), L @ x) < 1e-5
