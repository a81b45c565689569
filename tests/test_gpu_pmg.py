"""GPU parity of the p-multigrid preconditioner of the pressure solves against the oracle
(oracle/pmg.py):

* one V-cycle, element by element, with the same Chebyshev bounds on both sides (taken from
  the oracle's exact eigenvalues): FP64 to 1e-11 relative, FP32 to 1e-5; meshes in 2D and 3D,
  periodic and with Neumann sides, with two and three levels, several blocks and ragged tails;
* the level structure, and the context's own Chebyshev bounds (a power-iteration estimate,
  times 1.15) within [1.03, 1.15] of the exact largest eigenvalue of D^{-1} A on every level;
* Poisson solves preconditioned by the V-cycle equal to the oracle's bordered-LU solution,
  in a handful of iterations, and whole Alg. 3 steps through it equal to the oracle's steps;
* batches of uneven instances preconditioned by the V-cycle equal to the same instances alone.
"""
import numpy as np
import pytest

from oracle import dg, flows, ns, pmg
from tests import inputs

pytestmark = pytest.mark.gpu

imex = pytest.importorskip("paper_2112_04167_gb300.imex")
TWO_PI = 2 * np.pi

CASES = [
    # d, P, nelem, periodic
    (2, 8, (7, 5), (True, True)),          # N 8 -> 4 -> 2
    (2, 5, (4, 3), (False, True)),         # N 5 -> 3 -> 2
    (2, 4, (3, 5), (False, False)),        # N 4 -> 2
    (3, 7, (3, 2, 3), (True, True, True)),  # N 7 -> 4 -> 2
    (3, 6, (2, 3, 2), (False, True, False)),  # N 6 -> 3 -> 2
    (3, 3, (3, 3, 2), (True, False, True)),  # N 3 -> 2
]
LO = [0.1, -0.3, 0.0]
HI = [1.3, 0.9, 2.0]


def rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2112_04167_gb300 import build
    build.build()
    imex.load()


def make(case, **kw):
    d, P, n, per = case
    ctx = imex.Context(d, P, n, LO[:d], HI[:d], per, **kw)
    ctx.set_pressure_precond(imex.PRECOND_PMG)
    return ctx, dg.Mesh(d, P, n, LO[:d], HI[:d], per)


@pytest.fixture(scope="module")
def oracles():
    out = {}
    for case in CASES:
        mesh = dg.Mesh(case[0], case[1], case[2], LO[:case[0]], HI[:case[0]], case[3])
        M = pmg.PMG(mesh, case[1])
        exact = [pmg.largest_eig(A, dv) for A, dv in zip(M.A, M.dinv)]
        out[case] = (M, exact)
    return out


@pytest.mark.parametrize("case", CASES)
def test_vcycle_parity(case, oracles):
    M, _ = oracles[case]
    ctx, _ = make(case)
    N, _ = ctx.pmg_info()
    assert N == M.N
    r = inputs.field(ctx.npres, seed=61)
    ref = M.vcycle(r)
    assert rel(ctx.op_pmg_vcycle(r, lmax=M.lmax), ref) < 1e-11
    assert rel(ctx.op_pmg_vcycle(r, lmax=M.lmax, arith=imex.ARITH_FP32), ref) < 1e-5


@pytest.mark.parametrize("case", [(2, 6, (6, 1), (True, True)), (3, 5, (4, 1, 1), (True, True, True)),
                                  (3, 4, (1, 3, 2), (True, False, True))])
def test_vcycle_single_element_periodic(case):
    """One element across a periodic direction is its own neighbour there: the Jacobi diagonal
    of every level and the V-cycle equal the oracle's (assembled matrix)."""
    d, P, n, per = case
    mesh = dg.Mesh(d, P, n, LO[:d], HI[:d], per)
    M = pmg.PMG(mesh, P)
    ctx, _ = make(case)
    r = inputs.field(ctx.npres, seed=64)
    ref = M.vcycle(r)
    assert rel(ctx.op_pmg_vcycle(r, lmax=M.lmax), ref) < 1e-11
    assert rel(ctx.op_pmg_vcycle(r, lmax=M.lmax, arith=imex.ARITH_FP32), ref) < 1e-5


@pytest.mark.parametrize("n", [(5, 4, 3), (3, 2, 3), (17, 2, 2), (17, 1, 1)])
def test_coarsest_level_on_one_cluster(n, monkeypatch):
    """The FP32 coarsest level (N = 2) of a 3D periodic mesh smoothed in one cluster launch
    (elements split over the CTAs, neighbours across CTAs read from their shared memory)
    gives the oracle's V-cycle and that of one launch per Chebyshev step, with fewer launches
    (meshes with several elements per CTA, idle CTAs, a ragged last CTA)."""
    case = (3, 7, n, (True, True, True))
    mesh = dg.Mesh(3, 7, n, LO, HI, case[3])
    M = pmg.PMG(mesh, 7)
    r = inputs.field(M.A[0].shape[0], seed=63)
    ref = M.vcycle(r)
    out = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("IMEX_PMG_CLUSTER", flag)
        ctx, _ = make(case)
        ctx.op_pmg_vcycle(r, lmax=M.lmax, arith=imex.ARITH_FP32)         # set-up, tuning
        before = imex.launch_count()
        out[flag] = ctx.op_pmg_vcycle(r, lmax=M.lmax, arith=imex.ARITH_FP32)
        out[flag + "n"] = imex.launch_count() - before
    errs = (rel(out["1"], ref), rel(out["0"], ref), rel(out["1"], out["0"]))
    assert max(errs) < 1e-5, errs
    assert out["1n"] < out["0n"]


@pytest.mark.parametrize("case", CASES)
def test_chebyshev_bounds_estimate(case, oracles):
    _, exact = oracles[case]
    ctx, _ = make(case)
    _, lmax = ctx.pmg_info()
    for got, ex in zip(lmax, exact):
        assert 1.03 * ex <= got <= 1.15 * ex + 1e-12, (got, ex)


@pytest.mark.parametrize("precision,tol,bar", [(imex.FP64, 1e-14, 1e-10), (imex.MIXED, 1e-12, 1e-9)])
@pytest.mark.parametrize("case", [CASES[0], CASES[3], CASES[4]])
def test_poisson_solve_pmg(case, precision, tol, bar):
    ctx, mesh = make(case, precision=precision, tol=tol, maxit=5000)
    disc = ns.Discretization(mesh, flows.Flow("tgtravel", 0.01))
    b = inputs.field(ctx.npres, seed=62)
    psi = ctx.solve_poisson(b)
    assert rel(psi, disc.poisson(b.copy())) < bar
    assert ctx.stats()["poisson_iters"] <= 40


@pytest.mark.parametrize("precision,bar", [(imex.FP64, 1e-11), (imex.MIXED, 1e-9)])
def test_rk_steps_tg3d_pmg(precision, bar):
    P, n = 4, (3, 2, 3)
    ctx = imex.Context(3, P, n, [0, 0, 0], [TWO_PI] * 3, (1, 1, 1), precision=precision,
                       tol=1e-14 if precision == imex.FP64 else 1e-12, maxit=50000)
    ctx.set_pressure_precond(imex.PRECOND_PMG)
    ctx.set_viscosity_const(1.0 / 1600)
    mesh = dg.Mesh(3, P, n, [0, 0, 0], [TWO_PI] * 3, (True, True, True))
    fl = flows.Flow("tg3d", 1.0 / 1600)
    disc = ns.Discretization(mesh, fl)
    v, t = fl.initial(disc.X).reshape(3, -1), 0.0
    for _ in range(2):
        ctx.set_state(t, v)
        ctx.step(0.05, 1)
        v = ns.rk_step(disc, "CB3e", v, t, 0.05)[0]
        t += 0.05
        assert rel(ctx.get_velocity(), v) < bar


def test_rk_steps_mms_dirichlet_pmg():
    """Neumann pressure sides, variable viscosity, final projection: Alg. 3 through the V-cycle."""
    P, n = 5, 3
    ctx = imex.Context(2, P, (n, n), [0, 0], [1, 1], (0, 0), tol=1e-14, maxit=50000)
    ctx.set_pressure_precond(imex.PRECOND_PMG)
    ctx.set_viscosity_model(imex.NU_VARXYT, [0.01])
    ctx.set_boundary(imex.FLOW_TGTRAVEL, [0.01])
    ctx.set_forcing(imex.FORCE_TGTRAVEL_VARNU, [0.01])
    mesh = dg.Mesh(2, P, (n, n), [0, 0], [1, 1], (False, False))
    fl = flows.Flow("tgtravel", 0.01, nu_kind="varxyt")
    disc = ns.Discretization(mesh, fl)
    v, t = fl.initial(disc.X).reshape(2, -1), 0.0
    for _ in range(2):
        ctx.set_state(t, v)
        ctx.step(2e-3, 1)
        v = ns.rk_step(disc, "CB3e", v, t, 2e-3)[0]
        t += 2e-3
        assert rel(ctx.get_velocity(), v) < 1e-11


@pytest.mark.parametrize("precision,bar", [(imex.FP64, 1e-10), (imex.MIXED, 1e-7)])
def test_batch_pmg_matches_alone(precision, bar):
    specs = [(4, 3, 0.01), (6, 5, 0.003), (4, 6, 0.05), (6, 2, 0.02), (8, 4, 0.01)]
    tol = 1e-13 if precision == imex.FP64 else 1e-10

    def make_tg(P, n, nu):
        c = imex.Context(2, P, (n, n), [0, 0], [TWO_PI, TWO_PI], (1, 1), precision=precision, tol=tol, maxit=50000)
        c.set_pressure_precond(imex.PRECOND_PMG)
        c.set_viscosity_const(nu)
        c.init_flow(imex.FLOW_TG2D, [nu], 0.0)
        return c
    dts = [0.02, 0.01, 0.015, 0.02, 0.01]
    alone = [make_tg(*s) for s in specs]
    for c, dt in zip(alone, dts):
        c.step(dt, 3)
    batch = imex.Batch([make_tg(*s) for s in specs])
    batch.step(dts, 3)
    for i, c in enumerate(alone):
        assert rel(batch.get_velocity(i), c.get_velocity()) < bar, i
    assert batch.stats()["poisson_iters"] > 0
