"""The launch-shape tuner of the periodic constant-viscosity SIPG applies: every shape (the
default elements per block, half and twice as many, one more in 3D FP32 at N = 7, 9) gives the oracle's operator element by
element (FP64 1e-12, FP32 1e-5) in 2D and 3D on meshes with ragged last blocks, and the tuner
records a timed choice for the applies a solve uses, with the solve still equal to the
oracle's."""
import numpy as np
import pytest

from oracle import dg, flows, ns
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


@pytest.mark.parametrize("case", [(2, 6, (7, 5)), (2, 3, (11, 9)), (3, 7, (3, 2, 3)), (3, 4, (3, 3, 2))])
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_every_launch_shape(case, variant):
    d, P, n = case
    lo, hi = [0.1, -0.3, 0.0][:d], [1.3, 0.9, 2.0][:d]
    ctx = imex.Context(d, P, n, lo, hi, (1,) * d)
    mesh = dg.Mesh(d, P, n, lo, hi, (True,) * d)
    ne = int(np.prod(n))
    x = inputs.field(ctx.npres, seed=91)
    L = dg.sipg_matrix(mesh, P, 1.0, dirichlet=False)
    for fp32, tol in ((True, 1e-5), (False, 1e-12)):
        if (d == 2 and not fp32 and variant == 2) or (variant == 3 and (d == 2 or not fp32 or P not in (7, 9))):
            continue
        imex.set_apply_variant(d, P, fp32, ne, variant)
        y = ctx.op_sipg(x, space=imex.SPACE_PRESSURE, precision=imex.ARITH_FP32 if fp32 else imex.ARITH_FP64)
        assert rel(y, L @ x) < tol, (fp32, variant)


def test_tuner_records_and_solve_matches():
    d, P, n = 3, 5, (4, 3, 3)
    ctx = imex.Context(d, P, n, [0, 0, 0], [TWO_PI] * 3, (1, 1, 1), precision=imex.MIXED, tol=1e-12, maxit=5000)
    mesh = dg.Mesh(d, P, n, [0, 0, 0], [TWO_PI] * 3, (True, True, True))
    disc = ns.Discretization(mesh, flows.Flow("tg3d", 0.01))
    b = inputs.field(ctx.npres, seed=92)
    psi = ctx.solve_poisson(b)
    assert rel(psi, disc.poisson(b.copy())) < 1e-9
    tuned = [t for t in imex.tuning_info() if t["d"] == 3 and t["elements"] == 36 and t["fp32"]]
    assert {t["N"] for t in tuned} >= {5, 3, 2}          # the CG apply and the V-cycle levels
    for t in tuned:
        timed = 4 if t["N"] in (7, 9) else 3           # the one-more-element shape: N = 7, 9
        assert t["variant"] in range(timed) and min(t["us"][:timed]) > 0.0
