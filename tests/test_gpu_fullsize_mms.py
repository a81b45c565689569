"""Parity at the full size of the 2D manufactured-solution configuration (unit square, 32^2
quadrilaterals, P = 8, time-dependent Dirichlet data on all sides, nodal variable
viscosity), on sampled elements the oracle computes one by one.

The operators couple an element to its face neighbours only, so the output on an element of
the 32^2 mesh equals the output on the same element of the patch of its neighbours (3 x 3,
clipped at the domain boundary, where the patch keeps the domain's Dirichlet sides) holding
the same element fields: the oracle assembles the patch, the GPU runs the whole mesh."""
import numpy as np
import pytest

from oracle import dg
from tests import inputs

pytestmark = pytest.mark.gpu

imex = pytest.importorskip("paper_2112_04167_gb300.imex")
NE, P = 32, 8
N = P + 1
H = 1.0 / NE


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2112_04167_gb300 import build
    build.build()
    imex.load()


@pytest.fixture(scope="module")
def full():
    return imex.Context(2, P, (NE, NE), [0, 0], [1, 1], (0, 0), tol=1e-12, maxit=20000)


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


# interior, corner, edge and near-edge elements (x, y)
SAMPLES = [(0, 0), (31, 31), (0, 17), (15, 16), (31, 5), (7, 0), (30, 1)]


def patch(ec):
    """Element range of the clipped neighbour patch, its mesh, the full-mesh indices of its
    elements (x fastest, as in the library) and the position of ec in it."""
    x0, x1 = max(ec[0] - 1, 0), min(ec[0] + 1, NE - 1)
    y0, y1 = max(ec[1] - 1, 0), min(ec[1] + 1, NE - 1)
    nx, ny = x1 - x0 + 1, y1 - y0 + 1
    mesh = dg.Mesh(2, P, (nx, ny), [x0 * H, y0 * H], [(x1 + 1) * H, (y1 + 1) * H], (False, False))
    idx = [x + NE * y for y in range(y0, y1 + 1) for x in range(x0, x1 + 1)]
    centre = (ec[0] - x0) + nx * (ec[1] - y0)
    return mesh, idx, centre


def comps(a, d):
    return a.reshape(d, NE * NE, -1)


@pytest.mark.parametrize("precision,tol", [(imex.FP64, 1e-12), (imex.MIXED, 1e-5)])
def test_sipg_velocity_sampled(full, precision, tol):
    nv = full.nvel
    x = inputs.field(nv, seed=41)
    nu = inputs.positive_field(nv, seed=42)
    g = inputs.field(nv, seed=43)
    y = full.op_sipg(x, alpha=0.7, beta=1.3, nu=nu, g=g, precision=precision)
    xs, nus, gs, ys = (a.reshape(NE * NE, -1) for a in (x, nu, g, y))
    for ec in SAMPLES:
        mesh, idx, c = patch(ec)
        xp, nup, gp = xs[idx].ravel(), nus[idx].ravel(), gs[idx].ravel()
        ref = 0.7 * dg.mass_diag(mesh, N) * xp + 1.3 * (dg.sipg_matrix(mesh, N, nup, dirichlet=True) @ xp -
                                                        dg.sipg_dirichlet_rhs(mesh, N, nup, gp))
        ref = ref.reshape(len(idx), -1)[c]
        assert rel(ys[idx[c]], ref) < tol, ec


def test_sipg_pressure_sampled(full):
    x = inputs.field(full.npres, seed=44)
    y = full.op_sipg(x, space=imex.SPACE_PRESSURE)
    xs, ys = x.reshape(NE * NE, -1), y.reshape(NE * NE, -1)
    for ec in SAMPLES:
        mesh, idx, c = patch(ec)
        ref = (dg.sipg_matrix(mesh, P, 1.0, dirichlet=False) @ xs[idx].ravel()).reshape(len(idx), -1)[c]
        assert rel(ys[idx[c]], ref) < 1e-12, ec


def test_convection_sampled(full):
    v = inputs.field(2 * full.nvel, seed=45)
    vb = inputs.field(2 * full.nvel, seed=46)
    y = comps(full.op_conv(v, vb), 2)
    vs, vbs = comps(v, 2), comps(vb, 2)
    for ec in SAMPLES:
        mesh, idx, c = patch(ec)
        ref = dg.Convection(mesh)(vs[:, idx].ravel(), vbs[:, idx].ravel()).reshape(2, len(idx), -1)[:, c]
        assert rel(y[:, idx[c]], ref) < 1e-12, ec


def test_divergence_and_gradient_sampled(full):
    v = inputs.field(2 * full.nvel, seed=47)
    w = inputs.field(2 * full.nvel, seed=48)
    psi = inputs.field(full.npres, seed=49)
    b = full.op_div(v, w=w, mode=1).reshape(NE * NE, -1)
    gr = comps(full.op_grad(psi), 2)
    vs, ws, ps = comps(v, 2), comps(w, 2), psi.reshape(NE * NE, -1)
    for ec in SAMPLES:
        mesh, idx, c = patch(ec)
        B = dg.div_matrix(mesh, N, P)
        vp, wp = vs[:, idx].ravel(), ws[:, idx].ravel()
        ref_b = (B @ vp - dg.div_boundary_vector(mesh, N, P, wp)).reshape(len(idx), -1)[c]
        assert rel(b[idx[c]], ref_b) < 1e-12, ec
        Mv = dg.mass_diag(mesh, N)
        ref_g = ((B.T @ ps[idx].ravel()).reshape(2, -1) / Mv[None, :]).reshape(2, len(idx), -1)[:, c]
        assert rel(gr[:, idx[c]], ref_g) < 1e-12, ec
