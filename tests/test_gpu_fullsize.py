"""Parity at the benchmark's full size (3D Taylor-Green, 16^3 hexahedra, P = 7, the
configuration bench.py times), on sampled outputs the oracle can compute one by one.

The operators are element-local with face coupling to the six neighbours, and the mesh is
uniform and periodic, so the output on an element of the 16^3 mesh equals the output on the
centre element of a periodic 3^3 mesh with the same element size holding the same 27
element fields (its neighbours are the same elements, none wrapped).  The oracle assembles
that 3^3 problem; the GPU runs the full mesh.  A whole step is checked by a property that
holds at any size: the mixed form equals the FP64 form to the solver tolerance."""
import numpy as np
import pytest

from oracle import dg
from tests import inputs

pytestmark = pytest.mark.gpu

imex = pytest.importorskip("paper_2112_04167_gb300.imex")
TWO_PI = 2 * np.pi
NE, P = 16, 7


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2112_04167_gb300 import build
    build.build()
    imex.load()


@pytest.fixture(scope="module")
def full():
    return imex.Context(3, P, (NE, NE, NE), [0, 0, 0], [TWO_PI] * 3, (1, 1, 1), tol=1e-10, maxit=20000)


def patch_indices(ec, n=NE):
    """Elements of the 3x3x3 patch around element coordinates ec, in the 3^3 mesh's order."""
    out = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                x, y, z = (ec[0] + dx) % n, (ec[1] + dy) % n, (ec[2] + dz) % n
                out.append(x + n * (y + n * z))
    return out


@pytest.fixture(scope="module")
def local_ops():
    h = TWO_PI / NE
    mesh3 = dg.Mesh(3, P, (3, 3, 3), [0, 0, 0], [3 * h] * 3, (True, True, True))
    return mesh3, dg.sipg_matrix(mesh3, P, 1.0, dirichlet=False), dg.Convection(mesh3)


SAMPLES = [(0, 0, 0), (15, 7, 3), (8, 15, 0), (4, 9, 12), (15, 15, 15)]


@pytest.mark.parametrize("precision,tol", [(imex.FP64, 1e-12), (imex.MIXED, 1e-5)])
def test_pressure_apply_sampled(full, local_ops, precision, tol):
    mesh3, L3, _ = local_ops
    ndp = P ** 3
    x = inputs.field(full.npres, seed=31)
    y = full.op_sipg(x, space=imex.SPACE_PRESSURE, precision=precision)
    xs, ys = x.reshape(-1, ndp), y.reshape(-1, ndp)
    for ec in SAMPLES:
        idx = patch_indices(ec)
        ref = (L3 @ xs[idx].ravel()).reshape(27, ndp)[13]       # the centre element
        got = ys[idx[13]]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol, ec


@pytest.mark.parametrize("precision,tol", [(imex.FP64, 1e-12), (imex.ARITH_FF, 1e-12), (imex.ARITH_FP32, 1e-5)])
def test_velocity_helmholtz_apply_sampled(full, local_ops, precision, tol):
    """The velocity operator of the Helmholtz solves, M + gamma nu A (N = P + 1 = 8), for the
    three velocity components at once, in each arithmetic the solves use."""
    mesh3 = local_ops[0]
    nu, gamma = 1.0 / 1600, 0.01
    full.set_viscosity_const(nu)
    A3 = dg.sipg_matrix(mesh3, P + 1, nu, dirichlet=True)
    M3 = dg.mass_diag(mesh3, P + 1)
    ndv = (P + 1) ** 3
    x = inputs.field(3 * full.nvel, seed=33)
    y = full.op_sipg(x, nsys=3, alpha=1.0, beta=gamma, precision=precision).reshape(3, -1, ndv)
    xs = x.reshape(3, -1, ndv)
    for ec in SAMPLES:
        idx = patch_indices(ec)
        for c in range(3):
            xp = xs[c, idx].ravel()
            ref = (M3 * xp + gamma * (A3 @ xp)).reshape(27, ndv)[13]
            got = y[c, idx[13]]
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol, (ec, c)


def test_convection_sampled(full, local_ops):
    _, _, conv3 = local_ops
    ndv = (P + 1) ** 3
    v = inputs.field(3 * full.nvel, seed=32)
    y = full.op_conv(v).reshape(3, -1, ndv)
    vs = v.reshape(3, -1, ndv)
    for ec in SAMPLES:
        idx = patch_indices(ec)
        ref = conv3(vs[:, idx].reshape(-1), None).reshape(3, 27, ndv)[:, 13]
        got = y[:, idx[13]]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12, ec


def test_fullsize_step_mixed_equals_fp64():
    def run(prec):
        c = imex.Context(3, P, (NE, NE, NE), [0, 0, 0], [TWO_PI] * 3, (1, 1, 1), precision=prec, tol=1e-10,
                         maxit=20000)
        c.set_viscosity_const(1.0 / 1600)
        c.set_tableau_named("CB3e")
        c.init_flow(imex.FLOW_TG3D, [0.0])
        c.step(0.01, 1)
        return c.get_velocity(), c.stats()
    vm, sm = run(imex.MIXED)
    v64, _ = run(imex.FP64)
    assert np.linalg.norm(vm - v64) / np.linalg.norm(v64) < 1e-10
    assert sm["max_poisson_res"] <= 1e-10 and sm["refinements"] > 0
    # the flow stays bounded by its initial maximum (decaying vortex at this time)
    assert np.abs(vm).max() <= 1.0 + 1e-6
