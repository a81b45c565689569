"""GPU parity of the flow statistics of Sec. 4.3 (imex_dissipation, imex_energy_spectrum)
against the oracle (oracle/diagnostics.py): the dissipation rate to 1e-12 relative and the
energy spectrum shell by shell to 1e-10 of the total energy, for random fields in 2D and 3D,
periodic and bounded, constant and variable viscosity, and the Taylor-Green closed forms."""
import numpy as np
import pytest

from oracle import dg, diagnostics, flows
from tests import inputs

pytestmark = pytest.mark.gpu

imex = pytest.importorskip("paper_2112_04167_gb300.imex")
TWO_PI = 2 * np.pi


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2112_04167_gb300 import build
    build.build()
    imex.load()


CASES = [(2, 5, (3, 4), (True, True), [0.0, -1.0], [1.5, 1.0]),
         (3, 4, (2, 3, 2), (True, True, True), [0.0, 0.0, 0.0], [TWO_PI] * 3),
         (2, 7, (4, 2), (False, False), [0.0, 0.0], [1.0, 1.0])]


@pytest.mark.parametrize("case", CASES)
def test_dissipation_random_fields(case):
    d, P, n, per, lo, hi = case
    ctx = imex.Context(d, P, n, lo, hi, per)
    mesh = dg.Mesh(d, P, n, lo, hi, per)
    v = inputs.field(d * ctx.nvel, seed=71)
    ctx.set_state(0.0, v)
    ctx.set_viscosity_const(0.013)
    ref = diagnostics.dissipation(mesh, v, 0.013)
    assert abs(ctx.dissipation() - ref) < 1e-12 * ref
    if d == 2:
        ctx.set_viscosity_model(imex.NU_VARXYT, [0.01])
        nu = flows.nu_varxyt(mesh.node_coords(P + 1), 0.0, 0.01).ravel()
        ref = diagnostics.dissipation(mesh, v, nu)
        assert abs(ctx.dissipation() - ref) < 1e-12 * ref


@pytest.mark.parametrize("case,M", [(CASES[0], 16), (CASES[1], 8)])
def test_spectrum_random_fields(case, M):
    d, P, n, per, lo, hi = case
    ctx = imex.Context(d, P, n, lo, hi, per)
    mesh = dg.Mesh(d, P, n, lo, hi, per)
    v = inputs.field(d * ctx.nvel, seed=72)
    ctx.set_state(0.0, v)
    kmax = M
    ref = diagnostics.energy_spectrum(mesh, v, M, kmax)
    got = ctx.energy_spectrum(M, kmax)
    assert np.abs(got - ref).max() < 1e-10 * ref.sum()


def test_taylor_green_statistics():
    ctx = imex.Context(3, 7, (4, 4, 4), [0, 0, 0], [TWO_PI] * 3, (1, 1, 1))
    nu = 1.0 / 1600
    ctx.set_viscosity_const(nu)
    ctx.init_flow(imex.FLOW_TG3D, [0.0])
    assert abs(ctx.dissipation() - 0.75 * nu) < 1e-5 * 0.75 * nu
    E = ctx.energy_spectrum(32, 8)
    assert abs(E[2] - np.pi ** 3) < 1e-5 * np.pi ** 3
    assert np.abs(np.delete(E, 2)).max() < 1e-5 * np.pi ** 3


def test_statistics_reject_bad_arguments():
    ctx = imex.Context(2, 3, (2, 2), [0, 0], [1, 1], (1, 1))
    with pytest.raises(imex.ImexError):
        ctx.energy_spectrum(12, 4)          # not a power of two
