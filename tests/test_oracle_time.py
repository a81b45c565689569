"""Pins of the oracle's time integrators: tableaux (Table 1, appendix), Table 2,
orders of the IMEX RK and SDC methods on the scalar test equation (Sec. 2)."""
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import scalar, tableaux

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RK_NAMES = ["TR", "CB2", "CB3c", "CB3e", "CB4", "ARS3"]


def _read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.mark.parametrize("name", RK_NAMES + ["EULER"])
def test_ck_structure(name):
    t = tableaux.get(name)
    s = t.s
    assert t.c[0] == 0 and t.AI[0][0] == 0          # CK form, Eq. (imex-rk:butcher)
    for i in range(s):
        # row sums equal the shared nodes; the published rationals of the CB methods
        # are ~12-digit approximations, so compare to 1e-10
        assert float(sum(t.AI[i]) - t.c[i]) == pytest.approx(0.0, abs=1e-10)
        assert float(sum(t.AE[i]) - t.c[i]) == pytest.approx(0.0, abs=1e-10)
        for j in range(i + 1, s):
            assert t.AI[i][j] == 0
        for j in range(i, s):
            assert t.AE[i][j] == 0                   # explicit part strictly lower


def test_table1_properties():
    for name, stages, order, sa, exlast, beq in _read_table("table1_properties.txt"):
        t = tableaux.get(name)
        assert t.s == int(stages)
        assert t.order == int(order)
        if name == "CB3c":
            # Table 1 and the text of Sec. 2.2 say CB3c is not stiffly accurate, but the
            # appendix prints its last implicit row equal to b^IM; the tableau is used as
            # printed (it meets the third-order conditions), so it is SA here.
            assert t.AI[-1] == t.bI and not bool(int(sa))
        else:
            assert (t.AI[-1] == t.bI) == bool(int(sa))
        assert (t.AE[-1] == t.bE) == bool(int(exlast))
        assert (t.bE == t.bI) == bool(int(beq))
        assert t.c[-1] == 1                          # all methods have c_s = 1 (Sec. 2.2)


def _dot(a, b):
    return sum(x * y for x, y in zip(a, b))


def _matvec(A, x):
    return [_dot(r, x) for r in A]


@pytest.mark.parametrize("name", RK_NAMES)
def test_order_conditions(name):
    """Classical and coupling conditions up to order min(order, 3), evaluated in exact
    rationals; the published CB coefficients are ~12-digit rationals, hence the 1e-10."""
    t = tableaux.get(name)
    c = t.c

    def close(x, y):
        return abs(float(x - y)) < 1e-10
    for b in (t.bI, t.bE):
        assert close(sum(b), 1)
        assert close(_dot(b, c), Fr(1, 2))
    if t.order >= 3:
        for b in (t.bI, t.bE):
            assert close(_dot(b, [x * x for x in c]), Fr(1, 3))
            for A in (t.AI, t.AE):
                assert close(_dot(b, _matvec(A, c)), Fr(1, 6))


def test_table2_zim():
    """z_im* of Table 2: computed critical values truncate to the printed digits."""
    for method, printed in _read_table("table2_zim.txt"):
        z = scalar.critical_imag(method)
        assert np.floor(z * 100) / 100 == pytest.approx(float(printed), abs=1e-12), (method, z)


def _eoc(method, lc=1.0j, ld=-1.0, T=1.0, ns=(20, 40)):
    step = scalar.method_step(method)
    errs = []
    for n in ns:
        dt = T / n
        u = 1.0 + 0j
        for _ in range(n):
            u = step(u, dt, lc, ld)
        errs.append(abs(u - np.exp((lc + ld) * T)))
    return np.log(errs[0] / errs[1]) / np.log(ns[1] / ns[0])


@pytest.mark.parametrize("name", RK_NAMES)
def test_rk_order_scalar(name):
    order = tableaux.get(name).order
    assert _eoc(name) == pytest.approx(order, abs=0.25)


@pytest.mark.parametrize("method,order", [("SDC-Eu(3,1)", 2), ("SDC-Eu(3,2)", 3),
                                          ("SDC-Eu(2,5)", 4), ("SDC-CB3e(2,1)", 4)])
def test_sdc_order_scalar(method, order):
    """SDC-Eu(M,K) gains one order per sweep up to 2M (Sec. 2.4)."""
    assert _eoc(method, ns=(8, 16)) == pytest.approx(order, abs=0.3)


def test_sdc_converged_is_lobatto_iiia():
    """Many sweeps converge to the M-stage Lobatto IIIA collocation solution (order 2M)."""
    step = scalar.method_step("SDC-Eu(2,30)")
    u = step(1.0 + 0j, 0.5, 1.0j, -1.0)
    # Lobatto IIIA with 3 nodes (Simpson-type collocation) on y' = l y: R(z) = (1 + z/2 + z^2/12)/(1 - z/2 + z^2/12)
    z = 0.5 * (1.0j - 1.0)
    R = (1 + z / 2 + z * z / 12) / (1 - z / 2 + z * z / 12)
    assert abs(u - R) < 1e-12


def test_substep_counts():
    assert scalar.substeps("CB3e") == 3
    assert scalar.substeps("ARS3") == 4
    assert scalar.substeps("SDC-Eu(3,5)") == 18
    assert scalar.substeps("SDC-CB3e(3,3)") == 18


def test_alg2_matches_alg1_for_constant_nu():
    """Alg. 2 reduces to Alg. 1 when the diffusivity does not depend on u."""
    tab = tableaux.get("ARS3")
    lc, ld = 2.0j, -3.0
    fc = lambda u: lc * u
    u1 = scalar.imex_rk_step(tab, 1.0 + 0j, 0.1, fc, lambda u: ld * u, lambda r, g: r / (1 - g * ld))
    u2 = scalar.semi_implicit_rk_step(tab, 1.0 + 0j, 0.1, fc, lambda nu, u: nu * u, lambda v: ld,
                                      lambda r, g, nu: r / (1 - g * nu))
    assert abs(u1 - u2) < 1e-15


@pytest.mark.parametrize("name,ns", [("ARS3", (20, 40)), ("CB3e", (80, 160))])
def test_alg2_order_nonlinear(name, ns):
    """Alg. 2 keeps third order for a solution-dependent diffusivity (Sec. 2.3).
    CB3e's error constant is small, so its asymptotic range starts at finer steps."""
    tab = tableaux.get(name)
    fc = lambda u: 0.5 * u
    fd = lambda nu, u: -nu * u
    nu_of = lambda u: 1.0 + 0.5 * u * u
    solve = lambda r, g, nu: r / (1 + g * nu)
    ref = None
    errs = []
    for n in (3200,) + ns:
        dt = 1.0 / n
        u = 1.0
        for _ in range(n):
            u = scalar.semi_implicit_rk_step(tab, u, dt, fc, fd, nu_of, solve)
        if ref is None:
            ref = u
        else:
            errs.append(abs(u - ref))
    assert np.log(errs[0] / errs[1]) / np.log(2) == pytest.approx(3.0, abs=0.3)


@pytest.mark.parametrize("name", RK_NAMES + ["EULER"])
def test_stability_function_is_the_partitioned_rk_closed_form(name):
    """On u' = z_E u + z_I u the stages of an additive RK method solve the linear system
    (I - z_E A^EX - z_I A^IM) U = 1 and R = 1 + (z_E b^EX + z_I b^IM)^T U (the textbook
    stability function of a partitioned RK method, here with z_E = i Im z and z_I = Re z as
    Sec. 2.5 assigns them); the stage-by-stage step of Alg. 1 must give the same number."""
    t = tableaux.get(name)
    _, AI, bI, AE, bE = (np.array(a, dtype=float) for a in t.as_float())
    rng = np.random.default_rng(3)
    for _ in range(20):
        z = complex(-3.0 * rng.random(), 4.0 * rng.standard_normal())
        zE, zI = 1j * z.imag, z.real
        U = np.linalg.solve(np.eye(t.s) - zE * AE - zI * AI, np.ones(t.s))
        R = 1 + (zE * bE + zI * bI) @ U
        assert abs(scalar.stability_function("RK-" + name if name != "EULER" else "EULER", z) - R) < 1e-13 * max(1, abs(R))


def test_imex_euler_and_one_node_sdc_closed_form():
    """IMEX Euler: R(x + i y) = (1 + i y) / (1 - x); SDC with one subinterval and no sweep
    is that predictor step."""
    for z in (complex(-0.3, 0.8), complex(-2.0, -1.5), complex(0.0, 3.0)):
        R = (1 + 1j * z.imag) / (1 - z.real)
        assert abs(scalar.stability_function("EULER", z) - R) < 1e-15
        assert abs(scalar.stability_function("SDC-Eu(1,0)", z) - R) < 1e-15


@pytest.mark.parametrize("M", [1, 2, 3, 5])
def test_sdc_nodes_and_subinterval_weights(M):
    """The SDC sub-nodes are the M+1 GLL points mapped to [0, 1] (symmetric, ends included),
    and the weights w_{q,m} integrate every polynomial of degree <= M exactly over each
    subinterval (t_{m-1}, t_m): sum_q w_{q,m} t_q^k = (t_m^{k+1} - t_{m-1}^{k+1}) / (k+1)."""
    tau, W = scalar.sdc_nodes(M)
    assert tau[0] == 0.0 and tau[-1] == 1.0 and np.all(np.diff(tau) > 0)
    assert np.abs(tau + tau[::-1] - 1.0).max() < 1e-14
    for m in range(1, M + 1):
        for k in range(M + 1):
            exact = (tau[m] ** (k + 1) - tau[m - 1] ** (k + 1)) / (k + 1)
            assert abs(W[m] @ tau ** k - exact) < 1e-12   # power-basis rounding at M = 5
    if M == 2:
        # over the whole step the subinterval weights add up to the 3-point GLL weights on
        # [0, 1], Simpson's 1/6, 2/3, 1/6
        assert np.abs(W[1:].sum(axis=0) - np.array([1 / 6, 2 / 3, 1 / 6])).max() < 1e-15
