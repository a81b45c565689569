"""Pins of the oracle's DG-SEM operators (Sec. 3.3 readings) against closed forms,
exact integrals, invariants and hand-computed cases."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import dg, gll


# --------------------------------------------------------------------- basis
def test_gll_closed_forms():
    x, w = gll.gll_nodes_weights(2)
    assert np.allclose(x, [-1, 1]) and np.allclose(w, [1, 1])
    x, w = gll.gll_nodes_weights(3)
    assert np.allclose(x, [-1, 0, 1]) and np.allclose(w, [1 / 3, 4 / 3, 1 / 3])
    x, w = gll.gll_nodes_weights(4)
    r = 1 / np.sqrt(5)
    assert np.allclose(x, [-1, -r, r, 1]) and np.allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6])


@pytest.mark.parametrize("n", [2, 3, 5, 8, 9])
def test_gll_exactness(n):
    x, w = gll.gll_nodes_weights(n)
    p = n - 1
    for k in range(2 * p):                       # exact up to degree 2P-1
        exact = (1 - (-1) ** (k + 1)) / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-13
    k = 2 * p                                    # and not beyond
    assert abs(np.dot(w, x ** k) - 2 / (k + 1)) > 1e-6


@pytest.mark.parametrize("n", [3, 6, 9])
def test_derivative_matrix_exact(n):
    x, _ = gll.gll_nodes_weights(n)
    D = gll.lagrange_eval(x, x, deriv=1)
    for k in range(n):
        assert np.abs(D @ x ** k - k * x ** max(k - 1, 0) * (k > 0)).max() < 1e-11


def test_interpolation_exact():
    xp, _ = gll.gll_nodes_weights(4)
    xv, _ = gll.gll_nodes_weights(5)
    I = gll.lagrange_eval(xp, xv)
    f = lambda t: 2 * t ** 3 - t + 0.5
    assert np.abs(I @ f(xp) - f(xv)).max() < 1e-14


# ---------------------------------------------------------------------- SIPG
MESHES = [
    (2, 3, (2, 3), (True, False)),
    (2, 4, (3, 3), (True, True)),
    (3, 2, (2, 2, 1), (True, True, False)),
    (3, 3, (1, 2, 2), (False, True, True)),
]


def _mesh(d, P, n, per):
    return dg.Mesh(d, P, n, [0.0] * d, [1.0, 2.0, 1.5][:d], per)


@pytest.mark.parametrize("d,P,n,per", MESHES)
def test_sipg_symmetric_positive(d, P, n, per):
    m = _mesh(d, P, n, per)
    N = P + 1
    nu = 0.5 + np.random.default_rng(1).random(m.ne * N ** d)
    A = dg.sipg_matrix(m, N, nu, dirichlet=True).toarray()
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()
    ev = np.linalg.eigvalsh(A)
    if all(per):
        assert abs(ev[0]) < 1e-10 * ev[-1] and ev[1] > 1e-6 * ev[-1]   # only constants
        assert np.abs(A @ np.ones(A.shape[0])).max() < 1e-10 * np.abs(A).max()
    else:
        assert ev[0] > 1e-8 * ev[-1]


@pytest.mark.parametrize("d,P,n,per", MESHES)
def test_pressure_operators_nullspace(d, P, n, per):
    """SIPG (Neumann faces) and B M^-1 B^T on Q_{P-1}: SPD up to the constants only."""
    m = _mesh(d, P, n, per)
    L = dg.sipg_matrix(m, P, 1.0, dirichlet=False).toarray()
    B = dg.div_matrix(m, P + 1, P)
    Mv = np.tile(dg.mass_diag(m, P + 1), d)
    Lc = (B @ sp.diags(1 / Mv) @ B.T).toarray()
    for Op in (L, Lc):
        ev = np.linalg.eigvalsh(Op)
        assert abs(ev[0]) < 1e-10 * ev[-1]
        assert ev[1] > 1e-6 * ev[-1]


def _poly_case(d):
    if d == 2:
        u = lambda x, y: x ** 4 * y ** 2 - 3 * x * y ** 3 + y ** 4
        lap = lambda x, y: 12 * x ** 2 * y ** 2 + 2 * x ** 4 - 18 * x * y + 12 * y ** 2
        return u, lap
    u = lambda x, y, z: x ** 3 * z - y ** 2 * z ** 2 + x * y
    lap = lambda x, y, z: 6 * x * z - 2 * z ** 2 - 2 * y ** 2
    return u, lap


@pytest.mark.parametrize("d,P,n", [(2, 4, (3, 2)), (3, 3, (2, 1, 2))])
def test_sipg_polynomial_consistency(d, P, n):
    """A u - r_b(u) = -nu M lap(u) exactly for a global polynomial in Q_P (Dirichlet box):
    GLL quadrature is exact enough and summation by parts holds on GLL points."""
    m = dg.Mesh(d, P, n, [0.0] * d, [1.0, 0.7, 1.3][:d], [False] * d)
    N = P + 1
    X = m.node_coords(N).reshape(-1, d)
    u_f, lap_f = _poly_case(d)
    u = u_f(*X.T)
    lap = lap_f(*X.T)
    nu = 0.3
    A = dg.sipg_matrix(m, N, nu, dirichlet=True)
    r = dg.sipg_dirichlet_rhs(m, N, nu, u)
    M = dg.mass_diag(m, N)
    assert np.abs(A @ u - r + nu * M * lap).max() < 1e-12 * np.abs(nu * M * lap).max()


def test_sipg_helmholtz_convergence():
    """(M + A(nu)) u = M f + r_b with variable nu; error decays like h^(P+1)."""
    P = 3
    errs = []
    for ne in (2, 4):
        m = dg.Mesh(2, P, (ne, ne), [0, 0], [1, 1], (False, False))
        N = P + 1
        X = m.node_coords(N).reshape(-1, 2)
        x, y = X.T
        u = np.sin(2 * x + 1) * np.cos(3 * y)
        ux, uy = 2 * np.cos(2 * x + 1) * np.cos(3 * y), -3 * np.sin(2 * x + 1) * np.sin(3 * y)
        nu = 1 + 0.3 * x * y
        nux, nuy = 0.3 * y, 0.3 * x
        lap = -13 * u
        f = u - (nu * lap + nux * ux + nuy * uy)
        A = dg.sipg_matrix(m, N, nu, dirichlet=True)
        M = dg.mass_diag(m, N)
        rhs = M * f + dg.sipg_dirichlet_rhs(m, N, nu, u)
        uh = sp.linalg.spsolve((sp.diags(M) + A).tocsc(), rhs)
        errs.append(np.sqrt(np.sum(M * (uh - u) ** 2)))
    rate = np.log2(errs[0] / errs[1])
    assert rate > P + 0.5, (errs, rate)


# ------------------------------------------------------------- div / grad / D_k
def test_div_exact_for_polynomials():
    """B(v, q) = int v . grad q for continuous polynomials (quadrature exact on affine elements)."""
    d, P = 2, 4
    m = dg.Mesh(d, P, (3, 2), [0, 0], [1.0, 0.7], (False, False))
    Xv = m.node_coords(P + 1).reshape(-1, 2)
    Xp = m.node_coords(P).reshape(-1, 2)
    x, y = Xv.T
    xp, yp = Xp.T
    q = xp ** 3 * yp - yp ** 2 * xp + 1
    v = np.concatenate([x ** 2 * y ** 4, x * y - y ** 4 * x ** 3])
    val = q @ (dg.div_matrix(m, P + 1, P) @ v)
    xg, wg = np.polynomial.legendre.leggauss(20)
    GX, GY = np.meshgrid(0.5 * (xg + 1), 0.35 * (xg + 1), indexing="ij")
    W = np.outer(wg * 0.5, wg * 0.35)
    qx, qy = 3 * GX ** 2 * GY - GY ** 2, GX ** 3 - 2 * GY * GX
    exact = np.sum(W * ((GX ** 2 * GY ** 4) * qx + (GX * GY - GY ** 4 * GX ** 3) * qy))
    assert abs(val - exact) < 1e-14


def test_gradient_of_constant_vanishes():
    m = _mesh(3, 3, (2, 1, 2), (True, False, True))
    B = dg.div_matrix(m, 4, 3)
    assert np.abs(B.T @ np.ones(B.shape[0])).max() < 1e-13


def test_dg_derivative_exact_and_commuting():
    d, P = 2, 4
    m = dg.Mesh(d, P, (3, 2), [0, 0], [1.0, 0.7], (False, False))
    X = m.node_coords(P + 1).reshape(-1, 2)
    x, y = X.T
    u = x ** 4 * y ** 2 - 3 * x * y ** 3 + y ** 4
    D0 = dg.dg_derivative_matrix(m, P + 1, 0)
    D1 = dg.dg_derivative_matrix(m, P + 1, 1)
    assert np.abs(D0 @ u - (4 * x ** 3 * y ** 2 - 3 * y ** 3)).max() < 1e-12
    assert np.abs(D1 @ u - (2 * x ** 4 * y - 9 * x * y ** 2 + 4 * y ** 3)).max() < 1e-12
    assert abs(D0 @ D1 - D1 @ D0).max() < 1e-10 * abs(D0 @ D1).max()


def test_dg_derivative_is_central_on_jumps():
    """Hand case: u = 0 on element 0 and 1 on element 1 of a periodic 2 x 1 mesh; the
    lifting at a face node is (2/h)/w_end * (u+ - u-)/2 times the outward normal."""
    P = 2
    m = dg.Mesh(2, P, (2, 1), [0, 0], [2.0, 1.0], (True, True))
    N = P + 1
    u = np.concatenate([np.zeros(N * N), np.ones(N * N)])
    Du = dg.dg_derivative_matrix(m, N, 0) @ u
    w_end = 1.0 / 3.0
    lift = (2.0 / 1.0) / w_end * 0.5
    e0 = Du[:N * N].reshape(N, N)     # [iy, ix]
    assert np.allclose(e0[:, -1], lift) and np.allclose(e0[:, 0], -lift) and np.allclose(e0[:, 1], 0)


# ---------------------------------------------------------------- convection
def test_convection_exact_weak_form():
    """For a continuous polynomial field with v_b = v, M F_c equals the exact integral
    -int div(v v) . phi_j (over-integration exact, LLF dissipation vanishes)."""
    d, P = 2, 3
    m = dg.Mesh(d, P, (2, 2), [0, 0], [1.0, 1.0], (False, False))
    N = P + 1
    X = m.node_coords(N).reshape(-1, 2)
    x, y = X.T
    vx = lambda x, y: x * x * y - y ** 3
    vy = lambda x, y: x * y * y + 2 * x ** 3
    v = np.stack([vx(x, y), vy(x, y)])
    Fc = dg.Convection(m)(v, v)
    M = dg.mass_diag(m, N)
    xi, _ = gll.gll_nodes_weights(N)
    xg, wg = np.polynomial.legendre.leggauss(12)
    L = gll.lagrange_eval(xi, xg)

    def div_vv(x, y):
        a, b = vx(x, y), vy(x, y)
        ax, ay = 2 * x * y, x * x - 3 * y * y
        bx, by = y * y + 6 * x * x, 2 * x * y
        return np.stack([2 * a * ax + ay * b + a * by, bx * a + b * ax + 2 * b * by])

    nd = N * N
    for e in range(m.ne):
        ec = m.ecoords(e)
        gx = m.lo[0] + (ec[0] + 0.5 * (xg + 1)) * m.h[0]
        gy = m.lo[1] + (ec[1] + 0.5 * (xg + 1)) * m.h[1]
        GX, GY = np.meshgrid(gx, gy, indexing="xy")       # [iy, ix]
        W = np.outer(wg, wg) * m.jac()
        dv = div_vv(GX, GY)
        for j in range(nd):
            jx, jy = j % N, j // N
            phi = np.outer(L[:, jy], L[:, jx])
            for c in range(2):
                exact = -np.sum(W * dv[c] * phi)
                got = M[e * nd + j] * Fc[c, e * nd + j]
                assert abs(got - exact) < 1e-12, (e, j, c, got, exact)


def test_convection_llf_hand_case():
    """Piecewise-constant v = (1, 0) | (2, 0) on a periodic 2 x 1 mesh: the LLF flux is
    1.5 at the middle face and -3.5 (outward from element 0) at the periodic face, so
    the x-momentum of element 0 changes by -(1.5 - 3.5) * |F| and element 1's by the negative."""
    P = 2
    m = dg.Mesh(2, P, (2, 1), [0, 0], [2.0, 0.5], (True, True))
    N = P + 1
    nd = N * N
    vx = np.concatenate([np.ones(nd), 2 * np.ones(nd)])
    v = np.stack([vx, np.zeros(2 * nd)])
    Fc = dg.Convection(m)(v, None)
    M = dg.mass_diag(m, N)
    mom0 = np.sum((M * Fc[0])[:nd])
    mom1 = np.sum((M * Fc[0])[nd:])
    face = 0.5
    assert abs(mom0 - 2.0 * face) < 1e-13 and abs(mom1 + 2.0 * face) < 1e-13
    assert np.abs(Fc[1]).max() < 1e-14


def test_convection_conservative_periodic():
    m = dg.Mesh(3, 2, (2, 2, 1), [0, 0, 0], [1, 1, 1], (True, True, True))
    N = 3
    v = np.random.default_rng(3).standard_normal((3, m.ne * N ** 3))
    Fc = dg.Convection(m)(v, None)
    M = dg.mass_diag(m, N)
    assert np.abs((M[None, :] * Fc).sum(axis=1)).max() < 1e-12


def test_sipg_single_element_periodic_direction():
    """One element across a periodic direction is the same operator as two elements on a
    doubled box with the field repeated (translation invariance)."""
    N = 4
    m1 = dg.Mesh(2, 3, (2, 1), [0, 0], [1, 1], (False, True))
    m2 = dg.Mesh(2, 3, (2, 2), [0, 0], [1, 2], (False, True))
    rng = np.random.default_rng(0)
    nu1 = 0.5 + rng.random(m1.ne * N * N)
    u1 = rng.standard_normal(m1.ne * N * N)
    y1 = dg.sipg_matrix(m1, N, nu1, True) @ u1
    y2 = dg.sipg_matrix(m2, N, np.concatenate([nu1, nu1]), True) @ np.concatenate([u1, u1])
    assert np.abs(y2[:32] - y1).max() < 1e-12 and np.abs(y2[32:] - y1).max() < 1e-12


# ------------------------------------------------------ locality of the operators
# The full-size GPU parity tests compare sampled elements of a large mesh with the same
# elements of a small patch of their neighbours; this pins that reduction on meshes the
# oracle assembles whole: every operator's output on an element depends only on the element
# and its face neighbours (with the same fields and element sizes).
def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def test_operator_locality_clipped_patches_2d():
    # Dirichlet unit square: 3 x 3 patches clipped at the domain boundary keep its sides
    ne, P = 6, 3
    N, h = P + 1, 1.0 / 6
    mesh = dg.Mesh(2, P, (ne, ne), [0, 0], [1, 1], (False, False))
    nv, rng = ne * ne * N * N, np.random.default_rng(7)
    x, g = rng.standard_normal(nv), rng.standard_normal(nv)
    nu = 0.5 + rng.random(nv)
    v, vb, w = (rng.standard_normal(2 * nv) for _ in range(3))
    psi = rng.standard_normal(ne * ne * P * P)
    B = dg.div_matrix(mesh, N, P)
    full = {
        "sipg": (dg.sipg_matrix(mesh, N, nu) @ x - dg.sipg_dirichlet_rhs(mesh, N, nu, g)).reshape(ne * ne, -1),
        "conv": dg.Convection(mesh)(v, vb).reshape(2, ne * ne, -1),
        "div": (B @ v - dg.div_boundary_vector(mesh, N, P, w)).reshape(ne * ne, -1),
        "grad": ((B.T @ psi).reshape(2, -1) / dg.mass_diag(mesh, N)[None, :]).reshape(2, ne * ne, -1),
    }
    for ec in [(0, 0), (5, 5), (0, 3), (2, 3), (5, 1)]:
        x0, x1 = max(ec[0] - 1, 0), min(ec[0] + 1, ne - 1)
        y0, y1 = max(ec[1] - 1, 0), min(ec[1] + 1, ne - 1)
        nx, ny = x1 - x0 + 1, y1 - y0 + 1
        pm = dg.Mesh(2, P, (nx, ny), [x0 * h, y0 * h], [(x1 + 1) * h, (y1 + 1) * h], (False, False))
        idx = [i + ne * j for j in range(y0, y1 + 1) for i in range(x0, x1 + 1)]
        c = (ec[0] - x0) + nx * (ec[1] - y0)
        e = idx[c]
        el = lambda a: a.reshape(ne * ne, -1)[idx].ravel()
        vl = lambda a: a.reshape(2, ne * ne, -1)[:, idx].ravel()
        sip = dg.sipg_matrix(pm, N, el(nu)) @ el(x) - dg.sipg_dirichlet_rhs(pm, N, el(nu), el(g))
        assert _rel(full["sipg"][e], sip.reshape(len(idx), -1)[c]) < 1e-13
        cv = dg.Convection(pm)(vl(v), vl(vb)).reshape(2, len(idx), -1)[:, c]
        assert _rel(full["conv"][:, e], cv) < 1e-13
        Bp = dg.div_matrix(pm, N, P)
        dv = (Bp @ vl(v) - dg.div_boundary_vector(pm, N, P, vl(w))).reshape(len(idx), -1)[c]
        assert _rel(full["div"][e], dv) < 1e-13
        gr = ((Bp.T @ psi.reshape(ne * ne, -1)[idx].ravel()).reshape(2, -1) /
              dg.mass_diag(pm, N)[None, :]).reshape(2, len(idx), -1)[:, c]
        assert _rel(full["grad"][:, e], gr) < 1e-13


def test_operator_locality_periodic_patch_3d():
    # periodic box: the centre of a periodic 3 x 3 x 3 patch of the same element size sees
    # the same neighbours as the element of the large mesh (no wrap reaches it)
    ne, P = 4, 2
    N, L = P + 1, 2 * np.pi
    h = L / ne
    mesh = dg.Mesh(3, P, (ne, ne, ne), [0, 0, 0], [L] * 3, (True, True, True))
    nd, rng = N ** 3, np.random.default_rng(8)
    x = rng.standard_normal(ne ** 3 * nd)
    v = rng.standard_normal(3 * ne ** 3 * nd)
    xp = rng.standard_normal(ne ** 3 * P ** 3)
    A = dg.sipg_matrix(mesh, N, 0.3) @ x
    Lp = dg.sipg_matrix(mesh, P, 1.0, dirichlet=False) @ xp
    cv = dg.Convection(mesh)(v, None).reshape(3, ne ** 3, -1)
    pm = dg.Mesh(3, P, (3, 3, 3), [0, 0, 0], [3 * h] * 3, (True, True, True))
    for ec in [(0, 0, 0), (3, 1, 2), (2, 3, 3)]:
        idx = [((ec[0] + dx) % ne) + ne * (((ec[1] + dy) % ne) + ne * ((ec[2] + dz) % ne))
               for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
        e = idx[13]
        xs = x.reshape(ne ** 3, -1)[idx].ravel()
        assert _rel(A.reshape(ne ** 3, -1)[e], (dg.sipg_matrix(pm, N, 0.3) @ xs).reshape(27, -1)[13]) < 1e-13
        xps = xp.reshape(ne ** 3, -1)[idx].ravel()
        ref = (dg.sipg_matrix(pm, P, 1.0, dirichlet=False) @ xps).reshape(27, -1)[13]
        assert _rel(Lp.reshape(ne ** 3, -1)[e], ref) < 1e-13
        vs = v.reshape(3, ne ** 3, -1)[:, idx].ravel()
        assert _rel(cv[:, e], dg.Convection(pm)(vs, None).reshape(3, 27, -1)[:, 13]) < 1e-13
