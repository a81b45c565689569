"""Closed-form flows, viscosity laws, forcing and boundary data for the oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* ``tg2d``: decaying 2D Taylor-Green vortex u = (sin x cos y, -cos x sin y) e^{-2 nu t},
  p = 1/4 (cos 2x + cos 2y) e^{-4 nu t}; an exact Navier-Stokes solution for
  constant nu (the periodic 2D workload on [0, 2 pi]^2).
* ``tg3d``: the disturbed Taylor-Green initial field of Sec. 4.3, Eq.
  (transition:v0), evaluated at the point shifted by -pi/2 in x and +pi/2 in y
  and z, so that it reads (sin x cos y cos z, -cos x sin y cos z, 0) on
  [0, 2 pi]^3 (pinned in tests/test_oracle_flows.py).
* ``tgtravel``: the traveling Taylor-Green vortex of Sec. 4.1 with phase speed 1,
  decay rate 8 pi^2 nu_0.
* ``vv``: the travelling 3D vortex array of Sec. 4.2, Eq. (var-visc-test), with wave length 1,
  maximum speed 2 and phase speed 1 in each direction, and its pressure; with the
  velocity-dependent viscosity it is exact under the forcing ``forcing_vv``, Eq.
  (var-visc-test:rhs): f = d_t v + div(v v) - div[nu(v) (grad v + grad v^T)] + grad p,
  here with div v = 0 written as d_t v + (grad v) v - nu lap v - (grad v + grad v^T) grad nu
  + grad p;
* viscosity laws: constant; nu(x, y, t) = nu_0 (1 + 1/2 sin 2 pi x sin 2 pi y cos t);
  nu(v) = nu_0 + nu_1 (|v| / v_max)^2 (Sec. 4.2).
* forcing ``tgtravel_varnu``: f = (nu_0 - nu) lap v - (grad v + grad v^T) grad nu, the
  right-hand side that makes the traveling vortex exact under the variable viscosity
  (pattern of Eq. var-visc-test:rhs: f = d_t v + div(v v) - div(nu (grad v + grad v^T)) + grad p).
"""
import numpy as np

TWO_PI = 2.0 * np.pi


def tg2d_velocity(X, t, nu):
    """Decaying 2D Taylor-Green velocity, an exact solution of Eqs. (momentum), (continuity) of
    Sec. 3.1 with constant nu (the 2D periodic test flow)."""
    x, y = X[..., 0], X[..., 1]
    F = np.exp(-2.0 * nu * t)
    return np.stack([np.sin(x) * np.cos(y) * F, -np.cos(x) * np.sin(y) * F])


def tg2d_pressure(X, t, nu):
    """Pressure of the decaying 2D Taylor-Green vortex, mean-free."""
    x, y = X[..., 0], X[..., 1]
    return 0.25 * (np.cos(2 * x) + np.cos(2 * y)) * np.exp(-4.0 * nu * t)


def tg3d_velocity(X):
    """Initial field of the Taylor-Green transition, Eq. (transition:v0) of Sec. 4.3, at the
    point shifted by -pi/2 in x and +pi/2 in y and z."""
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    return np.stack([np.sin(x) * np.cos(y) * np.cos(z),
                     -np.cos(x) * np.sin(y) * np.cos(z),
                     np.zeros_like(x)])


def tgtravel_velocity(X, t, nu0):
    """Traveling Taylor-Green vortex of Sec. 4.1 on [0, 1]^2: phase speed 1 in x and y,
    decay rate 8 pi^2 nu_0."""
    x, y = X[..., 0], X[..., 1]
    a = TWO_PI * (x - t)
    b = TWO_PI * (y - 0.125 - t)
    F = np.exp(-8.0 * np.pi ** 2 * nu0 * t)
    return np.stack([1.0 + np.sin(a) * np.cos(b) * F, 1.0 - np.cos(a) * np.sin(b) * F])


def tgtravel_grad(X, t, nu0):
    """G[c, k] = d v_c / d x_k of the traveling vortex."""
    x, y = X[..., 0], X[..., 1]
    a = TWO_PI * (x - t)
    b = TWO_PI * (y - 0.125 - t)
    F = np.exp(-8.0 * np.pi ** 2 * nu0 * t)
    G = np.zeros((2, 2) + x.shape)
    G[0, 0] = TWO_PI * np.cos(a) * np.cos(b) * F
    G[0, 1] = -TWO_PI * np.sin(a) * np.sin(b) * F
    G[1, 0] = TWO_PI * np.sin(a) * np.sin(b) * F
    G[1, 1] = -TWO_PI * np.cos(a) * np.cos(b) * F
    return G


def nu_varxyt(X, t, nu0):
    """Viscosity nu(x, y, t) = nu_0 (1 + sin 2 pi x sin 2 pi y cos t / 2) of the manufactured
    variable-viscosity flow (the pattern of Sec. 4.1)."""
    x, y = X[..., 0], X[..., 1]
    return nu0 * (1.0 + 0.5 * np.sin(TWO_PI * x) * np.sin(TWO_PI * y) * np.cos(t))


def nu_varxyt_grad(X, t, nu0):
    """Spatial gradient of nu_varxyt."""
    x, y = X[..., 0], X[..., 1]
    c = 0.5 * nu0 * np.cos(t) * TWO_PI
    return np.stack([c * np.cos(TWO_PI * x) * np.sin(TWO_PI * y),
                     c * np.sin(TWO_PI * x) * np.cos(TWO_PI * y)])


def forcing_tgtravel_varnu(X, t, nu0):
    """Forcing that keeps the traveling vortex exact under nu(x, y, t): f = (nu_0 - nu) lap v
    - (grad v + grad v^T) grad nu, the right-hand side of the pattern of Eq.
    (var-visc-test:rhs) with the constant-nu_0 solution."""
    v = tgtravel_velocity(X, t, nu0)
    lap = -8.0 * np.pi ** 2 * (v - 1.0)          # Laplacian of the oscillating part
    nu = nu_varxyt(X, t, nu0)
    gnu = nu_varxyt_grad(X, t, nu0)
    G = tgtravel_grad(X, t, nu0)
    f = np.zeros_like(v)
    for c in range(2):
        f[c] = (nu0 - nu) * lap[c]
        for k in range(2):
            f[c] -= gnu[k] * (G[c, k] + G[k, c])
    return f


def vv_velocity(X, t):
    """Travelling 3D vortex array of Sec. 4.2, Eq. (var-visc-test): wave length 1, phase speed
    1 in each direction, maximum speed 2."""
    A, B, Cz = (TWO_PI * (X[..., k] + t) for k in range(3))
    return np.stack([(np.sin(A) + np.cos(B)) * np.sin(Cz),
                     (np.cos(A) + np.sin(B)) * np.sin(Cz),
                     (np.cos(A) + np.cos(B)) * np.cos(Cz)])


def vv_pressure(X, t):
    """Pressure of the vortex array, Eq. (var-visc-test:p)."""
    A, B, Cz = (TWO_PI * (X[..., k] + t) for k in range(3))
    return np.sin(A) * np.sin(B) * np.sin(Cz)


def vv_grad(X, t):
    """G[c, k] = d v_c / d x_k of the vortex array."""
    A, B, Cz = (TWO_PI * (X[..., k] + t) for k in range(3))
    sA, cA, sB, cB, sC, cC = np.sin(A), np.cos(A), np.sin(B), np.cos(B), np.sin(Cz), np.cos(Cz)
    k = TWO_PI
    G = np.zeros((3, 3) + A.shape)
    G[0, 0], G[0, 1], G[0, 2] = k * cA * sC, -k * sB * sC, k * (sA + cB) * cC
    G[1, 0], G[1, 1], G[1, 2] = -k * sA * sC, k * cB * sC, k * (cA + sB) * cC
    G[2, 0], G[2, 1], G[2, 2] = -k * sA * cC, -k * sB * cC, -k * (cA + cB) * sC
    return G


def forcing_vv(X, t, nu0, nu1, vmax):
    """Forcing of Eq. (var-visc-test:rhs) for the vortex array under nu(v) = nu_0 + nu_1
    (|v| / v_max)^2 (Sec. 4.2), in closed form with div v = 0."""
    v = vv_velocity(X, t)
    G = vv_grad(X, t)
    k = TWO_PI
    A, B, Cz = (TWO_PI * (X[..., j] + t) for j in range(3))
    gp = k * np.stack([np.cos(A) * np.sin(B) * np.sin(Cz), np.sin(A) * np.cos(B) * np.sin(Cz),
                       np.sin(A) * np.sin(B) * np.cos(Cz)])
    nu = nu0 + nu1 * np.sum(v ** 2, axis=0) / vmax ** 2
    gnu = np.stack([2.0 * nu1 / vmax ** 2 * sum(v[j] * G[j, i] for j in range(3)) for i in range(3)])
    f = np.zeros_like(v)
    for c in range(3):
        dt = G[c, 0] + G[c, 1] + G[c, 2]                  # every argument is (x_k + t)
        adv = sum(v[i] * G[c, i] for i in range(3))
        lap = -2.0 * k * k * v[c]                         # each term varies along two directions
        f[c] = dt + adv - nu * lap - sum((G[c, i] + G[i, c]) * gnu[i] for i in range(3)) + gp[c]
    return f


class Flow:
    """A flow case: initial data, viscosity law, forcing, boundary data, exact solution."""

    def __init__(self, kind, nu0, nu_kind="const", nu1=0.0, vmax=1.0):
        self.kind = kind
        self.nu0 = float(nu0)
        self.nu_kind = nu_kind
        self.nu1 = float(nu1)
        self.vmax = float(vmax)

    # --- viscosity ------------------------------------------------------
    def variable_nu(self):
        """True unless nu is constant (Alg. 2 / Alg. 3 then update nu per stage)."""
        return self.nu_kind != "const"

    def nu(self, X, t, v):
        """The viscosity law nu(x, t, v) of Eq. (momentum) at the points X (Sec. 3.1, 4.1, 4.2)."""
        if self.nu_kind == "const":
            return np.full(X.shape[:-1], self.nu0)
        if self.nu_kind == "varxyt":
            return nu_varxyt(X, t, self.nu0)
        if self.nu_kind == "velocity":
            mag2 = np.sum(np.asarray(v) ** 2, axis=0).reshape(X.shape[:-1])
            return self.nu0 + self.nu1 * mag2 / self.vmax ** 2
        raise ValueError(self.nu_kind)

    # --- fields -----------------------------------------------------------
    def exact(self, X, t):
        """The closed-form velocity at time t (the reference of the error and order pins)."""
        if self.kind == "tg2d":
            return tg2d_velocity(X, t, self.nu0)
        if self.kind == "tgtravel":
            return tgtravel_velocity(X, t, self.nu0)
        if self.kind == "vv":
            return vv_velocity(X, t)
        if self.kind == "tg3d":
            if t != 0.0:
                raise ValueError("tg3d has no closed form for t > 0")
            return tg3d_velocity(X)
        raise ValueError(self.kind)

    def initial(self, X):
        """Initial condition, Eq. (ic)."""
        return self.exact(X, 0.0)

    def boundary(self, X, t):
        """Dirichlet data v_b of Eq. (bc): the closed form on the boundary."""
        return self.exact(X, t)

    def has_forcing(self):
        """Whether the case carries a manufactured forcing f (Eq. (momentum))."""
        return (self.kind == "tgtravel" and self.nu_kind == "varxyt") or self.kind == "vv"

    def forcing(self, X, t):
        """The forcing f of Eq. (momentum) at the points X, d components."""
        if self.kind == "vv":
            return forcing_vv(X, t, self.nu0, self.nu1, self.vmax)
        if self.has_forcing():
            return forcing_tgtravel_varnu(X, t, self.nu0)
        return np.zeros((X.shape[-1],) + X.shape[:-1])
