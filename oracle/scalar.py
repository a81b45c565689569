"""Scalar IMEX harness: Alg. 1, Alg. 2, the SDC corrector and R(z) of Sec. 2.5.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The model problem is Eq. (model) of Sec. 2.1, du/dt = f_c(u) + f_d(nu, u), with
the linear test case f_c = lambda_c u, f_d = lambda_d u (Eq. conv-diff:ode).
Everything is plain Python complex arithmetic (double precision).
"""
import functools

import numpy as np

from . import gll
from .tableaux import get as get_tableau


def imex_rk_step(tab, u, dt, fc, fd, solve_d):
    """One step of Alg. 1 (IMEX RK, constant diffusivity).

    fc(u), fd(u): explicit and implicit right-hand sides.
    solve_d(rhs, gamma): returns u_i with u_i - gamma * fd(u_i) = rhs.
    """
    c, AI, bI, AE, bE = tab.as_float()
    s = tab.s
    us = [u]
    Fc = [fc(u)]
    Fd = [fd(u)]
    for i in range(1, s):
        rhs = u
        for j in range(i):
            rhs = rhs + dt * (AE[i][j] * Fc[j] + AI[i][j] * Fd[j])
        ui = solve_d(rhs, dt * AI[i][i])
        us.append(ui)
        Fc.append(fc(ui))
        Fd.append(fd(ui))
    out = u
    for i in range(s):
        out = out + dt * (bE[i] * Fc[i] + bI[i] * Fd[i])
    return out


def semi_implicit_rk_step(tab, u, dt, fc, fd, nu_of, solve_d):
    """One step of Alg. 2 (semi-implicit partitioned RK for variable diffusivity).

    fd(nu, u) is linear in u for fixed nu; nu_of(v) evaluates the diffusivity;
    solve_d(rhs, gamma, nu) returns u_i with u_i - gamma * fd(nu, u_i) = rhs.
    """
    c, AI, bI, AE, bE = tab.as_float()
    s = tab.s
    nus = [nu_of(u)]
    Fc = [fc(u)]
    Fd = [fd(nus[0], u)]
    for i in range(1, s):
        v = u
        for j in range(i):
            v = v + dt * AE[i][j] * (Fc[j] + Fd[j])
        nu_i = nu_of(v)
        rhs = u
        for j in range(i):
            rhs = rhs + dt * (AE[i][j] * Fc[j] + AI[i][j] * Fd[j])
        ui = solve_d(rhs, dt * AI[i][i], nu_i)
        nus.append(nu_i)
        Fc.append(fc(ui))
        Fd.append(fd(nu_i, ui))
    out = u
    for i in range(s):
        out = out + dt * (bE[i] * Fc[i] + bI[i] * Fd[i])
    return out


@functools.lru_cache(maxsize=None)
def sdc_nodes(M):
    """GLL sub-nodes on the unit step [0, 1] (Sec. 2.4) and the weights w_{q,m}.

    Reading of the weight interval: w_{q,m} integrates l_q over the subinterval
    (t_{m-1}, t_m) that the corrector Eq. (model:corrector) advances over.
    Returned weights are for a step of length 1 (scale by dt).
    """
    x, _ = gll.gll_nodes_weights(M + 1)
    tau = 0.5 * (x + 1.0)
    W = np.zeros((M + 1, M + 1))          # W[m, q], m = 1..M used
    for m in range(1, M + 1):
        W[m, :] = gll.lagrange_integrals(tau, tau[m - 1], tau[m])
    return tau, W


def sdc_step(M, K, predictor, u, dt, fc, fd, solve_d):
    """One step of the semi-implicit SDC method of Sec. 2.4 (linear / constant nu).

    predictor: name of an IMEX RK tableau applied once per subinterval
    ('EULER' gives SDC-Eu).  The corrector is Eq. (model:corrector) with the
    IMEX Euler rule for the first integral and Lagrange quadrature of f^k.
    """
    tau, W = sdc_nodes(M)
    t = dt * tau
    dts = np.diff(t)
    tab = get_tableau(predictor)
    uk = [u]
    for m in range(1, M + 1):
        uk.append(imex_rk_step(tab, uk[-1], dts[m - 1], fc, fd, solve_d))
    for _k in range(K):
        f_k = [fc(x) + fd(x) for x in uk]
        fc_k = [fc(x) for x in uk]
        fd_k = [fd(x) for x in uk]
        new = [uk[0]]
        for m in range(1, M + 1):
            S = sum(dt * W[m, q] * f_k[q] for q in range(M + 1))
            rhs = (new[m - 1] + dts[m - 1] * (fc(new[m - 1]) - fc_k[m - 1] - fd_k[m]) + S)
            new.append(solve_d(rhs, dts[m - 1]))
        uk = new
    return uk[-1]


def linear_problem(lc, ld):
    """f_c, f_d and the implicit solve of the linear test equation, Eq. (conv-diff:ode) of Sec. 2.1."""
    fc = lambda u: lc * u
    fd = lambda u: ld * u
    solve = lambda rhs, g: rhs / (1.0 - g * ld)
    return fc, fd, solve


def method_step(method):
    """Return step(u, dt, lc, ld) for 'RK-<name>' (Alg. 1) or 'SDC-<pred>(M,K)' (Sec. 2.4)."""
    name = method.strip()
    if name.upper().startswith("SDC-"):
        inner = name[4:]
        pred, rest = inner.split("(")
        M, K = [int(v) for v in rest.rstrip(")").split(",")]
        pred = "EULER" if pred.upper() in ("EU", "EULER") else pred

        def step(u, dt, lc, ld):
            fc, fd, solve = linear_problem(lc, ld)
            return sdc_step(M, K, pred, u, dt, fc, fd, solve)
        return step
    tab = get_tableau(name)

    def step(u, dt, lc, ld):
        fc, fd, solve = linear_problem(lc, ld)
        return imex_rk_step(tab, u, dt, fc, fd, solve)
    return step


def stability_function(method, z):
    """R(z) by the procedure of Sec. 2.5: one step with dt = 1,
    lambda_c = i Im z (explicit), lambda_d = Re z (implicit), u0 = 1."""
    step = method_step(method)
    return step(1.0 + 0j, 1.0, 1j * np.imag(z), np.real(z))


def critical_imag(method, re=-0.1, y_max=10.0, dy=1e-3, tol=1e-10):
    """Smallest y > 0 with |R(re + i y)| > 1 (Table 2's z_im^*), by scan + bisection."""
    y = dy
    prev = 0.0
    while y <= y_max:
        if abs(stability_function(method, re + 1j * y)) > 1.0:
            lo, hi = prev, y
            while hi - lo > tol:
                mid = 0.5 * (lo + hi)
                if abs(stability_function(method, re + 1j * mid)) > 1.0:
                    hi = mid
                else:
                    lo = mid
            return 0.5 * (lo + hi)
        prev = y
        y += dy
    return float("inf")


def substeps(method):
    """Number of nontrivial substeps per step (Sec. 2.5): s-1 for RK,
    M(K+1) for SDC with Euler predictor, M(K+s-1) with an RK predictor."""
    name = method.strip()
    if name.upper().startswith("SDC-"):
        inner = name[4:]
        pred, rest = inner.split("(")
        M, K = [int(v) for v in rest.rstrip(")").split(",")]
        if pred.upper() in ("EU", "EULER"):
            return M * (K + 1)
        return M * (K + get_tableau(pred).s - 1)
    return get_tableau(name).s - 1


# IMEX BDF2 of Eq. (bdf2:constant-nu), Sec. 2.2: gamma_0 = 3/2, alpha = (2, -1/2),
# beta = (2, -1); not self-starting, so its first step is IMEX Euler (all coefficients 1 or 0)
BDF2 = {"alpha": (2.0, -0.5), "beta": (2.0, -1.0), "gamma0": 1.5}
EULER_START = {"alpha": (1.0, 0.0), "beta": (1.0, 0.0), "gamma0": 1.0}


def bdf2_run(u0, dt, nsteps, fc, fd_solve):
    """nsteps of IMEX BDF2 on du/dt = f_c(u) + f_d(u), the first an IMEX Euler step.

    Each step solves (gamma_0 u^{n+1} - alpha_0 u^n - alpha_1 u^{n-1}) / dt
        = beta_0 f_c(u^n) + beta_1 f_c(u^{n-1}) + f_d(u^{n+1})
    for u^{n+1}; fd_solve(rhs, g) returns u with u - g f_d(u) = rhs.  Returns the list u^0..u^n.
    """
    us = [u0]
    for n in range(nsteps):
        co = EULER_START if n == 0 else BDF2
        a0, a1 = co["alpha"]
        b0, b1 = co["beta"]
        g0 = co["gamma0"]
        u, up = us[-1], (us[-2] if n > 0 else us[-1])
        rhs = (a0 * u + a1 * up + dt * (b0 * fc(u) + b1 * fc(up))) / g0
        us.append(fd_solve(rhs, dt / g0))
    return us
