"""Alg. 3 (IMEX RK) and Alg. 4 (SISDC) for incompressible flow, plain FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The right-hand side splits as in Sec. 3.2, F = F_c + F_d1 + F_d2 + F_d3 + F_p + F_s:

* F_c  = -div(v v)                   (dg.Convection, LLF flux, over-integration)
* F_d1 = div(nu grad v)              = -M^{-1} (A(nu) v - r_b(nu, v_b))   (SIPG)
* F_d2 = div(nu (grad v)^T)          = sum_k D_k (nu D_c v_k)
* F_d3 = -grad(nu div v)             = -D_c (nu sum_k D_k v_k)
* F_s  = f(x, t)

with D_k the nodal DG derivative of dg.dg_derivative_matrix.  The pressure
Poisson problems of Alg. 3 (line "psi'' <- solve ...") and Alg. 4 are solved in
the weak form  L psi = B v' - int_{dOmega} (n . v_b) q, with L either the SIPG
matrix on Q_{P-1} (homogeneous Neumann faces) or, in the "consistent" mode,
L = B M^{-1} B^T, which makes the projected velocity discretely
divergence-free.  The velocity update is v'' = v' - G psi with G = M^{-1} B^T.
All linear systems are solved directly (sparse LU); the singular pressure
problems are bordered with the constant vector.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import dg, gll
from .scalar import sdc_nodes
from .tableaux import get as get_tableau


class Discretization:
    """The DG-SEM discretisation of Sec. 3.3 on a mesh: GLL velocity space of degree P and
    pressure space of degree P-1, the assembled operators of Sec. 3.2's splitting of
    the right-hand side and the pressure Poisson operator of the projection (SIPG on Q_{P-1}
    with Neumann faces, or B M^{-1} B^T)."""

    def __init__(self, mesh, flow, poisson="sipg", stab=None):
        if mesh.P < 2:
            raise ValueError("velocity degree P must be at least 2")
        self.mesh = mesh
        self.flow = flow
        self.poisson_mode = poisson
        self.stab = stab                  # (zeta_D, zeta_C) of the stabilisation, or None
        d = mesh.d
        self.d = d
        self.Nv = mesh.P + 1
        self.Np = mesh.P
        self.X = mesh.node_coords(self.Nv)          # (ne, ndv, d)
        self.nv = mesh.ne * self.Nv ** d
        self.npr = mesh.ne * self.Np ** d
        self.Mv = dg.mass_diag(mesh, self.Nv)
        self.Mp = dg.mass_diag(mesh, self.Np)
        self.B = dg.div_matrix(mesh, self.Nv, self.Np)
        self.BT = self.B.T.tocsr()
        self.Dk = [dg.dg_derivative_matrix(mesh, self.Nv, k) for k in range(d)]
        self.conv = dg.Convection(mesh)
        if poisson == "sipg":
            L = dg.sipg_matrix(mesh, self.Np, 1.0, dirichlet=False)
        elif poisson == "consistent":
            L = (self.B @ sp.diags(1.0 / np.tile(self.Mv, d)) @ self.BT).tocsr()
        else:
            raise ValueError(poisson)
        self.L = L
        one = sp.csr_matrix(np.ones((self.npr, 1)))
        bordered = sp.bmat([[L, one], [one.T, None]], format="csc")
        self._poisson_lu = spla.splu(bordered)
        self._helm_cache = {}
        self._A_const = None
        self.has_boundary = not all(mesh.periodic)

    # ------------------------------------------------------------------ fields
    def nodal(self, field_fn, t):
        """A closed-form field at the velocity nodes, d blocks."""
        return np.asarray(field_fn(self.X, t)).reshape(self.d, -1) if field_fn else None

    def nu_field(self, t, v):
        """Nodal viscosity nu(x, t, v) of Eq. (momentum) (Alg. 3: the stage viscosity)."""
        X = self.X
        return np.asarray(self.flow.nu(X, t, np.asarray(v).reshape(self.d, *X.shape[:-1]))).ravel()

    def vb(self, t):
        """Nodal Dirichlet data v_b(t) of Eq. (bc), or None on a periodic mesh."""
        if not self.has_boundary:
            return None
        return np.asarray(self.flow.boundary(self.X, t)).reshape(self.d, -1)

    def fs(self, t):
        """F_s = f(x, t) of Sec. 3.2's splitting at the velocity nodes."""
        return np.asarray(self.flow.forcing(self.X, t)).reshape(self.d, -1)

    # -------------------------------------------------------------- operators
    def A(self, nu):
        """The assembled SIPG matrix of the viscous operator (Sec. 3.3; penalty N^2 / h max(nu-, nu+)) for nodal nu."""
        if not self.flow.variable_nu():
            if self._A_const is None:
                self._A_const = dg.sipg_matrix(self.mesh, self.Nv, self.flow.nu0, dirichlet=True)
            return self._A_const
        return dg.sipg_matrix(self.mesh, self.Nv, nu, dirichlet=True)

    def Fc(self, v, vb):
        """F_c = -div(v v) of Sec. 3.2 (LLF flux, over-integration on Gauss points)."""
        return self.conv(v, vb)

    def Fd1(self, v, nu, vb, A=None):
        """F_d1 = div(nu grad v) of Sec. 3.2 = -M^{-1}(A(nu) v - r_b(nu, v_b)) (SIPG)."""
        A = self.A(nu) if A is None else A
        out = np.empty((self.d, self.nv))
        for c in range(self.d):
            r = A @ v[c]
            if vb is not None:
                r -= dg.sipg_dirichlet_rhs(self.mesh, self.Nv, nu, vb[c])
            out[c] = -r / self.Mv
        return out

    def divergence_nodal(self, v):
        """sum_k D_k v_k, the nodal DG divergence (central lifting inside, own trace on the boundary)."""
        return sum(self.Dk[k] @ v[k] for k in range(self.d))

    def Fd3(self, v, nu):
        """F_d3 = -grad(nu div v) of Sec. 3.2 with the nodal DG derivatives."""
        phi = nu * self.divergence_nodal(v)
        return np.stack([-(self.Dk[c] @ phi) for c in range(self.d)])

    def Fd2(self, v, nu):
        """F_d2 = div(nu (grad v)^T) of Sec. 3.2 with the nodal DG derivatives."""
        out = np.zeros((self.d, self.nv))
        for c in range(self.d):
            for k in range(self.d):
                out[c] += self.Dk[k] @ (nu * (self.Dk[c] @ v[k]))
        return out

    def stabilized(self, v, dt):
        """The projected velocity after the divergence / mass-flux stabilisation (oracle/stab.py),
        with the time step dt in its penalty factors; unchanged without stabilisation."""
        if self.stab is None:
            return v
        from .stab import stabilize
        return stabilize(self.mesh, v, dt, *self.stab)

    def grad_p(self, psi):
        """G psi = M^{-1} B^T psi, the DG gradient of the projection's correction (Alg. 3)."""
        g = self.BT @ psi
        return g.reshape(self.d, self.nv) / self.Mv[None, :]

    def div_rhs(self, v, vb_or_none, mode):
        """B v - int (n . w) q with w = v_b (mode 'data') or w = v (mode 'trace')."""
        b = self.B @ np.asarray(v).ravel()
        if self.has_boundary:
            w = vb_or_none if mode == "data" else v
            b -= dg.div_boundary_vector(self.mesh, self.Nv, self.Np, w)
        return b

    def poisson(self, b):
        """Solve L psi = b on the mean-free subspace; returns psi with zero mass-weighted mean."""
        b = b - b.mean()
        rhs = np.concatenate([b, [0.0]])
        sol = self._poisson_lu.solve(rhs)
        psi = sol[:-1]
        return psi - np.dot(self.Mp, psi) / self.Mp.sum()

    def helmholtz(self, g, nu, gamma, vb):
        """(M + gamma A(nu)) u = M g + gamma r_b(nu, v_b), one solve per component."""
        key = gamma if not self.flow.variable_nu() else None
        lu = self._helm_cache.get(key) if key is not None else None
        if lu is None:
            H = (sp.diags(self.Mv) + gamma * self.A(nu)).tocsc()
            lu = spla.splu(H)
            if key is not None:
                self._helm_cache[key] = lu
        out = np.empty_like(g)
        for c in range(self.d):
            rhs = self.Mv * g[c]
            if vb is not None:
                rhs = rhs + gamma * dg.sipg_dirichlet_rhs(self.mesh, self.Nv, nu, vb[c])
            out[c] = lu.solve(rhs)
        return out

    def stage_rhs(self, v, nu, t, vb):
        """E = F_c + F_d2 + F_d3, F_d1, F_d3, F_s at one stage."""
        Fc = self.Fc(v, vb)
        Fd1 = self.Fd1(v, nu, vb)
        Fd3 = self.Fd3(v, nu)
        E = Fc + self.Fd2(v, nu) + Fd3
        Fs = self.fs(t)
        return E, Fd1, Fd3, Fs


def divergence_norm(disc, v, vb, t):
    """RMS of the weak divergence residual B v - int (n . v_b) q (zero after a consistent projection)."""
    b = disc.div_rhs(v, vb, "data")
    return float(np.sqrt(np.mean(b ** 2)))


# ---------------------------------------------------------------------------
# Alg. 3: IMEX RK for incompressible flow with variable viscosity
# ---------------------------------------------------------------------------
def rk_step(disc, tab, v, t, dt, final_projection=None):
    """One step of Alg. 3; returns (v_new, info)."""
    if isinstance(tab, str):
        tab = get_tableau(tab)
    c, AI, bI, AE, bE = tab.as_float()
    s = tab.s
    varnu = disc.flow.variable_nu()
    if final_projection is None:
        final_projection = varnu
    v = np.asarray(v, dtype=np.float64).reshape(disc.d, disc.nv)
    E, Fd1, Fd3, Fs = [None] * s, [None] * s, [None] * s, [None] * s
    nu1 = disc.nu_field(t, v)
    E[0], Fd1[0], Fd3[0], Fs[0] = disc.stage_rhs(v, nu1, t, disc.vb(t))
    vi = v
    psi = None
    for i in range(1, s):
        ti = t + c[i] * dt
        vb_i = disc.vb(ti)
        Fs[i] = disc.fs(ti)
        vp = v.copy()
        for j in range(i):
            vp += dt * AE[i][j] * (E[j] + Fd1[j] + Fd3[j])
        for j in range(i + 1):
            vp += dt * AI[i][j] * Fs[j]
        psi = disc.poisson(disc.div_rhs(vp, vb_i, "data"))
        vpp = disc.stabilized(vp - disc.grad_p(psi), dt)
        nu_i = disc.nu_field(ti, vpp)
        g = vpp.copy()
        for j in range(i):
            g += dt * ((AI[i][j] - AE[i][j]) * Fd1[j] - AE[i][j] * Fd3[j])
        vi = disc.helmholtz(g, nu_i, dt * AI[i][i], vb_i)
        E[i], Fd1[i], Fd3[i], _ = disc.stage_rhs(vi, nu_i, ti, vb_i)
    vnew = vi.copy()
    for i in range(s):
        fe = bE[i] - AE[s - 1][i]
        fi = bI[i] - AI[s - 1][i]
        if fe != 0.0:
            vnew += dt * fe * E[i]
        if fi != 0.0:
            vnew += dt * fi * (Fd1[i] + Fs[i])
    if final_projection:
        psi_f = disc.poisson(disc.div_rhs(vnew, None, "trace"))
        vnew = vnew - disc.grad_p(psi_f)
    return vnew, {"psi": psi}


# ---------------------------------------------------------------------------
# Alg. 4: SISDC corrector with an RK (or IMEX Euler) predictor
# ---------------------------------------------------------------------------
def sdc_step(disc, M, K, predictor, v, t, dt, final_projection=None):
    """One step of the SISDC method of Sec. 3.2.3 (predictor sweep + K corrector sweeps).

    Readings: the quadrature term sums w_{q,m} F(x, t_q, v^k_q, 0) over the
    sub-nodes q with F = F_c + F_d1 + F_d2 + F_d3 + F_s evaluated with
    nu(x, t_q, v^k_q); w_{q,m} integrates l_q over (t_{m-1}, t_m); the updated
    F^{IM,k+1}_m uses nu^{k+1}_{m-1}, the lag of its initialisation.
    """
    d = disc.d
    varnu = disc.flow.variable_nu()
    if final_projection is None:
        final_projection = varnu
    tau, W = sdc_nodes(M)
    tm = t + dt * tau
    dts = np.diff(tm)
    v0 = np.asarray(v, dtype=np.float64).reshape(d, disc.nv)
    # predictor: one RK step per subinterval
    vk = [v0]
    for m in range(1, M + 1):
        vn, _ = rk_step(disc, predictor, vk[-1], tm[m - 1], dts[m - 1],
                        final_projection=final_projection)
        vk.append(vn)

    def f_ex(vm, num, tq):
        """F(t_q, v_q) = F_c + F_d1 + F_d2 + F_d3 + F_s at one sub-node t_q (Alg. 4's quadrature term)."""
        vb = disc.vb(tq)
        return disc.Fc(vm, vb) + disc.Fd2(vm, num) + disc.Fd3(vm, num)

    # initial viscosity and RHS
    nuk = [disc.nu_field(tm[m], vk[m]) for m in range(M + 1)]
    FEX = [f_ex(vk[m], nuk[m], tm[m]) if m < M else None for m in range(M + 1)]
    FIM = [None] + [disc.Fd1(vk[m], nuk[m - 1], disc.vb(tm[m])) for m in range(1, M + 1)]
    for _k in range(K):
        # full right-hand side at the sub-nodes for the quadrature term
        Fq = []
        for q in range(M + 1):
            vbq = disc.vb(tm[q])
            Fq.append(f_ex(vk[q], nuk[q], tm[q]) + disc.Fd1(vk[q], nuk[q], vbq) + disc.fs(tm[q]))
        vnew = [vk[0]]
        nunew = [nuk[0]]
        FEXn = [FEX[0]]
        FIMn = [None]
        for m in range(1, M + 1):
            vb_m = disc.vb(tm[m])
            Fd1p = disc.Fd1(vk[m], nunew[m - 1], vb_m)
            Fd3p = disc.Fd3(vk[m], nunew[m - 1])
            S = sum(dt * W[m, q] * Fq[q] for q in range(M + 1))
            vp = vnew[m - 1] + dts[m - 1] * (FEXn[m - 1] + Fd1p + Fd3p - (FEX[m - 1] + FIM[m])) + S
            psi = disc.poisson(disc.div_rhs(vp, vb_m, "data"))
            vpp = disc.stabilized(vp - disc.grad_p(psi), dt)
            g = vpp - dts[m - 1] * (Fd1p + Fd3p)
            vppp = disc.helmholtz(g, nunew[m - 1], dts[m - 1], vb_m)
            if final_projection:
                psi_f = disc.poisson(disc.div_rhs(vppp, None, "trace"))
                vppp = vppp - disc.grad_p(psi_f)
            vnew.append(vppp)
            nunew.append(disc.nu_field(tm[m], vppp))
            FEXn.append(f_ex(vppp, nunew[m], tm[m]) if m < M else None)
            # F^{IM,k+1}_m with the viscosity lagged by one node, as in the initialisation
            # of Alg. 4 and in the corrector Eq. (model:corrector)
            FIMn.append(disc.Fd1(vppp, nunew[m - 1], vb_m))
        vk, nuk, FEX, FIM = vnew, nunew, FEXn, FIMn
    return vk[-1]


def rms(x):
    """Root mean square (the norm of Sec. 4's residuals and errors)."""
    return float(np.sqrt(np.mean(np.asarray(x) ** 2)))


def relative_l2(a, b):
    """||a - b|| / ||b|| (the relative L2 error of Sec. 4)."""
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


# ---------------------------------------------------------------------------
# IMEX BDF2 of Sec. 3.2.1: extrapolation, projection, diffusion, additional projection
# ---------------------------------------------------------------------------
def bdf2_step(disc, v, t, dt, prev=None, final_projection=None):
    """One step of IMEX BDF2 from v = v^n at t = t^n (the first step, prev = None, with the
    IMEX Euler coefficients of its start).  prev: the history returned by the previous step
    (v^{n-1} and its right-hand sides).  Returns (v^{n+1}, history for the next step, info).

    Readings: the projection solves psi = (dt / gamma_0) p'' from the same Poisson problem as
    Alg. 3 (weak divergence of v' with the boundary flux of v_b(t^{n+1})); the diffusion step
    uses the extrapolated viscosity beta_0 nu^n + beta_1 nu^{n-1} with nu^n = nu(x, t^n, v^n);
    the additional projection (variable viscosity) uses homogeneous Neumann data for the
    pressure increment, as the final projection of Alg. 3 does.
    """
    from .scalar import BDF2, EULER_START
    co = EULER_START if prev is None else BDF2
    a0, a1 = co["alpha"]
    b0, b1 = co["beta"]
    g0 = co["gamma0"]
    varnu = disc.flow.variable_nu()
    if final_projection is None:
        final_projection = varnu
    v = np.asarray(v, dtype=np.float64).reshape(disc.d, disc.nv)
    nu_n = disc.nu_field(t, v)
    E, Fd1, Fd3, _ = disc.stage_rhs(v, nu_n, t, disc.vb(t))
    cur = {"v": v, "E": E, "Fd1": Fd1, "Fd3": Fd3, "nu": nu_n}
    old = prev if prev is not None else cur
    t1 = t + dt
    vb1 = disc.vb(t1)
    # 1. extrapolation (forcing implicit: at t^{n+1})
    vp = (a0 * v + a1 * old["v"]
          + dt * (b0 * (E + Fd1 + Fd3) + b1 * (old["E"] + old["Fd1"] + old["Fd3"]) + disc.fs(t1))) / g0
    # 2. projection
    psi = disc.poisson(disc.div_rhs(vp, vb1, "data"))
    vpp = disc.stabilized(vp - disc.grad_p(psi), dt)
    # 3. diffusion with the extrapolated viscosity
    nu_star = b0 * nu_n + b1 * old["nu"]
    g = vpp - (dt / g0) * (b0 * (Fd1 + Fd3) + b1 * (old["Fd1"] + old["Fd3"]))
    vnew = disc.helmholtz(g, nu_star, dt / g0, vb1)
    # 4. additional projection
    if final_projection:
        psi_f = disc.poisson(disc.div_rhs(vnew, None, "trace"))
        vnew = vnew - disc.grad_p(psi_f)
    return vnew, cur, {"psi": psi, "pressure": g0 / dt * psi}
