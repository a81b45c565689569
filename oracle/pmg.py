"""p-multigrid preconditioned CG for the pressure Poisson problems of Alg. 3 and Alg. 4.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain FP64 NumPy/SciPy.

Sec. 3.3 of the paper solves its Poisson problems by CG with the multigrid / Schwarz
preconditioners of its library, which it does not describe.  This module states the
preconditioner of this project from textbook pieces, in the order a V-cycle uses them:

* levels: the pressure degree p_0 = P - 1, then p_{l+1} = floor(p_l / 2) down to degree 1,
  all on the same mesh (p-multigrid);
* level operators: the SIPG pressure operator rediscretised at each degree (nu = 1,
  homogeneous Neumann faces), the matrix dg.sipg_matrix assembles;
* transfers: prolongation by element-local interpolation from the GLL(p_c) nodes to the
  GLL(p_f) nodes (the tensor product of the 1D Lagrange interpolation matrix, exact for
  polynomials of degree p_c), restriction its transpose;
* smoother: Chebyshev iteration accelerating the Jacobi iteration on the interval
  [lmax / ratio, lmax] of the spectrum of D^{-1} A (the three-term recurrence of Saad,
  Iterative Methods for Sparse Linear Systems, Sec. 12.3, Alg. 12.1), the same polynomial
  before and after the coarse correction;
* coarsest level (degree 1): the same Chebyshev iteration from zero with more steps, a fixed
  polynomial, so that the V-cycle stays a fixed symmetric linear operator;
* V-cycle: pre-smooth from zero, restrict the residual, recurse, prolongate and add,
  post-smooth;
* CG preconditioned by one V-cycle per iteration, the residual and the preconditioned
  residual kept mean-free (the constants are the null space of every level operator, and
  prolongation maps constants to constants).

The solution of the preconditioned CG is the solution of the Poisson problem; the
preconditioner only changes how many iterations reach it.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import dg, gll

# default V-cycle parameters (the values the CUDA path uses unless told otherwise)
PRE_POST = 3          # Chebyshev steps before and after the coarse correction
COARSE_STEPS = 10     # Chebyshev steps of the coarsest level
RATIO = 10.0          # smoothing interval [lmax / RATIO, lmax]
COARSE_RATIO = 100.0  # interval of the coarsest level's iteration
SAFETY = 1.1          # lmax = SAFETY x the estimated largest eigenvalue of D^{-1} A


def level_points(P):
    """Points per direction of the pressure levels, finest first: degree P-1, then halved."""
    deg = [P - 1]
    while deg[-1] > 1:
        deg.append(deg[-1] // 2)
    return [p + 1 for p in deg]


def interp_1d(Nc, Nf):
    """I[i, j] = l_j(x_i): the GLL(Nc) cardinal polynomials at the GLL(Nf) nodes."""
    xc, _ = gll.gll_nodes_weights(Nc)
    xf, _ = gll.gll_nodes_weights(Nf)
    return gll.lagrange_eval(xc, xf)


def prolongation(mesh, Nc, Nf):
    """Block-diagonal prolongation: the element-local tensor-product interpolation."""
    Ie = dg.kron_dims([interp_1d(Nc, Nf)] * mesh.d)
    return sp.kron(sp.identity(mesh.ne, format="csr"), sp.csr_matrix(Ie), format="csr")


def chebyshev(A, dinv, b, x0, steps, lmax, ratio):
    """`steps` Chebyshev-accelerated Jacobi steps for A x = b from x0 on [lmax/ratio, lmax].

    theta, delta: centre and half-width of the interval; with sigma = theta / delta the
    recurrence is d_0 = D^{-1} r_0 / theta, rho_0 = 1 / sigma, and for k >= 1
    rho_k = 1 / (2 sigma - rho_{k-1}),  d_k = rho_k rho_{k-1} d_{k-1} + 2 rho_k / delta D^{-1} r_k,
    with x_{k+1} = x_k + d_k and r_{k+1} = r_k - A d_k.
    """
    lmin = lmax / ratio
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b.copy() if x0 is None else b - A @ x
    rho = 1.0 / sigma
    dvec = dinv * r / theta
    for k in range(steps):
        x = x + dvec
        if k == steps - 1:
            break
        r = r - A @ dvec
        rho_new = 1.0 / (2.0 * sigma - rho)
        dvec = rho_new * rho * dvec + (2.0 * rho_new / delta) * (dinv * r)
        rho = rho_new
    return x


class PMG:
    """The V-cycle of the pressure operator of a mesh with velocity degree P (the multigrid
    preconditioner Sec. 3.3 names for the pressure solves, in this library's form)."""

    def __init__(self, mesh, P, lmax=None, pre_post=PRE_POST, coarse_steps=COARSE_STEPS, ratio=RATIO,
                 coarse_ratio=COARSE_RATIO):
        self.mesh = mesh
        self.N = level_points(P)
        self.A = [dg.sipg_matrix(mesh, N, 1.0, dirichlet=False).tocsr() for N in self.N]
        self.dinv = [1.0 / A.diagonal() for A in self.A]
        self.Pr = [prolongation(mesh, self.N[l + 1], self.N[l]) for l in range(len(self.N) - 1)]
        self.pre_post = pre_post
        self.coarse_steps = coarse_steps
        self.ratio = ratio
        self.coarse_ratio = coarse_ratio
        self.lmax = list(lmax) if lmax is not None else [SAFETY * largest_eig(A, d) for A, d in zip(self.A, self.dinv)]

    def vcycle(self, r, level=0):
        """z = B r: one V-cycle from level `level` applied to the residual r."""
        A, dinv, lm = self.A[level], self.dinv[level], self.lmax[level]
        if level == len(self.N) - 1:
            return chebyshev(A, dinv, r, None, self.coarse_steps, lm, self.coarse_ratio)
        z = chebyshev(A, dinv, r, None, self.pre_post, lm, self.ratio)
        Pl = self.Pr[level]
        rc = Pl.T @ (r - A @ z)
        z = z + Pl @ self.vcycle(rc, level + 1)
        return chebyshev(A, dinv, r, z, self.pre_post, lm, self.ratio)


def largest_eig(A, dinv):
    """Largest eigenvalue of D^{-1} A (symmetric form D^{-1/2} A D^{-1/2}), by ARPACK (the
    Chebyshev smoothing interval)."""
    s = np.sqrt(dinv)
    S = sp.diags(s) @ A @ sp.diags(s)
    n = A.shape[0]
    if n <= 400:
        return float(np.linalg.eigvalsh(S.toarray())[-1])
    return float(spla.eigsh(S, k=1, which="LA", tol=1e-10, return_eigenvectors=False)[0])


def pcg(A, b, precond, tol, maxit=1000, weights=None):
    """CG on the singular system A x = b - mean(b) (constants as null space), preconditioned
    by `precond`; the residual and the preconditioned residual are kept mean-free, the
    result has zero weighted mean (weights: the pressure mass).  Returns (x, iterations)."""
    b = b - b.mean()
    x = np.zeros_like(b)
    r = b.copy()
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0
    z = precond(r)
    z -= z.mean()
    p = z.copy()
    rz = r @ z
    its = 0
    for its in range(1, maxit + 1):
        Ap = A @ p
        alpha = rz / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        r -= r.mean()
        if np.linalg.norm(r) <= tol * bn:
            break
        z = precond(r)
        z -= z.mean()
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    if weights is not None:
        x -= (weights @ x) / weights.sum()
    return x, its
