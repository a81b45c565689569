"""DG-SEM spatial operators of the oracle, assembled as plain sparse matrices.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain FP64 NumPy/SciPy.

Sec. 3.3 of the paper fixes the ingredients (hexahedral / quadrilateral
elements, tensor-product Lagrange bases on GLL points, velocity degree P,
pressure degree P-1, DG-SEM with consistent integration and local
Lax-Friedrichs fluxes for convection, interior penalty for the pressure and
viscous problems) and defers the details to another paper that is not
available here.  The forms below are the readings used by this project, each
written out in its textbook weak form and assembled element by element from
dense per-element matrices (Kronecker products of 1D matrices on the affine
Cartesian elements):

* mass: GLL collocation quadrature, diagonal;
* SIPG bilinear form for -div(nu grad u), nodal nu, GLL quadrature on
  volumes and faces, penalty tau = N^2 / h_perp * max(nu-, nu+) on interior
  faces (N = nodes per direction = degree + 1) and 2 tau on Dirichlet faces;
* weak divergence B(v, q) = sum_K int_K v . grad q - sum_F int_F {v}.n [q]
  with velocity in Q_P and pressure test functions in Q_{P-1}, integrated on
  the velocity GLL points; DG gradient G = M^{-1} B^T;
* nodal DG derivative (central flux at interior faces, one-sided at domain
  boundaries) in weak form, used for the grad-div terms F_d2, F_d3;
* convection -div(v v) with the LLF flux, over-integrated on Gauss points.

Layout (the same one the library uses at its boundary): a scalar field is a
vector of length N_e * N^d, element-major, nodes lexicographic with x
fastest; a vector field is d such blocks, component-major.
"""
import itertools

import numpy as np
import scipy.sparse as sp

from . import gll


# ----------------------------------------------------------------------------
# mesh
# ----------------------------------------------------------------------------
class Mesh:
    """Cartesian box [lo, hi] split into n[0] x ... x n[d-1] equal elements (the hexahedral /
    quadrilateral meshes of Sec. 3.3 on the boxes of Sec. 4).

    periodic[k]: True for a periodic direction; a non-periodic direction has
    Dirichlet velocity data (and Neumann pressure data) on both of its ends.
    """

    def __init__(self, d, P, n, lo, hi, periodic):
        self.d = d
        self.P = P
        self.n = tuple(int(x) for x in n[:d])
        self.lo = tuple(float(x) for x in lo[:d])
        self.hi = tuple(float(x) for x in hi[:d])
        self.periodic = tuple(bool(x) for x in periodic[:d])
        self.h = tuple((self.hi[k] - self.lo[k]) / self.n[k] for k in range(d))
        self.ne = int(np.prod(self.n))

    def ecoords(self, e):
        out = []
        for k in range(self.d):
            out.append(e % self.n[k])
            e //= self.n[k]
        return out

    def eindex(self, ec):
        e = 0
        for k in reversed(range(self.d)):
            e = e * self.n[k] + ec[k]
        return e

    def neighbor(self, e, k, side):
        """Element across the face of element e normal to k (side -1 / +1), or None."""
        ec = self.ecoords(e)
        j = ec[k] + side
        if j < 0 or j >= self.n[k]:
            if not self.periodic[k]:
                return None
            j %= self.n[k]
        ec[k] = j
        return self.eindex(ec)

    def node_coords(self, N):
        """Physical coordinates, shape (ne, N^d, d), of the GLL(N) nodes."""
        xi, _ = gll.gll_nodes_weights(N)
        nd = N ** self.d
        X = np.zeros((self.ne, nd, self.d))
        for e in range(self.ne):
            ec = self.ecoords(e)
            for a, idx in enumerate(node_multi_indices(N, self.d)):
                for k in range(self.d):
                    X[e, a, k] = self.lo[k] + (ec[k] + 0.5 * (xi[idx[k]] + 1.0)) * self.h[k]
        return X

    def jac(self):
        return float(np.prod([hk / 2.0 for hk in self.h]))


def node_multi_indices(N, d):
    """(i_0, ..., i_{d-1}) for the lexicographic node order with i_0 fastest (the tensor-product
    GLL nodes of Sec. 3.3)."""
    out = []
    for flat in range(N ** d):
        idx = []
        for _ in range(d):
            idx.append(flat % N)
            flat //= N
        out.append(tuple(idx))
    return out


def kron_dims(mats):
    """Kronecker product with mats[0] acting on the fastest (x) index (the tensor-product
    element matrices of Sec. 3.3 on affine elements)."""
    out = np.array([[1.0]])
    for m in mats:
        out = np.kron(m, out)
    return out


def face_nodes(N, d, k, side):
    """Element-local indices of the nodes on face (k, side); side 0: i_k = 0, 1: i_k = N-1.
    Ordered lexicographically over the remaining directions (lowest fastest)."""
    fix = 0 if side == 0 else N - 1
    return np.array([a for a, idx in enumerate(node_multi_indices(N, d)) if idx[k] == fix])


def face_weights(mesh, N, k):
    """GLL quadrature weights (with the face Jacobian) of the nodes of a face normal to k (the
    face integrals of Sec. 3.3 on GLL points)."""
    _, w = gll.gll_nodes_weights(N)
    mats = []
    for j in range(mesh.d):
        if j == k:
            continue
        mats.append(np.diag(w * mesh.h[j] / 2.0))
    if not mats:
        return np.array([1.0])
    return np.diag(kron_dims(mats))


def volume_weights(mesh, N):
    """GLL volume quadrature weights of one element's nodes (collocation quadrature, Sec. 3.3)."""
    _, w = gll.gll_nodes_weights(N)
    return np.diag(kron_dims([np.diag(w * mesh.h[k] / 2.0) for k in range(mesh.d)]))


def grad_mats(mesh, N):
    """G[k] (N^d x N^d): nodal values of d/dx_k of the element's Lagrange basis (the GLL
    basis of Sec. 3.3)."""
    xi, _ = gll.gll_nodes_weights(N)
    Dh = gll.lagrange_eval(xi, xi, deriv=1)
    I = np.eye(N)
    G = []
    for k in range(mesh.d):
        mats = [Dh * (2.0 / mesh.h[k]) if j == k else I for j in range(mesh.d)]
        G.append(kron_dims(mats))
    return G


def mass_diag(mesh, N):
    """Diagonal of the GLL mass matrix, whole mesh (collocation quadrature)."""
    return np.tile(volume_weights(mesh, N), mesh.ne)


def _bc_kind(mesh, k, velocity):
    """Face kind of direction k: periodic, Dirichlet velocity (Eq. (bc)) or Neumann pressure."""
    if mesh.periodic[k]:
        return "periodic"
    return "dirichlet" if velocity else "neumann"


# ----------------------------------------------------------------------------
# SIPG
# ----------------------------------------------------------------------------
def sipg_matrix(mesh, N, nu, dirichlet=True):
    """Assembled SIPG matrix A with a(u, w) = w^T A u (the interior penalty form of Sec. 3.3 for
    -div(nu grad u); penalty N^2 / h_perp max(nu-, nu+), twice that on Dirichlet faces).

    nu: scalar or nodal array (ne * N^d).  dirichlet: non-periodic directions
    carry Dirichlet faces (velocity problems); False gives homogeneous Neumann
    faces there (the pressure problem), which contribute nothing.
    """
    d = mesh.d
    nd = N ** d
    nuv = np.broadcast_to(np.asarray(nu, dtype=np.float64), (mesh.ne * nd,)).reshape(mesh.ne, nd)
    G = grad_mats(mesh, N)
    W = volume_weights(mesh, N)
    rows, cols, vals = [], [], []

    def add(ei, ej, blk):
        r = ei * nd + np.arange(nd)
        c = ej * nd + np.arange(nd)
        rr, cc = np.meshgrid(r, c, indexing="ij")
        rows.append(rr.ravel())
        cols.append(cc.ravel())
        vals.append(blk.ravel())

    # volume: sum_q W_q nu_q grad u . grad w
    for e in range(mesh.ne):
        K = np.zeros((nd, nd))
        for k in range(d):
            K += G[k].T @ (((W * nuv[e])[:, None]) * G[k])
        add(e, e, K)

    for k in range(d):
        Wf = face_weights(mesh, N, k)
        nf = len(Wf)
        fl = face_nodes(N, d, k, 1)   # high face of the "minus" element
        fr = face_nodes(N, d, k, 0)   # low face of the "plus" element
        lo_nodes = face_nodes(N, d, k, 0)
        hi_nodes = face_nodes(N, d, k, 1)
        EL = np.zeros((nf, nd)); EL[np.arange(nf), fl] = 1.0
        ER = np.zeros((nf, nd)); ER[np.arange(nf), fr] = 1.0
        DnL = EL @ G[k]          # d/dx_k on the face, n = +e_k from minus to plus
        DnR = ER @ G[k]
        for e in range(mesh.ne):
            nb = mesh.neighbor(e, k, +1)
            if nb is not None:
                nuL = nuv[e][fl]
                nuR = nuv[nb][fr]
                tau = (N * N / mesh.h[k]) * np.maximum(nuL, nuR)
                # jump [u] = u- - u+ ; average {nu du/dn} = (nuL DnL uL + nuR DnR uR)/2
                Jl, Jr = EL, -ER
                Al, Ar = 0.5 * nuL[:, None] * DnL, 0.5 * nuR[:, None] * DnR
                # (a list, not a dict: with one element in a periodic direction e == nb
                # and all four blocks land on the same diagonal block)
                blocks = [
                    (e, e, -Jl.T @ (Wf[:, None] * Al) - Al.T @ (Wf[:, None] * Jl) + Jl.T @ ((Wf * tau)[:, None] * Jl)),
                    (e, nb, -Jl.T @ (Wf[:, None] * Ar) - Al.T @ (Wf[:, None] * Jr) + Jl.T @ ((Wf * tau)[:, None] * Jr)),
                    (nb, e, -Jr.T @ (Wf[:, None] * Al) - Ar.T @ (Wf[:, None] * Jl) + Jr.T @ ((Wf * tau)[:, None] * Jl)),
                    (nb, nb, -Jr.T @ (Wf[:, None] * Ar) - Ar.T @ (Wf[:, None] * Jr) + Jr.T @ ((Wf * tau)[:, None] * Jr)),
                ]
                for a, b, blk in blocks:
                    add(a, b, blk)
            if dirichlet and not mesh.periodic[k]:
                ec = mesh.ecoords(e)
                for side, nodes, sign in ((0, lo_nodes, -1.0), (1, hi_nodes, +1.0)):
                    if (side == 0 and ec[k] != 0) or (side == 1 and ec[k] != mesh.n[k] - 1):
                        continue
                    E = np.zeros((nf, nd)); E[np.arange(nf), nodes] = 1.0
                    Dn = sign * (E @ G[k])        # outward normal derivative
                    nub = nuv[e][nodes]
                    tau = 2.0 * (N * N / mesh.h[k]) * nub
                    blk = (-E.T @ ((Wf * nub)[:, None] * Dn) - Dn.T @ ((Wf * nub)[:, None] * E)
                           + E.T @ ((Wf * tau)[:, None] * E))
                    add(e, e, blk)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(mesh.ne * nd, mesh.ne * nd)).tocsr()
    A.sum_duplicates()
    return A


def sipg_dirichlet_rhs(mesh, N, nu, g):
    """r_b(w) = sum over Dirichlet faces of int (-nu dn w g + 2 tau g w) (Nitsche data term of
    the SIPG form of Sec. 3.3 with the data v_b of Eq. (bc)).

    g: nodal array (ne * N^d); only its values on Dirichlet-face nodes are used.
    """
    d = mesh.d
    nd = N ** d
    nuv = np.broadcast_to(np.asarray(nu, dtype=np.float64), (mesh.ne * nd,)).reshape(mesh.ne, nd)
    gv = np.asarray(g).reshape(mesh.ne, nd)
    G = grad_mats(mesh, N)
    r = np.zeros((mesh.ne, nd))
    for k in range(d):
        if mesh.periodic[k]:
            continue
        Wf = face_weights(mesh, N, k)
        nf = len(Wf)
        for e in range(mesh.ne):
            ec = mesh.ecoords(e)
            for side, sign in ((0, -1.0), (1, +1.0)):
                if (side == 0 and ec[k] != 0) or (side == 1 and ec[k] != mesh.n[k] - 1):
                    continue
                nodes = face_nodes(N, d, k, side)
                E = np.zeros((nf, nd)); E[np.arange(nf), nodes] = 1.0
                Dn = sign * (E @ G[k])
                nub = nuv[e][nodes]
                tau = 2.0 * (N * N / mesh.h[k]) * nub
                gb = gv[e][nodes]
                r[e] += -Dn.T @ (Wf * nub * gb) + E.T @ (Wf * tau * gb)
    return r.ravel()


# ----------------------------------------------------------------------------
# divergence / gradient between Q_P (velocity) and Q_{P-1} (pressure)
# ----------------------------------------------------------------------------
def div_matrix(mesh, Nv, Np):
    """B with B(v, q) = q^T B v, v = [v_0; ...; v_{d-1}] (component-major): the weak divergence
    of the projection's Poisson problem (Alg. 3, Sec. 3.3).

    B(v, q) = sum_K sum_x W_x v(x).grad q(x) - sum_{interior F} sum_f W_f {v}.n [q],
    quadrature on the velocity GLL(Nv) points (exact for affine elements).
    """
    d = mesh.d
    ndv, ndp = Nv ** d, Np ** d
    xv, _ = gll.gll_nodes_weights(Nv)
    xp, _ = gll.gll_nodes_weights(Np)
    Ip = gll.lagrange_eval(xp, xv)              # pressure basis at velocity points
    Dp = gll.lagrange_eval(xp, xv, deriv=1)     # its derivative there
    W = volume_weights(mesh, Nv)
    rows, cols, vals = [], [], []
    nv_tot = mesh.ne * ndv

    def add(ep, ev, comp, blk):
        r = ep * ndp + np.arange(ndp)
        c = comp * nv_tot + ev * ndv + np.arange(ndv)
        rr, cc = np.meshgrid(r, c, indexing="ij")
        rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(blk.ravel())

    for k in range(d):
        Gq = kron_dims([Dp * (2.0 / mesh.h[k]) if j == k else Ip for j in range(d)])  # ndv x ndp
        vol = Gq.T * W[None, :]                                                    # ndp x ndv
        for e in range(mesh.ne):
            add(e, e, k, vol)
        # interior faces normal to k
        Wf = face_weights(mesh, Nv, k)
        nf = len(Wf)
        fl_v = face_nodes(Nv, d, k, 1); fr_v = face_nodes(Nv, d, k, 0)
        EvL = np.zeros((nf, ndv)); EvL[np.arange(nf), fl_v] = 1.0
        EvR = np.zeros((nf, ndv)); EvR[np.arange(nf), fr_v] = 1.0
        # pressure trace at the velocity face points: pressure basis at xi_k = +-1
        ends = [np.array([[1.0 if i == 0 else 0.0 for i in range(Np)]]),
                np.array([[1.0 if i == Np - 1 else 0.0 for i in range(Np)]])]
        EqL = kron_dims([ends[1] if j == k else Ip for j in range(d)])   # nf x ndp
        EqR = kron_dims([ends[0] if j == k else Ip for j in range(d)])
        for e in range(mesh.ne):
            nb = mesh.neighbor(e, k, +1)
            if nb is None:
                continue
            # -W_f * 1/2 (vL + vR)_k * (qL - qR)
            add(e, e, k, -0.5 * EqL.T @ (Wf[:, None] * EvL))
            add(e, nb, k, -0.5 * EqL.T @ (Wf[:, None] * EvR))
            add(nb, e, k, 0.5 * EqR.T @ (Wf[:, None] * EvL))
            add(nb, nb, k, 0.5 * EqR.T @ (Wf[:, None] * EvR))
    B = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(mesh.ne * ndp, d * nv_tot)).tocsr()
    B.sum_duplicates()
    return B


def div_boundary_vector(mesh, Nv, Np, vb):
    """int over the Dirichlet boundary of (n . v_b) q for every pressure test function q (the
    boundary flux of the projection's Poisson right-hand side, Alg. 3).

    vb: (d, ne*Nv^d) nodal boundary velocity (only face values are used).
    """
    d = mesh.d
    ndv, ndp = Nv ** d, Np ** d
    xv, _ = gll.gll_nodes_weights(Nv)
    xp, _ = gll.gll_nodes_weights(Np)
    Ip = gll.lagrange_eval(xp, xv)
    vbv = np.asarray(vb).reshape(d, mesh.ne, ndv)
    out = np.zeros((mesh.ne, ndp))
    for k in range(d):
        if mesh.periodic[k]:
            continue
        Wf = face_weights(mesh, Nv, k)
        for side, sign in ((0, -1.0), (1, 1.0)):
            nodes = face_nodes(Nv, d, k, side)
            end = np.array([[1.0 if i == (0 if side == 0 else Np - 1) else 0.0 for i in range(Np)]])
            Eq = kron_dims([end if j == k else Ip for j in range(d)])
            for e in range(mesh.ne):
                ec = mesh.ecoords(e)
                if (side == 0 and ec[k] != 0) or (side == 1 and ec[k] != mesh.n[k] - 1):
                    continue
                out[e] += Eq.T @ (Wf * sign * vbv[k, e][nodes])
    return out.ravel()


# ----------------------------------------------------------------------------
# nodal DG derivative (grad-div terms)
# ----------------------------------------------------------------------------
def dg_derivative_matrix(mesh, N, k):
    """Nodal DG derivative along x_k (the derivatives of F_d2, F_d3 of Sec. 3.2):
    M (Dk u) = w-weak form
        -sum_K int u d_k w + sum_{interior F} int {u} [w]_k + sum_{boundary} int u n_k w,
    i.e. central flux inside, the element's own trace on the domain boundary."""
    d = mesh.d
    nd = N ** d
    G = grad_mats(mesh, N)
    W = volume_weights(mesh, N)
    Minv = 1.0 / W
    Wf = face_weights(mesh, N, k)
    nf = len(Wf)
    lo = face_nodes(N, d, k, 0); hi = face_nodes(N, d, k, 1)
    rows, cols, vals = [], [], []

    def add(ei, ej, blk):
        r = ei * nd + np.arange(nd)
        c = ej * nd + np.arange(nd)
        rr, cc = np.meshgrid(r, c, indexing="ij")
        rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(blk.ravel())

    vol = -(G[k].T * W[None, :])      # -sum_q W_q d_k w(x_q) u(x_q), rows = w
    EL = np.zeros((nf, nd)); EL[np.arange(nf), hi] = 1.0
    ER = np.zeros((nf, nd)); ER[np.arange(nf), lo] = 1.0
    for e in range(mesh.ne):
        add(e, e, Minv[:, None] * vol)
        nb = mesh.neighbor(e, k, +1)
        if nb is not None:
            # {u} [w]_k with n = +e_k from e to nb: w_e gets +, w_nb gets -
            add(e, e, Minv[:, None] * (0.5 * EL.T @ (Wf[:, None] * EL)))
            add(e, nb, Minv[:, None] * (0.5 * EL.T @ (Wf[:, None] * ER)))
            add(nb, e, Minv[:, None] * (-0.5 * ER.T @ (Wf[:, None] * EL)))
            add(nb, nb, Minv[:, None] * (-0.5 * ER.T @ (Wf[:, None] * ER)))
        ec = mesh.ecoords(e)
        if not mesh.periodic[k]:
            if ec[k] == 0:
                add(e, e, Minv[:, None] * (-ER.T @ (Wf[:, None] * ER)))
            if ec[k] == mesh.n[k] - 1:
                add(e, e, Minv[:, None] * (EL.T @ (Wf[:, None] * EL)))
    Dk = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(mesh.ne * nd, mesh.ne * nd)).tocsr()
    Dk.sum_duplicates()
    return Dk


# ----------------------------------------------------------------------------
# convection with LLF flux and over-integration
# ----------------------------------------------------------------------------
class Convection:
    """The convective term F_c of Sec. 3.2 as Sec. 3.3 discretises it:
    M F_c(v) = sum_K int (v v) : grad w - sum_F int H(v-, v+, n) . w, with
    H = 1/2 (v- (v-.n) + v+ (v+.n)) + 1/2 lambda (v- - v+),
    lambda = max(|v-.n|, |v+.n|) pointwise, volume and face integrals on
    Q = ceil(3(P+1)/2) Gauss points per direction; v+ = v_b on Dirichlet faces."""

    def __init__(self, mesh):
        self.mesh = mesh
        d = mesh.d
        N = mesh.P + 1
        self.N = N
        Q = gll.over_integration_points(mesh.P)
        self.Q = Q
        xi, _ = gll.gll_nodes_weights(N)
        xg, wg = gll.gauss_nodes_weights(Q)
        I1 = gll.lagrange_eval(xi, xg)
        D1 = gll.lagrange_eval(xi, xg, deriv=1)
        self.Ivol = kron_dims([I1] * d)
        self.Dvol = [kron_dims([D1 * (2.0 / mesh.h[k]) if j == k else I1 for j in range(d)])
                     for k in range(d)]
        self.Wvol = np.diag(kron_dims([np.diag(wg * mesh.h[k] / 2.0) for k in range(d)]))
        self.Iface, self.Wface, self.fnodes = {}, {}, {}
        for k in range(d):
            mats, wm = [], []
            for j in range(d):
                if j == k:
                    continue
                mats.append(I1)
                wm.append(np.diag(wg * mesh.h[j] / 2.0))
            self.Iface[k] = kron_dims(mats) if mats else np.array([[1.0]])
            self.Wface[k] = np.diag(kron_dims(wm)) if wm else np.array([1.0])
            self.fnodes[k] = (face_nodes(N, d, k, 0), face_nodes(N, d, k, 1))
        self.Minv = 1.0 / volume_weights(mesh, N)

    def __call__(self, v, vb=None):
        mesh, d = self.mesh, self.mesh.d
        nd = self.N ** d
        V = np.asarray(v).reshape(d, mesh.ne, nd)
        VB = None if vb is None else np.asarray(vb).reshape(d, mesh.ne, nd)
        out = np.zeros((d, mesh.ne, nd))
        for e in range(mesh.ne):
            vq = self.Ivol @ V[:, e, :].T                    # (nq, d)
            for c in range(d):
                acc = np.zeros(nd)
                for k in range(d):
                    acc += self.Dvol[k].T @ (self.Wvol * vq[:, c] * vq[:, k])
                out[c, e] += acc
            for k in range(d):
                lo, hi = self.fnodes[k]
                If, Wf = self.Iface[k], self.Wface[k]
                for side, own_nodes, sign in ((-1, lo, -1.0), (+1, hi, +1.0)):
                    nb = mesh.neighbor(e, k, side)
                    vm = If @ V[:, e, own_nodes].T               # (nfq, d)
                    if nb is not None:
                        nb_nodes = hi if side == -1 else lo
                        vp = If @ V[:, nb, nb_nodes].T
                    else:
                        vp = If @ VB[:, e, own_nodes].T
                    vmn = sign * vm[:, k]
                    vpn = sign * vp[:, k]
                    lam = np.maximum(np.abs(vmn), np.abs(vpn))
                    for c in range(d):
                        H = 0.5 * (vm[:, c] * vmn + vp[:, c] * vpn) + 0.5 * lam * (vm[:, c] - vp[:, c])
                        contrib = If.T @ (Wf * H)
                        out[c, e, own_nodes] -= contrib
        out *= self.Minv[None, None, :]
        return out.reshape(d, -1)
