"""Divergence / mass-flux stabilisation of the projected velocity (Sec. 3.3 adds it "for
pressure robustness" after the works it cites, without stating its form).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain FP64 NumPy/SciPy.

Reading used by this project (the penalised projection common to those works): after each
projection v'' = v' - grad psi, the velocity is replaced by the solution v~ of

    (M + A_D + A_C) v~ = M v'',
    A_D = sum_K tau_D,K  B_K^T W_K B_K,       tau_D,K = zeta_D |u_K| h_K / (P + 1) dt,
    A_C = sum_F tau_C,F  J_F^T W_F J_F,       tau_C,F = zeta_C (|u_K-| + |u_K+|) / 2 dt,

where B_K is the element-local (broken) divergence at the GLL nodes of element K, W_K its GLL
volume weights, J_F the jump u_k(K-) - u_k(K+) of the normal velocity component across an
interior face F normal to direction k (periodic faces included, boundary faces excluded),
W_F the face's GLL weights, |u_K| the magnitude of the mean velocity of v'' over K (mass
weighted), h_K = (h_1 ... h_d)^(1/d) and dt the time step.  The matrix is symmetric positive
definite; a continuous, divergence-free velocity is left unchanged.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import dg, gll


def mean_speed(mesh, v):
    """|u_K|: magnitude of the mass-weighted mean velocity of every element (the speed in the
    penalty factors of the stabilisation)."""
    N = mesh.P + 1
    W = dg.volume_weights(mesh, N)
    u = np.asarray(v).reshape(mesh.d, mesh.ne, -1)
    means = (u * W).sum(axis=2) / W.sum()
    return np.sqrt((means ** 2).sum(axis=0))


def penalty_matrix(mesh, v, dt, zeta_d, zeta_c):
    """A_D + A_C (d components, component-major) for the element speeds of v: the divergence and
    normal-jump penalties of the stabilisation Sec. 3.3 adds (this library's reading of its
    form: a penalised projection)."""
    d, N = mesh.d, mesh.P + 1
    nd = N ** d
    nv = mesh.ne * nd
    x, w = gll.gll_nodes_weights(N)
    Dh = gll.lagrange_eval(x, x, deriv=1)
    I = np.eye(N)
    W = dg.volume_weights(mesh, N)
    speed = mean_speed(mesh, v)
    hK = float(np.prod(mesh.h)) ** (1.0 / d)
    rows, cols, vals = [], [], []

    def add(r, c, blk):
        rr, cc = np.meshgrid(r, c, indexing="ij")
        rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(np.asarray(blk).ravel())

    # element-local divergence: B_K = [D_0, ..., D_{d-1}] acting on the d components
    Dk = [dg.kron_dims([(2.0 / mesh.h[k]) * Dh if j == k else I for j in range(d)]) for k in range(d)]
    for e in range(mesh.ne):
        tau = zeta_d * speed[e] * hK / (mesh.P + 1) * dt
        B = np.hstack(Dk)                                         # nd x (d nd)
        blk = tau * B.T @ (W[:, None] * B)
        idx = np.concatenate([c * nv + e * nd + np.arange(nd) for c in range(d)])
        add(idx, idx, blk)
    # normal-velocity jumps on interior faces normal to k (each face once: its left element)
    multi = dg.node_multi_indices(N, d)
    for k in range(d):
        wf = np.ones(nd)
        for a, idx in enumerate(multi):
            for j in range(d):
                if j != k:
                    wf[a] *= w[idx[j]] * mesh.h[j] / 2.0
        right = [a for a, idx in enumerate(multi) if idx[k] == N - 1]
        for e in range(mesh.ne):
            nb = mesh.neighbor(e, k, +1)
            if nb is None:
                continue
            tau = zeta_c * 0.5 * (speed[e] + speed[nb]) * dt
            for a in right:
                idx = list(multi[a])
                idx[k] = 0
                b = multi.index(tuple(idx))
                i0, i1 = k * nv + e * nd + a, k * nv + nb * nd + b
                t = tau * wf[a]
                add([i0, i1], [i0, i1], [[t, -t], [-t, t]])
    n = d * nv
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def stabilize(mesh, v, dt, zeta_d, zeta_c):
    """v~ = (M + A_D + A_C)^{-1} M v for the velocity v ([d][nv]): the stabilised projection
    (Sec. 3.3)."""
    d = mesh.d
    M = np.tile(dg.mass_diag(mesh, mesh.P + 1), d)
    A = (sp.diags(M) + penalty_matrix(mesh, v, dt, zeta_d, zeta_c)).tocsc()
    return spla.spsolve(A, M * np.asarray(v).ravel()).reshape(d, -1)
