"""reduceLocalProblems (Alg. 1; Sec. 3, Eq. "mat_global"): gather the local
contributions into the saddle-point system
        [ A  B^T ] [L]   [E + G]
        [ B  0   ] [P] = [F    ]
with A_ij = sum_K (s psi_j, eta_i)_{dK}, B_{K,j} = (s psi_j, 1)_{dK},
E_j = -sum_K (s psi_j, eta_f)_{dK}, F_K = (f, 1)_K (Eq. "global" with
mu = psi_j and q0 the indicator of K), and solve it directly.

The paper treats homogeneous Dirichlet data only; for u = g on the
boundary the first equation of Eq. "global" gains (g, psi_j)_F on every
boundary face F (where s = +1): G_j below.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse
import scipy.sparse.linalg

from .mesh import CoarseMesh, legendre
from .quadrature import gauss_legendre_01


def assemble(mesh: CoarseMesh, locals_):
    """Sparse A (L x L), B (N_K x L), vectors E (L), F (N_K) from the per-K results."""
    L = mesh.n_lambda
    rows, cols, vals = [], [], []
    B = np.zeros((mesh.n_K, L))
    E = np.zeros(L)
    F = np.zeros(mesh.n_K)
    for K, loc in enumerate(locals_):
        ids = mesh.local_lambda(K)
        rr, cc = np.meshgrid(ids, ids, indexing="ij")
        rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(loc.AK.ravel())
        E[ids] += loc.EK
        B[K, ids] += loc.BK
        F[K] = loc.FK
    A = scipy.sparse.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                shape=(L, L)).tocsr()
    return A, scipy.sparse.csr_matrix(B), E, F


def dirichlet_term(mesh: CoarseMesh, g, N=1) -> np.ndarray:
    """G_j = (g, psi_j)_F for boundary faces F (None = homogeneous), by Gauss
    quadrature on every piece between consecutive subface breakpoints and the
    N fine nodes of the face (exact for g piecewise polynomial on the submesh).
    N: segments per face, one number or one per coarse element (a boundary face
    takes the value of its element)."""
    G = np.zeros(mesh.n_lambda)
    if g is None:
        return G
    for e in range(mesh.n_e):
        if not mesh.boundary[e]:
            continue
        x_lo, x_hi = mesh.verts[mesh.edges[e, 0]], mesh.verts[mesh.edges[e, 1]]
        length = float(np.linalg.norm(x_hi - x_lo))
        m_e, l_e = int(mesh.m_e[e]), int(mesh.l_e[e])
        gx, gw = gauss_legendre_01(l_e + 4)
        N_e = int(N) if np.ndim(N) == 0 else int(N[mesh.edge_tris[e][0]])
        cuts = sorted(set([k / N_e for k in range(N_e + 1)] + [q / m_e for q in range(m_e + 1)]))
        for alpha, beta in zip(cuts[:-1], cuts[1:]):
            q = int(np.floor(0.5 * (alpha + beta) * m_e))
            for xk, wk in zip(gx, gw):
                tau = alpha + (beta - alpha) * xk
                x = x_lo + tau * (x_hi - x_lo)
                gv = float(g(x[0], x[1]))
                xi = 2.0 * (tau * m_e - q) - 1.0
                for p in range(l_e + 1):
                    G[mesh.lam_offset[e] + q * (l_e + 1) + p] += wk * (beta - alpha) * length * gv * float(legendre(p, xi))
    return G


def saddle_matrix(A, B):
    return scipy.sparse.bmat([[A, B.T], [B, None]], format="csc")


def solve(mesh: CoarseMesh, A, B, E, F, G=None):
    """(lambda, u0) by sparse LU of the saddle-point matrix (a library primitive)."""
    rhs = np.concatenate([E + (0.0 if G is None else G), F])
    x = scipy.sparse.linalg.spsolve(saddle_matrix(A, B), rhs)
    return x[:mesh.n_lambda], x[mesh.n_lambda:]
