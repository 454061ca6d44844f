"""solveLocalProblem (Alg. 1; Sec. 3, Eqs. "etaf_comb"; Sec. 4.2, Eq.
"source_term" and the multiplier subproblems below it).

For one coarse triangle K this computes, in FP64:

* the stiffness matrix A = [a(phi_j, phi_i)] with a(u,w) = (kappa grad u,
  grad w)_K, element by element on the refined submesh (element matrices
  by quadrature of the basis gradients; kappa constant per fine triangle);
* the load vectors: F = [(f, phi_w)_K] for the source subproblem (Eq.
  "etaf") and N_i = [-(s psi_i, phi_w)_{dK}] for the N_I multiplier
  subproblems (Eq. "etai"; psi_i changes sign with s = n . n_F^K);
* the solutions eta_f, eta_i in V_h(K), a subspace of the zero-mean space
  V_0^perp(K) (Sec. 2, item 2: the orthogonal complement of the piecewise
  constants; read as int_K eta = 0).  The test functions are zero-mean too,
  so each solve is the bordered system
        [ A   m ] [eta]   [g]
        [ m^T 0 ] [mu ] = [0],      m_w = int_K phi_w,
  solved densely by LU with partial pivoting (a library primitive);
* the local contributions to the skeleton system (Eq. "mat_global"):
  A_K[j,i] = (s psi_j, eta_i)_{dK}, E_K[j] = -(s psi_j, eta_f)_{dK},
  B_K[j] = (s psi_j, 1)_{dK}, F_K = (f, 1)_K, the boundary integrals taken
  by Gauss quadrature of the traces of eta on every piece of the coarse
  face between consecutive fine nodes and subface breakpoints.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg

from .fem import Submesh, basis, basis_grad_ref
from .mesh import CoarseMesh, legendre
from .quadrature import duffy_triangle, face_points, gauss_legendre_01


@dataclass
class FacePoint:
    """One Gauss point on the boundary of K."""
    weight: float            # quadrature weight times piece length
    tri: int                 # fine triangle owning the boundary segment
    dofs: np.ndarray         # its local DOF ids
    phi: np.ndarray          # basis values there
    lam_ids: np.ndarray      # local multiplier ids p = 0..l of the subface
    psi: np.ndarray          # psi values P_p(xi)
    sign: int


def boundary_points(mesh: CoarseMesh, K: int, sub: Submesh):
    """Gauss points on dK, split at fine nodes and subface breakpoints."""
    tri = mesh.tris[K]
    V = mesh.verts[tri]
    pts = []
    lam_off = 0
    for a in range(3):
        e = int(mesh.tri_edges[K, a])
        s = int(mesh.signs[K, a])
        m_e, l_e = int(mesh.m_e[e]), int(mesh.l_e[e])
        x_lo, x_hi = mesh.verts[mesh.edges[e, 0]], mesh.verts[mesh.edges[e, 1]]
        d = x_hi - x_lo
        length = float(np.linalg.norm(d))
        P0, Q0 = V[(a + 1) % 3], V[(a + 2) % 3]
        face_dir = Q0 - P0

        def on_face(x):
            c = face_dir[0] * (x[1] - P0[1]) - face_dir[1] * (x[0] - P0[0])
            return abs(c) <= 1e-12 * (1.0 + length * length)

        gx, gw = gauss_legendre_01(face_points(sub.P, l_e))
        for t in range(sub.tri_xy.shape[0]):
            X = sub.tri_xy[t]
            for u, v in ((0, 1), (1, 2), (2, 0)):
                if not (on_face(X[u]) and on_face(X[v])):
                    continue
                tau = sorted([float((X[u] - x_lo) @ d) / length ** 2, float((X[v] - x_lo) @ d) / length ** 2])
                cuts = [tau[0]] + [q / m_e for q in range(1, m_e) if tau[0] < q / m_e < tau[1]] + [tau[1]]
                for alpha, beta in zip(cuts[:-1], cuts[1:]):
                    q = int(np.floor(0.5 * (alpha + beta) * m_e))
                    for xk, wk in zip(gx, gw):
                        tau_k = alpha + (beta - alpha) * xk
                        x = x_lo + tau_k * d
                        lam = sub.barycentric(t, x[None, :])
                        xi = 2.0 * (tau_k * m_e - q) - 1.0
                        psi = np.array([float(legendre(p, xi)) for p in range(l_e + 1)])
                        ids = lam_off + q * (l_e + 1) + np.arange(l_e + 1)
                        pts.append(FacePoint(wk * (beta - alpha) * length, t, sub.dofs[t],
                                             basis(sub.P, lam)[0], ids, psi, s))
        lam_off += m_e * (l_e + 1)
    return pts, lam_off


def assemble_stiffness(sub: Submesh, kappa_K: np.ndarray) -> scipy.sparse.csr_matrix:
    """A = sum_T kappa_T [int_T grad phi_a . grad phi_b] (element by element)."""
    ref, w = duffy_triangle(4)
    lam = np.stack([1.0 - ref[:, 0] - ref[:, 1], ref[:, 0], ref[:, 1]], axis=1)
    G = basis_grad_ref(sub.P, lam)                           # (nq, nb, 2)
    Jinv = np.linalg.inv(sub.J)                              # (nT, 2, 2)
    grad = np.einsum("qbk,tkc->tqbc", G, Jinv)               # grad_x phi_b = J^{-T} grad_ref phi_b
    S = np.einsum("q,tqac,tqbc->tab", w, grad, grad) * np.abs(sub.detJ)[:, None, None]
    S *= np.asarray(kappa_K, dtype=np.float64)[:, None, None]
    nb = sub.dofs.shape[1]
    rows = np.repeat(sub.dofs, nb, axis=1).ravel()
    cols = np.tile(sub.dofs, (1, nb)).ravel()
    return scipy.sparse.coo_matrix((S.ravel(), (rows, cols)), shape=(sub.n, sub.n)).tocsr()


def cell_integrals(sub: Submesh, f):
    """(m, F, F_K): m_w = int phi_w, F_w = int f phi_w, F_K = int f (Duffy 4x4 per fine triangle)."""
    ref, w = duffy_triangle(4)
    lam = np.stack([1.0 - ref[:, 0] - ref[:, 1], ref[:, 0], ref[:, 1]], axis=1)
    phi = basis(sub.P, lam)                                  # (nq, nb)
    nT = sub.tri_xy.shape[0]
    X = sub.physical(np.arange(nT), ref)                     # (nT, nq, 2)
    fx = f(X[..., 0], X[..., 1]) if callable(f) else np.full(X.shape[:2], float(f))
    jac = np.abs(sub.detJ)[:, None]
    mass = np.zeros(sub.n)
    load = np.zeros(sub.n)
    np.add.at(mass, sub.dofs, jac * (w @ phi)[None, :])
    np.add.at(load, sub.dofs, np.einsum("tq,q,qb->tb", fx, w, phi) * jac)
    FK = float(np.sum(fx * w[None, :] * jac))
    return mass, load, FK


@dataclass
class LocalResult:
    AK: np.ndarray      # (N_I, N_I)
    EK: np.ndarray      # (N_I,)
    BK: np.ndarray      # (N_I,)
    FK: float
    eta: np.ndarray     # (n, N_I + 1): eta_0..eta_{N_I-1}, eta_f
    rhs: np.ndarray     # (n, N_I + 1): N_0..N_{N_I-1}, (f, phi_w)_K
    mass: np.ndarray    # (n,)
    sub: Submesh


def solve_local(mesh: CoarseMesh, K: int, r: int, P: int, kappa_K, f) -> LocalResult:
    sub = Submesh(mesh.verts[mesh.tris[K]], r, P)
    A = assemble_stiffness(sub, kappa_K)
    mass, load, FK = cell_integrals(sub, f)
    fpts, n_I = boundary_points(mesh, K, sub)

    # Right-hand sides: N_i = -(s psi_i, phi_w)_{dK} (Eq. "etai"), then (f, phi_w)_K (Eq. "etaf").
    rhs = np.zeros((sub.n, n_I + 1))
    for fp in fpts:
        rhs[np.ix_(fp.dofs, fp.lam_ids)] -= fp.sign * fp.weight * np.outer(fp.phi, fp.psi)
    rhs[:, n_I] = load

    # Zero-mean solutions by the bordered system (V_h(K) inside V_0^perp(K)).
    n = sub.n
    if n <= 2200:
        M = np.zeros((n + 1, n + 1))
        M[:n, :n] = A.toarray()
        M[:n, n] = mass
        M[n, :n] = mass
        sol = scipy.linalg.solve(M, np.vstack([rhs, np.zeros((1, n_I + 1))]))
    else:
        M = scipy.sparse.bmat([[A, mass[:, None]], [mass[None, :], None]], format="csc")
        sol = scipy.sparse.linalg.splu(M).solve(np.vstack([rhs, np.zeros((1, n_I + 1))]))
    eta = sol[:n]

    # Face integrals of the traces (Eq. "mat_global" entries).
    AK = np.zeros((n_I, n_I))
    EK = np.zeros(n_I)
    BK = np.zeros(n_I)
    for fp in fpts:
        trace = fp.phi @ eta[fp.dofs]                        # (N_I + 1,) values of every eta here
        spw = fp.sign * fp.psi * fp.weight
        AK[fp.lam_ids, :] += np.outer(spw, trace[:n_I])
        EK[fp.lam_ids] -= spw * trace[n_I]
        BK[fp.lam_ids] += spw
    return LocalResult(AK, EK, BK, FK, eta, rhs, mass, sub)
