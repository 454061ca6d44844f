"""Second-level space V_h(K): continuous Lagrange P_k (k = P = 1 or 2) on a
submesh of K obtained by r uniform (red) refinements (Sec. 2: each K_t is a
domain on its own with an internal triangulation; the local problems use
the continuous Galerkin method with a Lagrange basis of P_h^k).

Conventions:

* N = 2^r fine segments per coarse face.  Lattice point (i,j), i+j <= P N,
  of K = (v0,v1,v2) sits at v0 + i/(PN) (v1-v0) + j/(PN) (v2-v0) and is
  local DOF sum_{j'<j} (PN+1-j') + i.
* Fine triangles of the N-lattice, row j = 0..N-1: the "up" triangles
  (i,j),(i+1,j),(i,j+1) for i = 0..N-1-j, then the "down" triangles
  (i+1,j),(i+1,j+1),(i,j+1) for i = 0..N-2-j (the order of the kappa array).
* Element DOFs: P1 the three vertices A,B,C; P2 the vertices then the
  midpoints of BC, CA, AB.  Basis in barycentrics (l0,l1,l2):
  P1 l_a; P2 l_a(2 l_a - 1) and 4 l1 l2, 4 l2 l0, 4 l0 l1.
"""
from __future__ import annotations

import numpy as np


def n_local(P: int, N: int) -> int:
    pn = P * N
    return (pn + 1) * (pn + 2) // 2


def lattice_index(i, j, PN):
    return j * (PN + 1) - j * (j - 1) // 2 + i


def lattice_points(PN: int):
    """(n, 2) integer lattice coordinates of the local DOFs, in DOF order."""
    return np.array([(i, j) for j in range(PN + 1) for i in range(PN + 1 - j)], dtype=np.int64)


def fine_triangles(N: int):
    """(N*N, 3, 2) vertex lattice coordinates (units 1/N) of the fine triangles, CCW."""
    out = []
    for j in range(N):
        for i in range(N - j):
            out.append(((i, j), (i + 1, j), (i, j + 1)))
        for i in range(N - 1 - j):
            out.append(((i + 1, j), (i + 1, j + 1), (i, j + 1)))
    return np.asarray(out, dtype=np.int64)


def element_dofs(P: int, N: int) -> np.ndarray:
    """(N*N, 3 or 6) local DOF ids of each fine triangle's element nodes."""
    PN = P * N
    tri = fine_triangles(N) * P
    rows = []
    for t in tri:
        A, B, C = t
        nodes = [A, B, C]
        if P == 2:
            nodes += [(B + C) // 2, (C + A) // 2, (A + B) // 2]
        rows.append([lattice_index(int(x), int(y), PN) for x, y in nodes])
    return np.asarray(rows, dtype=np.int64)


def basis(P: int, lam: np.ndarray) -> np.ndarray:
    """Basis values (nq, nb) at barycentric points lam (nq, 3)."""
    l0, l1, l2 = lam[:, 0], lam[:, 1], lam[:, 2]
    if P == 1:
        return np.stack([l0, l1, l2], axis=1)
    return np.stack([l0 * (2 * l0 - 1), l1 * (2 * l1 - 1), l2 * (2 * l2 - 1),
                     4 * l1 * l2, 4 * l2 * l0, 4 * l0 * l1], axis=1)


def basis_grad_ref(P: int, lam: np.ndarray) -> np.ndarray:
    """Gradients (nq, nb, 2) w.r.t. reference coordinates (xi, eta) = (l1, l2),
    with l0 = 1 - xi - eta."""
    nq = lam.shape[0]
    l0, l1, l2 = lam[:, 0], lam[:, 1], lam[:, 2]
    if P == 1:
        g = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
        return np.broadcast_to(g, (nq, 3, 2)).copy()
    g = np.empty((nq, 6, 2))
    g[:, 0, 0] = -(4 * l0 - 1); g[:, 0, 1] = -(4 * l0 - 1)
    g[:, 1, 0] = 4 * l1 - 1;    g[:, 1, 1] = 0.0
    g[:, 2, 0] = 0.0;           g[:, 2, 1] = 4 * l2 - 1
    g[:, 3, 0] = 4 * l2;        g[:, 3, 1] = 4 * l1
    g[:, 4, 0] = -4 * l2;       g[:, 4, 1] = 4 * (l0 - l2)
    g[:, 5, 0] = 4 * (l0 - l1); g[:, 5, 1] = -4 * l1
    return g


class Submesh:
    """The refined submesh of one coarse triangle with its P1/P2 space."""

    def __init__(self, verts: np.ndarray, r: int, P: int):
        self.verts = np.asarray(verts, dtype=np.float64)   # (3, 2)
        self.r, self.P, self.N = r, P, 1 << r
        self.PN = P * self.N
        self.n = n_local(P, self.N)
        self.dofs = element_dofs(P, self.N)                  # (nT, nb)
        v0, v1, v2 = self.verts
        lat = fine_triangles(self.N).astype(np.float64) / self.N   # (nT, 3, 2)
        self.tri_xy = v0 + lat[..., 0:1] * (v1 - v0) + lat[..., 1:2] * (v2 - v0)   # (nT, 3, 2)
        pts = lattice_points(self.PN).astype(np.float64) / self.PN
        self.node_xy = v0 + pts[:, 0:1] * (v1 - v0) + pts[:, 1:2] * (v2 - v0)
        A, B, C = self.tri_xy[:, 0], self.tri_xy[:, 1], self.tri_xy[:, 2]
        self.J = np.stack([B - A, C - A], axis=2)          # (nT, 2, 2): columns B-A, C-A
        self.detJ = self.J[:, 0, 0] * self.J[:, 1, 1] - self.J[:, 0, 1] * self.J[:, 1, 0]
        self.area = 0.5 * np.abs(self.detJ)

    def barycentric(self, t: int, x: np.ndarray) -> np.ndarray:
        """Barycentric coordinates (npts, 3) of points x (npts, 2) in fine triangle t."""
        ref = np.linalg.solve(self.J[t], (x - self.tri_xy[t, 0]).T).T
        return np.stack([1.0 - ref[:, 0] - ref[:, 1], ref[:, 0], ref[:, 1]], axis=1)

    def physical(self, t_idx: np.ndarray, ref: np.ndarray) -> np.ndarray:
        """Physical points (nT, nq, 2) of reference points ref (nq, 2) in triangles t_idx."""
        A = self.tri_xy[t_idx, 0]
        return A[:, None, :] + np.einsum("tij,qj->tqi", self.J[t_idx], ref)
