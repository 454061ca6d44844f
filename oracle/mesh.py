"""Coarse mesh T_H, skeleton E_H, normals and the multiplier space
Lambda_H^{m,l} (Sec. 2: the family of triangulations with globally indexed
elements K_t and faces F_e, one unit normal n per face, outward on the
domain boundary, and the outward normal n_F^K of face F seen from K;
definition (i) of Lambda_H^{m,l}).

Conventions (the paper asks only for global indexing):

* Vertex (i,j) of the (nx+1) x (ny+1) grid on (0,1)^2 has id j(nx+1)+i.
* Square (i,j) (rows j, then columns i) is split along its (i,j)-(i+1,j+1)
  diagonal: K = 2(j nx + i) has CCW vertices (i,j),(i+1,j),(i+1,j+1) and
  K+1 has (i,j),(i+1,j+1),(i,j+1).
* Local face a of K is the face opposite local vertex a, run CCW from
  vertex a+1 to vertex a+2 (mod 3).  Global face ids are given in order of
  first encounter, K ascending then a = 0, 1, 2.
* Face normal n: outward on the boundary; on an interior face with global
  vertices g0 < g1, n = (t_y, -t_x) for the unit tangent t from g0 to g1.
  The sign seen from K is s = n . n_F^K = +-1.
* Lambda_H^{m,l} on face e: m uniform subfaces q = 0..m-1 counted from the
  lower-id vertex, and on each the Legendre polynomials P_p(xi), p = 0..l,
  of the subface coordinate xi in [-1,1] increasing away from the
  lower-id vertex.  Global index offset(e) + q(l+1) + p; inside K the local
  index runs over the local faces a = 0,1,2 in turn.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CoarseMesh:
    nx: int
    ny: int
    verts: np.ndarray        # (n_v, 2)
    tris: np.ndarray         # (n_K, 3) vertex ids, CCW
    edges: np.ndarray        # (n_e, 2) vertex ids, sorted (lower id first)
    tri_edges: np.ndarray    # (n_K, 3) global face id of local face a
    edge_tris: list          # per face: ascending list of adjacent K
    normals: np.ndarray      # (n_e, 2)
    signs: np.ndarray        # (n_K, 3) int, s = n . n_F^K
    boundary: np.ndarray     # (n_e,) bool
    m_e: np.ndarray          # (n_e,) subfaces per face
    l_e: np.ndarray          # (n_e,) polynomial degree per face
    lam_offset: np.ndarray   # (n_e + 1,) global multiplier offsets

    @property
    def n_K(self):
        return self.tris.shape[0]

    @property
    def n_e(self):
        return self.edges.shape[0]

    @property
    def n_lambda(self):
        return int(self.lam_offset[-1])

    def face_dofs(self, e):
        return int(self.m_e[e] * (self.l_e[e] + 1))

    def local_lambda(self, K):
        """Global multiplier ids of K's local basis, in local order (faces a = 0,1,2)."""
        ids = []
        for a in range(3):
            e = self.tri_edges[K, a]
            ids.extend(range(self.lam_offset[e], self.lam_offset[e + 1]))
        return np.asarray(ids, dtype=np.int64)


def build_mesh(nx: int, ny: int, m=1, l=0) -> CoarseMesh:
    """splitProblem's mesh side (Alg. 1, first step): T_H, faces, normals.

    `m` and `l` are either scalars or callables face_id -> value; per-face
    arrays may also be given (indexed by global face id)."""
    verts = np.array([(i / nx, j / ny) for j in range(ny + 1) for i in range(nx + 1)], dtype=np.float64)
    vid = lambda i, j: j * (nx + 1) + i
    tris = []
    for j in range(ny):
        for i in range(nx):
            tris.append((vid(i, j), vid(i + 1, j), vid(i + 1, j + 1)))
            tris.append((vid(i, j), vid(i + 1, j + 1), vid(i, j + 1)))
    tris = np.asarray(tris, dtype=np.int64)
    n_K = tris.shape[0]

    key_to_edge = {}
    edges = []
    edge_tris = []
    tri_edges = np.zeros((n_K, 3), dtype=np.int64)
    for K in range(n_K):
        for a in range(3):
            p, q = tris[K, (a + 1) % 3], tris[K, (a + 2) % 3]
            key = (min(p, q), max(p, q))
            if key not in key_to_edge:
                key_to_edge[key] = len(edges)
                edges.append(key)
                edge_tris.append([])
            e = key_to_edge[key]
            tri_edges[K, a] = e
            edge_tris[e].append(K)
    edges = np.asarray(edges, dtype=np.int64)
    n_e = edges.shape[0]
    boundary = np.array([len(t) == 1 for t in edge_tris])

    def outward(K, a):
        p, q = verts[tris[K, (a + 1) % 3]], verts[tris[K, (a + 2) % 3]]
        d = q - p
        return np.array([d[1], -d[0]]) / np.linalg.norm(d)

    normals = np.zeros((n_e, 2))
    for e in range(n_e):
        if boundary[e]:
            K = edge_tris[e][0]
            a = int(np.where(tri_edges[K] == e)[0][0])
            normals[e] = outward(K, a)
        else:
            t = verts[edges[e, 1]] - verts[edges[e, 0]]
            t = t / np.linalg.norm(t)
            normals[e] = (t[1], -t[0])
    signs = np.zeros((n_K, 3), dtype=np.int64)
    for K in range(n_K):
        for a in range(3):
            s = float(normals[tri_edges[K, a]] @ outward(K, a))
            signs[K, a] = int(round(s))
            assert abs(abs(s) - 1.0) < 1e-12

    def per_face(v):
        if callable(v):
            return np.array([int(v(e)) for e in range(n_e)], dtype=np.int64)
        v = np.asarray(v, dtype=np.int64)
        return np.full(n_e, int(v)) if v.ndim == 0 else v.copy()

    m_e = per_face(m)
    l_e = per_face(l)
    lam_offset = np.zeros(n_e + 1, dtype=np.int64)
    lam_offset[1:] = np.cumsum(m_e * (l_e + 1))
    return CoarseMesh(nx, ny, verts, tris, edges, tri_edges, edge_tris, normals, signs, boundary,
                      m_e, l_e, lam_offset)


def legendre(p: int, xi):
    """Legendre polynomial P_p(xi) by the three-term recurrence."""
    xi = np.asarray(xi, dtype=np.float64)
    if p == 0:
        return np.ones_like(xi)
    p0, p1 = np.ones_like(xi), xi
    for k in range(1, p):
        p0, p1 = p1, ((2 * k + 1) * xi * p1 - k * p0) / (k + 1)
    return p1
