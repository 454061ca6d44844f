"""The three-dimensional form of the method, as run in the paper's experiment
(Sec. 5: the Darcy model problem on the unit cube, tetrahedral coarse
elements, each with its own tetrahedral submesh; multipliers of degree
l = 0 on m = 4 or 16 subfaces per face; local Lagrange degree k = 2).
Test infrastructure, FP64, like the rest of this package.

It follows the same definitions as the two-dimensional modules (Sec. 2,
Eqs. "etaf", "etai", "global", "mat_global", "u_Hh"), with triangles
replaced by tetrahedra and edges by triangular faces.  The paper generates
its submeshes with TetGen and does not describe its coarse mesh beyond the
element counts 24, 192, 1536, 12288; the readings below replace both by
structured meshes with those counts.

Conventions (readings where the paper is silent):

* Coarse mesh.  nc^3 cubes of side 1/nc.  Corner (i,j,k) has vertex id
  i + (nc+1)(j + (nc+1)k); then the cube centres, cube (ci,cj,ck) at
  n_corner + ci + nc(cj + nc ck); then the centres of the grid faces normal
  to x, y, z in turn (closed-form ids below).  Each cube is cut into 24
  tetrahedra (centre, face centre, and the two ends of one edge of that
  face): faces in the order -x, +x, -y, +y, -z, +z, and on each face its
  corners (0,0),(1,0),(1,1),(0,1) in the two other axes taken in
  increasing order, the edge from corner q to corner q+1 (mod 4).  Element
  K = 24 cube + 4 face + edge, vertices (centre, face centre, corner q,
  corner q+1).  nc = 1, 2, 4, 8 give 24, 192, 1536, 12288 elements.
* Local face a of K is the face opposite local vertex a; its vertices are
  the other three in increasing local order.  Global faces are numbered in
  order of first encounter, K ascending then a = 0..3.
* Face normal: outward on the boundary of the cube; on an interior face
  with sorted global vertex ids g0 < g1 < g2 it is the unit vector along
  (x_g1 - x_g0) x (x_g2 - x_g0).  s = n . n_F^K = +-1.
* Lambda_H^{m,0}: m = 4^s subfaces per face, the uniform refinement of the
  face triangle with M = 2^s segments per side in the frame of its sorted
  vertices: P(i,j) = x_g0 + (i/M)(x_g1 - x_g0) + (j/M)(x_g2 - x_g0); row j
  holds first the "up" triangles P(i,j),P(i+1,j),P(i,j+1), i = 0..M-1-j,
  then the "down" triangles P(i+1,j),P(i+1,j+1),P(i,j+1), i = 0..M-2-j.
  psi_{F,q} is the indicator of subface q.  Global multiplier id
  F m + q; local id inside K: a m + q.
* Submesh of K = (v0,v1,v2,v3): the Freudenthal refinement of K seen as the
  simplex {N >= A >= B >= C >= 0} with N = 2^r, through the barycentric
  coordinates l0 = (N - A)/N, l1 = (A - B)/N, l2 = (B - C)/N, l3 = C/N.  Its
  8^r tetrahedra are, for base points z = (z1,z2,z3) in [0,N)^3 (z3 outer,
  then z2, then z1) and the permutations pi of (0,1,2) in lexicographic
  order, the simplices z, z + e_pi0, z + e_pi0 + e_pi1, z + (1,1,1) that lie
  in that simplex; kappa is stored in this order.
* Local DOFs: lattice points of spacing 1/(kN) in the same coordinates,
  enumerated C ascending, then B = C..kN, then A = B..kN.  Element DOFs: the
  four vertices, then (k = 2) the midpoints of the edges 01, 02, 03, 12,
  13, 23.  Basis in barycentrics: k = 1 l_a; k = 2 l_a (2 l_a - 1) and
  4 l_a l_b.
* Quadrature: a collapsed Gauss-Legendre rule on tetrahedra (n^3 points),
  the collapsed rule of the two-dimensional modules on triangles.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg

from .quadrature import duffy_triangle, gauss_legendre_01

PERMS = list(itertools.permutations(range(3)))     # lexicographic
EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


# ---------------------------------------------------------------- quadrature

def duffy_tet(n: int = 4):
    """Collapsed Gauss rule on the reference tetrahedron {x >= 0, sum <= 1}:
    x1 = a, x2 = b (1 - a), x3 = c (1 - a)(1 - b), weight
    w_a w_b w_c (1 - a)^2 (1 - b).  Points (n^3, 3), weights sum to 1/6."""
    g, w = gauss_legendre_01(n)
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                a, b, c = g[i], g[j], g[k]
                pts.append((a, b * (1.0 - a), c * (1.0 - a) * (1.0 - b)))
                wts.append(w[i] * w[j] * w[k] * (1.0 - a) ** 2 * (1.0 - b))
    return np.asarray(pts), np.asarray(wts)


# ---------------------------------------------------------------- coarse mesh

@dataclass
class CoarseMesh3D:
    nc: int
    m: int
    verts: np.ndarray        # (n_v, 3)
    tets: np.ndarray         # (n_K, 4)
    faces: np.ndarray        # (n_f, 3) sorted vertex ids
    tet_faces: np.ndarray    # (n_K, 4) global face of local face a
    face_tets: list          # per face: ascending adjacent K
    normals: np.ndarray      # (n_f, 3)
    signs: np.ndarray        # (n_K, 4)
    boundary: np.ndarray     # (n_f,) bool

    @property
    def n_K(self):
        return self.tets.shape[0]

    @property
    def n_f(self):
        return self.faces.shape[0]

    @property
    def n_lambda(self):
        return self.n_f * self.m

    def local_lambda(self, K):
        """Global multiplier ids of K's local basis (local faces a = 0..3 in turn)."""
        return np.concatenate([self.tet_faces[K, a] * self.m + np.arange(self.m) for a in range(4)]).astype(np.int64)


def build_mesh3d(nc: int, m: int = 4) -> CoarseMesh3D:
    """splitProblem's mesh side in 3-D (Alg. 1, first step; Sec. 5's cube)."""
    s = int(round(math.log(m, 4)))
    if 4 ** s != m:
        raise ValueError("m must be a power of 4")
    n1 = nc + 1
    corner = lambda i, j, k: i + n1 * (j + n1 * k)
    n_corner = n1 ** 3
    centre = lambda ci, cj, ck: n_corner + ci + nc * (cj + nc * ck)
    base = [n_corner + nc ** 3, n_corner + nc ** 3 + n1 * nc * nc, n_corner + nc ** 3 + 2 * n1 * nc * nc]

    def face_centre(d, p):
        # centre of the grid face normal to axis d at grid position p (p[d] in 0..nc, others < nc)
        i, j, k = p
        if d == 0:
            return base[0] + i + n1 * (j + nc * k)
        if d == 1:
            return base[1] + i + nc * (j + n1 * k)
        return base[2] + i + nc * (j + nc * k)

    nv = base[2] + n1 * nc * nc
    verts = np.zeros((nv, 3))
    for k in range(n1):
        for j in range(n1):
            for i in range(n1):
                verts[corner(i, j, k)] = (i / nc, j / nc, k / nc)
    for ck in range(nc):
        for cj in range(nc):
            for ci in range(nc):
                verts[centre(ci, cj, ck)] = ((ci + 0.5) / nc, (cj + 0.5) / nc, (ck + 0.5) / nc)
    for d in range(3):
        u, v = [x for x in range(3) if x != d]
        rng = [range(nc), range(nc), range(nc)]
        rng[d] = range(n1)
        for k in rng[2]:
            for j in rng[1]:
                for i in rng[0]:
                    p = [i, j, k]
                    x = np.array([i, j, k], dtype=np.float64) / nc
                    x[u] += 0.5 / nc
                    x[v] += 0.5 / nc
                    verts[face_centre(d, p)] = x

    tets = []
    for ck in range(nc):
        for cj in range(nc):
            for ci in range(nc):
                c = (ci, cj, ck)
                for d in range(3):
                    u, v = [x for x in range(3) if x != d]
                    for side in (0, 1):
                        p = list(c)
                        p[d] += side
                        fc = face_centre(d, p)
                        corners = []
                        for du, dv in ((0, 0), (1, 0), (1, 1), (0, 1)):
                            q = list(p)
                            q[u] += du
                            q[v] += dv
                            corners.append(corner(*q))
                        for e in range(4):
                            tets.append((centre(*c), fc, corners[e], corners[(e + 1) % 4]))
    tets = np.asarray(tets, dtype=np.int64)

    key_to_face, faces, face_tets = {}, [], []
    tet_faces = np.zeros((len(tets), 4), dtype=np.int64)
    for K, t in enumerate(tets):
        for a in range(4):
            key = tuple(sorted(int(t[b]) for b in range(4) if b != a))
            if key not in key_to_face:
                key_to_face[key] = len(faces)
                faces.append(key)
                face_tets.append([])
            f = key_to_face[key]
            tet_faces[K, a] = f
            face_tets[f].append(K)
    faces = np.asarray(faces, dtype=np.int64)
    boundary = np.array([len(ft) == 1 for ft in face_tets])
    normals = np.zeros((len(faces), 3))
    for f, (g0, g1, g2) in enumerate(faces):
        n = np.cross(verts[g1] - verts[g0], verts[g2] - verts[g0])
        n /= np.linalg.norm(n)
        if boundary[f]:
            K = face_tets[f][0]
            a = [b for b in range(4) if tet_faces[K, b] == f][0]
            if n @ (verts[g0] - verts[tets[K, a]]) < 0:
                n = -n
        normals[f] = n
    signs = np.zeros((len(tets), 4), dtype=np.int64)
    for K, t in enumerate(tets):
        for a in range(4):
            f = tet_faces[K, a]
            out = verts[faces[f, 0]] - verts[t[a]]          # points away from the opposite vertex
            signs[K, a] = 1 if normals[f] @ out > 0 else -1
    return CoarseMesh3D(nc, m, verts, tets, faces, tet_faces, face_tets, normals, signs, boundary)


def subface_index(mu1: float, mu2: float, M: int) -> int:
    """Subface q holding the interior point with face coordinates (mu1, mu2)
    (x = x_g0 + mu1 (x_g1 - x_g0) + mu2 (x_g2 - x_g0)), in the row order of
    the module docstring."""
    X, Y = M * mu1, M * mu2
    i, j = int(math.floor(X)), int(math.floor(Y))
    up = (X - i) + (Y - j) < 1.0
    row = sum(2 * M - 2 * jj - 1 for jj in range(j))
    return row + i if up else row + (M - j) + i


def face_coords(mesh: CoarseMesh3D, f: int, x: np.ndarray):
    """(mu1, mu2) of point x in the frame of face f's sorted vertices."""
    g0, g1, g2 = mesh.faces[f]
    E = np.stack([mesh.verts[g1] - mesh.verts[g0], mesh.verts[g2] - mesh.verts[g0]], axis=1)
    mu, *_ = np.linalg.lstsq(E, x - mesh.verts[g0], rcond=None)
    return float(mu[0]), float(mu[1])


# ---------------------------------------------------------------- submesh

def lattice_nodes(PN: int):
    """(n, 3) lattice coordinates (A, B, C), PN >= A >= B >= C >= 0, in DOF order."""
    return np.array([(A, B, C) for C in range(PN + 1) for B in range(C, PN + 1) for A in range(B, PN + 1)],
                    dtype=np.int64)


def sub_tets(N: int):
    """(N^3, 4, 3) vertex lattice coordinates (units 1/N) and (N^3,) permutation
    index of the Freudenthal simplices of {N >= A >= B >= C >= 0}, in kappa order."""
    out, cls = [], []
    inside = lambda p: N >= p[0] >= p[1] >= p[2] >= 0
    for z3 in range(N):
        for z2 in range(N):
            for z1 in range(N):
                for pi_i, pi in enumerate(PERMS):
                    p = [np.array([z1, z2, z3])]
                    for d in pi:
                        q = p[-1].copy()
                        q[d] += 1
                        p.append(q)
                    if all(inside(q) for q in p):
                        out.append(p)
                        cls.append(pi_i)
    out = np.asarray(out, dtype=np.int64)
    assert out.shape[0] == N ** 3
    return out, np.asarray(cls, dtype=np.int64)


def basis3d(P: int, lam: np.ndarray) -> np.ndarray:
    """(nq, nb) values of the P1 / P2 basis at barycentric points lam (nq, 4)."""
    if P == 1:
        return lam.copy()
    cols = [lam[:, a] * (2.0 * lam[:, a] - 1.0) for a in range(4)]
    cols += [4.0 * lam[:, a] * lam[:, b] for a, b in EDGES]
    return np.stack(cols, axis=1)


def basis3d_grad_bary(P: int, lam: np.ndarray) -> np.ndarray:
    """(nq, nb, 4) derivatives of the basis with respect to the barycentrics."""
    nq = lam.shape[0]
    if P == 1:
        return np.broadcast_to(np.eye(4), (nq, 4, 4)).copy()
    G = np.zeros((nq, 10, 4))
    for a in range(4):
        G[:, a, a] = 4.0 * lam[:, a] - 1.0
    for e, (a, b) in enumerate(EDGES):
        G[:, 4 + e, a] = 4.0 * lam[:, b]
        G[:, 4 + e, b] = 4.0 * lam[:, a]
    return G


class Submesh3D:
    """V_h(K) on the r-times refined K (P1 or P2, continuous)."""

    def __init__(self, V: np.ndarray, r: int, P: int):
        self.V, self.r, self.P = np.asarray(V, dtype=np.float64), r, P
        N = 1 << r
        self.N = N
        PN = P * N
        self.nodes = lattice_nodes(PN)
        self.n = self.nodes.shape[0]
        index = {tuple(x): i for i, x in enumerate(self.nodes)}
        self.tet_lat, self.tet_cls = sub_tets(N)
        dofs = []
        for T in self.tet_lat:
            nodes = [P * T[a] for a in range(4)]
            if P == 2:
                nodes += [T[a] + T[b] for a, b in EDGES]
            dofs.append([index[tuple(int(v) for v in x)] for x in nodes])
        self.dofs = np.asarray(dofs, dtype=np.int64)
        self.tet_xyz = self.lattice_to_x(self.tet_lat.reshape(-1, 3), N).reshape(-1, 4, 3)
        X = self.tet_xyz
        self.J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)  # columns
        self.detJ = np.linalg.det(self.J)

    def lattice_to_x(self, L: np.ndarray, scale: int) -> np.ndarray:
        A, B, C = L[:, 0] / scale, L[:, 1] / scale, L[:, 2] / scale
        lam = np.stack([1.0 - A, A - B, B - C, C], axis=1)
        return lam @ self.V

    def physical(self, ref: np.ndarray) -> np.ndarray:
        """(nT, nq, 3) physical points of reference points ref (nq, 3) on every sub-tet."""
        return self.tet_xyz[:, 0][:, None, :] + np.einsum("tij,qj->tqi", self.J, ref)

    def barycentric(self, t: int, x: np.ndarray) -> np.ndarray:
        ref = np.linalg.solve(self.J[t], (x - self.tet_xyz[t, 0]).T).T
        return np.concatenate([1.0 - ref.sum(axis=1, keepdims=True), ref], axis=1)


# ---------------------------------------------------------------- local problem

def _ref_bary(ref):
    return np.concatenate([1.0 - ref.sum(axis=1, keepdims=True), ref], axis=1)


def assemble_stiffness3d(sub: Submesh3D, kappa_K) -> scipy.sparse.csr_matrix:
    """A = sum_T kappa_T [int_T grad phi_a . grad phi_b] by quadrature (Sec. 2, a(.,.)_K)."""
    ref, w = duffy_tet(3)
    lam = _ref_bary(ref)
    Gb = basis3d_grad_bary(sub.P, lam)                       # (nq, nb, 4)
    D = np.array([[-1.0, -1.0, -1.0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    Gr = Gb @ D                                              # (nq, nb, 3) d/dref
    Jinv = np.linalg.inv(sub.J)
    grad = np.einsum("qbk,tkc->tqbc", Gr, Jinv)
    S = np.einsum("q,tqac,tqbc->tab", w, grad, grad) * np.abs(sub.detJ)[:, None, None]
    S *= np.asarray(kappa_K, dtype=np.float64)[:, None, None]
    nb = sub.dofs.shape[1]
    rows = np.repeat(sub.dofs, nb, axis=1).ravel()
    cols = np.tile(sub.dofs, (1, nb)).ravel()
    return scipy.sparse.coo_matrix((S.ravel(), (rows, cols)), shape=(sub.n, sub.n)).tocsr()


def cell_integrals3d(sub: Submesh3D, f):
    """(m, F, F_K): int phi_w, int f phi_w, int f, by the collapsed 4^3 rule per sub-tet."""
    ref, w = duffy_tet(4)
    phi = basis3d(sub.P, _ref_bary(ref))
    X = sub.physical(ref)
    fx = f(X[..., 0], X[..., 1], X[..., 2]) if callable(f) else np.full(X.shape[:2], float(f))
    jac = np.abs(sub.detJ)[:, None]
    mass = np.zeros(sub.n)
    load = np.zeros(sub.n)
    np.add.at(mass, sub.dofs, jac * (w @ phi)[None, :])
    np.add.at(load, sub.dofs, np.einsum("tq,q,qb->tb", fx, w, phi) * jac)
    return mass, load, float(np.sum(fx * w[None, :] * jac))


@dataclass
class FacePoint3D:
    weight: float
    dofs: np.ndarray
    phi: np.ndarray
    lam_id: int
    sign: int


def on_local_face(a: int, p, N: int) -> bool:
    """Lattice point p (units 1/N) on local face a (the face where l_a = 0)."""
    A, B, C = p
    return (A == N, A == B, B == C, C == 0)[a]


def boundary_points3d(mesh: CoarseMesh3D, K: int, sub: Submesh3D):
    """Quadrature points on dK: the collapsed 4x4 triangle rule on every fine
    face triangle, each inside exactly one subface (r >= log_4 m)."""
    M = int(round(math.sqrt(mesh.m)))
    if sub.N < M:
        raise ValueError("submesh coarser than the subfaces")
    ref2, w2 = duffy_triangle(4)
    pts = []
    for t in range(sub.tet_lat.shape[0]):
        T = sub.tet_lat[t]
        for a in range(4):
            for omit in range(4):
                tri = [b for b in range(4) if b != omit]
                if not all(on_local_face(a, T[b], sub.N) for b in tri):
                    continue
                X = sub.tet_xyz[t, tri]
                area2 = float(np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0])))
                f = int(mesh.tet_faces[K, a])
                q = subface_index(*face_coords(mesh, f, X.mean(axis=0)), M)
                for (u, v), wk in zip(ref2, w2):
                    x = X[0] + u * (X[1] - X[0]) + v * (X[2] - X[0])
                    lam = sub.barycentric(t, x[None, :])
                    pts.append(FacePoint3D(wk * area2, sub.dofs[t], basis3d(sub.P, lam)[0], a * mesh.m + q,
                                           int(mesh.signs[K, a])))
    return pts


@dataclass
class LocalResult3D:
    AK: np.ndarray
    EK: np.ndarray
    BK: np.ndarray
    FK: float
    eta: np.ndarray
    rhs: np.ndarray
    mass: np.ndarray
    sub: Submesh3D


def solve_local3d(mesh: CoarseMesh3D, K: int, r: int, P: int, kappa_K, f) -> LocalResult3D:
    """solveLocalProblem for one tetrahedron (Sec. 3, Eqs. "etaf", "etai"): the
    zero-mean Neumann solutions by the bordered system, then the face
    integrals of their traces (Eq. "mat_global" entries)."""
    sub = Submesh3D(mesh.verts[mesh.tets[K]], r, P)
    A = assemble_stiffness3d(sub, kappa_K)
    mass, load, FK = cell_integrals3d(sub, f)
    fpts = boundary_points3d(mesh, K, sub)
    n_I = 4 * mesh.m
    rhs = np.zeros((sub.n, n_I + 1))
    for fp in fpts:
        rhs[fp.dofs, fp.lam_id] -= fp.sign * fp.weight * fp.phi
    rhs[:, n_I] = load
    n = sub.n
    if n <= 2200:
        Mx = np.zeros((n + 1, n + 1))
        Mx[:n, :n] = A.toarray()
        Mx[:n, n] = mass
        Mx[n, :n] = mass
        sol = scipy.linalg.solve(Mx, np.vstack([rhs, np.zeros((1, n_I + 1))]))
    else:
        Mx = scipy.sparse.bmat([[A, mass[:, None]], [mass[None, :], None]], format="csc")
        sol = scipy.sparse.linalg.splu(Mx).solve(np.vstack([rhs, np.zeros((1, n_I + 1))]))
    eta = sol[:n]
    AK = np.zeros((n_I, n_I))
    EK = np.zeros(n_I)
    BK = np.zeros(n_I)
    for fp in fpts:
        trace = fp.phi @ eta[fp.dofs]
        sw = fp.sign * fp.weight
        AK[fp.lam_id, :] += sw * trace[:n_I]
        EK[fp.lam_id] -= sw * trace[n_I]
        BK[fp.lam_id] += sw
    return LocalResult3D(AK, EK, BK, FK, eta, rhs, mass, sub)


# ---------------------------------------------------------------- global problem

def dirichlet_term3d(mesh: CoarseMesh3D, g, N: int) -> np.ndarray:
    """G_j = (g, psi_j)_F on the boundary faces (s = +1): the collapsed 4x4 rule on
    the N^2 fine triangles of each face, each inside one subface."""
    G = np.zeros(mesh.n_lambda)
    if g is None:
        return G
    M = int(round(math.sqrt(mesh.m)))
    ref2, w2 = duffy_triangle(4)
    for f in range(mesh.n_f):
        if not mesh.boundary[f]:
            continue
        x0, x1, x2 = mesh.verts[mesh.faces[f]]
        for j in range(N):
            for i in range(N - j):
                for up in (True, False):
                    if not up and i > N - 2 - j:
                        continue
                    if up:
                        tri = [(i, j), (i + 1, j), (i, j + 1)]
                    else:
                        tri = [(i + 1, j), (i + 1, j + 1), (i, j + 1)]
                    X = [x0 + (a / N) * (x1 - x0) + (b / N) * (x2 - x0) for a, b in tri]
                    cen = np.mean([(a / N, b / N) for a, b in tri], axis=0)
                    q = subface_index(cen[0], cen[1], M)
                    area2 = float(np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0])))
                    for (u, v), wk in zip(ref2, w2):
                        x = X[0] + u * (X[1] - X[0]) + v * (X[2] - X[0])
                        G[f * mesh.m + q] += wk * area2 * float(g(x[0], x[1], x[2]))
    return G


def source3d_fn(kind: str, value: float = 1.0, freq: float = 2.0):
    """f of the model problem: constant, or 3 (freq pi)^2 prod sin(freq pi x_i)
    (freq = 2: the paper's 12 pi^2 sin sin sin, exact u = sin sin sin, Sec. 5)."""
    if kind == "const":
        return float(value)
    if kind == "sinsinsin":
        c = 3.0 * (freq * math.pi) ** 2 * value
        return lambda x, y, z: c * np.sin(freq * math.pi * x) * np.sin(freq * math.pi * y) * np.sin(freq * math.pi * z)
    raise ValueError(kind)


@dataclass
class OracleRun3D:
    mesh: CoarseMesh3D
    locals: list
    lam: np.ndarray
    u0: np.ndarray
    A: object = None
    B: object = None
    E: np.ndarray = None
    F: np.ndarray = None


def run3d(nc, r, P, m, kappa, f, g=None, K_subset=None) -> OracleRun3D:
    """Algorithm 1 on the cube: kappa per K (8^r values in sub-tet order)."""
    from . import globalsys
    mesh = build_mesh3d(nc, m)
    Ks = range(mesh.n_K) if K_subset is None else K_subset
    locals_ = [solve_local3d(mesh, K, r, P, kappa[i], f) for i, K in enumerate(Ks)]
    if K_subset is not None:
        return OracleRun3D(mesh, locals_, None, None)
    A, B, E, F = globalsys.assemble(mesh, locals_)
    G = dirichlet_term3d(mesh, g, 1 << r)
    lam, u0 = globalsys.solve(mesh, A, B, E, F, G)
    return OracleRun3D(mesh, locals_, lam, u0, A, B, E, F)


def local_u3d(mesh, K, loc, lam, u0):
    """Nodal values of u_{H,h} on K's submesh (Eq. "u_Hh")."""
    ids = mesh.local_lambda(K)
    return u0[K] + loc.eta[:, :len(ids)] @ lam[ids] + loc.eta[:, len(ids)]


def errors3d(mesh, locals_, lam, u0, exact, exact_grad=None):
    """(L2 error, broken H1 seminorm error) by the collapsed 4^3 rule per sub-tet."""
    ref, w = duffy_tet(4)
    lamq = _ref_bary(ref)
    D = np.array([[-1.0, -1.0, -1.0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    e2, h2 = 0.0, 0.0
    for K, loc in enumerate(locals_):
        sub = loc.sub
        u = local_u3d(mesh, K, loc, lam, u0)
        phi = basis3d(sub.P, lamq)
        X = sub.physical(ref)
        uh = np.einsum("qb,tb->tq", phi, u[sub.dofs])
        jac = np.abs(sub.detJ)[:, None]
        e2 += float(np.sum(w[None, :] * jac * (uh - exact(X[..., 0], X[..., 1], X[..., 2])) ** 2))
        if exact_grad is not None:
            Gr = basis3d_grad_bary(sub.P, lamq) @ D
            grad = np.einsum("qbk,tkc->tqbc", Gr, np.linalg.inv(sub.J))
            guh = np.einsum("tqbc,tb->tqc", grad, u[sub.dofs])
            gx = np.stack(exact_grad(X[..., 0], X[..., 1], X[..., 2]), axis=-1)
            h2 += float(np.sum(w[None, :] * jac * np.sum((guh - gx) ** 2, axis=-1)))
    return math.sqrt(e2), math.sqrt(h2)
