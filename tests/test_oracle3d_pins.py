"""Pins of the three-dimensional oracle (oracle/tet3d.py; the paper's experiment,
Sec. 5: tetrahedral coarse mesh of the unit cube, tetrahedral submeshes, l = 0
multipliers on m = 4 or 16 subfaces, local degree k = 2) against closed forms,
invariants and exact solutions, none of which reuses the oracle's arithmetic."""
import math

import numpy as np
import pytest

from oracle import tet3d as T
from oracle import globalsys
from tests._golden import reference_tet_golden

REF_TET = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])


def _tet_volume(V):
    return abs(np.linalg.det(np.stack([V[1] - V[0], V[2] - V[0], V[3] - V[0]], axis=1))) / 6.0


def test_tet_rule_exact_monomials():
    gold = reference_tet_golden()["moments"]
    pts, w = T.duffy_tet(4)
    for (a, b, c), val in gold.items():
        got = float(np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c))
        assert abs(got - val) <= 1e-15, (a, b, c, got, val)


@pytest.mark.parametrize("nc", [1, 2])
def test_mesh3d_counts_and_orientation(nc):
    M = T.build_mesh3d(nc, 4)
    assert M.n_K == 24 * nc ** 3
    assert M.n_f == 36 * nc ** 3 + 12 * nc * nc * (nc + 1)
    assert int(M.boundary.sum()) == 24 * nc * nc
    edges = {tuple(sorted((int(t[a]), int(t[b])))) for t in M.tets for a in range(4) for b in range(a + 1, 4)}
    nv = (nc + 1) ** 3 + nc ** 3 + 3 * nc * nc * (nc + 1)
    assert len(set(M.tets.ravel().tolist())) == nv
    assert nv - len(edges) + M.n_f - M.n_K == 1              # Euler characteristic of a ball
    vol = sum(_tet_volume(M.verts[t]) for t in M.tets)
    assert abs(vol - 1.0) < 1e-13
    assert all(abs(_tet_volume(M.verts[t]) - 1.0 / (24 * nc ** 3)) < 1e-15 for t in M.tets)
    assert np.allclose(np.linalg.norm(M.normals, axis=1), 1.0)
    for f in range(M.n_f):
        ts = M.face_tets[f]
        x = M.verts[M.faces[f]]
        assert len(ts) == (1 if M.boundary[f] else 2)
        if M.boundary[f]:
            assert M.normals[f] @ (x.mean(axis=0) - 0.5) > 0     # outward from the cube
        else:
            (K0, K1) = ts
            a0 = list(M.tet_faces[K0]).index(f)
            a1 = list(M.tet_faces[K1]).index(f)
            assert M.signs[K0, a0] == -M.signs[K1, a1]
        for K in ts:
            a = list(M.tet_faces[K]).index(f)
            opp = M.verts[M.tets[K, a]]
            # s = +1 exactly when n points away from the opposite vertex
            assert M.signs[K, a] == (1 if M.normals[f] @ (x[0] - opp) > 0 else -1)


@pytest.mark.parametrize("P,r", [(1, 0), (1, 2), (2, 1), (2, 2), (1, 3)])
def test_submesh3d_structure(P, r):
    rng = np.random.default_rng(3)
    V = REF_TET + 0.2 * rng.standard_normal((4, 3))
    sub = T.Submesh3D(V, r, P)
    N = 1 << r
    assert sub.tet_lat.shape[0] == N ** 3
    assert sub.n == (P * N + 1) * (P * N + 2) * (P * N + 3) // 6
    vol = np.abs(sub.detJ) / 6.0
    assert np.allclose(vol, _tet_volume(V) / N ** 3, rtol=1e-12, atol=0)
    X = sub.lattice_to_x(sub.nodes, P * N)
    assert len({tuple(np.round(x, 12)) for x in X}) == sub.n
    # conformity: each face of a sub-tet is shared by two sub-tets or lies on dK (4 N^2 of them)
    count = {}
    for T4 in sub.tet_lat:
        for omit in range(4):
            key = tuple(sorted(tuple(int(v) for v in T4[b]) for b in range(4) if b != omit))
            count[key] = count.get(key, 0) + 1
    assert set(count.values()) <= {1, 2}
    assert sum(1 for c in count.values() if c == 1) == 4 * N * N
    assert sub.dofs.min() == 0 and sub.dofs.max() == sub.n - 1
    assert len(np.unique(sub.dofs)) == sub.n


def test_p1_stiffness_golden():
    gold = reference_tet_golden()["p1_stiffness"]
    sub = T.Submesh3D(REF_TET, 0, 1)
    S = T.assemble_stiffness3d(sub, [1.0]).toarray()
    assert np.abs(S - gold).max() < 1e-15


def test_p2_mass_golden_and_partition_of_unity():
    gold = reference_tet_golden()["p2_mass"]
    sub = T.Submesh3D(REF_TET, 0, 2)
    mass, load, FK = T.cell_integrals3d(sub, 2.0)
    vol = 1.0 / 6.0
    vert = sub.dofs[0, :4]
    edge = sub.dofs[0, 4:]
    assert np.abs(mass[vert] - gold["vertex"] * vol).max() < 1e-16
    assert np.abs(mass[edge] - gold["edge"] * vol).max() < 1e-16
    assert abs(FK - 2.0 * vol) < 1e-15 and np.abs(load - 2.0 * mass).max() < 1e-15
    rng = np.random.default_rng(5)
    V = REF_TET + 0.3 * rng.standard_normal((4, 3))
    sub = T.Submesh3D(V, 2, 2)
    mass, _, _ = T.cell_integrals3d(sub, 1.0)
    assert abs(mass.sum() - _tet_volume(V)) < 1e-14


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_p2_energy_of_quadratics(seed):
    """u^T S u = int |grad q|^2 for the P2 interpolant of a quadratic q on a random tet,
    the right side from the golden monomial moments by the affine change of variables."""
    rng = np.random.default_rng(seed)
    V = REF_TET + 0.3 * rng.standard_normal((4, 3))
    H = rng.standard_normal((3, 3))
    H = H + H.T
    b = rng.standard_normal(3)
    q = lambda X: 0.5 * np.einsum("ni,ij,nj->n", X, H, X) + X @ b
    sub = T.Submesh3D(V, 0, 2)
    S = T.assemble_stiffness3d(sub, [1.0]).toarray()
    u = q(sub.lattice_to_x(sub.nodes, 2))
    mom = reference_tet_golden()["moments"]
    J = np.stack([V[1] - V[0], V[2] - V[0], V[3] - V[0]], axis=1)
    c, D = H @ V[0] + b, H @ J
    first = np.array([mom[(1, 0, 0)], mom[(0, 1, 0)], mom[(0, 0, 1)]])
    # int xi_i xi_j: x^2 on the diagonal, xy, xz, yz off it (the tetrahedron is symmetric in its axes)
    second = np.array([[mom[(2, 0, 0)], mom[(1, 1, 0)], mom[(1, 0, 1)]],
                       [mom[(1, 1, 0)], mom[(2, 0, 0)], mom[(0, 1, 1)]],
                       [mom[(1, 0, 1)], mom[(0, 1, 1)], mom[(2, 0, 0)]]])
    exact = abs(np.linalg.det(J)) * (c @ c * mom[(0, 0, 0)] + 2 * c @ D @ first + np.sum(D.T @ D * second))
    assert abs(u @ S @ u - exact) <= 1e-12 * abs(exact)
    assert np.abs(S.sum(axis=1)).max() < 1e-12 * np.abs(S).max()


def _subface_centroid_area(mesh, f, q):
    """Closed-form centroid and area of subface q of face f (its definition in the frame
    of the sorted face vertices, row j: up triangles then down triangles)."""
    M = int(round(math.sqrt(mesh.m)))
    x0, x1, x2 = mesh.verts[mesh.faces[f]]
    k = 0
    for j in range(M):
        tris = [[(i, j), (i + 1, j), (i, j + 1)] for i in range(M - j)]
        tris += [[(i + 1, j), (i + 1, j + 1), (i, j + 1)] for i in range(M - 1 - j)]
        for tri in tris:
            if k == q:
                P = np.array([x0 + (a / M) * (x1 - x0) + (b / M) * (x2 - x0) for a, b in tri])
                return P.mean(axis=0), 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
            k += 1
    raise IndexError(q)


@pytest.mark.parametrize("P,r,m", [(2, 1, 4), (1, 2, 4), (2, 2, 16)])
def test_local3d_rhs_subface_moments(P, r, m):
    """Column j of the multiplier right-hand sides is -s (psi_j, phi_w): its sum is
    -s |subface j| and its first moment sum_w x_w (...) is -s |subface| centroid, since
    the P_k interpolant of x is exact (pins the subface numbering and the signs)."""
    mesh = T.build_mesh3d(1, m)
    rng = np.random.default_rng(7)
    for K in (0, 5, 13, 23):
        loc = T.solve_local3d(mesh, K, r, P, rng.uniform(0.5, 2.0, 8 ** r), 1.0)
        X = loc.sub.lattice_to_x(loc.sub.nodes, P * loc.sub.N)
        for a in range(4):
            f = int(mesh.tet_faces[K, a])
            s = int(mesh.signs[K, a])
            for q in range(m):
                j = a * m + q
                cen, area = _subface_centroid_area(mesh, f, q)
                col = loc.rhs[:, j]
                assert abs(-s * col.sum() - area) < 1e-14
                assert np.abs(-s * (col @ X) - area * cen).max() < 1e-14
                assert abs(loc.BK[j] - s * area) < 1e-14


@pytest.mark.parametrize("P,r", [(1, 1), (2, 1)])
def test_local3d_zero_mean_and_bordered_equation(P, r):
    mesh = T.build_mesh3d(1, 4)
    rng = np.random.default_rng(11)
    kap = 10.0 ** rng.uniform(-2, 2, 8 ** r)
    loc = T.solve_local3d(mesh, 3, r, P, kap, T.source3d_fn("sinsinsin"))
    A = T.assemble_stiffness3d(loc.sub, kap).toarray()
    vol = _tet_volume(mesh.verts[mesh.tets[3]])
    assert abs(loc.mass.sum() - vol) < 1e-15
    assert np.abs(loc.mass @ loc.eta).max() <= 1e-13 * np.abs(loc.eta).max()
    mu = loc.rhs.sum(axis=0) / vol                            # 1^T A = 0 fixes the border multiplier
    res = A @ loc.eta - (loc.rhs - np.outer(loc.mass, mu))
    assert np.abs(res).max() <= 1e-11 * np.abs(loc.rhs).max()


def _nodal_error(run, u, P):
    err = 0.0
    for K, loc in enumerate(run.locals):
        uh = T.local_u3d(run.mesh, K, loc, run.lam, run.u0)
        X = loc.sub.lattice_to_x(loc.sub.nodes, P * loc.sub.N)
        err = max(err, float(np.abs(uh - u(X[:, 0], X[:, 1], X[:, 2])).max()))
    return err


@pytest.mark.parametrize("P,r,m", [(2, 1, 4), (1, 2, 4), (2, 2, 16), (1, 3, 16)])
def test_exact_linear_recovery_3d(P, r, m):
    """kappa = 1, u linear, f = 0, g = u: the flux -grad u . n is constant on every face, so it
    lies in Lambda_H^{m,0} and the method reproduces u and lambda = -grad u . n exactly.
    (The local traces must outnumber the multipliers: P1 needs N >= 2 sqrt(m).)"""
    grad = np.array([2.0, -3.0, 0.5])
    u = lambda x, y, z: 1.0 + grad[0] * x + grad[1] * y + grad[2] * z
    mesh = T.build_mesh3d(1, m)
    run = T.run3d(1, r, P, m, [np.ones(8 ** r)] * mesh.n_K, 0.0, g=u)
    assert _nodal_error(run, u, P) < 1e-12
    # lambda to 1e-10: with m = 16 the skeleton matrix's spectrum spans 1e3 (small subfaces)
    assert np.abs(run.lam - np.repeat(-(mesh.normals @ grad), m)).max() < 1e-10
    assert np.abs(run.u0).max() < 10.0


def test_exact_layered_recovery_3d():
    """kappa constant on the slabs i/nc < x < (i+1)/nc (1, 100): u = phi(x) + b y + c z with
    kappa phi' the same on every slab solves -div(kappa grad u) = 0; its flux is constant
    on every coarse face, so the method reproduces it."""
    nc, r, P, m = 2, 1, 2, 4
    kap_slab = [1.0, 100.0]
    q, b, c = 3.0, 0.7, -1.1
    x_if = 0.5
    phi = lambda x: np.where(x < x_if, q * x / kap_slab[0], q * x_if / kap_slab[0] + q * (x - x_if) / kap_slab[1])
    u = lambda x, y, z: phi(x) + b * y + c * z
    mesh = T.build_mesh3d(nc, m)
    kap = [np.full(8 ** r, kap_slab[int(mesh.verts[t].mean(axis=0)[0] > x_if)]) for t in mesh.tets]
    run = T.run3d(nc, r, P, m, kap, 0.0, g=u)
    assert _nodal_error(run, u, P) < 1e-11


def test_skeleton3d_symmetric_nsd_and_flux():
    nc, r, P, m = 1, 1, 2, 4
    mesh = T.build_mesh3d(nc, m)
    rng = np.random.default_rng(2)
    kap = [10.0 ** rng.uniform(-1, 1, 8 ** r) for _ in range(mesh.n_K)]
    run = T.run3d(nc, r, P, m, kap, T.source3d_fn("sinsinsin"))
    A = run.A.toarray()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.max() <= 1e-12 * np.abs(ev).max()
    # flux compatibility: sum_F (s lambda, 1)_F = (f, 1)_K on every K (second row of Eq. "mat_global")
    assert np.abs(run.B @ run.lam - run.F).max() <= 1e-11 * max(1.0, np.abs(run.F).max())
    # the assembled system is the brute-force sum of the local blocks
    Ad = np.zeros_like(A)
    for K, loc in enumerate(run.locals):
        ids = mesh.local_lambda(K)
        Ad[np.ix_(ids, ids)] += loc.AK
    assert np.abs(Ad - A).max() == 0.0


def test_convergence_3d_model_problem():
    """The paper's model problem (Sec. 5: kappa = 1, u = sin(2 pi x) sin(2 pi y) sin(2 pi z)):
    the L2 error falls with finer multipliers (m = 4 -> 16) and with a finer coarse mesh."""
    u = lambda x, y, z: np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) * np.sin(2 * np.pi * z)
    f = T.source3d_fn("sinsinsin", 1.0, 2.0)
    err = {}
    for m in (4, 16):
        mesh = T.build_mesh3d(1, m)
        run = T.run3d(1, 2, 2, m, [np.ones(64)] * mesh.n_K, f)
        err[m] = T.errors3d(run.mesh, run.locals, run.lam, run.u0, u)[0]
    assert err[16] < err[4] / 5.0
    assert err[4] < 0.25


def test_dirichlet3d_subface_moments():
    """G_j = (g, psi_j)_F for a linear g is |subface| g(centroid)."""
    g = lambda x, y, z: 1.0 + 2.0 * x - y + 4.0 * z
    mesh = T.build_mesh3d(1, 16)
    G = T.dirichlet_term3d(mesh, g, 4)
    for f in range(mesh.n_f):
        for q in range(16):
            if not mesh.boundary[f]:
                assert G[f * 16 + q] == 0.0
                continue
            cen, area = _subface_centroid_area(mesh, f, q)
            assert abs(G[f * 16 + q] - area * g(*cen)) < 1e-14
