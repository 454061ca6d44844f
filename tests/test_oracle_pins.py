"""Pins of the FP64 oracle against facts fixed by the paper and by the
mathematics, not by the oracle itself: closed forms, invariants, exact
recovery of solutions that lie in the discrete spaces, convergence rates and
brute-force dense solves.  CPU only."""
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import globalsys, reconstruct
from oracle.fem import Submesh, basis_grad_ref, lattice_points, n_local
from oracle.local import assemble_stiffness, cell_integrals, solve_local
from oracle.mesh import build_mesh
from oracle.quadrature import duffy_triangle, gauss_legendre_01
from oracle.run import run, source_fn
from _golden import dirichlet_moment, legendre_golden

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden_matrices():
    mats, cur, den = {}, None, None
    for line in open(os.path.join(GOLDEN, "reference_elements.txt")):
        if line.startswith("#") or not line.strip():
            continue
        tok = line.split()
        if tok[0] in ("P1", "P2"):
            cur, den = tok[0], float(tok[2])
            mats[cur] = []
            continue
        mats[cur].append([float(t) / den for t in tok])
    return {k: np.array(v) for k, v in mats.items()}


def _table(section):
    out, cur = [], None
    for line in open(os.path.join(GOLDEN, "mesh_counts.txt")):
        if line.startswith("#") or not line.strip():
            continue
        if line.startswith("["):
            cur = line[1:line.index("]")]
            continue
        if cur == section:
            out.append([int(t) for t in line.split()])
    return out


# --------------------------------------------------------------- quadrature
@pytest.mark.parametrize("p,q", [(a, b) for a in range(7) for b in range(7) if a + b <= 6])
def test_duffy_rule_exact_monomials(p, q):
    # int_ref xi^p eta^q = p! q! / (p+q+2)!
    pts, w = duffy_triangle(4)
    got = float(np.sum(w * pts[:, 0] ** p * pts[:, 1] ** q))
    exact = math.factorial(p) * math.factorial(q) / math.factorial(p + q + 2)
    assert got == pytest.approx(exact, rel=1e-13, abs=1e-16)


def test_gauss_legendre_exact():
    x, w = gauss_legendre_01(3)
    for k in range(6):
        assert float(np.sum(w * x ** k)) == pytest.approx(1.0 / (k + 1), rel=1e-14)


# --------------------------------------------------------------- mesh
def test_mesh_counts_closed_form():
    for nx, ny, nK, ne in _table("faces"):
        assert 2 * nx * ny == nK and nx * (ny + 1) + ny * (nx + 1) + nx * ny == ne
        if nK <= 2048:
            m = build_mesh(nx, ny)
            assert m.n_K == nK and m.n_e == ne
            assert len(m.verts) - m.n_e + m.n_K == 1          # Euler


def test_mesh_orientation_and_signs():
    m = build_mesh(3, 2)
    assert int(m.boundary.sum()) == 2 * (3 + 2)
    for e in range(m.n_e):
        assert abs(np.linalg.norm(m.normals[e]) - 1) < 1e-14
        Ks = m.edge_tris[e]
        ss = [m.signs[K, list(m.tri_edges[K]).index(e)] for K in Ks]
        if m.boundary[e]:
            assert ss == [1]
            mid = 0.5 * (m.verts[m.edges[e, 0]] + m.verts[m.edges[e, 1]])
            assert float(m.normals[e] @ (mid - 0.5)) > 0      # outward on the unit square
        else:
            assert sorted(ss) == [-1, 1] and Ks == sorted(Ks)
    # every triangle is CCW and local face a is opposite local vertex a
    for K in range(m.n_K):
        v = m.verts[m.tris[K]]
        d1, d2 = v[1] - v[0], v[2] - v[0]
        assert d1[0] * d2[1] - d1[1] * d2[0] > 0
        for a in range(3):
            assert m.tris[K, a] not in m.edges[m.tri_edges[K, a]]


def test_lattice_sizes():
    for P, r, n, nb in _table("lattice"):
        N = 1 << r
        assert n_local(P, N) == n
        pts = lattice_points(P * N)
        on_bdry = (pts[:, 0] == 0) | (pts[:, 1] == 0) | (pts[:, 0] + pts[:, 1] == P * N)
        assert len(pts) == n and int(on_bdry.sum()) == nb


# --------------------------------------------------------------- elements
@pytest.mark.parametrize("P", [1, 2])
def test_reference_stiffness_golden(P):
    gold = _read_golden_matrices()["P%d" % P]
    sub = Submesh(np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]), 0, P)
    A = assemble_stiffness(sub, np.ones(1)).toarray()
    d = sub.dofs[0]                      # element node order A,B,C(,BC,CA,AB) -> lattice DOF ids
    assert np.allclose(A[np.ix_(d, d)], gold, atol=1e-14)


@pytest.mark.parametrize("P", [1, 2])
def test_stiffness_invariants(P):
    rng = np.random.default_rng(0)
    v = np.array([[0.1, 0.2], [0.7, 0.25], [0.3, 0.9]])
    sub = Submesh(v, 3, P)
    kap = 10.0 ** rng.uniform(-2, 2, sub.tri_xy.shape[0])
    A = assemble_stiffness(sub, kap).toarray()
    assert np.allclose(A, A.T, atol=1e-12)
    assert np.abs(A.sum(axis=1)).max() < 1e-11 * np.abs(A).max()        # constants in the kernel
    ev = np.linalg.eigvalsh(A)
    assert ev[0] > -1e-10 * ev[-1] and ev[1] > 1e-10 * ev[-1]         # PSD with a 1-D kernel
    # energy of a linear function: a(x, x) = sum_T kappa_T |T| for grad x = (1,0)
    lin = sub.node_xy[:, 0]
    assert float(lin @ A @ lin) == pytest.approx(float(np.sum(kap * sub.area)), rel=1e-12)


def test_mass_vector_closed_form():
    v = np.array([[0.0, 0.0], [0.25, 0.0], [0.25, 0.25]])
    sub = Submesh(v, 3, 1)
    m, load, FK = cell_integrals(sub, 2.0)
    area = 0.5 * 0.25 * 0.25
    assert m.sum() == pytest.approx(area, rel=1e-14)
    count = np.zeros(sub.n)
    np.add.at(count, sub.dofs, 1)
    assert np.allclose(m, count * sub.area[0] / 3.0, rtol=1e-13)
    assert FK == pytest.approx(2.0 * area, rel=1e-14) and np.allclose(load, 2 * m)
    sub2 = Submesh(v, 2, 2)
    m2, _, _ = cell_integrals(sub2, 1.0)
    pts = lattice_points(sub2.PN)
    vertex = (pts[:, 0] % 2 == 0) & (pts[:, 1] % 2 == 0)
    assert np.abs(m2[vertex]).max() < 1e-16 and m2.sum() == pytest.approx(area, rel=1e-14)


# --------------------------------------------------------------- local problems
def _local_case(P=1, r=2, m=2, l=1, seed=1):
    mesh = build_mesh(2, 2, m, l)
    rng = np.random.default_rng(seed)
    kap = 10.0 ** rng.uniform(-2, 2, (1 << r) ** 2)
    f = source_fn("sinsin", 1.0, 1.0)
    return mesh, solve_local(mesh, 3, r, P, kap, f), kap


@pytest.mark.parametrize("P", [1, 2])
def test_local_solutions_zero_mean_and_equation(P):
    """eta in V_0^perp (int_K eta = 0) and a(eta, w) = (g, w) for every zero-mean
    w, i.e. A eta - g is a multiple of the mass vector m."""
    mesh, loc, kap = _local_case(P)
    A = assemble_stiffness(loc.sub, kap).toarray()
    assert np.abs(loc.mass @ loc.eta).max() < 1e-13 * np.abs(loc.eta).max()
    d = A @ loc.eta - loc.rhs
    mu = (loc.mass @ d) / (loc.mass @ loc.mass)
    assert np.abs(d - np.outer(loc.mass, mu)).max() < 1e-11 * np.abs(loc.rhs).max()
    # the multiplier loads integrate to -B_K: sum_w N_i[w] = -(s psi_i, 1)_{dK}
    n_I = loc.AK.shape[0]
    assert np.allclose(loc.rhs[:, :n_I].sum(axis=0), -loc.BK, atol=1e-15)


def test_local_bordered_vs_pseudoinverse():
    """The bordered solve equals the pseudo-inverse route: project g onto
    1^T g = 0, take the minimum-norm least-squares solution, shift to zero mean."""
    mesh, loc, kap = _local_case(1, 3, 2, 2, seed=3)
    A = assemble_stiffness(loc.sub, kap).toarray()
    m = loc.mass
    area = m.sum()
    gt = loc.rhs - np.outer(m, loc.rhs.sum(axis=0) / area)
    z = np.linalg.lstsq(A, gt, rcond=None)[0]
    z -= np.outer(np.ones(len(m)), (m @ z) / area)
    assert np.allclose(z, loc.eta, rtol=0, atol=1e-10 * np.abs(z).max())


def test_local_face_integrals_structure():
    mesh, loc, kap = _local_case(1, 3, 2, 2)
    AK = loc.AK
    assert np.abs(AK - AK.T).max() < 1e-12 * np.abs(AK).max()             # symmetric
    ev = np.linalg.eigvalsh(0.5 * (AK + AK.T))
    assert ev.max() < 1e-12 * np.abs(ev).max()                              # negative semidefinite
    # B_K[j] = s |F| / m for p = 0, zero for p > 0 (int of P_p over a subface)
    K = 3
    j = 0
    for a in range(3):
        e = mesh.tri_edges[K, a]
        length = np.linalg.norm(mesh.verts[mesh.edges[e, 1]] - mesh.verts[mesh.edges[e, 0]])
        for q in range(mesh.m_e[e]):
            for p in range(mesh.l_e[e] + 1):
                want = mesh.signs[K, a] * length / mesh.m_e[e] if p == 0 else 0.0
                assert loc.BK[j] == pytest.approx(want, abs=1e-15)
                j += 1


def test_local_gram_identity():
    """A_K = -Y^T Y and E_K = Y^T y_f with Y = L^{-1} N~, y_f = L^{-1} f~ (Cholesky
    of the system pinned at DOF 0, loads projected onto 1^T g = 0): a second
    route to the face integrals, which the oracle takes by trace quadrature."""
    mesh, loc, kap = _local_case(1, 3, 2, 2)
    A = assemble_stiffness(loc.sub, kap).toarray()
    m = loc.mass
    n_I = loc.AK.shape[0]
    gt = loc.rhs - np.outer(m, loc.rhs.sum(axis=0) / m.sum())
    Lc = np.linalg.cholesky(A[1:, 1:])
    Y = scipy.linalg.solve_triangular(Lc, gt[1:], lower=True)
    scale = np.abs(loc.AK).max()
    assert np.allclose(-Y[:, :n_I].T @ Y[:, :n_I], loc.AK, rtol=0, atol=1e-10 * scale)
    assert np.allclose(Y[:, :n_I].T @ Y[:, n_I], loc.EK, rtol=0, atol=1e-10 * np.abs(loc.EK).max())


def test_cell_integral_sinsin_closed_form():
    mesh = build_mesh(4, 4, 1, 1)
    f = source_fn("sinsin", 1.0, 1.0)
    loc = solve_local(mesh, 5, 3, 1, np.ones(64), f)
    # K = 5 is the upper triangle of square (2, 0); by the x<->y symmetry of sin sin
    # it carries half of the square's integral.
    i, j = 2, 0
    sx = (math.cos(math.pi * i / 4) - math.cos(math.pi * (i + 1) / 4)) / math.pi
    sy = (math.cos(math.pi * j / 4) - math.cos(math.pi * (j + 1) / 4)) / math.pi
    full = 2 * math.pi ** 2 * sx * sy
    lower = solve_local(mesh, 4, 3, 1, np.ones(64), f).FK
    assert lower + loc.FK == pytest.approx(full, rel=1e-11)


# --------------------------------------------------------------- global problem
def _max_nodal_error(o, exact):
    err = 0.0
    for K, loc in enumerate(o.locals):
        u = reconstruct.local_u(o.mesh, K, loc, o.lam, o.u0)
        err = max(err, float(np.abs(u - exact(loc.sub.node_xy[:, 0], loc.sub.node_xy[:, 1])).max()))
    return err


def test_exact_linear_recovery_config1():
    """kappa = 1, u = 1 + 2x - 3y: the flux is constant per face, so it lies in
    Lambda_H and the P1 locals reproduce u exactly."""
    g = lambda x, y: 1 + 2 * x - 3 * y
    o = run(4, 4, 3, 1, 1, 1, np.ones((32, 64)), 0.0, g=g)
    assert _max_nodal_error(o, g) < 1e-12


@pytest.mark.parametrize("P,m,l", [(1, 1, 0), (1, 2, 1), (2, 1, 0), (2, 3, 1)])
def test_exact_recovery_layered_heterogeneous(P, m, l):
    """kappa(y) piecewise constant on horizontal strips of height h = H/N (every
    fine triangle lies in one strip), f = 0, u(y) = int_0^y 1/kappa: the flux
    kappa u' = 1 is constant, u is piecewise linear on the submesh, so the
    method is exact for any contrast."""
    from paper_1703_10435_gb300 import workloads as W
    nx = ny = 2
    r = 2
    N = 1 << r
    cen = W.fine_centroids(W.coarse_vertices(nx, ny), N)
    hs = 1.0 / (ny * N)
    ks = 10.0 ** (-2 + 4 * W.uniform01(5, np.arange(ny * N, dtype=np.uint64), 0, 0))
    kap = ks[np.floor(cen[..., 1] / hs).astype(int)]
    cum = np.concatenate([[0.0], np.cumsum(hs / ks)])

    def u(x, y):
        y = np.asarray(y, dtype=float)
        s = np.clip(np.floor(y / hs).astype(int), 0, ny * N - 1)
        return cum[s] + (y - s * hs) / ks[s]

    o = run(nx, ny, r, P, m, l, kap, 0.0, g=u)
    assert _max_nodal_error(o, u) < 1e-11 * cum[-1]


def test_exact_quadratic_recovery_p2():
    u = lambda x, y: x ** 2 - 2 * x * y + 3 * y ** 2 + x
    o = run(2, 2, 2, 2, 1, 1, np.ones((8, 16)), -8.0, g=u)
    assert _max_nodal_error(o, u) < 1e-12
    # P1 locals cannot represent it: the pin would catch a P2 path silently using P1
    o1 = run(2, 2, 2, 1, 1, 1, np.ones((8, 16)), -8.0, g=u)
    assert _max_nodal_error(o1, u) > 1e-4


def test_skeleton_symmetric_negative_definite_and_flux():
    rng = np.random.default_rng(7)
    kap = 10.0 ** rng.uniform(-2, 2, (8, 16))
    o = run(2, 2, 2, 1, 1, 1, kap, 1.0)
    A = o.A.toarray()
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.max() < -1e-8 * np.abs(ev).max()          # definite: 2 DOFs/face vs 5 trace nodes
    # with as many multiplier DOFs per K as boundary nodes (m=2, l=1 on N=4) A keeps
    # a kernel but stays negative semidefinite
    o2 = run(2, 2, 2, 1, 2, 1, kap, 1.0)
    ev2 = np.linalg.eigvalsh(o2.A.toarray())
    assert ev2.max() < 1e-12 * np.abs(ev2).max()
    # second equation of Eq. "global": sum_F (s lambda, 1)_F = (f, 1)_K on every K
    assert np.abs(o.B @ o.lam - o.F).max() < 1e-12


@pytest.mark.parametrize("nx", [1, 2])
def test_brute_force_dense_saddle_point(nx):
    rng = np.random.default_rng(nx)
    kap = 10.0 ** rng.uniform(-1, 1, (2 * nx * nx, 16))
    o = run(nx, nx, 2, 1, 1, 1, kap, source_fn("sinsin"), g=lambda x, y: x * y)
    A, B = o.A.toarray(), o.B.toarray()
    L = A.shape[0]
    M = np.block([[A, B.T], [B, np.zeros((B.shape[0], B.shape[0]))]])
    x = np.linalg.solve(M, np.concatenate([o.E + o.G, o.F]))
    assert np.allclose(x[:L], o.lam, rtol=0, atol=1e-11 * np.abs(x).max())
    assert np.allclose(x[L:], o.u0, rtol=0, atol=1e-11 * np.abs(x).max())


@pytest.mark.slow
def test_convergence_rates_sinsin():
    """u = sin(pi x) sin(pi y), kappa = 1, fixed r = 3 (h proportional to H):
    L2 error ~ H^2 and broken H1 error ~ H (P1 locals dominate)."""
    ex = lambda x, y: np.sin(math.pi * x) * np.sin(math.pi * y)
    exg = lambda x, y: (math.pi * np.cos(math.pi * x) * np.sin(math.pi * y),
                        math.pi * np.sin(math.pi * x) * np.cos(math.pi * y))
    e = []
    for nx in (2, 4, 8, 16):
        o = run(nx, nx, 3, 1, 1, 1, np.ones((2 * nx * nx, 64)), source_fn("sinsin"))
        e.append(reconstruct.errors(o.mesh, o.locals, o.lam, o.u0, ex, exg))
    e = np.array(e)
    rates = np.log2(e[:-1] / e[1:])
    assert 1.8 < rates[-1, 0] < 2.3, rates
    assert 0.9 < rates[-1, 1] < 1.15, rates


# ---- refinement level per coarse element (the multipliers live on the coarse faces;
# every element's submesh is its own)

def test_per_element_levels_equal_uniform():
    """A per-element level list that is uniform gives the uniform run's system exactly."""
    rng = np.random.default_rng(3)
    kap = 10.0 ** rng.uniform(-1, 1, (8, 16))
    a = run(2, 2, 2, 1, 1, 1, kap, 1.0)
    b = run(2, 2, [2] * 8, 1, 1, 1, list(kap), 1.0)
    assert np.array_equal(a.A.toarray(), b.A.toarray()) and np.array_equal(a.E, b.E)
    assert np.array_equal(a.lam, b.lam)


def test_per_element_levels_exact_linear():
    """kappa = 1, u linear: exact on every submesh, whatever each element's level."""
    g = lambda x, y: 1 + 2 * x - 3 * y
    rng = np.random.default_rng(4)
    rs = rng.integers(1, 4, 18)
    o = run(3, 3, rs, 1, 1, 1, [np.ones(4 ** int(r)) for r in rs], 0.0, g=g)
    assert _max_nodal_error(o, g) < 1e-12
    assert sorted(set(len(loc.eta) for loc in o.locals)) == sorted(set((2 ** int(r) + 1) * (2 ** int(r) + 2) // 2 for r in rs))


@pytest.mark.parametrize("P", [1, 2])
def test_per_element_levels_exact_layered(P):
    """Layered kappa on strips of height H / 2^r_min with f = 0 and u(y) = int 1/kappa:
    every fine triangle of every element lies in one strip, so the method is exact
    with elements of different levels side by side."""
    from paper_1703_10435_gb300 import workloads as W
    nx = ny = 2
    rng = np.random.default_rng(5)
    rs = rng.integers(1, 4, 2 * nx * ny)
    rmin = int(rs.min())
    hs = 1.0 / (ny * (1 << rmin))
    ks = 10.0 ** (-2 + 4 * W.uniform01(6, np.arange(ny * (1 << rmin), dtype=np.uint64), 0, 0))
    kap = []
    for K, r in enumerate(rs):
        cen = W.fine_centroids(W.coarse_vertices(nx, ny), 1 << int(r))[K]
        kap.append(ks[np.floor(cen[..., 1] / hs).astype(int)])
    cum = np.concatenate([[0.0], np.cumsum(hs / ks)])

    def u(x, y):
        y = np.asarray(y, dtype=float)
        s = np.clip(np.floor(y / hs).astype(int), 0, len(ks) - 1)
        return cum[s] + (y - s * hs) / ks[s]

    o = run(nx, ny, rs, P, 1, 1, kap, 0.0, g=u)
    assert _max_nodal_error(o, u) < 1e-11 * cum[-1]


def test_per_face_degree_uniform_equals_scalar():
    """A per-face degree array with one value gives the scalar-degree run's system exactly."""
    rng = np.random.default_rng(8)
    kap = 10.0 ** rng.uniform(-1, 1, (8, 16))
    a = run(2, 2, 2, 1, 2, 1, kap, 1.0)
    ne = 2 * 3 + 2 * 3 + 4
    b = run(2, 2, 2, 1, 2, np.ones(ne, dtype=np.int64), kap, 1.0)
    assert np.array_equal(a.A.toarray(), b.A.toarray()) and np.array_equal(a.E, b.E)
    assert np.array_equal(a.lam, b.lam)


@pytest.mark.parametrize("m,lmax", [(1, 3), (2, 1)])
def test_per_face_degree_exact_linear_and_layered(m, lmax):
    """Degrees 0..lmax face by face, levels 2..4 element by element: kappa = 1 with u
    linear, and layered kappa with u(y) = int 1/kappa (flux constant per face, so it lies in
    every face's space), are both reproduced exactly.  Every face keeps m(l_e+1) <= 4
    multipliers against the >= 5 trace nodes of a level-2 submesh (a richer multiplier
    space than the trace makes the saddle-point system singular)."""
    from paper_1703_10435_gb300 import workloads as W
    nx = ny = 3
    ne = nx * (ny + 1) + ny * (nx + 1) + nx * ny
    rng = np.random.default_rng(9 + m)
    lf = rng.integers(0, lmax + 1, ne)
    rs = rng.integers(2, 5, 2 * nx * ny)
    g = lambda x, y: 1 + 2 * x - 3 * y
    o = run(nx, ny, rs, 1, m, lf, [np.ones(4 ** int(r)) for r in rs], 0.0, g=g)
    assert sorted(set(int(v) for v in o.mesh.l_e)) == list(range(lmax + 1))
    assert _max_nodal_error(o, g) < 1e-12
    rmin = int(rs.min())
    hs = 1.0 / (ny * (1 << rmin))
    ks = 10.0 ** (-2 + 4 * W.uniform01(7, np.arange(ny * (1 << rmin), dtype=np.uint64), 0, 0))
    kap = []
    for K, r in enumerate(rs):
        cen = W.fine_centroids(W.coarse_vertices(nx, ny), 1 << int(r))[K]
        kap.append(ks[np.floor(cen[..., 1] / hs).astype(int)])
    cum = np.concatenate([[0.0], np.cumsum(hs / ks)])

    def u(x, y):
        y = np.asarray(y, dtype=float)
        s = np.clip(np.floor(y / hs).astype(int), 0, len(ks) - 1)
        return cum[s] + (y - s * hs) / ks[s]

    o = run(nx, ny, rs, 1, m, lf, kap, 0.0, g=u)
    assert _max_nodal_error(o, u) < 1e-11 * cum[-1]


def test_per_face_degree_exact_quadratic_p2():
    """P2 locals, levels 1..3 element by element, degrees 1..3 face by face: the flux of a
    quadratic u is linear along every face, so it lies in every face's space (l_e >= 1), and
    u is reproduced exactly (m(l_e+1) <= 4 against the >= 5 P2 trace nodes of a level-1
    face keeps the system nonsingular).  Degree 0 on one face breaks the exactness."""
    u = lambda x, y: x ** 2 - 2 * x * y + 3 * y ** 2 + x
    nx = ny = 2
    ne = nx * (ny + 1) + ny * (nx + 1) + nx * ny
    rng = np.random.default_rng(12)
    lf = rng.integers(1, 4, ne)
    rs = rng.integers(1, 4, 2 * nx * ny)
    kap = [np.ones(4 ** int(r)) for r in rs]
    o = run(nx, ny, rs, 2, 1, lf, kap, -8.0, g=u)
    assert sorted(set(int(v) for v in o.mesh.l_e)) == [1, 2, 3]
    assert _max_nodal_error(o, u) < 1e-11
    lf0 = lf.copy()
    lf0[[e for e in range(ne) if not o.mesh.boundary[e]][0]] = 0   # one interior face at degree 0
    o0 = run(nx, ny, rs, 2, 1, lf0, kap, -8.0, g=u)
    assert _max_nodal_error(o0, u) > 1e-6


# --------------------------------------------------------------- Legendre basis
def test_legendre_golden_values_norms_moments():
    """The multiplier basis P_p of Lambda_H^{m,l} (Sec. 2, definition (i)) against the
    closed forms: point values (a wrong recurrence coefficient or normalisation moves
    P_2(1/2) = -1/8 and P_3(1/2) = -7/16), the norms 2/(2p+1) and the moments."""
    from oracle.mesh import legendre
    gold = legendre_golden()
    for row in gold["values"]:
        x, vals = row[0], row[1:]
        for p, v in enumerate(vals):
            assert float(legendre(p, x)) == pytest.approx(v, abs=1e-15), (p, x)
    xg, wg = np.polynomial.legendre.leggauss(8)
    for p, v in gold["norms"].items():
        assert float(np.sum(wg * legendre(p, xg) ** 2)) == pytest.approx(v, rel=1e-14)
    for (k, p), v in gold["moments"].items():
        assert float(np.sum(wg * xg ** k * legendre(p, xg))) == pytest.approx(v, abs=1e-14)


@pytest.mark.parametrize("m,l", [(1, 0), (2, 2), (3, 3)])
def test_dirichlet_term_face_moments(m, l):
    """The oracle's boundary term (g, psi_j)_F (Eq. "global" with u = g on the boundary)
    for g = x^2 + y^2 equals the closed form built from the Legendre moments: pins the
    basis normalisation, the direction of xi on every boundary face and the subface
    coordinates."""
    gold = legendre_golden()
    mesh = build_mesh(2, 3, m, l)
    G = globalsys.dirichlet_term(mesh, lambda x, y: x * x + y * y, 4)
    for e in range(mesh.n_e):
        for q in range(m):
            for p in range(l + 1):
                j = mesh.lam_offset[e] + q * (l + 1) + p
                want = dirichlet_moment(mesh, e, q, p, m, gold) if mesh.boundary[e] else 0.0
                assert G[j] == pytest.approx(want, abs=1e-14), (e, q, p)
