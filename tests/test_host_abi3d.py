"""CPU-side checks of the three-dimensional C ABI (include/mhm3d.h): host-only meshes
(no GPU) reproduce the oracle's connectivity, signs, lattice and sub-tetrahedra bit for
bit, the face-load table rebuilds the oracle's multiplier right-hand sides, the skeleton
pattern is the union of the elements' multiplier pairs, and unstable or oversized
configurations are refused."""
import numpy as np
import pytest

from oracle import tet3d as T
from paper_1703_10435_gb300 import build, mhm


@pytest.fixture(scope="module")
def lib():
    build.build()
    return mhm.lib()


@pytest.mark.parametrize("nc,r,P,m", [(1, 1, 2, 4), (2, 2, 2, 16), (2, 3, 1, 16), (3, 2, 1, 4)])
def test_connectivity_bit_exact(lib, nc, r, P, m):
    M = mhm.Mesh3D(nc, r, P, m, device=-1)
    o = T.build_mesh3d(nc, m)
    assert (M.n_K, M.n_faces, M.n_vertices, M.n_lambda, M.n_I) == (o.n_K, o.n_f, len(o.verts), o.n_lambda, 4 * m)
    assert np.array_equal(M.query(mhm.Q3_TETS, np.int32, 4 * M.n_K).reshape(-1, 4), o.tets)
    assert np.array_equal(M.query(mhm.Q3_TET_FACES, np.int32, 4 * M.n_K).reshape(-1, 4), o.tet_faces)
    assert np.array_equal(M.query(mhm.Q3_TET_SIGNS, np.int8, 4 * M.n_K).reshape(-1, 4), o.signs)
    assert np.array_equal(M.query(mhm.Q3_FACES, np.int32, 3 * M.n_faces).reshape(-1, 3), o.faces)
    assert np.array_equal(M.query(mhm.Q3_VERTICES, np.float64, 3 * M.n_vertices).reshape(-1, 3), o.verts)
    assert np.abs(M.query(mhm.Q3_NORMALS, np.float64, 3 * M.n_faces).reshape(-1, 3) - o.normals).max() < 1e-15


@pytest.mark.parametrize("r,P", [(0, 2), (1, 2), (2, 2), (2, 1), (3, 1)])
def test_lattice_and_sub_tets_bit_exact(lib, r, P):
    m = 4 if r >= 1 and (P == 2 or r >= 2) else 1
    M = mhm.Mesh3D(1, r, P, m, device=-1)
    sub = T.Submesh3D(np.eye(4, 3), r, P)
    assert (M.n_local, M.n_sub) == (sub.n, 8 ** r)
    assert np.array_equal(M.query(mhm.Q3_NODES, np.int32, 3 * M.n_local).reshape(-1, 3), sub.nodes)
    nb = 4 if P == 1 else 10
    assert np.array_equal(M.query(mhm.Q3_SUB_DOFS, np.int32, M.n_sub * nb).reshape(-1, nb), sub.dofs)


def test_quadrature_table_matches_oracle_rule(lib):
    M = mhm.Mesh3D(1, 1, 2, 4, device=-1)
    q = M.query(mhm.Q3_QUAD, np.float64, 64 * 14)
    pts, w = T.duffy_tet(4)
    assert np.abs(q[:256].reshape(64, 4)[:, :3] - pts).max() < 1e-15
    assert np.abs(q[:256].reshape(64, 4)[:, 3] - w).max() < 1e-16
    lam = np.concatenate([1.0 - pts.sum(axis=1, keepdims=True), pts], axis=1)
    assert np.abs(q[256:].reshape(64, 10) - T.basis3d(2, lam)).max() < 1e-15


@pytest.mark.parametrize("nc,r,P,m", [(1, 1, 2, 4), (1, 2, 2, 16), (1, 2, 1, 4), (2, 2, 2, 4)])
def test_face_table_rebuilds_oracle_rhs(lib, nc, r, P, m):
    """-s |fine face| / 3 x count per table entry reproduces the oracle's quadrature of
    N_j = -(s psi_j, phi_w)_{dK} for every element (every face orientation that occurs)."""
    M = mhm.Mesh3D(nc, r, P, m, device=-1)
    o = T.build_mesh3d(nc, m)
    perm = M.query(mhm.Q3_FACE_PERM, np.int8, 4 * M.n_K).reshape(-1, 4)
    off = M.query(mhm.Q3_FTAB_OFF, np.int32, 24 * (m + 1))
    ne = int(off[-1])
    node = M.query(mhm.Q3_FTAB_NODE, np.int16, ne)
    cnt = M.query(mhm.Q3_FTAB_COUNT, np.int8, ne)
    N = 1 << r
    Ks = range(o.n_K) if o.n_K <= 24 else range(0, o.n_K, 7)
    seen = set()
    for K in Ks:
        loc = T.solve_local3d(o, K, r, P, np.ones(8 ** r), 0.0)
        V = o.verts[o.tets[K]]
        rhs = np.zeros((loc.sub.n, 4 * m))
        for a in range(4):
            b = [v for v in range(4) if v != a]
            area = 0.5 * np.linalg.norm(np.cross(V[b[1]] - V[b[0]], V[b[2]] - V[b[0]])) / N ** 2
            p = int(perm[K, a])
            seen.add((a, p))
            for q in range(m):
                base = (a * 6 + p) * (m + 1) + q
                for e in range(off[base], off[base + 1]):
                    rhs[node[e], a * m + q] = -o.signs[K, a] * area / 3.0 * cnt[e]
        assert np.abs(rhs - loc.rhs[:, :4 * m]).max() < 1e-15
    assert len(seen) >= 6     # several face orientations occur (6 of the 24 on one cube)


def test_skeleton_pattern_is_union_of_local_pairs(lib):
    M = mhm.Mesh3D(2, 1, 2, 4, device=-1)
    o = T.build_mesh3d(2, 4)
    rowptr = M.query(mhm.Q3_CSR_ROWPTR, np.int32, M.n_lambda + 1)
    cols = M.query(mhm.Q3_CSR_COLS, np.int32, M.nnz)
    want = [set() for _ in range(o.n_lambda)]
    for K in range(o.n_K):
        ids = o.local_lambda(K)
        for j in ids:
            want[j].update(int(i) for i in ids)
    assert rowptr[-1] == M.nnz == sum(len(w) for w in want)
    for row in range(o.n_lambda):
        got = cols[rowptr[row]:rowptr[row + 1]]
        assert np.array_equal(got, np.array(sorted(want[row])))


@pytest.mark.parametrize("nc,r,P,m", [(1, 1, 1, 4), (1, 2, 1, 16), (1, 1, 2, 16), (1, 2, 2, 8), (0, 1, 2, 4),
                                      (1, 1, 3, 4)])
def test_refusals(lib, nc, r, P, m):
    with pytest.raises(mhm.MHMError) as e:
        mhm.Mesh3D(nc, r, P, m, device=-1)
    assert e.value.code == mhm.MHM_ERR_INVALID_ARG


@pytest.mark.parametrize("case", ["kind", "precision", "it_max", "tol", "range", "null"])
def test_local_solve_argument_errors(lib, case):
    """Arguments are checked before the device: refusals on a host-only mesh (no pointer is
    dereferenced on the host)."""
    import torch
    M = mhm.Mesh3D(1, 1, 2, 4, device=-1)
    t = torch.zeros(8)
    st = torch.zeros(8, dtype=torch.int32)
    src = mhm.Source3D(7 if case == "kind" else mhm.MHM3D_SRC_CONST, 1.0, 2.0)
    kw = dict(stream=type("S", (), {"cuda_stream": 0})())
    if case == "precision":
        kw["precision"] = 5
    if case == "it_max":
        kw["opts"] = mhm.Opts3D(0, 1e-9, 0)
    if case == "tol":
        kw["opts"] = mhm.Opts3D(4, 0.0, 0)
    if case == "range":
        kw["K0"], kw["K1"] = 3, M.n_K + 1
    with pytest.raises(mhm.MHMError) as e:
        mhm.mhm3d_local_solve_batch(M, None if case == "null" else t, src, t, t, t, t, st, **kw)
    assert e.value.code == mhm.MHM_ERR_INVALID_ARG


def test_host_only_mesh_has_no_compute(lib):
    import torch
    M = mhm.Mesh3D(1, 1, 2, 4, device=-1)
    t = torch.zeros(8)
    with pytest.raises(mhm.MHMError) as e:
        mhm.mhm3d_local_solve_batch(M, t, mhm.Source3D(0, 1.0, 2.0), t, t, t, t, torch.zeros(8, dtype=torch.int32),
                                    stream=type("S", (), {"cuda_stream": 0})())
    assert e.value.code == mhm.MHM_ERR_UNSUPPORTED
