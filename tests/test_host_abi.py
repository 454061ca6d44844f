"""CPU-side checks of the C ABI: the library loads, exports every symbol the
header declares, and its host mesh builder reproduces the oracle's
connectivity, signs and multiplier numbering bit for bit (host-only meshes,
no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.mesh import build_mesh
from paper_1703_10435_gb300 import build, mhm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return mhm.lib()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "mhm.h")).read()
    declared = set(re.findall(r"\b(mhm_[a-z_0-9]+)\s*\(", hdr))
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert set(mhm.EXPORTED) <= declared
    hdr3 = open(os.path.join(ROOT, "include", "mhm3d.h")).read()
    declared3 = set(re.findall(r"\b(mhm3d_[a-z_0-9]+)\s*\(", hdr3))
    assert declared3 == set(mhm.EXPORTED_3D)
    for name in declared3:
        assert hasattr(lib, name), name


def _host_mesh(nx, ny, r=2, P=1, m=2, l=1):
    return mhm.Mesh(nx, ny, r, P, m, l, device=-1)


@pytest.mark.parametrize("nx,ny,m,l", [(1, 1, 1, 0), (4, 4, 1, 1), (3, 5, 2, 2), (8, 2, 3, 1)])
def test_connectivity_bit_exact(lib, nx, ny, m, l):
    M = _host_mesh(nx, ny, 2, 1, m, l)
    o = build_mesh(nx, ny, m, l)
    assert (M.n_K, M.n_faces, M.n_vertices, M.n_lambda) == (o.n_K, o.n_e, len(o.verts), o.n_lambda)
    assert np.array_equal(M.query(mhm.Q_TRI_VERTS, np.int32, 3 * M.n_K).reshape(-1, 3), o.tris)
    assert np.array_equal(M.query(mhm.Q_TRI_FACES, np.int32, 3 * M.n_K).reshape(-1, 3), o.tri_edges)
    assert np.array_equal(M.query(mhm.Q_TRI_SIGNS, np.int8, 3 * M.n_K).reshape(-1, 3), o.signs)
    assert np.array_equal(M.query(mhm.Q_FACE_VERTS, np.int32, 2 * M.n_faces).reshape(-1, 2), o.edges)
    assert np.array_equal(M.query(mhm.Q_LAMBDA_OFFSET, np.int64, M.n_faces + 1), o.lam_offset)
    kl = M.query(mhm.Q_K_LAMBDA, np.int32, M.n_K * M.n_I).reshape(M.n_K, M.n_I)
    for K in range(M.n_K):
        assert np.array_equal(kl[K], o.local_lambda(K))
    assert np.array_equal(M.query(mhm.Q_VERTEX_XY, np.float64, 2 * M.n_vertices).reshape(-1, 2), o.verts)
    assert np.array_equal(M.query(mhm.Q_FACE_NORMALS, np.float64, 2 * M.n_faces).reshape(-1, 2), o.normals)


def test_skeleton_pattern_matches_oracle(lib):
    import scipy.sparse
    M = _host_mesh(3, 2, 2, 1, 2, 1)
    o = build_mesh(3, 2, 2, 1)
    rowptr = M.query(mhm.Q_CSR_ROWPTR, np.int32, M.n_lambda + 1)
    cols = M.query(mhm.Q_CSR_COLS, np.int32, M.nnz)
    assert np.all(np.diff(rowptr) > 0)
    for j in range(M.n_lambda):
        c = cols[rowptr[j]:rowptr[j + 1]]
        assert np.all(np.diff(c) > 0)          # strictly ascending columns
    # the oracle's pattern: (j, i) couple iff some K holds both
    want = set()
    for K in range(o.n_K):
        ids = o.local_lambda(K)
        want.update((int(a), int(b)) for a in ids for b in ids)
    got = {(j, int(c)) for j in range(M.n_lambda) for c in cols[rowptr[j]:rowptr[j + 1]]}
    assert got == want


@pytest.mark.parametrize("nx,ny,m", [(3, 2, 1), (4, 3, 2)])
def test_per_face_degree_numbering_matches_oracle(lib, nx, ny, m):
    """A multiplier degree per face: offsets, the per-K slots (face a at a d + u, d =
    m(l_max+1), unused slots -1) and the skeleton pattern against the oracle's mesh."""
    rng = np.random.default_rng(5 + nx)
    ne = nx * (ny + 1) + ny * (nx + 1) + nx * ny
    lf = rng.integers(0, 4, ne).astype(np.int8)
    M = mhm.Mesh(nx, ny, 2, 1, m, 0, device=-1, l_per_face=lf)
    o = build_mesh(nx, ny, m, lf)
    d = m * (int(lf.max()) + 1)
    assert (M.n_faces, M.n_lambda, M.n_I) == (o.n_e, o.n_lambda, 3 * d)
    assert np.array_equal(M.face_degree, lf)
    assert np.array_equal(M.query(mhm.Q_LAMBDA_OFFSET, np.int64, M.n_faces + 1), o.lam_offset)
    kl = M.query(mhm.Q_K_LAMBDA, np.int32, M.n_K * M.n_I).reshape(M.n_K, M.n_I)
    for K in range(M.n_K):
        used = []
        for a in range(3):
            e = int(o.tri_edges[K, a])
            n = m * (int(lf[e]) + 1)
            assert np.array_equal(kl[K, a * d:a * d + n], o.lam_offset[e] + np.arange(n))
            assert np.all(kl[K, a * d + n:(a + 1) * d] == -1)
            used.extend(kl[K, a * d:a * d + n])
        assert np.array_equal(used, o.local_lambda(K))
    rowptr = M.query(mhm.Q_CSR_ROWPTR, np.int32, M.n_lambda + 1)
    cols = M.query(mhm.Q_CSR_COLS, np.int32, M.nnz)
    want = set()
    for K in range(o.n_K):
        ids = o.local_lambda(K)
        want.update((int(a), int(b)) for a in ids for b in ids)
    got = {(j, int(c)) for j in range(M.n_lambda) for c in cols[rowptr[j]:rowptr[j + 1]]}
    assert got == want
    for j in range(M.n_lambda):
        assert np.all(np.diff(cols[rowptr[j]:rowptr[j + 1]]) > 0)


def test_errors_are_reported(lib):
    with pytest.raises(mhm.MHMError) as e:
        mhm.Mesh(0, 1, 2, 1, 1, 1, device=-1)
    assert e.value.code == mhm.MHM_ERR_INVALID_ARG and "nx" in str(e.value)
    with pytest.raises(mhm.MHMError) as e:
        mhm.Mesh(1, 1, 2, 3, 1, 1, device=-1)
    assert e.value.code == mhm.MHM_ERR_INVALID_ARG
    M = _host_mesh(2, 2)
    # compute calls on a host-only mesh fail loudly instead of falling back
    code = lib.mhm_local_solve_batch(M.handle, None, None, 0, None, None, None, None, None, None, None,
                                     None, 0, None)
    assert code == mhm.MHM_ERR_UNSUPPORTED
    code = lib.mhm_local_solve_waves(M.handle, None, 0, None, 0, None, None, None, None, None, None, None,
                                     None, 0, None, None)
    assert code == mhm.MHM_ERR_UNSUPPORTED
    # a degree per face: negative degrees and more than 16 multipliers per face are refused
    ne = 2 * 3 + 2 * 3 + 4
    with pytest.raises(mhm.MHMError) as e:
        mhm.Mesh(2, 2, 2, 1, 1, 0, device=-1, l_per_face=[-1] + [1] * (ne - 1))
    assert e.value.code == mhm.MHM_ERR_INVALID_ARG
    with pytest.raises(mhm.MHMError) as e:
        mhm.Mesh(2, 2, 2, 1, 4, 0, device=-1, l_per_face=[4] + [1] * (ne - 1))
    assert e.value.code == mhm.MHM_ERR_INVALID_ARG


def test_per_element_levels_queries():
    """A level per K: the queries give each K's level, its kappa block (4^r_K values)
    and its block of nodal values (n_local of its level), in K order."""
    from paper_1703_10435_gb300 import mhm
    rng = np.random.default_rng(11)
    rs = rng.integers(0, 5, 2 * 3 * 2)
    for P in (1, 2):
        m = mhm.Mesh(3, 2, 0, P, 1, 1, device=-1, r_per_K=rs)
        assert np.array_equal(m.r_of_K, rs)
        N = 2 ** rs.astype(np.int64)
        assert np.array_equal(m.kappa_offset, np.concatenate([[0], np.cumsum(N * N)]))
        nloc = (P * N + 1) * (P * N + 2) // 2
        assert np.array_equal(m.nodal_offset, np.concatenate([[0], np.cumsum(nloc)]))
        assert m.n_fine == int((N * N).max()) and m.n_local == int(nloc.max())
        # the skeleton does not depend on the levels
        u = mhm.Mesh(3, 2, 2, P, 1, 1, device=-1)
        assert (m.n_lambda, m.n_I, m.nnz) == (u.n_lambda, u.n_I, u.nnz)
        assert np.array_equal(u.kappa_offset, np.arange(13) * 16) and np.all(u.r_of_K == 2)


def test_per_element_levels_reject_out_of_range():
    from paper_1703_10435_gb300 import mhm
    with pytest.raises(mhm.MHMError):
        mhm.Mesh(1, 1, 0, 1, 1, 1, device=-1, r_per_K=[3, 8])


@pytest.mark.parametrize("nx,ny,m,l,per_face", [(1, 1, 1, 0, False), (3, 2, 4, 3, False), (4, 3, 2, 2, True)])
def test_system_count_equals_built_pattern(lib, nx, ny, m, l, per_face):
    """The entry count behind mhm_create_mesh's int32 guard equals the saddle-point CSR
    the mesh then builds (uniform degree and a degree per face)."""
    lf = None
    if per_face:
        ne = nx * (ny + 1) + ny * (nx + 1) + nx * ny
        lf = np.random.default_rng(3).integers(0, l + 1, ne)
    M = mhm.Mesh(nx, ny, 2, 1, m, l, -1, None, lf)
    counted, built = M.query(mhm.Q_SYSTEM_NNZ, np.int64, 2)
    assert counted == built > 0


def test_mesh_beyond_int32_entries_refused(lib):
    """760 x 760 squares with 16 multipliers per face: about 2.2e9 saddle-point entries,
    beyond int32 indexing; refused with INVALID_ARG before any table of that size exists."""
    with pytest.raises(mhm.MHMError) as ei:
        mhm.Mesh(760, 760, 1, 1, 4, 3, -1)
    assert ei.value.code == mhm.MHM_ERR_INVALID_ARG and "2^31" in str(ei.value)
