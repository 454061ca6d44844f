"""A refinement level per coarse element (each local problem on its own submesh;
the multipliers on the coarse faces): every K against the oracle on a small mesh
with levels 1..7, exact recovery through the whole pipeline, and the uneven
channel workload at full size sampled per level.  Level 7 (256-row level window)
runs the global-memory window of the FP64 path."""
from types import SimpleNamespace

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.local import solve_local
from oracle.mesh import build_mesh
from oracle.run import run
from paper_1703_10435_gb300 import mhm, workloads as W
from _blocks import assert_blocks, gram_entry_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_10435_gb300 import build
    build.build()


def _levels_case():
    nx = ny = 3
    rng = np.random.default_rng(21)
    rs = rng.integers(1, 6, 2 * nx * ny).astype(np.int8)
    rs[[4, 11]] = 6                                   # two level-6 locals (64-wide levels)
    rs[7] = 7                                         # one level-7 local (8385 unknowns)
    kap = [10.0 ** rng.uniform(-2, 2, 4 ** int(r)) for r in rs]
    return nx, ny, rs, kap


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _degrees(tri_faces, rs):
    """Per-face multiplier degrees by the level recipe on one side's own face numbering."""
    tf = np.asarray(tri_faces).reshape(-1, 3)
    rmax = np.zeros(int(tf.max()) + 1, dtype=np.int64)
    np.maximum.at(rmax, tf.ravel(), np.repeat(np.asarray(rs, dtype=np.int64), 3))
    return W.face_degree_from_levels(rmax)


def _slots(mesh, K, m, d, blk):
    """The oracle's per-K vector or matrix (local multipliers face by face, m(l_a+1) each)
    in the library's slot layout: face a at a d .. a d + m(l_a+1) - 1, zeros elsewhere."""
    idx = []
    for a in range(3):
        e = int(mesh.tri_edges[K, a])
        idx.extend(a * d + np.arange(m * (int(mesh.l_e[e]) + 1)))
    idx = np.asarray(idx)
    blk = np.asarray(blk)
    if blk.ndim == 2:
        out = np.zeros((3 * d, 3 * d))
        out[np.ix_(idx, idx)] = blk
    else:
        out = np.zeros(3 * d)
        out[idx] = blk
    return out


def _fp64_bound(o, kap, base):
    """base, or the FP64 error bound 10 u cond(A) (u = 2^-53; cond on the mean-zero space,
    from the largest and the smallest non-zero eigenvalue) where that is larger: two FP64
    solvers (dense or sparse LU in the oracle, pinned Cholesky on the GPU) agree only to
    about that."""
    import scipy.sparse.linalg as sla
    from oracle.local import assemble_stiffness
    A = assemble_stiffness(o.sub, kap)
    if A.shape[0] <= 2500:
        ev = np.linalg.eigvalsh(A.toarray())
        lo, hi = ev[1], ev[-1]
    else:
        hi = float(sla.eigsh(A, k=1, which="LA", return_eigenvectors=False)[0])
        # the two eigenvalues nearest a small negative shift: 0 (constants) and the smallest non-zero
        ev = np.sort(sla.eigsh(A, k=2, sigma=-1e-6 * hi, which="LM", return_eigenvectors=False))
        lo = float(ev[1])
    return max(base, 10 * 2.0 ** -53 * hi / lo)


# the mixed path at the refinement tolerance of the other mixed parity tests (1e-13)
OPTS_PARITY = mhm.SolveOpts(10, 1e-13, 0, 0)


@pytest.mark.parametrize("precision,tol", [(mhm.MHM_FP64, 1e-10), (mhm.MHM_MIXED, 1e-9)])
def test_levels_every_element_vs_oracle(precision, tol):
    from paper_1703_10435_gb300.pipeline import Pipeline
    nx, ny, rs, kap = _levels_case()
    m, l = 1, 2
    p = Pipeline(nx, ny, 0, 1, m, l, 0, precision, r_per_K=rs)
    kd = torch.as_tensor(np.concatenate(kap), device="cuda")
    src = mhm.Source(mhm.MHM_SRC_CONST, 1.0, 1.0)
    p.local(kd, src, OPTS_PARITY)
    torch.cuda.synchronize()
    assert int(p.status.abs().sum()) == 0
    NI = p.mesh.n_I
    AK = p.AK.view(-1, NI, NI).cpu().numpy()
    EK = p.EK.view(-1, NI).cpu().numpy()
    BK = p.BK.view(-1, NI).cpu().numpy()
    FK = p.FK.cpu().numpy()
    mesh = build_mesh(nx, ny, m, l)
    for K in range(len(rs)):
        o = solve_local(mesh, K, int(rs[K]), 1, kap[K], 1.0)
        tk = _fp64_bound(o, kap[K], tol) if rs[K] >= 7 else tol
        assert_blocks(AK[K], EK[K], BK[K], FK[K], o, tk, (K, int(rs[K]), tk))
    if precision == mhm.MHM_MIXED:   # the allocation-free entry runs the same levels
        AK2 = torch.empty_like(p.AK)
        EK2, BK2, FK2 = torch.empty_like(p.EK), torch.empty_like(p.BK), torch.empty_like(p.FK)
        st2 = torch.empty_like(p.status)
        mhm.mhm_local_solve_batch_noalloc(p.mesh, kd, src, OPTS_PARITY, AK2, EK2, BK2, FK2, st2)
        torch.cuda.synchronize()
        assert int(st2.abs().sum()) == 0
        assert _rel(AK2.cpu().numpy(), p.AK.cpu().numpy()) < tol


@pytest.mark.parametrize("precision", [mhm.MHM_FP64, mhm.MHM_MIXED])
def test_levels_exact_linear_pipeline(precision):
    """kappa = 1, u = 1 + 2x - 3y: recovered exactly at every node of every level."""
    from paper_1703_10435_gb300.pipeline import Pipeline
    nx, ny, rs, _ = _levels_case()
    p = Pipeline(nx, ny, 0, 1, 1, 1, 0, precision, r_per_K=rs)
    kd = torch.ones(int(p.mesh.kappa_offset[-1]), dtype=torch.float64, device="cuda")
    src = mhm.Source(mhm.MHM_SRC_CONST, 0.0, 1.0)
    gd = mhm.Dirichlet((mhm.ctypes.c_double * 6)(1.0, 2.0, -3.0, 0.0, 0.0, 0.0))
    p.step(kd, src, gd)
    p.solve_global()
    ex = mhm.Exact(mhm.MHM_EXACT_POLY, (mhm.ctypes.c_double * 6)(1.0, 2.0, -3.0, 0.0, 0.0, 0.0))
    u, err = p.reconstruct(kd, src, ex)
    torch.cuda.synchronize()
    assert int(p.status.abs().sum()) == 0
    assert float(err.sum()) < 1e-18
    # nodal values against g at the lattice points of each K's own level
    o = run(nx, ny, rs, 1, 1, 1, [np.ones(4 ** int(r)) for r in rs], 0.0, g=lambda x, y: 1 + 2 * x - 3 * y)
    uh = u.cpu().numpy()
    for K, loc in enumerate(o.locals):
        a, b = int(p.mesh.nodal_offset[K]), int(p.mesh.nodal_offset[K + 1])
        xy = loc.sub.node_xy
        assert np.abs(uh[a:b] - (1 + 2 * xy[:, 0] - 3 * xy[:, 1])).max() < 1e-10, K


def test_levels_solution_vs_oracle():
    """Random kappa on levels 1..7 through the whole pipeline: the multipliers and the
    reconstructed u of every element against the oracle.  Covers the global-memory
    window of the level-7 reconstruction and pinned DOFs moved off DOF 0 (the stiffest
    triangle of the first fine rows).  Bound 1e-9: the level-7 block alone carries the
    FP64 bound 10 u cond ~ 2e-10."""
    from oracle import reconstruct as orec
    from paper_1703_10435_gb300.pipeline import Pipeline
    nx, ny, rs, kap = _levels_case()
    p = Pipeline(nx, ny, 0, 1, 1, 2, 0, mhm.MHM_FP64, r_per_K=rs)
    kd = torch.as_tensor(np.concatenate(kap), device="cuda")
    src = mhm.Source(mhm.MHM_SRC_CONST, 1.0, 1.0)
    p.step(kd, src)
    lam, u0 = p.solve_global()
    u, _ = p.reconstruct(kd, src)
    torch.cuda.synchronize()
    assert int(p.status.abs().sum()) == 0
    o = run(nx, ny, rs, 1, 1, 2, kap, 1.0)
    assert _rel(lam.cpu().numpy(), o.lam) < 1e-9
    assert _rel(u0.cpu().numpy(), o.u0) < 1e-9
    uh = u.cpu().numpy()
    for K, loc in enumerate(o.locals):
        a, b = int(p.mesh.nodal_offset[K]), int(p.mesh.nodal_offset[K + 1])
        assert _rel(uh[a:b], orec.local_u(o.mesh, K, loc, o.lam, o.u0)) < 1e-9, (K, int(rs[K]))


@pytest.mark.parametrize("precision,tol", [(mhm.MHM_FP64, 1e-10), (mhm.MHM_MIXED, 1e-9)])
def test_face_degrees_every_element_vs_oracle(precision, tol):
    """A multiplier degree per face (1 + [r >= 5] + [r >= 7] over the adjacent levels, so
    degrees 1..3 meet levels 1..7): every element's blocks against the oracle in the slot
    layout (unused slots of lower-degree faces exactly zero)."""
    from paper_1703_10435_gb300.pipeline import Pipeline
    nx, ny, rs, kap = _levels_case()
    m = 1
    h = mhm.Mesh(nx, ny, 0, 1, m, 0, -1, rs)
    lf = _degrees(h.query(mhm.Q_TRI_FACES, np.int32, 3 * h.n_K), rs)
    mesh = build_mesh(nx, ny, m, _degrees(build_mesh(nx, ny, 1, 0).tri_edges, rs))
    assert np.array_equal(lf, mesh.l_e) and set(lf.tolist()) == {1, 2, 3}
    p = Pipeline(nx, ny, 0, 1, m, 3, 0, precision, r_per_K=rs, l_per_face=lf)
    d = p.mesh.n_I // 3
    kd = torch.as_tensor(np.concatenate(kap), device="cuda")
    src = mhm.Source(mhm.MHM_SRC_CONST, 1.0, 1.0)
    p.local(kd, src, OPTS_PARITY)
    torch.cuda.synchronize()
    assert int(p.status.abs().sum()) == 0
    NI = p.mesh.n_I
    AK = p.AK.view(-1, NI, NI).cpu().numpy()
    EK, BK = p.EK.view(-1, NI).cpu().numpy(), p.BK.view(-1, NI).cpu().numpy()
    FK = p.FK.cpu().numpy()
    for K in range(len(rs)):
        o = solve_local(mesh, K, int(rs[K]), 1, kap[K], 1.0)
        oA, oE, oB = _slots(mesh, K, m, d, o.AK), _slots(mesh, K, m, d, o.EK), _slots(mesh, K, m, d, o.BK)
        unused = _slots(mesh, K, m, d, np.ones(len(o.BK))) == 0.0
        assert unused.sum() == 3 * d - len(o.BK)
        assert np.all(AK[K][unused] == 0.0) and np.all(AK[K][:, unused] == 0.0), K
        assert np.all(EK[K][unused] == 0.0) and np.all(BK[K][unused] == 0.0), K
        tk = _fp64_bound(o, kap[K], tol) if rs[K] >= 7 else tol
        os_ = SimpleNamespace(AK=oA, EK=oE, BK=oB, FK=o.FK)
        assert_blocks(AK[K], EK[K], BK[K], FK[K], os_, tk, (K, int(rs[K]), tk))
        assert np.abs(BK[K] - oB).max() < 1e-13 * np.abs(oB).max(), K
    if precision == mhm.MHM_MIXED:   # the allocation-free entry runs the same levels
        AK2 = torch.empty_like(p.AK)
        EK2, BK2, FK2 = torch.empty_like(p.EK), torch.empty_like(p.BK), torch.empty_like(p.FK)
        st2 = torch.empty_like(p.status)
        mhm.mhm_local_solve_batch_noalloc(p.mesh, kd, src, OPTS_PARITY, AK2, EK2, BK2, FK2, st2)
        torch.cuda.synchronize()
        assert int(st2.abs().sum()) == 0
        assert _rel(AK2.cpu().numpy(), p.AK.cpu().numpy()) < tol


@pytest.mark.parametrize("precision,tol", [(mhm.MHM_FP64, 1e-9), (mhm.MHM_MIXED, 1e-8)])
def test_face_degrees_solution_vs_oracle(precision, tol):
    """Degrees 1..3 per face through the whole pipeline (skeleton of mixed block sizes,
    global solve, reconstruction): multipliers, u0 and u of every element against the
    oracle; sinsin source."""
    from oracle import reconstruct as orec
    from oracle.run import source_fn
    from paper_1703_10435_gb300.pipeline import Pipeline
    nx, ny, rs, kap = _levels_case()
    m = 1
    h = mhm.Mesh(nx, ny, 0, 1, m, 0, -1, rs)
    lf = _degrees(h.query(mhm.Q_TRI_FACES, np.int32, 3 * h.n_K), rs)
    p = Pipeline(nx, ny, 0, 1, m, 3, 0, precision, r_per_K=rs, l_per_face=lf)
    kd = torch.as_tensor(np.concatenate(kap), device="cuda")
    src = mhm.Source(mhm.MHM_SRC_SINSIN, 1.0, 1.0)
    p.step(kd, src, None, mhm.SolveOpts(10, 1e-13, 0, 0))
    lam, u0 = p.solve_global()
    u, _ = p.reconstruct(kd, src)
    torch.cuda.synchronize()
    assert int(p.status.abs().sum()) == 0
    o = run(nx, ny, rs, 1, m, _degrees(build_mesh(nx, ny, 1, 0).tri_edges, rs), kap, source_fn("sinsin"))
    assert _rel(lam.cpu().numpy(), o.lam) < tol
    assert _rel(u0.cpu().numpy(), o.u0) < tol
    uh = u.cpu().numpy()
    for K, loc in enumerate(o.locals):
        a, b = int(p.mesh.nodal_offset[K]), int(p.mesh.nodal_offset[K + 1])
        assert _rel(uh[a:b], orec.local_u(o.mesh, K, loc, o.lam, o.u0)) < tol, (K, int(rs[K]))


@pytest.mark.parametrize("precision", [mhm.MHM_FP64, mhm.MHM_MIXED])
def test_face_degrees_exact_linear_pipeline(precision):
    """Degrees 0..3 face by face, levels 2..4 element by element, kappa = 1 and
    u = 1 + 2x - 3y: recovered exactly at every node (the flux is constant per face, so it
    lies in every face's space; m(l_e+1) <= 4 against >= 5 trace nodes keeps the system
    nonsingular)."""
    from paper_1703_10435_gb300.pipeline import Pipeline
    nx = ny = 3
    ne = nx * (ny + 1) + ny * (nx + 1) + nx * ny
    rng = np.random.default_rng(10)
    lf = rng.integers(0, 4, ne).astype(np.int8)
    rs = rng.integers(2, 5, 2 * nx * ny).astype(np.int8)
    p = Pipeline(nx, ny, 0, 1, 1, 3, 0, precision, r_per_K=rs, l_per_face=lf)
    kd = torch.ones(int(p.mesh.kappa_offset[-1]), dtype=torch.float64, device="cuda")
    src = mhm.Source(mhm.MHM_SRC_CONST, 0.0, 1.0)
    gd = mhm.Dirichlet((mhm.ctypes.c_double * 6)(1.0, 2.0, -3.0, 0.0, 0.0, 0.0))
    p.step(kd, src, gd)
    p.solve_global()
    ex = mhm.Exact(mhm.MHM_EXACT_POLY, (mhm.ctypes.c_double * 6)(1.0, 2.0, -3.0, 0.0, 0.0, 0.0))
    u, err = p.reconstruct(kd, src, ex)
    torch.cuda.synchronize()
    assert int(p.status.abs().sum()) == 0
    assert float(err.sum()) < 1e-18
    o = run(nx, ny, rs, 1, 1, lf, [np.ones(4 ** int(r)) for r in rs], 0.0, g=lambda x, y: 1 + 2 * x - 3 * y)
    uh = u.cpu().numpy()
    for K, loc in enumerate(o.locals):
        a, b = int(p.mesh.nodal_offset[K]), int(p.mesh.nodal_offset[K + 1])
        xy = loc.sub.node_xy
        assert np.abs(uh[a:b] - (1 + 2 * xy[:, 0] - 3 * xy[:, 1])).max() < 1e-10, K


@pytest.mark.parametrize("precision", [mhm.MHM_FP64, mhm.MHM_MIXED])
def test_levels_k_ranges_equal_one_shot(precision):
    """The K-range option (one rank's contiguous share of the elements) on a mesh of levels
    1..7 and face degrees 1..3: two calls over an uneven split give the one-shot blocks bit
    for bit (each level maps the range to its own element list)."""
    from paper_1703_10435_gb300.pipeline import Pipeline
    nx, ny, rs, kap = _levels_case()
    h = mhm.Mesh(nx, ny, 0, 1, 1, 0, -1, rs)
    lf = _degrees(h.query(mhm.Q_TRI_FACES, np.int32, 3 * h.n_K), rs)
    kd = torch.as_tensor(np.concatenate(kap), device="cuda")
    src = mhm.Source(mhm.MHM_SRC_CONST, 1.0, 1.0)
    one = Pipeline(nx, ny, 0, 1, 1, 3, 0, precision, r_per_K=rs, l_per_face=lf)
    one.local(kd, src)
    two = Pipeline(nx, ny, 0, 1, 1, 3, 0, precision, r_per_K=rs, l_per_face=lf)
    n = two.mesh.n_K
    split = n // 2 + 1
    two.local(kd, src, mhm.SolveOpts(8, 1e-12, 0, split))
    two.local(kd, src, mhm.SolveOpts(8, 1e-12, split, n))
    torch.cuda.synchronize()
    for name in ("AK", "EK", "BK", "FK", "status", "iters"):
        assert torch.equal(getattr(one, name), getattr(two, name)), name


def test_channel_workload_full_size():
    """The uneven channel workload (8192 K, levels 3..7, face degrees 1..3): every level
    present, FP64 and mixed agree, and sampled elements of each level match the oracle."""
    from paper_1703_10435_gb300.pipeline import Pipeline, source_of
    w = W.WORKLOADS["c4_channels"]
    rk = w.r_per_K
    assert set(np.unique(rk).tolist()) == {3, 4, 5, 6, 7}
    kd = torch.as_tensor(W.kappa_for(w), device="cuda")
    out = {}
    for prec in (mhm.MHM_FP64, mhm.MHM_MIXED):
        p = Pipeline.for_workload(w, 0, prec)
        p.local(kd, source_of(w))
        torch.cuda.synchronize()
        assert int(p.status.abs().sum()) == 0
        out[prec] = p.AK.view(w.n_K, -1)
        if prec == mhm.MHM_MIXED:
            # levels 3..5 converge in FP32 + refinement; the 64- and 128-wide levels 6
            # and 7 in FP64 conjugate gradients preconditioned by the FP32 factor (a few
            # elements whose pinned DOF lies on lattice row 1 are solved in FP64: -1)
            it = p.iters.cpu().numpy()
            assert np.all(it[rk <= 5] >= 2)
            w67 = it[rk >= 6]
            assert np.all((w67 == -1) | ((w67 >= 1) & (w67 <= 8))) and np.mean(w67 == -1) < 0.01
            assert float(w67[w67 > 0].mean()) <= 4.0
    d = (torch.linalg.norm(out[mhm.MHM_MIXED] - out[mhm.MHM_FP64], dim=1) /
         torch.linalg.norm(out[mhm.MHM_FP64], dim=1)).cpu().numpy()
    # levels 3..5: the same pinned solution to 1e-9.  Levels 6, 7: the two paths reach it by
    # different FP64 arithmetic (Cholesky Gram form; CG residuals and the corrected bilinear
    # form), each to about 10 u cond(A) per entry (scaled by sqrt(A_ii A_jj)): on the element
    # where they differ most, the norm-relative difference stays below 2 sqrt(N_I) times that
    # bound (cond from the oracle's matrix; sum_ij A_ii A_jj <= N_I ||A||_F^2).
    assert float(d[rk <= 5].max()) < 1e-9
    Kw = int(np.flatnonzero(rk >= 6)[np.argmax(d[rk >= 6])])
    from oracle.fem import Submesh
    from oracle.local import assemble_stiffness
    import scipy.sparse.linalg as sla
    kw = W.kappa_levels(w, [Kw])[0]
    A = assemble_stiffness(Submesh(W.coarse_vertices(w.nx, w.ny)[Kw], int(rk[Kw]), 1), kw)
    hi = float(sla.eigsh(A, k=1, which="LA", return_eigenvectors=False)[0])
    lo = float(np.sort(sla.eigsh(A, k=2, sigma=-1e-6 * hi, which="LM", return_eigenvectors=False))[1])
    NIw = out[mhm.MHM_FP64].shape[1] ** 0.5
    assert float(d[Kw]) < 2 * np.sqrt(NIw) * max(1e-10, 10 * 2.0 ** -53 * hi / lo), (Kw, float(d[Kw]), hi / lo)
    # Per level: the median element and the first element crossing a channel (kappa 1 and
    # 1e4 inside it), each path against the oracle.  The bound is 1e-10, or the FP64
    # error bound 10 u cond(A) (u = 2^-53, cond on the mean-zero space) where that is
    # larger: crossing elements have cond ~2e7 (level 6) to ~1.5e8 (level 7), and the
    # pinned Cholesky on the GPU reproduces them only to about u cond (the oracle's
    # bordered LU is accurate to ~4e-12 there).
    mesh = build_mesh(w.nx, w.ny, w.m, w.l_per_face(build_mesh(w.nx, w.ny, 1, 0).tri_edges))
    assert set(mesh.l_e.tolist()) == {1, 2, 3}
    NI = 3 * w.m * (w.l + 1)
    d = NI // 3
    for r in (3, 4, 5, 6, 7):
        idx = np.flatnonzero(rk == r)
        picks = [int(idx[len(idx) // 2])]
        for K in idx:
            if W.kappa_levels(w, [int(K)])[0].max() > 1.0:
                picks.append(int(K))
                break
        for K in picks:
            kap = W.kappa_levels(w, [K])[0]
            o = solve_local(mesh, K, r, 1, kap, 1.0)
            tol = _fp64_bound(o, kap, 1e-10)
            for prec in (mhm.MHM_FP64, mhm.MHM_MIXED):
                got = out[prec][K].view(NI, NI).cpu().numpy()
                assert gram_entry_error(got, _slots(mesh, K, w.m, d, o.AK)) < tol, (r, K, prec, tol)


@pytest.mark.parametrize("precision", [mhm.MHM_FP64, mhm.MHM_MIXED])
def test_levels_graph_replay(precision):
    """The step on a mesh of several levels (levels forked to side streams and joined
    back) captured once in a CUDA graph: every replay gives the eager result bit for bit.
    The first, eager call creates the side streams before the capture."""
    from paper_1703_10435_gb300.pipeline import Pipeline
    nx, ny, rs, kap = _levels_case()
    p = Pipeline(nx, ny, 0, 1, 1, 2, 0, precision, r_per_K=rs)
    kd = torch.as_tensor(np.concatenate(kap), device="cuda")
    src = mhm.Source(mhm.MHM_SRC_CONST, 1.0, 1.0)
    p.step(kd, src)
    torch.cuda.synchronize()
    ref_A, ref_AK = p.A_vals.clone(), p.AK.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            p.step(kd, src, stream=s)
    torch.cuda.synchronize()
    for _ in range(3):
        p.A_vals.zero_()
        p.AK.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(p.A_vals, ref_A) and torch.equal(p.AK, ref_AK)


@pytest.mark.parametrize("precision", [mhm.MHM_FP64, mhm.MHM_MIXED])
def test_p2_r5_wide_window_vs_oracle(precision):
    """P2 at r = 5 (2145 unknowns per element, a 253-row level window kept in global
    memory; MIXED runs it on the FP64 path): every element of a 2 x 1 mesh against the
    oracle, log-uniform kappa."""
    from paper_1703_10435_gb300.pipeline import Pipeline
    nx, ny, r, m, l = 2, 1, 5, 2, 2
    rng = np.random.default_rng(33)
    kap = 10.0 ** rng.uniform(-1, 1, (2 * nx * ny, 4 ** r))
    p = Pipeline(nx, ny, r, 2, m, l, 0, precision)
    p.local(torch.as_tensor(kap.ravel(), device="cuda"), mhm.Source(mhm.MHM_SRC_CONST, 1.0, 1.0))
    torch.cuda.synchronize()
    assert int(p.status.abs().sum()) == 0
    assert np.all(p.iters.cpu().numpy() == 1)
    NI = p.mesh.n_I
    AK = p.AK.view(-1, NI, NI).cpu().numpy()
    EK = p.EK.view(-1, NI).cpu().numpy()
    BK, FK = p.BK.view(-1, NI).cpu().numpy(), p.FK.cpu().numpy()
    mesh = build_mesh(nx, ny, m, l)
    for K in range(2 * nx * ny):
        o = solve_local(mesh, K, r, 2, kap[K], 1.0)
        tk = _fp64_bound(o, kap[K], 1e-10)
        assert_blocks(AK[K], EK[K], BK[K], FK[K], o, tk, (K, tk))


def test_mixed_levels_in_one_persistent_launch():
    """Coarse elements of five refinement levels on the mixed level-Schur path go into one
    factor launch and one persistent solve launch (the levels as work buckets, the largest
    first), with the blocks of the single-level launches: a mesh whose elements all sit at
    one level runs those, so the same elements at the same level agree to rounding (the
    two kernels are separate compilations of the same code)."""
    from paper_1703_10435_gb300.pipeline import Pipeline
    nx, ny, rs, kap = _levels_case()
    keep = rs <= 5                     # the level-Schur levels only (6 and 7 run in FP64)
    rs2 = np.where(keep, rs, 5).astype(np.int8)
    kap2 = [k if kp else 10.0 ** np.random.default_rng(K).uniform(-2, 2, 4 ** 5) for K, (k, kp) in
            enumerate(zip(kap, keep))]
    p = Pipeline(nx, ny, 0, 1, 1, 2, 0, mhm.MHM_MIXED, r_per_K=rs2)
    kd = torch.as_tensor(np.concatenate(kap2), device="cuda")
    src = mhm.Source(mhm.MHM_SRC_CONST, 1.0, 1.0)
    mhm.mhm_set_timing(p.mesh, True)
    p.local(kd, src, mhm.SolveOpts(10, 1e-13, 0, 0))
    times = mhm.mhm_kernel_times(p.mesh)
    assert times["k_local_mixed"][0] == 1 and times["k_schur_factor"][0] == 1, times
    assert int(p.status.abs().sum()) == 0
    # each element against a mesh that holds only its own level (single-level launches)
    NI = p.mesh.n_I
    for r in sorted(set(rs2.tolist())):
        idx = np.flatnonzero(rs2 == r)
        q = Pipeline(nx, ny, 0, 1, 1, 2, 0, mhm.MHM_MIXED, r_per_K=np.full_like(rs2, r))
        kq = [kap2[K] if rs2[K] == r else np.ones(4 ** r) for K in range(len(rs2))]
        q.local(torch.as_tensor(np.concatenate(kq), device="cuda"), src, mhm.SolveOpts(10, 1e-13, 0, 0))
        torch.cuda.synchronize()
        for K in idx:
            for a, b in ((p.AK[K * NI * NI:(K + 1) * NI * NI], q.AK[K * NI * NI:(K + 1) * NI * NI]),
                         (p.EK[K * NI:(K + 1) * NI], q.EK[K * NI:(K + 1) * NI])):
                assert float((a - b).abs().max()) <= 1e-12 * float(b.abs().max()), (r, K)


def test_mixed_levels_launch_falls_back_to_fp64():
    """The persistent launch across levels with a one-pass limit: the refinement of most
    elements stops short, and each level's failed elements are solved again by the FP64 path
    (status OK, iters -1, blocks equal to the FP64 path's); without the re-solve they keep
    MHM_ERR_NOT_CONVERGED and the outcome word says so."""
    from paper_1703_10435_gb300.pipeline import Pipeline
    nx, ny, rs, kap = _levels_case()
    keep = rs <= 5
    rs2 = np.where(keep, rs, 5).astype(np.int8)
    kap2 = [k if kp else 10.0 ** np.random.default_rng(K).uniform(-2, 2, 4 ** 5) for K, (k, kp) in
            enumerate(zip(kap, keep))]
    kd = torch.as_tensor(np.concatenate(kap2), device="cuda")
    src = mhm.Source(mhm.MHM_SRC_CONST, 1.0, 1.0)
    p = Pipeline(nx, ny, 0, 1, 1, 2, 0, mhm.MHM_MIXED, r_per_K=rs2)
    q = Pipeline(nx, ny, 0, 1, 1, 2, 0, mhm.MHM_FP64, r_per_K=rs2)
    mhm.mhm_set_timing(p.mesh, True)
    p.local(kd, src, mhm.SolveOpts(1, 1e-13, 0, 0))
    times = mhm.mhm_kernel_times(p.mesh)
    assert times["k_local_mixed"][0] == 1, times
    q.local(kd, src)
    torch.cuda.synchronize()
    assert set(p.status.cpu().tolist()) == {0}
    failed = np.flatnonzero(p.iters.cpu().numpy() == -1)   # (the smallest levels may finish in one pass)
    assert len(failed) >= len(rs2) // 2
    NI = p.mesh.n_I
    for K in failed:
        assert torch.equal(p.AK[K * NI * NI:(K + 1) * NI * NI], q.AK[K * NI * NI:(K + 1) * NI * NI]), K
        assert torch.equal(p.EK[K * NI:(K + 1) * NI], q.EK[K * NI:(K + 1) * NI]), K
    p.local(kd, src, mhm.SolveOpts(1, 1e-13, 0, 0, 1))
    torch.cuda.synchronize()
    st = p.status.cpu().numpy()
    assert set(st.tolist()) <= {0, mhm.MHM_ERR_NOT_CONVERGED} and (st[failed] == mhm.MHM_ERR_NOT_CONVERGED).all()
    assert mhm.mhm_sync_status(p.mesh)[0] == mhm.MHM_ERR_NOT_CONVERGED
