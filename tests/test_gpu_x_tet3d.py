"""Parity of the three-dimensional CUDA path (include/mhm3d.h, through the C ABI) with
the FP64 oracle (oracle/tet3d.py) on the same seeded inputs: the per-element blocks
A_K, E_K, B_K, F_K entry by entry, the assembled skeleton, the full-size workload of
the paper's experiment (Sec. 5: 12288 tetrahedra, m = 4) on sampled elements and by
properties that hold at any size, and the exact recovery of a linear solution."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import globalsys
from oracle import tet3d as T
from paper_1703_10435_gb300 import mhm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_10435_gb300 import build
    build.build()


def _run(M, kappa, src, K0=0, K1=0, precision=mhm.MHM_FP64, opts=None):
    dev = torch.device("cuda", 0)
    nK, NI = M.n_K, M.n_I
    out = dict(AK=torch.zeros(nK, NI, NI, dtype=torch.float64, device=dev),
               EK=torch.zeros(nK, NI, dtype=torch.float64, device=dev),
               BK=torch.zeros(nK, NI, dtype=torch.float64, device=dev),
               FK=torch.zeros(nK, dtype=torch.float64, device=dev),
               status=torch.full((nK,), -7, dtype=torch.int32, device=dev),
               iters=torch.full((nK,), -9, dtype=torch.int32, device=dev))
    kap = torch.as_tensor(np.ascontiguousarray(kappa, dtype=np.float64).reshape(-1), device=dev)
    mhm.mhm3d_local_solve_batch(M, kap, src, out["AK"], out["EK"], out["BK"], out["FK"], out["status"], K0, K1,
                                precision=precision, opts=opts, iters=out["iters"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _errors(got, K, o, amp_volK):
    """Worst error ratios of element K's blocks against the oracle's: A_K on the Gram
    scale sqrt(|A_ii| |A_jj|), E_K on max(|E_K|, |A_K| |F_K| / |B_K|) (E_K vanishes for a
    constant source), B_K on its largest entry, F_K on the bound int |f| <= amp |K|."""
    d = np.sqrt(np.abs(np.diag(o.AK)))
    eA = float((np.abs(got["AK"][K] - o.AK) / np.maximum(np.outer(d, d), 1e-300)).max())
    bmax = float(np.abs(o.BK).max())
    sE = max(float(np.abs(o.EK).max()), float(np.abs(o.AK).max()) * abs(o.FK) / bmax, 1e-300)
    eE = float(np.abs(got["EK"][K] - o.EK).max()) / sE
    eB = float(np.abs(got["BK"][K] - o.BK).max()) / bmax
    eF = abs(float(got["FK"][K]) - o.FK) / amp_volK
    return {"A": eA, "E": eE, "B": eB, "F": eF}


CASES = [
    # nc, r, k, m, source (kind, value, freq), log10 kappa range, tolerance
    (1, 1, 2, 4, (mhm.MHM3D_SRC_CONST, 1.0, 2.0), 1.0, 1e-10),
    (1, 2, 2, 4, (mhm.MHM3D_SRC_SINSINSIN, 1.0, 2.0), 1.0, 1e-10),
    (1, 2, 2, 16, (mhm.MHM3D_SRC_SINSINSIN, 1.0, 2.0), 2.0, 1e-9),
    (1, 2, 1, 4, (mhm.MHM3D_SRC_SINSINSIN, 0.7, 1.0), 2.0, 1e-9),
    (1, 3, 1, 16, (mhm.MHM3D_SRC_CONST, 2.5, 2.0), 1.0, 1e-10),
]


@pytest.mark.parametrize("precision", [mhm.MHM_FP64, mhm.MHM_MIXED])
@pytest.mark.parametrize("nc,r,P,m,src,decades,tol", CASES)
def test_local_blocks_entrywise(nc, r, P, m, src, decades, tol, precision):
    """Both precisions against the oracle at the same bound: MIXED (m = 4) refines its FP32
    solutions in FP64 and uses the corrected bilinear form, whose error is second order in
    the solution error; MIXED with m = 16 runs the FP64 kernel."""
    M = mhm.Mesh3D(nc, r, P, m, device=0)
    o = T.build_mesh3d(nc, m)
    rng = np.random.default_rng(100 * r + m + P)
    kappa = 10.0 ** rng.uniform(-decades, decades, (M.n_K, 8 ** r))
    got = _run(M, kappa, mhm.Source3D(*src), precision=precision)
    assert np.all(got["status"] == 0)
    if precision == mhm.MHM_MIXED and m <= 4:
        assert np.all((got["iters"] >= 1) & (got["iters"] <= 8) | (got["iters"] == -1))
    else:
        assert np.all(got["iters"] == 1)
    f = src[1] if src[0] == mhm.MHM3D_SRC_CONST else T.source3d_fn("sinsinsin", src[1], src[2])
    amp = abs(src[1]) * (3.0 * (src[2] * math.pi) ** 2 if src[0] == mhm.MHM3D_SRC_SINSINSIN else 1.0)
    worst = {}
    for K in range(M.n_K):
        loc = T.solve_local3d(o, K, r, P, kappa[K], f)
        e = _errors(got, K, loc, amp / M.n_K)
        for k, v in e.items():
            worst[k] = max(worst.get(k, 0.0), v)
        assert max(e["A"], e["E"], e["B"]) < tol and e["F"] < 1e-13, (K, e)
    # symmetric by construction; every other block checked against the oracle above
    assert np.array_equal(got["AK"], np.transpose(got["AK"], (0, 2, 1)))


def test_mixed_fallback_and_no_fallback():
    """One refinement pass with an unreachable target: every element is solved again by the
    FP64 kernel (iters -1, blocks equal to the FP64 path's up to the assembly order), or,
    with no_fallback, keeps MHM_ERR_NOT_CONVERGED."""
    M = mhm.Mesh3D(1, 1, 2, 4, device=0)
    rng = np.random.default_rng(4)
    kappa = 10.0 ** rng.uniform(-1, 1, (M.n_K, 8))
    src = mhm.Source3D(mhm.MHM3D_SRC_SINSINSIN, 1.0, 2.0)
    ref = _run(M, kappa, src)
    fb = _run(M, kappa, src, precision=mhm.MHM_MIXED, opts=mhm.Opts3D(1, 1e-300, 0))
    assert np.all(fb["status"] == 0) and np.all(fb["iters"] == -1)
    for k in ("AK", "EK", "BK", "FK"):   # the FP64 kernel again: bit for bit
        assert np.array_equal(fb[k], ref[k]), k
    nf = _run(M, kappa, src, precision=mhm.MHM_MIXED, opts=mhm.Opts3D(1, 1e-300, 1))
    assert np.all(nf["status"] == mhm.MHM_ERR_NOT_CONVERGED) and np.all(nf["iters"] == 1)
    with pytest.raises(mhm.MHMError) as e:
        _run(M, kappa, src, precision=mhm.MHM_MIXED, opts=mhm.Opts3D(0, 1e-9, 0))
    assert e.value.code == mhm.MHM_ERR_INVALID_ARG


@pytest.mark.parametrize("precision", [mhm.MHM_FP64, mhm.MHM_MIXED])
def test_k_range_matches_full_call(precision):
    M = mhm.Mesh3D(1, 2, 2, 4, device=0)
    rng = np.random.default_rng(3)
    kappa = 10.0 ** rng.uniform(-1, 1, (M.n_K, 64))
    src = mhm.Source3D(mhm.MHM3D_SRC_SINSINSIN, 1.0, 2.0)
    full = _run(M, kappa, src, precision=precision)
    part = _run(M, kappa, src, 5, 17, precision=precision)
    assert np.all(part["status"][:5] == -7) and np.all(part["status"][17:] == -7)
    # the same elements bit for bit (every sum in the kernels runs in a fixed order)
    for k in ("AK", "EK", "BK", "FK"):
        assert np.array_equal(part[k][5:17], full[k][5:17]), k
        assert not np.any(part[k][17:])


@pytest.mark.parametrize("precision", [mhm.MHM_FP64, mhm.MHM_MIXED])
def test_repeated_calls_bit_identical(precision):
    """No atomics: assembly, loads and residuals are gathered per DOF in a fixed order."""
    M = mhm.Mesh3D(1, 2, 2, 4, device=0)
    rng = np.random.default_rng(12)
    kappa = 10.0 ** rng.uniform(-2, 2, (M.n_K, 64))
    src = mhm.Source3D(mhm.MHM3D_SRC_SINSINSIN, 1.0, 2.0)
    a = _run(M, kappa, src, precision=precision)
    b = _run(M, kappa, src, precision=precision)
    for k in ("AK", "EK", "BK", "FK", "status", "iters"):
        assert np.array_equal(a[k], b[k]), k


def test_skeleton_matches_oracle_assembly():
    import scipy.sparse
    nc, r, P, m = 2, 1, 2, 4
    M = mhm.Mesh3D(nc, r, P, m, device=0)
    o = T.build_mesh3d(nc, m)
    rng = np.random.default_rng(9)
    kappa = 10.0 ** rng.uniform(-1, 1, (M.n_K, 8 ** r))
    f = T.source3d_fn("sinsinsin", 1.0, 2.0)
    got = _run(M, kappa, mhm.Source3D(mhm.MHM3D_SRC_SINSINSIN, 1.0, 2.0))
    dev = torch.device("cuda", 0)
    AK, EK = torch.as_tensor(got["AK"], device=dev), torch.as_tensor(got["EK"], device=dev)
    vals = torch.zeros(M.nnz, dtype=torch.float64, device=dev)
    E = torch.zeros(M.n_lambda, dtype=torch.float64, device=dev)
    mhm.mhm3d_assemble_skeleton(M, AK, EK, vals, E)
    torch.cuda.synchronize()
    rowptr = M.query(mhm.Q3_CSR_ROWPTR, np.int32, M.n_lambda + 1)
    cols = M.query(mhm.Q3_CSR_COLS, np.int32, M.nnz)
    A_gpu = scipy.sparse.csr_matrix((vals.cpu().numpy(), cols, rowptr), shape=(M.n_lambda, M.n_lambda)).toarray()
    locs = [T.solve_local3d(o, K, r, P, kappa[K], f) for K in range(o.n_K)]
    A_or, B_or, E_or, F_or = globalsys.assemble(o, locs)
    A_or = A_or.toarray()
    d = np.sqrt(np.abs(np.diag(A_or)))
    assert (np.abs(A_gpu - A_or) / np.maximum(np.outer(d, d), 1e-300)).max() < 1e-10
    assert np.abs(E.cpu().numpy() - E_or).max() < 1e-10 * np.abs(E_or).max()
    # the second row of Eq. "mat_global": B and F are the per-element blocks as they are
    B_gpu = np.zeros((o.n_K, o.n_lambda))
    for K in range(o.n_K):
        B_gpu[K, o.local_lambda(K)] += got["BK"][K]
    assert np.abs(B_gpu - B_or.toarray()).max() < 1e-14
    assert np.abs(got["FK"] - F_or).max() < 1e-13 * 12 * math.pi ** 2


def test_exact_linear_recovery_through_gpu_blocks():
    """kappa = 1, f = 0, u linear: the saddle-point system built from the GPU's blocks (and
    the boundary moments of g = u) gives lambda = -grad u . n on every subface."""
    import scipy.sparse
    import scipy.sparse.linalg
    nc, r, P, m = 1, 1, 2, 4
    M = mhm.Mesh3D(nc, r, P, m, device=0)
    o = T.build_mesh3d(nc, m)
    got = _run(M, np.ones((M.n_K, 8 ** r)), mhm.Source3D(mhm.MHM3D_SRC_CONST, 0.0, 1.0))
    grad = np.array([2.0, -3.0, 0.5])
    g = lambda x, y, z: 1.0 + grad[0] * x + grad[1] * y + grad[2] * z
    L = o.n_lambda
    A = np.zeros((L, L))
    B = np.zeros((o.n_K, L))
    E = np.zeros(L)
    for K in range(o.n_K):
        ids = o.local_lambda(K)
        A[np.ix_(ids, ids)] += got["AK"][K]
        B[K, ids] += got["BK"][K]
        E[ids] += got["EK"][K]
    G = T.dirichlet_term3d(o, g, 1 << r)
    S = np.block([[A, B.T], [B, np.zeros((o.n_K, o.n_K))]])
    x = np.linalg.solve(S, np.concatenate([E + G, got["FK"]]))
    lam = x[:L]
    assert np.abs(lam - np.repeat(-(o.normals @ grad), m)).max() < 1e-10


@pytest.mark.parametrize("nc,m", [(8, 4), (4, 16)])
def test_full_size_sampled_parity_and_properties(nc, m):
    """The paper's configurations (Sec. 5, k = 2, here 64 sub-tetrahedra per element for
    TetGen's 59): 12288 coarse tetrahedra with m = 4 and 1536 with m = 16 (MIXED runs the FP64
    kernel there), kappa = 1 and f = 12 pi^2 sin sin sin as in the paper (FP64 and MIXED), then
    a log-uniform kappa (MIXED): sampled elements against the oracle, and at
    every element B_K = s |face| / m, a symmetric negative semidefinite A_K (checked on 256
    elements) and status 0."""
    r, P = 2, 2
    M = mhm.Mesh3D(nc, r, P, m, device=0)
    o = T.build_mesh3d(nc, m)
    src = mhm.Source3D(mhm.MHM3D_SRC_SINSINSIN, 1.0, 2.0)
    f = T.source3d_fn("sinsinsin", 1.0, 2.0)
    amp = 12.0 * math.pi ** 2
    rng = np.random.default_rng(2026)
    runs = []
    for kappa, precision in ((np.ones((M.n_K, 64)), mhm.MHM_FP64), (np.ones((M.n_K, 64)), mhm.MHM_MIXED),
                             (10.0 ** rng.uniform(-1, 1, (M.n_K, 64)), mhm.MHM_MIXED)):
        got = _run(M, kappa, src, precision=precision)
        runs.append(got)
        assert np.all(got["status"] == 0)
        sample = [0, M.n_K - 1] + [int(k) for k in rng.choice(M.n_K, 4, replace=False)]
        for K in sample:
            loc = T.solve_local3d(o, K, r, P, kappa[K], f)
            e = _errors(got, K, loc, amp / M.n_K)
            assert max(e["A"], e["E"], e["B"]) < 1e-10 and e["F"] < 1e-13, (K, e)
        # B_K = s |face| / m for every element and subface
        V = o.verts[o.tets]                                   # (n_K, 4, 3)
        for a in range(4):
            b = [v for v in range(4) if v != a]
            area = 0.5 * np.linalg.norm(np.cross(V[:, b[1]] - V[:, b[0]], V[:, b[2]] - V[:, b[0]]), axis=1)
            want = (o.signs[:, a] * area / m)[:, None]
            assert np.abs(got["BK"][:, a * m:(a + 1) * m] - want).max() < 1e-15
        for K in rng.choice(M.n_K, 256, replace=False):
            ev = np.linalg.eigvalsh(got["AK"][K])
            assert ev.max() <= 1e-12 * np.abs(ev).max()
    # every element: the two precisions on the same input agree on the Gram scale
    a64, amx = runs[0]["AK"], runs[1]["AK"]
    d = np.sqrt(np.abs(np.einsum("kii->ki", a64)))
    assert float((np.abs(amx - a64) / np.maximum(d[:, :, None] * d[:, None, :], 1e-300)).max()) < 1e-10
    assert float(np.abs(runs[1]["EK"] - runs[0]["EK"]).max()) <= 1e-10 * float(np.abs(runs[0]["EK"]).max())


def test_device_refusals():
    for args in ((1, 3, 2, 4), (1, 4, 1, 16)):
        with pytest.raises(mhm.MHMError) as e:
            mhm.Mesh3D(*args, device=0)
        assert e.value.code == mhm.MHM_ERR_UNSUPPORTED
