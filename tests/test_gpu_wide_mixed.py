"""Mixed precision on the wide P1 levels r = 6 and 7 (lattice rows of 64 and 128
unknowns): the FP32 level-Schur factor as the preconditioner of FP64 conjugate
gradients.  Every element against the oracle; the elements the kernel leaves to the FP64
path (pinned DOF on lattice row 1; CG not converged within it_max) re-solved there, or
reported with the re-solve turned off."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.local import solve_local
from oracle.mesh import build_mesh
from paper_1703_10435_gb300 import mhm
from _blocks import assert_blocks

pytestmark = pytest.mark.gpu

M, L = 2, 1          # N_I = 12, 13 right-hand sides (the channel workload's slot stride)
OPTS = mhm.SolveOpts(10, 1e-13, 0, 0)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_10435_gb300 import build
    build.build()


def _kappa(N, kind, seed):
    """kappa per fine triangle (row j: up i = 0..N-j-1, then down i = 0..N-j-2).
    "bands": 1, and 1e4 on a band of fine rows across the middle and on a diagonal band
    from the corner (0, 0), so the stiffest triangles of rows 0 and 1 touch lattice row 0
    (pinned DOF there).  "row1": log-uniform 10^[-1, 1], row 0 at 1e-2 and one triangle
    of row 1 at 1e3, so the pinned DOF lies on lattice row 1."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(N):
        for up in (True, False):
            for i in range(N - j if up else N - j - 1):
                if kind == "bands":
                    stiff = (N // 2 - 4 <= j < N // 2 + 4) or abs(i - j) < 3
                    out.append(1e4 if stiff else 1.0)
                else:
                    out.append(10.0 ** rng.uniform(-1, 1))
    k = np.array(out)
    if kind == "row1":
        k[:2 * N - 1] = 1e-2
        k[(2 * N - 1) + N // 3] = 1e3
    return k


def _fp64_bound(o, kap, base):
    """base, or 10 u cond(A) on the mean-zero space where larger (the FP64 path and the
    oracle's LU agree only to about that on high-contrast level-7 elements)."""
    import scipy.sparse.linalg as sla
    from oracle.local import assemble_stiffness
    A = assemble_stiffness(o.sub, kap)
    hi = float(sla.eigsh(A, k=1, which="LA", return_eigenvectors=False)[0])
    ev = np.sort(sla.eigsh(A, k=2, sigma=-1e-6 * hi, which="LM", return_eigenvectors=False))
    return max(base, 10 * 2.0 ** -53 * hi / float(ev[1]))


def _case(r):
    N = 1 << r
    kap = [_kappa(N, "bands", 1), _kappa(N, "row1", 2)]
    return N, kap


@pytest.mark.parametrize("r", [6, 7])
def test_wide_level_vs_oracle(r):
    """K = 0 runs the mixed kernel (CG converged, iters >= 1); K = 1 (pinned DOF on row 1)
    is solved again by the FP64 path (iters -1).  Both against the oracle entry by entry;
    one wide-kernel launch and one FP64 re-solve launch."""
    from paper_1703_10435_gb300.pipeline import Pipeline
    N, kap = _case(r)
    p = Pipeline(1, 1, r, 1, M, L, 0, mhm.MHM_MIXED)
    kd = torch.as_tensor(np.concatenate(kap), device="cuda")
    src = mhm.Source(mhm.MHM_SRC_SINSIN, 1.0, 1.0)
    mhm.mhm_set_timing(p.mesh, True)
    p.local(kd, src, OPTS)
    times = mhm.mhm_kernel_times(p.mesh)
    torch.cuda.synchronize()
    assert times["k_local_mixed"][0] == 1 and times["k_local_fp64"][0] == 1, times
    assert p.status.cpu().tolist() == [0, 0]
    it = p.iters.cpu().tolist()
    assert 1 <= it[0] <= 6 and it[1] == -1, it
    NI = p.mesh.n_I
    AK = p.AK.view(-1, NI, NI).cpu().numpy()
    EK = p.EK.view(-1, NI).cpu().numpy()
    BK, FK = p.BK.view(-1, NI).cpu().numpy(), p.FK.cpu().numpy()
    mesh = build_mesh(1, 1, M, L)
    f = lambda x, y: 2 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y)
    for K in range(2):
        o = solve_local(mesh, K, r, 1, kap[K], f)
        tol = _fp64_bound(o, kap[K], 1e-9) if r == 7 else 1e-9
        assert_blocks(AK[K], EK[K], BK[K], FK[K], o, tol, (r, K, tol))


@pytest.mark.parametrize("r", [6, 7])
def test_wide_level_fallback_and_no_fallback(r):
    """With one CG iteration allowed the mixed element does not converge: it is solved
    again by the FP64 path, and its blocks equal the FP64 path's bit for bit.  With the
    re-solve off, the elements keep MHM_ERR_NOT_CONVERGED and MHM_ERR_UNSUPPORTED (pinned
    DOF on row 1), and the outcome word carries both."""
    from paper_1703_10435_gb300.pipeline import Pipeline
    N, kap = _case(r)
    kd = torch.as_tensor(np.concatenate(kap), device="cuda")
    src = mhm.Source(mhm.MHM_SRC_CONST, 1.0, 1.0)
    p = Pipeline(1, 1, r, 1, M, L, 0, mhm.MHM_MIXED)
    q = Pipeline(1, 1, r, 1, M, L, 0, mhm.MHM_FP64)
    q.local(kd, src)
    p.local(kd, src, mhm.SolveOpts(1, 1e-13, 0, 0))
    torch.cuda.synchronize()
    assert p.status.cpu().tolist() == [0, 0]
    assert p.iters.cpu().tolist() == [-1, -1]
    assert torch.equal(p.AK, q.AK) and torch.equal(p.EK, q.EK)
    mhm.mhm_sync_status(p.mesh)
    p.local(kd, src, mhm.SolveOpts(1, 1e-13, 0, 0, 1))
    torch.cuda.synchronize()
    assert p.status.cpu().tolist() == [mhm.MHM_ERR_NOT_CONVERGED, mhm.MHM_ERR_UNSUPPORTED]
    code, word = mhm.mhm_sync_status(p.mesh)
    assert code == mhm.MHM_ERR_UNSUPPORTED
    assert word & (1 << mhm.MHM_ERR_NOT_CONVERGED) and word & (1 << mhm.MHM_ERR_UNSUPPORTED)


def test_wide_level_mixed_vs_fp64_on_channel_elements():
    """Level-7 elements of the channel workload (contrast 1e4 across 0.01-wide channels),
    on the 8 right isosceles triangles of a 2 x 2 mesh: CG converges within it_max (8) and
    in 4 iterations or fewer on average at the default tolerance.  The two paths reach the pinned solution by different FP64
    arithmetic (a Cholesky factor's Gram form; CG residuals with the corrected bilinear
    form), each to about u cond(A) (u = 2^-53, cond on the mean-zero space, ~1e8 here):
    on the element where they differ most, both are held to the oracle at max(1e-10,
    10 u cond), entry by entry."""
    from paper_1703_10435_gb300 import workloads as W
    from paper_1703_10435_gb300.pipeline import Pipeline
    from _blocks import gram_entry_error
    w = W.WORKLOADS["c4_channels"]
    rk = w.r_per_K
    idx = np.flatnonzero(rk == 7)
    crossing = [int(K) for K in idx if W.kappa_levels(w, [int(K)])[0].max() > 1.0][:8]
    kap = W.kappa_levels(w, crossing)
    out = {}
    for prec in (mhm.MHM_FP64, mhm.MHM_MIXED):
        p = Pipeline(2, 2, 7, 1, 1, 3, 0, prec)
        p.local(torch.as_tensor(np.concatenate(kap), device="cuda"), mhm.Source(mhm.MHM_SRC_CONST, 1.0, 1.0))
        torch.cuda.synchronize()
        assert int(p.status.abs().sum()) == 0
        out[prec] = (p.AK.view(len(crossing), -1).cpu().numpy(), p.iters.cpu().numpy())
    a64, amx = out[mhm.MHM_FP64][0], out[mhm.MHM_MIXED][0]
    it = out[mhm.MHM_MIXED][1]
    assert np.all((it == -1) | ((it >= 1) & (it <= 8))) and float(it[it > 0].mean()) <= 4.0, it
    d = np.linalg.norm(amx - a64, axis=1) / np.linalg.norm(a64, axis=1)
    K = int(np.argmax(d))
    o = solve_local(build_mesh(2, 2, 1, 3), K, 7, 1, kap[K], 1.0)
    tol = _fp64_bound(o, kap[K], 1e-10)
    NI = o.AK.shape[0]
    e_mx = gram_entry_error(amx[K].reshape(NI, NI), o.AK)
    e_64 = gram_entry_error(a64[K].reshape(NI, NI), o.AK)
    assert e_mx < tol and e_64 < tol, (K, d[K], e_mx, e_64, tol)
