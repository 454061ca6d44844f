"""The allocation-free mixed-precision entry point (for callers that cannot
allocate device memory while they run, e.g. when a framework's memory pool
owns the device, or inside a loop that must not call cudaMalloc): called
through the C ABI twice in a row, it must give the same per-element blocks as
the workspace-taking entry point, within the mixed-precision tolerance the
other tests use.  Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1703_10435_gb300 import mhm, workloads as W

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-9


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_10435_gb300 import build
    build.build()


def _outputs(mesh):
    f64 = dict(dtype=torch.float64, device="cuda")
    n, ni = mesh.n_K, mesh.n_I
    return (torch.full((n * ni * ni,), float("nan"), **f64), torch.full((n * ni,), float("nan"), **f64),
            torch.full((n * ni,), float("nan"), **f64), torch.full((n,), float("nan"), **f64),
            torch.full((n,), -1, dtype=torch.int32, device="cuda"),
            torch.zeros(n, dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("name,nx", [("c2_hetero_fp64", 32), ("c5_p2_large", 4)])
def test_noalloc_matches_workspace_entry_point_twice(name, nx):
    w0 = W.WORKLOADS[name]
    w = W.Workload(w0.name, nx, nx, w0.r, w0.degree, w0.m, w0.l, w0.field, w0.source, w0.source_value, seed=w0.seed)
    mesh = mhm.Mesh(w.nx, w.ny, w.r, w.degree, w.m, w.l, 0)
    kap = torch.as_tensor(W.kappa_for(w), device="cuda").contiguous()
    src = mhm.Source(mhm.MHM_SRC_CONST, w.source_value, 1.0)
    opts = mhm.SolveOpts(10, 1e-13, 0, 0)

    ref = _outputs(mesh)
    ws = torch.empty(mhm.mhm_local_workspace_size(mesh, mhm.MHM_MIXED), dtype=torch.uint8, device="cuda")
    mhm.mhm_local_solve_batch(mesh, kap, src, mhm.MHM_MIXED, opts, *ref[:5], ref[5], ws)
    torch.cuda.synchronize()
    assert int(ref[4].abs().sum()) == 0

    for call in range(2):
        out = _outputs(mesh)
        mhm.mhm_local_solve_batch_noalloc(mesh, kap, src, opts, *out)
        torch.cuda.synchronize()
        assert int(out[4].abs().sum()) == 0, "call %d: status" % call
        A, Ar = out[0].view(mesh.n_K, -1).cpu().numpy(), ref[0].view(mesh.n_K, -1).cpu().numpy()
        err = np.linalg.norm(A - Ar, axis=1) / np.linalg.norm(Ar, axis=1)
        assert err.max() < TOL_MIXED, (call, err.max())
        for a, b in zip(out[1:4], ref[1:4]):
            a, b = a.cpu().numpy(), b.cpu().numpy()
            assert np.all(np.isfinite(a))
            assert np.abs(a - b).max() <= TOL_MIXED * max(np.abs(b).max(), np.abs(Ar).max())


def test_noalloc_rejects_null_arguments():
    mesh = mhm.Mesh(1, 1, 2, 1, 1, 1, 0)
    code = mhm.lib().mhm_local_solve_batch_noalloc(mesh.handle, None, None, None, None, None, None, None,
                                                   None, None, None)
    assert code == mhm.MHM_ERR_INVALID_ARG
