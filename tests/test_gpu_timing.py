"""Per-kernel timing of the local solves (mhm_set_timing / mhm_kernel_times): the
library's CUDA events around each launch report the kernels each precision runs."""
import pytest

torch = pytest.importorskip("torch")

from paper_1703_10435_gb300 import mhm, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_10435_gb300 import build
    build.build()


@pytest.mark.parametrize("precision,expect", [
    (mhm.MHM_FP64, {"k_local_fp64": 1}),
    # mixed: factor, solve, and the FP64 re-solve of failed elements (launched with a
    # device-side count, here zero)
    (mhm.MHM_MIXED, {"k_schur_factor": 1, "k_local_mixed": 1, "k_local_fp64": 1}),
])
def test_kernel_times(precision, expect):
    from paper_1703_10435_gb300.pipeline import Pipeline, source_of
    w = W.WORKLOADS["c1_sin"]
    kap = torch.as_tensor(W.kappa_for(w), device="cuda")
    p = Pipeline.for_workload(w, 0, precision)
    p.local(kap, source_of(w))
    mhm.mhm_set_timing(p.mesh, True)
    for _ in range(2):
        p.local(kap, source_of(w))
    kt = mhm.mhm_kernel_times(p.mesh)
    assert {k: v[0] for k, v in kt.items()} == {k: 2 * n for k, n in expect.items()}
    assert all(ms > 0.0 for _, ms in kt.values())
    assert mhm.mhm_kernel_times(p.mesh) == {}          # a reading starts the next one
    mhm.mhm_set_timing(p.mesh, False)
    p.local(kap, source_of(w))
    assert mhm.mhm_kernel_times(p.mesh) == {}
