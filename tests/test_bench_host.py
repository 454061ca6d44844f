"""Host-side checks of bench.py's accounting (no GPU): the FP64 work of one refinement
pass equals the nonzero stencil weights of the pinned stiffness matrix, as the oracle
assembles it, times the right-hand sides; the config object names the workload's shape."""
import numpy as np
import pytest

import bench
from oracle.fem import Submesh
from oracle.local import assemble_stiffness
from oracle.mesh import build_mesh
from paper_1703_10435_gb300 import workloads as W


@pytest.mark.parametrize("r", [1, 2, 3, 5])
def test_residual_fmas_equal_stencil_nonzeros(r):
    w = W.Workload("t", 1, 1, r, 1, 2, 2, "one", "const")
    mesh = build_mesh(1, 1, 2, 2)
    nnz = 0
    for K in (0, 1):   # the two orientations of the coarse triangles
        sub = Submesh(mesh.verts[mesh.tris[K]], r, 1)
        A = assemble_stiffness(sub, np.ones(4 ** r)).toarray()[1:, 1:]   # DOF 0 pinned
        nnz += int((np.abs(A) > 1e-12 * np.abs(A).max()).sum())
    assert bench.residual_fmas_per_pass(w) == nnz / 2 * (w.n_I + 1)


def test_workload_config_shapes():
    c2 = bench.workload_config(W.WORKLOADS["c2_hetero_fp64"])
    assert (c2["r"], c2["n_local"], c2["l"], c2["rhs"]) == (5, 561, 2, 19)
    c4 = bench.workload_config(W.WORKLOADS["c4_channels"])
    assert "r" not in c4 and sum(c4["elements_per_level"].values()) == 8192
    assert set(c4["elements_per_level"]) == {"3", "4", "5", "6", "7"}
    assert "l_per_face" in c4 and c4["rhs"] == 13
    assert [bench.mixed_level(W.WORKLOADS["c4_channels"], r) for r in (3, 5, 6, 7)] == [True, True, False, False]
    assert bench.mixed_level(W.WORKLOADS["c5_p2_large"], 4) and not bench.mixed_level(W.WORKLOADS["c5_p2_large"], 5)
