"""Device buffers around the C calls: one object per mesh that owns the
torch tensors the library writes into (per-K blocks, skeleton CSR values,
right-hand side, status) and runs mhm_local_solve_batch followed by
mhm_assemble_skeleton on a stream."""
from __future__ import annotations

import numpy as np
import torch

from . import mhm
from .workloads import Workload


def source_of(w: Workload) -> mhm.Source:
    if w.source == "const":
        return mhm.Source(mhm.MHM_SRC_CONST, w.source_value, 1.0)
    return mhm.Source(mhm.MHM_SRC_SINSIN, w.source_value, w.source_freq)


def dirichlet_of(w: Workload):
    if w.dirichlet is None:
        return None
    c = list(w.dirichlet) + [0.0] * (6 - len(w.dirichlet))
    return mhm.Dirichlet((mhm.ctypes.c_double * 6)(*c))


class Pipeline:
    def __init__(self, nx, ny, r, degree, m, l, device: int = 0, precision: int = mhm.MHM_FP64, r_per_K=None,
                 l_per_face=None):
        self.mesh = mhm.Mesh(nx, ny, r, degree, m, l, device, r_per_K, l_per_face)
        self.device = torch.device("cuda", device)
        self.precision = precision
        M = self.mesh
        f64 = dict(dtype=torch.float64, device=self.device)
        i32 = dict(dtype=torch.int32, device=self.device)
        self.AK = torch.zeros(M.n_K * M.n_I * M.n_I, **f64)
        self.EK = torch.zeros(M.n_K * M.n_I, **f64)
        self.BK = torch.zeros(M.n_K * M.n_I, **f64)
        self.FK = torch.zeros(M.n_K, **f64)
        self.status = torch.zeros(M.n_K, **i32)
        self.iters = torch.zeros(M.n_K, **i32)
        self.A_vals = torch.zeros(M.nnz, **f64)
        self.E = torch.zeros(M.n_lambda, **f64)
        self.workspace = None
        self.set_precision(precision)

    @classmethod
    def for_workload(cls, w: Workload, device: int = 0, precision: int = mhm.MHM_FP64):
        rk = w.r_per_K
        lf = None
        if w.face_degree is not None:
            # the face numbering from a host-only mesh of the same T_H
            h = mhm.Mesh(w.nx, w.ny, w.r, w.degree, w.m, w.l, -1, rk)
            lf = w.l_per_face(h.query(mhm.Q_TRI_FACES, np.int32, 3 * h.n_K))
            h.close()
        return cls(w.nx, w.ny, w.r, w.degree, w.m, w.l, device, precision, rk, lf)

    def set_precision(self, precision: int):
        self.precision = precision
        ws = mhm.mhm_local_workspace_size(self.mesh, precision)
        if ws > 0 and (self.workspace is None or self.workspace.numel() < ws):
            self.workspace = torch.empty(ws, dtype=torch.uint8, device=self.device)

    def local(self, kappa, source: mhm.Source, opts: mhm.SolveOpts | None = None, stream=None):
        mhm.mhm_local_solve_batch(self.mesh, kappa, source, self.precision, opts, self.AK, self.EK, self.BK,
                                  self.FK, self.status, self.iters, self.workspace, stream)

    def skeleton(self, dirichlet=None, stream=None):
        mhm.mhm_assemble_skeleton(self.mesh, self.AK, self.EK, dirichlet, self.A_vals, self.E, stream)

    def step(self, kappa, source, dirichlet=None, opts=None, stream=None):
        self.local(kappa, source, opts, stream)
        self.skeleton(dirichlet, stream)

    def solve_global(self, stream=None):
        """lambda, u0 of Eq. "mat_global" from the current skeleton and per-K blocks."""
        M = self.mesh
        self.lam = torch.zeros(M.n_lambda, dtype=torch.float64, device=self.device)
        self.u0 = torch.zeros(M.n_K, dtype=torch.float64, device=self.device)
        mhm.mhm_solve_global(M, self.A_vals, self.E, self.BK, self.FK, self.lam, self.u0, stream)
        return self.lam, self.u0

    def reconstruct(self, kappa, source, exact=None, stream=None):
        """Nodal u_{H,h} per K (n_K x n_local; with a level per K a flat array, K's values
        at mesh.nodal_offset[K]) and, with `exact`, per-K squared L2/H1 errors."""
        M = self.mesh
        u = torch.empty(int(M.nodal_offset[-1]), dtype=torch.float64, device=self.device)
        err = torch.empty(2 * M.n_K, dtype=torch.float64, device=self.device) if exact is not None else None
        mhm.mhm_reconstruct(M, kappa, source, self.lam, self.u0, exact, u, err, stream)
        uv = u if len(set(M.r_of_K.tolist())) > 1 else u.view(M.n_K, M.n_local)
        return uv, (None if err is None else err.view(M.n_K, 2))

    def local_waves(self, kappa_host, source, budget_bytes: int, opts=None, stream=None):
        """Local solves with kappa on the host, in memory-admitted waves
        (mhm_local_solve_waves): contiguous K ranges whose kappa fits in half of
        `budget_bytes`, two device buffers alternating so that the copy of the next wave
        overlaps the solves of the current one.  Returns the number of waves."""
        kh = torch.as_tensor(kappa_host, dtype=torch.float64).reshape(-1).contiguous()
        if not kh.is_pinned():
            kh = kh.pin_memory()
        n = mhm.mhm_local_solve_waves(self.mesh, kh, budget_bytes, source, self.precision, opts, self.AK, self.EK,
                                      self.BK, self.FK, self.status, self.iters, self.workspace, stream)
        # the copies read kh until the work on the stream is done
        (torch.cuda.current_stream() if stream is None else stream).synchronize()
        return n

    # host-side views for tests and reports
    def blocks(self):
        M = self.mesh
        return (self.AK.view(M.n_K, M.n_I, M.n_I).cpu().numpy(), self.EK.view(M.n_K, M.n_I).cpu().numpy(),
                self.BK.view(M.n_K, M.n_I).cpu().numpy(), self.FK.cpu().numpy())

    def skeleton_scipy(self):
        import scipy.sparse
        M = self.mesh
        rowptr = M.query(mhm.Q_CSR_ROWPTR, np.int32, M.n_lambda + 1)
        cols = M.query(mhm.Q_CSR_COLS, np.int32, M.nnz)
        return scipy.sparse.csr_matrix((self.A_vals.cpu().numpy(), cols, rowptr), shape=(M.n_lambda, M.n_lambda))
