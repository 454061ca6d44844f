"""Python binding of the C ABI in include/mhm.h (argument marshalling only).

Functions keep the C names.  Device arrays are torch tensors on the mesh's
device; their data pointers and the current CUDA stream are passed straight
to the library, which runs every step of the pipeline in its own kernels.
The library must be built (``paper_1703_10435_gb300.build.build()``); there
is no fallback when it is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmhm.so")

MHM_OK = 0
MHM_ERR_INVALID_ARG = 1
MHM_ERR_OOM = 2
MHM_ERR_CUDA = 3
MHM_ERR_NOT_CONVERGED = 4
MHM_ERR_TIMEOUT = 5
MHM_ERR_UNSUPPORTED = 6

MHM_FP64 = 0
MHM_MIXED = 1
MHM_SRC_CONST = 0
MHM_SRC_SINSIN = 1
MHM_SRC_QUAD = 2
MHM_STATUS_REFINED_IN_FP64 = 1 << 16

Q_SIZES, Q_TRI_VERTS, Q_TRI_FACES, Q_TRI_SIGNS, Q_FACE_VERTS, Q_LAMBDA_OFFSET, Q_K_LAMBDA, \
    Q_CSR_ROWPTR, Q_CSR_COLS, Q_VERTEX_XY, Q_FACE_NORMALS, Q_R_OF_K, Q_KAPPA_OFFSET, Q_NODAL_OFFSET, \
    Q_FACE_DEGREE, Q_SYSTEM_NNZ = range(16)

EXPORTED = [
    "mhm_create_mesh", "mhm_destroy_mesh", "mhm_mesh_query", "mhm_local_workspace_size",
    "mhm_local_solve_batch", "mhm_assemble_skeleton", "mhm_last_error", "mhm_measure_pipes",
    "mhm_local_solve_batch_noalloc", "mhm_solve_global", "mhm_reconstruct", "mhm_set_timing", "mhm_kernel_times",
    "mhm_local_solve_waves", "mhm_sync_status", "mhm_factor_store_size", "mhm_set_tuning", "mhm_get_tuning",
    "mhm_autotune",
]
MHM_KERNEL_LOCAL_FP64, MHM_KERNEL_LOCAL_MIXED, MHM_KERNEL_SCHUR_FACTOR = range(3)
MHM_N_KERNELS = 3
KERNEL_NAMES = ("k_local_fp64", "k_local_mixed", "k_schur_factor")
MHM_EXACT_SINSIN = 1
MHM_EXACT_POLY = 2


class MeshDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("r", ctypes.c_int32),
                ("degree", ctypes.c_int32), ("m", ctypes.c_int32), ("l", ctypes.c_int32),
                ("r_per_K", ctypes.c_void_p), ("l_per_face", ctypes.c_void_p)]


class Source(ctypes.Structure):
    """mhm_source: kind, value, freq, and for MHM_SRC_QUAD the device pointer of the point
    values (keep the tensor alive while the calls that use it run)."""
    _fields_ = [("kind", ctypes.c_int32), ("value", ctypes.c_double), ("freq", ctypes.c_double),
                ("values_dev", ctypes.c_void_p)]


def quad_source(values) -> Source:
    """A source given by its values at the 16 collapsed-Gauss points of every fine triangle
    (a contiguous float64 device tensor laid out like kappa, 16 values per fine triangle)."""
    src = Source(MHM_SRC_QUAD, 0.0, 0.0, ctypes.c_void_p(values.data_ptr()))
    src._values = values   # keeps the tensor alive with the struct
    return src


class Dirichlet(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double * 6)]


class Exact(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("c", ctypes.c_double * 6)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("it_max", ctypes.c_int32), ("tol", ctypes.c_double),
                ("K_begin", ctypes.c_int64), ("K_end", ctypes.c_int64), ("no_fallback", ctypes.c_int32),
                ("factor_store", ctypes.c_void_p), ("factor_store_bytes", ctypes.c_size_t),
                ("factor_reuse", ctypes.c_int32), ("tuner_cache", ctypes.c_char_p)]


class Tuning(ctypes.Structure):
    """mhm_tuning: launch shape of the mixed local solves of one level."""
    _fields_ = [("chunk", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("op_buffers", ctypes.c_int32),
                ("l2_prefetch", ctypes.c_int32), ("prefetch_all", ctypes.c_int32), ("op_policy", ctypes.c_int32),
                ("ms_per_K", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def solve_opts(it_max=8, tol=1e-12, K_begin=0, K_end=0, no_fallback=0, factor_store=None, factor_reuse=0,
               tuner_cache=None):
    """mhm_solve_opts with an optional factor store (a uint8 device tensor of at least
    mhm_factor_store_size bytes) and tuning cache path."""
    o = SolveOpts(it_max, tol, K_begin, K_end, no_fallback)
    if tuner_cache is not None:
        o._cache = str(tuner_cache).encode()
        o.tuner_cache = o._cache
    if factor_store is not None:
        o.factor_store = ctypes.c_void_p(factor_store.data_ptr())
        o.factor_store_bytes = factor_store.numel() * factor_store.element_size()
        o.factor_reuse = factor_reuse
        o._store = factor_store   # keeps the tensor alive with the struct
    return o


class MHMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("mhm error %d: %s" % (code, msg))
        self.code = code


_lib = None


def lib():
    """The loaded libmhm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise MHMError(MHM_ERR_UNSUPPORTED, "libmhm.so is not built; run paper_1703_10435_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        L.mhm_create_mesh.argtypes = [ctypes.POINTER(MeshDesc), i32, ctypes.POINTER(vp)]
        L.mhm_destroy_mesh.argtypes = [vp]
        L.mhm_destroy_mesh.restype = None
        L.mhm_mesh_query.argtypes = [vp, i32, vp, sz]
        L.mhm_local_workspace_size.argtypes = [vp, i32, ctypes.POINTER(sz)]
        L.mhm_local_solve_batch.argtypes = [vp, vp, ctypes.POINTER(Source), i32, ctypes.POINTER(SolveOpts),
                                            vp, vp, vp, vp, vp, vp, vp, sz, vp]
        L.mhm_local_solve_waves.argtypes = [vp, vp, sz, ctypes.POINTER(Source), i32, ctypes.POINTER(SolveOpts),
                                            vp, vp, vp, vp, vp, vp, vp, sz, vp, ctypes.POINTER(i32)]
        L.mhm_assemble_skeleton.argtypes = [vp, vp, vp, ctypes.POINTER(Dirichlet), vp, vp, vp]
        L.mhm_local_solve_batch_noalloc.argtypes = [vp, vp, ctypes.POINTER(Source), ctypes.POINTER(SolveOpts),
                                                    vp, vp, vp, vp, vp, vp, vp]
        L.mhm_solve_global.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
        L.mhm_reconstruct.argtypes = [vp, vp, ctypes.POINTER(Source), vp, vp, ctypes.POINTER(Exact), vp, vp, vp]
        L.mhm_last_error.restype = ctypes.c_char_p
        L.mhm_measure_pipes.argtypes = [i32, ctypes.POINTER(ctypes.c_double)]
        L.mhm_set_timing.argtypes = [vp, i32]
        L.mhm_kernel_times.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)]
        L.mhm_sync_status.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_uint32)]
        L.mhm_factor_store_size.argtypes = [vp, ctypes.POINTER(sz)]
        L.mhm_factor_store_size.restype = i32
        L.mhm_set_tuning.argtypes = [vp, i32, ctypes.POINTER(Tuning)]
        L.mhm_get_tuning.argtypes = [vp, i32, ctypes.POINTER(Tuning)]
        L.mhm_autotune.argtypes = [vp, vp, ctypes.POINTER(Source), ctypes.POINTER(SolveOpts), vp, vp, vp, vp, vp, vp,
                                   vp, sz, ctypes.c_char_p, vp]
        for name in ("mhm_set_tuning", "mhm_get_tuning", "mhm_autotune"):
            getattr(L, name).restype = i32
        L.mhm_sync_status.restype = i32
        for name in ("mhm_create_mesh", "mhm_mesh_query", "mhm_local_workspace_size", "mhm_local_solve_batch",
                     "mhm_assemble_skeleton", "mhm_measure_pipes", "mhm_local_solve_batch_noalloc",
                     "mhm_solve_global", "mhm_reconstruct", "mhm_set_timing", "mhm_kernel_times",
                     "mhm_local_solve_waves"):
            getattr(L, name).restype = i32
        _bind3d(L)
        _lib = L
    return _lib


def _check(code):
    if code != MHM_OK:
        raise MHMError(code, lib().mhm_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Mesh:
    """Owning handle of an mhm_mesh (splitProblem)."""

    def __init__(self, nx, ny, r, degree, m, l, device: int = 0, r_per_K=None, l_per_face=None):
        """r_per_K: optional refinement level of every K (sequence of n_K ints); r is
        then ignored.  l_per_face: optional multiplier degree of every face (global face
        numbering); l is then ignored."""
        rk = lf = None
        if r_per_K is not None:
            rk = np.ascontiguousarray(np.asarray(r_per_K, dtype=np.int8))
        if l_per_face is not None:
            lf = np.ascontiguousarray(np.asarray(l_per_face, dtype=np.int8))
        self.desc = MeshDesc(nx, ny, r, degree, m, l, None if rk is None else rk.ctypes.data,
                             None if lf is None else lf.ctypes.data)
        h = ctypes.c_void_p()
        _check(lib().mhm_create_mesh(ctypes.byref(self.desc), device, ctypes.byref(h)))
        self.handle = h
        self.device = device
        s = self.query(Q_SIZES, np.int64, 8)
        (self.n_K, self.n_faces, self.n_vertices, self.n_lambda, self.n_fine, self.n_local,
         self.n_I, self.nnz) = [int(v) for v in s]
        self.r_of_K = self.query(Q_R_OF_K, np.int8, self.n_K)
        self.kappa_offset = self.query(Q_KAPPA_OFFSET, np.int64, self.n_K + 1)   # 4^r_K values per K
        self.nodal_offset = self.query(Q_NODAL_OFFSET, np.int64, self.n_K + 1)   # n_local(r_K) values per K
        self.face_degree = self.query(Q_FACE_DEGREE, np.int8, self.n_faces)

    def query(self, what, dtype, count):
        out = np.empty(count, dtype=dtype)
        _check(lib().mhm_mesh_query(self.handle, what, out.ctypes.data_as(ctypes.c_void_p), out.nbytes))
        return out

    def close(self):
        if self.handle is not None and _lib is not None:
            _lib.mhm_destroy_mesh(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mhm_create_mesh(nx, ny, r, degree, m, l, device: int = 0, r_per_K=None, l_per_face=None) -> Mesh:
    return Mesh(nx, ny, r, degree, m, l, device, r_per_K, l_per_face)


def mhm_factor_store_size(mesh: Mesh) -> int:
    n = ctypes.c_size_t()
    _check(lib().mhm_factor_store_size(mesh.handle, ctypes.byref(n)))
    return int(n.value)


def mhm_local_workspace_size(mesh: Mesh, precision: int) -> int:
    n = ctypes.c_size_t()
    _check(lib().mhm_local_workspace_size(mesh.handle, precision, ctypes.byref(n)))
    return int(n.value)


def mhm_local_solve_waves(mesh: Mesh, kappa_host, budget_bytes: int, source: Source, precision,
                          opts: SolveOpts | None, AK, EK, BK, FK, status, iters=None, workspace=None,
                          stream=None) -> int:
    """kappa_host: a contiguous float64 CPU tensor (pinned for overlapped copies) holding the
    whole batch's kappa; returns the number of waves."""
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    if kappa_host.is_cuda or not kappa_host.is_contiguous():
        raise ValueError("kappa_host must be a contiguous CPU tensor")
    n = ctypes.c_int32(0)
    _check(lib().mhm_local_solve_waves(mesh.handle, _ptr(kappa_host), int(budget_bytes), ctypes.byref(source),
                                       precision, None if opts is None else ctypes.byref(opts),
                                       _ptr(AK), _ptr(EK), _ptr(BK), _ptr(FK), _ptr(status), _ptr(iters),
                                       _ptr(workspace), ws_bytes, _stream(stream), ctypes.byref(n)))
    return int(n.value)


def mhm_local_solve_batch(mesh: Mesh, kappa, source: Source, precision, opts: SolveOpts | None,
                          AK, EK, BK, FK, status, iters=None, workspace=None, stream=None):
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(lib().mhm_local_solve_batch(mesh.handle, _ptr(kappa), ctypes.byref(source), precision,
                                       None if opts is None else ctypes.byref(opts),
                                       _ptr(AK), _ptr(EK), _ptr(BK), _ptr(FK), _ptr(status), _ptr(iters),
                                       _ptr(workspace), ws_bytes, _stream(stream)))


def mhm_local_solve_batch_noalloc(mesh: Mesh, kappa, source: Source, opts: SolveOpts | None,
                                  AK, EK, BK, FK, status, iters=None, stream=None):
    """Mixed-precision local solves with the library's fixed scratch array (no allocation)."""
    _check(lib().mhm_local_solve_batch_noalloc(mesh.handle, _ptr(kappa), ctypes.byref(source),
                                               None if opts is None else ctypes.byref(opts),
                                               _ptr(AK), _ptr(EK), _ptr(BK), _ptr(FK), _ptr(status),
                                               _ptr(iters), _stream(stream)))


def mhm_assemble_skeleton(mesh: Mesh, AK, EK, dirichlet: Dirichlet | None, A_vals, E, stream=None):
    _check(lib().mhm_assemble_skeleton(mesh.handle, _ptr(AK), _ptr(EK),
                                       None if dirichlet is None else ctypes.byref(dirichlet),
                                       _ptr(A_vals), _ptr(E), _stream(stream)))


def mhm_solve_global(mesh: Mesh, A_vals, E, BK, FK, lam, u0, stream=None):
    _check(lib().mhm_solve_global(mesh.handle, _ptr(A_vals), _ptr(E), _ptr(BK), _ptr(FK), _ptr(lam), _ptr(u0),
                                  _stream(stream)))


def mhm_reconstruct(mesh: Mesh, kappa, source: Source, lam, u0, exact: Exact | None, u_nodal, err_sq=None,
                    stream=None):
    _check(lib().mhm_reconstruct(mesh.handle, _ptr(kappa), ctypes.byref(source), _ptr(lam), _ptr(u0),
                                 None if exact is None else ctypes.byref(exact), _ptr(u_nodal), _ptr(err_sq),
                                 _stream(stream)))


def mhm_measure_pipes(device: int = 0):
    out = (ctypes.c_double * 2)()
    _check(lib().mhm_measure_pipes(device, out))
    return {"fp64_gflops": out[0], "fp32_gflops": out[1]}


def mhm_set_timing(mesh: Mesh, enable: bool = True):
    """Record CUDA events around each kernel launch of the following local solves on `mesh`."""
    _check(lib().mhm_set_timing(mesh.handle, 1 if enable else 0))


def mhm_kernel_times(mesh: Mesh):
    """{kernel name: (launches, total ms)} of the timed local solves on `mesh` since the last reading."""
    n = (ctypes.c_int32 * MHM_N_KERNELS)()
    ms = (ctypes.c_double * MHM_N_KERNELS)()
    _check(lib().mhm_kernel_times(mesh.handle, n, ms))
    return {KERNEL_NAMES[k]: (int(n[k]), float(ms[k])) for k in range(MHM_N_KERNELS) if n[k] > 0}


def mhm_sync_status(mesh: Mesh, stream=None):
    """(most severe final code recorded since the last read, the outcome word); waits for the
    work on `stream` and clears the word.  The code is returned, not raised."""
    w = ctypes.c_uint32(0)
    code = lib().mhm_sync_status(mesh.handle, _stream(stream), ctypes.byref(w))
    if code not in (MHM_OK, MHM_ERR_NOT_CONVERGED, MHM_ERR_INVALID_ARG, MHM_ERR_TIMEOUT, MHM_ERR_UNSUPPORTED) or (
            code in (MHM_ERR_INVALID_ARG, MHM_ERR_UNSUPPORTED) and not w.value):
        _check(code)
    return code, int(w.value)


def mhm_set_tuning(mesh: Mesh, r: int, t: Tuning):
    _check(lib().mhm_set_tuning(mesh.handle, r, ctypes.byref(t)))


def mhm_get_tuning(mesh: Mesh, r: int) -> Tuning:
    t = Tuning()
    _check(lib().mhm_get_tuning(mesh.handle, r, ctypes.byref(t)))
    return t


def mhm_autotune(mesh: Mesh, kappa, source: Source, opts: SolveOpts | None, AK, EK, BK, FK, status, iters=None,
                 workspace=None, cache_path=None, stream=None):
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(lib().mhm_autotune(mesh.handle, _ptr(kappa), ctypes.byref(source), None if opts is None else ctypes.byref(opts),
                              _ptr(AK), _ptr(EK), _ptr(BK), _ptr(FK), _ptr(status), _ptr(iters), _ptr(workspace),
                              ws_bytes, None if cache_path is None else str(cache_path).encode(), _stream(stream)))


# ---------------------------------------------------------------- include/mhm3d.h
# The three-dimensional local problems (the paper's experiment, Sec. 5).

MHM3D_SRC_CONST = 0
MHM3D_SRC_SINSINSIN = 1
Q3_SIZES, Q3_TETS, Q3_TET_FACES, Q3_TET_SIGNS, Q3_FACES, Q3_VERTICES, Q3_NORMALS, Q3_CSR_ROWPTR, \
    Q3_CSR_COLS, Q3_SUB_DOFS, Q3_NODES, Q3_FACE_PERM, Q3_FTAB_OFF, Q3_FTAB_NODE, Q3_FTAB_COUNT, Q3_QUAD = range(16)
EXPORTED_3D = ["mhm3d_create_mesh", "mhm3d_destroy_mesh", "mhm3d_mesh_query", "mhm3d_local_solve_batch",
               "mhm3d_assemble_skeleton"]


class Mesh3DDesc(ctypes.Structure):
    _fields_ = [("nc", ctypes.c_int32), ("r", ctypes.c_int32), ("degree", ctypes.c_int32), ("m", ctypes.c_int32)]


class Source3D(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("value", ctypes.c_double), ("freq", ctypes.c_double)]


class Opts3D(ctypes.Structure):
    """mhm3d_opts: MIXED refinement passes, scaled residual target, no FP64 re-solve."""
    _fields_ = [("it_max", ctypes.c_int32), ("tol", ctypes.c_double), ("no_fallback", ctypes.c_int32)]


def _bind3d(L):
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    L.mhm3d_create_mesh.argtypes = [ctypes.POINTER(Mesh3DDesc), i32, ctypes.POINTER(vp)]
    L.mhm3d_destroy_mesh.argtypes = [vp]
    L.mhm3d_destroy_mesh.restype = None
    L.mhm3d_mesh_query.argtypes = [vp, i32, vp, sz]
    L.mhm3d_local_solve_batch.argtypes = [vp, vp, ctypes.POINTER(Source3D), i32, ctypes.POINTER(Opts3D), i64, i64,
                                          vp, vp, vp, vp, vp, vp, vp]
    L.mhm3d_assemble_skeleton.argtypes = [vp, vp, vp, vp, vp, vp]
    for name in ("mhm3d_create_mesh", "mhm3d_mesh_query", "mhm3d_local_solve_batch", "mhm3d_assemble_skeleton"):
        getattr(L, name).restype = i32


class Mesh3D:
    """Owning handle of an mhm3d_mesh (splitProblem on the unit cube)."""

    def __init__(self, nc, r, degree, m, device: int = 0):
        self.desc = Mesh3DDesc(nc, r, degree, m)
        h = ctypes.c_void_p()
        _check(lib().mhm3d_create_mesh(ctypes.byref(self.desc), device, ctypes.byref(h)))
        self.handle = h
        self.device = device
        (self.n_K, self.n_faces, self.n_vertices, self.n_lambda, self.n_local, self.n_I, self.n_sub,
         self.nnz) = [int(v) for v in self.query(Q3_SIZES, np.int64, 8)]

    def query(self, what, dtype, count):
        out = np.empty(count, dtype=dtype)
        _check(lib().mhm3d_mesh_query(self.handle, what, out.ctypes.data_as(ctypes.c_void_p), out.nbytes))
        return out

    def close(self):
        if self.handle is not None and _lib is not None:
            _lib.mhm3d_destroy_mesh(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mhm3d_create_mesh(nc, r, degree, m, device: int = 0) -> Mesh3D:
    return Mesh3D(nc, r, degree, m, device)


def mhm3d_local_solve_batch(mesh: Mesh3D, kappa, source: Source3D, AK, EK, BK, FK, status, K0=0, K1=0,
                            precision=MHM_FP64, opts: Opts3D | None = None, iters=None, stream=None):
    _check(lib().mhm3d_local_solve_batch(mesh.handle, _ptr(kappa), ctypes.byref(source), precision,
                                         None if opts is None else ctypes.byref(opts), K0, K1, _ptr(AK), _ptr(EK),
                                         _ptr(BK), _ptr(FK), _ptr(status), _ptr(iters), _stream(stream)))


def mhm3d_assemble_skeleton(mesh: Mesh3D, AK, EK, A_vals, E, stream=None):
    _check(lib().mhm3d_assemble_skeleton(mesh.handle, _ptr(AK), _ptr(EK), _ptr(A_vals), _ptr(E), _stream(stream)))
