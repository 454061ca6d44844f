"""Seeded synthetic inputs for the MHM local-problem pipeline.

This module holds input generators only: the counter-based random numbers,
the coefficient fields kappa sampled at fine-triangle centroids, the
workload descriptions (coarse mesh size, refinement, local degree,
multiplier space) and the manufactured sources.  It contains none of the
method's arithmetic; both the CUDA path and the CPU oracle consume the arrays
it returns, and neither is imported here.

Layout of a kappa array: one value per fine triangle, coarse elements in
ascending order, and inside each coarse element the fine triangles of its
N = 2^r lattice row by row (j = 0..N-1): first the N-j "up" triangles
(i,j),(i+1,j),(i,j+1) for i = 0..N-1-j, then the N-1-j "down" triangles
(i+1,j),(i+1,j+1),(i,j+1) for i = 0..N-2-j.  Lattice point (i,j) of the
coarse triangle (v0,v1,v2) sits at v0 + (i/N)(v1-v0) + (j/N)(v2-v0).

The coarse mesh of (0,1)^2 is nx*ny squares, square (i,j) split along its
(i,j)-(i+1,j+1) diagonal into K = 2(j*nx+i) with vertices
(i,j),(i+1,j),(i+1,j+1) and K+1 with vertices (i,j),(i+1,j+1),(i,j+1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


# ---------------------------------------------------------------------------
# Counter-based random numbers (SplitMix64 finaliser, Steele/Lea/Flood 2014)
# ---------------------------------------------------------------------------

def _mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def hash_u64(seed, a, b, stream) -> np.ndarray:
    """64-bit hash of the counter (seed, a, b, stream); broadcasts over arrays."""
    g = np.uint64(GOLDEN)
    with np.errstate(over="ignore"):
        h = _mix64(np.uint64(seed) + g)
        h = _mix64(h ^ (np.asarray(a, dtype=np.uint64) + g))
        h = _mix64(h ^ (np.asarray(b, dtype=np.uint64) + g))
        h = _mix64(h ^ (np.asarray(stream, dtype=np.uint64) + g))
    return h


def uniform01(seed, a, b, stream) -> np.ndarray:
    """Uniform in [0,1): the top 53 bits of the hash times 2^-53."""
    h = hash_u64(seed, a, b, stream)
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def gaussian(seed, a, b, stream) -> np.ndarray:
    """Standard normal by Box-Muller from two hashed uniforms (streams 2s, 2s+1)."""
    u1 = uniform01(seed, a, b, 2 * np.asarray(stream) + 0)
    u2 = uniform01(seed, a, b, 2 * np.asarray(stream) + 1)
    u1 = np.maximum(u1, 1e-300)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ---------------------------------------------------------------------------
# Geometry of the structured mesh, needed to place field samples
# ---------------------------------------------------------------------------

def coarse_vertices(nx: int, ny: int) -> np.ndarray:
    """(N_K, 3, 2) vertex coordinates of every coarse triangle, CCW."""
    ks = []
    for j in range(ny):
        for i in range(nx):
            p00 = (i / nx, j / ny)
            p10 = ((i + 1) / nx, j / ny)
            p11 = ((i + 1) / nx, (j + 1) / ny)
            p01 = (i / nx, (j + 1) / ny)
            ks.append((p00, p10, p11))
            ks.append((p00, p11, p01))
    return np.asarray(ks, dtype=np.float64)


def fine_centroid_lattice(N: int) -> np.ndarray:
    """(N*N, 2) lattice coordinates (in units of 1/N) of fine-triangle centroids."""
    out = []
    for j in range(N):
        for i in range(N - j):
            out.append((i + 1.0 / 3.0, j + 1.0 / 3.0))
        for i in range(N - 1 - j):
            out.append((i + 2.0 / 3.0, j + 2.0 / 3.0))
    return np.asarray(out, dtype=np.float64)


def fine_centroids(verts: np.ndarray, N: int) -> np.ndarray:
    """(N_K, N*N, 2) physical centroids for coarse triangles `verts` at N = 2^r."""
    lat = fine_centroid_lattice(N) / N
    v0 = verts[:, 0, None, :]
    e1 = (verts[:, 1] - verts[:, 0])[:, None, :]
    e2 = (verts[:, 2] - verts[:, 0])[:, None, :]
    return v0 + lat[None, :, 0, None] * e1 + lat[None, :, 1, None] * e2


def duffy_points_ref() -> np.ndarray:
    """(16, 2) reference points (xi, eta) of the collapsed 4 x 4 Gauss rule, point 4 i + j at
    xi = a_i, eta = a_j (1 - a_i) with a the 4-point Gauss-Legendre nodes on [0, 1] (the
    point order of a source given by its values, MHM_SRC_QUAD)."""
    a = 0.5 * (np.polynomial.legendre.leggauss(4)[0] + 1.0)
    return np.array([(a[i], a[j] * (1.0 - a[i])) for i in range(4) for j in range(4)])


def fine_triangle_lattice(N: int) -> np.ndarray:
    """(N*N, 3, 2) lattice coordinates (units of 1/N) of the fine-triangle vertices in the
    kappa order: "up" (i,j),(i+1,j),(i,j+1), then "down" (i+1,j),(i+1,j+1),(i,j+1)."""
    out = []
    for j in range(N):
        for i in range(N - j):
            out.append(((i, j), (i + 1, j), (i, j + 1)))
        for i in range(N - 1 - j):
            out.append(((i + 1, j), (i + 1, j + 1), (i, j + 1)))
    return np.asarray(out, dtype=np.float64)


def source_points(verts: np.ndarray, N: int) -> np.ndarray:
    """(N_K, N*N, 16, 2) physical positions of the 16 source points of every fine triangle
    of the coarse triangles `verts` (N_K, 3, 2) at N = 2^r, in the layout of a source given
    by its values: X0 + xi (X1 - X0) + eta (X2 - X0) per fine triangle (X0, X1, X2)."""
    lat = fine_triangle_lattice(N) / N                                    # (T, 3, 2)
    ref = duffy_points_ref()                                              # (16, 2)
    bary = lat[:, 0, None, :] + ref[None, :, 0, None] * (lat[:, 1] - lat[:, 0])[:, None, :] \
        + ref[None, :, 1, None] * (lat[:, 2] - lat[:, 0])[:, None, :]     # (T, 16, 2) in (s, t)
    v0 = verts[:, 0, None, None, :]
    e1 = (verts[:, 1] - verts[:, 0])[:, None, None, :]
    e2 = (verts[:, 2] - verts[:, 0])[:, None, None, :]
    return v0 + bary[None, ..., 0, None] * e1 + bary[None, ..., 1, None] * e2


# ---------------------------------------------------------------------------
# Coefficient fields
# ---------------------------------------------------------------------------

def kappa_log_uniform(n_K: int, n_fine: int, seed: int, lo: float = -2.0, hi: float = 2.0) -> np.ndarray:
    """kappa = 10^U with U ~ U[lo, hi] independently per fine triangle."""
    K = np.arange(n_K, dtype=np.uint64)[:, None]
    t = np.arange(n_fine, dtype=np.uint64)[None, :]
    u = uniform01(seed, K, t, 0)
    return 10.0 ** (lo + (hi - lo) * u)


@dataclass
class FourierField:
    """Gaussian random field by random Fourier features: g(x) = sqrt(2/F) sum cos(w_k.x + p_k),
    w_k ~ N(0, ell^-2 I), p_k ~ U[0, 2pi); unit variance."""
    seed: int
    ell: float = 0.02
    n_features: int = 512
    omega: np.ndarray = field(init=False)
    phase: np.ndarray = field(init=False)

    def __post_init__(self):
        k = np.arange(self.n_features, dtype=np.uint64)
        big = np.uint64(0xFFFFFFFF)
        self.omega = np.stack([gaussian(self.seed, big, k, 0), gaussian(self.seed, big, k, 1)], axis=1) / self.ell
        self.phase = 2.0 * math.pi * uniform01(self.seed, big, k, 7)

    def eval_numpy(self, xy: np.ndarray, chunk: int = 1 << 16) -> np.ndarray:
        flat = xy.reshape(-1, 2)
        out = np.empty(flat.shape[0], dtype=np.float64)
        s = math.sqrt(2.0 / self.n_features)
        for a in range(0, flat.shape[0], chunk):
            arg = flat[a:a + chunk] @ self.omega.T + self.phase[None, :]
            out[a:a + chunk] = s * np.cos(arg).sum(axis=1)
        return out.reshape(xy.shape[:-1])

    def eval_torch(self, xy, chunk: int = 1 << 18):
        import torch
        dev = xy.device
        om = torch.as_tensor(self.omega, dtype=torch.float64, device=dev)
        ph = torch.as_tensor(self.phase, dtype=torch.float64, device=dev)
        flat = xy.reshape(-1, 2)
        out = torch.empty(flat.shape[0], dtype=torch.float64, device=dev)
        s = math.sqrt(2.0 / self.n_features)
        for a in range(0, flat.shape[0], chunk):
            out[a:a + chunk] = s * torch.cos(flat[a:a + chunk] @ om.T + ph[None, :]).sum(dim=1)
        return out.reshape(xy.shape[:-1])


def kappa_from_gaussian(g, decades: float):
    """kappa = 10^(decades * clip(g/3, -1, 1)); contrast 10^(2*decades)."""
    if isinstance(g, np.ndarray):
        return 10.0 ** (decades * np.clip(g / 3.0, -1.0, 1.0))
    import torch
    return torch.pow(10.0, decades * torch.clamp(g / 3.0, -1.0, 1.0))


@dataclass
class ChannelField:
    """Background 1 with n straight channels of half-width w and value kappa_hi."""
    seed: int
    n_channels: int = 16
    half_width: float = 0.005
    kappa_hi: float = 1e4
    points: np.ndarray = field(init=False)
    dirs: np.ndarray = field(init=False)

    def __post_init__(self):
        c = np.arange(self.n_channels, dtype=np.uint64)
        big = np.uint64(0xFFFFFFFE)
        self.points = np.stack([uniform01(self.seed, big, c, 0), uniform01(self.seed, big, c, 1)], axis=1)
        ang = math.pi * uniform01(self.seed, big, c, 2)
        self.dirs = np.stack([np.cos(ang), np.sin(ang)], axis=1)

    def distance(self, xy: np.ndarray) -> np.ndarray:
        d = xy[..., None, :] - self.points
        normal = np.stack([-self.dirs[:, 1], self.dirs[:, 0]], axis=1)
        return np.abs((d * normal).sum(axis=-1)).min(axis=-1)

    def kappa(self, xy: np.ndarray) -> np.ndarray:
        return np.where(self.distance(xy) <= self.half_width, self.kappa_hi, 1.0)


# ---------------------------------------------------------------------------
# Workload descriptions
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    r: int
    degree: int
    m: int
    l: int
    field: str            # "one" | "log_uniform" | "grf4" | "grf6" | "channels"
    source: str           # "const" | "sinsin"
    source_value: float = 1.0
    source_freq: float = 1.0
    dirichlet: tuple | None = None   # (a, b, c) for g = a + b x + c y, None = homogeneous
    seed: int = 0
    levels: str | None = None        # None: every K at r; "channels": level per K from the channel field
    r_cap: int = 7                   # largest level a K gets ("channels")
    face_degree: str | None = None   # None: every face at l; "levels": l_e from the adjacent levels
                                     # (face_degree_from_levels; l is then the largest degree)

    @property
    def r_per_K(self):
        """Refinement level of every K (None: uniform r).  "channels": r_K = 7, 6, 5, 4, 3
        for a centroid within H/2, H, 2H, 4H of the nearest channel line, else (H the
        coarse square size), capped at r_cap."""
        if self.levels is None:
            return None
        if self.levels != "channels":
            raise ValueError(self.levels)
        cen = coarse_vertices(self.nx, self.ny).mean(axis=1)
        d = ChannelField(self.seed).distance(cen)
        H = 1.0 / self.nx
        r = np.full(self.n_K, 3, dtype=np.int8)
        for thr, lev in ((4 * H, 4), (2 * H, 5), (H, 6), (0.5 * H, 7)):
            r[d < thr] = lev
        return np.minimum(r, self.r_cap).astype(np.int8)

    def l_per_face(self, tri_faces):
        """Multiplier degree of every face (None: every face at l), given the global face
        id of each K's local faces (n_K x 3, any consistent face numbering)."""
        if self.face_degree is None:
            return None
        if self.face_degree != "levels":
            raise ValueError(self.face_degree)
        tf = np.asarray(tri_faces).reshape(-1, 3)
        rk = self.r_per_K if self.r_per_K is not None else np.full(self.n_K, self.r, dtype=np.int8)
        rmax = np.zeros(int(tf.max()) + 1, dtype=np.int64)
        np.maximum.at(rmax, tf.ravel(), np.repeat(rk.astype(np.int64), 3))
        return face_degree_from_levels(rmax)

    @property
    def n_K(self) -> int:
        return 2 * self.nx * self.ny

    @property
    def N(self) -> int:
        return 1 << self.r

    @property
    def n_fine(self) -> int:
        return self.N * self.N

    @property
    def n_local(self) -> int:
        pn = self.degree * self.N
        return (pn + 1) * (pn + 2) // 2

    @property
    def n_I(self) -> int:
        return 3 * self.m * (self.l + 1)


def face_degree_from_levels(r_adjacent_max):
    """Degree of a face's multipliers from the largest refinement level among its (one or
    two) coarse elements: 1 + [r >= 5] + [r >= 7], so finer submeshes meet richer
    multiplier spaces."""
    r = np.asarray(r_adjacent_max)
    return (1 + (r >= 5).astype(np.int64) + (r >= 7).astype(np.int64)).astype(np.int8)


WORKLOADS = {
    # 4x4 squares (32 K), r=3 P1, m=1 l=1, kappa = 1, u = sin(pi x) sin(pi y)
    "c1_sin": Workload("c1_sin", 4, 4, 3, 1, 1, 1, "one", "sinsin", 1.0, 1.0),
    # same mesh, linear u = 1 + 2x - 3y (f = 0, g = u) recovered exactly
    "c1_linear": Workload("c1_linear", 4, 4, 3, 1, 1, 1, "one", "const", 0.0, dirichlet=(1.0, 2.0, -3.0)),
    # 32x32 squares (2048 K), r=5 P1 (561 DOFs), m=2 l=2 (18 lambda-RHS), log-uniform kappa, f = 1
    "c2_hetero_fp64": Workload("c2_hetero_fp64", 32, 32, 5, 1, 2, 2, "log_uniform", "const", 1.0),
    # 128x128 squares (32768 K), r=5 P1, m=2 l=2, GRF contrast 1e4, f = 1
    "c3_grf_mixed": Workload("c3_grf_mixed", 128, 128, 5, 1, 2, 2, "grf4", "const", 1.0),
    # 256x256 squares (131072 K), r=4 P2 (561 DOFs), m=3 l=1, GRF contrast 1e6, f = 1
    "c5_p2_large": Workload("c5_p2_large", 256, 256, 4, 2, 3, 1, "grf6", "const", 1.0),
    # uneven levels 3..7: 64x64 squares, level per K from 16 channels of kappa = 1e4, P1,
    # one subface per face with degree 1..3 multipliers by the adjacent levels
    "c4_channels": Workload("c4_channels", 64, 64, 3, 1, 1, 3, "channels", "const", 1.0, levels="channels",
                            face_degree="levels"),
}


def kappa_levels(w: Workload, K_index=None):
    """Per K (all, or those in K_index) the kappa values of its own level (4^r_K values,
    fine-triangle order): a list of arrays.  For a workload with a level per K."""
    rk = w.r_per_K
    verts = coarse_vertices(w.nx, w.ny)
    Ks = np.arange(w.n_K) if K_index is None else np.asarray(K_index)
    out = [None] * len(Ks)
    for r in sorted(set(int(rk[K]) for K in Ks)):
        sel = [i for i, K in enumerate(Ks) if rk[K] == r]
        cen = fine_centroids(verts[Ks[sel]], 1 << r)
        if w.field == "channels":
            vals = ChannelField(w.seed).kappa(cen)
        elif w.field == "one":
            vals = np.ones(cen.shape[:-1])
        else:
            raise ValueError(w.field)
        for j, i in enumerate(sel):
            out[i] = vals[j].reshape(-1)
    return out


def kappa_for(w: Workload, K_index: np.ndarray | None = None) -> np.ndarray:
    """kappa array (n_K_selected, N*N) for workload `w` (all K, or the K in `K_index`);
    for a workload with a level per K the concatenated per-K blocks (flat)."""
    if w.r_per_K is not None:
        return np.concatenate(kappa_levels(w, K_index))
    verts = coarse_vertices(w.nx, w.ny)
    Ks = np.arange(w.n_K) if K_index is None else np.asarray(K_index)
    if w.field == "one":
        return np.ones((len(Ks), w.n_fine))
    if w.field == "log_uniform":
        K = Ks.astype(np.uint64)[:, None]
        t = np.arange(w.n_fine, dtype=np.uint64)[None, :]
        return 10.0 ** (-2.0 + 4.0 * uniform01(w.seed, K, t, 0))
    if w.field in ("grf4", "grf6"):
        ff = FourierField(w.seed)
        g = ff.eval_numpy(fine_centroids(verts[Ks], w.N))
        return kappa_from_gaussian(g, 2.0 if w.field == "grf4" else 3.0)
    if w.field == "channels":
        return ChannelField(w.seed).kappa(fine_centroids(verts[Ks], w.N))
    raise ValueError(w.field)


def kappa_for_torch(w: Workload, device):
    """Same field as `kappa_for` for all K, generated with torch on `device` (float64)."""
    import torch
    if w.field in ("one", "log_uniform", "channels"):
        return torch.as_tensor(kappa_for(w), dtype=torch.float64).to(device)
    ff = FourierField(w.seed)
    verts = coarse_vertices(w.nx, w.ny)
    out = torch.empty((w.n_K, w.n_fine), dtype=torch.float64, device=device)
    step = max(1, (1 << 22) // w.n_fine)
    for a in range(0, w.n_K, step):
        xy = torch.as_tensor(fine_centroids(verts[a:a + step], w.N), device=device)
        out[a:a + step] = kappa_from_gaussian(ff.eval_torch(xy), 2.0 if w.field == "grf4" else 3.0)
    return out
