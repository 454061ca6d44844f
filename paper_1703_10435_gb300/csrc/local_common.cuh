// Device helpers shared by the local-problem kernels: the level structure of
// the refined submesh, element matrices and loads, face loads.
//
// Level structure.  The lattice rows of the submesh of K (N = 2^r segments per
// face, degree P, PN = P N) are grouped into levels that couple only with their
// neighbours, so the stiffness matrix is block tridiagonal in levels:
//   P1: level j = lattice row j (j = 0..N);
//   P2: level J = lattice rows 2J and 2J+1 (J = 0..N-1), level N = row 2N.
// Fine row j of triangles (between vertex rows j and j+1) touches levels j and
// j+1 only.  Local DOF 0 (lattice point (0,0)) is pinned to remove the constant
// kernel of the Neumann operator; it is left out of level 0.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "mhm_internal.h"

namespace mhm {

struct LevelGeom {
    int P, N, PN;
    int pin_x = 0, pin_y = 0;   // the pinned lattice point (in level 0 or 1; default DOF 0)
    __device__ __forceinline__ int n_levels() const { return N + 1; }
    __device__ __forceinline__ int level_of_row(int y) const { return P == 1 ? y : (y >> 1); }
    // number of unknowns of level `lev` (pinned DOF excluded)
    __device__ __forceinline__ int size(int lev) const {
        const int pinned = lev == level_of_row(pin_y);
        if (P == 1) return N + 1 - lev - pinned;
        if (lev == N) return 1 - pinned;
        return (2 * N - 2 * lev + 1) + (2 * N - 2 * lev) - pinned;
    }
    // position of lattice point (x, y) inside its level; -1 for the pinned DOF
    __device__ __forceinline__ int pos(int x, int y) const {
        const int sx = (y == pin_y && x > pin_x);   // points after the pin in its row move up one
        if (y == pin_y && x == pin_x) return -1;
        if (P == 1 || (y & 1) == 0) return x - sx;
        // odd row: behind the PN-y+2 points of row y-1 (one fewer when the pin is there)
        return (PN - y + 2) - (pin_y == y - 1) + x - sx;
    }
    // inverse of pos: lattice point of position p in level lev
    __device__ __forceinline__ void point(int lev, int p, int* x, int* y) const {
        if (P == 1) {
            *y = lev;
            *x = p + (lev == pin_y && p >= pin_x);
            return;
        }
        const int y0 = 2 * lev;
        const int len0 = PN - y0 + 1 - (pin_y == y0);
        if (p < len0 || lev == N) {
            *y = y0;
            *x = p + (pin_y == y0 && p >= pin_x);
        } else {
            const int q = p - len0;
            *y = y0 + 1;
            *x = q + (pin_y == y0 + 1 && q >= pin_x);
        }
    }
};

// Element stiffness of a triangle with vertices X0, X1, X2 (element node order
// A, B, C; for P2 then the midpoints of BC, CA, AB) for the Laplacian:
// S[a][b] = int grad phi_a . grad phi_b, with grad_x = J^{-T} grad_ref and
// J = [X1 - X0, X2 - X0].  P2 integrates the quadratic integrand exactly with the
// three edge-midpoint rule of the reference triangle.
__device__ inline void element_stiffness(int P, const double X[3][2], double* S /* nb*nb */) {
    const double j00 = X[1][0] - X[0][0], j10 = X[1][1] - X[0][1];
    const double j01 = X[2][0] - X[0][0], j11 = X[2][1] - X[0][1];
    const double det = j00 * j11 - j01 * j10;
    const double adet = fabs(det);
    // G = J^{-1} J^{-T}; J^{-1} = [[j11, -j01], [-j10, j00]] / det
    const double i00 = j11 / det, i01 = -j01 / det, i10 = -j10 / det, i11 = j00 / det;
    const double g00 = i00 * i00 + i01 * i01, g01 = i00 * i10 + i01 * i11, g11 = i10 * i10 + i11 * i11;
    if (P == 1) {
        const double gx[3] = {-1.0, 1.0, 0.0}, gy[3] = {-1.0, 0.0, 1.0};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                S[a * 3 + b] = 0.5 * adet * (gx[a] * (g00 * gx[b] + g01 * gy[b]) + gy[a] * (g01 * gx[b] + g11 * gy[b]));
        return;
    }
    for (int k = 0; k < 36; ++k) S[k] = 0.0;
    const double qx[3] = {0.5, 0.5, 0.0}, qy[3] = {0.0, 0.5, 0.5};
    for (int q = 0; q < 3; ++q) {
        const double l1 = qx[q], l2 = qy[q], l0 = 1.0 - l1 - l2;
        double gx[6], gy[6];
        gx[0] = -(4 * l0 - 1); gy[0] = -(4 * l0 - 1);
        gx[1] = 4 * l1 - 1;    gy[1] = 0.0;
        gx[2] = 0.0;           gy[2] = 4 * l2 - 1;
        gx[3] = 4 * l2;        gy[3] = 4 * l1;
        gx[4] = -4 * l2;       gy[4] = 4 * (l0 - l2);
        gx[5] = 4 * (l0 - l1); gy[5] = -4 * l1;
        for (int a = 0; a < 6; ++a)
            for (int b = 0; b < 6; ++b)
                S[a * 6 + b] += (adet / 6.0) * (gx[a] * (g00 * gx[b] + g01 * gy[b]) + gy[a] * (g01 * gx[b] + g11 * gy[b]));
    }
}

// Lattice coordinates (P-lattice) of the element nodes of fine triangle
// (type up/down, column i, fine row j).
__device__ __forceinline__ void element_nodes(int P, bool up, int i, int j, int nx[6], int ny[6]) {
    int ax, ay, bx, by, cx, cy;
    if (up) { ax = i; ay = j; bx = i + 1; by = j; cx = i; cy = j + 1; }
    else    { ax = i + 1; ay = j; bx = i + 1; by = j + 1; cx = i; cy = j + 1; }
    nx[0] = P * ax; ny[0] = P * ay;
    nx[1] = P * bx; ny[1] = P * by;
    nx[2] = P * cx; ny[2] = P * cy;
    if (P == 2) {
        nx[3] = bx + cx; ny[3] = by + cy;
        nx[4] = cx + ax; ny[4] = cy + ay;
        nx[5] = ax + bx; ny[5] = ay + by;
    }
}

// The pinned DOF of a local problem (Sec. 2: the local solutions are fixed up to a
// constant; one DOF is set to zero, then the mean is removed): a lattice point of
// levels 0 and 1 (level 0 alone when N = 1) on a fine triangle of largest kappa among
// the triangles of fine rows 0 and 1, the first such point in DOF order; DOF 0 when kappa
// is uniform there.  Pinning inside a stiff region keeps the pinned solution free of a
// large constant offset on it; the face integrals would otherwise cancel that offset
// in rounding (relative errors up to 1e5 times larger on high-contrast elements).
// kap: the element's kappa in fine-triangle order (row j: up i = 0..N-j-1, down
// i = 0..N-j-2).  Called by one thread.
__device__ inline void choose_pin(int P, int N, const double* kap, int* pin_x, int* pin_y) {
    const int PN = P * N;
    const int ymax = N == 1 ? (P == 1 ? 0 : 1) : (P == 1 ? 1 : 3);   // lattice rows of the candidate levels
    const int jmax = N == 1 ? 1 : 2;                                  // fine rows touching them
    double best = -1.0;
    for (int j = 0; j < jmax; ++j) {
        const int rs = j * (2 * N - j);
        for (int t = 0; t < 2 * (N - j) - 1; ++t) best = fmax(best, kap[rs + t]);
    }
    int bd = 1 << 30, bx = 0, by = 0;
    for (int j = 0; j < jmax; ++j) {
        const int rs = j * (2 * N - j);
        for (int t = 0; t < 2 * (N - j) - 1; ++t) {
            if (kap[rs + t] != best) continue;
            const bool up = t < N - j;
            int nx[6], ny[6];
            element_nodes(P, up, up ? t : t - (N - j), j, nx, ny);
            for (int a = 0; a < (P == 1 ? 3 : 6); ++a) {
                const int x = nx[a], y = ny[a];
                if (y > ymax) continue;
                const int d = y * (PN + 1) - y * (y - 1) / 2 + x;
                if (d < bd) { bd = d; bx = x; by = y; }
            }
        }
    }
    *pin_x = bx;
    *pin_y = by;
}

// Degree + 1 of local face a of K (Lambda_H^{m,l} with a degree per face, Sec. 2).
__device__ __forceinline__ int face_la1(const DeviceMesh& dm, int64_t K, int a) {
    return dm.lface ? dm.lface[3 * K + a] + 1 : dm.lmax1;
}

// Row of the face-load table (rows q lmax1 + p, built for the largest degree) of local
// slot jf = q la1 + p of a face of degree la1 - 1; -1 for the unused slots jf >= m la1
// of a face below the largest degree (no load: zero rows and columns in A_K).
__device__ __forceinline__ int face_row(int jf, int la1, int fm, int lmax1) {
    if (la1 == lmax1) return jf;
    if (jf >= fm * la1) return -1;
    const int q = jf / la1;
    return q * lmax1 + (jf - q * la1);
}

// int_T phi_a / |T|: P1 1/3 at every vertex; P2 0 at vertices, 1/3 at midpoints.
__device__ __forceinline__ double element_mass_frac(int P, int a) {
    return (P == 1 || a >= 3) ? (1.0 / 3.0) : 0.0;
}

__device__ __forceinline__ double source_value(int kind, double value, double freq, double x, double y) {
    if (kind == MHM_SRC_CONST) return value;
    const double c = 2.0 * (freq * M_PI) * (freq * M_PI) * value;
    return c * sinpi(freq * x) * sinpi(freq * y);
}

// f at point k = 4 i + j of the collapsed 4 x 4 Gauss rule of a fine triangle: the caller's
// value there (MHM_SRC_QUAD; fq holds the triangle's 16 values), else the analytic source.
__device__ __forceinline__ double source_at(int kind, double value, double freq, double x, double y,
                                            const double* fq, int k) {
    if (kind == MHM_SRC_QUAD) return fq[k];
    return source_value(kind, value, freq, x, y);
}

// The 16 point values of f on fine triangle (up, i, j) of the element whose kappa starts at
// kap (the values array is laid out like kappa with 16 values per fine triangle), or NULL
// when f is not given by values.
__device__ __forceinline__ const double* quad_of(const double* vals, const double* kappa, const double* kap, int N,
                                                 bool up, int i, int j) {
    if (!vals) return nullptr;
    return vals + 16 * ((kap - kappa) + (int64_t)j * (2 * N - j) + (up ? i : (N - j) + i));
}

// Faces of lattice point (x, y): bit a set if it lies on local face a
// (face 2: y = 0, face 0: x + y = PN, face 1: x = 0), with the face-local
// position k_loc along the face (from vertex a+1 towards vertex a+2).
__device__ __forceinline__ int face_position(int PN, int x, int y, int a) {
    if (a == 2) return y == 0 ? x : -1;
    if (a == 0) return (x + y == PN) ? y : -1;
    return x == 0 ? PN - y : -1;
}

}  // namespace mhm

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA, non-tensor) global -> shared with an mbarrier.
// Addresses and sizes must be multiples of 16 bytes.
namespace mhm {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// The same copy with an L2 eviction-priority policy (a createpolicy value).
__device__ __forceinline__ void bulk_copy_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                                   uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// Asynchronous prefetch of [src, src + bytes) into L2 (16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// L2 policies: keep the lines (evict last) or let them go first (evict first).
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of `bar` with an iteration limit; returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (int it = 0; it < (1 << 24); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Orders this thread's earlier generic-proxy global writes before later async-proxy reads.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace mhm

// ---------------------------------------------------------------------------
// Blocked right-looking Cholesky of the b pivots of a level window.
namespace mhm {

template <typename T> __device__ __forceinline__ T rsqrt_t(T d);
template <> __device__ __forceinline__ float rsqrt_t<float>(float d) { return rsqrtf(d); }
// FP64: two Newton-Raphson steps y <- y (3 - d y^2) / 2 from the FP32 estimate
// (each step doubles the correct bits), a handful of FP64 operations instead of
// a correctly rounded sqrt and division; plain expression outside FP32 range.
template <> __device__ __forceinline__ double rsqrt_t<double>(double d) {
    if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
    double y = (double)rsqrtf((float)d);
    double t = d * y;
    y = y * fma(-0.5 * t, y, 1.5);
    t = d * y;
    y = y * fma(-0.5 * t, y, 1.5);
    return y;
}

// Loads the NB panel entries row[p0 .. p0+NB) (16-byte aligned) into registers.
template <int NB> __device__ __forceinline__ void load_panel(const float* row, float (&v)[NB]) {
#pragma unroll
    for (int q = 0; q < NB; q += 4) {
        const float4 t = *reinterpret_cast<const float4*>(row + q);
        v[q] = t.x; v[q + 1] = t.y; v[q + 2] = t.z; v[q + 3] = t.w;
    }
}
template <int NB> __device__ __forceinline__ void load_panel(const double* row, double (&v)[NB]) {
#pragma unroll
    for (int q = 0; q < NB; q += 2) {
        const double2 t = *reinterpret_cast<const double2*>(row + q);
        v[q] = t.x; v[q + 1] = t.y;
    }
}

// M (row-major, leading dimension ld, lower triangle used) holds the window rows
// [0, nr): the b pivots of the current level first, then the next level.  Rhs
// (row-major, ldr) holds ncols right-hand-side columns for rows [0, rhs_rows).
// On return: rows [0, b) x cols [0, b) of M hold L (diagonal sqrt of the
// pivots), rows [b, nr) x cols [0, b) hold L_{next,cur}, rows/cols [b, nr) the
// Schur complement; Rhs rows [0, b) hold L^{-1} Rhs and rows [b, rhs_rows) are
// reduced by -L_{next,cur} (L^{-1} Rhs).  Panels of NB pivots are factored by
// warp 0 (warp-synchronous), then all threads apply the rank-NB update.
// ld and ldr must keep every row 16-byte aligned; nr <= 32 RPL and
// ncols <= 32 CPL; *bad gets the first non-positive pivot (+1).  Ends with a
// block barrier.
template <typename T, int NB, int RPL, int CPL>
__device__ void blocked_cholesky_level(T* M, int ld, int b, int nr, T* Rhs, int ldr, int rhs_rows, int ncols,
                                       int* bad) {
    using T_ = T;
    for (int p0 = 0; p0 < b; p0 += NB) {
        const int pe = min(p0 + NB, b);
        if (threadIdx.x < 32) {
            // Panel in registers: lane owns rows i = lane + 32 s of the panel columns and
            // columns c = lane + 32 s of the panel's right-hand-side rows.
            const int lane = threadIdx.x;
            const int nbk = pe - p0;
            T pr[RPL][NB];   // pr[s][q] = M[lane + 32 s][p0 + q]
            T rh[NB][CPL];   // rh[q][s] = Rhs[p0 + q][lane + 32 s]
#pragma unroll
            for (int s2 = 0; s2 < RPL; ++s2) {
                const int i = lane + 32 * s2;
#pragma unroll
                for (int q = 0; q < NB; ++q) pr[s2][q] = (i < nr && q < nbk && i >= p0 + q) ? M[i * ld + p0 + q] : T(0);
            }
#pragma unroll
            for (int q = 0; q < NB; ++q)
#pragma unroll
                for (int s2 = 0; s2 < CPL; ++s2) {
                    const int cidx = lane + 32 * s2;
                    rh[q][s2] = (q < nbk && cidx < ncols) ? Rhs[(p0 + q) * ldr + cidx] : T(0);
                }
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                if (q < nbk) {
                    const int k = p0 + q;
                    // pivot value from the lane owning row k
                    T srcv = pr[0][q];
#pragma unroll
                    for (int s2 = 1; s2 < RPL; ++s2)
                        if (s2 == (k >> 5)) srcv = pr[s2][q];
                    const T d = __shfl_sync(0xffffffffu, srcv, k & 31);
                    const T inv = rsqrt_t<T>(d);
                    if (lane == 0 && !(d > T(0)) && *bad == 0) *bad = k + 1;
                    // scale column q below the pivot; the diagonal becomes sqrt(d)
#pragma unroll
                    for (int s2 = 0; s2 < RPL; ++s2) {
                        const int i = lane + 32 * s2;
                        if (i > k) pr[s2][q] *= inv;
                        else if (i == k) pr[s2][q] = d * inv;
                    }
#pragma unroll
                    for (int s2 = 0; s2 < CPL; ++s2) rh[q][s2] *= inv;
                    // rank-1 update of the remaining panel columns and panel right-hand-side rows
#pragma unroll
                    for (int q2 = 0; q2 < NB; ++q2) {
                        if (q2 > q && q2 < nbk) {
                            const int j = p0 + q2;
                            T srcl = pr[0][q];
#pragma unroll
                            for (int s2 = 1; s2 < RPL; ++s2)
                                if (s2 == (j >> 5)) srcl = pr[s2][q];
                            const T ljk = __shfl_sync(0xffffffffu, srcl, j & 31);
#pragma unroll
                            for (int s2 = 0; s2 < RPL; ++s2) {
                                const int i = lane + 32 * s2;
                                if (i >= j) pr[s2][q2] -= pr[s2][q] * ljk;
                            }
#pragma unroll
                            for (int s2 = 0; s2 < CPL; ++s2) rh[q2][s2] -= ljk * rh[q][s2];
                        }
                    }
                }
            }
#pragma unroll
            for (int s2 = 0; s2 < RPL; ++s2) {
                const int i = lane + 32 * s2;
#pragma unroll
                for (int q = 0; q < NB; ++q)
                    if (i < nr && q < nbk && i >= p0 + q) M[i * ld + p0 + q] = pr[s2][q];
            }
#pragma unroll
            for (int q = 0; q < NB; ++q)
#pragma unroll
                for (int s2 = 0; s2 < CPL; ++s2) {
                    const int cidx = lane + 32 * s2;
                    if (q < nbk && cidx < ncols) Rhs[(p0 + q) * ldr + cidx] = rh[q][s2];
                }
        }
        __syncthreads();
        const int nbk = pe - p0;
        // symmetric part: rows/cols [pe, nr), folded row pairs (pe+m-1-p, pe+p)
        const int m = nr - pe;
        if (m > 0) {
            const int H = (m + 1) / 2, Wd = m + 1, total = H * Wd;
#pragma unroll 2
            for (int e = threadIdx.x; e < total; e += blockDim.x) {
                const int p = e / Wd, cc = e - p * Wd;
                const bool second = cc >= m - p;
                const int i = pe + (second ? p : m - 1 - p);
                const int j = pe + (second ? cc - (m - p) : cc);
                if (second && m - 1 - p == p) continue;
                T acc = M[i * ld + j];
                if (nbk == NB) {
                    T li[NB], lj[NB];
                    load_panel<NB>(M + i * ld + p0, li);
                    load_panel<NB>(M + j * ld + p0, lj);
#pragma unroll
                    for (int q = 0; q < NB; ++q) acc -= li[q] * lj[q];
                } else {
                    for (int q = 0; q < nbk; ++q) acc -= M[i * ld + p0 + q] * M[j * ld + p0 + q];
                }
                M[i * ld + j] = acc;
            }
        }
        // right-hand sides: rows [pe, rhs_rows)
        const int rr = rhs_rows - pe;
        if (rr > 0) {
#pragma unroll 2
            for (int e = threadIdx.x; e < rr * ncols; e += blockDim.x) {
                const int i = pe + e / ncols, c = e - (e / ncols) * ncols;
                T acc = Rhs[i * ldr + c];
                if (nbk == NB) {
                    T li[NB];
                    load_panel<NB>(M + i * ld + p0, li);
#pragma unroll
                    for (int q = 0; q < NB; ++q) acc -= li[q] * Rhs[(p0 + q) * ldr + c];
                } else {
                    for (int q = 0; q < nbk; ++q) acc -= M[i * ld + p0 + q] * Rhs[(p0 + q) * ldr + c];
                }
                Rhs[i * ldr + c] = acc;
            }
        }
        __syncthreads();
    }
}

// The same factorisation for a window held in global memory (one too large for
// shared memory).  Each panel of NB pivots is copied to shared memory (Ps: window
// rows [p0, nr) x NB columns, 16-byte aligned; Rs: NB x ncols; invd: NB), its
// NB x NB diagonal block is factored there by warp 0 together with the panel's
// right-hand-side rows, the rows below it are solved against that block row by
// row, the panel goes back to M and Rhs, and the trailing window is updated from
// the shared copy: every trailing entry is read and written once per panel.  Panel
// rows are wide_panel_stride(NB) doubles apart (NB + 2: consecutive rows start four
// banks apart, so the 16-byte loads of 8 rows cover all 32 banks).  gram
// (ncols x ncols, upper triangle; NULL: none) accumulates (L^{-1} Rhs)^T
// (L^{-1} Rhs) over the b pivot rows.  Same results and contract as
// blocked_cholesky_level (up to rounding order); no alignment asked of M or Rhs.
// Ends with a block barrier.
template <int NB>
__host__ __device__ constexpr int wide_panel_stride() { return NB + 2; }

template <int NB>
__device__ void wide_cholesky_level(double* M, int ld, int b, int nr, double* Rhs, int ldr, int rhs_rows, int ncols,
                                    int* bad, double* Ps, double* Rs, double* invd, double* gram) {
    constexpr int PS = wide_panel_stride<NB>();
    for (int p0 = 0; p0 < b; p0 += NB) {
        const int nbk = min(NB, b - p0), pe = p0 + nbk, np = nr - p0;
        for (int t = threadIdx.x; t < np * NB; t += blockDim.x) {
            const int i = t / NB, q = t - i * NB;
            Ps[i * PS + q] = (q < nbk && i >= q) ? M[(size_t)(p0 + i) * ld + p0 + q] : 0.0;
        }
        for (int t = threadIdx.x; t < NB * ncols; t += blockDim.x) {   // rows past nbk: zero
            const int q = t / ncols, cc = t - q * ncols;
            Rs[t] = q < nbk ? Rhs[(size_t)(p0 + q) * ldr + cc] : 0.0;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            // diagonal block (lane = row) and the panel's right-hand-side rows (lane = column)
            const int lane = threadIdx.x;
            for (int q = 0; q < nbk; ++q) {
                const double d = Ps[q * PS + q];
                const double inv = rsqrt_t<double>(d);
                __syncwarp();
                if (lane == 0) {
                    if (!(d > 0.0) && *bad == 0) *bad = p0 + q + 1;
                    Ps[q * PS + q] = d * inv;
                    invd[q] = inv;
                }
                if (lane > q && lane < nbk) Ps[lane * PS + q] *= inv;
                for (int cc = lane; cc < ncols; cc += 32) Rs[q * ncols + cc] *= inv;
                __syncwarp();
                if (lane > q && lane < nbk) {
                    const double liq = Ps[lane * PS + q];
                    for (int j = q + 1; j <= lane; ++j) Ps[lane * PS + j] -= liq * Ps[j * PS + q];
                }
                for (int q2 = q + 1; q2 < nbk; ++q2) {
                    const double l2 = Ps[q2 * PS + q];
                    for (int cc = lane; cc < ncols; cc += 32) Rs[q2 * ncols + cc] -= l2 * Rs[q * ncols + cc];
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // rows below the diagonal block: l_i = (a_i - sum_{k<q} l_ik L_qk) / L_qq, one row per thread
        for (int ii = nbk + threadIdx.x; ii < np; ii += blockDim.x) {
            double l[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q) l[q] = Ps[ii * PS + q];
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                if (q < nbk) {
                    double v = l[q];
#pragma unroll
                    for (int k = 0; k < NB; ++k)
                        if (k < q) v -= l[k] * Ps[q * PS + k];
                    l[q] = v * invd[q];
                }
            }
#pragma unroll
            for (int q = 0; q < NB; ++q) Ps[ii * PS + q] = l[q];
        }
        __syncthreads();
        // panel back to M and Rhs (columns [p0, pe), rows [p0, pe) of Rhs)
        for (int t = threadIdx.x; t < np * nbk; t += blockDim.x) {
            const int i = t / nbk, q = t - i * nbk;
            if (i >= q) M[(size_t)(p0 + i) * ld + p0 + q] = Ps[i * PS + q];
        }
        for (int t = threadIdx.x; t < nbk * ncols; t += blockDim.x) {
            const int q = t / ncols, cc = t - q * ncols;
            Rhs[(size_t)(p0 + q) * ldr + cc] = Rs[t];
        }
        if (gram) {
            for (int t = threadIdx.x; t < ncols * (ncols + 1) / 2; t += blockDim.x) {
                int c1 = 0, c2 = t;   // t-th pair of the upper triangle, row by row
                while (c2 >= ncols - c1) { c2 -= ncols - c1; ++c1; }
                c2 += c1;
                double s = 0.0;
                for (int q = 0; q < nbk; ++q) s += Rs[q * ncols + c1] * Rs[q * ncols + c2];
                gram[c1 * ncols + c2] += s;
            }
        }
        // trailing symmetric part: rows/cols [pe, nr), folded row pairs (pe+m-1-p, pe+p)
        const int m = nr - pe;
        if (m > 0) {
            const int H = (m + 1) / 2, Wd = m + 1, total = H * Wd;
#pragma unroll 2
            for (int e = threadIdx.x; e < total; e += blockDim.x) {
                const int p = e / Wd, cc = e - p * Wd;
                const bool second = cc >= m - p;
                const int i = pe + (second ? p : m - 1 - p);
                const int j = pe + (second ? cc - (m - p) : cc);
                if (second && m - 1 - p == p) continue;
                double li[NB], lj[NB];
                load_panel<NB>(Ps + (size_t)(i - p0) * PS, li);
                load_panel<NB>(Ps + (size_t)(j - p0) * PS, lj);
                double acc = M[(size_t)i * ld + j];
#pragma unroll
                for (int q = 0; q < NB; ++q) acc -= li[q] * lj[q];
                M[(size_t)i * ld + j] = acc;
            }
        }
        // trailing right-hand-side rows [pe, rhs_rows)
        const int rr = rhs_rows - pe;
        for (int e = threadIdx.x; e < rr * ncols; e += blockDim.x) {
            const int i = pe + e / ncols, cc = e - (e / ncols) * ncols;
            double li[NB];
            load_panel<NB>(Ps + (size_t)(i - p0) * PS, li);
            double acc = Rhs[(size_t)i * ldr + cc];
#pragma unroll
            for (int q = 0; q < NB; ++q) acc -= li[q] * Rs[q * ncols + cc];
            Rhs[(size_t)i * ldr + cc] = acc;
        }
        __syncthreads();
    }
}

}  // namespace mhm
