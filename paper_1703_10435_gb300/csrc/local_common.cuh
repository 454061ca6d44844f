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
    __device__ __forceinline__ int n_levels() const { return N + 1; }
    // number of unknowns of level `lev` (pinned DOF excluded)
    __device__ __forceinline__ int size(int lev) const {
        if (P == 1) return N + 1 - lev - (lev == 0);
        if (lev == N) return 1;
        return (2 * N - 2 * lev + 1) + (2 * N - 2 * lev) - (lev == 0);
    }
    __device__ __forceinline__ int level_of_row(int y) const { return P == 1 ? y : (y >> 1); }
    // position of lattice point (x, y) inside its level; -1 for the pinned DOF
    __device__ __forceinline__ int pos(int x, int y) const {
        if (y == 0) return x - 1;
        if (P == 1 || (y & 1) == 0) return x;
        return (PN - y + 2) - (y == 1) + x;  // row y-1 has PN-y+2 points
    }
    // inverse of pos: lattice point of position p in level lev
    __device__ __forceinline__ void point(int lev, int p, int* x, int* y) const {
        if (P == 1) {
            *y = lev;
            *x = p + (lev == 0);
            return;
        }
        int y0 = 2 * lev;
        int len0 = PN - y0 + 1 - (lev == 0);
        if (p < len0 || lev == N) {
            *y = y0;
            *x = p + (lev == 0);
        } else {
            *y = y0 + 1;
            *x = p - len0;
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

// int_T phi_a / |T|: P1 1/3 at every vertex; P2 0 at vertices, 1/3 at midpoints.
__device__ __forceinline__ double element_mass_frac(int P, int a) {
    return (P == 1 || a >= 3) ? (1.0 / 3.0) : 0.0;
}

__device__ __forceinline__ double source_value(int kind, double value, double freq, double x, double y) {
    if (kind == MHM_SRC_CONST) return value;
    const double c = 2.0 * (freq * M_PI) * (freq * M_PI) * value;
    return c * sinpi(freq * x) * sinpi(freq * y);
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

}  // namespace mhm
