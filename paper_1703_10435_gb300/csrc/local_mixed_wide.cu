// solveLocalProblem in mixed precision for wide P1 levels (Alg. 1; Sec. 3, Eqs. "etaf",
// "etai", "etaf_comb"): submeshes of r = 6 and 7, whose lattice rows (the levels of the
// block-tridiagonal stiffness matrix) hold 64 and 128 unknowns.
//
// What is computed (as on the FP64 path): with A_p the stiffness matrix pinned at one DOF
// (choose_pin) and G = [N~_0 .. N~_{N_I-1}, f~] the compatible right-hand sides, the
// solutions Z = A_p^{-1} G and the local contributions to Eq. "mat_global"
//     A_K = -N~^T Z,  E_K = N~^T z_f,
// taken through the corrected bilinear form X = G^T Z + Z^T Res (Res = G - A_p Z), whose
// error is quadratic in the error of Z.
//
// How.  One thread block per coarse triangle (a persistent grid, one workspace slot per
// block):
//  1. FP64 set-up: the diagonal scaling s = diag(A_p)^{-1/2}, the scaled couplings of
//     every node to its left/right neighbours and to the row below (Ah = S A_p S, FP32),
//     and G, all from kappa and the two element matrices of the fine triangles;
//  2. FP32 level-Schur factor of Ah: S_0 = Ah_00, S_lev = Ah_ll - C_lev T_{lev-1} C_lev^T
//     and T_lev = S_lev^{-1} by the symmetric sweep (Gauss-Jordan) with the rows of S_lev
//     in registers, two threads per row; the inverses go to the slot;
//  3. preconditioned conjugate gradients in FP64 on A_p Z = G, all columns at once, the
//     preconditioner M = S (block LDL^T of Ah)^{-1} S applied in FP32 by a forward and a
//     backward sweep over the levels:
//        forward   v_lev = T_lev (s r_lev - C_lev v_{lev-1})
//        backward  x_lev = v_lev - T_lev C_{lev+1}^T x_{lev+1},   z = s x;
//     products with A_p are taken in FP64 straight from kappa (7-point rows).  A column
//     stops when r^T M r <= tol g^T M g (energy-norm error estimate, as in the
//     refinement of the narrower levels);
//  4. the outputs in FP64.
// Why CG and not the plain refinement of the narrower levels: on the high-contrast
// channel elements of r = 7 the FP32 factor of Ah is accurate to a few per cent only, so
// refinement contracts slowly (up to 9 passes at the working tolerance), while CG with
// the same factor converges in 2 or 3 iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "local_common.cuh"
#include "mixed_wide.h"

namespace mhm {

namespace {

constexpr int kRp = 16;            // padded right-hand-side count of the FP32 level arrays
constexpr int kMaxWideLev = 129;   // levels of r = 7

struct WideArgs {
    DeviceMesh dm;
    const double* kappa;
    int N, dpf, NI, R, nunk;
    int src_kind;
    const double* src_vals;   // MHM_SRC_QUAD: 16 values per fine triangle, laid out like kappa
    double src_value, src_freq;
    uint32_t* sword;          // the mesh's outcome word (mhm_sync_status)
    int word_final;           // 1: a failed status is final (no FP64 re-solve follows)
    int64_t K0, K1;           // launch indices within the level
    int it_max;
    double tol;
    char* ws;
    size_t slot_bytes;
    // slot layout (bytes): FP64 n x R node-major G, X, Res, P, Q; FP32 n x kRp Z, V;
    // FP64 scale (n); FP32 x 4 couplings (n); FP32 level inverses
    size_t off_G, off_X, off_R, off_P, off_Q, off_Z, off_V, off_s, off_cw, off_T;
    double *AK, *EK, *BK, *FK;
    int32_t *status, *iters;
};

struct WCtx {
    double X[3][2];
    double Sup[9], Sdn[9];
    double area, area_fine, flen[3];
    int sgn[3], rev[3], la1[3];
    double cproj[kMaxNI + 1];
    double FK;
    int pin_x, pin_y, bad;
    int u0[kMaxWideLev + 1];     // first unknown of each level
    int toff[kMaxWideLev + 1];   // first float of each level's inverse
    double gamma[kRp], rz[kRp], alpha[kRp], beta[kRp], red[kRp];
    int done[kRp], failed[kRp];
    int all_done, iters;
};

__device__ __forceinline__ int kap_index(int N, bool up, int i, int j) {
    return j * (2 * N - j) + (up ? i : (N - j) + i);
}
__device__ __forceinline__ bool up_ok(int N, int i, int j) { return i >= 0 && j >= 0 && i + j <= N - 1; }
__device__ __forceinline__ bool dn_ok(int N, int i, int j) { return i >= 0 && j >= 0 && i + j <= N - 2; }

// Unknown of lattice point (x, y) (P1: level y), -1 outside the triangle or pinned.
__device__ __forceinline__ int unknown_of(const WCtx& c, const LevelGeom& lg, int x, int y) {
    if (x < 0 || y < 0 || x + y > lg.N) return -1;
    const int p = lg.pos(x, y);
    return p < 0 ? -1 : c.u0[y] + p;
}

// Lattice point of unknown u (binary search over the level offsets).
__device__ __forceinline__ void node_of(const WCtx& c, const LevelGeom& lg, int u, int* x, int* y) {
    int lo = 0, hi = lg.N;   // u0[lo] <= u < u0[hi + 1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (c.u0[mid] <= u) lo = mid;
        else hi = mid - 1;
    }
    lg.point(lo, u - c.u0[lo], x, y);
}

// The P1 stiffness row of node (x, y): weights of the node itself and of its neighbours
// E (x+1, y), W (x-1, y), N (x, y+1), S (x, y-1), SE (x+1, y-1), NW (x-1, y+1), summed
// over the (up to six) fine triangles around it, each kappa_T times its element matrix.
// Up triangle (i, j): vertices (i, j), (i+1, j), (i, j+1); down triangle (i, j):
// (i+1, j), (i+1, j+1), (i, j+1).
enum { kSelf = 0, kE, kW, kN, kS, kSE, kNW };
__device__ __forceinline__ void stiffness_row(const WCtx& c, int N, const double* kap, int x, int y, double w[7]) {
    for (int d = 0; d < 7; ++d) w[d] = 0.0;
    const double* U = c.Sup;
    const double* D = c.Sdn;
    if (up_ok(N, x, y)) {            // node = vertex 0
        const double k = kap[kap_index(N, true, x, y)];
        w[kSelf] += k * U[0]; w[kE] += k * U[1]; w[kN] += k * U[2];
    }
    if (up_ok(N, x - 1, y)) {        // node = vertex 1
        const double k = kap[kap_index(N, true, x - 1, y)];
        w[kSelf] += k * U[4]; w[kW] += k * U[3]; w[kNW] += k * U[5];
    }
    if (up_ok(N, x, y - 1)) {        // node = vertex 2
        const double k = kap[kap_index(N, true, x, y - 1)];
        w[kSelf] += k * U[8]; w[kS] += k * U[6]; w[kSE] += k * U[7];
    }
    if (dn_ok(N, x - 1, y - 1)) {    // node = vertex 1; vertex 0 = (x, y-1), vertex 2 = (x-1, y)
        const double k = kap[kap_index(N, false, x - 1, y - 1)];
        w[kSelf] += k * D[4]; w[kS] += k * D[3]; w[kW] += k * D[5];
    }
    if (dn_ok(N, x - 1, y)) {        // node = vertex 0; vertex 1 = (x, y+1), vertex 2 = (x-1, y+1)
        const double k = kap[kap_index(N, false, x - 1, y)];
        w[kSelf] += k * D[0]; w[kN] += k * D[1]; w[kNW] += k * D[2];
    }
    if (dn_ok(N, x, y - 1)) {        // node = vertex 2; vertex 0 = (x+1, y-1), vertex 1 = (x+1, y)
        const double k = kap[kap_index(N, false, x, y - 1)];
        w[kSelf] += k * D[8]; w[kSE] += k * D[6]; w[kE] += k * D[7];
    }
}

__device__ __forceinline__ void neighbour_unknowns(const WCtx& c, const LevelGeom& lg, int x, int y, int v[7]) {
    v[kSelf] = unknown_of(c, lg, x, y);
    v[kE] = unknown_of(c, lg, x + 1, y);
    v[kW] = unknown_of(c, lg, x - 1, y);
    v[kN] = unknown_of(c, lg, x, y + 1);
    v[kS] = unknown_of(c, lg, x, y - 1);
    v[kSE] = unknown_of(c, lg, x + 1, y - 1);
    v[kNW] = unknown_of(c, lg, x - 1, y + 1);
}

// int_K phi_w for the P1 vertex (x, y): a third of each fine triangle around it.
__device__ __forceinline__ double vertex_mass(int N, int x, int y, double area_fine) {
    const int n = up_ok(N, x, y) + up_ok(N, x - 1, y) + up_ok(N, x, y - 1) + dn_ok(N, x - 1, y - 1) +
                  dn_ok(N, x - 1, y) + dn_ok(N, x, y - 1);
    return n * (area_fine / 3.0);
}

__device__ __forceinline__ void fine_tri_vertices(const WCtx& c, int N, bool up, int i, int j, double X[3][2]) {
    const double e1x = (c.X[1][0] - c.X[0][0]) / N, e1y = (c.X[1][1] - c.X[0][1]) / N;
    const double e2x = (c.X[2][0] - c.X[0][0]) / N, e2y = (c.X[2][1] - c.X[0][1]) / N;
    int a[3][2];
    if (up) { a[0][0] = i; a[0][1] = j; a[1][0] = i + 1; a[1][1] = j; a[2][0] = i; a[2][1] = j + 1; }
    else    { a[0][0] = i + 1; a[0][1] = j; a[1][0] = i + 1; a[1][1] = j + 1; a[2][0] = i; a[2][1] = j + 1; }
    for (int v = 0; v < 3; ++v) {
        X[v][0] = c.X[0][0] + a[v][0] * e1x + a[v][1] * e2x;
        X[v][1] = c.X[0][1] + a[v][0] * e1y + a[v][1] * e2y;
    }
}

// int_T f lambda_a (a = -1: int_T f) over a fine triangle by the collapsed 4 x 4 Gauss rule.
__device__ double tri_source(const WideArgs& g, const double X[3][2], int a, const double* fq) {
    const double* gx = g.dm.gauss_x + 3 * kMaxGauss;
    const double* gw = g.dm.gauss_w + 3 * kMaxGauss;
    const double adet = fabs((X[1][0] - X[0][0]) * (X[2][1] - X[0][1]) - (X[2][0] - X[0][0]) * (X[1][1] - X[0][1]));
    double s = 0.0;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            const double xi = gx[i], eta = gx[j] * (1.0 - gx[i]), w = gw[i] * gw[j] * (1.0 - gx[i]);
            const double x = X[0][0] + xi * (X[1][0] - X[0][0]) + eta * (X[2][0] - X[0][0]);
            const double y = X[0][1] + xi * (X[1][1] - X[0][1]) + eta * (X[2][1] - X[0][1]);
            const double phi = a < 0 ? 1.0 : (a == 0 ? 1.0 - xi - eta : (a == 1 ? xi : eta));
            s += w * adet * source_at(g.src_kind, g.src_value, g.src_freq, x, y, fq, 4 * i + j) * phi;
        }
    return s;
}

// (f, phi_w)_K of a source that is not constant: the cell integrals of the fine triangles
// around vertex (x, y), each with the vertex's own barycentric weight.
__device__ double vertex_source(const WideArgs& g, const WCtx& c, const double* kap, int x, int y) {
    const int N = g.N;
    double s = 0.0;
    double X[3][2];
    auto add = [&](bool up, int i, int j, int a) {
        fine_tri_vertices(c, N, up, i, j, X);
        s += tri_source(g, X, a, quad_of(g.src_vals, g.kappa, kap, N, up, i, j));
    };
    if (up_ok(N, x, y)) add(true, x, y, 0);
    if (up_ok(N, x - 1, y)) add(true, x - 1, y, 1);
    if (up_ok(N, x, y - 1)) add(true, x, y - 1, 2);
    if (dn_ok(N, x - 1, y - 1)) add(false, x - 1, y - 1, 1);
    if (dn_ok(N, x - 1, y)) add(false, x - 1, y, 0);
    if (dn_ok(N, x, y - 1)) add(false, x, y - 1, 2);
    return s;
}

// Sum over the block of up to kRp per-thread column values; out[c] for c < kRp (all
// threads see it after the call).
template <int NT>
__device__ __forceinline__ void block_sum_cols(double (&acc)[kRp], double* red, double* out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int col = 0; col < kRp; ++col) {
        double v = acc[col];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp * kRp + col] = v;
    }
    __syncthreads();
    if (threadIdx.x < kRp) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += red[w * kRp + threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// As block_sum_cols for per-thread sums of 8 columns, column half h = lane & 1 (columns
// 8 h .. 8 h + 7): out[c] for c < kRp.
template <int NT>
__device__ __forceinline__ void block_sum_halves(double (&acc)[8], double* red, double* out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        double v = acc[e];
        for (int o = 16; o > 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane < 2) red[warp * kRp + lane * 8 + e] = v;
    }
    __syncthreads();
    if (threadIdx.x < kRp) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += red[w * kRp + threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// acc[e] = sum_k T[k][i] Gs[k][8 h + e] for row i < b of a level inverse T (b x b,
// row-major, symmetric: column i is read as row entries, coalesced over i).
__device__ __forceinline__ void level_product(const float* Tl, int b, int i, int h, const float* Gs,
                                              float (&acc)[8]) {
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] = 0.0f;
    if (i >= b) return;
    const float* Gc = Gs + h * 8;
    auto step = [&](float t, int k) {
        const float4 g0 = *reinterpret_cast<const float4*>(Gc + k * kRp);
        const float4 g1 = *reinterpret_cast<const float4*>(Gc + k * kRp + 4);
        acc[0] = fmaf(t, g0.x, acc[0]); acc[1] = fmaf(t, g0.y, acc[1]);
        acc[2] = fmaf(t, g0.z, acc[2]); acc[3] = fmaf(t, g0.w, acc[3]);
        acc[4] = fmaf(t, g1.x, acc[4]); acc[5] = fmaf(t, g1.y, acc[5]);
        acc[6] = fmaf(t, g1.z, acc[6]); acc[7] = fmaf(t, g1.w, acc[7]);
    };
    int k = 0;
    for (; k + 8 <= b; k += 8) {
        float t[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) t[q] = Tl[(size_t)(k + q) * b + i];
#pragma unroll
        for (int q = 0; q < 8; ++q) step(t[q], k + q);
    }
    for (; k < b; ++k) step(Tl[(size_t)k * b + i], k);
}

// Shared memory of a block (floats): the previous level's inverse (BMAX rows of BMAX + 1),
// the staged level operand and the previous level's vector (BMAX x kRp each), the pivot
// rows (2 x BMAX), the diagonal of the sweep (BMAX), the pivots (4), the level's couplings
// (BMAX float4) and the reduction scratch (NT / 32 x kRp doubles).
template <int BMAX> struct WideSmem {
    static constexpr int NT = 2 * BMAX, LDT = BMAX + 1;
    static constexpr int Gs = BMAX * LDT;
    static constexpr int Vp = Gs + BMAX * kRp;
    static constexpr int rb = Vp + BMAX * kRp;
    static constexpr int dg = rb + 2 * BMAX;
    static constexpr int dsh = dg + BMAX;
    static constexpr int cws = dsh + 4;
    static constexpr int red = cws + 4 * BMAX;
    static constexpr int floats = red + 2 * (NT / 32) * kRp;
    static_assert(Gs % 4 == 0 && cws % 4 == 0 && red % 2 == 0, "alignment");
};

template <int BMAX>
__global__ void __launch_bounds__(2 * BMAX, BMAX == 128 ? 2 : 4) k_local_mixed_wide(const __grid_constant__ WideArgs g) {
    using SM = WideSmem<BMAX>;
    constexpr int NT = SM::NT, H = BMAX / 2, LDT = SM::LDT;
    extern __shared__ __align__(16) float wsm[];
    float* Tp = wsm;
    float* Gs = wsm + SM::Gs;
    float* Vp = wsm + SM::Vp;
    float* rb = wsm + SM::rb;
    float* dg = wsm + SM::dg;
    float* dsh = wsm + SM::dsh;
    float4* cws = reinterpret_cast<float4*>(wsm + SM::cws);
    double* red = reinterpret_cast<double*>(wsm + SM::red);
    __shared__ WCtx c;
    const int tid = threadIdx.x, i = tid >> 1, h = tid & 1;   // row i of a level, half h
    const int N = g.N, R = g.R, n = g.nunk;
    char* slot = g.ws + (size_t)blockIdx.x * g.slot_bytes;
    double* G = reinterpret_cast<double*>(slot + g.off_G);
    double* X = reinterpret_cast<double*>(slot + g.off_X);
    double* Rv = reinterpret_cast<double*>(slot + g.off_R);
    double* Pv = reinterpret_cast<double*>(slot + g.off_P);
    double* Qv = reinterpret_cast<double*>(slot + g.off_Q);
    float* Zg = reinterpret_cast<float*>(slot + g.off_Z);
    float* Vg = reinterpret_cast<float*>(slot + g.off_V);
    double* sc = reinterpret_cast<double*>(slot + g.off_s);
    float4* cw = reinterpret_cast<float4*>(slot + g.off_cw);
    float* Tg = reinterpret_cast<float*>(slot + g.off_T);

    for (int64_t ki = g.K0 + blockIdx.x; ki < g.K1; ki += gridDim.x) {
        const int64_t K = g.dm.klist ? (int64_t)g.dm.klist[ki] : ki;
        const double* kap = g.kappa + (g.dm.kap_off ? g.dm.kap_off[K] : K * (int64_t)N * N);

        // ---- per-K set-up
        if (tid == 0) {
            for (int v = 0; v < 3; ++v) {
                c.X[v][0] = g.dm.geom[6 * K + 2 * v];
                c.X[v][1] = g.dm.geom[6 * K + 2 * v + 1];
            }
            c.area = 0.5 * fabs((c.X[1][0] - c.X[0][0]) * (c.X[2][1] - c.X[0][1]) -
                                (c.X[2][0] - c.X[0][0]) * (c.X[1][1] - c.X[0][1]));
            c.area_fine = c.area / ((double)N * N);
            for (int a = 0; a < 3; ++a) {
                const double* P0 = c.X[(a + 1) % 3];
                const double* Q0 = c.X[(a + 2) % 3];
                c.flen[a] = sqrt((Q0[0] - P0[0]) * (Q0[0] - P0[0]) + (Q0[1] - P0[1]) * (Q0[1] - P0[1]));
                c.sgn[a] = g.dm.sign[3 * K + a];
                c.rev[a] = g.dm.rev[3 * K + a];
                c.la1[a] = face_la1(g.dm, K, a);
            }
            double Xu[3][2], Xd[3][2];
            fine_tri_vertices(c, N, true, 0, 0, Xu);
            fine_tri_vertices(c, N, false, 0, 0, Xd);
            element_stiffness(1, Xu, c.Sup);
            element_stiffness(1, Xd, c.Sdn);
            choose_pin(1, N, kap, &c.pin_x, &c.pin_y);
            c.bad = 0;
            const LevelGeom lg0{1, N, N, c.pin_x, c.pin_y};
            int u = 0, t = 0;
            for (int lev = 0; lev <= N; ++lev) {
                const int b = lg0.size(lev);
                c.u0[lev] = u;
                c.toff[lev] = t;
                u += b;
                t += b * b;
            }
            c.u0[N + 1] = u;
            c.toff[N + 1] = t;
        }
        __syncthreads();
        if (c.pin_y != 0) {
            // pinned DOF on lattice row 1: level 0 keeps all N + 1 points of row 0, one more
            // than the kernel's rows; left to the FP64 re-solve (zero blocks, MHM_ERR_UNSUPPORTED)
            const int NI = g.NI;
            for (int t = tid; t < NI * NI; t += NT) g.AK[K * NI * NI + t] = 0.0;
            for (int j = tid; j < NI; j += NT) g.EK[K * NI + j] = g.BK[K * NI + j] = 0.0;
            if (tid == 0) {
                g.FK[K] = 0.0;
                g.status[K] = MHM_ERR_UNSUPPORTED;
                if (g.iters) g.iters[K] = 0;
                if (g.sword && g.word_final) atomicOr(g.sword, 1u << MHM_ERR_UNSUPPORTED);
            }
            __syncthreads();
            continue;
        }
        const LevelGeom lg{1, N, N, c.pin_x, c.pin_y};
        // F_K = (f, 1)_K and the projection coefficients (1^T g) / |K| of every right-hand side
        double FK;
        if (g.src_kind == MHM_SRC_CONST) {
            FK = g.src_value * c.area;
        } else {
            double acc[kRp];
#pragma unroll
            for (int col = 0; col < kRp; ++col) acc[col] = 0.0;
            for (int t = tid; t < N * N; t += NT) {
                // fine triangle t in kappa order: row j starts at j (2N - j)
                int j = (int)((double)N - sqrt((double)N * N - (double)t));
                while (j > 0 && j * (2 * N - j) > t) --j;
                while ((j + 1) * (2 * N - j - 1) <= t) ++j;
                const int o = t - j * (2 * N - j);
                const bool up = o < N - j;
                const int ii = up ? o : o - (N - j);
                double Xt[3][2];
                fine_tri_vertices(c, N, up, ii, j, Xt);
                acc[0] += tri_source(g, Xt, -1, quad_of(g.src_vals, g.kappa, kap, N, up, ii, j));
            }
            block_sum_cols<NT>(acc, red, c.red);
            FK = c.red[0];
        }
        for (int col = tid; col <= g.NI; col += NT) {
            if (col == g.NI) {
                c.cproj[col] = FK / c.area;
            } else {
                const int a = col / g.dpf, jf = col - a * g.dpf;
                const int row = face_row(jf, c.la1[a], g.dm.fm, g.dm.lmax1);
                c.cproj[col] = row < 0 ? 0.0 : -c.sgn[a] * c.flen[a] * g.dm.btab_sum[row] / c.area;
            }
        }
        if (tid == 0) c.FK = FK;
        // the scaling s_u = A_uu^{-1/2}
        for (int u = tid; u < n; u += NT) {
            int x, y;
            node_of(c, lg, u, &x, &y);
            double w[7];
            stiffness_row(c, N, kap, x, y, w);
            sc[u] = w[kSelf] > 0.0 ? 1.0 / sqrt(w[kSelf]) : 0.0;
        }
        __syncthreads();
        // scaled couplings (row below, right neighbour, diagonal) and the right-hand sides:
        // face loads -(s psi_j, phi_w)_{dK}, the compatible projection -(1^T g / |K|) m_w,
        // the source load (f, phi_w)_K
        for (int u = tid; u < n; u += NT) {
            int x, y;
            node_of(c, lg, u, &x, &y);
            double w[7];
            stiffness_row(c, N, kap, x, y, w);
            int v[7];
            neighbour_unknowns(c, lg, x, y, v);
            const double su = sc[u];
            float4 q;
            q.x = v[kS] >= 0 ? (float)(su * w[kS] * sc[v[kS]]) : 0.0f;
            q.y = v[kSE] >= 0 ? (float)(su * w[kSE] * sc[v[kSE]]) : 0.0f;
            q.z = v[kE] >= 0 ? (float)(su * w[kE] * sc[v[kE]]) : 0.0f;
            q.w = (float)(su * w[kSelf] * su);
            cw[u] = q;
            const double m = vertex_mass(N, x, y, c.area_fine);
            const double fsrc = g.src_kind == MHM_SRC_CONST ? g.src_value * m : vertex_source(g, c, kap, x, y);
            for (int col = 0; col < R; ++col) {
                double val = -c.cproj[col] * m;
                if (col == g.NI) {
                    val += fsrc;
                } else {
                    const int a = col / g.dpf, jf = col - a * g.dpf;
                    const int kl = face_position(N, x, y, a);
                    const int row = face_row(jf, c.la1[a], g.dm.fm, g.dm.lmax1);
                    if (kl >= 0 && row >= 0) {
                        const int k = c.rev[a] ? N - kl : kl;
                        val += -c.sgn[a] * c.flen[a] * g.dm.btab[row * (N + 1) + k];
                    }
                }
                const size_t e = (size_t)u * R + col;
                G[e] = val;
                Rv[e] = val;
                X[e] = 0.0;
            }
        }
        __syncthreads();

        // ---- FP32 level-Schur factor of Ah, level by level
        // position in level lev - 1 of lattice point (x, lev - 1), -1 for the pinned DOF
        auto prev_pos = [&](int lev, int x) {
            if (lev - 1 != c.pin_y) return x;
            return x == c.pin_x ? -1 : x - (x > c.pin_x);
        };
        for (int lev = 0; lev <= N; ++lev) {
            const int b = lg.size(lev), ub = c.u0[lev];
            for (int p = tid; p < b; p += NT) cws[p] = cw[ub + p];
            __syncthreads();
            // row i of S_lev = Ah_ll - C T_{lev-1} C^T in registers (positions 64 h .. of this half)
            float a[H];
            float dd = 0.0f;
            {
                const bool row_ok = i < b;
                int qi0 = 0, qi1 = 0;
                float ci0 = 0.0f, ci1 = 0.0f, cri = 0.0f;
                if (row_ok) {
                    const float4 cwi = cws[i];
                    cri = cwi.z;
                    if (lev > 0) {
                        const int xi = i + (lev == c.pin_y && i >= c.pin_x);
                        const int q0 = prev_pos(lev, xi), q1 = prev_pos(lev, xi + 1);
                        ci0 = q0 >= 0 ? cwi.x : 0.0f;
                        ci1 = q1 >= 0 ? cwi.y : 0.0f;
                        qi0 = max(q0, 0);
                        qi1 = max(q1, 0);
                    }
                }
#pragma unroll
                for (int jj = 0; jj < H; ++jj) {
                    const int j = h * H + jj;
                    float v = 0.0f;
                    if (row_ok && j < b) {
                        const float4 cwj = cws[j];
                        if (j == i) v = cwj.w;
                        else if (j == i + 1) v = cri;
                        else if (j == i - 1) v = cwj.z;
                        if (lev > 0) {
                            const int xj = j + (lev == c.pin_y && j >= c.pin_x);
                            int qj0 = prev_pos(lev, xj), qj1 = prev_pos(lev, xj + 1);
                            const float cj0 = qj0 >= 0 ? cwj.x : 0.0f, cj1 = qj1 >= 0 ? cwj.y : 0.0f;
                            qj0 = max(qj0, 0);
                            qj1 = max(qj1, 0);
                            const float u0v = fmaf(cj0, Tp[qi0 * LDT + qj0], cj1 * Tp[qi0 * LDT + qj1]);
                            const float u1v = fmaf(cj0, Tp[qi1 * LDT + qj0], cj1 * Tp[qi1 * LDT + qj1]);
                            v -= fmaf(ci0, u0v, ci1 * u1v);
                        }
                    }
                    a[jj] = v;
                    if (j == i) dd = v;
                }
                if (row_ok && h == i / H) dg[i] = dd;
            }
            __syncthreads();
            // symmetric sweep: per pivot k the pivot row (entry k replaced by d - 1) is
            // broadcast and every row takes a_i -= (rb[i] / d) rb; by symmetry rb[i] is
            // the row's own column-k entry.  Ends with a = 2 I - S^{-1}.
            for (int k = 0; k < b; ++k) {
                float* rbk = rb + (k & 1) * BMAX;
                if (i == k) {
                    float4* dst = reinterpret_cast<float4*>(rbk + h * H);
#pragma unroll
                    for (int q = 0; q < H / 4; ++q) dst[q] = make_float4(a[4 * q], a[4 * q + 1], a[4 * q + 2], a[4 * q + 3]);
                    if (h == k / H) {
                        const float d = dg[k];
                        rbk[k] = d - 1.0f;
                        dsh[k & 1] = d;
                    }
                }
                __syncthreads();
                const float d = dsh[k & 1];
                float dinv = 0.0f;
                if (d > 0.0f) dinv = 1.0f / d;
                else if (tid == 0) c.bad = 1;
                const float m = rbk[i];
                const float s = m * dinv;
                const float4* src = reinterpret_cast<const float4*>(rbk + h * H);
#pragma unroll
                for (int q = 0; q < H / 4; ++q) {
                    const float4 r4 = src[q];
                    a[4 * q] = fmaf(-s, r4.x, a[4 * q]);
                    a[4 * q + 1] = fmaf(-s, r4.y, a[4 * q + 1]);
                    a[4 * q + 2] = fmaf(-s, r4.z, a[4 * q + 2]);
                    a[4 * q + 3] = fmaf(-s, r4.w, a[4 * q + 3]);
                }
                if (i < b && h == i / H) dg[i] = fmaf(-s, m, dg[i]);
            }
            __syncthreads();
            if (i < b) {
#pragma unroll
                for (int jj = 0; jj < H; ++jj) {
                    const int j = h * H + jj;
                    if (j < b) Tp[i * LDT + j] = (j == i) ? 2.0f - a[jj] : -a[jj];
                }
            }
            __syncthreads();
            float* Tl = Tg + c.toff[lev];
            for (int r = tid >> 5; r < b; r += NT / 32)
                for (int col = tid & 31; col < b; col += 32) Tl[r * b + col] = Tp[r * LDT + col];
        }
        __syncthreads();

        // ---- preconditioned CG, all columns at once
        // z = M r: forward then backward sweep over the levels; with upd, the update
        // X += alpha P, Res -= alpha Q of the iteration is applied as the residual is staged.
        // Returns r^T z per column in c.red.
        auto apply = [&](bool upd) {
            double racc[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) racc[e] = 0.0;
            for (int lev = 0; lev <= N; ++lev) {
                const int b = lg.size(lev), ub = c.u0[lev];
                for (int t = tid; t < b * kRp; t += NT) {
                    const int p = t >> 4, col = t & (kRp - 1);
                    float gv = 0.0f;
                    if (col < R) {
                        const int u = ub + p;
                        const size_t e = (size_t)u * R + col;
                        double r = Rv[e];
                        if (upd) {
                            const double al = c.alpha[col];
                            if (al != 0.0) {
                                r = fma(-al, Qv[e], r);
                                Rv[e] = r;
                                X[e] = fma(al, Pv[e], X[e]);
                            }
                        }
                        gv = (float)(sc[u] * r);
                        if (lev > 0) {
                            const int x = p + (lev == c.pin_y && p >= c.pin_x);
                            const int q0 = prev_pos(lev, x), q1 = prev_pos(lev, x + 1);
                            const float4 cu = cw[u];
                            if (q0 >= 0) gv = fmaf(-cu.x, Vp[q0 * kRp + col], gv);
                            if (q1 >= 0) gv = fmaf(-cu.y, Vp[q1 * kRp + col], gv);
                        }
                    }
                    Gs[p * kRp + col] = gv;
                }
                __syncthreads();
                float acc[8];
                level_product(Tg + c.toff[lev], b, i, h, Gs, acc);
                if (i < b) {
                    const float4 v0 = make_float4(acc[0], acc[1], acc[2], acc[3]);
                    const float4 v1 = make_float4(acc[4], acc[5], acc[6], acc[7]);
                    float4* vd = reinterpret_cast<float4*>(Vg + (size_t)(ub + i) * kRp + h * 8);
                    vd[0] = v0;
                    vd[1] = v1;
                    float4* vs = reinterpret_cast<float4*>(Vp + i * kRp + h * 8);
                    vs[0] = v0;
                    vs[1] = v1;
                }
                __syncthreads();
            }
            for (int lev = N; lev >= 0; --lev) {
                const int b = lg.size(lev), ub = c.u0[lev];
                for (int t = tid; t < b * kRp; t += NT) {
                    const int p = t >> 4, col = t & (kRp - 1);
                    float hv = 0.0f;
                    if (col < R && lev < N) {
                        // C_{lev+1}^T x_{lev+1}: node (x, lev) is the S neighbour of (x, lev+1)
                        // and the SE neighbour of (x-1, lev+1)
                        const int x = p + (lev == c.pin_y && p >= c.pin_x);
                        const int ua = unknown_of(c, lg, x, lev + 1), ub2 = unknown_of(c, lg, x - 1, lev + 1);
                        const int un = c.u0[lev + 1];
                        if (ua >= 0) hv = fmaf(cw[ua].x, Vp[(ua - un) * kRp + col], hv);
                        if (ub2 >= 0) hv = fmaf(cw[ub2].y, Vp[(ub2 - un) * kRp + col], hv);
                    }
                    Gs[p * kRp + col] = hv;
                }
                __syncthreads();
                float acc[8];
                level_product(Tg + c.toff[lev], b, i, h, Gs, acc);
                if (i < b) {
                    const int u = ub + i;
                    const float4* vv = reinterpret_cast<const float4*>(Vg + (size_t)u * kRp + h * 8);
                    const float4 v0 = vv[0], v1 = vv[1];
                    float xv[8] = {v0.x - acc[0], v0.y - acc[1], v0.z - acc[2], v0.w - acc[3],
                                   v1.x - acc[4], v1.y - acc[5], v1.z - acc[6], v1.w - acc[7]};
                    float4* vs = reinterpret_cast<float4*>(Vp + i * kRp + h * 8);
                    vs[0] = make_float4(xv[0], xv[1], xv[2], xv[3]);
                    vs[1] = make_float4(xv[4], xv[5], xv[6], xv[7]);
                    const double su = sc[u];
                    float zv[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) zv[e] = (float)(su * (double)xv[e]);
                    float4* zd = reinterpret_cast<float4*>(Zg + (size_t)u * kRp + h * 8);
                    zd[0] = make_float4(zv[0], zv[1], zv[2], zv[3]);
                    zd[1] = make_float4(zv[4], zv[5], zv[6], zv[7]);
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int col = h * 8 + e;
                        if (col < R) racc[e] = fma(Rv[(size_t)u * R + col], (double)zv[e], racc[e]);
                    }
                }
                __syncthreads();
            }
            block_sum_halves<NT>(racc, red, c.red);
        };

        apply(false);
        if (tid == 0) {
            int all = 1;
            for (int col = 0; col < kRp; ++col) {
                const double gm = col < R ? c.red[col] : 0.0;
                c.gamma[col] = c.rz[col] = gm;
                c.done[col] = !(gm > 0.0);
                c.failed[col] = 0;
                c.alpha[col] = c.beta[col] = 0.0;
                all &= c.done[col];
            }
            c.all_done = all || c.bad;
            c.iters = 0;
        }
        __syncthreads();
        for (int u = tid; u < n; u += NT)
            for (int col = 0; col < R; ++col) Pv[(size_t)u * R + col] = (double)Zg[(size_t)u * kRp + col];
        __syncthreads();
        while (!c.all_done) {
            // Q = A_p P (FP64 7-point rows), p^T q per column
            {
                double acc[kRp];
#pragma unroll
                for (int col = 0; col < kRp; ++col) acc[col] = 0.0;
                for (int u = tid; u < n; u += NT) {
                    int x, y;
                    node_of(c, lg, u, &x, &y);
                    double w[7];
                    stiffness_row(c, N, kap, x, y, w);
                    int v[7];
                    neighbour_unknowns(c, lg, x, y, v);
#pragma unroll
                    for (int col = 0; col < kRp; ++col) {
                        if (col < R) {
                            double q = 0.0;
#pragma unroll
                            for (int d = 0; d < 7; ++d)
                                if (v[d] >= 0) q = fma(w[d], Pv[(size_t)v[d] * R + col], q);
                            Qv[(size_t)u * R + col] = q;
                            acc[col] = fma(Pv[(size_t)u * R + col], q, acc[col]);
                        }
                    }
                }
                block_sum_cols<NT>(acc, red, c.red);
            }
            if (tid == 0) {
                for (int col = 0; col < R; ++col) {
                    c.alpha[col] = 0.0;
                    if (c.done[col]) continue;
                    const double pq = c.red[col];
                    if (pq > 0.0 && c.rz[col] == c.rz[col]) c.alpha[col] = c.rz[col] / pq;
                    else c.failed[col] = c.done[col] = 1;
                }
            }
            __syncthreads();
            apply(true);
            if (tid == 0) {
                int all = 1;
                ++c.iters;
                for (int col = 0; col < R; ++col) {
                    c.beta[col] = 0.0;
                    if (!c.done[col]) {
                        const double rzn = c.red[col];
                        if (rzn <= g.tol * c.gamma[col]) c.done[col] = 1;
                        else c.beta[col] = rzn / c.rz[col];
                        c.rz[col] = rzn;
                    }
                    all &= c.done[col];
                }
                c.all_done = all || c.iters >= g.it_max;
            }
            __syncthreads();
            if (c.all_done) break;
            for (int u = tid; u < n; u += NT)
                for (int col = 0; col < R; ++col) {
                    if (c.done[col]) continue;
                    const size_t e = (size_t)u * R + col;
                    Pv[e] = fma(c.beta[col], Pv[e], (double)Zg[(size_t)u * kRp + col]);
                }
            __syncthreads();
        }

        // ---- outputs: X[j][i] = G_j^T z_i + z_j^T Res_i over node chunks in shared memory;
        // A_K = -(X + X^T) / 2, E_K = X[:, f]
        {
            constexpr int CH = BMAX / 2;
            double* cG = reinterpret_cast<double*>(Tp);
            double* cX = cG + CH * kRp;
            double* cR = cX + CH * kRp;
            // pairs (j, i) = tid and tid + NT (R^2 <= 256 <= 2 NT)
            const int t0 = tid < R * R ? tid : 0, t1 = tid + NT < R * R ? tid + NT : 0;
            const int pj0 = t0 / R, pi0 = t0 - pj0 * R, pj1 = t1 / R, pi1 = t1 - pj1 * R;
            double xacc0 = 0.0, xacc1 = 0.0;
            for (int base = 0; base < n; base += CH) {
                const int cnt = min(CH, n - base);
                for (int t = tid; t < CH * kRp; t += NT) {
                    const int uu = t >> 4, col = t & (kRp - 1);
                    const bool ok = uu < cnt && col < R;
                    const size_t e = (size_t)(base + uu) * R + col;
                    cG[t] = ok ? G[e] : 0.0;
                    cX[t] = ok ? X[e] : 0.0;
                    cR[t] = ok ? Rv[e] : 0.0;
                }
                __syncthreads();
                for (int uu = 0; uu < cnt; ++uu) {
                    const double* gr = cG + uu * kRp;
                    const double* xr = cX + uu * kRp;
                    const double* rr = cR + uu * kRp;
                    xacc0 = fma(gr[pj0], xr[pi0], fma(xr[pj0], rr[pi0], xacc0));
                    xacc1 = fma(gr[pj1], xr[pi1], fma(xr[pj1], rr[pi1], xacc1));
                }
                __syncthreads();
            }
            double* xb = cG;   // R x R
            if (tid < R * R) xb[t0] = xacc0;
            if (tid + NT < R * R) xb[t1] = xacc1;
            __syncthreads();
            const int NI = g.NI;
            for (int t = tid; t < NI * NI; t += NT) {
                const int j = t / NI, ii = t - j * NI;
                g.AK[K * NI * NI + t] = -0.5 * (xb[j * R + ii] + xb[ii * R + j]);
            }
            for (int j = tid; j < NI; j += NT) {
                g.EK[K * NI + j] = xb[j * R + NI];
                const int a = j / g.dpf, jf = j - a * g.dpf;
                const int row = face_row(jf, c.la1[a], g.dm.fm, g.dm.lmax1);
                g.BK[K * NI + j] = row < 0 ? 0.0 : c.sgn[a] * c.flen[a] * g.dm.btab_sum[row];
            }
            if (tid == 0) {
                int conv = 1;
                for (int col = 0; col < R; ++col) conv &= c.done[col] && !c.failed[col];
                const int code = c.bad ? MHM_ERR_INVALID_ARG : (conv ? 0 : MHM_ERR_NOT_CONVERGED);
                g.FK[K] = c.FK;
                g.status[K] = code;
                if (g.iters) g.iters[K] = c.iters;
                if (code && g.sword && g.word_final) atomicOr(g.sword, 1u << code);
            }
            __syncthreads();   // the context, the slot and shared memory serve the next element
        }
    }
}

__global__ void k_collect_failed_wide(const int32_t* klist, int64_t i0, int64_t i1, const int32_t* status,
                                      int32_t* list, int32_t* count) {
    for (int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < i1; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t K = klist ? (int64_t)klist[i] : i;
        if (status[K] != MHM_OK) list[atomicAdd(count, 1)] = (int32_t)K;
    }
}

// Slot layout of a level (bytes, each array on a 256-byte boundary) and the launch shape.
struct WideLayout {
    int bmax = 0, threads = 0, R = 0, nunk = 0;
    size_t smem = 0, slot = 0;
    size_t off_G, off_X, off_R, off_P, off_Q, off_Z, off_V, off_s, off_cw, off_T;
};

WideLayout wide_layout(const mhm_mesh* mesh, const Level& lv) {
    WideLayout L;
    const int N = lv.N;
    L.bmax = N == 64 ? 64 : 128;
    L.threads = 2 * L.bmax;
    L.R = (int)mesh->NI + 1;
    L.nunk = (N + 1) * (N + 2) / 2 - 1;
    L.smem = (size_t)(L.bmax == 64 ? WideSmem<64>::floats : WideSmem<128>::floats) * sizeof(float);
    const size_t n = (size_t)L.nunk;
    auto take = [&](size_t bytes) {
        const size_t at = L.slot;
        L.slot += (bytes + 255) & ~(size_t)255;
        return at;
    };
    L.off_G = take(n * L.R * sizeof(double));
    L.off_X = take(n * L.R * sizeof(double));
    L.off_R = take(n * L.R * sizeof(double));
    L.off_P = take(n * L.R * sizeof(double));
    L.off_Q = take(n * L.R * sizeof(double));
    L.off_Z = take(n * kRp * sizeof(float));
    L.off_V = take(n * kRp * sizeof(float));
    L.off_s = take(n * sizeof(double));
    L.off_cw = take(n * 4 * sizeof(float));
    // level inverses: sum of b^2 over the levels, bounded by the unpinned sizes N + 1 - lev
    const size_t tf = (size_t)(N + 1) * (N + 2) * (2 * N + 3) / 6;
    L.off_T = take(tf * sizeof(float));
    return L;
}

int wide_sm_count(const mhm_mesh* mesh) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, mesh->device);
    return sms > 0 ? sms : 1;
}

// Resident blocks per SM of the level's kernel (its registers and shared memory).
int wide_blocks_per_sm(const WideLayout& L) {
    int nb = 0;
    cudaError_t e;
    if (L.bmax == 64) {
        cudaFuncSetAttribute(k_local_mixed_wide<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_local_mixed_wide<64>, L.threads, L.smem);
    } else {
        cudaFuncSetAttribute(k_local_mixed_wide<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_local_mixed_wide<128>, L.threads, L.smem);
    }
    return (e == cudaSuccess && nb > 0) ? nb : 1;
}

// Slots of a level: one per resident block, at most one per element.
int64_t wide_slots(const mhm_mesh* mesh, const Level& lv, const WideLayout& L) {
    const int64_t blocks = (int64_t)wide_blocks_per_sm(L) * wide_sm_count(mesh);
    return std::max<int64_t>(1, std::min<int64_t>(blocks, std::max<int64_t>(lv.nK, 1)));
}

// Workspace of a level: the slots (also the FP64 re-solve's window), then the failed-
// element count (256 bytes) and list (one entry per element of the level).
size_t wide_list_offset(const mhm_mesh* mesh, const Level& lv, const WideLayout& L) {
    const size_t slots = (size_t)wide_slots(mesh, lv, L) * L.slot;
    return (std::max(slots, fp64_level_workspace(mesh, lv)) + 255) & ~(size_t)255;
}

}  // namespace

bool wide_mixed_level(const mhm_mesh* mesh, const Level& lv) {
    return mesh->desc.degree == 1 && (lv.N == 64 || lv.N == 128) && mesh->NI + 1 <= kRp;
}

size_t wide_mixed_workspace(const mhm_mesh* mesh, const Level& lv) {
    if (mesh->device < 0 || !wide_mixed_level(mesh, lv)) return 0;
    const WideLayout L = wide_layout(mesh, lv);
    return wide_list_offset(mesh, lv, L) + 256 + (size_t)std::max<int64_t>(lv.nK, 1) * sizeof(int32_t);
}

mhm_status launch_local_mixed_wide(const mhm_mesh* mesh, const Level& lv, const double* kappa, const mhm_source& f,
                                   const mhm_solve_opts& opts, int64_t K0, int64_t K1, double* AK, double* EK,
                                   double* BK, double* FK, int32_t* status, int32_t* iters, void* ws,
                                   size_t ws_bytes, cudaStream_t stream) {
    if (!wide_mixed_level(mesh, lv))
        return fail(MHM_ERR_UNSUPPORTED, "mhm_local_solve_batch: level not on the wide mixed path");
    const int64_t nblk = K1 - K0;
    if (nblk <= 0) return MHM_OK;
    const WideLayout L = wide_layout(mesh, lv);
    const size_t need = wide_mixed_workspace(mesh, lv);
    if (!ws || ws_bytes < need)
        return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch: workspace smaller than mhm_local_workspace_size");
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0)
        return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch: workspace must be 256-byte aligned");
    WideArgs g;
    g.dm = mesh->dev(lv);
    g.kappa = kappa;
    g.N = lv.N;
    g.dpf = mesh->dpf;
    g.NI = (int)mesh->NI;
    g.R = L.R;
    g.nunk = L.nunk;
    g.src_kind = f.kind;
    g.src_vals = f.kind == MHM_SRC_QUAD ? f.values_dev : nullptr;
    g.src_value = f.value;
    g.src_freq = f.freq;
    g.sword = mesh->d_sword;
    g.word_final = opts.no_fallback != 0;
    g.K0 = K0;
    g.K1 = K1;
    g.it_max = opts.it_max;
    g.tol = opts.tol;
    g.ws = static_cast<char*>(ws);
    g.slot_bytes = L.slot;
    g.off_G = L.off_G; g.off_X = L.off_X; g.off_R = L.off_R; g.off_P = L.off_P; g.off_Q = L.off_Q;
    g.off_Z = L.off_Z; g.off_V = L.off_V; g.off_s = L.off_s; g.off_cw = L.off_cw; g.off_T = L.off_T;
    g.AK = AK; g.EK = EK; g.BK = BK; g.FK = FK;
    g.status = status;
    g.iters = iters;
    const int64_t grid = std::min<int64_t>(wide_slots(mesh, lv, L), nblk);
    timing_mark(mesh, MHM_KERNEL_LOCAL_MIXED, stream, true);
    if (L.bmax == 64) {
        MHM_CUDA_TRY(cudaFuncSetAttribute(k_local_mixed_wide<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem));
        k_local_mixed_wide<64><<<(unsigned)grid, L.threads, L.smem, stream>>>(g);
    } else {
        MHM_CUDA_TRY(cudaFuncSetAttribute(k_local_mixed_wide<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem));
        k_local_mixed_wide<128><<<(unsigned)grid, L.threads, L.smem, stream>>>(g);
    }
    timing_mark(mesh, MHM_KERNEL_LOCAL_MIXED, stream, false);
    MHM_CUDA_TRY(cudaGetLastError());
    if (opts.no_fallback) return MHM_OK;
    // elements whose CG did not converge (or whose FP32 factor met a non-positive pivot):
    // solved again by the FP64 path, its window in the slots' memory
    char* base = static_cast<char*>(ws);
    const size_t lo = wide_list_offset(mesh, lv, L);
    int32_t* fcount = reinterpret_cast<int32_t*>(base + lo);
    int32_t* flist = reinterpret_cast<int32_t*>(base + lo + 256);
    MHM_CUDA_TRY(cudaMemsetAsync(fcount, 0, sizeof(int32_t), stream));
    const int64_t nb = std::min<int64_t>((nblk + 255) / 256, 1024);
    k_collect_failed_wide<<<(unsigned)nb, 256, 0, stream>>>(g.dm.klist, K0, K1, status, flist, fcount);
    MHM_CUDA_TRY(cudaGetLastError());
    return launch_local_fp64_list_ws(mesh, lv, kappa, f, flist, fcount, nblk, AK, EK, BK, FK, status, iters, ws, lo,
                                     stream);
}
}  // namespace mhm
