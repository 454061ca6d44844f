// Three-dimensional local problems (the paper's experiment, Sec. 5) on the GPU:
// solveLocalProblem for every coarse tetrahedron (Sec. 3, Eqs. "etaf", "etai") in FP64
// or mixed precision, and the gather of the skeleton system (Eq. "mat_global").
// Conventions in mhm3d.h.
//
// Both local kernels run one block of kThreads threads per coarse element, everything in
// shared memory, with no atomics (every sum in a fixed order: repeated calls are
// bit-identical):
//   1. one element matrix per class of congruent sub-tetrahedra (the Freudenthal
//      refinement has six: its sub-tetrahedra of one permutation class are translates),
//      from the closed forms of the P1 / P2 Lagrange stiffness in barycentric gradients;
//   2. per local DOF, over the sub-tetrahedra that hold it: its row of the pinned lower
//      triangle (local DOF 0 removed), its mass int phi_w and its source load; the
//      multiplier loads -s (psi_j, phi_w) from the face table (a fine face triangle puts
//      a third of its area on each load node);
//   3. the compatibility projection g - (1^T g / |K|) m of every right-hand side;
// then k_local3d (FP64):
//   4. a right-looking Cholesky factorisation of the pinned matrix with the forward
//      substitution of all right-hand sides fused in;
//   5. the face integrals in Gram form, (s psi_j, eta_i)_{dK} = -Y_j . Y_i with Y = L^{-1}
//      times the projected loads (symmetric by construction), and E_K = Y_j . y_f;
// or k_local3d_mixed: an FP32 factor of the diagonally scaled matrix, FP64 refinement
// against the matrix-free residual, and the corrected bilinear form (see the kernel).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "mhm3d_internal.h"

namespace mhm3 {

namespace {

struct Local3DArgs {
    const double* geom;
    const int8_t* signs;
    const int8_t* perm;
    const int32_t* sub_dofs;
    const int8_t* sub_cls;
    const int8_t* sub_base;
    const int32_t* inc_off;   // per local DOF, its slots t nb + a (ascending)
    const int32_t* inc_ent;
    const int32_t* ftab_off;
    const int16_t* ftab_node;
    const int8_t* ftab_cnt;
    const double* quad;
    const double* kappa;
    int src_kind;
    double src_value, src_freq;
    int64_t K0;
    int N, P, n, nb, nsub, m, NI, R;
    double* AK;
    double* EK;
    double* BK;
    double* FK;
    int32_t* status;
    int32_t* iters;       // may be NULL
    int only_failed;      // FP64 kernel: solve only the elements whose status is nonzero (iters -1)
    int it_max;           // mixed kernel: refinement passes
    double tol;           // mixed kernel: scaled residual target per column
    int qs;               // the source's quadrature points of a sub-tetrahedron in qs groups of 64/qs
};

__constant__ int c_perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
__constant__ int c_edges[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

// packed lower triangle, row i >= column j
__device__ __forceinline__ int pk(int i, int j) { return i * (i + 1) / 2 + j; }

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Row of entry t of a packed lower triangle (t = row (row + 1) / 2 + col, col <= row).
__device__ __forceinline__ int tri_row(int t) {
    int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while (r * (r + 1) / 2 > t) --r;
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    return r;
}

// shared-memory layout of the FP64 kernel (doubles), in this order
struct Smem3 {
    int T, Y, mass, S6, G6, J6, red, misc, total;
};

// doubles of the source's partial loads: per group of quadrature points of every
// sub-tetrahedron, its nb loads and its part of F_K
__host__ __device__ inline int partial_loads(int nsub, int nb, int qs) { return qs * nsub * (nb + 1); }

__host__ __device__ inline Smem3 smem_layout(int n, int NI, int nb, int nsub, int qs) {
    const int R = NI + 1, n1 = n - 1, npk = n1 * (n1 + 1) / 2, pl = partial_loads(nsub, nb, qs);
    Smem3 s{};
    int o = 0;
    s.T = o;    o += npk > pl ? npk : pl;           // the source's partial loads, then the pinned factor
    s.Y = o;    o += n * R;                         // right-hand sides, then solutions
    s.mass = o; o += n;
    s.S6 = o;   o += 6 * nb * nb;                   // element matrix per class
    s.G6 = o;   o += 6 * 12;                        // barycentric gradients per class
    s.J6 = o;   o += 6 * 9;                         // edge vectors per class (columns)
    s.red = o;  o += R;
    s.misc = o; o += 16;                            // |K|, |face a| / N^2 (4), V_sub, F_K, pivot flag, done flag
    s.total = o;
    return s;
}

// shared-memory layout of the mixed kernel (doubles; the FP32 factor and solve vectors
// take half a double per value)
struct Smem3M {
    int Lf, G, Z, Rr, W, sc, dg, invf, mass, S6, G6, J6, red, gn, misc, total;
};

__host__ __device__ inline Smem3M smem_layout_mixed(int n, int NI, int nb, int nsub, int qs) {
    const int R = NI + 1, n1 = n - 1, npk = n1 * (n1 + 1) / 2, pl = partial_loads(nsub, nb, qs);
    Smem3M s{};
    int o = 0;
    s.Lf = o;   o += (npk + 1) / 2;                 // FP32 factor of the scaled pinned matrix
    s.G = o;    o += n * R;                         // projected loads g~ (FP64)
    s.Z = o;    o += n * R;                         // solutions (FP64)
    s.Rr = o;   o += n * R > pl ? n * R : pl;       // the source's partial loads, then residuals g~ - A z
    s.W = o;    o += (n1 * R + 1) / 2;              // FP32 preconditioner solves
    s.sc = o;   o += n1;                            // 1 / sqrt(diag) of the pinned matrix
    s.dg = o;   o += n;                             // FP64 diagonal
    s.invf = o; o += (n1 + 1) / 2;                  // FP32 1 / L_kk
    s.mass = o; o += n;
    s.S6 = o;   o += 6 * nb * nb;
    s.G6 = o;   o += 6 * 12;
    s.J6 = o;   o += 6 * 9;
    s.red = o;  o += R;
    s.gn = o;   o += R;                             // |S g~|^2 per column
    s.misc = o; o += 16;
    s.total = o;
    return s;
}

// Geometry of element K into shared memory: misc[0] = |K|, misc[1 + a] = |face a| / N^2,
// misc[5] = |sub-tetrahedron|, misc[6] = F_K accumulator, misc[7] = failure flag,
// misc[8] = done flag; per class c: edge vectors J6[9c + 3 comp + v] and the gradients of
// the four barycentrics G6[12c + 3 l + comp].  No barrier.
__device__ __forceinline__ void element_geometry(const Local3DArgs& g, const double* V, double* misc, double* G6,
                                                 double* J6) {
    const int tid = threadIdx.x, N = g.N;
    if (tid == 0) {
        double e[3][3];
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < 3; ++k) e[k][c] = V[3 * (k + 1) + c] - V[c];
        const double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                           e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                           e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
        misc[0] = fabs(det) / 6.0;
        misc[5] = misc[0] / ((double)N * N * N);
        misc[6] = 0.0;
        misc[7] = 0.0;
        misc[8] = 0.0;
    }
    if (tid < 4) {   // area of local face a over N^2
        int b[3], k = 0;
        for (int v = 0; v < 4; ++v)
            if (v != tid) b[k++] = v;
        double u[3], w[3];
        for (int c = 0; c < 3; ++c) u[c] = V[3 * b[1] + c] - V[3 * b[0] + c], w[c] = V[3 * b[2] + c] - V[3 * b[0] + c];
        const double cx = u[1] * w[2] - u[2] * w[1], cy = u[2] * w[0] - u[0] * w[2], cz = u[0] * w[1] - u[1] * w[0];
        misc[1 + tid] = 0.5 * sqrt(cx * cx + cy * cy + cz * cz) / ((double)N * N);
    }
    if (tid < 6) {   // class tid: edge vectors X_v - X_0 = D p_v / N and barycentric gradients
        double D[3][3];   // columns: v1 - v0, v2 - v1, v3 - v2
        for (int c = 0; c < 3; ++c) {
            D[c][0] = V[3 + c] - V[c];
            D[c][1] = V[6 + c] - V[3 + c];
            D[c][2] = V[9 + c] - V[6 + c];
        }
        int p[3] = {0, 0, 0};
        double J[3][3];   // J[c][v]: component c of edge vector v
        for (int v = 0; v < 3; ++v) {
            p[c_perm[tid][v]] += 1;
            for (int c = 0; c < 3; ++c) J[c][v] = (D[c][0] * p[0] + D[c][1] * p[1] + D[c][2] * p[2]) / N;
        }
        for (int c = 0; c < 3; ++c)
            for (int v = 0; v < 3; ++v) J6[tid * 9 + 3 * c + v] = J[c][v];
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        const double id = 1.0 / det;
        // rows of J^{-1} are the gradients of the barycentrics l1, l2, l3
        double Ji[3][3];
        Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * id;
        Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
        Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
        Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * id;
        Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
        Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
        Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * id;
        Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
        Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
        double* G = G6 + tid * 12;
        for (int c = 0; c < 3; ++c) {
            G[3 + c] = Ji[0][c], G[6 + c] = Ji[1][c], G[9 + c] = Ji[2][c];
            G[c] = -(Ji[0][c] + Ji[1][c] + Ji[2][c]);
        }
    }
}

// Element matrix of each class from the closed forms in the barycentric gradients
// (Vs the common volume of the sub-tetrahedra).  No barrier.
__device__ __forceinline__ void class_matrices(const Local3DArgs& g, double Vs, const double* G6, double* S6) {
    const int nb = g.nb;
    for (int it = threadIdx.x; it < 6 * nb * nb; it += blockDim.x) {
        const int c = it / (nb * nb), a = (it / nb) % nb, b = it % nb;
        const double* G = G6 + c * 12;
        auto d = [&](int i, int j) { return G[3 * i] * G[3 * j] + G[3 * i + 1] * G[3 * j + 1] + G[3 * i + 2] * G[3 * j + 2]; };
        double v;
        if (g.P == 1) {
            v = Vs * d(a, b);
        } else if (a < 4 && b < 4) {
            v = Vs * d(a, b) * (a == b ? 0.6 : -0.2);
        } else if (a < 4 || b < 4) {
            const int x = a < 4 ? a : b, e = (a < 4 ? b : a) - 4;
            const int j = c_edges[e][0], k = c_edges[e][1];
            const double cj = x == j ? 0.15 : -0.05, ck = x == k ? 0.15 : -0.05;
            v = 4.0 * Vs * (d(x, k) * cj + d(x, j) * ck);
        } else {
            const int i = c_edges[a - 4][0], j = c_edges[a - 4][1], k = c_edges[b - 4][0], l = c_edges[b - 4][1];
            v = 0.8 * Vs * (d(j, l) * (1 + (i == k)) + d(j, k) * (1 + (i == l)) + d(i, l) * (1 + (j == k)) +
                            d(i, k) * (1 + (j == l)));
        }
        S6[it] = v;
    }
}

// The source's partial loads (sin sin sin by the collapsed Gauss rule of every
// sub-tetrahedron, its 64 points in qs groups): PL[(t qs + grp) nb + a] and, after the
// qs nsub nb loads, the group's part of F_K.  No barrier.
__device__ __forceinline__ void source_partials(const Local3DArgs& g, const double* V, const double* J6,
                                                const double* misc, double* PL) {
    if (g.src_kind != MHM3D_SRC_SINSINSIN) return;
    const int nb = g.nb, N = g.N, qs = g.qs, per = kQuad / qs;
    const double* qp = g.quad;
    const double* qphi = g.quad + 4 * kQuad;
    const double w6 = 6.0 * misc[5];
    const double kf = g.src_freq * M_PI, amp = g.src_value * 3.0 * kf * kf;
    for (int it = threadIdx.x; it < g.nsub * qs; it += blockDim.x) {
        const int t = it / qs, grp = it % qs;
        const double* Jc = J6 + 9 * g.sub_cls[t];
        const int zA = g.sub_base[3 * t], zB = g.sub_base[3 * t + 1], zC = g.sub_base[3 * t + 2];
        double x0[3];
        for (int c = 0; c < 3; ++c)
            x0[c] = V[c] + ((V[3 + c] - V[c]) * zA + (V[6 + c] - V[3 + c]) * zB + (V[9 + c] - V[6 + c]) * zC) / N;
        double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, fk = 0.0;
        for (int q = grp * per; q < (grp + 1) * per; ++q) {
            double x[3];
            for (int c = 0; c < 3; ++c)
                x[c] = x0[c] + Jc[3 * c] * qp[4 * q] + Jc[3 * c + 1] * qp[4 * q + 1] + Jc[3 * c + 2] * qp[4 * q + 2];
            const double wf = qp[4 * q + 3] * w6 * amp * sin(kf * x[0]) * sin(kf * x[1]) * sin(kf * x[2]);
            fk += wf;
#pragma unroll
            for (int a = 0; a < 10; ++a)
                if (a < nb) acc[a] += wf * qphi[q * nb + a];
        }
#pragma unroll
        for (int a = 0; a < 10; ++a)
            if (a < nb) PL[(size_t)it * nb + a] = acc[a];
        PL[(size_t)g.nsub * qs * nb + it] = fk;
    }
}

// After the partial loads' barrier: per local DOF, in the fixed order of its incidence
// list, the mass int phi_w and the source load (f, phi_w)_K (column N_I of Y, n x R); the
// multiplier loads -s |fine face| / 3 per load node and fine face triangle (columns
// a m + q of Y, zeroed by the caller); F_K into misc[6] (thread 0, in order).  No barrier.
__device__ __forceinline__ void element_loads(const Local3DArgs& g, int64_t K, double* Y, double* mass,
                                              const double* PL, double* misc) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int nb = g.nb, m = g.m, R = g.R, NI = g.NI, qs = g.qs;
    const double Vs = misc[5];
    const bool src = g.src_kind == MHM3D_SRC_SINSINSIN;
    for (int w = tid; w < g.n; w += nthr) {
        double ms = 0.0, ld = 0.0;
        for (int e = g.inc_off[w]; e < g.inc_off[w + 1]; ++e) {
            const int slot = g.inc_ent[e], t = slot / nb, a = slot % nb;
            ms += (g.P == 1 ? 0.25 : (a < 4 ? -0.05 : 0.2)) * Vs;
            if (src)
                for (int grp = 0; grp < qs; ++grp) ld += PL[(size_t)(t * qs + grp) * nb + a];
        }
        mass[w] = ms;
        if (src) Y[w * R + NI] = ld;
    }
    for (int it = tid; it < 4 * m; it += nthr) {
        const int a = it / m, q = it % m;
        const int p = g.perm[4 * K + a];
        const double w = -(double)g.signs[4 * K + a] * misc[1 + a] / 3.0;
        const int base = (a * 6 + p) * (m + 1) + q;
        for (int e = g.ftab_off[base]; e < g.ftab_off[base + 1]; ++e)
            Y[g.ftab_node[e] * R + it] = w * g.ftab_cnt[e];
    }
    if (src && tid == 0) {
        double fk = 0.0;
        for (int i = 0; i < g.nsub * qs; ++i) fk += PL[(size_t)g.nsub * qs * nb + i];
        misc[6] = fk;
    }
}

// Row w of the pinned lower triangle (DOF w >= 1, pinned row w - 1), gathered from the
// element matrices of the sub-tetrahedra at w in the fixed order of its incidence list;
// one thread owns the row (no atomics).  TL: double (FP64 factor) or float (FP32 factor).
template <typename TL>
__device__ __forceinline__ void assemble_row(const Local3DArgs& g, int w, const double* kap, const double* S6,
                                             TL* Lrow, double* diag) {
    const int nb = g.nb;
    for (int j = 0; j < w; ++j) Lrow[j] = (TL)0;
    double dsum = 0.0;
    for (int e = g.inc_off[w]; e < g.inc_off[w + 1]; ++e) {
        const int slot = g.inc_ent[e], t = slot / nb, a = slot % nb;
        const double kt = kap[t];
        const double* Sa = S6 + (g.sub_cls[t] * nb + a) * nb;
        const int32_t* dofs = g.sub_dofs + t * nb;
        for (int b = 0; b < nb; ++b) {
            const int col = dofs[b];
            if (col < 1 || col > w) continue;
            const double v = kt * Sa[b];
            Lrow[col - 1] += (TL)v;
            if (col == w) dsum += v;
        }
    }
    if (diag) *diag = dsum;
}

// After the loads' barrier: a constant source, then the compatibility projection
// g - (1^T g / |K|) m of every column.  Ends with a barrier.
__device__ __forceinline__ void const_source_and_projection(const Local3DArgs& g, double* Y, const double* mass,
                                                            double* red, double* misc) {
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const int n = g.n, R = g.R, NI = g.NI;
    if (g.src_kind == MHM3D_SRC_CONST) {
        for (int w = tid; w < n; w += nthr) Y[w * R + NI] = g.src_value * mass[w];
        if (tid == 0) misc[6] = g.src_value * misc[0];
        __syncthreads();
    }
    const double volK = misc[0];
    for (int r = warp; r < R; r += nwarp) {
        double s = 0.0;
        for (int w = lane; w < n; w += 32) s += Y[w * R + r];
        s = warp_sum(s);
        if (lane == 0) red[r] = s / volK;
    }
    __syncthreads();
    for (int it = tid; it < n * R; it += nthr) Y[it] -= red[it % R] * mass[it / R];
    __syncthreads();
}

// B_K[j] = (s psi_j, 1)_{dK} = s |subface j| from the face-load table, F_K, status.
__device__ __forceinline__ void element_tail(const Local3DArgs& g, int64_t K, const double* misc, int32_t code,
                                            int32_t iters) {
    const int m = g.m, NI = g.NI;
    for (int j = threadIdx.x; j < NI; j += blockDim.x) {
        const int a = j / m, q = j % m;
        const int p = g.perm[4 * K + a];
        const int base = (a * 6 + p) * (m + 1) + q;
        int c = 0;
        for (int e = g.ftab_off[base]; e < g.ftab_off[base + 1]; ++e) c += g.ftab_cnt[e];
        g.BK[K * NI + j] = (double)g.signs[4 * K + a] * misc[1 + a] / 3.0 * c;
    }
    if (threadIdx.x == 0) {
        g.FK[K] = misc[6];
        g.status[K] = code;
        if (g.iters) g.iters[K] = iters;
    }
}

__global__ void __launch_bounds__(kThreads) k_local3d(Local3DArgs g) {
    extern __shared__ double sm[];
    const Smem3 L = smem_layout(g.n, g.NI, g.nb, g.nsub, g.qs);
    double* Lp = sm + L.T;
    double* Y = sm + L.Y;
    double* mass = sm + L.mass;
    double* S6 = sm + L.S6;
    double* G6 = sm + L.G6;
    double* J6 = sm + L.J6;
    double* red = sm + L.red;
    double* misc = sm + L.misc;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int64_t K = g.K0 + blockIdx.x;
    if (g.only_failed && g.status[K] == MHM_OK) return;   // the whole block, before any barrier
    const int n = g.n, n1 = n - 1, R = g.R, NI = g.NI;
    const double* V = g.geom + 12 * K;   // v0..v3
    const double* kap = g.kappa + K * (int64_t)g.nsub;

    // ---- zero the right-hand sides; geometry; class matrices; the source's partial loads
    for (int i = L.Y + tid; i < L.mass; i += nthr) sm[i] = 0.0;
    element_geometry(g, V, misc, G6, J6);
    __syncthreads();
    class_matrices(g, misc[5], G6, S6);
    source_partials(g, V, J6, misc, Lp);
    __syncthreads();
    // ---- loads and mass per DOF, then the pinned lower triangle row by row (pinned DOF 0
    // dropped), over the partial loads once they are summed: no atomics, a fixed order
    element_loads(g, K, Y, mass, Lp, misc);
    __syncthreads();
    for (int w = 1 + tid; w < n; w += nthr) assemble_row<double>(g, w, kap, S6, Lp + pk(w - 1, 0), nullptr);
    const_source_and_projection(g, Y, mass, red, misc);

    // ---- Cholesky of the pinned matrix (rows 1..n-1), forward substitution fused
    for (int k = 0; k < n1; ++k) {
        double d = Lp[pk(k, k)];
        if (!(d > 0.0)) {
            d = 1.0;
            if (tid == 0) misc[7] = 1.0;
        }
        const double inv = 1.0 / sqrt(d);
        for (int i = k + 1 + tid; i < n1; i += nthr) Lp[pk(i, k)] *= inv;
        for (int r = tid; r < R; r += nthr) Y[(k + 1) * R + r] *= inv;
        __syncthreads();
        // trailing update of the triangle below pivot k and of the right-hand sides, as one
        // flat list of items over all threads (every lane busy: the FP64 pipe is the limit)
        const int mt = n1 - k - 1, tri = mt * (mt + 1) / 2, items = tri + mt * R;
        for (int t = tid; t < items; t += nthr) {
            if (t < tri) {
                const int ii = tri_row(t);
                const int i = k + 1 + ii, j = k + 1 + (t - ii * (ii + 1) / 2);
                Lp[pk(i, j)] -= Lp[pk(i, k)] * Lp[pk(j, k)];
            } else {
                const int u = t - tri, i = k + 1 + u / R, r = u % R;
                Y[(i + 1) * R + r] -= Lp[pk(i, k)] * Y[(k + 1) * R + r];
            }
        }
        __syncthreads();
    }
    // ---- face integrals by the Gram form.  With Y = L^{-1} g~ over the pinned rows,
    // (s psi_j, eta_i)_{dK} = -N_j^T eta_i = -N~_j^T z_i = -Y_j . Y_i: the zero-mean shift of
    // eta_i cancels against the compatibility projection of N_j (N~_j^T 1 = 0), and z_i
    // vanishes on the pinned DOF.  Likewise -(s psi_j, eta_f)_{dK} = Y_j . y_f.  No backward
    // substitution is needed.
    double* AK = g.AK + K * (int64_t)NI * NI;
    const int pairs = NI * (NI + 1) / 2;   // each pair i <= j once, then the E_K entries (i = N_I)
    for (int it = tid; it < pairs + NI; it += nthr) {
        const int j = it < pairs ? tri_row(it) : it - pairs, i = it < pairs ? it - j * (j + 1) / 2 : NI;
        double s = 0.0;
        for (int w = 1; w < n; ++w) s += Y[w * R + j] * Y[w * R + i];
        if (i == NI) {
            g.EK[K * NI + j] = s;
        } else {
            AK[j * NI + i] = -s;
            AK[i * NI + j] = -s;
        }
    }
    element_tail(g, K, misc, misc[7] != 0.0 ? MHM_ERR_INVALID_ARG : MHM_OK, g.only_failed ? -1 : 1);
}

// Mixed precision (Sec. 3: the local matrix is factored once and each further solve is
// only products with the factor): the pinned matrix, scaled by its diagonal, is factored
// in FP32 (Cholesky, shared memory); the N_I + 1 solutions are refined in FP64 against
// the matrix-free FP64 residual r = g~ - A z (element matrices of the six classes times
// kappa), each pass one FP32 forward and backward substitution per column (a warp per
// column), until every column's scaled residual |S r| <= tol |S g~| or it_max passes.  The
// face integrals use the corrected bilinear form
//   (s psi_j, eta_i)_{dK} = -(g~_j . z_i + z_j . r_i),
// whose error is the product of the two solution errors in the energy norm (second order),
// averaged with its transpose.  An element whose FP32 factor breaks down or that does not
// converge gets MHM_ERR_NOT_CONVERGED (the host then re-solves it in FP64 unless asked not to).
__global__ void __launch_bounds__(kThreads) k_local3d_mixed(Local3DArgs g) {
    extern __shared__ double sm[];
    const Smem3M L = smem_layout_mixed(g.n, g.NI, g.nb, g.nsub, g.qs);
    float* Lf = reinterpret_cast<float*>(sm + L.Lf);
    double* G = sm + L.G;
    double* Z = sm + L.Z;
    double* Rr = sm + L.Rr;
    float* W = reinterpret_cast<float*>(sm + L.W);
    double* sc = sm + L.sc;
    double* dg = sm + L.dg;
    float* invf = reinterpret_cast<float*>(sm + L.invf);
    double* mass = sm + L.mass;
    double* S6 = sm + L.S6;
    double* G6 = sm + L.G6;
    double* J6 = sm + L.J6;
    double* red = sm + L.red;
    double* gn = sm + L.gn;
    double* misc = sm + L.misc;
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const int64_t K = g.K0 + blockIdx.x;
    const int n = g.n, n1 = n - 1, R = g.R, NI = g.NI, nb = g.nb, npk = n1 * (n1 + 1) / 2;
    const double* V = g.geom + 12 * K;
    const double* kap = g.kappa + K * (int64_t)g.nsub;

    // ---- zero the loads and solutions; geometry; classes; the source's partial loads
    for (int i = L.G + tid; i < L.Rr; i += nthr) sm[i] = 0.0;
    element_geometry(g, V, misc, G6, J6);
    __syncthreads();
    class_matrices(g, misc[5], G6, S6);
    source_partials(g, V, J6, misc, Rr);
    __syncthreads();
    // ---- loads and mass per DOF; the pinned lower triangle in FP32 row by row with its
    // diagonal in FP64 (no atomics, a fixed order)
    element_loads(g, K, G, mass, Rr, misc);
    for (int w = 1 + tid; w < n; w += nthr) assemble_row<float>(g, w, kap, S6, Lf + pk(w - 1, 0), dg + w);
    __syncthreads();
    const_source_and_projection(g, G, mass, red, misc);

    // ---- diagonal scaling S A S (S = diag^-1/2), then the FP32 Cholesky
    for (int i = tid; i < n1; i += nthr) {
        const double d = dg[i + 1];
        if (!(d > 0.0)) misc[7] = 1.0;
        sc[i] = d > 0.0 ? 1.0 / sqrt(d) : 1.0;
    }
    __syncthreads();
    for (int it = tid; it < npk; it += nthr) {
        const int i = tri_row(it), j = it - i * (i + 1) / 2;
        Lf[it] = (float)((double)Lf[it] * sc[i] * sc[j]);
    }
    __syncthreads();
    for (int k = 0; k < n1; ++k) {
        float d = Lf[pk(k, k)];
        if (!(d > 0.0f)) {
            d = 1.0f;
            if (tid == 0) misc[7] = 1.0;
        }
        const float inv = 1.0f / sqrtf(d);
        for (int i = k + 1 + tid; i < n1; i += nthr) Lf[pk(i, k)] *= inv;
        if (tid == 0) invf[k] = inv;
        __syncthreads();
        const int mt = n1 - k - 1, tri = mt * (mt + 1) / 2;   // the trailing triangle, one flat list
        for (int t = tid; t < tri; t += nthr) {
            const int ii = tri_row(t);
            const int i = k + 1 + ii, j = k + 1 + (t - ii * (ii + 1) / 2);
            Lf[pk(i, j)] -= Lf[pk(i, k)] * Lf[pk(j, k)];
        }
        __syncthreads();
    }

    // ---- FP64 refinement: z = 0, r = g~; |S g~|^2 per column
    for (int it = tid; it < n * R; it += nthr) Rr[it] = it < R ? 0.0 : G[it];
    for (int c = warp; c < R; c += nwarp) {
        double s = 0.0;
        for (int i = lane; i < n1; i += 32) s += (sc[i] * G[(i + 1) * R + c]) * (sc[i] * G[(i + 1) * R + c]);
        s = warp_sum(s);
        if (lane == 0) gn[c] = s;
    }
    __syncthreads();
    int passes = 0;
    const double tol2 = g.tol * g.tol;
    for (int pass = 0; pass < g.it_max && misc[7] == 0.0; ++pass) {
        // w = S r (FP32), then L^-1 and L^-T by a warp per column
        for (int it = tid; it < n1 * R; it += nthr) {
            const int i = it / R, c = it % R;
            W[it] = (float)(sc[i] * Rr[(i + 1) * R + c]);
        }
        __syncthreads();
        for (int c = warp; c < R; c += nwarp) {
            for (int k = 0; k < n1; ++k) {
                const float xk = W[k * R + c] * invf[k];
                __syncwarp();
                for (int i = k + 1 + lane; i < n1; i += 32) W[i * R + c] -= Lf[pk(i, k)] * xk;
                if (lane == 0) W[k * R + c] = xk;
                __syncwarp();
            }
            for (int k = n1 - 1; k >= 0; --k) {
                float s = 0.0f;
                for (int i = k + 1 + lane; i < n1; i += 32) s += Lf[pk(i, k)] * W[i * R + c];
                s = warp_sumf(s);
                const float xk = (W[k * R + c] - s) * invf[k];
                __syncwarp();
                if (lane == 0) W[k * R + c] = xk;
                __syncwarp();
            }
        }
        __syncthreads();
        // z += S w; then r = g~ - A z on the pinned rows, gathered per DOF from the element
        // matrices at it (z vanishes on the pinned DOF)
        for (int it = tid; it < n1 * R; it += nthr) {
            const int i = it / R, c = it % R;
            Z[(i + 1) * R + c] += sc[i] * (double)W[it];
        }
        __syncthreads();
        for (int it = tid; it < n1 * R; it += nthr) {
            const int w = it / R + 1, c = it % R;
            double s = 0.0;
            for (int e = g.inc_off[w]; e < g.inc_off[w + 1]; ++e) {
                const int slot = g.inc_ent[e], t = slot / nb, a = slot % nb;
                const double* Sa = S6 + (g.sub_cls[t] * nb + a) * nb;
                const int32_t* dofs = g.sub_dofs + t * nb;
                double sa = 0.0;
                for (int b = 0; b < nb; ++b) sa += Sa[b] * Z[dofs[b] * R + c];
                s += kap[t] * sa;
            }
            Rr[w * R + c] = G[w * R + c] - s;
        }
        __syncthreads();
        // converged when every column's |S r|^2 <= tol^2 |S g~|^2
        for (int c = warp; c < R; c += nwarp) {
            double s = 0.0;
            for (int i = lane; i < n1; i += 32) s += (sc[i] * Rr[(i + 1) * R + c]) * (sc[i] * Rr[(i + 1) * R + c]);
            s = warp_sum(s);
            if (lane == 0) red[c] = s;
        }
        __syncthreads();
        passes = pass + 1;
        bool done = true;
        for (int c = 0; c < R; ++c) done = done && red[c] <= tol2 * gn[c];
        if (done) break;   // the same decision in every thread (read after the barrier)
        __syncthreads();   // red is rewritten in the next pass
    }
    const bool converged = misc[7] == 0.0 && passes > 0 && [&] {
        bool ok = true;
        for (int c = 0; c < R; ++c) ok = ok && red[c] <= tol2 * gn[c];
        return ok;
    }();

    // ---- corrected face integrals T_ji = -(g~_j . z_i + z_j . r_i), averaged with T_ij
    double* AK = g.AK + K * (int64_t)NI * NI;
    const int pairs = NI * (NI + 1) / 2;   // each pair i <= j once, then the E_K entries (i = N_I)
    for (int it = tid; it < pairs + NI; it += nthr) {
        const int j = it < pairs ? tri_row(it) : it - pairs, i = it < pairs ? it - j * (j + 1) / 2 : NI;
        double a1 = 0.0, a2 = 0.0;
        for (int w = 1; w < n; ++w) {
            a1 += G[w * R + j] * Z[w * R + i] + Z[w * R + j] * Rr[w * R + i];
            a2 += G[w * R + i] * Z[w * R + j] + Z[w * R + i] * Rr[w * R + j];
        }
        const double v = 0.5 * (a1 + a2);
        if (i == NI) {
            g.EK[K * NI + j] = v;
        } else {
            AK[j * NI + i] = -v;
            AK[i * NI + j] = -v;
        }
    }
    element_tail(g, K, misc, converged ? MHM_OK : MHM_ERR_NOT_CONVERGED, passes);
}

// skeleton values: one thread per entry of a neighbour block
__global__ void k_skeleton3d_A(const Nbr3* nbrs, int64_t nblocks, const int32_t* rowptr, int m, int NI,
                               const double* AK, double* vals) {
    const int64_t mm = (int64_t)m * m;
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < nblocks * mm;
         it += (int64_t)gridDim.x * blockDim.x) {
        const Nbr3 b = nbrs[it / mm];
        const int q = (int)((it % mm) / m), q2 = (int)(it % m);
        double v = AK[((int64_t)b.K0 * NI + b.a0 * m + q) * NI + b.b0 * m + q2];
        if (b.K1 >= 0) v += AK[((int64_t)b.K1 * NI + b.a1 * m + q) * NI + b.b1 * m + q2];
        vals[rowptr[(int64_t)b.f * m + q] + b.col_off + q2] = v;
    }
}

__global__ void k_skeleton3d_E(const int32_t* face_ka, int64_t nlam, int m, int NI, const double* EK, double* E) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < nlam; l += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = l / m;
        const int q = (int)(l % m);
        const int32_t* k = face_ka + 4 * f;
        double v = EK[(int64_t)k[0] * NI + k[1] * m + q];
        if (k[2] >= 0) v += EK[(int64_t)k[2] * NI + k[3] * m + q];
        E[l] = v;
    }
}

template <typename T>
mhm_status upload3(const std::vector<T>& h, T** d) {
    if (h.empty()) {
        *d = nullptr;
        return MHM_OK;
    }
    cudaError_t e = cudaMalloc((void**)d, h.size() * sizeof(T));
    if (e == cudaErrorMemoryAllocation) return mhm::fail(MHM_ERR_OOM, "cudaMalloc failed for 3-D mesh tables");
    if (e != cudaSuccess) return mhm::cuda_fail(e, "cudaMalloc");
    e = cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return mhm::cuda_fail(e, "cudaMemcpy");
    return MHM_OK;
}

void free_device(mhm_mesh3d* m) {
    void* ptrs[] = {m->d_geom, m->d_signs, m->d_perm, m->d_sub_dofs, m->d_sub_cls, m->d_sub_base, m->d_ftab_off,
                    m->d_ftab_node, m->d_ftab_cnt, m->d_quad, m->d_rowptr, m->d_nbrs, m->d_face_ka, m->d_inc_off,
                    m->d_inc_ent};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

}  // namespace

int local3d_qsplit(int nsub) {
    int qs = 8;   // groups of the 64 points: as many as keep one item per thread
    while (qs > 1 && qs * nsub > kThreads) qs >>= 1;
    return qs;
}
size_t local3d_smem(int n, int NI, int nb, int nsub) {
    return (size_t)smem_layout(n, NI, nb, nsub, local3d_qsplit(nsub)).total * sizeof(double);
}
size_t local3d_smem_mixed(int n, int NI, int nb, int nsub) {
    return (size_t)smem_layout_mixed(n, NI, nb, nsub, local3d_qsplit(nsub)).total * sizeof(double);
}

}  // namespace mhm3

using namespace mhm3;

extern "C" mhm_status mhm3d_create_mesh(const mhm3d_mesh_desc* desc, int32_t device, mhm3d_mesh** out) {
    if (!desc || !out) return mhm::fail(MHM_ERR_INVALID_ARG, "mhm3d_create_mesh: NULL argument");
    *out = nullptr;
    const mhm3d_mesh_desc d = *desc;
    if (d.nc < 1 || d.nc > 64 || d.r < 0 || d.r > 4 || (d.degree != 1 && d.degree != 2))
        return mhm::fail(MHM_ERR_INVALID_ARG, "mhm3d_create_mesh: need 1 <= nc <= 64, 0 <= r <= 4, degree 1 or 2");
    int s = 0;
    while ((1 << (2 * s)) < d.m && s < 8) ++s;
    if (d.m < 1 || (1 << (2 * s)) != d.m || s > d.r)
        return mhm::fail(MHM_ERR_INVALID_ARG, "mhm3d_create_mesh: m must be 4^s with s <= r");
    if (d.degree == 1 && (1 << d.r) < 2 * (1 << s))
        return mhm::fail(MHM_ERR_INVALID_ARG,
                         "mhm3d_create_mesh: degree 1 needs 2^r >= 2 sqrt(m) (the local traces must outnumber "
                         "the multipliers, else A_K is singular)");
    const int PN = d.degree << d.r;
    const int64_t n = (int64_t)(PN + 1) * (PN + 2) * (PN + 3) / 6;
    const int64_t nK = 24LL * d.nc * d.nc * d.nc;
    if (nK * 16LL * d.m * d.m > (1LL << 34))   // A_K alone: n_K N_I^2 doubles
        return mhm::fail(MHM_ERR_INVALID_ARG, "mhm3d_create_mesh: the per-element blocks would exceed 2^34 values");
    if (device >= 0) {
        if (!mhm::device_supported(device))
            return mhm::fail(MHM_ERR_UNSUPPORTED, "mhm3d_create_mesh: device is not an sm_103 GPU");
        if (n > kMaxLocal || d.m > kMaxM ||
            local3d_smem((int)n, 4 * d.m, d.degree == 1 ? 4 : 10, 1 << (3 * d.r)) > 227 * 1024)
            return mhm::fail(MHM_ERR_UNSUPPORTED,
                             "mhm3d_create_mesh: the local factor and right-hand sides exceed shared memory "
                             "(degree 2: r <= 2, degree 1: r <= 3, m <= 16)");
    }
    mhm_mesh3d* m = new mhm_mesh3d();
    m->device = device;
    m->desc = d;
    m->s = s;
    const std::string err = build_mesh3d_host(m);
    if (!err.empty()) {
        delete m;
        return mhm::fail(MHM_ERR_INVALID_ARG, "mhm3d_create_mesh: " + err);
    }
    if (device >= 0) {
        cudaError_t ce = cudaSetDevice(device);
        if (ce != cudaSuccess) {
            delete m;
            return mhm::cuda_fail(ce, "cudaSetDevice");
        }
        mhm_status st = MHM_OK;
        if (!st) st = upload3(m->geom, &m->d_geom);
        if (!st) st = upload3(m->signs, &m->d_signs);
        if (!st) st = upload3(m->perm, &m->d_perm);
        if (!st) st = upload3(m->sub_dofs, &m->d_sub_dofs);
        if (!st) st = upload3(m->sub_cls, &m->d_sub_cls);
        if (!st) st = upload3(m->sub_base, &m->d_sub_base);
        if (!st) st = upload3(m->inc_off, &m->d_inc_off);
        if (!st) st = upload3(m->inc_ent, &m->d_inc_ent);
        if (!st) st = upload3(m->ftab_off, &m->d_ftab_off);
        if (!st) st = upload3(m->ftab_node, &m->d_ftab_node);
        if (!st) st = upload3(m->ftab_cnt, &m->d_ftab_cnt);
        if (!st) st = upload3(m->quad, &m->d_quad);
        if (!st) st = upload3(m->rowptr, &m->d_rowptr);
        if (!st) st = upload3(m->nbrs, &m->d_nbrs);
        if (!st) st = upload3(m->face_ka, &m->d_face_ka);
        if (st) {
            free_device(m);
            delete m;
            return st;
        }
    }
    *out = m;
    return MHM_OK;
}

extern "C" void mhm3d_destroy_mesh(mhm3d_mesh* mesh) {
    if (!mesh) return;
    if (mesh->device >= 0) {
        cudaSetDevice(mesh->device);
        free_device(mesh);
    }
    delete mesh;
}

extern "C" mhm_status mhm3d_mesh_query(const mhm3d_mesh* m, int32_t what, void* host_out, size_t bytes) {
    if (!m || !host_out) return mhm::fail(MHM_ERR_INVALID_ARG, "mhm3d_mesh_query: NULL argument");
    auto copy = [&](const void* src, size_t n) -> mhm_status {
        if (bytes < n) return mhm::fail(MHM_ERR_INVALID_ARG, "mhm3d_mesh_query: output buffer too small");
        if (n) std::memcpy(host_out, src, n);
        return MHM_OK;
    };
    switch (what) {
        case MHM3D_Q_SIZES: {
            const int64_t s[8] = {m->nK, m->nf, m->nv, m->nlam, m->n, m->NI, m->nsub, m->nnz};
            return copy(s, sizeof(s));
        }
        case MHM3D_Q_TETS: return copy(m->tets.data(), m->tets.size() * 4);
        case MHM3D_Q_TET_FACES: return copy(m->tet_faces.data(), m->tet_faces.size() * 4);
        case MHM3D_Q_TET_SIGNS: return copy(m->signs.data(), m->signs.size());
        case MHM3D_Q_FACES: return copy(m->faces.data(), m->faces.size() * 4);
        case MHM3D_Q_VERTICES: return copy(m->verts.data(), m->verts.size() * 8);
        case MHM3D_Q_NORMALS: return copy(m->normals.data(), m->normals.size() * 8);
        case MHM3D_Q_CSR_ROWPTR: return copy(m->rowptr.data(), m->rowptr.size() * 4);
        case MHM3D_Q_CSR_COLS: return copy(m->cols.data(), m->cols.size() * 4);
        case MHM3D_Q_SUB_DOFS: return copy(m->sub_dofs.data(), m->sub_dofs.size() * 4);
        case MHM3D_Q_NODES: return copy(m->nodes.data(), m->nodes.size() * 4);
        case MHM3D_Q_FACE_PERM: return copy(m->perm.data(), m->perm.size());
        case MHM3D_Q_FTAB_OFF: return copy(m->ftab_off.data(), m->ftab_off.size() * 4);
        case MHM3D_Q_FTAB_NODE: return copy(m->ftab_node.data(), m->ftab_node.size() * 2);
        case MHM3D_Q_FTAB_COUNT: return copy(m->ftab_cnt.data(), m->ftab_cnt.size());
        case MHM3D_Q_QUAD: return copy(m->quad.data(), m->quad.size() * 8);
        default: return mhm::fail(MHM_ERR_INVALID_ARG, "mhm3d_mesh_query: unknown query");
    }
}

extern "C" mhm_status mhm3d_local_solve_batch(const mhm3d_mesh* m, const double* kappa, const mhm3d_source* f,
                                              int32_t precision, const mhm3d_opts* opts, int64_t K0, int64_t K1,
                                              double* AK, double* EK, double* BK, double* FK, int32_t* status,
                                              int32_t* iters, void* stream) {
    // every argument is checked before the device: a host-only mesh reports argument errors too
    if (!m) return mhm::fail(MHM_ERR_INVALID_ARG, "mhm3d_local_solve_batch: NULL mesh");
    if (!kappa || !f || !AK || !EK || !BK || !FK || !status)
        return mhm::fail(MHM_ERR_INVALID_ARG, "mhm3d_local_solve_batch: NULL pointer argument");
    if (f->kind != MHM3D_SRC_CONST && f->kind != MHM3D_SRC_SINSINSIN)
        return mhm::fail(MHM_ERR_INVALID_ARG, "mhm3d_local_solve_batch: unknown source kind");
    if (precision != MHM_FP64 && precision != MHM_MIXED)
        return mhm::fail(MHM_ERR_INVALID_ARG, "mhm3d_local_solve_batch: precision must be MHM_FP64 or MHM_MIXED");
    mhm3d_opts o{8, 1e-9, 0};
    if (opts) o = *opts;
    if (o.it_max < 1 || !(o.tol > 0.0))
        return mhm::fail(MHM_ERR_INVALID_ARG, "mhm3d_local_solve_batch: it_max >= 1 and tol > 0 required");
    if (K1 <= 0) K1 = m->nK;
    if (K0 < 0 || K1 > m->nK || K0 > K1) return mhm::fail(MHM_ERR_INVALID_ARG, "mhm3d_local_solve_batch: K range");
    if (m->device < 0) return mhm::fail(MHM_ERR_UNSUPPORTED, "mhm3d_local_solve_batch: host-only mesh");
    if (K1 == K0) return MHM_OK;
    MHM_CUDA_TRY(cudaSetDevice(m->device));
    Local3DArgs g{};
    g.geom = m->d_geom, g.signs = m->d_signs, g.perm = m->d_perm;
    g.sub_dofs = m->d_sub_dofs, g.sub_cls = m->d_sub_cls, g.sub_base = m->d_sub_base;
    g.inc_off = m->d_inc_off, g.inc_ent = m->d_inc_ent;
    g.ftab_off = m->d_ftab_off, g.ftab_node = m->d_ftab_node, g.ftab_cnt = m->d_ftab_cnt;
    g.quad = m->d_quad, g.kappa = kappa;
    g.src_kind = f->kind, g.src_value = f->value, g.src_freq = f->freq;
    g.K0 = K0;
    g.N = m->N, g.P = m->desc.degree, g.n = (int)m->n, g.nb = m->nb, g.nsub = (int)m->nsub, g.m = m->desc.m;
    g.NI = (int)m->NI, g.R = (int)m->NI + 1;
    g.AK = AK, g.EK = EK, g.BK = BK, g.FK = FK, g.status = status, g.iters = iters;
    g.it_max = o.it_max, g.tol = o.tol;
    const unsigned grid = (unsigned)(K1 - K0);
    cudaStream_t s = (cudaStream_t)stream;
    // the shared-memory attribute is per kernel, not per mesh: set it for this mesh every call
    g.qs = local3d_qsplit(g.nsub);
    const size_t smem64 = local3d_smem(g.n, g.NI, g.nb, g.nsub);
    const size_t smemmx = local3d_smem_mixed(g.n, g.NI, g.nb, g.nsub);
    const bool mixed = precision == MHM_MIXED && smemmx <= 227 * 1024;
    if (mixed) {
        MHM_CUDA_TRY(cudaFuncSetAttribute(k_local3d_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemmx));
        k_local3d_mixed<<<grid, kThreads, smemmx, s>>>(g);
        MHM_CUDA_TRY(cudaGetLastError());
        if (o.no_fallback) return MHM_OK;
        g.only_failed = 1;   // the elements the refinement could not finish, again in FP64
    }
    MHM_CUDA_TRY(cudaFuncSetAttribute(k_local3d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64));
    k_local3d<<<grid, kThreads, smem64, s>>>(g);
    MHM_CUDA_TRY(cudaGetLastError());
    return MHM_OK;
}

extern "C" mhm_status mhm3d_assemble_skeleton(const mhm3d_mesh* m, const double* AK, const double* EK,
                                              double* A_vals, double* E, void* stream) {
    if (!m) return mhm::fail(MHM_ERR_INVALID_ARG, "mhm3d_assemble_skeleton: NULL mesh");
    if (!AK || !EK || !A_vals || !E) return mhm::fail(MHM_ERR_INVALID_ARG, "mhm3d_assemble_skeleton: NULL pointer");
    if (m->device < 0) return mhm::fail(MHM_ERR_UNSUPPORTED, "mhm3d_assemble_skeleton: host-only mesh");
    MHM_CUDA_TRY(cudaSetDevice(m->device));
    const int64_t nblocks = (int64_t)m->nbrs.size();
    const int64_t items = nblocks * m->desc.m * m->desc.m;
    const int threads = 256;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
    const int64_t want = (items + threads - 1) / threads;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
    k_skeleton3d_A<<<grid, threads, 0, (cudaStream_t)stream>>>(m->d_nbrs, nblocks, m->d_rowptr, m->desc.m,
                                                               (int)m->NI, AK, A_vals);
    MHM_CUDA_TRY(cudaGetLastError());
    const int64_t want_e = (m->nlam + threads - 1) / threads;
    const unsigned grid_e = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want_e, (int64_t)sms * 8));
    k_skeleton3d_E<<<grid_e, threads, 0, (cudaStream_t)stream>>>(m->d_face_ka, m->nlam, m->desc.m, (int)m->NI, EK, E);
    MHM_CUDA_TRY(cudaGetLastError());
    return MHM_OK;
}
