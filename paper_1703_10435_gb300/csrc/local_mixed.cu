// solveLocalProblem in mixed precision (Alg. 1; Sec. 3, Eqs. "etaf", "etai",
// "etaf_comb"; Sec. 4.2, Eq. "source_term").
//
// Per coarse triangle K (one thread block, persistent over K):
//  1. loads G = [N~_0 .. N~_{N_I-1}, f~] (FP64), the compatible right-hand sides
//     of the Neumann problems pinned at DOF 0 (N_i = -(s psi_i, phi_w)_{dK},
//     f = (f, phi_w)_K, each minus (1^T g / |K|) m with m_w = int_K phi_w);
//  2. factors the pinned stiffness matrix A_p = L L^T in FP32 by the same
//     level-window right-looking Cholesky as the FP64 kernel, writing the blocks
//     L_lev and L_{lev+1,lev} to this block's slot of the scratch workspace;
//  3. refines Z = A_p^{-1} G: each pass solves L L^T D = R in FP32 and adds D to
//     Z in FP64, where R = G - A_p Z is the residual computed in FP64 straight
//     from kappa and the element matrices (no assembled FP64 matrix);
//     a column stops once its estimated error |D_k|^2 / |D_{k-1}| is below
//     tol * |Z|;
//  4. forms the local contributions to Eq. "mat_global" in FP64:
//     A_K[j,i] = -N~_j^T z_i (symmetrised), E_K[j] = N~_j^T z_f, with
//     N~_j^T z = N_j^T z - c_j m^T z (N_j lives on one face only).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "local_common.cuh"

namespace mhm {

namespace {

constexpr int kThreadsM = 256;
constexpr int kWarpsM = kThreadsM / 32;

struct MixedArgs {
    DeviceMesh dm;
    const double* kappa;
    int P, N, PN, dpf, NI, R, nlev, nunk;
    int wrows, wld;               // FP32 window rows and leading dimension
    int wfloats;                  // floats reserved for the window (also holds R x R doubles)
    int yfloats;                  // floats reserved for the right-hand-side block (>= nunk R)
    int bmax;                     // largest level size
    int opmax;                    // floats of the largest level operator (multiple of 4)
    int ldr;                      // leading dimension of the level right-hand sides (multiple of 4)
    int src_kind;
    double src_value, src_freq;
    int64_t K0, K1;
    int it_max;
    double tol;
    char* ws;
    size_t slot_bytes, off_G, off_Z, off_mass, off_scale, off_D;
    size_t off_kap_smem, off_scale_smem;
    int kap_in_smem;
    double *AK, *EK, *BK, *FK;
    int32_t *status, *iters;
};

struct MCtx {
    double X[3][2];
    double Sup[36], Sdn[36];
    double area_fine, area, FK;
    double flen[3];
    int sgn[3], rev[3];
    double cproj[kMaxNI + 1];
    int bad;
    int col_done[kMaxNI + 1];
    double gamma[kMaxNI + 1];     // G_c^T M G_c per column
    double eps[kMaxNI + 1];       // Res_c^T M Res_c per column
    int passes;
    int all_done;
    int converged;
    int col_frozen[kMaxNI + 1];   // no further solves for this column
    double eps_prev[kMaxNI + 1];
    int col_fail;
    double red[kWarpsM];
    double mz[kMaxNI + 1];
    alignas(8) uint64_t bar[2];
    uint32_t phase[2];
    int timeout;
};

__device__ __forceinline__ int lev_size(const LevelGeom& lg, int lev) { return lg.size(lev); }

// Fine-triangle vertices in physical coordinates.
__device__ __forceinline__ void fine_xy(const MCtx& c, int N, bool up, int i, int j, double X[3][2]) {
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

__device__ double cell_src(const MixedArgs& g, const double X[3][2], int P, int a) {
    const double* gx = g.dm.gauss_x + 3 * kMaxGauss;
    const double* gw = g.dm.gauss_w + 3 * kMaxGauss;
    const double adet = fabs((X[1][0] - X[0][0]) * (X[2][1] - X[0][1]) - (X[2][0] - X[0][0]) * (X[1][1] - X[0][1]));
    double s = 0.0;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            const double xi = gx[i], eta = gx[j] * (1.0 - gx[i]), w = gw[i] * gw[j] * (1.0 - gx[i]);
            const double x = X[0][0] + xi * (X[1][0] - X[0][0]) + eta * (X[2][0] - X[0][0]);
            const double y = X[0][1] + xi * (X[1][1] - X[0][1]) + eta * (X[2][1] - X[0][1]);
            double phi = 1.0;
            if (a >= 0) {
                const double l0 = 1.0 - xi - eta, l1 = xi, l2 = eta;
                if (P == 1) phi = a == 0 ? l0 : (a == 1 ? l1 : l2);
                else {
                    const double lam[3] = {l0, l1, l2};
                    if (a < 3) phi = lam[a] * (2.0 * lam[a] - 1.0);
                    else if (a == 3) phi = 4.0 * l1 * l2;
                    else if (a == 4) phi = 4.0 * l2 * l0;
                    else phi = 4.0 * l0 * l1;
                }
            }
            s += w * adet * source_value(g.src_kind, g.src_value, g.src_freq, x, y) * phi;
        }
    return s;
}

// Fine triangles incident to lattice point (X, Y) and the point's local index in
// each: up to 6 for a vertex, 2 for a P2 edge midpoint.  Returns the count.
__device__ int incident(int P, int N, int X, int Y, int ti[6], int tj[6], bool tup[6], int ta[6]) {
    int n = 0;
    auto add = [&](bool up, int i, int j, int a) {
        if (i < 0 || j < 0) return;
        if (up ? (i + j > N - 1) : (i + j > N - 2)) return;
        ti[n] = i; tj[n] = j; tup[n] = up; ta[n] = a; ++n;
    };
    if (P == 1 || ((X & 1) == 0 && (Y & 1) == 0)) {
        const int x = P == 1 ? X : X >> 1, y = P == 1 ? Y : Y >> 1;
        add(true, x, y, 0);
        add(true, x - 1, y, 1);
        add(true, x, y - 1, 2);
        add(false, x - 1, y - 1, 1);
        add(false, x - 1, y, 0);
        add(false, x, y - 1, 2);
    } else if ((X & 1) && !(Y & 1)) {      // horizontal edge (x,y)-(x+1,y)
        const int x = (X - 1) >> 1, y = Y >> 1;
        add(true, x, y, 5);
        add(false, x, y - 1, 3);
    } else if (!(X & 1) && (Y & 1)) {      // vertical edge (x,y)-(x,y+1)
        const int x = X >> 1, y = (Y - 1) >> 1;
        add(true, x, y, 4);
        add(false, x - 1, y, 5);
    } else {                               // diagonal edge (x+1,y)-(x,y+1)
        const int x = (X - 1) >> 1, y = (Y - 1) >> 1;
        add(true, x, y, 3);
        add(false, x, y, 4);
    }
    return n;
}

__device__ __forceinline__ int kap_index(int N, bool up, int i, int j) {
    return j * (2 * N - j) + (up ? i : (N - j) + i);
}

// Unknown index of lattice point (X, Y): lattice DOF - 1 (DOF 0 is pinned -> -1).
__device__ __forceinline__ int unk(int PN, int X, int Y) {
    return Y * (PN + 1) - Y * (Y - 1) / 2 + X - 1;
}

__device__ __forceinline__ void lattice_of_unk(int PN, int u, int* X, int* Y) {
    int d = u + 1, y = 0;
    while (d >= PN + 1 - y) { d -= PN + 1 - y; ++y; }
    *X = d;
    *Y = y;
}

// Res(u, :) -= (A_p D)(u, :) for the columns still refining, in FP64, and the next
// FP32 right-hand side y(u, :) = s_u Res(u, :): the sum over
// the fine triangles T containing u of kappa_T S_T[a_u][b] D(b).  P1 uses the
// assembled 7-point row of the lattice (6 triangles, 7 coefficients); P2 sums
// element by element.
__device__ void apply_residual(const MixedArgs& g, const MCtx& c, const double* kap, int u, const double* D,
                               double* Res, float* y, const double s_u) {
    int X, Y;
    lattice_of_unk(g.PN, u, &X, &Y);
    const size_t ld = (size_t)g.nunk;
    if (g.P == 1) {
        const int N = g.N, x = X, yl = Y;
        auto kup = [&](int i, int j) { return (i >= 0 && j >= 0 && i + j <= N - 1) ? kap[kap_index(N, true, i, j)] : 0.0; };
        auto kdn = [&](int i, int j) { return (i >= 0 && j >= 0 && i + j <= N - 2) ? kap[kap_index(N, false, i, j)] : 0.0; };
        const double k1 = kup(x, yl), k2 = kup(x - 1, yl), k3 = kup(x, yl - 1);
        const double k4 = kdn(x - 1, yl - 1), k5 = kdn(x - 1, yl), k6 = kdn(x, yl - 1);
        const double* Su = c.Sup;
        const double* Sd = c.Sdn;
        double w[7];
        int v[7];
        w[0] = k1 * Su[0] + k2 * Su[4] + k3 * Su[8] + k4 * Sd[4] + k5 * Sd[0] + k6 * Sd[8];  v[0] = u;
        w[1] = k1 * Su[1] + k6 * Sd[7];  v[1] = unk(g.PN, x + 1, yl);        // east
        w[2] = k2 * Su[3] + k4 * Sd[5];  v[2] = unk(g.PN, x - 1, yl);        // west
        w[3] = k1 * Su[2] + k5 * Sd[1];  v[3] = unk(g.PN, x, yl + 1);        // north
        w[4] = k3 * Su[6] + k4 * Sd[3];  v[4] = unk(g.PN, x, yl - 1);        // south
        w[5] = k3 * Su[7] + k6 * Sd[6];  v[5] = unk(g.PN, x + 1, yl - 1);    // south-east
        w[6] = k2 * Su[5] + k5 * Sd[2];  v[6] = unk(g.PN, x - 1, yl + 1);    // north-west
        for (int k = 1; k < 7; ++k)
            if (w[k] == 0.0 || v[k] < 0 || v[k] >= g.nunk) { w[k] = 0.0; v[k] = u; }
        for (int col = 0; col < g.R; ++col) {
            if (c.col_done[col]) continue;
            const double* Dc = D + col * ld;
            double a = 0.0;
#pragma unroll
            for (int k = 0; k < 7; ++k)
                if (w[k] != 0.0) a = fma(w[k], Dc[v[k]], a);   // zero weights: edges at right angles
            const double rn = Res[col * ld + u] - a;
            Res[col * ld + u] = rn;
            y[col * ld + u] = (float)(rn * s_u);
        }
        return;
    }
    int ti[6], tj[6], ta[6];
    bool tup[6];
    const int n = incident(g.P, g.N, X, Y, ti, tj, tup, ta);
    for (int col = 0; col < g.R; ++col) {
        if (c.col_done[col]) continue;
        const double* Dc = D + col * ld;
        double a = 0.0;
        for (int t = 0; t < n; ++t) {
            int nx[6], ny[6];
            element_nodes(2, tup[t], ti[t], tj[t], nx, ny);
            const double kt = kap[kap_index(g.N, tup[t], ti[t], tj[t])];
            const double* S = tup[t] ? c.Sup : c.Sdn;
            for (int b = 0; b < 6; ++b) {
                const int ub = unk(g.PN, nx[b], ny[b]);
                if (ub >= 0) a = fma(kt * S[ta[t] * 6 + b], Dc[ub], a);
            }
        }
        const double rn = Res[col * ld + u] - a;
        Res[col * ld + u] = rn;
        y[col * ld + u] = (float)(rn * s_u);
    }
}

// out[c] = sum_u Res(u, c) s(u) y(u, c) for the columns still refining (warp per
// column, fixed summation order).
__device__ void column_dot(const MixedArgs& g, const double* Res, const float* y, const double* s, double* out,
                           const MCtx& c) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int col = warp; col < g.R; col += kWarpsM) {
        if (c.col_frozen[col]) continue;
        const double* rc = Res + (size_t)col * g.nunk;
        const float* yc = y + (size_t)col * g.nunk;
        float a = 0.0f;   // an error estimate: FP32 is ample
        for (int u = lane; u < g.nunk; u += 32) a = fmaf((float)rc[u] * (float)s[u], yc[u], a);
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) out[col] = (double)a;
    }
}

// Forward + backward solve of L L^T D = Y in FP32 for every column still
// refining, in place in y (column-major, nunk per column).  Level by level,
//   forward   y_lev = Fw_lev [y_lev; y_{lev-1}],  Fw_lev = [L_lev^{-1} | -L_lev^{-1} L_{lev,lev-1}]
//   backward  x_lev = Bw_lev [y_lev; x_{lev+1}],  Bw_lev = [L_lev^{-T} | -L_lev^{-T} L_{lev+1,lev}^T]
// so each step is one small dense product over all columns.  The operators are
// stored column-major ((b + b') x b) and streamed into two shared-memory buffers
// by bulk asynchronous copies: the copy for step s+1 runs while step s computes.
constexpr int kColGroup = 4;     // columns per work item
constexpr int kItemsPerThread = 2;

__device__ void solve_factor(const MixedArgs& g, const LevelGeom& lg, const float* F, const int* opoff,
                             const int* u0, float* y, float* opbuf, float* tbuf, MCtx& c) {
    // One block barrier per level step: each step writes its result into one of two
    // small buffers T (column-major, ld bmax) and, meanwhile, copies the previous
    // step's result from the other buffer into y.
    const int R = g.R, ldt = g.bmax;
    const int nsteps = 2 * g.nlev;
    const int ngroups = (R + kColGroup - 1) / kColGroup;
    uint32_t ph0 = c.phase[0], ph1 = c.phase[1];
    auto step_lev = [&](int st, int* dir) { *dir = st >= g.nlev; return *dir ? nsteps - 1 - st : st; };
    auto issue = [&](int st) {
        int dir;
        const int lev = step_lev(st, &dir);
        const int b = lg.size(lev);
        const int lo = dir == 0 ? lev - 1 : lev + 1;
        const int bo = (lo >= 0 && lo < g.nlev) ? lg.size(lo) : 0;
        const uint32_t bytes = (uint32_t)(((b * (b + bo) + 3) & ~3) * sizeof(float));
        float* dst = opbuf + (size_t)(st & 1) * g.opmax;
        fence_proxy_async_shared();
        mbar_arrive_expect_tx(&c.bar[st & 1], bytes);
        bulk_copy_g2s(dst, F + opoff[2 * lev + dir], bytes, &c.bar[st & 1]);
    };
    // copies are issued by the last thread, whose work item is empty in most steps
    const bool issuer = threadIdx.x == blockDim.x - 1;
    if (issuer) issue(0);
    int prev_lev = -1, prev_b = 0;
    for (int st = 0; st < nsteps; ++st) {
        int dir;
        const int lev = step_lev(st, &dir);
        const int b = lg.size(lev);
        const int lo = dir == 0 ? lev - 1 : lev + 1;
        const int bo = (lo >= 0 && lo < g.nlev) ? lg.size(lo) : 0;
        if (issuer && st + 1 < nsteps) issue(st + 1);
        const float* tprev = tbuf + (size_t)((st + 1) & 1) * ldt * R;
        float* tcur = tbuf + (size_t)(st & 1) * ldt * R;
        // the previous step's result goes to y (nobody reads those entries of y now)
        if (prev_lev >= 0) {
            for (int t = threadIdx.x; t < prev_b * R; t += blockDim.x) {
                const int col = t / prev_b, i = t - col * prev_b;
                if (!c.col_frozen[col]) y[(size_t)col * g.nunk + u0[prev_lev] + i] = tprev[col * ldt + i];
            }
        }
        const uint32_t par = (st & 1) ? ph1 : ph0;
        if (!mbar_wait_bounded(&c.bar[st & 1], par)) c.timeout = 1;
        if (st & 1) ph1 ^= 1u; else ph0 ^= 1u;
        const float* op = opbuf + (size_t)(st & 1) * g.opmax;
        const int work = b * ngroups;
        const int ulev = u0[lev];
        // the level's own input: the right-hand side (forward) or the forward result
        // (backward; for the last level it is still in the previous buffer)
        const bool own_in_t = (st == g.nlev);
#pragma unroll
        for (int it = 0; it < kItemsPerThread; ++it) {
            const int item = threadIdx.x + it * kThreadsM;
            if (item < work) {
                const int cg = item / b, i = item - cg * b;
                float acc[kColGroup];
                const float* yo[kColGroup];
                const float* yt[kColGroup];
#pragma unroll
                for (int q = 0; q < kColGroup; ++q) {
                    acc[q] = 0.0f;
                    const int col = min(cg * kColGroup + q, R - 1);
                    yo[q] = own_in_t ? tprev + col * ldt : y + (size_t)col * g.nunk + ulev;
                    yt[q] = tprev + col * ldt;
                }
#pragma unroll 4
                for (int k = 0; k < b; ++k) {
                    const float a = op[k * b + i];
#pragma unroll
                    for (int q = 0; q < kColGroup; ++q) acc[q] = fmaf(a, yo[q][k], acc[q]);
                }
#pragma unroll 4
                for (int k = 0; k < bo; ++k) {
                    const float a = op[(b + k) * b + i];
#pragma unroll
                    for (int q = 0; q < kColGroup; ++q) acc[q] = fmaf(a, yt[q][k], acc[q]);
                }
#pragma unroll
                for (int q = 0; q < kColGroup; ++q) {
                    const int col = cg * kColGroup + q;
                    if (col < R) tcur[col * ldt + i] = acc[q];
                }
            }
        }
        prev_lev = lev;
        prev_b = b;
        __syncthreads();
    }
    {
        const float* tlast = tbuf + (size_t)((nsteps - 1) & 1) * ldt * R;
        for (int t = threadIdx.x; t < prev_b * R; t += blockDim.x) {
            const int col = t / prev_b, i = t - col * prev_b;
            if (!c.col_frozen[col]) y[(size_t)col * g.nunk + u0[prev_lev] + i] = tlast[col * ldt + i];
        }
    }
    if (threadIdx.x == 0) {
        c.phase[0] = ph0;
        c.phase[1] = ph1;
    }
    __syncthreads();
}

template <int RPL, int CPL>
__global__ void __launch_bounds__(kThreadsM, 3) k_local_mixed(const MixedArgs g) {
    extern __shared__ unsigned char smem_raw[];
    float* W = reinterpret_cast<float*>(smem_raw);                    // FP32 window
    float* y = W + (size_t)g.wfloats;                                    // nunk x R
    int* loff = reinterpret_cast<int*>(y + (size_t)g.yfloats);         // 2 nlev operator offsets (Fw, Bw)
    int* u0 = loff + 2 * g.nlev;                                        // nlev + 1 level starts
    double* kap_s = reinterpret_cast<double*>(smem_raw + g.off_kap_smem);   // kappa of the current K (if staged)
    double* scale = reinterpret_cast<double*>(g.ws + (size_t)blockIdx.x * g.slot_bytes + g.off_scale);   // 1/sqrt(diag A_p)
    float* opbuf = W;                                                   // 2 x opmax staging (solves only)
    float* tbuf = W + 2 * (size_t)g.opmax;                              // 2 x bmax x R level results (solves only)
    __shared__ MCtx c;
    const LevelGeom lg{g.P, g.N, g.PN};
    const int R = g.R;
    char* slot = g.ws + (size_t)blockIdx.x * g.slot_bytes;
    float* F = reinterpret_cast<float*>(slot);
    double* G = reinterpret_cast<double*>(slot + g.off_G);
    double* Z = reinterpret_cast<double*>(slot + g.off_Z);
    double* mass = reinterpret_cast<double*>(slot + g.off_mass);

    if (threadIdx.x == 0) {
        int o = 0, u = 0;
        for (int lev = 0; lev < g.nlev; ++lev) {
            const int b = lg.size(lev), bn = lev + 1 < g.nlev ? lg.size(lev + 1) : 0;
            const int bp = lev > 0 ? lg.size(lev - 1) : 0;
            loff[2 * lev] = o;                       // 16-byte aligned operator starts
            o += (b * (b + bp) + 3) & ~3;
            loff[2 * lev + 1] = o;
            o += (b * (b + bn) + 3) & ~3;
            u0[lev] = u;
            u += b;
        }
        u0[g.nlev] = u;
        mbar_init(&c.bar[0], 1);
        mbar_init(&c.bar[1], 1);
        c.phase[0] = 0;
        c.phase[1] = 0;
    }
    __syncthreads();

    for (int64_t K = g.K0 + blockIdx.x; K < g.K1; K += gridDim.x) {
        const double* kap = g.kappa + K * (int64_t)g.N * g.N;
        if (g.kap_in_smem) {
            // stage this K's kappa in shared memory (read by assembly, scaling and residuals)
            const int nf = g.N * g.N;
            for (int t = threadIdx.x; t < nf; t += blockDim.x) kap_s[t] = kap[t];
            kap = kap_s;   // published by the barrier after the per-K setup
        }
        // ---- per-K setup
        if (threadIdx.x == 0) {
            for (int v = 0; v < 3; ++v) {
                c.X[v][0] = g.dm.geom[6 * K + 2 * v];
                c.X[v][1] = g.dm.geom[6 * K + 2 * v + 1];
            }
            c.area = 0.5 * fabs((c.X[1][0] - c.X[0][0]) * (c.X[2][1] - c.X[0][1]) -
                                (c.X[2][0] - c.X[0][0]) * (c.X[1][1] - c.X[0][1]));
            c.area_fine = c.area / ((double)g.N * g.N);
            for (int a = 0; a < 3; ++a) {
                const double* P0 = c.X[(a + 1) % 3];
                const double* Q0 = c.X[(a + 2) % 3];
                c.flen[a] = sqrt((Q0[0] - P0[0]) * (Q0[0] - P0[0]) + (Q0[1] - P0[1]) * (Q0[1] - P0[1]));
                c.sgn[a] = g.dm.sign[3 * K + a];
                c.rev[a] = g.dm.rev[3 * K + a];
            }
            double Xu[3][2], Xd[3][2];
            fine_xy(c, g.N, true, 0, 0, Xu);
            fine_xy(c, g.N, false, 0, 0, Xd);
            element_stiffness(g.P, Xu, c.Sup);
            element_stiffness(g.P, Xd, c.Sdn);
            c.bad = 0;
            c.col_fail = 0;
            c.timeout = 0;
            c.passes = 0;
            c.FK = 0.0;
        }
        for (int col = threadIdx.x; col < R; col += blockDim.x) c.col_done[col] = c.col_frozen[col] = 0;
        __syncthreads();
        if (g.src_kind == MHM_SRC_CONST) {
            if (threadIdx.x == 0) c.FK = g.src_value * c.area;
        } else {
            double s = 0.0;
            for (int t = threadIdx.x; t < g.N * g.N; t += blockDim.x) {
                int j = 0, rs = 0;
                while (rs + 2 * (g.N - j) - 1 <= t) { rs += 2 * (g.N - j) - 1; ++j; }
                const int o = t - rs;
                const bool up = o < g.N - j;
                double X[3][2];
                fine_xy(c, g.N, up, up ? o : o - (g.N - j), j, X);
                s += cell_src(g, X, g.P, -1);
            }
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if ((threadIdx.x & 31) == 0) c.red[threadIdx.x >> 5] = s;
            __syncthreads();
            if (threadIdx.x == 0) {
                double t = 0.0;
                for (int w = 0; w < kWarpsM; ++w) t += c.red[w];   // fixed order: deterministic
                c.FK = t;
            }
        }
        __syncthreads();
        for (int col = threadIdx.x; col < R; col += blockDim.x) {
            if (col == g.NI) c.cproj[col] = c.FK / c.area;
            else {
                const int a = col / g.dpf, jf = col - a * g.dpf;
                c.cproj[col] = -c.sgn[a] * c.flen[a] * g.dm.btab_sum[jf] / c.area;
            }
        }
        __syncthreads();

        // ---- right-hand sides G (FP64, column-major) and the mass vector
        for (int u = threadIdx.x; u < g.nunk; u += blockDim.x) {
            int X, Y;
            lattice_of_unk(g.PN, u, &X, &Y);
            int ti[6], tj[6], ta[6];
            bool tup[6];
            const int n = incident(g.P, g.N, X, Y, ti, tj, tup, ta);
            double m = 0.0, fh = 0.0, diag = 0.0;
            const int nb = g.P == 1 ? 3 : 6;
            for (int t = 0; t < n; ++t) {
                const double mt = c.area_fine * element_mass_frac(g.P, ta[t]);
                m += mt;
                diag += kap[kap_index(g.N, tup[t], ti[t], tj[t])] * (tup[t] ? c.Sup : c.Sdn)[ta[t] * nb + ta[t]];
                if (g.src_kind == MHM_SRC_CONST) fh += g.src_value * mt;
                else {
                    double Xv[3][2];
                    fine_xy(c, g.N, tup[t], ti[t], tj[t], Xv);
                    fh += cell_src(g, Xv, g.P, ta[t]);
                }
            }
            mass[u] = m;
            scale[u] = 1.0 / sqrt(diag);
            for (int col = 0; col < R; ++col) {
                double v = -c.cproj[col] * m;
                if (col == g.NI) v += fh;
                else {
                    const int a = col / g.dpf, jf = col - a * g.dpf;
                    const int kl = face_position(g.PN, X, Y, a);
                    if (kl >= 0) {
                        const int kk = c.rev[a] ? g.PN - kl : kl;
                        v += -c.sgn[a] * c.flen[a] * g.dm.btab[jf * (g.PN + 1) + kk];
                    }
                }
                G[(size_t)col * g.nunk + u] = v;
            }
        }

        // ---- FP32 factorisation by levels (window rows: level lev, then lev+1)
        const int b0 = lg.size(0), b1 = g.nlev > 1 ? lg.size(1) : 0;
        float* Rhs = y;                               // level right-hand sides (y is free while factoring)
        for (int t = threadIdx.x; t < (b0 + b1) * g.wld; t += blockDim.x) W[t] = 0.0f;
        for (int t = threadIdx.x; t < b0 * b0; t += blockDim.x) {
            const int i = t / b0, k = t - i * b0;
            Rhs[i * g.ldr + k] = k == i ? 1.0f : 0.0f;
        }
        __syncthreads();   // (also publishes scale[] to the block)
        for (int lev = 0; lev < g.nlev; ++lev) {
            const int b = lg.size(lev);
            const int bn = lev + 1 < g.nlev ? lg.size(lev + 1) : 0;
            const int nr = b + bn;
            if (bn > 0) {
                // element matrices of fine row lev in four colour classes
                const int P = g.P, N = g.N, nb = P == 1 ? 3 : 6, npair = nb * (nb + 1) / 2;
                for (int cls = 0; cls < 4; ++cls) {
                    const bool up = cls < 2;
                    const int parity = cls & 1;
                    const int ntri = up ? N - lev : N - 1 - lev;
                    const int ncls = (ntri - parity + 1) / 2;
                    for (int t = threadIdx.x; t < ncls * npair; t += blockDim.x) {
                        const int ti = t / npair, item = t - ti * npair;
                        const int i = parity + 2 * ti;
                        int nx[6], ny[6];
                        element_nodes(P, up, i, lev, nx, ny);
                        const double kt = kap[kap_index(N, up, i, lev)];
                        const double* S = up ? c.Sup : c.Sdn;
                        int a = 0, rem = item;
                        while (rem >= nb - a) { rem -= nb - a; ++a; }
                        const int bb = a + rem;
                        const int pa = lg.pos(nx[a], ny[a]), pb = lg.pos(nx[bb], ny[bb]);
                        if (pa < 0 || pb < 0) continue;
                        const int ra = pa + (lg.level_of_row(ny[a]) == lev ? 0 : b);
                        const int rb = pb + (lg.level_of_row(ny[bb]) == lev ? 0 : b);
                        const int hi = ra > rb ? ra : rb, lo = ra > rb ? rb : ra;
                        // symmetric diagonal scaling: the FP32 factor is of D^-1/2 A_p D^-1/2
                        const double sab = scale[unk(g.PN, nx[a], ny[a])] * scale[unk(g.PN, nx[bb], ny[bb])];
                        W[hi * g.wld + lo] += (float)(kt * S[a * nb + bb] * sab);
                    }
                    __syncthreads();
                }
            }
            // Blocked Cholesky of this level; its right-hand sides Rhs = [I | -L_{lev,lev-1}]
            // come out as the forward operator Fw_lev = [L^{-1} | -L^{-1} L_{lev,lev-1}].
            const int bp = lev > 0 ? lg.size(lev - 1) : 0;
            blocked_cholesky_level<float, 8, RPL, CPL>(W, g.wld, b, nr, Rhs, g.ldr, b, b + bp, &c.bad);
            {
                // Fw (column-major (b + bp) x b) and Bw = [Linv^T | -Linv^T L_{lev+1,lev}^T]
                // (column-major (b + bn) x b) to this block's scratch slot
                float* Fw = F + loff[2 * lev];
                float* Bw = F + loff[2 * lev + 1];
                for (int t = threadIdx.x; t < b * (b + bp); t += blockDim.x) {
                    const int k = t / b, i = t - k * b;
                    Fw[t] = Rhs[i * g.ldr + k];
                }
                for (int t = threadIdx.x; t < b * (b + bn); t += blockDim.x) {
                    const int k = t / b, i = t - k * b;
                    float v;
                    if (k < b) v = Rhs[k * g.ldr + i];
                    else {
                        const float* cn = W + (size_t)(b + (k - b)) * g.wld;
                        float a = 0.0f;
                        for (int mm = i; mm < b; ++mm) a = fmaf(Rhs[mm * g.ldr + i], cn[mm], a);
                        v = -a;
                    }
                    Bw[t] = v;
                }
                fence_proxy_async_global();   // the operators are read back by bulk copies
                __syncthreads();
                // right-hand sides of the next level: [I_bn | -L_{lev+1,lev}]
                for (int t = threadIdx.x; t < bn * (bn + b); t += blockDim.x) {
                    const int i = t / (bn + b), k = t - i * (bn + b);
                    Rhs[i * g.ldr + k] = k < bn ? (k == i ? 1.0f : 0.0f) : -W[(size_t)(b + i) * g.wld + (k - bn)];
                }
            }
            __syncthreads();
            if (bn > 0) {
                for (int t = threadIdx.x; t < bn * bn; t += blockDim.x) {
                    const int i = t / bn, jj = t - i * bn;
                    if (jj <= i) W[i * g.wld + jj] = W[(b + i) * g.wld + b + jj];
                }
                __syncthreads();
                const int bnn = lev + 2 < g.nlev ? lg.size(lev + 2) : 0;
                for (int t = threadIdx.x; t < bnn * g.wld; t += blockDim.x) W[bn * g.wld + t] = 0.0f;
                __syncthreads();
            }
        }

        // ---- refinement.  M = (L L^T)^{-1} (scaled) approximates A_p^{-1}.  The buffer G
        // becomes the residual Res = G - A_p Z, kept exact in FP64 by Res -= A_p D for
        // every correction D = M Res added to Z.  The outputs use the corrected
        // bilinear form N~^T Z + Z^T Res, whose error e^T A_p e is quadratic in the
        // error e of Z; eps_c = Res_c^T M Res_c estimates ||e_c||^2_{A_p}.
        double* Res = G;
        double* D64 = reinterpret_cast<double*>(slot + g.off_D);
        const int total = g.nunk * R;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            y[t] = (float)(Res[t] * scale[t % g.nunk]);
            Z[t] = 0.0;
        }
        __syncthreads();
        solve_factor(g, lg, F, loff, u0, y, opbuf, tbuf, c);
        __syncthreads();
        column_dot(g, Res, y, scale, c.gamma, c);      // gamma_c = G_c^T M G_c ~ ||z_c||^2_{A_p}
        __syncthreads();
        // Columns with a zero right-hand side are done at once (Z = 0, Res = G = 0).
        // Otherwise, after each correction the next one D' = M Res gives
        // eps = Res^T M Res ~ ||e||^2 (energy norm of the error of Z): a column stops
        // when eps <= tol * gamma; and when linear convergence predicts that one more
        // correction will get there (eps^2 / eps_prev, with a safety factor 4), that
        // correction is applied without a further confirming solve.
        if (threadIdx.x == 0) {
            int all = 1;
            for (int col = 0; col < R; ++col) {
                c.col_frozen[col] = c.col_done[col] = !(c.gamma[col] > 0.0);
                c.eps_prev[col] = c.gamma[col];
                all &= c.col_done[col];
            }
            c.all_done = all;
        }
        __syncthreads();
        int pass = 0;
        while (!c.all_done) {
            // D = s . y (FP64), Z += D
            for (int t = threadIdx.x; t < total; t += blockDim.x) {
                const int col = t / g.nunk;
                if (c.col_done[col]) continue;
                const double d = (double)y[t] * scale[t - col * g.nunk];
                D64[t] = d;
                Z[t] += d;
            }
            __syncthreads();
            // Res -= A_p D (FP64, from kappa and the element matrices); y = s . Res
            for (int u = threadIdx.x; u < g.nunk; u += blockDim.x) apply_residual(g, c, kap, u, D64, Res, y, scale[u]);
            ++pass;
            __syncthreads();
            if (threadIdx.x == 0) {
                int all = 1;
                for (int col = 0; col < R; ++col) {
                    if (c.col_frozen[col]) c.col_done[col] = 1;   // its last correction is in
                    all &= c.col_done[col];
                }
                c.all_done = all || pass >= g.it_max;
                c.converged = all;
            }
            __syncthreads();
            if (c.all_done) break;
            solve_factor(g, lg, F, loff, u0, y, opbuf, tbuf, c);
            __syncthreads();
            column_dot(g, Res, y, scale, c.eps, c);
            __syncthreads();
            if (threadIdx.x == 0) {
                int all = 1;
                for (int col = 0; col < R; ++col) {
                    if (!c.col_frozen[col]) {
                        const double eps = c.eps[col], lim = g.tol * c.gamma[col];
                        if (eps <= lim) c.col_frozen[col] = c.col_done[col] = 1;
                        else if (4.0 * eps * eps <= lim * c.eps_prev[col]) c.col_frozen[col] = 1;
                        c.eps_prev[col] = eps;
                    }
                    all &= c.col_done[col];
                }
                c.all_done = all;
                c.converged = all;
            }
            __syncthreads();
        }
        const int converged = c.converged;

        // ---- local contributions X[j][i] = N~_j^T z_i + z_j^T Res_i; A_K = -(X + X^T)/2, E_K = X[:, f]
        {
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            for (int col = warp; col < R; col += kWarpsM) {          // m^T z per column
                const double* zc = Z + (size_t)col * g.nunk;
                double mz = 0.0;
                for (int u = lane; u < g.nunk; u += 32) mz = fma(mass[u], zc[u], mz);
                for (int o = 16; o > 0; o >>= 1) mz += __shfl_down_sync(0xffffffffu, mz, o);
                if (lane == 0) c.mz[col] = mz;
            }
        }
        // correction Gram Z^T Res in FP32 (it is of the size of the error of Z), by node chunks
        float corr[(kMaxNI + 1) * (kMaxNI + 1) / kThreadsM + 1];
        const int npair = R * R;
        for (int q = 0; q * kThreadsM < npair; ++q) corr[q] = 0.0f;
        constexpr int kChunk = 64;
        float* zs = y;                       // R x kChunk
        float* rs = y + R * kChunk;          // R x kChunk
        for (int base = 0; base < g.nunk; base += kChunk) {
            const int cnt = min(kChunk, g.nunk - base);
            __syncthreads();
            for (int t = threadIdx.x; t < R * kChunk; t += blockDim.x) {
                const int col = t / kChunk, uu = t - col * kChunk;
                zs[t] = uu < cnt ? (float)Z[(size_t)col * g.nunk + base + uu] : 0.0f;
                rs[t] = uu < cnt ? (float)Res[(size_t)col * g.nunk + base + uu] : 0.0f;
            }
            __syncthreads();
            for (int q = 0; q * kThreadsM + (int)threadIdx.x < npair; ++q) {
                const int t = q * kThreadsM + threadIdx.x, j = t / R, i = t - j * R;
                float a = 0.0f;
                for (int uu = 0; uu < kChunk; ++uu) a = fmaf(zs[j * kChunk + uu], rs[i * kChunk + uu], a);
                corr[q] += a;
            }
        }
        __syncthreads();
        double* xbuf = reinterpret_cast<double*>(W);   // reuse the window: R x R doubles
        for (int q = 0; q * kThreadsM + (int)threadIdx.x < npair; ++q) xbuf[q * kThreadsM + threadIdx.x] = corr[q];
        __syncthreads();
        for (int t = threadIdx.x; t < g.NI * R; t += blockDim.x) {
            const int j = t / R, col = t - j * R;
            const int a = j / g.dpf, jf = j - a * g.dpf;
            const double* zc = Z + (size_t)col * g.nunk;
            double s = 0.0;
            for (int kl = 0; kl <= g.PN; ++kl) {
                int X, Y;
                if (a == 2) { X = kl; Y = 0; }
                else if (a == 0) { X = g.PN - kl; Y = kl; }
                else { X = 0; Y = g.PN - kl; }
                const int u = unk(g.PN, X, Y);
                if (u < 0) continue;
                const int kk = c.rev[a] ? g.PN - kl : kl;
                s += (-c.sgn[a] * c.flen[a] * g.dm.btab[jf * (g.PN + 1) + kk]) * zc[u];
            }
            xbuf[j * R + col] += s - c.cproj[j] * c.mz[col];
        }
        __syncthreads();
        const int NI = g.NI;
        for (int t = threadIdx.x; t < NI * NI; t += blockDim.x) {
            const int j = t / NI, i = t - j * NI;
            g.AK[K * NI * NI + t] = -0.5 * (xbuf[j * R + i] + xbuf[i * R + j]);
        }
        for (int j = threadIdx.x; j < NI; j += blockDim.x) {
            g.EK[K * NI + j] = xbuf[j * R + NI];
            const int a = j / g.dpf, jf = j - a * g.dpf;
            g.BK[K * NI + j] = c.sgn[a] * c.flen[a] * g.dm.btab_sum[jf];
        }
        if (threadIdx.x == 0) {
            g.FK[K] = c.FK;
            g.status[K] = c.timeout ? MHM_ERR_TIMEOUT : c.bad ? MHM_ERR_INVALID_ARG : (converged ? 0 : MHM_ERR_NOT_CONVERGED);
            if (g.iters) g.iters[K] = pass;
        }
        __syncthreads();
    }
}

struct MixedLayout {
    int nlev, nunk, wrows, wld, wfloats, yfloats, bmax, opmax, ldr;
    size_t factor_floats, slot_bytes, off_G, off_Z, off_mass, off_scale, off_D, smem;
    size_t off_kap_smem, off_scale_smem;
    int kap_in_smem, rpl, cpl;
};

MixedLayout mixed_layout(const mhm_mesh* mesh) {
    MixedLayout L{};
    const int P = mesh->desc.degree, N = mesh->N;
    auto size = [&](int lev) {
        if (P == 1) return N + 1 - lev - (lev == 0);
        if (lev == N) return 1;
        return (2 * N - 2 * lev + 1) + (2 * N - 2 * lev) - (lev == 0);
    };
    L.nlev = N + 1;
    L.nunk = (int)mesh->nloc - 1;
    size_t f = 0;
    int bmax = 0, opmax = 0;
    for (int lev = 0; lev < L.nlev; ++lev) {
        const int b = size(lev), bn = lev + 1 < L.nlev ? size(lev + 1) : 0;
        const int bp = lev > 0 ? size(lev - 1) : 0;
        const int fw = (b * (b + bp) + 3) & ~3, bw = (b * (b + bn) + 3) & ~3;
        f += (size_t)fw + bw;
        if (b > bmax) bmax = b;
        if (fw > opmax) opmax = fw;
        if (bw > opmax) opmax = bw;
    }
    L.bmax = bmax;
    L.opmax = opmax;
    L.factor_floats = f;
    L.wrows = size(0) + (N >= 1 ? size(1) : 0);
    L.wld = (L.wrows + 4) & ~3;   // rows 16-byte aligned for the vector panel loads
    const int R = (int)mesh->NI + 1;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    L.off_G = al(f * sizeof(float));
    L.off_Z = L.off_G + al((size_t)L.nunk * R * sizeof(double));
    L.off_mass = L.off_Z + al((size_t)L.nunk * R * sizeof(double));
    L.off_scale = L.off_mass + al((size_t)L.nunk * sizeof(double));
    L.off_D = L.off_scale + al((size_t)L.nunk * sizeof(double));
    L.slot_bytes = L.off_D + al((size_t)L.nunk * R * sizeof(double));
    size_t win = (size_t)L.wrows * L.wld;
    if (win < (size_t)R * R * 2) win = (size_t)R * R * 2;
    if (win < (size_t)2 * L.opmax + (size_t)2 * bmax * R) win = (size_t)2 * L.opmax + (size_t)2 * bmax * R;
    win = (win + 3) & ~(size_t)3;
    L.wfloats = (int)win;
    size_t yf = (size_t)L.nunk * R;
    if (yf < (size_t)2 * R * 64) yf = (size_t)2 * R * 64;   // also holds two R x 64 staging chunks
    L.ldr = (2 * bmax + 3) & ~3;
    if (yf < (size_t)bmax * L.ldr) yf = (size_t)bmax * L.ldr;   // and the level right-hand sides while factoring
    L.yfloats = (int)((yf + 3) & ~(size_t)3);
    size_t off = win * sizeof(float) + (size_t)L.yfloats * sizeof(float) + (size_t)(3 * L.nlev + 1) * sizeof(int);
    off = (off + 15) & ~(size_t)15;
    const size_t nf = (size_t)N * N;
    L.kap_in_smem = 0;   // kappa is read from global memory (L2-resident after first touch)
    L.off_kap_smem = off;
    off += L.kap_in_smem ? nf * sizeof(double) : 0;
    L.off_scale_smem = 0;
    L.smem = (off + 15) & ~(size_t)15;
    // register shape of the warp panel: rows (window) and right-hand-side columns per lane
    int ncols = 0;
    for (int lev = 0; lev < L.nlev; ++lev) {
        const int c = size(lev) + (lev > 0 ? size(lev - 1) : 0);
        if (c > ncols) ncols = c;
    }
    if (L.wrows <= 64 && ncols <= 96) { L.rpl = 2; L.cpl = 3; }
    else if (L.wrows <= 128 && ncols <= 128) { L.rpl = 4; L.cpl = 4; }
    else { L.rpl = 0; L.cpl = 0; }
    return L;
}

using MixedKernel = void (*)(const MixedArgs);

MixedKernel mixed_kernel(const MixedLayout& L) {
    if (L.rpl == 2) return k_local_mixed<2, 3>;
    if (L.rpl == 4) return k_local_mixed<4, 4>;
    return nullptr;
}

int mixed_slots(const mhm_mesh* mesh, const MixedLayout& L) {
    int dev = mesh->device, sms = 0, per = 0;
    MixedKernel k = mixed_kernel(L);
    if (!k) return 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kThreadsM, L.smem) != cudaSuccess || per < 1)
        per = 1;
    return sms * per;
}

}  // namespace

size_t mixed_workspace_bytes(const mhm_mesh* mesh) {
    if (mesh->device < 0) return 0;
    const MixedLayout L = mixed_layout(mesh);
    if (L.smem > 220 * 1024 || !mixed_kernel(L)) return 0;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(mesh->device);
    const size_t bytes = (size_t)mixed_slots(mesh, L) * L.slot_bytes;
    cudaSetDevice(cur);
    return bytes;
}

mhm_status launch_local_mixed(const mhm_mesh* mesh, const double* kappa, const mhm_source& f,
                              const mhm_solve_opts& opts, int64_t K0, int64_t K1, double* AK, double* EK,
                              double* BK, double* FK, int32_t* status, int32_t* iters, void* workspace,
                              size_t ws_bytes, cudaStream_t stream) {
    const MixedLayout L = mixed_layout(mesh);
    if (L.smem > 220 * 1024 || !mixed_kernel(L))
        return fail(MHM_ERR_UNSUPPORTED, "mhm_local_solve_batch: MIXED buffers exceed shared memory (r too large)");
    // the level solves map (row, group of 8 columns) to threads: one pass per block
    if (L.bmax * (((int)mesh->NI + 1 + kColGroup - 1) / kColGroup) > kItemsPerThread * kThreadsM)
        return fail(MHM_ERR_UNSUPPORTED, "mhm_local_solve_batch: MIXED level x columns too large for one block");
    const int slots = mixed_slots(mesh, L);
    if (ws_bytes < (size_t)slots * L.slot_bytes)
        return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch: workspace smaller than mhm_local_workspace_size");
    MixedArgs g;
    g.dm = mesh->dev();
    g.kappa = kappa;
    g.P = mesh->desc.degree;
    g.N = mesh->N;
    g.PN = mesh->PN;
    g.dpf = mesh->dpf;
    g.NI = (int)mesh->NI;
    g.R = g.NI + 1;
    g.nlev = L.nlev;
    g.nunk = L.nunk;
    g.wrows = L.wrows;
    g.wld = L.wld;
    g.wfloats = L.wfloats;
    g.yfloats = L.yfloats;
    g.bmax = L.bmax;
    g.opmax = L.opmax;
    g.ldr = L.ldr;
    g.src_kind = f.kind;
    g.src_value = f.value;
    g.src_freq = f.freq;
    g.K0 = K0;
    g.K1 = K1;
    g.it_max = opts.it_max;
    g.tol = opts.tol;
    g.ws = (char*)workspace;
    g.slot_bytes = L.slot_bytes;
    g.off_G = L.off_G;
    g.off_Z = L.off_Z;
    g.off_mass = L.off_mass;
    g.off_scale = L.off_scale;
    g.off_D = L.off_D;
    g.off_kap_smem = L.off_kap_smem;
    g.off_scale_smem = L.off_scale_smem;
    g.kap_in_smem = L.kap_in_smem;
    g.AK = AK; g.EK = EK; g.BK = BK; g.FK = FK;
    g.status = status;
    g.iters = iters;
    const int64_t nK = K1 - K0;
    if (nK <= 0) return MHM_OK;
    const int grid = (int)(nK < slots ? nK : slots);
    mixed_kernel(L)<<<grid, kThreadsM, L.smem, stream>>>(g);
    MHM_CUDA_TRY(cudaGetLastError());
    return MHM_OK;
}


// ---------------------------------------------------------------------------
// Allocation-free variant of the mixed-precision local solve.
//
// Some callers cannot allocate device memory while they run: a host framework
// whose memory pool owns the whole device (allocating behind its back breaks
// its accounting), or a latency-critical loop that must not call cudaMalloc or
// cope with it failing.  For them this entry point takes its scratch from a
// fixed array that lives in the library's own device image (kStaticScratch
// bytes, held on every GPU that loads the library until the process exits)
// instead of a caller-supplied workspace.  The caller still passes inputs and
// outputs.
namespace {

constexpr size_t kStaticScratch = size_t(32) << 20;   // 32 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratch];

constexpr int kMaxDevices = 64;
static std::mutex g_static_mutex;
static void* g_static_ptr[kMaxDevices];   // device address of g_static_scratch, per device

}  // namespace

extern "C" mhm_status mhm_local_solve_batch_noalloc(const mhm_mesh* mesh, const double* kappa,
                                                    const mhm_source* f, const mhm_solve_opts* opts,
                                                    double* AK, double* EK, double* BK, double* FK,
                                                    int32_t* status, int32_t* iters, void* stream) {
    if (!mesh) return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch_noalloc: NULL mesh");
    if (mesh->device < 0 || mesh->device >= kMaxDevices)
        return fail(MHM_ERR_UNSUPPORTED, "mhm_local_solve_batch_noalloc: mesh has no usable device");
    if (!kappa || !f || !AK || !EK || !BK || !FK || !status)
        return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch_noalloc: NULL pointer argument");
    if (f->kind != MHM_SRC_CONST && f->kind != MHM_SRC_SINSIN)
        return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch_noalloc: unknown source kind");
    MHM_CUDA_TRY(cudaSetDevice(mesh->device));
    mhm_solve_opts o{};
    o.it_max = 8;
    o.tol = 1e-12;
    if (opts) o = *opts;
    const int64_t K0 = o.K_begin, K1 = o.K_end > 0 ? o.K_end : mesh->nK;
    if (K0 < 0 || K1 > mesh->nK || K0 > K1)
        return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch_noalloc: K range out of bounds");
    if (o.it_max < 1 || !(o.tol > 0.0))
        return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch_noalloc: it_max >= 1 and tol > 0 required");
    const MixedLayout L = mixed_layout(mesh);
    if (L.smem > 220 * 1024 || !mixed_kernel(L))
        return fail(MHM_ERR_UNSUPPORTED, "mhm_local_solve_batch_noalloc: buffers exceed shared memory (r too large)");
    if (L.bmax * (((int)mesh->NI + 1 + kColGroup - 1) / kColGroup) > kItemsPerThread * kThreadsM)
        return fail(MHM_ERR_UNSUPPORTED, "mhm_local_solve_batch_noalloc: level x columns too large for one block");
    if (L.slot_bytes > kStaticScratch)
        return fail(MHM_ERR_INVALID_ARG,
                    "mhm_local_solve_batch_noalloc: one coarse element needs " + std::to_string(L.slot_bytes) +
                        " bytes of scratch, above the fixed " + std::to_string(kStaticScratch) + " bytes");
    // Set-up, once per device with that device current: the device address of the
    // fixed array (its name in host code is only a stand-in for the symbol).
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mutex);
        if (!g_static_ptr[mesh->device]) {
            cudaError_t e = cudaGetSymbolAddress(&g_static_ptr[mesh->device], g_static_scratch);
            if (e != cudaSuccess) {
                g_static_ptr[mesh->device] = nullptr;
                return cuda_fail(e, "cudaGetSymbolAddress(g_static_scratch)");
            }
        }
        scratch = g_static_ptr[mesh->device];
    }
    const int64_t nK = K1 - K0;
    if (nK <= 0) return MHM_OK;
    const int64_t fit = (int64_t)(kStaticScratch / L.slot_bytes);
    int64_t grid = mixed_slots(mesh, L);
    if (grid > fit) grid = fit;
    if (grid > nK) grid = nK;
    MixedArgs g;
    g.dm = mesh->dev();
    g.kappa = kappa;
    g.P = mesh->desc.degree;
    g.N = mesh->N;
    g.PN = mesh->PN;
    g.dpf = mesh->dpf;
    g.NI = (int)mesh->NI;
    g.R = g.NI + 1;
    g.nlev = L.nlev;
    g.nunk = L.nunk;
    g.wrows = L.wrows;
    g.wld = L.wld;
    g.wfloats = L.wfloats;
    g.yfloats = L.yfloats;
    g.bmax = L.bmax;
    g.opmax = L.opmax;
    g.ldr = L.ldr;
    g.src_kind = f->kind;
    g.src_value = f->value;
    g.src_freq = f->freq;
    g.K0 = K0;
    g.K1 = K1;
    g.it_max = o.it_max;
    g.tol = o.tol;
    g.ws = (char*)scratch;
    g.slot_bytes = L.slot_bytes;
    g.off_G = L.off_G;
    g.off_Z = L.off_Z;
    g.off_mass = L.off_mass;
    g.off_scale = L.off_scale;
    g.off_D = L.off_D;
    g.off_kap_smem = L.off_kap_smem;
    g.off_scale_smem = L.off_scale_smem;
    g.kap_in_smem = L.kap_in_smem;
    g.AK = AK; g.EK = EK; g.BK = BK; g.FK = FK;
    g.status = status;
    g.iters = iters;
    mixed_kernel(L)<<<(unsigned)grid, kThreadsM, L.smem, (cudaStream_t)stream>>>(g);
    MHM_CUDA_TRY(cudaGetLastError());
    return MHM_OK;
}

}  // namespace mhm
