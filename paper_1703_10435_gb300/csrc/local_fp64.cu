// solveLocalProblem in FP64 (Alg. 1; Sec. 3, Eqs. "etaf", "etai", "etaf_comb";
// Sec. 4.2, Eq. "source_term"), one thread block per coarse triangle K.
//
// What is computed.  With A the stiffness matrix of a(.,.)_K on the submesh,
// m_w = int_K phi_w, and the loads N_i = -(s psi_i, phi_w)_{dK}, F = (f, phi_w)_K,
// the zero-mean solutions are eta = z - (m^T z / |K|) 1 where z solves the
// system pinned at one DOF (choose_pin: inside the stiffest region touching the
// first two levels) with the compatible loads g~ = g - (1^T g / |K|) m.
// The face integrals of Eq. "mat_global" then reduce to a Gram matrix:
//     A_K = -N~^T A_p^{-1} N~ = -Y^T Y,   E_K = Y^T y_f,
// with Y = L^{-1} N~, y_f = L^{-1} f~ and A_p = L L^T (Cholesky of the pinned
// matrix).  Only the forward elimination is needed; no factor is stored.
//
// How.  A_p is block tridiagonal in the levels of the submesh (local_common.cuh).
// The kernel slides a window over two consecutive levels held in shared memory:
// rows [0, b) hold level lev (already reduced by the previous levels), rows
// [b, b + b') the fresh level lev+1, the columns are the symmetric part (lower
// triangle used) followed by the R = N_I + 1 right-hand sides.  It adds the
// element matrices and loads of fine row lev (the only triangles touching both
// levels), eliminates the b pivots of level lev by right-looking Cholesky on the
// augmented rows (which produces L, W = L^{-1} C^T, the Schur complement of
// level lev+1 and the forward-solved right-hand sides in one pass), accumulates
// Y_lev^T Y_lev into the Gram matrix and moves the reduced level lev+1 to the
// top of the window.
//
// Levels whose window does not fit in shared memory (P1 r = 7: 256 rows; P2 r = 5)
// keep it in global memory instead, one workspace slot per block of a persistent
// grid (one block per SM, so the slots stay in L2), and factor it panel by panel
// through shared memory (wide_cholesky_level).
#include <cuda_runtime.h>

#include "local_common.cuh"
#include "mixed_wide.h"

namespace mhm {

namespace {

constexpr int kThreads = 128;
constexpr int kThreadsWide = 512;   // wide window: one block per SM
constexpr int kNBWide = 16;         // wide window: pivots per panel

struct Fp64Args {
    DeviceMesh dm;
    const double* kappa;
    int P, N, PN, M, L, dpf, NI, R;
    int ld;        // leading dimension of the window (doubles)
    int rhs0;      // first right-hand-side column of the window
    int rows;      // window rows (largest b + b')
    int src_kind;
    const double* src_vals;   // MHM_SRC_QUAD: 16 values per fine triangle, laid out like kappa
    uint32_t* sword;          // the mesh's outcome word (mhm_sync_status)
    double src_value, src_freq;
    int64_t K0, K1;  // launch indices [K0, K1) within the level
    double* win;     // wide window: slots of win_doubles per block (NULL: window in shared memory)
    size_t win_doubles;
    double *AK, *EK, *BK, *FK;
    int32_t *status, *iters;
    const int32_t* kcount;   // launch indices >= *kcount do nothing (NULL: no bound)
    int fallback;            // 1: re-solving elements of a failed mixed refinement (iters = -1)
};

struct KCtx {
    double X[3][2];      // coarse vertices
    double Sup[36], Sdn[36];
    double area_fine;    // |T| of every fine triangle
    double area;         // |K|
    double flen[3];      // face lengths
    int sgn[3], rev[3], la1[3];  // la1: degree + 1 of each face
    double cproj[kMaxNI + 1];  // projection coefficient of each right-hand side
    double FK;
    int bad;             // first failing pivot (+1), 0 if none
    int pin_x, pin_y;    // the pinned lattice point (choose_pin)
};

// Sum over the block of one value per thread.
__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        red[0] = s;
    }
    __syncthreads();
    s = red[0];
    __syncthreads();
    return s;
}

// Cell integral of f phi_a over fine triangle (X0, X1, X2) by the collapsed
// 4 x 4 Gauss rule; phi_a = -1 means the integral of f itself.
__device__ double cell_source(const Fp64Args& g, const double X[3][2], int P, int a, const double* fq) {
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
            s += w * adet * source_at(g.src_kind, g.src_value, g.src_freq, x, y, fq, 4 * i + j) * phi;
        }
    return s;
}

// Vertices of fine triangle (up/down, i, j) in physical coordinates.
__device__ __forceinline__ void fine_vertices(const KCtx& c, int N, bool up, int i, int j, double X[3][2]) {
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

// Mass m_w = int_K phi_w of lattice point (x, y) of the (P N)-lattice: a third of the fine
// triangles around a P1 vertex; for P2 a third of the (one or two) triangles sharing an edge
// midpoint, zero at a vertex.
__device__ __forceinline__ double node_mass(int P, int N, int x, int y, double area_fine) {
    auto up_ok = [&](int i, int j) { return i >= 0 && j >= 0 && i + j <= N - 1; };
    auto dn_ok = [&](int i, int j) { return i >= 0 && j >= 0 && i + j <= N - 2; };
    int n = 0;
    if (P == 1) {
        n = up_ok(x, y) + up_ok(x - 1, y) + up_ok(x, y - 1) + dn_ok(x - 1, y - 1) + dn_ok(x - 1, y) + dn_ok(x, y - 1);
    } else if ((x & 1) && !(y & 1)) {          // horizontal edge midpoint
        n = up_ok((x - 1) >> 1, y >> 1) + dn_ok((x - 1) >> 1, (y >> 1) - 1);
    } else if (!(x & 1) && (y & 1)) {          // vertical edge midpoint
        n = up_ok(x >> 1, (y - 1) >> 1) + dn_ok((x >> 1) - 1, (y - 1) >> 1);
    } else if ((x & 1) && (y & 1)) {           // diagonal edge midpoint
        n = up_ok((x - 1) >> 1, (y - 1) >> 1) + dn_ok((x - 1) >> 1, (y - 1) >> 1);
    }
    return n * (area_fine / 3.0);
}

// Right-hand sides at the nodes of level lev (window rows row0 + p), once per node and
// column: the face load -(s psi_j, phi_w)_{dK} of multiplier column j on the nodes of its
// face, the compatible projection -(1^T g / |K|) m_w of every column, and a constant
// source's load f m_w (other sources' loads are added triangle by triangle in add_fine_row).
__device__ void add_node_loads(const Fp64Args& g, const KCtx& c, const LevelGeom& lg, int lev, int row0,
                               double* W) {
    const int b = lg.size(lev), R = g.R;
    for (int t = threadIdx.x; t < b * R; t += blockDim.x) {
        const int p = t / R, col = t - p * R;
        int x, y;
        lg.point(lev, p, &x, &y);
        const double m = node_mass(g.P, g.N, x, y, c.area_fine);
        double v = -c.cproj[col] * m;
        if (col == g.NI) {
            if (g.src_kind == MHM_SRC_CONST) v += g.src_value * m;
        } else {
            const int a = col / g.dpf, jf = col - a * g.dpf;
            const int kl = face_position(g.PN, x, y, a);
            const int row = face_row(jf, c.la1[a], g.dm.fm, g.dm.lmax1);
            if (kl >= 0 && row >= 0) {   // (an unused slot of a lower-degree face has no load)
                const int k = c.rev[a] ? g.PN - kl : kl;
                v += -c.sgn[a] * c.flen[a] * g.dm.btab[row * (g.PN + 1) + k];
            }
        }
        W[(row0 + p) * g.ld + g.rhs0 + col] += v;
    }
}

// Element contributions of fine row j (triangles touching levels j and j+1),
// in four colour classes of pairwise disjoint triangles; level j at window rows
// [0, b), level j+1 at [b, ...).
__device__ void add_fine_row(const Fp64Args& g, const KCtx& c, const LevelGeom& lg, int j, int b,
                             const double* kap, double* W) {
    const int P = g.P, N = g.N, nb = P == 1 ? 3 : 6, npair = nb * (nb + 1) / 2;
    const int rowstart = j * (2 * N - j);
    for (int cls = 0; cls < 4; ++cls) {
        const bool up = cls < 2;
        const int parity = cls & 1;
        const int ntri = up ? N - j : N - 1 - j;
        const int ncls = (ntri - parity + 1) / 2;
        const int per = npair + (g.src_kind == MHM_SRC_CONST ? 0 : nb);   // (the source load per vertex)
        for (int t = threadIdx.x; t < ncls * per; t += blockDim.x) {
            const int ti = t / per, item = t - ti * per;
            const int i = parity + 2 * ti;
            int nx[6], ny[6];
            element_nodes(P, up, i, j, nx, ny);
            const double kt = kap[rowstart + (up ? i : (N - j) + i)];
            const double* S = up ? c.Sup : c.Sdn;
            if (item < npair) {
                // pair (a <= bb) by row-major enumeration of the upper triangle
                int a = 0, rem = item;
                while (rem >= nb - a) { rem -= nb - a; ++a; }
                const int bb = a + rem;
                const int pa = lg.pos(nx[a], ny[a]), pb = lg.pos(nx[bb], ny[bb]);
                if (pa < 0 || pb < 0) continue;  // pinned DOF
                const int ra = pa + (lg.level_of_row(ny[a]) == j ? 0 : b);
                const int rb = pb + (lg.level_of_row(ny[bb]) == j ? 0 : b);
                const int hi = ra > rb ? ra : rb, lo = ra > rb ? rb : ra;
                W[hi * g.ld + lo] += kt * S[a * nb + bb];
            } else {
                // (f, phi_a)_T of a source that is not constant, in the source column
                const int a = item - npair;
                const int pa = lg.pos(nx[a], ny[a]);
                if (pa < 0) continue;
                const int ra = pa + (lg.level_of_row(ny[a]) == j ? 0 : b);
                double X[3][2];
                fine_vertices(c, N, up, i, j, X);
                W[ra * g.ld + g.rhs0 + g.NI] += cell_source(g, X, P, a, quad_of(g.src_vals, g.kappa, kap, N, up, i, j));
            }
        }
        __syncthreads();
    }
}

// Shared memory of the wide variant: the Gram matrix (R x R, rounded to an even count
// so the panel stays 16-byte aligned), the panel (rows x wide_panel_stride), its right-hand-side
// rows (kNBWide x R) and the inverse pivots (kNBWide).
__host__ __device__ inline size_t wide_gram_doubles(int R) { return ((size_t)R * R + 1) & ~(size_t)1; }
inline size_t wide_smem_bytes(int rows, int R) {
    return (wide_gram_doubles(R) + (size_t)rows * wide_panel_stride<kNBWide>() + (size_t)kNBWide * R + kNBWide) *
           sizeof(double);
}

template <int RPL, bool WIDE>
__global__ void __launch_bounds__(WIDE ? kThreadsWide : kThreads, WIDE ? 1 : 4) k_local_fp64(const Fp64Args g) {
    extern __shared__ double smem[];
    __shared__ KCtx c;
    __shared__ double red[32];
    const int R = g.R;
    // window rows x ld: shared memory, or this block's workspace slot
    double* W = WIDE ? g.win + (size_t)blockIdx.x * g.win_doubles : smem;
    double* gram = WIDE ? smem : smem + (size_t)g.rows * g.ld;   // R x R, upper triangle used
    double* Ps = smem + wide_gram_doubles(R);                      // (wide) panel
    double* Rs = Ps + (size_t)g.rows * wide_panel_stride<kNBWide>();
    double* invd = Rs + (size_t)kNBWide * R;
    // launch indices within the level: one per block, or (wide) strided over the grid
    for (int64_t ki = g.K0 + blockIdx.x; ki < g.K1; ki += gridDim.x) {
    if (g.kcount && ki >= *g.kcount) break;                        // (whole block)
    const int64_t K = g.dm.klist ? (int64_t)g.dm.klist[ki] : ki;  // coarse element
    const double* kap = g.kappa + (g.dm.kap_off ? g.dm.kap_off[K] : K * (int64_t)g.N * g.N);

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
            c.la1[a] = face_la1(g.dm, K, a);
        }
        double Xu[3][2], Xd[3][2];
        fine_vertices(c, g.N, true, 0, 0, Xu);
        fine_vertices(c, g.N, false, 0, 0, Xd);
        element_stiffness(g.P, Xu, c.Sup);
        element_stiffness(g.P, Xd, c.Sdn);
        c.bad = 0;
        choose_pin(g.P, g.N, kap, &c.pin_x, &c.pin_y);
    }
    __syncthreads();
    const LevelGeom lg{g.P, g.N, g.PN, c.pin_x, c.pin_y};
    // F_K = (f, 1)_K and the projection coefficients (1^T g) / |K| of every right-hand side
    double FK;
    if (g.src_kind == MHM_SRC_CONST) {
        FK = g.src_value * c.area;
    } else {
        double s = 0.0;
        for (int t = threadIdx.x; t < g.N * g.N; t += blockDim.x) {
            // fine triangle t in kappa order: row j, then up/down, column i
            int j = 0, rs = 0;
            while (rs + 2 * (g.N - j) - 1 <= t) { rs += 2 * (g.N - j) - 1; ++j; }
            const int o = t - rs;
            const bool up = o < g.N - j;
            const int i = up ? o : o - (g.N - j);
            double X[3][2];
            fine_vertices(c, g.N, up, i, j, X);
            s += cell_source(g, X, g.P, -1, quad_of(g.src_vals, g.kappa, kap, g.N, up, i, j));
        }
        FK = block_sum(s, red);
    }
    for (int col = threadIdx.x; col <= g.NI; col += blockDim.x) {
        if (col == g.NI) c.cproj[col] = FK / c.area;
        else {
            const int a = col / g.dpf, jf = col - a * g.dpf;
            const int row = face_row(jf, c.la1[a], g.dm.fm, g.dm.lmax1);
            c.cproj[col] = row < 0 ? 0.0 : -c.sgn[a] * c.flen[a] * g.dm.btab_sum[row] / c.area;
        }
    }
    for (int t = threadIdx.x; t < R * R; t += blockDim.x) gram[t] = 0.0;
    const int b0 = lg.size(0), b1 = lg.size(1);
    for (int t = threadIdx.x; t < (b0 + b1) * g.ld; t += blockDim.x) W[t] = 0.0;
    __syncthreads();
    add_node_loads(g, c, lg, 0, 0, W);
    __syncthreads();

    // ---- level sweep
    const int nlev = lg.n_levels();
    for (int lev = 0; lev < nlev; ++lev) {
        const int b = lg.size(lev);
        const int bn = lev + 1 < nlev ? lg.size(lev + 1) : 0;
        const int nr = b + bn;
        if (bn > 0) {
            add_node_loads(g, c, lg, lev + 1, b, W);
            __syncthreads();
            add_fine_row(g, c, lg, lev, b, kap, W);  // ends with a barrier
        }
        // Blocked right-looking Cholesky of the level's b pivots on the augmented window
        // rows; the right-hand-side columns (all window rows) are forward-substituted.
        if constexpr (WIDE) {
            // Gram += Y^T Y accumulated panel by panel
            wide_cholesky_level<kNBWide>(W, g.ld, b, nr, W + g.rhs0, g.ld, nr, R, &c.bad, Ps, Rs, invd, gram);
        } else {
            blocked_cholesky_level<double, 8, RPL, 2>(W, g.ld, b, nr, W + g.rhs0, g.ld, nr, R, &c.bad);
            // Gram += Y^T Y over the b rows of this level (upper triangle c1 <= c2)
            for (int t = threadIdx.x; t < R * (R + 1) / 2; t += blockDim.x) {
                int c1 = 0, c2 = t;   // t-th pair of the upper triangle, row by row
                while (c2 >= R - c1) { c2 -= R - c1; ++c1; }
                c2 += c1;
                double s = 0.0;
                for (int k = 0; k < b; ++k) s += W[k * g.ld + g.rhs0 + c1] * W[k * g.ld + g.rhs0 + c2];
                gram[c1 * R + c2] += s;
            }
            __syncthreads();
        }
        if (bn > 0) {
            // move the reduced level lev+1 (rows/cols [b, nr)) to the top; clear the next rows
            for (int t = threadIdx.x; t < bn * (bn + R); t += blockDim.x) {
                const int i = t / (bn + R), jj = t - i * (bn + R);
                if (jj < bn) {
                    if (jj <= i) W[i * g.ld + jj] = W[(b + i) * g.ld + b + jj];
                } else {
                    W[i * g.ld + g.rhs0 + (jj - bn)] = W[(b + i) * g.ld + g.rhs0 + (jj - bn)];
                }
            }
            __syncthreads();
            const int bnn = lev + 2 < nlev ? lg.size(lev + 2) : 0;
            for (int t = threadIdx.x; t < bnn * g.ld; t += blockDim.x) W[bn * g.ld + t] = 0.0;
            __syncthreads();
        }
    }

    // ---- outputs
    const int NI = g.NI;
    for (int t = threadIdx.x; t < NI * NI; t += blockDim.x) {
        const int j = t / NI, i = t - j * NI;
        const int lo = j < i ? j : i, hi = j < i ? i : j;
        g.AK[K * NI * NI + t] = -gram[lo * R + hi];
    }
    for (int j = threadIdx.x; j < NI; j += blockDim.x) {
        g.EK[K * NI + j] = gram[j * R + NI];
        const int a = j / g.dpf, jf = j - a * g.dpf;
        const int row = face_row(jf, c.la1[a], g.dm.fm, g.dm.lmax1);
        g.BK[K * NI + j] = row < 0 ? 0.0 : c.sgn[a] * c.flen[a] * g.dm.btab_sum[row];
    }
    if (threadIdx.x == 0) {
        g.FK[K] = FK;
        g.status[K] = c.bad ? MHM_ERR_INVALID_ARG : 0;
        if (g.iters) g.iters[K] = g.fallback ? -1 : 1;
        if (g.sword && (c.bad || g.fallback))
            atomicOr(g.sword, (c.bad ? 1u << MHM_ERR_INVALID_ARG : 0u) | (g.fallback ? MHM_STATUS_REFINED_IN_FP64 : 0u));
    }
    __syncthreads();   // the context, the Gram matrix and the window serve the next element
    }
}

}  // namespace

int fp64_window_rows(const mhm_mesh* mesh, const Level& lv) {
    // largest b + b' over consecutive levels: levels 0 and 1
    const int P = mesh->desc.degree, N = lv.N;
    auto size = [&](int lev) {
        if (P == 1) return N + 1 - lev - (lev == 0);
        if (lev == N) return 1;
        return (2 * N - 2 * lev + 1) + (2 * N - 2 * lev) - (lev == 0);
    };
    return size(0) + (N >= 1 ? size(1) : 0);
}

namespace {

// Window of a level: rows, leading dimension (even: 16-byte rows), shared memory, and
// whether it lives in global memory (more rows than the register panel holds, or more
// than the shared memory).
struct Fp64Shape {
    int rows, ld, R;
    size_t smem, win_doubles;
    bool wide;
};

Fp64Shape fp64_shape(const mhm_mesh* mesh, const Level& lv) {
    Fp64Shape sh;
    sh.R = (int)mesh->NI + 1;
    sh.rows = fp64_window_rows(mesh, lv);
    sh.ld = sh.rows + sh.R;
    if (sh.ld % 2 == 1) sh.ld += 1;
    sh.smem = ((size_t)sh.rows * sh.ld + (size_t)sh.R * sh.R) * sizeof(double);
    sh.wide = sh.rows > 128 || sh.smem > 220 * 1024;
    sh.win_doubles = ((size_t)sh.rows * sh.ld + 31) & ~(size_t)31;   // 256-byte slots
    if (sh.wide) sh.smem = wide_smem_bytes(sh.rows, sh.R);
    return sh;
}

int sm_count(const mhm_mesh* mesh) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, mesh->device);
    return sms > 0 ? sms : 1;
}

}  // namespace

size_t fp64_level_workspace(const mhm_mesh* mesh, const Level& lv) {
    if (mesh->device < 0) return 0;
    const Fp64Shape sh = fp64_shape(mesh, lv);
    if (!sh.wide) return 0;
    const int64_t slots = std::min<int64_t>(sm_count(mesh), std::max<int64_t>(lv.nK, 1));
    return (size_t)slots * sh.win_doubles * sizeof(double);
}

size_t fp64_slot_bytes(const mhm_mesh* mesh, const Level& lv) {
    const Fp64Shape sh = fp64_shape(mesh, lv);
    return sh.wide ? sh.win_doubles * sizeof(double) : 0;
}

bool fp64_level_launchable(const mhm_mesh* mesh, const Level& lv) {
    const Fp64Shape sh = fp64_shape(mesh, lv);
    return sh.smem <= 220 * 1024 && sh.R <= 64;
}

static mhm_status launch_fp64(const mhm_mesh* mesh, const Level& lv, const double* kappa, const mhm_source& f,
                              int64_t K0, int64_t K1, double* AK, double* EK, double* BK, double* FK,
                              int32_t* status, int32_t* iters, const int32_t* list, const int32_t* count,
                              void* ws, size_t ws_bytes, cudaStream_t stream) {
    Fp64Args g;
    g.dm = mesh->dev(lv);
    g.kcount = count;
    g.fallback = list != nullptr;
    if (list) g.dm.klist = list;
    g.kappa = kappa;
    g.P = mesh->desc.degree;
    g.N = lv.N;
    g.PN = lv.PN;
    g.M = mesh->desc.m;
    g.L = mesh->desc.l;
    g.dpf = mesh->dpf;
    g.NI = (int)mesh->NI;
    const Fp64Shape sh = fp64_shape(mesh, lv);
    g.R = sh.R;
    g.rows = sh.rows;
    g.rhs0 = sh.rows;
    g.ld = sh.ld;
    g.src_kind = f.kind;
    g.src_vals = f.kind == MHM_SRC_QUAD ? f.values_dev : nullptr;
    g.sword = mesh->d_sword;
    g.src_value = f.value;
    g.src_freq = f.freq;
    g.K0 = K0;
    g.K1 = K1;
    g.win = nullptr;
    g.win_doubles = sh.win_doubles;
    g.AK = AK; g.EK = EK; g.BK = BK; g.FK = FK;
    g.status = status;
    g.iters = iters;
    if (sh.smem > 220 * 1024)
        return fail(MHM_ERR_UNSUPPORTED, "mhm_local_solve_batch: FP64 window panel exceeds shared memory (r too large)");
    if (g.R > 64)
        return fail(MHM_ERR_UNSUPPORTED, "mhm_local_solve_batch: FP64 path takes at most 64 right-hand sides");
    const int64_t nblk = K1 - K0;
    if (nblk <= 0) return MHM_OK;
    void (*kern)(const Fp64Args);
    int64_t grid = nblk;
    int threads = kThreads;
    if (sh.wide) {
        // persistent grid: one block per SM and workspace slot
        const int64_t fit = ws ? (int64_t)(ws_bytes / (sh.win_doubles * sizeof(double))) : 0;
        grid = std::min<int64_t>(std::min<int64_t>(sm_count(mesh), fit), nblk);
        if (grid < 1)
            return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch: the FP64 window of this level needs a workspace of " +
                                                 std::to_string(sh.win_doubles * sizeof(double)) + " bytes or more");
        if (reinterpret_cast<uintptr_t>(ws) % 16 != 0)
            return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch: workspace must be 16-byte aligned");
        g.win = static_cast<double*>(ws);
        kern = k_local_fp64<4, true>;
        threads = kThreadsWide;
    } else {
        // register shape of the warp panel: window rows per lane
        kern = sh.rows <= 64 ? k_local_fp64<2, false> : k_local_fp64<4, false>;
    }
    MHM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem));
    timing_mark(mesh, MHM_KERNEL_LOCAL_FP64, stream, true);
    kern<<<(unsigned)grid, threads, sh.smem, stream>>>(g);
    timing_mark(mesh, MHM_KERNEL_LOCAL_FP64, stream, false);
    MHM_CUDA_TRY(cudaGetLastError());
    return MHM_OK;
}

mhm_status launch_local_fp64(const mhm_mesh* mesh, const Level& lv, const double* kappa, const mhm_source& f,
                             int64_t K0, int64_t K1, double* AK, double* EK, double* BK, double* FK, int32_t* status,
                             int32_t* iters, void* ws, size_t ws_bytes, cudaStream_t stream) {
    // K0, K1: launch indices within the level (its K list, or K itself on a uniform mesh)
    return launch_fp64(mesh, lv, kappa, f, K0, K1, AK, EK, BK, FK, status, iters, nullptr, nullptr, ws, ws_bytes,
                       stream);
}

mhm_status launch_local_fp64_list_ws(const mhm_mesh* mesh, const Level& lv, const double* kappa,
                                     const mhm_source& f, const int32_t* list, const int32_t* count, int64_t max_n,
                                     double* AK, double* EK, double* BK, double* FK, int32_t* status,
                                     int32_t* iters, void* ws, size_t ws_bytes, cudaStream_t stream) {
    // re-solves of failed elements of a wide mixed level: the window may need the workspace
    return launch_fp64(mesh, lv, kappa, f, 0, max_n, AK, EK, BK, FK, status, iters, list, count, ws, ws_bytes, stream);
}

mhm_status launch_local_fp64_list(const mhm_mesh* mesh, const Level& lv, const double* kappa, const mhm_source& f,
                                  const int32_t* list, const int32_t* count, int64_t max_n, double* AK, double* EK,
                                  double* BK, double* FK, int32_t* status, int32_t* iters, cudaStream_t stream) {
    // re-solves of failed mixed elements: mixed levels always have a shared-memory window
    return launch_fp64(mesh, lv, kappa, f, 0, max_n, AK, EK, BK, FK, status, iters, list, count, nullptr, 0, stream);
}

}  // namespace mhm
