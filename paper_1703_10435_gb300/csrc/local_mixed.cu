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

#include <algorithm>
#include <mutex>
#include <string>

#include "local_common.cuh"

namespace mhm {

namespace {

constexpr int kThreadsM = 256;
constexpr int kWarpsM = kThreadsM / 32;
constexpr int kMaxOpBufs = 4;   // level-Schur solves: shared-memory ring of staged level operators

struct MixedArgs {
    DeviceMesh dm;
    const double* kappa;
    int P, N, PN, dpf, NI, R, Rp, nlev, nunk;   // Rp: row length of y (= R)
    int wrows, wld;               // FP32 window rows and leading dimension
    int wfloats;                  // floats reserved for the window (also holds R x R doubles)
    int yfloats;                  // floats reserved for the right-hand-side block (>= nunk Rp)
    int bmax;                     // largest level size
    int opmax;                    // floats of the largest level operator (fragment order, multiple of 128)
    int stage_floats;             // floats of one staged solve operand (fragment order)
    int ldr;                      // leading dimension of the level right-hand sides (multiple of 4)
    int src_kind;
    const double* src_vals;       // MHM_SRC_QUAD: 16 values per fine triangle, laid out like kappa
    uint32_t* sword;              // the mesh's outcome word (mhm_sync_status)
    int word_final;               // 1: a failed status is final (no FP64 re-solve follows)
    double src_value, src_freq;
    int64_t K0, K1;
    int it_max;
    double tol;
    char* ws;
    size_t slot_bytes, off_G, off_Z, off_mass, off_scale, off_D;
    size_t off_kap_smem, off_scale_smem, off_sinfo, off_cw;
    int kap_in_smem;
    double *AK, *EK, *BK, *FK;
    int32_t *status, *iters;
    // level-Schur operators computed by the factor kernel for the chunk [Kc0, K1); the
    // per-K arrays below start at launch index Kbase (the chunk's first, or 0 for a factor
    // store that holds the whole level)
    float* Tall;                  // t_stride floats per K
    float* cwall;                 // 4 nunk floats per K
    int* fbad;                    // pivot flag per K
    double* scall;                // s_u = A_uu^-1/2, nunk per K
    double* ahall;                // scaled stencil S A S: 7 x nunk per K (self, E, W, N, S, SE, NW)
    int64_t Kc0, Kbase;
    size_t t_stride;
    int* kcounter;                // dynamic K assignment (zeroed before the launch); NULL: static
    // level-Schur solves (tuning knobs): operator buffers in the shared-memory ring (2..4;
    // the copy of step s + nbuf - 1 is issued at step s), L2 prefetch distance in steps
    // (0: none), prefetch of the element's whole operator set into L2 at the start of each
    // solve, and the L2 policy of the operator copies (0 default, 1 evict first, 2 evict last)
    int nbuf, l2pf, pf_all, op_policy;
};

struct MCtx {
    double X[3][2];
    double Sup[36], Sdn[36];
    double area_fine, area, FK;
    double flen[3];
    int sgn[3], rev[3], la1[3];   // la1: degree + 1 of each face
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
    float epsred[2][32];          // level-Schur solve: per row-tile partial sums of g^T T g per column
    uint32_t rmask[3][kWarpsM];   // level-Schur refinement: stencil directions each warp's rows use
    int64_t nextK;
    double mz[kMaxNI + 1];
    alignas(8) uint64_t bar[kMaxOpBufs];
    uint32_t phase[kMaxOpBufs];
    alignas(8) uint64_t ebar[kMaxOpBufs];   // level-Schur solves by column groups: slot released
    uint32_t ephase[kMaxOpBufs];
    int timeout;
};

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

__device__ double cell_src(const MixedArgs& g, const double X[3][2], int P, int a, const double* fq) {
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

// Row y of lattice DOF d = u + 1 solves S(y) <= d < S(y + 1), S(y) = y (2 PN + 3 - y) / 2
// (the first DOF of row y): the root of the quadratic in FP32, then an exact fix-up.
__device__ __forceinline__ void lattice_of_unk(int PN, int u, int* X, int* Y) {
    const int d = u + 1, b = 2 * PN + 3;
    int y = (int)(0.5f * ((float)b - sqrtf((float)(b * b - 8 * d))));
    y = max(0, min(y, PN));
    while (y < PN && (y + 1) * (b - y - 1) / 2 <= d) ++y;
    while (y > 0 && y * (b - y) / 2 > d) --y;
    *X = d - y * (b - y) / 2;
    *Y = y;
}

// Conversions between FP32 and FP64 by rearranging the IEEE-754 fields on the
// integer pipe (a hardware conversion occupies the FP64 pipe here, at the rate of
// an FP64 multiply-add).  f2d_bits is exact for zero and normal numbers (FP32
// subnormals flush to zero); d2f_bits truncates the significand (round toward
// zero) and flushes magnitudes below the FP32 normal range to zero.  Only finite
// values of FP32 range pass through them.
__device__ __forceinline__ double f2d_bits(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xffu;
    const uint32_t hi = e ? (b & 0x80000000u) | ((e + 896u) << 20) | ((b >> 3) & 0xfffffu) : (b & 0x80000000u);
    const uint32_t lo = e ? (b << 29) : 0u;
    return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ float d2f_bits(double d) {
    const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;
    if (e <= 0) return __uint_as_float(hi & 0x80000000u);
    return __uint_as_float((hi & 0x80000000u) | ((uint32_t)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

// x == 0 (either sign) tested on the integer pipe (a floating-point comparison of doubles
// occupies the FP64 pipe)
__device__ __forceinline__ bool is_zero(double x) { return (__double_as_longlong(x) << 1) == 0; }
__device__ __forceinline__ bool is_zero(float x) { return (__float_as_uint(x) << 1) == 0; }

// kappa in the arithmetic of an assembled row (FP32: converted on the integer pipe)
template <typename T> __device__ __forceinline__ T kappa_as(double k);
template <> __device__ __forceinline__ double kappa_as<double>(double k) { return k; }
template <typename T> __device__ __forceinline__ T kappa_as(float k) { return (T)k; }

// The assembled P1 row of unknown u at lattice point (x, yl): the weights of u and
// of its six lattice neighbours (east, west, north, south, south-east, north-west:
// the edges of the six fine triangles around it) and their unknown indices.  A
// neighbour outside K, the pinned DOF, or an edge of zero weight (a right angle)
// gets weight 0 and index u.
template <typename T, typename KT = double>
__device__ __forceinline__ void p1_row(int N, int PN, int nunk, const T* Su, const T* Sd, const KT* kap,
                                       int x, int yl, int u, T w[7], int v[7]) {
    auto kup = [&](int i, int j) { return (i >= 0 && j >= 0 && i + j <= N - 1) ? kappa_as<T>(kap[kap_index(N, true, i, j)]) : T(0); };
    auto kdn = [&](int i, int j) { return (i >= 0 && j >= 0 && i + j <= N - 2) ? kappa_as<T>(kap[kap_index(N, false, i, j)]) : T(0); };
    const T k1 = kup(x, yl), k2 = kup(x - 1, yl), k3 = kup(x, yl - 1);
    const T k4 = kdn(x - 1, yl - 1), k5 = kdn(x - 1, yl), k6 = kdn(x, yl - 1);
    w[0] = k1 * Su[0] + k2 * Su[4] + k3 * Su[8] + k4 * Sd[4] + k5 * Sd[0] + k6 * Sd[8];  v[0] = u;
    w[1] = k1 * Su[1] + k6 * Sd[7];  v[1] = unk(PN, x + 1, yl);        // east
    w[2] = k2 * Su[3] + k4 * Sd[5];  v[2] = unk(PN, x - 1, yl);        // west
    w[3] = k1 * Su[2] + k5 * Sd[1];  v[3] = unk(PN, x, yl + 1);        // north
    w[4] = k3 * Su[6] + k4 * Sd[3];  v[4] = unk(PN, x, yl - 1);        // south
    w[5] = k3 * Su[7] + k6 * Sd[6];  v[5] = unk(PN, x + 1, yl - 1);    // south-east
    w[6] = k2 * Su[5] + k5 * Sd[2];  v[6] = unk(PN, x - 1, yl + 1);    // north-west
    for (int k = 1; k < 7; ++k)
        if (is_zero(w[k]) || v[k] < 0 || v[k] >= nunk) { w[k] = T(0); v[k] = u; }
}

// The assembled P2 row of unknown u at point (X, Y) of the (2N)-lattice: the weights
// of u and of the points it shares a fine triangle with (19 around a vertex, 9 around
// an edge midpoint), summed over those triangles (x = X >> 1, y = Y >> 1 indexes the
// N-lattice), and their unknown indices.  Returns the number of entries (u first).
// An entry outside K, the pinned DOF, or of zero weight gets weight 0 and index u.
template <typename T, typename KT = double>
__device__ __forceinline__ int p2_row(int N, int PN, int nunk, const T* Su, const T* Sd, const KT* kap,
                                      int X, int Y, int u, T w[19], int v[19]) {
    auto kup = [&](int i, int j) { return (i >= 0 && j >= 0 && i + j <= N - 1) ? kappa_as<T>(kap[kap_index(N, true, i, j)]) : T(0); };
    auto kdn = [&](int i, int j) { return (i >= 0 && j >= 0 && i + j <= N - 2) ? kappa_as<T>(kap[kap_index(N, false, i, j)]) : T(0); };
    const int x = X >> 1, y = Y >> 1;
    int n;
#pragma unroll
    for (int k = 9; k < 19; ++k) { w[k] = T(0); v[k] = u; }   // (a midpoint's row has 9 entries)
    if (!(X & 1) && !(Y & 1)) {   // vertex
        const T k0 = kup(x, y), k1 = kup(x - 1, y), k2 = kup(x, y - 1), k3 = kdn(x - 1, y - 1), k4 = kdn(x - 1, y), k5 = kdn(x, y - 1);
        w[0] = k0 * Su[0] + k1 * Su[7] + k2 * Su[14] + k3 * Sd[7] + k4 * Sd[0] + k5 * Sd[14];  v[0] = u;
        w[1] = k2 * Su[12] + k3 * Sd[6];  v[1] = unk(PN, X, Y - 2);
        w[2] = k2 * Su[17];  v[2] = unk(PN, X + 1, Y - 2);
        w[3] = k2 * Su[13] + k5 * Sd[12];  v[3] = unk(PN, X + 2, Y - 2);
        w[4] = k3 * Sd[10];  v[4] = unk(PN, X - 1, Y - 1);
        w[5] = k2 * Su[16] + k3 * Sd[11];  v[5] = unk(PN, X, Y - 1);
        w[6] = k2 * Su[15] + k5 * Sd[16];  v[6] = unk(PN, X + 1, Y - 1);
        w[7] = k5 * Sd[17];  v[7] = unk(PN, X + 2, Y - 1);
        w[8] = k1 * Su[6] + k3 * Sd[8];  v[8] = unk(PN, X - 2, Y);
        w[9] = k1 * Su[11] + k3 * Sd[9];  v[9] = unk(PN, X - 1, Y);
        w[10] = k0 * Su[5] + k5 * Sd[15];  v[10] = unk(PN, X + 1, Y);
        w[11] = k0 * Su[1] + k5 * Sd[13];  v[11] = unk(PN, X + 2, Y);
        w[12] = k1 * Su[10];  v[12] = unk(PN, X - 2, Y + 1);
        w[13] = k1 * Su[9] + k4 * Sd[4];  v[13] = unk(PN, X - 1, Y + 1);
        w[14] = k0 * Su[4] + k4 * Sd[5];  v[14] = unk(PN, X, Y + 1);
        w[15] = k0 * Su[3];  v[15] = unk(PN, X + 1, Y + 1);
        w[16] = k1 * Su[8] + k4 * Sd[2];  v[16] = unk(PN, X - 2, Y + 2);
        w[17] = k4 * Sd[3];  v[17] = unk(PN, X - 1, Y + 2);
        w[18] = k0 * Su[2] + k4 * Sd[1];  v[18] = unk(PN, X, Y + 2);
        n = 19;
    } else if ((X & 1) && !(Y & 1)) {   // horizontal
        const T k0 = kup(x, y), k1 = kdn(x, y - 1);
        w[0] = k0 * Su[35] + k1 * Sd[21];  v[0] = u;
        w[1] = k1 * Sd[18];  v[1] = unk(PN, X + 1, Y - 2);
        w[2] = k1 * Sd[22];  v[2] = unk(PN, X, Y - 1);
        w[3] = k1 * Sd[23];  v[3] = unk(PN, X + 1, Y - 1);
        w[4] = k0 * Su[30] + k1 * Sd[20];  v[4] = unk(PN, X - 1, Y);
        w[5] = k0 * Su[31] + k1 * Sd[19];  v[5] = unk(PN, X + 1, Y);
        w[6] = k0 * Su[34];  v[6] = unk(PN, X - 1, Y + 1);
        w[7] = k0 * Su[33];  v[7] = unk(PN, X, Y + 1);
        w[8] = k0 * Su[32];  v[8] = unk(PN, X - 1, Y + 2);
        n = 9;
    } else if (!(X & 1) && (Y & 1)) {   // vertical
        const T k0 = kup(x, y), k1 = kdn(x - 1, y);
        w[0] = k0 * Su[28] + k1 * Sd[35];  v[0] = u;
        w[1] = k0 * Su[24] + k1 * Sd[30];  v[1] = unk(PN, X, Y - 1);
        w[2] = k0 * Su[29];  v[2] = unk(PN, X + 1, Y - 1);
        w[3] = k0 * Su[25];  v[3] = unk(PN, X + 2, Y - 1);
        w[4] = k1 * Sd[34];  v[4] = unk(PN, X - 1, Y);
        w[5] = k0 * Su[27];  v[5] = unk(PN, X + 1, Y);
        w[6] = k1 * Sd[32];  v[6] = unk(PN, X - 2, Y + 1);
        w[7] = k1 * Sd[33];  v[7] = unk(PN, X - 1, Y + 1);
        w[8] = k0 * Su[26] + k1 * Sd[31];  v[8] = unk(PN, X, Y + 1);
        n = 9;
    } else {   // diagonal
        const T k0 = kup(x, y), k1 = kdn(x, y);
        w[0] = k0 * Su[21] + k1 * Sd[28];  v[0] = u;
        w[1] = k0 * Su[18];  v[1] = unk(PN, X - 1, Y - 1);
        w[2] = k0 * Su[23];  v[2] = unk(PN, X, Y - 1);
        w[3] = k0 * Su[19] + k1 * Sd[24];  v[3] = unk(PN, X + 1, Y - 1);
        w[4] = k0 * Su[22];  v[4] = unk(PN, X - 1, Y);
        w[5] = k1 * Sd[29];  v[5] = unk(PN, X + 1, Y);
        w[6] = k0 * Su[20] + k1 * Sd[26];  v[6] = unk(PN, X - 1, Y + 1);
        w[7] = k1 * Sd[27];  v[7] = unk(PN, X, Y + 1);
        w[8] = k1 * Sd[25];  v[8] = unk(PN, X + 1, Y + 1);
        n = 9;
    }
#pragma unroll
    for (int k = 1; k < 19; ++k)
        if (is_zero(w[k]) || v[k] < 0 || v[k] >= nunk) { w[k] = T(0); v[k] = u; }
    return n;
}

// The assembled row of degree P (entries past the P1 row's seven: weight 0, index u).
template <typename T, typename KT = double>
__device__ __forceinline__ void assembled_row(int P, int N, int PN, int nunk, const T* Su, const T* Sd,
                                              const KT* kap, int X, int Y, int u, T w[19], int v[19]) {
    if (P == 2) {
        p2_row<T, KT>(N, PN, nunk, Su, Sd, kap, X, Y, u, w, v);
        return;
    }
    p1_row<T, KT>(N, PN, nunk, Su, Sd, kap, X, Y, u, w, v);
    for (int k = 7; k < 19; ++k) { w[k] = T(0); v[k] = u; }
}

// Res(u, :) -= (A_p D)(u, :) for the columns still refining, in FP64, and the next
// FP32 right-hand side y(u, :) = s_u Res(u, :), from the assembled row of u (the sum
// over the fine triangles T containing u of kappa_T S_T[a_u][b]): 7 entries for P1,
// up to 19 for P2.
__device__ void apply_residual(const MixedArgs& g, const MCtx& c, const double* kap, int u, const double* D,
                               double* Res, float* y, const double s_u) {
    int X, Y;
    lattice_of_unk(g.PN, u, &X, &Y);
    const size_t ld = (size_t)g.nunk;
    double w[19];
    int v[19];
    assembled_row(g.P, g.N, g.PN, g.nunk, c.Sup, c.Sdn, kap, X, Y, u, w, v);
    uint32_t nz = 0;   // non-zero weights (zero: edges at right angles), tested on the integer pipe
#pragma unroll
    for (int k = 0; k < 19; ++k)
        if ((__double_as_longlong(w[k]) << 1) != 0) nz |= 1u << k;
    for (int col = 0; col < g.R; ++col) {
        if (c.col_done[col]) continue;
        const double* Dc = D + col * ld;
        double a = 0.0;
#pragma unroll
        for (int k = 0; k < 19; ++k)
            if (nz >> k & 1) a = fma(w[k], Dc[v[k]], a);
        const double rn = Res[col * ld + u] - a;
        Res[col * ld + u] = rn;
        y[(size_t)u * g.Rp + col] = d2f_bits(rn * s_u);
    }
}

// out[c] = sum_u Res(u, c) s(u) y(u, c) for the columns still refining (warp per
// column, fixed summation order).
__device__ __noinline__ void column_dot(const MixedArgs& g, const double* Res, const float* y, const double* s, double* out,
                           const MCtx& c) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int col = warp; col < g.R; col += kWarpsM) {
        if (c.col_frozen[col]) continue;
        const double* rc = Res + (size_t)col * g.nunk;
        float a = 0.0f;   // an error estimate: FP32 is ample
        for (int u = lane; u < g.nunk; u += 32) a = fmaf(d2f_bits(rc[u]) * d2f_bits(s[u]), y[(size_t)u * g.Rp + col], a);
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) out[col] = (double)a;
    }
}

// Forward + backward solve of L L^T D = Y in FP32 for every column still
// refining, in place in y (node-major: y[u * R + col]).  Level by level,
//   forward   y_lev = Fw_lev [y_{lev-1}; y_lev],  Fw_lev = [-L_lev^{-1} L_{lev,lev-1} | L_lev^{-1}]
//   backward  x_lev = Bw_lev [x_{lev+1}; y_lev],  Bw_lev = [-L_lev^{-T} L_{lev+1,lev}^T | L_lev^{-T}]
// so each step is one small dense product T = Op B (b x K times K x R,
// K = b' + b, the neighbouring level's rows first).  It runs on the tensor
// cores as warp-level m16n8k8 TF32 products with a three-term split of both
// operands (x = hi + lo, both TF32; hi*hi + hi*lo + lo*hi in FP32
// accumulators), which keeps FP32 accuracy (hi keeps the 10 leading mantissa
// bits that the tensor core reads, lo = x - hi is exact in FP32, and the
// product drops lo*lo and the bits of lo below TF32: about 2^-20 relative):
// one warp per 16 x 8 output tile,
// its operands read as one 16-byte and one 8-byte shared load per 8 x 8 block.
// Op is stored by the factorisation in fragment order; B is staged in fragment
// order by the step before (its result tiles, which become the next level's
// neighbouring rows, and the next level's own rows copied from y), double
// buffered, so a step needs one block barrier.  The operators stream into two
// shared-memory buffers by bulk asynchronous copies, the copy for step s+1
// running while step s computes.
// Split by masking (the rounding conversion is a slow multi-cycle instruction here).
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    hi = __float_as_uint(x) & 0xffffe000u;
    lo = __float_as_uint(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ float4 lds4(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ float2 lds2(uint32_t a) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ float lds1(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts1(uint32_t a, float v) {
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

// Fragment positions (floats).  A operand (row-major 16 x 8 tiles, tile (mt, kt)
// of KT k-tiles, 128 floats each): lane = 4 g + t holds A[g][t], A[g+8][t],
// A[g][t+4], A[g+8][t+4] at 4 lane + 0..3 (the factorisation writes this order).
// B operand (8 x 8 tiles, tile (kt, nt) of NT n-tiles): lane = 4 g + t holds B[t][g], B[t+4][g].
__device__ __forceinline__ int frag_b_pos(int k, int n, int NT) {
    const int lane = (n & 7) * 4 + (k & 3);
    return (((k >> 3) * NT + (n >> 3)) * 32 + lane) * 2 + ((k >> 2) & 1);
}
// Floats of an operator of b rows and K columns in fragment order.
__host__ __device__ __forceinline__ int frag_op_floats(int b, int K) {
    return ((b + 15) / 16) * ((K + 7) / 8) * 128;
}

// One warp's 16 x 8 output tile: C = sum over the KT k-tiles of A(mt, kt) B(kt, nt)
// with the three-term split, in three independent accumulator chains (hi*hi,
// hi*lo, lo*hi) summed at the end.  KT > 0 is a compile-time trip count (the
// loop is fully unrolled and scheduled); KT = 0 takes the run-time count kt_n.
template <int KT>
__device__ __forceinline__ void tile_product(uint32_t aa, uint32_t ba, uint32_t bstep, int kt_n, float (&c)[4]) {
    float chh[4] = {0.f, 0.f, 0.f, 0.f}, chl[4] = {0.f, 0.f, 0.f, 0.f}, clh[4] = {0.f, 0.f, 0.f, 0.f};
    const int n = KT > 0 ? KT : kt_n;
    float4 av = lds4(aa);
    float2 bv = lds2(ba);
#pragma unroll
    for (int kt = 0; kt < n; ++kt) {
        float4 an = av;
        float2 bn = bv;
        if (kt + 1 < n) {
            aa += 512u;
            ba += bstep;
            an = lds4(aa);
            bn = lds2(ba);
        }
        uint32_t ah[4], al[4], bh0, bl0, bh1, bl1;
        split_tf32(av.x, ah[0], al[0]);
        split_tf32(av.y, ah[1], al[1]);
        split_tf32(av.z, ah[2], al[2]);
        split_tf32(av.w, ah[3], al[3]);
        split_tf32(bv.x, bh0, bl0);
        split_tf32(bv.y, bh1, bl1);
        mma_tf32(chh, ah, bh0, bh1);
        mma_tf32(chl, ah, bl0, bl1);
        mma_tf32(clh, al, bh0, bh1);
        av = an;
        bv = bn;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) c[e] = chh[e] + (chl[e] + clh[e]);
}

// tile_product with the k-steps in two halves, each with its own three accumulator chains
// (six in all) summed at the end: the dependent chain of MMAs is half as long.
template <int KT>
__device__ __forceinline__ void tile_product_split(uint32_t aa, uint32_t ba, uint32_t bstep, float (&c)[4]) {
    constexpr int H = (KT + 1) / 2;   // first half: k-steps 0 .. H-1; second: H .. KT-1
    float x0[4] = {0.f, 0.f, 0.f, 0.f}, x1[4] = {0.f, 0.f, 0.f, 0.f}, x2[4] = {0.f, 0.f, 0.f, 0.f};
    float y0[4] = {0.f, 0.f, 0.f, 0.f}, y1[4] = {0.f, 0.f, 0.f, 0.f}, y2[4] = {0.f, 0.f, 0.f, 0.f};
    auto step = [&](int kt, float (&hh)[4], float (&hl)[4], float (&lh)[4]) {
        const float4 av = lds4(aa + 512u * (uint32_t)kt);
        const float2 bv = lds2(ba + bstep * (uint32_t)kt);
        uint32_t ah[4], al[4], bh0, bl0, bh1, bl1;
        split_tf32(av.x, ah[0], al[0]);
        split_tf32(av.y, ah[1], al[1]);
        split_tf32(av.z, ah[2], al[2]);
        split_tf32(av.w, ah[3], al[3]);
        split_tf32(bv.x, bh0, bl0);
        split_tf32(bv.y, bh1, bl1);
        mma_tf32(hh, ah, bh0, bh1);
        mma_tf32(hl, ah, bl0, bl1);
        mma_tf32(lh, al, bh0, bh1);
    };
#pragma unroll
    for (int i = 0; i < H; ++i) {
        step(i, x0, x1, x2);
        if (i + H < KT) step(i + H, y0, y1, y2);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) c[e] = (x0[e] + y0[e]) + ((x1[e] + x2[e]) + (y1[e] + y2[e]));
}

// Per solve step, built once per block: (b | bo << 8, ulev | uo << 16, unused,
// operator offset in floats).
__device__ __forceinline__ int4 solve_step_info(const LevelGeom& lg, int nlev, const int* opoff, const int* u0,
                                                int st) {
    const int dir = st >= nlev, lev = dir ? 2 * nlev - 1 - st : st;
    const int b = lg.size(lev);
    const int lo = dir == 0 ? lev - 1 : lev + 1;
    const int bo = (lo >= 0 && lo < nlev) ? lg.size(lo) : 0;
    return make_int4(b | (bo << 8), u0[lev] | ((bo > 0 ? u0[lo] : 0) << 16), 0, opoff[2 * lev + dir]);
}

// Copies the own rows (b rows from y row u) of a step into B-fragment order at
// k = bo + i.  Element t = threadIdx.x + j * blockDim.x of the b x R block is
// (i0 + j rq + carry, c0 + j rr - carry R): (i0, c0, rq, rr) precomputed per solve.
__device__ __forceinline__ void stage_own(uint32_t y_s, uint32_t stg, int R, int NT, int b, int bo, int u, int i0,
                                          int c0, int rq, int rr) {
    int i = i0, col = c0;
    for (int t = threadIdx.x; t < b * R; t += kThreadsM) {
        sts1(stg + 4u * frag_b_pos(bo + i, col, NT), lds1(y_s + 4u * (uint32_t)((u + i) * R + col)));
        i += rq;
        col += rr;
        if (col >= R) { col -= R; ++i; }
    }
}

__device__ __noinline__ void solve_factor(const MixedArgs& g, const float* F, const int4* sinfo, float* y,
                                          float* opbuf, float* stage, MCtx& c) {
    const int R = g.R, NT = (R + 7) >> 3;
    const int nsteps = 2 * g.nlev;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
    const uint32_t y_s = smem_u32(y), op_s = smem_u32(opbuf), st_s = smem_u32(stage);
    uint32_t ph0 = c.phase[0], ph1 = c.phase[1];
    const int si0 = threadIdx.x / R, sc0 = threadIdx.x - si0 * R, srq = kThreadsM / R, srr = kThreadsM - srq * R;
    uint64_t frozen = 0;
    for (int col = 0; col < R; ++col)
        if (c.col_frozen[col]) frozen |= 1ull << col;
    auto issue = [&](int st) {
        const int4 si = sinfo[st];
        const int b = si.x & 0xff, bo = si.x >> 8;
        const uint32_t bytes = (uint32_t)frag_op_floats(b, b + bo) * 4u;
        fence_proxy_async_shared();
        mbar_arrive_expect_tx(&c.bar[st & 1], bytes);
        bulk_copy_g2s(opbuf + (size_t)(st & 1) * g.opmax, F + si.w, bytes, &c.bar[st & 1]);
    };
    // copies are issued by lane 0 of the last warp, which holds no output tile while
    // a level has at most 7 (16 x 8) tiles
    const bool issuer = threadIdx.x == kThreadsM - 32;
    if (issuer) issue(0);
    // both staging buffers start at zero (padding columns stay zero); step 0's rows
    for (int t = threadIdx.x; t < 2 * g.stage_floats; t += kThreadsM) stage[t] = 0.0f;
    __syncthreads();
    {
        const int4 si = sinfo[0];
        stage_own(y_s, st_s, R, NT, si.x & 0xff, si.x >> 8, si.y & 0xffff, si0, sc0, srq, srr);
    }
    __syncthreads();
    for (int st = 0; st < nsteps; ++st) {
        const int4 si = sinfo[st];
        const int b = si.x & 0xff, bo = si.x >> 8;
        const int ulev = si.y & 0xffff;
        const int K = b + bo, KT = (K + 7) >> 3, MT = (b + 15) >> 4;
        // the other operator buffer was last read in step st-1, which ended with a barrier
        if (issuer && st + 1 < nsteps) issue(st + 1);
        const uint32_t par = (st & 1) ? ph1 : ph0;
        if (!mbar_wait_bounded(&c.bar[st & 1], par)) c.timeout = 1;
        if (st & 1) ph1 ^= 1u; else ph0 ^= 1u;
        const uint32_t op0 = op_s + (uint32_t)((st & 1) * g.opmax) * 4u;
        const uint32_t sb0 = st_s + (uint32_t)((st & 1) * g.stage_floats) * 4u;
        const uint32_t sb1 = st_s + (uint32_t)(((st + 1) & 1) * g.stage_floats) * 4u;
        for (int q = warp; q < MT * NT; q += kWarpsM) {
            const int mt = q / NT, nt = q - mt * NT;
            const uint32_t aa = op0 + (uint32_t)(((mt * KT) * 32 + lane) * 16);
            const uint32_t ba = sb0 + (uint32_t)((nt * 32 + lane) * 8);
            const uint32_t bstep = (uint32_t)(NT * 32 * 8);
            float cv[4];
            switch (KT) {
                case 1: tile_product<1>(aa, ba, bstep, KT, cv); break;
                case 2: tile_product<2>(aa, ba, bstep, KT, cv); break;
                case 3: tile_product<3>(aa, ba, bstep, KT, cv); break;
                case 4: tile_product<4>(aa, ba, bstep, KT, cv); break;
                case 5: tile_product<5>(aa, ba, bstep, KT, cv); break;
                case 6: tile_product<6>(aa, ba, bstep, KT, cv); break;
                case 7: tile_product<7>(aa, ba, bstep, KT, cv); break;
                case 8: tile_product<8>(aa, ba, bstep, KT, cv); break;
                default: tile_product<0>(aa, ba, bstep, KT, cv); break;
            }
            // C tile: rows mt*16 + gq (+8), columns nt*8 + 2 tq (+1).  Result rows go to y
            // (columns still refining) and, as k = i, to the next step's operand.
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i = mt * 16 + gq + 8 * (e >> 1), col = nt * 8 + 2 * tq + (e & 1);
                if (i < b && col < R) {
                    const float v = cv[e];
                    if (!(frozen >> col & 1)) sts1(y_s + 4u * (uint32_t)((ulev + i) * R + col), v);
                    if (st + 1 < nsteps) sts1(sb1 + 4u * frag_b_pos(i, col, NT), v);
                }
            }
        }
        // the next step's own rows (at the turn from forward to backward they are this
        // step's result, already staged above)
        if (st + 1 < nsteps && st + 1 != g.nlev) {
            const int4 sn = sinfo[st + 1];
            stage_own(y_s, sb1, R, NT, sn.x & 0xff, sn.x >> 8, sn.y & 0xffff, si0, sc0, srq, srr);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        c.phase[0] = ph0;
        c.phase[1] = ph1;
    }
}

// ---------------------------------------------------------------------------
// P1 levels of at most 32 unknowns: block LDL^T by level Schur complements.
//
// With s = D^-1/2 (unit diagonal after scaling), level lev couples to the level
// below only through each point's south and south-east edges: C_lev (b_lev x
// b_{lev-1}) has two entries per row.  The scaled matrix factors as
// A = L diag(S_lev) L^T, L_{lev,lev-1} = C_lev T_{lev-1}, T = S^-1, with
//   S_0 = A_00,   S_lev = A_{lev,lev} - C_lev T_{lev-1} C_lev^T,
// so each level needs one sparse update (four entries of T_{lev-1} per entry of
// S_lev) and one dense inverse T_lev, computed by Gauss-Jordan elimination in a
// warp's registers (row p in lane p; SPD: no pivoting).  A solve is then
//   forward   v_lev = T_lev (r_lev - C_lev v_{lev-1})
//   backward  x_lev = v_lev - T_lev (C_{lev+1}^T x_{lev+1})
// one b x b tensor-core product per level step, with T_lev stored once for both
// directions.  Couplings cw (scaled, FP32): [east | west | south | south-east] x nunk.
constexpr int kSchurMax = 32;     // largest level handled by this path
constexpr int kSLd = kSchurMax + 1;

// Row k travels through shared memory (rowbuf: 2 x 32 floats per warp, row k
// published unscaled by lane k); every lane applies a[j] -= g_k r[j] with
// g_k = a_ik / a_kk, or 1 - 1/a_kk in lane k (which turns its row into r / a_kk).
// Pivots go in blocks of 8 with the register row rotated so that the block's pivot columns
// sit at positions 0..7 (the row turns left by 8 after each block): every register index
// stays static with a quarter of the fully unrolled code, and a chunk of 8 columns that
// lies past b is skipped.  Each entry of the inverse sees the same operations in the same
// order as in the unrotated elimination.
__device__ __forceinline__ void gauss_jordan_regs(float (&a)[kSchurMax], float* Tb, float* rowbuf, int b, int lev,
                                                  int* bad) {
    const int lane = threadIdx.x & 31;
    const int nblk = (b + 7) >> 3;
    for (int kb = 0; kb < nblk; ++kb) {
        uint32_t cm = 0;   // chunk m (positions 8m..8m+7) holds columns 8 ((kb + m) mod 4) + 0..7
#pragma unroll
        for (int m = 0; m < kSchurMax / 8; ++m)
            if ((((kb + m) & 3) << 3) < b) cm |= 1u << m;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const int k = kb * 8 + kk;
            if (k < b) {
                float* rb = rowbuf + (k & 1) * kSchurMax;
                if (lane == k) {
#pragma unroll
                    for (int j = 0; j < kSchurMax; j += 4)
                        *reinterpret_cast<float4*>(rb + j) = make_float4(a[j], a[j + 1], a[j + 2], a[j + 3]);
                }
                __syncwarp();
                const float piv = rb[kk];
                if (lane == 0 && !(piv > 0.0f) && *bad == 0) *bad = 1 + lev;
                const float d = __frcp_rn(piv);
                const float gk = lane == k ? 1.0f - d : a[kk] * d;
#pragma unroll
                for (int m = 0; m < kSchurMax / 8; ++m) {
                    if (cm >> m & 1) {
#pragma unroll
                        for (int t = 0; t < 8; t += 4) {
                            const float4 v = *reinterpret_cast<const float4*>(rb + 8 * m + t);
                            a[8 * m + t] = fmaf(-gk, v.x, a[8 * m + t]);
                            a[8 * m + t + 1] = fmaf(-gk, v.y, a[8 * m + t + 1]);
                            a[8 * m + t + 2] = fmaf(-gk, v.z, a[8 * m + t + 2]);
                            a[8 * m + t + 3] = fmaf(-gk, v.w, a[8 * m + t + 3]);
                        }
                    }
                }
                a[kk] = lane == k ? d : -gk;
            }
        }
        float t8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) t8[j] = a[j];
#pragma unroll
        for (int j = 0; j < kSchurMax - 8; ++j) a[j] = a[j + 8];
#pragma unroll
        for (int j = 0; j < 8; ++j) a[kSchurMax - 8 + j] = t8[j];
    }
    // position j now holds column (8 nblk + j) mod 32
#pragma unroll
    for (int j = 0; j < kSchurMax; ++j) Tb[lane * kSLd + ((8 * nblk + j) & (kSchurMax - 1))] = a[j];
}

__device__ __noinline__ void gauss_jordan_warp(const float* Sb, float* Tb, float* rowbuf, int b, int lev, int* bad) {
    const int lane = threadIdx.x & 31;
    float a[kSchurMax];
#pragma unroll
    for (int j = 0; j < kSchurMax; ++j) a[j] = (lane < b && j < b) ? Sb[lane * kSLd + j] : (lane == j ? 1.0f : 0.0f);
    gauss_jordan_regs(a, Tb, rowbuf, b, lev, bad);
}

// One level of the factor kernel in one warp: row p of S_lev (lane p; the same values as
// schur_update, built in registers in chunks of 8 columns, identity past b) and its
// inverse by gauss_jordan_regs, which leaves T_lev in Tb for the next level.
__device__ __noinline__ void schur_level_warp(const float* cwE, const float* cwW, const float* cwS, const float* cwSE,
                                              float* Tb, float* rowbuf, int lev, int b, int ul, int* bad) {
    const int p = threadIdx.x & 31;
    const int off = lev == 1 ? 1 : 0;   // level 0 starts at x = 1 (the pinned point)
    const bool row = p < b;
    const float cps = (row && lev > 0) ? cwS[ul + p] : 0.0f, cpse = (row && lev > 0) ? cwSE[ul + p] : 0.0f;
    const float ce = row ? cwE[ul + p] : 0.0f, cwv = row ? cwW[ul + p] : 0.0f;
    const int ps = p - off, pse = p + 1 - off;
    float a[kSchurMax];
#pragma unroll
    for (int m = 0; m < kSchurMax / 8; ++m) {
        if (8 * m < b) {
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int q = 8 * m + t;
                float sv = p == q ? 1.0f : 0.0f;
                if (row && q < b) {
                    sv = p == q ? 1.0f : (q == p + 1 ? ce : (q == p - 1 ? cwv : 0.0f));
                    if (lev > 0) {
                        const int qs = q - off, qse = q + 1 - off;
                        const float cqs = cwS[ul + q], cqse = cwSE[ul + q];
                        float acc = cpse * Tb[pse * kSLd + qse] * cqse;
                        if (qs >= 0) acc = fmaf(cpse * Tb[pse * kSLd + qs], cqs, acc);
                        if (ps >= 0) {
                            acc = fmaf(cps * Tb[ps * kSLd + qse], cqse, acc);
                            if (qs >= 0) acc = fmaf(cps * Tb[ps * kSLd + qs], cqs, acc);
                        }
                        sv -= acc;
                    }
                }
                a[q] = sv;
            }
        } else {
#pragma unroll
            for (int t = 0; t < 8; ++t) a[8 * m + t] = p == 8 * m + t ? 1.0f : 0.0f;
        }
    }
    __syncwarp();   // every lane has read T_{lev-1} before the elimination overwrites Tb
    gauss_jordan_regs(a, Tb, rowbuf, b, lev, bad);
}

// T (b x b, row-major ld kSLd in shared memory) to global memory in fragment order,
// zero beyond b; tiles are distributed over the warps [w0, w0 + nw) of the caller.
__device__ __forceinline__ void write_frag_op(const float* Tb, int b, float* dst, int w0, int nw) {
    const int KT = (b + 7) >> 3, MT = (b + 15) >> 4, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    for (int tile = warp - w0; tile < MT * KT; tile += nw) {
        const int mt = tile / KT, kt = tile - mt * KT;
        const int i0 = mt * 16 + g, i1 = i0 + 8, k0 = kt * 8 + t, k1 = k0 + 4;
        float4 v;
        v.x = (i0 < b && k0 < b) ? Tb[i0 * kSLd + k0] : 0.0f;
        v.y = (i1 < b && k0 < b) ? Tb[i1 * kSLd + k0] : 0.0f;
        v.z = (i0 < b && k1 < b) ? Tb[i0 * kSLd + k1] : 0.0f;
        v.w = (i1 < b && k1 < b) ? Tb[i1 * kSLd + k1] : 0.0f;
        reinterpret_cast<float4*>(dst)[tile * 32 + lane] = v;
    }
}

// S_lev = A_{lev,lev} - C_lev T_{lev-1} C_lev^T (row-major, ld kSLd): this thread's row
// p (if p < b), columns q0, q0 + qstride, ...
__device__ __forceinline__ void schur_update(const float* cwE, const float* cwW, const float* cwS, const float* cwSE,
                                             const float* Tb, float* Sb, int lev, int b, int ul, int p, int q0,
                                             int qstride) {
    const int off = lev == 1 ? 1 : 0;   // level 0 starts at x = 1 (the pinned point)
    if (p < b) {
        const float cps = lev > 0 ? cwS[ul + p] : 0.0f, cpse = lev > 0 ? cwSE[ul + p] : 0.0f;
        const int ps = p - off, pse = p + 1 - off;
        for (int q = q0; q < b; q += qstride) {
            float sv = p == q ? 1.0f : (q == p + 1 ? cwE[ul + p] : (q == p - 1 ? cwW[ul + p] : 0.0f));
            if (lev > 0) {
                const int qs = q - off, qse = q + 1 - off;
                const float cqs = cwS[ul + q], cqse = cwSE[ul + q];
                float acc = cpse * Tb[pse * kSLd + qse] * cqse;
                if (qs >= 0) acc = fmaf(cpse * Tb[pse * kSLd + qs], cqs, acc);
                if (ps >= 0) {
                    acc = fmaf(cps * Tb[ps * kSLd + qse], cqse, acc);
                    if (qs >= 0) acc = fmaf(cps * Tb[ps * kSLd + qs], cqs, acc);
                }
                sv -= acc;
            }
            Sb[p * kSLd + q] = sv;
        }
    }
}

// Factor pass: T_lev for every level, written to the scratch slot (F + loff[lev]) in
// tensor-core fragment order.  Sb, Tb: kSchurMax x kSLd floats of shared memory.
__device__ __noinline__ void schur_factor(const MixedArgs& g, const int* loff, const int* u0, const float* cw,
                                          float* Sb, float* Tb, float* rowbuf, float* F, MCtx& c) {
    const LevelGeom lg{g.P, g.N, g.PN};
    const int nu = g.nunk;
    for (int lev = 0; lev < g.nlev; ++lev) {
        const int b = lg.size(lev);
        schur_update(cw, cw + nu, cw + 2 * nu, cw + 3 * nu, Tb, Sb, lev, b, u0[lev], threadIdx.x & 31, threadIdx.x >> 5,
                     kWarpsM);
        __syncthreads();
        if (threadIdx.x < 32) gauss_jordan_warp(Sb, Tb, rowbuf, b, lev, &c.bad);
        __syncthreads();
        write_frag_op(Tb, b, F + loff[lev], 0, kWarpsM);   // Tb stays for the next level's update
    }
    fence_proxy_async_global();   // T is read back by bulk copies
    __syncthreads();
}

// Per solve step of this path: (b | dir << 8, ulev | uo << 16, b_other | lev << 16, T offset).
__device__ __forceinline__ int4 schur_step_info(const LevelGeom& lg, int nlev, const int* loff, const int* u0,
                                                int st) {
    const int dir = st >= nlev, lev = dir ? 2 * nlev - 2 - st : st;
    const int lo = dir ? lev + 1 : lev - 1;
    const int bo = (lo >= 0 && lo < nlev) ? lg.size(lo) : 0;
    return make_int4(lg.size(lev) | (dir << 8), u0[lev] | ((bo > 0 ? u0[lo] : 0) << 16), bo | (lev << 16), loff[lev]);
}

// Also returns eps[col] = r^T (L D L^T)^{-1} r = sum over levels of g_lev^T T_lev g_lev,
// accumulated from the forward steps (g_lev is a forward step's staged operand,
// T_lev g_lev its result) in a fixed order.  Needs R <= 32: one output tile per warp,
// warp w at (row tile w / NT, column tile w % NT) at every level.
__device__ __noinline__ void solve_schur(const MixedArgs& g, const float* F, const int4* sinfo, float* y,
                                         const float* cw, const double* Rh, float* opbuf, float* stage, double* eps,
                                         MCtx& c) {
    const int R = g.R, NT = (R + 7) >> 3, nu = g.nunk;
    const int nsteps = 2 * g.nlev - 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
    const uint32_t y_s = smem_u32(y), op_s = smem_u32(opbuf), st_s = smem_u32(stage);
    const float* cwS = cw + 2 * nu;
    const float* cwSE = cw + 3 * nu;
    uint32_t ph = 0;   // bit b: parity of buffer b's next wait
    for (int b = 0; b < kMaxOpBufs; ++b) ph |= (c.phase[b] & 1u) << b;
    uint64_t frozen = 0;
    for (int col = 0; col < R; ++col)
        if (c.col_frozen[col]) frozen |= 1ull << col;
    const int si0 = threadIdx.x / R, sc0 = threadIdx.x - si0 * R, srq = kThreadsM / R, srr = kThreadsM - srq * R;
    const int nb = g.nbuf;   // ring of staged operators: step st uses buffer st % nb
    const uint64_t pol = g.op_policy == 1 ? l2_policy_evict_first() : l2_policy_evict_last();
    auto op_bytes = [&](int st) { return (uint32_t)frag_op_floats(sinfo[st].x & 0xff, sinfo[st].x & 0xff) * 4u; };
    auto issue = [&](int st) {
        const uint32_t bytes = op_bytes(st);
        const int b = st % nb;
        fence_proxy_async_shared();
        mbar_arrive_expect_tx(&c.bar[b], bytes);
        if (g.op_policy) bulk_copy_g2s_hint(opbuf + (size_t)b * g.opmax, F + sinfo[st].w, bytes, &c.bar[b], pol);
        else bulk_copy_g2s(opbuf + (size_t)b * g.opmax, F + sinfo[st].w, bytes, &c.bar[b]);
    };
    // lane 0 of the last warp issues the copies (it holds no output tile while a level has <= 7 tiles)
    const bool issuer = threadIdx.x == kThreadsM - 32;
    if (issuer) {
        if (g.pf_all) {
            // the element's operators (one contiguous array, forward steps in level order)
            const int l = nsteps / 2;   // the last level's step
            bulk_prefetch_l2(F, (uint32_t)(sinfo[l].w * 4u + op_bytes(l)));
        } else {
            for (int st = nb - 1; st < nsteps && st < nb - 1 + g.l2pf; ++st) bulk_prefetch_l2(F + sinfo[st].w, op_bytes(st));
        }
        for (int st = 0; st < nb - 1 && st < nsteps; ++st) issue(st);
    }
    for (int t = threadIdx.x; t < g.stage_floats; t += kThreadsM) stage[t] = 0.0f;   // padding columns stay 0
    // the right-hand side r = FP32 rounding of Rh, in y (frozen columns keep their pending correction);
    // node-major on both sides, so the reads are coalesced and all in flight together
    for (int t = threadIdx.x; t < nu * R; t += kThreadsM) {
        const int col = t % R;
        if (!(frozen >> col & 1)) y[t] = d2f_bits(Rh[t]);
    }
    __syncthreads();
    float eacc0 = 0.0f, eacc1 = 0.0f;   // this lane's two columns (2 tq, 2 tq + 1 of its column tile)
    for (int st = 0; st < nsteps; ++st) {
        const int4 si = sinfo[st];
        const int b = si.x & 0xff, dir = si.x >> 8;
        const int ulev = si.y & 0xffff, uo = si.y >> 16;
        const int bo = si.z & 0xffff, lev = si.z >> 16;
        // buffer (st + nb - 1) % nb was last read in step st - 1, which ended with a barrier
        if (issuer && st + nb - 1 < nsteps) issue(st + nb - 1);
        if (issuer && g.l2pf && !g.pf_all && st + nb - 1 + g.l2pf < nsteps) {
            const int sp = st + nb - 1 + g.l2pf;
            bulk_prefetch_l2(F + sinfo[sp].w, op_bytes(sp));
        }
        // B (b x R) in fragment order: forward r_lev - C_lev v_{lev-1} (r = the FP32 rounding of
        // the scaled residual Rh); backward C_{lev+1}^T x_{lev+1}
        {
            const int xo = lev == 0 ? 1 : 0;       // lattice x of position 0
            const int off = lev == 1 ? 1 : 0;      // level below starts at x = 1
            int i = si0, col = sc0;
            for (int t = threadIdx.x; t < b * R; t += kThreadsM) {
                const int x = i + xo;
                float v;
                if (dir == 0) {
                    v = lds1(y_s + 4u * (uint32_t)((ulev + i) * R + col));   // right-hand side
                    if (lev > 0) {
                        const int ps = x - off, pse = x + 1 - off;
                        float a = cwSE[ulev + i] * lds1(y_s + 4u * (uint32_t)((uo + pse) * R + col));
                        if (ps >= 0) a = fmaf(cwS[ulev + i], lds1(y_s + 4u * (uint32_t)((uo + ps) * R + col)), a);
                        v -= a;
                    }
                } else {
                    v = 0.0f;
                    if (x < bo) v = cwS[uo + x] * lds1(y_s + 4u * (uint32_t)((uo + x) * R + col));
                    if (x >= 1) v = fmaf(cwSE[uo + x - 1], lds1(y_s + 4u * (uint32_t)((uo + x - 1) * R + col)), v);
                }
                sts1(st_s + 4u * frag_b_pos(i, col, NT), v);
                i += srq;
                col += srr;
                if (col >= R) { col -= R; ++i; }
            }
        }
        const int bu = st % nb;
        if (!mbar_wait_bounded(&c.bar[bu], (ph >> bu) & 1u)) c.timeout = 1;
        ph ^= 1u << bu;
        __syncthreads();
        const int KT = (b + 7) >> 3, MT = (b + 15) >> 4;
        const uint32_t op0 = op_s + (uint32_t)(bu * g.opmax) * 4u;
        for (int q = warp; q < MT * NT; q += kWarpsM) {
            const int mt = q / NT, nt = q - mt * NT;
            const uint32_t aa = op0 + (uint32_t)(((mt * KT) * 32 + lane) * 16);
            const uint32_t ba = st_s + (uint32_t)((nt * 32 + lane) * 8);
            const uint32_t bstep = (uint32_t)(NT * 32 * 8);
            float cv[4];
            switch (KT) {
                case 1: tile_product<1>(aa, ba, bstep, KT, cv); break;
                case 2: tile_product_split<2>(aa, ba, bstep, cv); break;
                case 3: tile_product_split<3>(aa, ba, bstep, cv); break;
                default: tile_product_split<4>(aa, ba, bstep, cv); break;
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i = mt * 16 + gq + 8 * (e >> 1), col = nt * 8 + 2 * tq + (e & 1);
                if (i < b && col < R) {
                    if (dir == 0) {
                        const float gv = lds1(st_s + 4u * frag_b_pos(i, col, NT)) * cv[e];
                        if (e & 1) eacc1 += gv; else eacc0 += gv;
                    }
                    if (!(frozen >> col & 1)) {
                        const uint32_t ya = y_s + 4u * (uint32_t)((ulev + i) * R + col);
                        sts1(ya, dir == 0 ? cv[e] : lds1(ya) - cv[e]);
                    }
                }
            }
        }
        __syncthreads();
    }
    // eps: sum over the 8 row lanes of each column (lanes with equal tq), then the two row tiles
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
        eacc0 += __shfl_xor_sync(0xffffffffu, eacc0, o);
        eacc1 += __shfl_xor_sync(0xffffffffu, eacc1, o);
    }
    if (warp < 2 * NT && gq == 0) {
        c.epsred[warp / NT][(warp % NT) * 8 + 2 * tq] = eacc0;
        c.epsred[warp / NT][(warp % NT) * 8 + 2 * tq + 1] = eacc1;
    }
    __syncthreads();
    if (threadIdx.x < R) eps[threadIdx.x] = (double)c.epsred[0][threadIdx.x] + (double)c.epsred[1][threadIdx.x];
    if (threadIdx.x == 0)
        for (int b = 0; b < kMaxOpBufs; ++b) c.phase[b] = (ph >> b) & 1u;
}

// The same solve with the column tiles decoupled (R <= 24: at most 3 tiles of 8
// columns).  A column of the solve depends only on the same column at the other levels, so
// each column tile runs its own chain of level steps in its own pair of warps (one per
// 16-row tile), synchronised by a named barrier of those 64 threads instead of the whole
// block; the groups drift against each other and hide one another's latencies.  The level
// operators they share stream through the ring fed by a producer (lane 0 of the last warp,
// which holds no tile): slot s mod nbuf is refilled once every group has released its step
// s - nbuf (an mbarrier with one arrival per group).
__device__ __forceinline__ void group_sync(int id) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(64) : "memory");
}

__device__ __noinline__ void solve_schur_groups(const MixedArgs& g, const float* F, const int4* sinfo, float* y,
                                                const float* cw, const double* Rh, float* opbuf, float* stage,
                                                double* eps, MCtx& c) {
    const int R = g.R, NT = (R + 7) >> 3, nu = g.nunk;
    const int nsteps = 2 * g.nlev - 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
    const int grp = warp >> 1, mt = warp & 1;          // column tile and row tile of this warp
    const uint32_t y_s = smem_u32(y), op_s = smem_u32(opbuf), st_s = smem_u32(stage);
    const float* cwS = cw + 2 * nu;
    const float* cwSE = cw + 3 * nu;
    const int nb = g.nbuf;
    uint32_t fph = 0, eph = 0;   // bit b: parity of slot b's full / empty barrier at the solve's start
    for (int b = 0; b < kMaxOpBufs; ++b) {
        fph |= (c.phase[b] & 1u) << b;
        eph |= (c.ephase[b] & 1u) << b;
    }
    uint64_t frozen = 0;
    for (int col = 0; col < R; ++col)
        if (c.col_frozen[col]) frozen |= 1ull << col;
    const uint64_t pol = g.op_policy == 1 ? l2_policy_evict_first() : l2_policy_evict_last();
    auto op_bytes = [&](int st) { return (uint32_t)frag_op_floats(sinfo[st].x & 0xff, sinfo[st].x & 0xff) * 4u; };
    for (int t = threadIdx.x; t < g.stage_floats; t += kThreadsM) stage[t] = 0.0f;   // padding columns stay 0
    for (int t = threadIdx.x; t < nu * R; t += kThreadsM) {
        const int col = t % R;
        if (!(frozen >> col & 1)) y[t] = d2f_bits(Rh[t]);
    }
    __syncthreads();
    float eacc0 = 0.0f, eacc1 = 0.0f;
    if (warp == kWarpsM - 1) {
        if (lane == 0) {
            // producer: the operator of every step into its slot, after the slot's last use
            if (g.pf_all) {
                const int l = nsteps / 2;
                bulk_prefetch_l2(F, (uint32_t)(sinfo[l].w * 4u + op_bytes(l)));
            }
            for (int st = 0; st < nsteps; ++st) {
                const int b = st % nb;
                if (st >= nb) {
                    const uint32_t k = (uint32_t)((st - nb) / nb);   // that use's index in this solve
                    if (!mbar_wait_bounded(&c.ebar[b], ((eph >> b) ^ k) & 1u)) c.timeout = 1;
                }
                if (g.l2pf && !g.pf_all && st + g.l2pf < nsteps)
                    bulk_prefetch_l2(F + sinfo[st + g.l2pf].w, op_bytes(st + g.l2pf));
                const uint32_t bytes = op_bytes(st);
                fence_proxy_async_shared();
                mbar_arrive_expect_tx(&c.bar[b], bytes);
                if (g.op_policy) bulk_copy_g2s_hint(opbuf + (size_t)b * g.opmax, F + sinfo[st].w, bytes, &c.bar[b], pol);
                else bulk_copy_g2s(opbuf + (size_t)b * g.opmax, F + sinfo[st].w, bytes, &c.bar[b]);
            }
        }
    } else if (grp < NT) {
        const int t64 = threadIdx.x & 63, c8 = t64 & 7, i0 = t64 >> 3;
        const int col = grp * 8 + c8;
        for (int st = 0; st < nsteps; ++st) {
            const int4 si = sinfo[st];
            const int b = si.x & 0xff, dir = si.x >> 8;
            const int ulev = si.y & 0xffff, uo = si.y >> 16;
            const int bo = si.z & 0xffff, lev = si.z >> 16;
            // this tile's columns of B (b x 8): forward r_lev - C_lev v_{lev-1}, backward
            // C_{lev+1}^T x_{lev+1}
            if (col < R) {
                const int xo = lev == 0 ? 1 : 0;       // lattice x of position 0
                const int off = lev == 1 ? 1 : 0;      // level below starts at x = 1
                for (int i = i0; i < b; i += 8) {
                    const int x = i + xo;
                    float v;
                    if (dir == 0) {
                        v = lds1(y_s + 4u * (uint32_t)((ulev + i) * R + col));
                        if (lev > 0) {
                            const int ps = x - off, pse = x + 1 - off;
                            float a = cwSE[ulev + i] * lds1(y_s + 4u * (uint32_t)((uo + pse) * R + col));
                            if (ps >= 0) a = fmaf(cwS[ulev + i], lds1(y_s + 4u * (uint32_t)((uo + ps) * R + col)), a);
                            v -= a;
                        }
                    } else {
                        v = 0.0f;
                        if (x < bo) v = cwS[uo + x] * lds1(y_s + 4u * (uint32_t)((uo + x) * R + col));
                        if (x >= 1) v = fmaf(cwSE[uo + x - 1], lds1(y_s + 4u * (uint32_t)((uo + x - 1) * R + col)), v);
                    }
                    sts1(st_s + 4u * frag_b_pos(i, col, NT), v);
                }
            }
            const int bu = st % nb;
            const uint32_t k = (uint32_t)(st / nb);   // use of slot bu in this solve
            if (!mbar_wait_bounded(&c.bar[bu], ((fph >> bu) ^ k) & 1u)) c.timeout = 1;
            group_sync(1 + grp);
            const int KT = (b + 7) >> 3, MT = (b + 15) >> 4;
            if (mt < MT) {
                const uint32_t op0 = op_s + (uint32_t)(bu * g.opmax) * 4u;
                const uint32_t aa = op0 + (uint32_t)(((mt * KT) * 32 + lane) * 16);
                const uint32_t ba = st_s + (uint32_t)((grp * 32 + lane) * 8);
                const uint32_t bstep = (uint32_t)(NT * 32 * 8);
                float cv[4];
                switch (KT) {
                    case 1: tile_product<1>(aa, ba, bstep, KT, cv); break;
                    case 2: tile_product_split<2>(aa, ba, bstep, cv); break;
                    case 3: tile_product_split<3>(aa, ba, bstep, cv); break;
                    default: tile_product_split<4>(aa, ba, bstep, cv); break;
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int i = mt * 16 + gq + 8 * (e >> 1), cc = grp * 8 + 2 * tq + (e & 1);
                    if (i < b && cc < R) {
                        if (dir == 0) {
                            const float gv = lds1(st_s + 4u * frag_b_pos(i, cc, NT)) * cv[e];
                            if (e & 1) eacc1 += gv; else eacc0 += gv;
                        }
                        if (!(frozen >> cc & 1)) {
                            const uint32_t ya = y_s + 4u * (uint32_t)((ulev + i) * R + cc);
                            sts1(ya, dir == 0 ? cv[e] : lds1(ya) - cv[e]);
                        }
                    }
                }
            }
            group_sync(1 + grp);
            if (t64 == 0) mbar_arrive(&c.ebar[bu]);   // this group is done with the slot
        }
    }
    // eps: sum over the 8 row lanes of each column (lanes with equal tq), then the two row tiles
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
        eacc0 += __shfl_xor_sync(0xffffffffu, eacc0, o);
        eacc1 += __shfl_xor_sync(0xffffffffu, eacc1, o);
    }
    if (grp < NT && warp < kWarpsM - 1 && gq == 0) {
        c.epsred[mt][grp * 8 + 2 * tq] = eacc0;
        c.epsred[mt][grp * 8 + 2 * tq + 1] = eacc1;
    }
    __syncthreads();
    if (threadIdx.x < R) eps[threadIdx.x] = (double)c.epsred[0][threadIdx.x] + (double)c.epsred[1][threadIdx.x];
    if (threadIdx.x == 0)
        for (int b = 0; b < kMaxOpBufs; ++b) {
            const uint32_t uses = b < nb ? (uint32_t)((nsteps - b + nb - 1) / nb) : 0u;
            c.phase[b] = ((fph >> b) ^ uses) & 1u;
            c.ephase[b] = ((eph >> b) ^ uses) & 1u;
        }
}

// One refinement pass of the level-Schur path, in scaled variables, for the columns
// not done: Zh_u += y_u and Rh_u -= sum_v Ah_uv y_v over the stencil points v of u,
// accumulated in FP64 (y widened on the integer pipe).  A node's entries are read 8
// columns at a time before they are used, so that their loads are in flight
// together.  Thread per node; `done` has bit col set for the columns to skip.
__device__ __noinline__ void fused_residual(int PN, int nu, int R, const double* __restrict__ ah, const float* y,
                                            double* __restrict__ Zh, double* __restrict__ Rh, uint64_t done,
                                            const uint32_t* rmask) {
    const uint32_t y_s = smem_u32(y);
    for (int u = threadIdx.x, rnd = 0; u < nu; u += kThreadsM, ++rnd) {
        int X, Y;
        lattice_of_unk(PN, u, &X, &Y);
        int v[7];
        v[0] = u;
        v[1] = unk(PN, X + 1, Y);
        v[2] = unk(PN, X - 1, Y);
        v[3] = unk(PN, X, Y + 1);
        v[4] = unk(PN, X, Y - 1);
        v[5] = unk(PN, X + 1, Y - 1);
        v[6] = unk(PN, X - 1, Y + 1);
        double a[7];
        uint32_t nz = 0;   // stencil points with a non-zero weight, tested once per node on the
                           // integer pipe (a double comparison would occupy the FP64 pipe)
#pragma unroll
        for (int d = 0; d < 7; ++d) {
            a[d] = ah[(size_t)d * nu + u];
            if (v[d] < 0 || v[d] >= nu) { a[d] = 0.0; v[d] = u; }   // (weight zero there)
            if ((__double_as_longlong(a[d]) << 1) != 0) nz |= 1u << d;   // a[d] != 0 (either zero sign)
        }
        // directions that no node of this warp's row set needs (the fine triangles' right
        // angles give zero weights): skipped by a warp-uniform branch
        const uint32_t any = rmask[rnd * kWarpsM + (threadIdx.x >> 5)];
        for (int c0 = 0; c0 < R; c0 += 8) {
            double zr[8], rr[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int col = c0 + j;
                const bool on = col < R && !(done >> col & 1);
                zr[j] = on ? Zh[(size_t)u * R + col] : 0.0;
                rr[j] = on ? Rh[(size_t)u * R + col] : 0.0;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int col = c0 + j;
                if (col < R && !(done >> col & 1)) {
                    const double d0 = f2d_bits(lds1(y_s + 4u * (uint32_t)(u * R + col)));
                    Zh[(size_t)u * R + col] = zr[j] + d0;
                    double r = fma(-a[0], d0, rr[j]);
#pragma unroll
                    for (int d = 1; d < 7; ++d)
                        if (any >> d & 1) {
                            if (nz >> d & 1) r = fma(-a[d], f2d_bits(lds1(y_s + 4u * (uint32_t)(v[d] * R + col))), r);
                        }
                    Rh[(size_t)u * R + col] = r;
                }
            }
        }
    }
}

// The level factorisation, the solves and the column dots run out of line: each
// then keeps its working set (register panel, accumulator tiles) in registers
// instead of sharing the kernel's register budget with the per-K state live
// around it.
template <int RPL, int CPL>
__device__ __noinline__ void cholesky_level_f32(float* M, int ld, int b, int nr, float* Rhs, int ldr, int rhs_rows,
                                                int ncols, int* bad) {
    blocked_cholesky_level<float, 8, RPL, CPL>(M, ld, b, nr, Rhs, ldr, rhs_rows, ncols, bad);
}

// ---------------------------------------------------------------------------
// Generic levels (P2: two lattice rows per level, at most 64 unknowns; P1 with more
// right-hand sides than the P1 level-Schur solve takes): the block LDL^T of Ah = S A_p S
// by levels, as on the P1 path, factored by k_schur_factor_gen.  Only a level's first
// lattice row couples to the level below (a P2 fine row's triangles span lattice rows
// 2j..2j+2), and the couplings come from the assembled rows, kept as tables:
//   forward   v_lev = T_lev (r_lev - C_lev v_{lev-1})
//   backward  x_lev = v_lev - T_lev (C_{lev+1}^T x_{lev+1})
// An element's operator block: T_lev of every level in fragment order, then per level
// lev >= 1 the forward table (kTabQ entries per first-row node of lev: its couplings into
// lev - 1), then per level lev <= nlev - 2 the backward table (kTabF entries per node of
// lev: its couplings into lev + 1); an entry is two floats, the position in the other
// level (int bits; -1: none) and the scaled FP32 weight.
constexpr int kGenMax = 64;            // largest level of this path
constexpr int kGenRow = 32;            // largest first lattice row of a level
constexpr int kTabF = 4;               // couplings of a node into the level above it
constexpr int kTabQ = 8;               // couplings of a first-row node into the level below it

// Number of unknowns in the first lattice row of level lev (the pinned DOF 0 excluded).
__device__ __forceinline__ int first_row_size(const LevelGeom& lg, int lev) {
    if (lg.P == 1 || lev == lg.N) return lg.size(lev);
    return lg.PN - 2 * lev + 1 - (lev == 0);
}

// Offsets (floats) of level lev's T, forward table and backward table in the operator block.
__device__ inline void gen_offsets(const LevelGeom& lg, int nlev, int lev, int* t_off, int* f_off, int* b_off) {
    int t = 0, tl = 0, fl = 0, bl = 0, fsum = 0, bsum = 0;
    for (int l = 0; l < nlev; ++l) {
        const int b = lg.size(l);
        if (l == lev) { tl = t; fl = fsum; bl = bsum; }
        t += frag_op_floats(b, b);
        if (l >= 1) fsum += 2 * kTabQ * first_row_size(lg, l);
        if (l + 1 < nlev) bsum += 2 * kTabF * b;
    }
    *t_off = tl;
    *f_off = t + fl;
    *b_off = t + fsum + bl;
}

// Per solve step: (b | dir << 8 | l0 << 16, ulev | uo << 16, table offset, T offset); l0 is
// the forward step's first-row size (0 at level 0), uo the first unknown of the other level.
__device__ inline int4 gen_step_info(const LevelGeom& lg, int nlev, const int* u0, int st) {
    const int dir = st >= nlev, lev = dir ? 2 * nlev - 2 - st : st;
    int t_off, f_off, b_off;
    gen_offsets(lg, nlev, lev, &t_off, &f_off, &b_off);
    const int b = lg.size(lev);
    if (!dir) {
        const int l0 = lev > 0 ? first_row_size(lg, lev) : 0;
        return make_int4(b | (l0 << 16), u0[lev] | ((lev > 0 ? u0[lev - 1] : 0) << 16), lev > 0 ? f_off : 0, t_off);
    }
    return make_int4(b | (1 << 8), u0[lev] | (u0[lev + 1] << 16), b_off, t_off);
}

// Forward + backward solve of the generic path for every column still refining, in place
// in y (node-major: y[u * R + col]): per level step the operand is staged from y through
// the coupling tables, then one b x b by b x R product with T_lev on the tensor cores
// (three-term TF32 split, as in solve_factor); T_lev streams into two shared-memory
// buffers by bulk copies, one step ahead.
__device__ __noinline__ void solve_gen(const MixedArgs& g, const float* F, const int4* sinfo, float* y,
                                       float* opbuf, float* stage, MCtx& c) {
    const int R = g.R, NT = (R + 7) >> 3;
    const int nsteps = 2 * g.nlev - 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
    const uint32_t y_s = smem_u32(y), op_s = smem_u32(opbuf), st_s = smem_u32(stage);
    uint32_t ph0 = c.phase[0], ph1 = c.phase[1];
    const int si0 = threadIdx.x / R, sc0 = threadIdx.x - si0 * R, srq = kThreadsM / R, srr = kThreadsM - srq * R;
    uint64_t frozen = 0;
    for (int col = 0; col < R; ++col)
        if (c.col_frozen[col]) frozen |= 1ull << col;
    auto issue = [&](int st) {
        const int4 si = sinfo[st];
        const int b = si.x & 0xff;
        const uint32_t bytes = (uint32_t)frag_op_floats(b, b) * 4u;
        fence_proxy_async_shared();
        mbar_arrive_expect_tx(&c.bar[st & 1], bytes);
        bulk_copy_g2s(opbuf + (size_t)(st & 1) * g.opmax, F + si.w, bytes, &c.bar[st & 1]);
    };
    const bool issuer = threadIdx.x == kThreadsM - 32;
    if (issuer) issue(0);
    for (int t = threadIdx.x; t < g.stage_floats; t += kThreadsM) stage[t] = 0.0f;   // padding stays 0
    __syncthreads();
    for (int st = 0; st < nsteps; ++st) {
        const int4 si = sinfo[st];
        const int b = si.x & 0xff, dir = (si.x >> 8) & 1, l0 = si.x >> 16;
        const int ulev = si.y & 0xffff, uo = si.y >> 16;
        const float2* tab = reinterpret_cast<const float2*>(F + si.z);
        // the other buffer was last read in step st - 1, which ended with a barrier
        if (issuer && st + 1 < nsteps) issue(st + 1);
        // operand (b x R, fragment order): forward r_lev - C_lev v_{lev-1}, backward
        // C_{lev+1}^T x_{lev+1}
        {
            int i = si0, col = sc0;
            for (int t = threadIdx.x; t < b * R; t += kThreadsM) {
                float v = 0.0f;
                if (dir == 0) {
                    v = lds1(y_s + 4u * (uint32_t)((ulev + i) * R + col));
                    if (i < l0) {
#pragma unroll
                        for (int m = 0; m < kTabQ; ++m) {
                            const float2 e = tab[i * kTabQ + m];
                            const int pos = __float_as_int(e.x);
                            if (pos >= 0) v = fmaf(-e.y, lds1(y_s + 4u * (uint32_t)((uo + pos) * R + col)), v);
                        }
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < kTabF; ++m) {
                        const float2 e = tab[i * kTabF + m];
                        const int pos = __float_as_int(e.x);
                        if (pos >= 0) v = fmaf(e.y, lds1(y_s + 4u * (uint32_t)((uo + pos) * R + col)), v);
                    }
                }
                sts1(st_s + 4u * frag_b_pos(i, col, NT), v);
                i += srq;
                col += srr;
                if (col >= R) { col -= R; ++i; }
            }
        }
        const uint32_t par = (st & 1) ? ph1 : ph0;
        if (!mbar_wait_bounded(&c.bar[st & 1], par)) c.timeout = 1;
        if (st & 1) ph1 ^= 1u; else ph0 ^= 1u;
        __syncthreads();
        const int KT = (b + 7) >> 3, MT = (b + 15) >> 4;
        const uint32_t op0 = op_s + (uint32_t)((st & 1) * g.opmax) * 4u;
        for (int q = warp; q < MT * NT; q += kWarpsM) {
            const int mt = q / NT, nt = q - mt * NT;
            const uint32_t aa = op0 + (uint32_t)(((mt * KT) * 32 + lane) * 16);
            const uint32_t ba = st_s + (uint32_t)((nt * 32 + lane) * 8);
            const uint32_t bstep = (uint32_t)(NT * 32 * 8);
            float cv[4];
            switch (KT) {
                case 1: tile_product<1>(aa, ba, bstep, KT, cv); break;
                case 2: tile_product_split<2>(aa, ba, bstep, cv); break;
                case 3: tile_product_split<3>(aa, ba, bstep, cv); break;
                case 4: tile_product_split<4>(aa, ba, bstep, cv); break;
                case 5: tile_product_split<5>(aa, ba, bstep, cv); break;
                case 6: tile_product_split<6>(aa, ba, bstep, cv); break;
                case 7: tile_product_split<7>(aa, ba, bstep, cv); break;
                default: tile_product_split<8>(aa, ba, bstep, cv); break;
            }
            // forward: y_lev = result; backward: y_lev -= result (columns still refining)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i = mt * 16 + gq + 8 * (e >> 1), col = nt * 8 + 2 * tq + (e & 1);
                if (i < b && col < R && !(frozen >> col & 1)) {
                    const uint32_t ya = y_s + 4u * (uint32_t)((ulev + i) * R + col);
                    sts1(ya, dir == 0 ? cv[e] : lds1(ya) - cv[e]);
                }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        c.phase[0] = ph0;
        c.phase[1] = ph1;
    }
}

// MODE 0: generic level operators (Cholesky) factored in this kernel; 1: level Schur
// complements factored in this kernel; 2: level Schur operators precomputed by
// k_schur_factor; 3: generic level operators precomputed by k_schur_factor_gen.
// The blocks of the launch take the coarse elements of one level (g) from its queue.
template <int RPL, int CPL, int MODE>
__device__ __forceinline__ void mixed_blocks(const MixedArgs& g) {
    constexpr bool SCHUR = MODE == 1 || MODE == 2;
    extern __shared__ unsigned char smem_raw[];
    float* W = reinterpret_cast<float*>(smem_raw);                    // FP32 window
    float* y = W + (size_t)g.wfloats;                                    // nunk x R
    int* loff = reinterpret_cast<int*>(y + (size_t)g.yfloats);         // 2 nlev operator offsets (Fw, Bw)
    int* u0 = loff + 2 * g.nlev;                                        // nlev + 1 level starts
    int4* sinfo = reinterpret_cast<int4*>(smem_raw + g.off_sinfo);      // 2 nlev solve steps
    double* kap_s = reinterpret_cast<double*>(smem_raw + g.off_kap_smem);   // kappa of the current K (if staged)
    double* scale = reinterpret_cast<double*>(g.ws + (size_t)blockIdx.x * g.slot_bytes + g.off_scale);   // 1/sqrt(diag A_p)
    float* opbuf = W;                                                   // nbuf x opmax staging (solves only)
    float* stage = W + (size_t)(SCHUR ? g.nbuf : 2) * g.opmax;          // staged solve operand(s) (solves only)
    float* cw = reinterpret_cast<float*>(smem_raw + g.off_cw);          // level-Schur path: 4 x nunk couplings
    __shared__ MCtx c;
    const LevelGeom lg{g.P, g.N, g.PN};
    const int R = g.R;
    char* slot = g.ws + (size_t)blockIdx.x * g.slot_bytes;
    float* F = reinterpret_cast<float*>(slot);   // level operators (MODE 2: per K, set below)
    double* G = reinterpret_cast<double*>(slot + g.off_G);
    double* Z = reinterpret_cast<double*>(slot + g.off_Z);
    double* mass = reinterpret_cast<double*>(slot + g.off_mass);

    if (threadIdx.x == 0) {
        int o = 0, u = 0;
        for (int lev = 0; lev < g.nlev; ++lev) {
            const int b = lg.size(lev), bn = lev + 1 < g.nlev ? lg.size(lev + 1) : 0;
            const int bp = lev > 0 ? lg.size(lev - 1) : 0;
            if (SCHUR) {
                loff[lev] = o;                       // T_lev in fragment order
                o += frag_op_floats(b, b);
            } else {
                loff[2 * lev] = o;                   // operators in fragment order (16-byte aligned)
                o += frag_op_floats(b, b + bp);
                loff[2 * lev + 1] = o;
                o += frag_op_floats(b, b + bn);
            }
            u0[lev] = u;
            u += b;
        }
        u0[g.nlev] = u;
        if (SCHUR)
            for (int st = 0; st < 2 * g.nlev - 1; ++st) sinfo[st] = schur_step_info(lg, g.nlev, loff, u0, st);
        else if (MODE == 3)
            for (int st = 0; st < 2 * g.nlev - 1; ++st) sinfo[st] = gen_step_info(lg, g.nlev, u0, st);
        else
            for (int st = 0; st < 2 * g.nlev; ++st) sinfo[st] = solve_step_info(lg, g.nlev, loff, u0, st);
        for (int b = 0; b < kMaxOpBufs; ++b) {
            mbar_init(&c.bar[b], 1);
            c.phase[b] = 0;
            mbar_init(&c.ebar[b], (g.R + 7) >> 3);   // one release per column group
            c.ephase[b] = 0;
        }
    }
    __syncthreads();

    // coarse triangles: K0 + blockIdx.x, then (dynamic) the next index from the counter
    // or (static) every gridDim.x-th
    if (threadIdx.x == 0) c.nextK = g.kcounter ? g.K0 + gridDim.x + atomicAdd(g.kcounter, 1) : 0;
    for (int64_t ki = g.K0 + blockIdx.x; ki < g.K1;) {                  // launch index within the level
        const int64_t K = g.dm.klist ? (int64_t)g.dm.klist[ki] : ki;      // coarse element
        const double* kap = g.kappa + (g.dm.kap_off ? g.dm.kap_off[K] : K * (int64_t)g.N * g.N);
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
                c.la1[a] = face_la1(g.dm, K, a);
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
                s += cell_src(g, X, g.P, -1, quad_of(g.src_vals, g.kappa, kap, g.N, up, up ? o : o - (g.N - j), j));
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
                const int row = face_row(jf, c.la1[a], g.dm.fm, g.dm.lmax1);
                c.cproj[col] = row < 0 ? 0.0 : -c.sgn[a] * c.flen[a] * g.dm.btab_sum[row] / c.area;
            }
        }
        __syncthreads();

        if constexpr (SCHUR) {
            // ---- Level-Schur path in scaled variables (node-major, index u R + col):
            //   Zh = S^-1 Z, Rh = S (G - A Z), Ah = S A S, S = diag(A_uu^-1/2).
            // A correction is Zh += y (the FP32 solve output, exactly), the residual update
            // Rh -= Ah y reads y at the stencil points, and z_j^T Res_i = Zh_j^T Rh_i.
            double* Rh = G;
            double* Zh = Z;
            double* smass = mass;   // s_u m_u
            const double* sc;
            const double* ah;       // 7 x nunk: self, E, W, N, S, SE, NW
            const int nu = g.nunk;
            if constexpr (MODE == 2) {
                __syncthreads();
                const int64_t kk = ki - g.Kbase;
                F = g.Tall + kk * (int64_t)g.t_stride;
                sc = g.scall + kk * (int64_t)nu;
                ah = g.ahall + kk * 7 * (int64_t)nu;
                cw = g.cwall + kk * 4 * (int64_t)nu;   // read in place (L1), no shared copy
                if (threadIdx.x == 0) c.bad = g.fbad[kk];
            } else {
                double* ahw = reinterpret_cast<double*>(slot + g.off_D);
                for (int u = threadIdx.x; u < nu; u += blockDim.x) {
                    int X, Y;
                    lattice_of_unk(g.PN, u, &X, &Y);
                    double w[7];
                    int v[7];
                    p1_row(g.N, g.PN, nu, c.Sup, c.Sdn, kap, X, Y, u, w, v);
                    scale[u] = 1.0 / sqrt(w[0]);
                }
                __syncthreads();
                for (int u = threadIdx.x; u < nu; u += blockDim.x) {
                    int X, Y;
                    lattice_of_unk(g.PN, u, &X, &Y);
                    double w[7];
                    int v[7];
                    p1_row(g.N, g.PN, nu, c.Sup, c.Sdn, kap, X, Y, u, w, v);
                    const double su = scale[u];
                    double a7[7];
                    for (int d = 0; d < 7; ++d) a7[d] = w[d] * su * scale[v[d]];
                    cw[u] = (float)a7[1];
                    cw[nu + u] = (float)a7[2];
                    cw[2 * nu + u] = (float)a7[4];
                    cw[3 * nu + u] = (float)a7[5];
                    for (int d = 0; d < 7; ++d) ahw[(size_t)d * nu + u] = a7[d];
                }
                __syncthreads();
                schur_factor(g, loff, u0, cw, W, W + kSchurMax * kSLd, W + 2 * kSchurMax * kSLd, F, c);
                sc = scale;
                ah = ahw;
            }
            // per warp and round of the residual's node loop: the stencil directions with a
            // non-zero weight at some node
            for (int ub = 0, rnd = 0; ub < nu; ub += kThreadsM, ++rnd) {
                const int u = ub + threadIdx.x;
                uint32_t nz = 0;
                if (u < nu) {
                    int X, Y;
                    lattice_of_unk(g.PN, u, &X, &Y);
                    const int vv[7] = {u, unk(g.PN, X + 1, Y), unk(g.PN, X - 1, Y), unk(g.PN, X, Y + 1),
                                       unk(g.PN, X, Y - 1), unk(g.PN, X + 1, Y - 1), unk(g.PN, X - 1, Y + 1)};
#pragma unroll
                    for (int d = 0; d < 7; ++d)
                        if (vv[d] >= 0 && vv[d] < nu && !is_zero(ah[(size_t)d * nu + u])) nz |= 1u << d;
                }
                nz = __reduce_or_sync(0xffffffffu, nz);
                if ((threadIdx.x & 31) == 0) c.rmask[rnd][threadIdx.x >> 5] = nz;
            }
            // ---- right-hand sides Rh = S G (compatible loads, pinned DOF left out), S m, Zh = 0
            for (int u = threadIdx.x; u < nu; u += blockDim.x) {
                int X, Y;
                lattice_of_unk(g.PN, u, &X, &Y);
                int ti[6], tj[6], ta[6];
                bool tup[6];
                const int n = incident(1, g.N, X, Y, ti, tj, tup, ta);
                double m = 0.0, fh = 0.0;
                for (int t = 0; t < n; ++t) {
                    const double mt = c.area_fine * element_mass_frac(1, ta[t]);
                    m += mt;
                    if (g.src_kind == MHM_SRC_CONST) fh += g.src_value * mt;
                    else {
                        double Xv[3][2];
                        fine_xy(c, g.N, tup[t], ti[t], tj[t], Xv);
                        fh += cell_src(g, Xv, 1, ta[t], quad_of(g.src_vals, g.kappa, kap, g.N, tup[t], ti[t], tj[t]));
                    }
                }
                const double su = sc[u];
                smass[u] = su * m;
                for (int col = 0; col < R; ++col) {
                    double v = -c.cproj[col] * m;
                    if (col == g.NI) v += fh;
                    else {
                        const int a = col / g.dpf, jf = col - a * g.dpf;
                        const int kl = face_position(g.PN, X, Y, a);
                        const int row = face_row(jf, c.la1[a], g.dm.fm, g.dm.lmax1);
                        if (kl >= 0 && row >= 0) {
                            const int kk2 = c.rev[a] ? g.PN - kl : kl;
                            v += -c.sgn[a] * c.flen[a] * g.dm.btab[row * (g.PN + 1) + kk2];
                        }
                    }
                    Rh[(size_t)u * R + col] = su * v;
                    Zh[(size_t)u * R + col] = 0.0;
                }
            }
            __syncthreads();
            // ---- refinement (as in the generic path, in scaled variables)
            if (R <= 24) solve_schur_groups(g, F, sinfo, y, cw, Rh, opbuf, stage, c.gamma, c);
            else solve_schur(g, F, sinfo, y, cw, Rh, opbuf, stage, c.gamma, c);
            __syncthreads();
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
                // Zh += y and Rh -= Ah y in one pass (y read at the node and its stencil points)
                {
                    uint64_t done = 0;
                    for (int col = 0; col < R; ++col)
                        if (c.col_done[col]) done |= 1ull << col;
                    fused_residual(g.PN, nu, R, ah, y, Zh, Rh, done, &c.rmask[0][0]);
                }
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
                if (R <= 24) solve_schur_groups(g, F, sinfo, y, cw, Rh, opbuf, stage, c.eps, c);
                else solve_schur(g, F, sinfo, y, cw, Rh, opbuf, stage, c.eps, c);
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
            // ---- outputs X[j][i] = N~_j^T z_i + z_j^T Res_i = (S N~_j)^T Zh_i + Zh_j^T Rh_i.
            // Lane = column, warps take node rows in turn: every row read is one coalesced
            // load of R doubles.  The Gram Zh^T Rh (the correction, of the size of the error
            // of Z) accumulates in FP32, one R x R partial per warp in shared memory; the mass
            // term (S m)^T Zh in FP64; partials are summed in a fixed warp order.
            {
                const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
                const bool lc = lane < R;
                // in y (free now): 8 R x R float partials, 8 x R double mass partials, R x R result
                const int gfl = (kWarpsM * R * R + 1) & ~1;
                float* gpart = y;
                double* mpart = reinterpret_cast<double*>(y + gfl);
                double* xbuf = reinterpret_cast<double*>(y + gfl + 2 * kWarpsM * R);
                // two 32-float rows per warp, used in turn: a node's Rh row (FP32) goes through
                // shared memory and is read back as 16-byte broadcasts
                float* rowb = y + ((gfl + 2 * kWarpsM * R + 2 * R * R + 3) & ~3) + warp * 64;
                float acc[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) acc[i] = 0.0f;
                double mzp = 0.0;
                int par = 0;
                for (int u = warp; u < nu; u += kWarpsM) {
                    const double zh = lc ? Zh[(size_t)u * R + lane] : 0.0;
                    const double rh = lc ? Rh[(size_t)u * R + lane] : 0.0;
                    mzp = fma(smass[u], zh, mzp);
                    const float zf = d2f_bits(zh);
                    float* rb = rowb + par * 32;
                    par ^= 1;
                    rb[lane] = d2f_bits(rh);
                    __syncwarp();
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        if (4 * q < R) {
                            const float4 r4 = *reinterpret_cast<const float4*>(rb + 4 * q);
                            acc[4 * q] = fmaf(zf, r4.x, acc[4 * q]);
                            if (4 * q + 1 < R) acc[4 * q + 1] = fmaf(zf, r4.y, acc[4 * q + 1]);
                            if (4 * q + 2 < R) acc[4 * q + 2] = fmaf(zf, r4.z, acc[4 * q + 2]);
                            if (4 * q + 3 < R) acc[4 * q + 3] = fmaf(zf, r4.w, acc[4 * q + 3]);
                        }
                    }
                }
                if (lc) {
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        if (i < R) gpart[(warp * R + lane) * R + i] = acc[i];
                    mpart[warp * R + lane] = mzp;
                }
                __syncthreads();
                for (int t = threadIdx.x; t < R * R; t += blockDim.x) {
                    float sg = 0.0f;
                    for (int w2 = 0; w2 < kWarpsM; ++w2) sg += gpart[w2 * R * R + t];
                    xbuf[t] = sg;
                }
                if (threadIdx.x < R) {
                    double mz = 0.0;
                    for (int w2 = 0; w2 < kWarpsM; ++w2) mz += mpart[w2 * R + threadIdx.x];
                    c.mz[threadIdx.x] = mz;
                }
                __syncthreads();
                // boundary terms (S N_j)^T Zh: warp per face, lane = column, FP64
                if (warp < 3 && lc) {
                    const int a = warp;
                    double sb[kMaxFaceDofs];
                    for (int jf = 0; jf < g.dpf; ++jf) sb[jf] = 0.0;
                    for (int kl = 0; kl <= g.PN; ++kl) {
                        int X, Y;
                        if (a == 2) { X = kl; Y = 0; }
                        else if (a == 0) { X = g.PN - kl; Y = kl; }
                        else { X = 0; Y = g.PN - kl; }
                        const int u = unk(g.PN, X, Y);
                        if (u < 0) continue;
                        const int kk2 = c.rev[a] ? g.PN - kl : kl;
                        const double zs = sc[u] * Zh[(size_t)u * R + lane] * (-c.sgn[a] * c.flen[a]);
                        for (int jf = 0; jf < g.dpf; ++jf) {
                            const int row = face_row(jf, c.la1[a], g.dm.fm, g.dm.lmax1);
                            if (row >= 0) sb[jf] = fma(g.dm.btab[row * (g.PN + 1) + kk2], zs, sb[jf]);
                        }
                    }
                    for (int jf = 0; jf < g.dpf; ++jf) {
                        const int j = a * g.dpf + jf;
                        xbuf[j * R + lane] += sb[jf] - c.cproj[j] * c.mz[lane];
                    }
                }
                __syncthreads();
            }
            const double* xbuf = reinterpret_cast<const double*>(y + ((kWarpsM * R * R + 1) & ~1) + 2 * kWarpsM * R);
            const int NI = g.NI;
            for (int t = threadIdx.x; t < NI * NI; t += blockDim.x) {
                const int j = t / NI, i = t - j * NI;
                g.AK[K * NI * NI + t] = -0.5 * (xbuf[j * R + i] + xbuf[i * R + j]);
            }
            for (int j = threadIdx.x; j < NI; j += blockDim.x) {
                g.EK[K * NI + j] = xbuf[j * R + NI];
                const int a = j / g.dpf, jf = j - a * g.dpf;
                const int row = face_row(jf, c.la1[a], g.dm.fm, g.dm.lmax1);
                g.BK[K * NI + j] = row < 0 ? 0.0 : c.sgn[a] * c.flen[a] * g.dm.btab_sum[row];
            }
            if (threadIdx.x == 0) {
                g.FK[K] = c.FK;
                const int code = c.timeout ? MHM_ERR_TIMEOUT : c.bad ? MHM_ERR_INVALID_ARG : (converged ? 0 : MHM_ERR_NOT_CONVERGED);
                g.status[K] = code;
                if (g.iters) g.iters[K] = pass;
                if (code && g.sword && g.word_final) atomicOr(g.sword, 1u << code);
            }
            __syncthreads();
        } else {
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
                        fh += cell_src(g, Xv, g.P, ta[t], quad_of(g.src_vals, g.kappa, kap, g.N, tup[t], ti[t], tj[t]));
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
                        const int row = face_row(jf, c.la1[a], g.dm.fm, g.dm.lmax1);
                        if (kl >= 0 && row >= 0) {
                            const int kk = c.rev[a] ? g.PN - kl : kl;
                            v += -c.sgn[a] * c.flen[a] * g.dm.btab[row * (g.PN + 1) + kk];
                        }
                    }
                    G[(size_t)col * g.nunk + u] = v;
                }
            }

            if constexpr (MODE == 3) {
                // ---- the level operators of this K, precomputed by the factor kernel
                __syncthreads();
                const int64_t kk = ki - g.Kbase;
                F = g.Tall + kk * (int64_t)g.t_stride;
                if (threadIdx.x == 0) c.bad = g.fbad[kk];
                __syncthreads();
            } else {
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
                    cholesky_level_f32<RPL, CPL>(W, g.wld, b, nr, Rhs, g.ldr, b, b + bp, &c.bad);
                    {
                        // Fw = [-Linv L_{lev,lev-1} | Linv] (b x (bp + b)) and
                        // Bw = [-Linv^T L_{lev+1,lev}^T | Linv^T] (b x (bn + b)) to this block's scratch
                        // slot in tensor-core fragment order, zero beyond the operator
                        float* Fw = F + loff[2 * lev];
                        float* Bw = F + loff[2 * lev + 1];
                        {
                            const int K = bp + b, KT = (K + 7) >> 3, n = frag_op_floats(b, K);
                            for (int t = threadIdx.x; t < n; t += blockDim.x) {
                                const int tile = t >> 7, r = t & 127, ln = r >> 2, e = r & 3;
                                const int i = (tile / KT) * 16 + (ln >> 2) + 8 * (e & 1);
                                const int k = (tile % KT) * 8 + (ln & 3) + 4 * (e >> 1);
                                float v = 0.0f;
                                if (i < b && k < K) v = k < bp ? Rhs[i * g.ldr + b + k] : Rhs[i * g.ldr + (k - bp)];
                                Fw[t] = v;
                            }
                        }
                        {
                            const int K = bn + b, KT = (K + 7) >> 3, n = frag_op_floats(b, K);
                            for (int t = threadIdx.x; t < n; t += blockDim.x) {
                                const int tile = t >> 7, r = t & 127, ln = r >> 2, e = r & 3;
                                const int i = (tile / KT) * 16 + (ln >> 2) + 8 * (e & 1);
                                const int k = (tile % KT) * 8 + (ln & 3) + 4 * (e >> 1);
                                float v = 0.0f;
                                if (i < b && k < K) {
                                    if (k >= bn) v = Rhs[(k - bn) * g.ldr + i];
                                    else {
                                        const float* cn = W + (size_t)(b + k) * g.wld;
                                        float a = 0.0f;
                                        for (int mm = i; mm < b; ++mm) a = fmaf(Rhs[mm * g.ldr + i], cn[mm], a);
                                        v = -a;
                                    }
                                }
                                Bw[t] = v;
                            }
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
            }

            // ---- refinement.  M = (L L^T)^{-1} (scaled) approximates A_p^{-1}.  The buffer G
            // becomes the residual Res = G - A_p Z, kept exact in FP64 by Res -= A_p D for
            // every correction D = M Res added to Z.  The outputs use the corrected
            // bilinear form N~^T Z + Z^T Res, whose error e^T A_p e is quadratic in the
            // error e of Z; eps_c = Res_c^T M Res_c estimates ||e_c||^2_{A_p}.
            double* Res = G;
            double* D64 = reinterpret_cast<double*>(slot + g.off_D);
            const int total = g.nunk * R;
            for (int t = threadIdx.x; t < g.nunk * g.Rp; t += blockDim.x) {
                const int u = t / g.Rp, col = t - u * g.Rp;
                y[t] = col < R ? d2f_bits(Res[(size_t)col * g.nunk + u] * scale[u]) : 0.0f;
            }
            for (int t = threadIdx.x; t < total; t += blockDim.x) Z[t] = 0.0;
            __syncthreads();
            // gamma_c = G_c^T M G_c ~ ||z_c||^2_{A_p}
            if constexpr (MODE == 3) solve_gen(g, F, sinfo, y, opbuf, stage, c);
            else solve_factor(g, F, sinfo, y, opbuf, stage, c);
            __syncthreads();
            column_dot(g, Res, y, scale, c.gamma, c);
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
                    const int col = t / g.nunk, u = t - col * g.nunk;
                    if (c.col_done[col]) continue;
                    const double d = f2d_bits(y[(size_t)u * g.Rp + col]) * scale[u];
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
                if constexpr (MODE == 3) solve_gen(g, F, sinfo, y, opbuf, stage, c);
                else solve_factor(g, F, sinfo, y, opbuf, stage, c);
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
                    zs[t] = uu < cnt ? d2f_bits(Z[(size_t)col * g.nunk + base + uu]) : 0.0f;
                    rs[t] = uu < cnt ? d2f_bits(Res[(size_t)col * g.nunk + base + uu]) : 0.0f;
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
                const int row = face_row(jf, c.la1[a], g.dm.fm, g.dm.lmax1);
                const double* zc = Z + (size_t)col * g.nunk;
                double s = 0.0;
                for (int kl = 0; kl <= g.PN && row >= 0; ++kl) {
                    int X, Y;
                    if (a == 2) { X = kl; Y = 0; }
                    else if (a == 0) { X = g.PN - kl; Y = kl; }
                    else { X = 0; Y = g.PN - kl; }
                    const int u = unk(g.PN, X, Y);
                    if (u < 0) continue;
                    const int kk = c.rev[a] ? g.PN - kl : kl;
                    s += (-c.sgn[a] * c.flen[a] * g.dm.btab[row * (g.PN + 1) + kk]) * zc[u];
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
                const int row = face_row(jf, c.la1[a], g.dm.fm, g.dm.lmax1);
                g.BK[K * NI + j] = row < 0 ? 0.0 : c.sgn[a] * c.flen[a] * g.dm.btab_sum[row];
            }
            if (threadIdx.x == 0) {
                g.FK[K] = c.FK;
                const int code = c.timeout ? MHM_ERR_TIMEOUT : c.bad ? MHM_ERR_INVALID_ARG : (converged ? 0 : MHM_ERR_NOT_CONVERGED);
                g.status[K] = code;
                if (g.iters) g.iters[K] = pass;
                if (code && g.sword && g.word_final) atomicOr(g.sword, 1u << code);
            }
            __syncthreads();
        }
        if (g.kcounter) {
            ki = c.nextK;
            __syncthreads();
            if (threadIdx.x == 0) c.nextK = g.K0 + gridDim.x + atomicAdd(g.kcounter, 1);
        } else {
            ki += gridDim.x;
        }
    }
}

template <int RPL, int CPL, int MODE, int MINB>
__global__ void __launch_bounds__(kThreadsM, MINB) k_local_mixed(const __grid_constant__ MixedArgs g) {
    mixed_blocks<RPL, CPL, MODE>(g);
}

// Coarse elements of uneven refinement level in one persistent launch: the level-Schur
// levels of a mesh are buckets of work (one per local size, the largest first); every
// block drains the current bucket's queue (its counter) and moves on to the next, so no
// block idles while a bucket has elements left.
constexpr int kMaxLevelLaunch = 5;
struct MixedLevels {
    int n;
    int block0[kMaxLevelLaunch + 1];   // factor launch: first block of each level
    MixedArgs lv[kMaxLevelLaunch];
};

__global__ void __launch_bounds__(kThreadsM, 3) k_local_mixed_levels(const __grid_constant__ MixedLevels P) {
    for (int l = 0; l < P.n; ++l) {
        mixed_blocks<2, 3, 2>(P.lv[l]);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// The level-Schur factorisation as its own kernel: one warp per coarse triangle
// (four per 128-thread block).  Each factorisation is a long chain of small
// dependent steps (a Gauss-Jordan inverse per level); run one per warp, many of
// them share an SM instead of each holding a whole block of the solve kernel.
// Per K of the chunk [Kc0, K1) it writes T_lev of every level (fragment order,
// t_stride floats), the scaled couplings (4 x nunk floats) and the pivot flag.
constexpr int kFactorWarps = 4;

struct FactorSmem {   // per warp
    float Tb[kSchurMax * kSLd];
    alignas(16) float rowbuf[2 * kSchurMax];
    double Su[9], Sd[9];
    int bad;
};

// blk: the block's index among the level's factor blocks
__device__ __forceinline__ void schur_factor_block(const MixedArgs& g, int blk) {
    extern __shared__ unsigned char fs_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ki = g.Kc0 + (int64_t)blk * kFactorWarps + warp;   // launch index within the level
    if (ki >= g.K1) return;
    const int64_t K = g.dm.klist ? (int64_t)g.dm.klist[ki] : ki;
    FactorSmem& fs = reinterpret_cast<FactorSmem*>(fs_raw)[warp];
    const int nu = g.nunk;
    double* scale = reinterpret_cast<double*>(fs_raw + kFactorWarps * sizeof(FactorSmem)) + (size_t)warp * nu;
    const double* kap = g.kappa + (g.dm.kap_off ? g.dm.kap_off[K] : K * (int64_t)g.N * g.N);
    const int64_t kk = ki - g.Kbase;
    float* cw = g.cwall + kk * 4 * (int64_t)nu;
    float* T = g.Tall + kk * (int64_t)g.t_stride;
    if (lane < 2) {
        // the two fine-triangle shapes of the uniform refinement: up (lane 0), down (lane 1)
        double V[3][2];
        for (int v = 0; v < 3; ++v) {
            V[v][0] = g.dm.geom[6 * K + 2 * v];
            V[v][1] = g.dm.geom[6 * K + 2 * v + 1];
        }
        const double e1x = (V[1][0] - V[0][0]) / g.N, e1y = (V[1][1] - V[0][1]) / g.N;
        const double e2x = (V[2][0] - V[0][0]) / g.N, e2y = (V[2][1] - V[0][1]) / g.N;
        const double Xu[3][2] = {{V[0][0], V[0][1]}, {V[0][0] + e1x, V[0][1] + e1y}, {V[0][0] + e2x, V[0][1] + e2y}};
        const double Xd[3][2] = {{V[0][0] + e1x, V[0][1] + e1y},
                                 {V[0][0] + e1x + e2x, V[0][1] + e1y + e2y},
                                 {V[0][0] + e2x, V[0][1] + e2y}};
        if (lane == 0) element_stiffness(1, Xu, fs.Su);
        else element_stiffness(1, Xd, fs.Sd);
        if (lane == 0) fs.bad = 0;
    }
    __syncwarp();
    for (int u = lane; u < nu; u += 32) {
        int X, Y;
        lattice_of_unk(g.PN, u, &X, &Y);
        double w[7];
        int v[7];
        p1_row(g.N, g.PN, nu, fs.Su, fs.Sd, kap, X, Y, u, w, v);
        scale[u] = 1.0 / sqrt(w[0]);
    }
    __syncwarp();
    for (int u = lane; u < nu; u += 32) {
        int X, Y;
        lattice_of_unk(g.PN, u, &X, &Y);
        double w[7];
        int v[7];
        p1_row(g.N, g.PN, nu, fs.Su, fs.Sd, kap, X, Y, u, w, v);
        const double su = scale[u];
        double ah[7];
        for (int d = 0; d < 7; ++d) ah[d] = w[d] * su * scale[v[d]];
        cw[u] = (float)ah[1];
        cw[nu + u] = (float)ah[2];
        cw[2 * nu + u] = (float)ah[4];
        cw[3 * nu + u] = (float)ah[5];
        double* ahK = g.ahall + kk * 7 * (int64_t)nu;
        for (int d = 0; d < 7; ++d) ahK[(size_t)d * nu + u] = ah[d];
        g.scall[kk * (int64_t)nu + u] = su;
    }
    __syncwarp();
    const LevelGeom lg{1, g.N, g.PN};
    int ul = 0, o = 0;
    for (int lev = 0; lev < g.nlev; ++lev) {
        const int b = lg.size(lev);
        schur_level_warp(cw, cw + nu, cw + 2 * nu, cw + 3 * nu, fs.Tb, fs.rowbuf, lev, b, ul, &fs.bad);
        __syncwarp();
        write_frag_op(fs.Tb, b, T + o, warp, 1);
        __syncwarp();
        o += frag_op_floats(b, b);
        ul += b;
    }
    if (lane == 0) g.fbad[kk] = fs.bad;
}

__global__ void __launch_bounds__(32 * kFactorWarps) k_schur_factor(const __grid_constant__ MixedArgs g) {
    schur_factor_block(g, blockIdx.x);
}

// The factorisations of several levels in one launch (blocks [block0[l], block0[l + 1]) take level l).
__global__ void __launch_bounds__(32 * kFactorWarps) k_schur_factor_levels(const __grid_constant__ MixedLevels P) {
    int l = 0;
    while (l + 1 < P.n && (int)blockIdx.x >= P.block0[l + 1]) ++l;
    schur_factor_block(P.lv[l], (int)blockIdx.x - P.block0[l]);
}

size_t factor_smem_bytes(int nunk) {
    return kFactorWarps * (sizeof(FactorSmem) + (size_t)nunk * sizeof(double));
}

// ---------------------------------------------------------------------------
// The generic path's level-Schur factorisation (see solve_gen) as its own kernel, one
// 128-thread block per coarse triangle, threads 2p and 2p + 1 holding row p of the level's matrix:
// S_0 = Ah_00, S_lev = Ah_{lev,lev} - C_lev T_{lev-1} C_lev^T (on the leading first-row
// block), T_lev = S_lev^-1 by Gauss-Jordan elimination in FP32, written with the coupling
// tables into the element's operator block.
constexpr int kGenThreads = 128;
constexpr int kGenLd = kGenMax + 4;    // tile row stride in floats (16-byte aligned rows)

struct GenSmem {
    alignas(16) float T[kGenMax * kGenLd];     // S_lev, then T_lev (row-major), then the next level's
                                               // Schur update C T C^T (first-row block)
    alignas(16) float rowbuf[2 * kGenMax];     // pivot rows of the Gauss-Jordan steps
    float Q[kGenMax * (kGenRow + 1)];          // T_lev C_{lev+1}^T, first-row columns of lev + 1
    int qpos[kGenRow * kTabQ];                 // per first-row node of lev + 1: positions in lev
    float qc[kGenRow * kTabQ];                 //   and couplings (position -1: none)
    double Su[36], Sd[36];                     // element stiffness of the two fine shapes
    float Suf[36], Sdf[36];                    // (FP32: the factor's assembled rows)
    int bad;
};

// T = S^-1 in place (b x b, b <= kGenMax, rows of stride kGenLd in shared memory) by
// Gauss-Jordan elimination without pivoting (S is SPD).  Row p is held in registers by the
// two threads 2p (positions 0..31) and 2p + 1 (positions 32..63) of a warp pair.  Pivots go
// in blocks of 8 with the row rotated so that the block's pivot columns sit at positions
// 0..7 (the row turns left by 8 after each block, the halves trading 8 values by shuffles),
// which keeps every register index static.  Row k travels through shared memory; each row
// applies a[j] -= g r[j] with g = a_pk / a_kk, or 1 - 1/a_kk in row k (which turns it into
// r / a_kk), then a_pk = -g (1 / a_kk in row k); a_pk reaches the second half by a shuffle.
// Ends with a block barrier.
__device__ __forceinline__ void gauss_jordan_gen(float* T, float* rowbuf, int b, int lev, int* bad) {
    constexpr int H = kGenMax / 2;   // positions per thread
    const int p = threadIdx.x >> 1, h = threadIdx.x & 1;
    const bool row = p < b;
    float a[H];
#pragma unroll
    for (int j = 0; j < H; j += 4) {
        const float4 v = row ? *reinterpret_cast<const float4*>(T + p * kGenLd + h * H + j) : make_float4(0.f, 0.f, 0.f, 0.f);
        a[j] = v.x; a[j + 1] = v.y; a[j + 2] = v.z; a[j + 3] = v.w;
    }
    const int nblk = (b + 7) >> 3;
    for (int kb = 0; kb < nblk; ++kb) {
        uint32_t cm = 0;   // this half's chunk m (positions 8(m + 4h) ..) holds columns 8 ((kb + m + 4h) mod 8) + 0..7
#pragma unroll
        for (int m = 0; m < H / 8; ++m)
            if ((((kb + m + 4 * h) & 7) << 3) < b) cm |= 1u << m;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const int k = kb * 8 + kk;
            if (k < b) {
                float* rb = rowbuf + (k & 1) * kGenMax;
                if (p == k) {
#pragma unroll
                    for (int j = 0; j < H; j += 4)
                        *reinterpret_cast<float4*>(rb + h * H + j) = make_float4(a[j], a[j + 1], a[j + 2], a[j + 3]);
                }
                __syncthreads();
                const float apk = __shfl_sync(0xffffffffu, a[kk], threadIdx.x & 30);   // position kk: first half
                if (row) {
                    const float piv = rb[kk];
                    if (threadIdx.x == 0 && !(piv > 0.0f) && *bad == 0) *bad = 1 + lev;
                    const float d = __frcp_rn(piv);
                    const float gk = p == k ? 1.0f - d : apk * d;
#pragma unroll
                    for (int m = 0; m < H / 8; ++m) {
                        if (cm >> m & 1) {
#pragma unroll
                            for (int t = 0; t < 8; t += 4) {
                                const float4 r4 = *reinterpret_cast<const float4*>(rb + h * H + 8 * m + t);
                                a[8 * m + t] = fmaf(-gk, r4.x, a[8 * m + t]);
                                a[8 * m + t + 1] = fmaf(-gk, r4.y, a[8 * m + t + 1]);
                                a[8 * m + t + 2] = fmaf(-gk, r4.z, a[8 * m + t + 2]);
                                a[8 * m + t + 3] = fmaf(-gk, r4.w, a[8 * m + t + 3]);
                            }
                        }
                    }
                    if (h == 0) a[kk] = p == k ? d : -gk;
                }
            }
        }
        // turn the row left by 8: each half passes its first 8 positions to the other half's tail
        float t8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) t8[j] = __shfl_xor_sync(0xffffffffu, a[j], 1);
#pragma unroll
        for (int j = 0; j < H - 8; ++j) a[j] = a[j + 8];
#pragma unroll
        for (int j = 0; j < 8; ++j) a[H - 8 + j] = t8[j];
    }
    // position h H + j now holds column (8 nblk + h H + j) mod kGenMax
    __syncthreads();
    if (row) {
#pragma unroll
        for (int j = 0; j < H; ++j) {
            const int col = (8 * nblk + h * H + j) & (kGenMax - 1);
            if (col < b) T[p * kGenLd + col] = a[j];
        }
    }
    __syncthreads();
}

// Couplings of unknown u into the unknowns [lo, lo + n): up to cap (position, scaled
// weight) pairs, position -1 after the last.  The factorisation assembles and scales in
// FP32 (it is an FP32 approximation of Ah; the refinement residual stays FP64).
__device__ __forceinline__ void coupling_table(const MixedArgs& g, const GenSmem& s, const float* kap,
                                               const float* scale, int u, int lo, int n, int cap, int* pos, float* cf) {
    int X, Y;
    lattice_of_unk(g.PN, u, &X, &Y);
    float w[19];
    int v[19];
    assembled_row<float>(g.P, g.N, g.PN, g.nunk, s.Suf, s.Sdf, kap, X, Y, u, w, v);
    const float su = scale[u];
    int m = 0;
#pragma unroll
    for (int k = 1; k < 19; ++k)
        if (v[k] != u && v[k] >= lo && v[k] < lo + n && m < cap) {
            pos[m] = v[k] - lo;
            cf[m] = w[k] * su * scale[v[k]];
            ++m;
        }
    for (; m < cap; ++m) { pos[m] = -1; cf[m] = 0.0f; }
}

// An operator of b rows and Kc columns to global memory in fragment order (one float4 per
// lane and 16 x 8 tile, the layout of write_frag_op), entry (i, k) from val(i, k) inside
// the operator and 0 in the padding.
template <class Val>
__device__ __forceinline__ void write_frag_gen(float* dst, int b, int Kc, const Val& val) {
    const int KT = (Kc + 7) >> 3, MT = (b + 15) >> 4, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    auto at = [&](int i, int k) { return (i < b && k < Kc) ? val(i, k) : 0.0f; };
    for (int tile = warp; tile < MT * KT; tile += kGenThreads / 32) {
        const int mt = tile / KT, kt = tile - mt * KT;
        const int i0 = mt * 16 + g, k0 = kt * 8 + t;
        reinterpret_cast<float4*>(dst)[tile * 32 + lane] =
            make_float4(at(i0, k0), at(i0 + 8, k0), at(i0, k0 + 4), at(i0 + 8, k0 + 4));
    }
}

__global__ void __launch_bounds__(kGenThreads) k_schur_factor_gen(const MixedArgs g) {
    extern __shared__ unsigned char gs_raw[];
    GenSmem& s = *reinterpret_cast<GenSmem*>(gs_raw);
    float* scale = reinterpret_cast<float*>(gs_raw + sizeof(GenSmem));   // nunk
    float* kap = scale + g.nunk;                                           // N^2 (FP32)
    const int64_t ki = g.Kc0 + blockIdx.x;   // launch index within the level
    if (ki >= g.K1) return;
    const int64_t K = g.dm.klist ? (int64_t)g.dm.klist[ki] : ki;
    const int p = threadIdx.x, nu = g.nunk;
    const double* kapg = g.kappa + (g.dm.kap_off ? g.dm.kap_off[K] : K * (int64_t)g.N * g.N);
    for (int t = p; t < g.N * g.N; t += kGenThreads) kap[t] = d2f_bits(kapg[t]);
    const int64_t kk = ki - g.Kbase;
    float* F = g.Tall + kk * (int64_t)g.t_stride;
    if (p == 0) {
        // the two fine-triangle shapes (up and down) of the uniform refinement
        double V[3][2];
        for (int v = 0; v < 3; ++v) {
            V[v][0] = g.dm.geom[6 * K + 2 * v];
            V[v][1] = g.dm.geom[6 * K + 2 * v + 1];
        }
        const double e1x = (V[1][0] - V[0][0]) / g.N, e1y = (V[1][1] - V[0][1]) / g.N;
        const double e2x = (V[2][0] - V[0][0]) / g.N, e2y = (V[2][1] - V[0][1]) / g.N;
        const double Xu[3][2] = {{V[0][0], V[0][1]}, {V[0][0] + e1x, V[0][1] + e1y}, {V[0][0] + e2x, V[0][1] + e2y}};
        const double Xd[3][2] = {{V[0][0] + e1x, V[0][1] + e1y},
                                 {V[0][0] + e1x + e2x, V[0][1] + e1y + e2y},
                                 {V[0][0] + e2x, V[0][1] + e2y}};
        element_stiffness(g.P, Xu, s.Su);
        element_stiffness(g.P, Xd, s.Sd);
        s.bad = 0;
    }
    __syncthreads();
    if (p < 36) {
        s.Suf[p] = d2f_bits(s.Su[p]);
        s.Sdf[p] = d2f_bits(s.Sd[p]);
    }
    __syncthreads();
    for (int u = p; u < nu; u += kGenThreads) {
        int X, Y;
        lattice_of_unk(g.PN, u, &X, &Y);
        float w[19];
        int v[19];
        assembled_row<float>(g.P, g.N, g.PN, nu, s.Suf, s.Sdf, kap, X, Y, u, w, v);
        scale[u] = 1.0f / sqrtf(w[0]);
    }
    __syncthreads();
    const LevelGeom lg{g.P, g.N, g.PN};
    int ul = 0;   // first unknown of the level
    for (int lev = 0; lev < g.nlev; ++lev) {
        const int b = lg.size(lev);
        const int bp = lev > 0 ? lg.size(lev - 1) : 0;
        const int bn = lev + 1 < g.nlev ? lg.size(lev + 1) : 0;
        const int l0 = first_row_size(lg, lev), l0n = bn > 0 ? first_row_size(lg, lev + 1) : 0;
        // S_lev: row p from the assembled row of its unknown, less the Schur update (which the
        // level before left in the first-row block of the tile)
        if (p < b) {
            float* row = s.T + p * kGenLd;
            const int keep = lev > 0 && p < l0 ? l0 : 0;
            for (int j = 0; j < keep; ++j) row[j] = -row[j];
            for (int j = keep; j < kGenMax; ++j) row[j] = 0.0f;
            const int u = ul + p;
            int X, Y;
            lattice_of_unk(g.PN, u, &X, &Y);
            float w[19];
            int v[19];
            assembled_row<float>(g.P, g.N, g.PN, nu, s.Suf, s.Sdf, kap, X, Y, u, w, v);
            const float su = scale[u];
#pragma unroll
            for (int k = 0; k < 19; ++k)
                if (v[k] >= ul && v[k] < ul + b) row[v[k] - ul] += w[k] * su * scale[v[k]];
        }
        int t_off, f_off, b_off;
        // backward table of the level below: its nodes' couplings into this level
        if (lev > 0) {
            gen_offsets(lg, g.nlev, lev - 1, &t_off, &f_off, &b_off);
            for (int k = p; k < bp; k += kGenThreads) {
                int pos[kTabF];
                float cf[kTabF];
                coupling_table(g, s, kap, scale, ul - bp + k, ul, b, kTabF, pos, cf);
                float2* e = reinterpret_cast<float2*>(F + b_off) + k * kTabF;
#pragma unroll
                for (int m = 0; m < kTabF; ++m) e[m] = make_float2(__int_as_float(pos[m]), cf[m]);
            }
        }
        // the next level's first-row couplings into this level (rows of C_{lev+1}): its
        // forward table, and kept for the Schur update
        if (l0n > 0) {
            gen_offsets(lg, g.nlev, lev + 1, &t_off, &f_off, &b_off);
            for (int q = p; q < l0n; q += kGenThreads) {
                coupling_table(g, s, kap, scale, ul + b + q, ul, b, kTabQ, s.qpos + q * kTabQ, s.qc + q * kTabQ);
                float2* e = reinterpret_cast<float2*>(F + f_off) + q * kTabQ;
#pragma unroll
                for (int m = 0; m < kTabQ; ++m) e[m] = make_float2(__int_as_float(s.qpos[q * kTabQ + m]), s.qc[q * kTabQ + m]);
            }
        }
        __syncthreads();
        gauss_jordan_gen(s.T, s.rowbuf, b, lev, &s.bad);
        // T_lev in fragment order
        gen_offsets(lg, g.nlev, lev, &t_off, &f_off, &b_off);
        write_frag_gen(F + t_off, b, b, [&](int i, int k) { return s.T[i * kGenLd + k]; });
        // Q = T C_{lev+1}^T on the next level's first-row columns
        for (int t = p; t < b * l0n; t += kGenThreads) {
            const int i = t / l0n, q = t - i * l0n;
            float acc = 0.0f;
#pragma unroll
            for (int m = 0; m < kTabQ; ++m) {
                const int a = s.qpos[q * kTabQ + m];
                if (a >= 0) acc = fmaf(s.T[i * kGenLd + a], s.qc[q * kTabQ + m], acc);
            }
            s.Q[i * (kGenRow + 1) + q] = acc;
        }
        __syncthreads();
        // C_{lev+1} Q on the next level's first-row block, into the tile (T_lev is written out)
        for (int t = p; t < l0n * l0n; t += kGenThreads) {
            const int i = t / l0n, q = t - i * l0n;
            float acc = 0.0f;
#pragma unroll
            for (int m = 0; m < kTabQ; ++m) {
                const int a = s.qpos[i * kTabQ + m];
                if (a >= 0) acc = fmaf(s.qc[i * kTabQ + m], s.Q[a * (kGenRow + 1) + q], acc);
            }
            s.T[i * kGenLd + q] = acc;
        }
        __syncthreads();
        ul += b;
    }
    if (p == 0) g.fbad[kk] = s.bad;
}

size_t gen_factor_smem_bytes(int nunk, int N) {
    return sizeof(GenSmem) + (size_t)(nunk + N * N) * sizeof(float);
}

struct MixedLayout {
    int nlev, nunk, wrows, wld, wfloats, yfloats, bmax, opmax, ldr, Rp, stage_floats;
    size_t factor_floats, slot_bytes, off_G, off_Z, off_mass, off_scale, off_D, smem;
    size_t off_kap_smem, off_scale_smem, off_sinfo, off_cw;
    int kap_in_smem, rpl, cpl;
    bool schur;   // P1 with levels of at most kSchurMax unknowns: level-Schur factorisation
    int mode;     // kernel MODE (0 generic, 1 Schur in the kernel, 2 Schur by k_schur_factor,
                  // 3 generic by k_schur_factor_gen)
};

constexpr int64_t kChunkMax = 8192;      // MODE 2: coarse triangles per factor + solve launch pair
constexpr int64_t kChunkMaxGen = 4096;   // MODE 3 (about 4x the operator floats per element)

// split: the level-Schur path factors in k_schur_factor (MODE 2) instead of in the
// solve kernel (MODE 1; the allocation-free entry, whose scratch cannot hold the
// per-K operators of a whole chunk).
MixedLayout mixed_layout(const mhm_mesh* mesh, const Level& lv, bool split = true) {
    MixedLayout L{};
    const int P = mesh->desc.degree, N = lv.N;
    auto size = [&](int lev) {
        if (P == 1) return N + 1 - lev - (lev == 0);
        if (lev == N) return 1;
        return (2 * N - 2 * lev + 1) + (2 * N - 2 * lev) - (lev == 0);
    };
    L.nlev = N + 1;
    L.nunk = (int)lv.nloc - 1;
    int bmax = 0;
    for (int lev = 0; lev < L.nlev; ++lev) bmax = std::max(bmax, size(lev));
    L.schur = P == 1 && bmax <= kSchurMax && mesh->NI + 1 <= 32;
    int row0 = 0;   // largest first lattice row of a level (unknowns)
    for (int lev = 0; lev < L.nlev; ++lev)
        row0 = std::max(row0, P == 1 || lev == N ? size(lev) : 2 * N - 2 * lev + 1 - (lev == 0));
    L.mode = L.schur ? (split ? 2 : 1) : (split && bmax <= kGenMax && row0 <= kGenRow ? 3 : 0);
    size_t f = 0;
    int opmax = 0;
    for (int lev = 0; lev < L.nlev; ++lev) {
        const int b = size(lev), bn = lev + 1 < L.nlev ? size(lev + 1) : 0;
        const int bp = lev > 0 ? size(lev - 1) : 0;
        if (L.schur || L.mode == 3) {
            const int t = frag_op_floats(b, b);
            f += (size_t)t;
            opmax = std::max(opmax, t);
            if (L.mode == 3) {   // coupling tables: forward (first rows of levels >= 1), backward
                const int l0 = P == 1 || lev == N ? b : 2 * N - 2 * lev + 1 - (lev == 0);
                if (lev >= 1) f += (size_t)2 * kTabQ * l0;
                if (lev + 1 < L.nlev) f += (size_t)2 * kTabF * b;
            }
        } else {
            const int fw = frag_op_floats(b, b + bp), bw = frag_op_floats(b, b + bn);
            f += (size_t)fw + bw;
            opmax = std::max(opmax, std::max(fw, bw));
        }
    }
    L.bmax = bmax;
    L.opmax = opmax;
    L.factor_floats = f;
    L.wrows = size(0) + (N >= 1 ? size(1) : 0);
    L.wld = (L.wrows + 4) & ~3;   // rows 16-byte aligned for the vector panel loads
    const int R = (int)mesh->NI + 1;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    L.off_G = L.mode >= 2 ? 0 : al(f * sizeof(float));   // MODEs 2 and 3 keep the operators outside the slots
    L.off_Z = L.off_G + al((size_t)L.nunk * R * sizeof(double));
    L.off_mass = L.off_Z + al((size_t)L.nunk * R * sizeof(double));
    L.off_scale = L.off_mass + al((size_t)L.nunk * sizeof(double));
    L.off_D = L.off_scale + al((size_t)L.nunk * sizeof(double));
    L.slot_bytes = L.off_D + al((size_t)L.nunk * R * sizeof(double));
    size_t win = (size_t)L.wrows * L.wld;
    if (win < (size_t)R * R * 2) win = (size_t)R * R * 2;
    // staged solve operand: K-tiles x n-tiles x 64 floats, K = b + b' of the largest step
    L.Rp = R;
    int ktmax = 0;
    for (int lev = 0; lev < L.nlev; ++lev) {
        const int b = size(lev), bn = lev + 1 < L.nlev ? size(lev + 1) : 0, bp = lev > 0 ? size(lev - 1) : 0;
        ktmax = std::max(ktmax, (b + std::max(bn, bp) + 7) / 8);
    }
    if (L.schur) {
        // one staged operand of K = b; the factorisation's S and T (kSchurMax x kSLd each)
        L.stage_floats = ((bmax + 7) / 8) * ((R + 7) / 8) * 64;
        // the ring of the level's tuned depth (the allocation-free entry keeps the default)
        const int nring = std::max(2, std::min(kMaxOpBufs, lv.tune.nbuf));
        win = std::max((size_t)nring * L.opmax + (size_t)L.stage_floats, (size_t)R * R * 2);
        if (L.mode == 1) win = std::max(win, (size_t)2 * kSchurMax * kSLd + 2 * kSchurMax);   // S, T, pivot rows
    } else {
        L.stage_floats = ktmax * ((R + 7) / 8) * 64;
        if (L.mode == 3) {
            // no factorisation window: two operator buffers and one staged operand of K = b
            L.stage_floats = ((bmax + 7) / 8) * ((R + 7) / 8) * 64;
            win = std::max((size_t)R * R * 2, (size_t)2 * L.opmax + (size_t)L.stage_floats);
        }
        if (win < (size_t)2 * L.opmax + (size_t)2 * L.stage_floats && L.mode != 3)
            win = (size_t)2 * L.opmax + (size_t)2 * L.stage_floats;
    }
    win = (win + 3) & ~(size_t)3;
    L.wfloats = (int)win;
    size_t yf = (size_t)L.nunk * L.Rp;
    if (yf < (size_t)2 * R * 64) yf = (size_t)2 * R * 64;   // also holds two R x 64 staging chunks
    L.ldr = (2 * bmax + 3) & ~3;
    if (L.mode == 0 && yf < (size_t)bmax * L.ldr) yf = (size_t)bmax * L.ldr;   // and the level right-hand sides while factoring
    if (L.schur) yf = std::max(yf, (size_t)(10 * R * R + 16 * R + 8 + 4 + kWarpsM * 64));   // and the output partials
    L.yfloats = (int)((yf + 3) & ~(size_t)3);
    size_t off = win * sizeof(float) + (size_t)L.yfloats * sizeof(float) + (size_t)(3 * L.nlev + 1) * sizeof(int);
    off = (off + 15) & ~(size_t)15;
    const size_t nf = (size_t)N * N;
    L.kap_in_smem = 0;   // kappa is read from global memory (L2-resident after first touch)
    L.off_kap_smem = off;
    off += L.kap_in_smem ? nf * sizeof(double) : 0;
    L.off_scale_smem = 0;
    off = (off + 15) & ~(size_t)15;
    L.off_sinfo = off;
    off += (size_t)2 * L.nlev * 16;
    L.off_cw = off;
    if (L.mode == 1) off += (size_t)4 * L.nunk * sizeof(float);   // MODE 2 reads the couplings in place
    L.smem = (off + 15) & ~(size_t)15;
    // register shape of the warp panel: rows (window) and right-hand-side columns per lane
    int ncols = 0;
    for (int lev = 0; lev < L.nlev; ++lev) {
        const int c = size(lev) + (lev > 0 ? size(lev - 1) : 0);
        if (c > ncols) ncols = c;
    }
    if (L.schur) { L.rpl = 2; L.cpl = 3; }
    else if (L.wrows <= 64 && ncols <= 96) { L.rpl = 2; L.cpl = 3; }
    else if (L.wrows <= 128 && ncols <= 128) { L.rpl = 4; L.cpl = 4; }
    else { L.rpl = 0; L.cpl = 0; }
    return L;
}

using MixedKernel = void (*)(const MixedArgs);

// four resident blocks per SM: the level-Schur solve kernel compiled for 64 registers
MixedKernel mixed_kernel(const MixedLayout& L, int blocks_per_sm = 3) {
    if (L.mode == 2) return blocks_per_sm >= 4 ? k_local_mixed<2, 3, 2, 4> : k_local_mixed<2, 3, 2, 3>;
    if (L.mode == 1) return k_local_mixed<2, 3, 1, 3>;
    if (L.mode == 3) return k_local_mixed<2, 3, 3, 2>;
    if (L.rpl == 2) return k_local_mixed<2, 3, 0, 3>;
    if (L.rpl == 4) return k_local_mixed<4, 4, 0, 3>;
    return nullptr;
}

// Resident blocks per SM of the kernel for this layout: the slots of the workspace.  The
// level-Schur path sizes them for the four-block variant (its shape may be tuned after the
// workspace was allocated).
int mixed_slots(const mhm_mesh* mesh, const MixedLayout& L) {
    int dev = mesh->device, sms = 0, per = 0;
    MixedKernel k = mixed_kernel(L);
    if (!k) return 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kThreadsM, L.smem) != cudaSuccess || per < 1)
        per = 1;
    if (L.mode == 2) per = std::max(per, 4);
    return sms * per;
}

}  // namespace

namespace {

// the workspace holds chunk regions of kChunkMax elements; a tuned chunk is at most that
int64_t chunk_of(const Level& lv, const MixedLayout& L) {
    return L.mode == 2 ? std::min<int64_t>(lv.nK, kChunkMax) : L.mode == 3 ? std::min<int64_t>(lv.nK, kChunkMaxGen) : 0;
}
int64_t tuned_chunk(const Level& lv, const MixedLayout& L) {
    return L.mode >= 2 ? std::min<int64_t>(chunk_of(lv, L), std::max(256, std::min<int>(lv.tune.chunk, (int)kChunkMax)))
                       : 0;
}

MixedArgs mixed_args(const mhm_mesh* mesh, const Level& lv, const MixedLayout& L, const double* kappa,
                     const mhm_source& f, const mhm_solve_opts& o, double* AK, double* EK, double* BK, double* FK,
                     int32_t* status, int32_t* iters, char* ws) {
    MixedArgs g{};
    g.dm = mesh->dev(lv);
    g.kappa = kappa;
    g.P = mesh->desc.degree;
    g.N = lv.N;
    g.PN = lv.PN;
    g.dpf = mesh->dpf;
    g.NI = (int)mesh->NI;
    g.R = g.NI + 1;
    g.Rp = L.Rp;
    g.nlev = L.nlev;
    g.nunk = L.nunk;
    g.wrows = L.wrows;
    g.wld = L.wld;
    g.wfloats = L.wfloats;
    g.yfloats = L.yfloats;
    g.bmax = L.bmax;
    g.opmax = L.opmax;
    g.stage_floats = L.stage_floats;
    g.ldr = L.ldr;
    g.src_kind = f.kind;
    g.src_vals = f.kind == MHM_SRC_QUAD ? f.values_dev : nullptr;
    g.sword = mesh->d_sword;
    g.word_final = o.no_fallback != 0;
    g.src_value = f.value;
    g.src_freq = f.freq;
    g.it_max = o.it_max;
    g.tol = o.tol;
    g.ws = ws;
    g.slot_bytes = L.slot_bytes;
    g.off_G = L.off_G;
    g.off_Z = L.off_Z;
    g.off_mass = L.off_mass;
    g.off_scale = L.off_scale;
    g.off_D = L.off_D;
    g.off_kap_smem = L.off_kap_smem;
    g.off_scale_smem = L.off_scale_smem;
    g.off_sinfo = L.off_sinfo;
    g.off_cw = L.off_cw;
    g.kap_in_smem = L.kap_in_smem;
    g.AK = AK; g.EK = EK; g.BK = BK; g.FK = FK;
    g.status = status;
    g.iters = iters;
    g.t_stride = L.factor_floats;
    g.nbuf = std::max(2, std::min(kMaxOpBufs, lv.tune.nbuf));
    g.l2pf = std::max(0, lv.tune.l2pf);
    g.pf_all = lv.tune.pf_all != 0;
    g.op_policy = std::max(0, std::min(2, lv.tune.op_policy));
    return g;
}

}  // namespace

// Per-K arrays of the factor kernel's output for n coarse elements starting at base: the
// level operators (fragment order), the pivot flags and, for MODE 2, the FP32 couplings,
// the FP64 scaling and the scaled stencil, each array 256-byte aligned.
static size_t region_bytes(int64_t n, const MixedLayout& L) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t ops = (size_t)n * al(L.factor_floats * sizeof(float)) + al((size_t)n * sizeof(int));
    if (L.mode == 3) return ops;
    return ops + al((size_t)n * 4 * L.nunk * sizeof(float)) + al((size_t)n * L.nunk * sizeof(double)) +
           al((size_t)n * 7 * L.nunk * sizeof(double));
}

static void region_ptrs(char* base, int64_t n, const MixedLayout& L, MixedArgs& g) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char* p = base;
    g.Tall = reinterpret_cast<float*>(p);
    p += (size_t)n * al(L.factor_floats * sizeof(float));
    if (L.mode == 3) {
        g.fbad = reinterpret_cast<int*>(p);
        g.cwall = nullptr;
        g.scall = nullptr;
        g.ahall = nullptr;
        return;
    }
    g.cwall = reinterpret_cast<float*>(p);
    p += al((size_t)n * 4 * L.nunk * sizeof(float));
    g.fbad = reinterpret_cast<int*>(p);
    p += al((size_t)n * sizeof(int));
    g.scall = reinterpret_cast<double*>(p);
    p += al((size_t)n * L.nunk * sizeof(double));
    g.ahall = reinterpret_cast<double*>(p);
}

// The K of launch indices [i0, i1) whose status is not OK, appended to list (order of
// arrival; each K's result does not depend on it).
__global__ void k_collect_failed(const int32_t* klist, int64_t i0, int64_t i1, const int32_t* status, int32_t* list,
                                 int32_t* count) {
    for (int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < i1; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t K = klist ? (int64_t)klist[i] : i;
        if (status[K] != MHM_OK) list[atomicAdd(count, 1)] = (int32_t)K;
    }
}

// Workspace of one level: the slots, the chunk arrays, the assignment counter, and the
// list of failed elements (count + one entry per element of the level).
// chunk regions of a level: two (factor of chunk c+1 beside the solve of chunk c) when
// the level spans several chunks
static int chunk_buffers(const Level& lv, const MixedLayout& L) {
    return (L.mode >= 2 && lv.nK > chunk_of(lv, L)) ? 2 : 1;
}

static size_t level_workspace(const mhm_mesh* mesh, const Level& lv, const MixedLayout& L) {
    return (size_t)mixed_slots(mesh, L) * L.slot_bytes + (size_t)chunk_buffers(lv, L) * region_bytes(chunk_of(lv, L), L) +
           256 + 256 + (((size_t)lv.nK * sizeof(int32_t) + 255) & ~(size_t)255);
}

// Factor store (kept level-Schur factors): the MODE 2 and 3 levels one after the other,
// each a region of all its elements.  Returns the store's size; *offset gets lv's region (or
// SIZE_MAX for a level without one).
size_t factor_store_layout(const mhm_mesh* mesh, const Level* lv, size_t* offset) {
    size_t bytes = 0;
    if (offset) *offset = SIZE_MAX;
    if (mesh->device < 0) return 0;
    for (const Level& l2 : mesh->levels) {
        if (fp64_level(mesh, l2)) continue;
        const MixedLayout L = mixed_layout(mesh, l2);
        if (L.mode < 2) continue;
        if (&l2 == lv && offset) *offset = bytes;
        bytes += (region_bytes(l2.nK, L) + 255) & ~(size_t)255;
    }
    return bytes;
}

bool schur_split_level(const mhm_mesh* mesh, const Level& lv) {
    if (mesh->device < 0 || fp64_level(mesh, lv)) return false;
    return mixed_layout(mesh, lv).mode == 2;
}

size_t mixed_level_workspace(const mhm_mesh* mesh, const Level& lv) {
    if (mesh->device < 0 || fp64_level(mesh, lv)) return 0;   // FP64 levels: fp64_level_workspace
    const MixedLayout L = mixed_layout(mesh, lv);
    if (L.smem > 220 * 1024 || !mixed_kernel(L)) return 0;
    return (level_workspace(mesh, lv, L) + 255) & ~(size_t)255;
}

mhm_status launch_local_mixed(const mhm_mesh* mesh, const Level& lv, const double* kappa, const mhm_source& f,
                              const mhm_solve_opts& opts, int64_t K0, int64_t K1, double* AK, double* EK,
                              double* BK, double* FK, int32_t* status, int32_t* iters, void* workspace,
                              size_t ws_bytes, cudaStream_t stream) {
    // K0, K1: launch indices within the level (its K list, or K itself on a uniform mesh)
    const MixedLayout L = mixed_layout(mesh, lv);
    if (L.smem > 220 * 1024 || !mixed_kernel(L))
        return fail(MHM_ERR_UNSUPPORTED, "mhm_local_solve_batch: MIXED buffers exceed shared memory (r too large)");
    const int slots = mixed_slots(mesh, L);
    const int64_t chunk = chunk_of(lv, L);
    const size_t slots_bytes = (size_t)slots * L.slot_bytes;
    if (ws_bytes < level_workspace(mesh, lv, L))
        return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch: workspace smaller than mhm_local_workspace_size");
    // dynamic assignment of coarse triangles to blocks: a counter behind the scratch,
    // zeroed in stream order before every solve launch
    const int nbuf = chunk_buffers(lv, L);
    int* counter = reinterpret_cast<int*>((char*)workspace + slots_bytes + (size_t)nbuf * region_bytes(chunk, L));
    MixedArgs g = mixed_args(mesh, lv, L, kappa, f, opts, AK, EK, BK, FK, status, iters, (char*)workspace);
    const int64_t nK = K1 - K0;
    if (nK <= 0) return MHM_OK;
    g.kcounter = counter;
    // elements whose refinement failed are solved again by the FP64 path (list behind the counter)
    auto fallback = [&]() -> mhm_status {
        if (opts.no_fallback) return MHM_OK;
        int32_t* fcount = reinterpret_cast<int32_t*>((char*)counter + 256);
        int32_t* flist = reinterpret_cast<int32_t*>((char*)counter + 512);
        MHM_CUDA_TRY(cudaMemsetAsync(fcount, 0, sizeof(int32_t), stream));
        const int64_t nb = std::min<int64_t>((nK + 255) / 256, 1024);
        k_collect_failed<<<(unsigned)nb, 256, 0, stream>>>(g.dm.klist, K0, K1, status, flist, fcount);
        MHM_CUDA_TRY(cudaGetLastError());
        return launch_local_fp64_list(mesh, lv, kappa, f, flist, fcount, nK, AK, EK, BK, FK, status, iters, stream);
    };
    if (L.mode < 2) {
        g.K0 = K0;
        g.K1 = K1;
        MHM_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), stream));
        const int grid = (int)(nK < slots ? nK : slots);
        timing_mark(mesh, MHM_KERNEL_LOCAL_MIXED, stream, true);
        mixed_kernel(L)<<<grid, kThreadsM, L.smem, stream>>>(g);
        timing_mark(mesh, MHM_KERNEL_LOCAL_MIXED, stream, false);
        MHM_CUDA_TRY(cudaGetLastError());
        return fallback();
    }
    // MODEs 2 and 3: per chunk, the factor kernel writes the level operators and pivot flags
    // (MODE 2 also the couplings, scaling and scaled stencil) into a chunk region behind the
    // slots; the solve kernel reads them.  With several chunks the factor launches run on
    // the level's own stream, one chunk ahead: region c % 2 is refilled once the solve of
    // chunk c - 2 is done with it.
    const bool gen = L.mode == 3;
    const size_t fsmem = gen ? gen_factor_smem_bytes(L.nunk, lv.N) : factor_smem_bytes(L.nunk);
    if (gen) MHM_CUDA_TRY(cudaFuncSetAttribute(k_schur_factor_gen, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
    else MHM_CUDA_TRY(cudaFuncSetAttribute(k_schur_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
    // the tuned chunk steps through the range; factor launches run one chunk ahead on the
    // level's stream when there are two chunk regions (or a factor store, whose regions
    // never repeat), otherwise in the caller's stream order
    const int64_t tchunk = tuned_chunk(lv, L);
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, mesh->device);
    const int tslots = std::max(1, std::min(slots, sms * std::max(1, lv.tune.blocks_per_sm)));
    const MixedKernel kern = mixed_kernel(L, lv.tune.blocks_per_sm);
    MHM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem));
    const bool pipelined = K1 - K0 > tchunk && (nbuf == 2 || opts.factor_store != nullptr);
    if (pipelined) {
        if (!lv.fstream) {
            MHM_CUDA_TRY(cudaStreamCreateWithFlags(&lv.fstream, cudaStreamNonBlocking));
            MHM_CUDA_TRY(cudaEventCreateWithFlags(&lv.fstart, cudaEventDisableTiming));
            for (int b = 0; b < 2; ++b) {
                MHM_CUDA_TRY(cudaEventCreateWithFlags(&lv.fdone[b], cudaEventDisableTiming));
                MHM_CUDA_TRY(cudaEventCreateWithFlags(&lv.mdone[b], cudaEventDisableTiming));
            }
        }
        MHM_CUDA_TRY(cudaEventRecord(lv.fstart, stream));
        MHM_CUDA_TRY(cudaStreamWaitEvent(lv.fstream, lv.fstart, 0));
    }
    cudaStream_t fs = pipelined ? lv.fstream : stream;
    // a factor store keeps every element's factors of the level (factor_reuse 0: the factor
    // launches fill it; 1: they are skipped and the solves read what it holds)
    char* store = nullptr;
    if (opts.factor_store) {
        size_t off = SIZE_MAX;
        factor_store_layout(mesh, &lv, &off);
        if (off == SIZE_MAX) return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch: level without a factor store region");
        store = (char*)opts.factor_store + off;
    }
    const bool reuse = store && opts.factor_reuse;
    int c = 0;
    for (int64_t c0 = K0; c0 < K1; c0 += tchunk, ++c) {
        const int64_t c1 = std::min(K1, c0 + tchunk);
        const int b = pipelined ? (c & 1) : 0;
        if (store) {
            region_ptrs(store, lv.nK, L, g);
            g.Kbase = 0;
        } else {
            region_ptrs((char*)workspace + slots_bytes + (size_t)b * region_bytes(chunk, L), chunk, L, g);
            g.Kbase = c0;
        }
        g.Kc0 = c0;
        g.K0 = c0;
        g.K1 = c1;
        if (!reuse) {
            if (pipelined && c >= 2 && !store) MHM_CUDA_TRY(cudaStreamWaitEvent(fs, lv.mdone[b], 0));
            timing_mark(mesh, MHM_KERNEL_SCHUR_FACTOR, fs, true);
            if (gen) k_schur_factor_gen<<<(unsigned)(c1 - c0), kGenThreads, fsmem, fs>>>(g);
            else k_schur_factor<<<(unsigned)((c1 - c0 + kFactorWarps - 1) / kFactorWarps), 32 * kFactorWarps, fsmem, fs>>>(g);
            timing_mark(mesh, MHM_KERNEL_SCHUR_FACTOR, fs, false);
            MHM_CUDA_TRY(cudaGetLastError());
            if (pipelined) {
                MHM_CUDA_TRY(cudaEventRecord(lv.fdone[b], fs));
                MHM_CUDA_TRY(cudaStreamWaitEvent(stream, lv.fdone[b], 0));
            }
        }
        MHM_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), stream));
        const int grid = (int)(c1 - c0 < tslots ? c1 - c0 : tslots);
        timing_mark(mesh, MHM_KERNEL_LOCAL_MIXED, stream, true);
        kern<<<grid, kThreadsM, L.smem, stream>>>(g);
        timing_mark(mesh, MHM_KERNEL_LOCAL_MIXED, stream, false);
        MHM_CUDA_TRY(cudaGetLastError());
        if (pipelined) MHM_CUDA_TRY(cudaEventRecord(lv.mdone[b], stream));
    }
    return fallback();
}

// Several level-Schur levels in one factor launch and one persistent solve launch (see
// k_local_mixed_levels); each level keeps its own workspace region (slots, one chunk
// region, queue counter), and its failed elements are re-solved in FP64 afterwards.
bool levels_launchable(const mhm_mesh* mesh, const std::vector<const Level*>& lvs, const std::vector<int64_t>& r0,
                       const std::vector<int64_t>& r1, const mhm_solve_opts& opts) {
    if (lvs.size() < 2 || lvs.size() > (size_t)kMaxLevelLaunch || opts.factor_store) return false;
    for (size_t i = 0; i < lvs.size(); ++i) {
        if (!schur_split_level(mesh, *lvs[i])) return false;
        const MixedLayout L = mixed_layout(mesh, *lvs[i]);
        if (r1[i] - r0[i] > chunk_of(*lvs[i], L)) return false;   // one chunk region per level
    }
    return true;
}

mhm_status launch_local_mixed_levels(const mhm_mesh* mesh, const std::vector<const Level*>& lvs,
                                     const std::vector<int64_t>& r0, const std::vector<int64_t>& r1,
                                     const std::vector<char*>& regions, const double* kappa, const mhm_source& f,
                                     const mhm_solve_opts& opts, double* AK, double* EK, double* BK, double* FK,
                                     int32_t* status, int32_t* iters, cudaStream_t stream) {
    const int n = (int)lvs.size();
    // buckets in order of decreasing work (elements x unknowns)
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::vector<MixedLayout> Ls(n);
    for (int i = 0; i < n; ++i) Ls[i] = mixed_layout(mesh, *lvs[i]);
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        return (double)(r1[a] - r0[a]) * Ls[a].nunk > (double)(r1[b] - r0[b]) * Ls[b].nunk;
    });
    MixedLevels P{};
    P.n = n;
    size_t smem = 0, fsmem = 0;
    int min_slots = INT32_MAX, fblocks = 0;
    std::vector<int*> counters(n);
    for (int j = 0; j < n; ++j) {
        const int i = order[j];
        const Level& lv = *lvs[i];
        const MixedLayout& L = Ls[i];
        const int slots = mixed_slots(mesh, L);
        min_slots = std::min(min_slots, slots);
        const size_t slots_bytes = (size_t)slots * L.slot_bytes;
        const int64_t chunk = chunk_of(lv, L);
        const int nbuf = chunk_buffers(lv, L);
        counters[j] = reinterpret_cast<int*>(regions[i] + slots_bytes + (size_t)nbuf * region_bytes(chunk, L));
        MixedArgs g = mixed_args(mesh, lv, L, kappa, f, opts, AK, EK, BK, FK, status, iters, regions[i]);
        region_ptrs(regions[i] + slots_bytes, chunk, L, g);
        g.Kbase = g.Kc0 = g.K0 = r0[i];
        g.K1 = r1[i];
        g.kcounter = counters[j];
        P.lv[j] = g;
        P.block0[j] = fblocks;
        fblocks += (int)((r1[i] - r0[i] + kFactorWarps - 1) / kFactorWarps);
        smem = std::max(smem, L.smem);
        fsmem = std::max(fsmem, factor_smem_bytes(L.nunk));
        MHM_CUDA_TRY(cudaMemsetAsync(counters[j], 0, sizeof(int), stream));
    }
    P.block0[n] = fblocks;
    MHM_CUDA_TRY(cudaFuncSetAttribute(k_schur_factor_levels, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
    MHM_CUDA_TRY(cudaFuncSetAttribute(k_local_mixed_levels, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, mesh->device);
    const int grid = std::min(min_slots, sms * 3);
    timing_mark(mesh, MHM_KERNEL_SCHUR_FACTOR, stream, true);
    k_schur_factor_levels<<<(unsigned)fblocks, 32 * kFactorWarps, fsmem, stream>>>(P);
    timing_mark(mesh, MHM_KERNEL_SCHUR_FACTOR, stream, false);
    MHM_CUDA_TRY(cudaGetLastError());
    timing_mark(mesh, MHM_KERNEL_LOCAL_MIXED, stream, true);
    k_local_mixed_levels<<<grid, kThreadsM, smem, stream>>>(P);
    timing_mark(mesh, MHM_KERNEL_LOCAL_MIXED, stream, false);
    MHM_CUDA_TRY(cudaGetLastError());
    if (opts.no_fallback) return MHM_OK;
    // elements whose refinement failed: solved again by the FP64 path, level by level
    for (int j = 0; j < n; ++j) {
        const int i = order[j];
        int32_t* fcount = reinterpret_cast<int32_t*>((char*)counters[j] + 256);
        int32_t* flist = reinterpret_cast<int32_t*>((char*)counters[j] + 512);
        const int64_t nK = r1[i] - r0[i];
        MHM_CUDA_TRY(cudaMemsetAsync(fcount, 0, sizeof(int32_t), stream));
        const int64_t nb = std::min<int64_t>((nK + 255) / 256, 1024);
        k_collect_failed<<<(unsigned)nb, 256, 0, stream>>>(P.lv[j].dm.klist, r0[i], r1[i], status, flist, fcount);
        MHM_CUDA_TRY(cudaGetLastError());
        const mhm_status st =
            launch_local_fp64_list(mesh, *lvs[i], kappa, f, flist, fcount, nK, AK, EK, BK, FK, status, iters, stream);
        if (st) return st;
    }
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
    {
        const mhm_status sst = check_source(f, "mhm_local_solve_batch_noalloc");
        if (sst) return sst;
    }
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
    // every level is checked before any is launched: the call either runs all of them or
    // launches nothing
    for (const Level& lv : mesh->levels) {
        if (fp64_level(mesh, lv)) {
            if (!fp64_level_launchable(mesh, lv))
                return fail(MHM_ERR_UNSUPPORTED, "mhm_local_solve_batch_noalloc: FP64 window panel exceeds shared memory");
            const size_t need = fp64_slot_bytes(mesh, lv);
            if (need > kStaticScratch)
                return fail(MHM_ERR_INVALID_ARG,
                            "mhm_local_solve_batch_noalloc: one coarse element's FP64 window needs " +
                                std::to_string(need) + " bytes of scratch, above the fixed " +
                                std::to_string(kStaticScratch) + " bytes");
            continue;
        }
        const MixedLayout L = mixed_layout(mesh, lv, false);   // factor inside the solve kernel
        if (L.smem > 220 * 1024 || !mixed_kernel(L))
            return fail(MHM_ERR_UNSUPPORTED, "mhm_local_solve_batch_noalloc: buffers exceed shared memory (r too large)");
        if (L.slot_bytes > kStaticScratch)
            return fail(MHM_ERR_INVALID_ARG,
                        "mhm_local_solve_batch_noalloc: one coarse element needs " + std::to_string(L.slot_bytes) +
                            " bytes of scratch, above the fixed " + std::to_string(kStaticScratch) + " bytes");
    }
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
    // one launch per refinement level, in stream order (each reuses the fixed array)
    for (const Level& lv : mesh->levels) {
        int64_t i0 = 0, i1 = 0;
        level_range(lv, K0, K1, &i0, &i1);
        const int64_t nK = i1 - i0;
        if (nK <= 0) continue;
        if (fp64_level(mesh, lv)) {   // a window wider than shared memory: as many blocks as the array holds
            const mhm_status st = launch_local_fp64(mesh, lv, kappa, *f, i0, i1, AK, EK, BK, FK, status, iters,
                                                    scratch, kStaticScratch, (cudaStream_t)stream);
            if (st) return st;
            continue;
        }
        const MixedLayout L = mixed_layout(mesh, lv, false);
        const int64_t fit = (int64_t)(kStaticScratch / L.slot_bytes);
        int64_t grid = mixed_slots(mesh, L);
        if (grid > fit) grid = fit;
        if (grid > nK) grid = nK;
        MixedArgs g = mixed_args(mesh, lv, L, kappa, *f, o, AK, EK, BK, FK, status, iters, (char*)scratch);
        g.word_final = 1;
        g.K0 = i0;
        g.K1 = i1;
        mixed_kernel(L)<<<(unsigned)grid, kThreadsM, L.smem, (cudaStream_t)stream>>>(g);
        MHM_CUDA_TRY(cudaGetLastError());
    }
    return MHM_OK;
}

}  // namespace mhm
