// computeSolution (Alg. 1; Sec. 2, Eq. "u_Hh"; Sec. 3): on every coarse
// triangle K,  u_{H,h} = u0_K + sum_i k_i eta_i + eta_f.  By linearity this is
// one zero-mean Neumann solve per K with the combined load
//     g = sum_i k_i N~_i + f~      (k_i: global multipliers of K's local basis),
// done here in FP64: the level-window Cholesky of the FP64 kernel with one
// right-hand side, storing L_lev and L_{lev+1,lev} per level in scratch, then a
// backward sweep by one warp.  Optional per-K squared L2 and broken-H1 errors
// against an exact solution by the collapsed 4 x 4 Gauss rule per fine triangle.
// Windows too large for shared memory (P1 r = 7, P2 r = 5) sit in the block's
// scratch slot behind the stored factors and are factored panel by panel
// (wide_cholesky_level).
#include <cuda_runtime.h>

#include "local_common.cuh"

namespace mhm {

namespace {

constexpr int kThreadsR = 128;
constexpr int kThreadsRWide = 256;
constexpr int kNBR = 16;   // wide window: pivots per panel

struct RecArgs {
    DeviceMesh dm;
    const double* kappa;
    const double* lambda;
    const double* u0;
    const int32_t* k_lambda;    // n_K * N_I global multiplier ids
    int P, N, PN, dpf, NI, nlev, nloc;
    int rows, ld, rhs;          // window rows, leading dimension, right-hand-side column
    int src_kind;
    const double* src_vals;   // MHM_SRC_QUAD: 16 values per fine triangle, laid out like kappa
    double src_value, src_freq;
    int ex_kind;                // 0 none, 1 sin sin, 2 quadratic polynomial
    double ex[6];
    char* ws;
    size_t slot_bytes;
    size_t win_offset;          // wide window: its byte offset in the slot (0: shared memory)
    int64_t nK;                 // launch indices of this level
    const int64_t* nod_off;     // first nodal value of each K in u_out (NULL: K * nloc)
    double* u_out;              // n_K * nloc (per-K levels: at nod_off)
    double* err_out;            // n_K * 2 (squared L2, squared H1 seminorm) or NULL
};

struct RCtx {
    double X[3][2];
    double Sup[36], Sdn[36];
    double area, area_fine, FK, cl;
    double flen[3];
    int sgn[3], rev[3], la1[3];  // la1: degree + 1 of each face
    int bad;
    int pin_x, pin_y;            // the pinned lattice point (choose_pin)
    double red[kThreadsRWide / 32];
    double mz;
};

__device__ __forceinline__ void fine_xy(const RCtx& c, int N, bool up, int i, int j, double X[3][2]) {
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

__device__ __forceinline__ void basis_eval(int P, double l0, double l1, double l2, double* phi, double* dxi,
                                           double* deta) {
    if (P == 1) {
        phi[0] = l0; phi[1] = l1; phi[2] = l2;
        dxi[0] = -1; dxi[1] = 1; dxi[2] = 0;
        deta[0] = -1; deta[1] = 0; deta[2] = 1;
        return;
    }
    phi[0] = l0 * (2 * l0 - 1); phi[1] = l1 * (2 * l1 - 1); phi[2] = l2 * (2 * l2 - 1);
    phi[3] = 4 * l1 * l2; phi[4] = 4 * l2 * l0; phi[5] = 4 * l0 * l1;
    dxi[0] = -(4 * l0 - 1); deta[0] = -(4 * l0 - 1);
    dxi[1] = 4 * l1 - 1;    deta[1] = 0;
    dxi[2] = 0;             deta[2] = 4 * l2 - 1;
    dxi[3] = 4 * l2;        deta[3] = 4 * l1;
    dxi[4] = -4 * l2;       deta[4] = 4 * (l0 - l2);
    dxi[5] = 4 * (l0 - l1); deta[5] = -4 * l1;
}

// Integral of f phi_a (a >= 0) or of f (a < 0) over a fine triangle, 4 x 4 collapsed Gauss.
__device__ double cell_source(const RecArgs& g, const double X[3][2], int a, const double* fq) {
    const double* gx = g.dm.gauss_x + 3 * kMaxGauss;
    const double* gw = g.dm.gauss_w + 3 * kMaxGauss;
    const double adet = fabs((X[1][0] - X[0][0]) * (X[2][1] - X[0][1]) - (X[2][0] - X[0][0]) * (X[1][1] - X[0][1]));
    double s = 0.0;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            const double xi = gx[i], eta = gx[j] * (1.0 - gx[i]), w = gw[i] * gw[j] * (1.0 - gx[i]);
            const double x = X[0][0] + xi * (X[1][0] - X[0][0]) + eta * (X[2][0] - X[0][0]);
            const double y = X[0][1] + xi * (X[1][1] - X[0][1]) + eta * (X[2][1] - X[0][1]);
            double phi[6], dx[6], dy[6];
            basis_eval(g.P, 1.0 - xi - eta, xi, eta, phi, dx, dy);
            s += w * adet * source_at(g.src_kind, g.src_value, g.src_freq, x, y, fq, 4 * i + j) * (a >= 0 ? phi[a] : 1.0);
        }
    return s;
}

__device__ void exact_eval(const RecArgs& g, double x, double y, double* u, double* ux, double* uy) {
    if (g.ex_kind == 1) {
        const double f = g.ex[0], amp = g.ex[1];
        const double sx = sinpi(f * x), sy = sinpi(f * y), cx = cospi(f * x), cy = cospi(f * y);
        *u = amp * sx * sy;
        *ux = amp * f * M_PI * cx * sy;
        *uy = amp * f * M_PI * sx * cy;
    } else {
        const double* c = g.ex;
        *u = c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y;
        *ux = c[1] + 2 * c[3] * x + c[4] * y;
        *uy = c[2] + c[4] * x + 2 * c[5] * y;
    }
}

__device__ double block_sum(double v, RCtx& c) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) c.red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += c.red[w];   // same order in every thread
    __syncthreads();
    return s;
}

template <bool WIDE>
__global__ void __launch_bounds__(WIDE ? kThreadsRWide : kThreadsR) k_reconstruct(const RecArgs g) {
    extern __shared__ double smem[];
    __shared__ RCtx c;
    const int rhs = g.rhs;
    char* slot = g.ws + (size_t)blockIdx.x * g.slot_bytes;
    double* Fst = reinterpret_cast<double*>(slot);   // per level: L (b x b), C (bn x b), y (b)
    // window rows x ld (column rhs is the right-hand side): shared memory or the slot
    double* W = WIDE ? reinterpret_cast<double*>(slot + g.win_offset) : smem;
    double* zs = WIDE ? smem : smem + (size_t)g.rows * g.ld;   // nloc: the solution z (pinned DOF 0 = 0)
    double* Ps = smem + (((size_t)g.nloc + 1) & ~(size_t)1);   // (wide) panel, 16-byte aligned
    double* Rs = Ps + (size_t)g.rows * wide_panel_stride<kNBR>();
    double* invd = Rs + kNBR;
    const int nb = g.P == 1 ? 3 : 6, npair = nb * (nb + 1) / 2;

    for (int64_t ki = blockIdx.x; ki < g.nK; ki += gridDim.x) {
        const int64_t K = g.dm.klist ? (int64_t)g.dm.klist[ki] : ki;      // coarse element
        const double* kap = g.kappa + (g.dm.kap_off ? g.dm.kap_off[K] : K * (int64_t)g.N * g.N);
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
            // sum_i k_i c_i, c_i = (1^T N_i) / |K| = -s |F| int psi / |K|
            double cl = 0.0;
            for (int i = 0; i < g.NI; ++i) {
                const int a = i / g.dpf, jf = i - a * g.dpf;
                const int row = face_row(jf, c.la1[a], g.dm.fm, g.dm.lmax1);
                if (row < 0) continue;   // unused slot
                cl += g.lambda[g.k_lambda[K * g.NI + i]] * (-c.sgn[a] * c.flen[a] * g.dm.btab_sum[row] / c.area);
            }
            c.cl = cl;
            c.bad = 0;
            choose_pin(g.P, g.N, kap, &c.pin_x, &c.pin_y);
        }
        __syncthreads();
        const LevelGeom lg{g.P, g.N, g.PN, c.pin_x, c.pin_y};
        double fk = 0.0;
        if (g.src_kind == MHM_SRC_CONST) fk = g.src_value * c.area;
        else {
            double s = 0.0;
            for (int t = threadIdx.x; t < g.N * g.N; t += blockDim.x) {
                int j = 0, rs = 0;
                while (rs + 2 * (g.N - j) - 1 <= t) { rs += 2 * (g.N - j) - 1; ++j; }
                const int o = t - rs;
                const bool up = o < g.N - j;
                double X[3][2];
                fine_xy(c, g.N, up, up ? o : o - (g.N - j), j, X);
                s += cell_source(g, X, -1, quad_of(g.src_vals, g.kappa, kap, g.N, up, up ? o : o - (g.N - j), j));
            }
            fk = block_sum(s, c);
        }
        const double cm = fk / c.area + c.cl;     // coefficient of the mass vector in g
        const int b0 = lg.size(0), b1 = g.nlev > 1 ? lg.size(1) : 0;
        for (int t = threadIdx.x; t < (b0 + b1) * g.ld; t += blockDim.x) W[t] = 0.0;
        __syncthreads();
        size_t foff = 0;
        for (int lev = 0; lev < g.nlev; ++lev) {
            const int b = lg.size(lev);
            const int bn = lev + 1 < g.nlev ? lg.size(lev + 1) : 0;
            const int nr = b + bn;
            // boundary loads sum_j k_j N_j of the fresh points (level 0 at the start too)
            for (int pass = (lev == 0 ? 0 : 1); pass < 2; ++pass) {
                const int l2 = lev + pass, row0 = pass ? b : 0;
                if (l2 >= g.nlev) continue;
                for (int p = threadIdx.x; p < lg.size(l2); p += blockDim.x) {
                    int x, y;
                    lg.point(l2, p, &x, &y);
                    double v = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        const int kl = face_position(g.PN, x, y, a);
                        if (kl < 0) continue;
                        const int kk = c.rev[a] ? g.PN - kl : kl;
                        for (int jf = 0; jf < g.dpf; ++jf) {
                            const int row = face_row(jf, c.la1[a], g.dm.fm, g.dm.lmax1);
                            if (row < 0) continue;   // unused slot
                            v += g.lambda[g.k_lambda[K * g.NI + a * g.dpf + jf]] *
                                 (-c.sgn[a] * c.flen[a] * g.dm.btab[row * (g.PN + 1) + kk]);
                        }
                    }
                    W[(row0 + p) * g.ld + rhs] += v;
                }
                __syncthreads();
            }
            if (bn > 0) {
                // element matrices and loads of fine row lev, four colour classes
                for (int cls = 0; cls < 4; ++cls) {
                    const bool up = cls < 2;
                    const int parity = cls & 1;
                    const int ntri = up ? g.N - lev : g.N - 1 - lev;
                    const int ncls = (ntri - parity + 1) / 2;
                    const int per = npair + nb;
                    for (int t = threadIdx.x; t < ncls * per; t += blockDim.x) {
                        const int ti = t / per, item = t - ti * per;
                        const int i = parity + 2 * ti;
                        int nx[6], ny[6];
                        element_nodes(g.P, up, i, lev, nx, ny);
                        const double kt = kap[lev * (2 * g.N - lev) + (up ? i : (g.N - lev) + i)];
                        const double* S = up ? c.Sup : c.Sdn;
                        if (item < npair) {
                            int a = 0, rem = item;
                            while (rem >= nb - a) { rem -= nb - a; ++a; }
                            const int bb = a + rem;
                            const int pa = lg.pos(nx[a], ny[a]), pb = lg.pos(nx[bb], ny[bb]);
                            if (pa < 0 || pb < 0) continue;
                            const int ra = pa + (lg.level_of_row(ny[a]) == lev ? 0 : b);
                            const int rb = pb + (lg.level_of_row(ny[bb]) == lev ? 0 : b);
                            W[max(ra, rb) * g.ld + min(ra, rb)] += kt * S[a * nb + bb];
                        } else {
                            const int a = item - npair;
                            const int pa = lg.pos(nx[a], ny[a]);
                            if (pa < 0) continue;
                            const int ra = pa + (lg.level_of_row(ny[a]) == lev ? 0 : b);
                            const double mass = c.area_fine * element_mass_frac(g.P, a);
                            double v = -cm * mass;
                            if (g.src_kind == MHM_SRC_CONST) v += g.src_value * mass;
                            else {
                                double X[3][2];
                                fine_xy(c, g.N, up, i, lev, X);
                                v += cell_source(g, X, a, quad_of(g.src_vals, g.kappa, kap, g.N, up, i, lev));
                            }
                            W[ra * g.ld + rhs] += v;
                        }
                    }
                    __syncthreads();
                }
            }
            if constexpr (WIDE)
                wide_cholesky_level<kNBR>(W, g.ld, b, nr, W + rhs, g.ld, nr, 1, &c.bad, Ps, Rs, invd, nullptr);
            else
                blocked_cholesky_level<double, 8, 4, 1>(W, g.ld, b, nr, W + rhs, g.ld, nr, 1, &c.bad);
            // keep L_lev, L_{lev+1,lev} and y_lev for the backward sweep
            for (int t = threadIdx.x; t < b * b + bn * b + b; t += blockDim.x) {
                double v;
                if (t < b * b) { const int i = t / b, k = t - i * b; v = k <= i ? W[i * g.ld + k] : 0.0; }
                else if (t < b * b + bn * b) { const int q = t - b * b, i = q / b, k = q - i * b; v = W[(b + i) * g.ld + k]; }
                else v = W[(t - b * b - bn * b) * g.ld + rhs];
                Fst[foff + t] = v;
            }
            foff += (size_t)b * b + (size_t)bn * b + b;
            __syncthreads();
            if (bn > 0) {
                for (int t = threadIdx.x; t < bn * bn; t += blockDim.x) {
                    const int i = t / bn, jj = t - i * bn;
                    if (jj <= i) W[i * g.ld + jj] = W[(b + i) * g.ld + b + jj];
                }
                for (int t = threadIdx.x; t < bn; t += blockDim.x) W[t * g.ld + rhs] = W[(b + t) * g.ld + rhs];
                __syncthreads();
                const int bnn = lev + 2 < g.nlev ? lg.size(lev + 2) : 0;
                for (int t = threadIdx.x; t < bnn * g.ld; t += blockDim.x) W[bn * g.ld + t] = 0.0;
                __syncthreads();
            }
        }
        // backward sweep x_lev = L_lev^{-T} (y_lev - L_{lev+1,lev}^T x_{lev+1}) by warp 0
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            size_t off = foff;
            int bnext = 0, u0n = 0;
            int ustart = g.nloc - 1;   // unknowns 0..nloc-2 at zs[1 ..]
            for (int lev = g.nlev - 1; lev >= 0; --lev) {
                const int b = lg.size(lev);
                const int bn = lev + 1 < g.nlev ? lg.size(lev + 1) : 0;
                off -= (size_t)b * b + (size_t)bn * b + b;
                const double* Lm = Fst + off;
                const double* Cm = Lm + (size_t)b * b;
                const double* yv = Cm + (size_t)bn * b;
                ustart -= b;
                for (int k = lane; k < b; k += 32) {
                    double t = yv[k];
                    for (int i = 0; i < bnext; ++i) t -= Cm[i * b + k] * zs[1 + u0n + i];
                    zs[1 + ustart + k] = t;
                }
                __syncwarp();
                for (int k = b - 1; k >= 0; --k) {
                    const double xk = zs[1 + ustart + k] / Lm[k * b + k];
                    __syncwarp();
                    for (int i = lane; i < k; i += 32) zs[1 + ustart + i] -= Lm[k * b + i] * xk;
                    if (lane == 0) zs[1 + ustart + k] = xk;
                    __syncwarp();
                }
                bnext = b;
                u0n = ustart;
            }
            // zs[1 + u] holds unknown u; the unknowns are the local DOFs in order without the
            // pinned one: shift the DOFs before it down by one and set the pinned DOF to 0
            const int pd = lg.pin_y * (g.PN + 1) - lg.pin_y * (lg.pin_y - 1) / 2 + lg.pin_x;
            for (int base = 0; base < pd; base += 32) {
                const double v = base + lane < pd ? zs[base + lane + 1] : 0.0;
                __syncwarp();
                if (base + lane < pd) zs[base + lane] = v;
                __syncwarp();
            }
            if (lane == 0) zs[pd] = 0.0;
        }
        __syncthreads();
        // zero mean: eta = z - (m^T z) / |K|, m_w = sum of int phi_w over the fine triangles
        double mzp = 0.0;
        for (int t = threadIdx.x; t < g.N * g.N; t += blockDim.x) {
            int j = 0, rs = 0;
            while (rs + 2 * (g.N - j) - 1 <= t) { rs += 2 * (g.N - j) - 1; ++j; }
            const int o = t - rs;
            const bool up = o < g.N - j;
            int nx[6], ny[6];
            element_nodes(g.P, up, up ? o : o - (g.N - j), j, nx, ny);
            for (int a = 0; a < nb; ++a) {
                const int dof = ny[a] * (g.PN + 1) - ny[a] * (ny[a] - 1) / 2 + nx[a];
                mzp += c.area_fine * element_mass_frac(g.P, a) * zs[dof];
            }
        }
        const double shift = g.u0[K] - block_sum(mzp, c) / c.area;
        double* uK = g.u_out + (g.nod_off ? g.nod_off[K] : K * (int64_t)g.nloc);
        for (int w = threadIdx.x; w < g.nloc; w += blockDim.x) uK[w] = zs[w] + shift;
        if (g.err_out) {
            const double* gx = g.dm.gauss_x + 3 * kMaxGauss;
            const double* gw = g.dm.gauss_w + 3 * kMaxGauss;
            double e2 = 0.0, h2 = 0.0;
            for (int t = threadIdx.x; t < g.N * g.N; t += blockDim.x) {
                int j = 0, rs = 0;
                while (rs + 2 * (g.N - j) - 1 <= t) { rs += 2 * (g.N - j) - 1; ++j; }
                const int o = t - rs;
                const bool up = o < g.N - j;
                const int i = up ? o : o - (g.N - j);
                int nx[6], ny[6];
                element_nodes(g.P, up, i, j, nx, ny);
                double X[3][2];
                fine_xy(c, g.N, up, i, j, X);
                const double j00 = X[1][0] - X[0][0], j10 = X[1][1] - X[0][1];
                const double j01 = X[2][0] - X[0][0], j11 = X[2][1] - X[0][1];
                const double det = j00 * j11 - j01 * j10;
                double uv[6];
                for (int a = 0; a < nb; ++a)
                    uv[a] = zs[ny[a] * (g.PN + 1) - ny[a] * (ny[a] - 1) / 2 + nx[a]] + shift;
                for (int qi = 0; qi < 4; ++qi)
                    for (int qj = 0; qj < 4; ++qj) {
                        const double xi = gx[qi], eta = gx[qj] * (1.0 - gx[qi]);
                        const double w = gw[qi] * gw[qj] * (1.0 - gx[qi]) * fabs(det);
                        double phi[6], dxi[6], deta[6];
                        basis_eval(g.P, 1.0 - xi - eta, xi, eta, phi, dxi, deta);
                        double uh = 0.0, gxi = 0.0, geta = 0.0;
                        for (int a = 0; a < nb; ++a) {
                            uh += phi[a] * uv[a];
                            gxi += dxi[a] * uv[a];
                            geta += deta[a] * uv[a];
                        }
                        // grad_x = J^{-T} grad_ref
                        const double ux = (j11 * gxi - j10 * geta) / det, uy = (-j01 * gxi + j00 * geta) / det;
                        const double x = X[0][0] + xi * j00 + eta * j01, y = X[0][1] + xi * j10 + eta * j11;
                        double ue, uex, uey;
                        exact_eval(g, x, y, &ue, &uex, &uey);
                        e2 += w * (uh - ue) * (uh - ue);
                        h2 += w * ((ux - uex) * (ux - uex) + (uy - uey) * (uy - uey));
                    }
            }
            const double E2 = block_sum(e2, c), H2 = block_sum(h2, c);
            if (threadIdx.x == 0) {
                g.err_out[2 * K] = E2;
                g.err_out[2 * K + 1] = H2;
            }
        }
        __syncthreads();
    }
}

}  // namespace

}  // namespace mhm

using namespace mhm;

extern "C" mhm_status mhm_reconstruct(const mhm_mesh* mesh, const double* kappa, const mhm_source* f,
                                      const double* lambda, const double* u0, const mhm_exact* exact,
                                      double* u_nodal, double* err_sq, void* stream) {
    if (!mesh) return fail(MHM_ERR_INVALID_ARG, "mhm_reconstruct: NULL mesh");
    if (mesh->device < 0) return fail(MHM_ERR_UNSUPPORTED, "mhm_reconstruct: mesh was created without a device");
    if (!kappa || !f || !lambda || !u0 || !u_nodal) return fail(MHM_ERR_INVALID_ARG, "mhm_reconstruct: NULL pointer argument");
    if (err_sq && !exact) return fail(MHM_ERR_INVALID_ARG, "mhm_reconstruct: err_sq needs an exact solution");
    {
        const mhm_status sst = check_source(f, "mhm_reconstruct");
        if (sst) return sst;
    }
    if (exact && exact->kind != MHM_EXACT_SINSIN && exact->kind != MHM_EXACT_POLY)
        return fail(MHM_ERR_INVALID_ARG, "mhm_reconstruct: unknown exact-solution kind");
    MHM_CUDA_TRY(cudaSetDevice(mesh->device));
    cudaStream_t s = (cudaStream_t)stream;
    // one launch per refinement level, in stream order
    for (const Level& lv : mesh->levels) {
        RecArgs g;
        g.dm = mesh->dev(lv);
        g.kappa = kappa;
        g.lambda = lambda;
        g.u0 = u0;
        g.k_lambda = mesh->d_k_lambda;
        g.P = mesh->desc.degree;
        g.N = lv.N;
        g.PN = lv.PN;
        g.dpf = mesh->dpf;
        g.NI = (int)mesh->NI;
        g.nlev = lv.N + 1;
        g.nloc = (int)lv.nloc;
        auto size = [&](int lev) {
            if (g.P == 1) return g.N + 1 - lev - (lev == 0);
            if (lev == g.N) return 1;
            return (2 * g.N - 2 * lev + 1) + (2 * g.N - 2 * lev) - (lev == 0);
        };
        g.rows = size(0) + (g.N >= 1 ? size(1) : 0);
        g.rhs = g.rows;                      // right-hand side right after the symmetric part
        g.ld = (g.rows + 2) & ~1;            // even: 16-byte rows for the vector panel loads
        g.src_kind = f->kind;
        g.src_vals = f->kind == MHM_SRC_QUAD ? f->values_dev : nullptr;
        g.src_value = f->value;
        g.src_freq = f->freq;
        g.ex_kind = exact ? (exact->kind == MHM_EXACT_SINSIN ? 1 : 2) : 0;
        for (int i = 0; i < 6; ++i) g.ex[i] = exact ? exact->c[i] : 0.0;
        size_t per = 0;
        for (int lev = 0; lev < g.nlev; ++lev) {
            const int b = size(lev), bn = lev + 1 < g.nlev ? size(lev + 1) : 0;
            per += (size_t)b * b + (size_t)bn * b + b;
        }
        g.slot_bytes = ((per * sizeof(double)) + 255) & ~(size_t)255;
        g.nK = lv.nK;
        g.nod_off = mesh->d_nod_off;
        g.u_out = u_nodal;
        g.err_out = err_sq;
        size_t smem = ((size_t)g.rows * g.ld + (size_t)g.nloc) * sizeof(double);
        const bool wide = g.rows > 128 || smem > 220 * 1024;
        g.win_offset = 0;
        if (wide) {
            // the window behind the stored factors in the slot; shared memory keeps z and the panel
            g.win_offset = g.slot_bytes;
            g.slot_bytes += (((size_t)g.rows * g.ld * sizeof(double)) + 255) & ~(size_t)255;
            smem = ((((size_t)g.nloc + 1) & ~(size_t)1) + (size_t)g.rows * wide_panel_stride<kNBR>() + 2 * kNBR) *
                   sizeof(double);
        }
        if (smem > 220 * 1024) return fail(MHM_ERR_UNSUPPORTED, "mhm_reconstruct: window exceeds shared memory");
        void (*kern)(const RecArgs) = wide ? k_reconstruct<true> : k_reconstruct<false>;
        const int threads = wide ? kThreadsRWide : kThreadsR;
        MHM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int sms = 0, occ = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, mesh->device);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
        int64_t grid = (int64_t)sms * (occ > 0 ? occ : 1);
        if (grid > lv.nK) grid = lv.nK;
        char* ws = nullptr;
        cudaError_t e = cudaMallocAsync((void**)&ws, (size_t)grid * g.slot_bytes, s);
        if (e != cudaSuccess) return cuda_fail(e, "mhm_reconstruct: cudaMallocAsync");
        g.ws = ws;
        kern<<<(unsigned)grid, threads, smem, s>>>(g);
        e = cudaGetLastError();
        cudaFreeAsync(ws, s);
        if (e != cudaSuccess) return cuda_fail(e, "mhm_reconstruct: launch");
    }
    return MHM_OK;
}
