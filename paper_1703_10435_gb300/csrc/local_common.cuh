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
