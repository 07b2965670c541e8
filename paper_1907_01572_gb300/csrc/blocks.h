// Block maps of multi-block meshes (Sec. II.A.1; the cubed-sphere domains of
// Sec. III) and the relative orientation of two block faces, for host code
// (connectivity) and device code (node coordinates, mortar geometry).
#pragma once
#include <cmath>

#include "dgell.h"

namespace dg {

// Frame of a wedge / shell block on cube face 2 d + s: reference axes 0, 1
// along e_t1, e_t2 and axis 2 outward (right-handed).
__host__ __device__ inline void wedge_frame(int face, int& d, double& sg, int& t1, int& t2) {
    d = face >> 1;
    if (face & 1) {
        sg = 1.0;
        t1 = (d + 1) % 3;
        t2 = (d + 2) % 3;
    } else {
        sg = -1.0;
        t1 = (d + 2) % 3;
        t2 = (d + 1) % 3;
    }
}

// x = block map of reference point xi in [-1, 1]^3.
__host__ __device__ inline void block_point(const dg_block& B, const double xi[3], double x[3]) {
    if (B.kind == DG_BLOCK_HEX8) {
        for (int i = 0; i < 3; ++i) x[i] = 0.0;
        for (int c = 0; c < 8; ++c) {
            double w = 1.0;
            for (int k = 0; k < 3; ++k) w *= ((c >> k) & 1) ? 0.5 * (1.0 + xi[k]) : 0.5 * (1.0 - xi[k]);
            for (int i = 0; i < 3; ++i) x[i] += w * B.corners[c][i];
        }
        return;
    }
    int d, t1, t2;
    double sg;
    wedge_frame(B.face, d, sg, t1, t2);
    double v[3];
    v[d] = sg;
    v[t1] = xi[0];
    v[t2] = xi[1];
    const double len = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const double t = 0.5 * (xi[2] + 1.0);
    if (B.kind == DG_BLOCK_WEDGE) {
        for (int i = 0; i < 3; ++i) x[i] = (1.0 - t) * B.a * v[i] + t * B.r * v[i] / len;
    } else {
        const double R = 1.0 / ((1.0 - t) / B.r1 + t / B.r2);
        for (int i = 0; i < 3; ++i) x[i] = R * v[i] / len;
    }
}

// J[i][l] = d x_i / d xi_l of the block map at xi, and x itself (exact
// derivatives of the formulas in block_point).
__host__ __device__ inline void block_jacobian(const dg_block& B, const double xi[3], double J[3][3], double x[3]) {
    if (B.kind == DG_BLOCK_HEX8) {
        for (int i = 0; i < 3; ++i) {
            x[i] = 0.0;
            for (int l = 0; l < 3; ++l) J[i][l] = 0.0;
        }
        for (int c = 0; c < 8; ++c) {
            double f[3], df[3];
            for (int k = 0; k < 3; ++k) {
                const bool hi = (c >> k) & 1;
                f[k] = hi ? 0.5 * (1.0 + xi[k]) : 0.5 * (1.0 - xi[k]);
                df[k] = hi ? 0.5 : -0.5;
            }
            const double w = f[0] * f[1] * f[2];
            const double dw[3] = {df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2]};
            for (int i = 0; i < 3; ++i) {
                x[i] += w * B.corners[c][i];
                for (int l = 0; l < 3; ++l) J[i][l] += dw[l] * B.corners[c][i];
            }
        }
        return;
    }
    int d, t1, t2;
    double sg;
    wedge_frame(B.face, d, sg, t1, t2);
    double v[3];
    v[d] = sg;
    v[t1] = xi[0];
    v[t2] = xi[1];
    const double len = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double u[3], du0[3], du1[3];   // u = v / |v| and its derivatives along xi_0, xi_1
    for (int i = 0; i < 3; ++i) u[i] = v[i] / len;
    for (int i = 0; i < 3; ++i) {
        du0[i] = ((i == t1 ? 1.0 : 0.0) - u[i] * u[t1]) / len;
        du1[i] = ((i == t2 ? 1.0 : 0.0) - u[i] * u[t2]) / len;
    }
    const double t = 0.5 * (xi[2] + 1.0);
    if (B.kind == DG_BLOCK_WEDGE) {
        for (int i = 0; i < 3; ++i) {
            x[i] = (1.0 - t) * B.a * v[i] + t * B.r * u[i];
            J[i][0] = (1.0 - t) * B.a * (i == t1 ? 1.0 : 0.0) + t * B.r * du0[i];
            J[i][1] = (1.0 - t) * B.a * (i == t2 ? 1.0 : 0.0) + t * B.r * du1[i];
            J[i][2] = 0.5 * (B.r * u[i] - B.a * v[i]);
        }
    } else {
        const double R = 1.0 / ((1.0 - t) / B.r1 + t / B.r2);
        const double dR = R * R * (1.0 / B.r1 - 1.0 / B.r2);   // dR / dt
        for (int i = 0; i < 3; ++i) {
            x[i] = R * u[i];
            J[i][0] = R * du0[i];
            J[i][1] = R * du1[i];
            J[i][2] = 0.5 * dR * u[i];
        }
    }
}

// H[i][l][m] = d^2 x_i / dxi_l dxi_m of the block map at xi (the second
// derivatives of the formulas in block_point, for the estimator's exact
// Laplacian of mapped polynomials).  Wedge and shell, with v linear in
// xi_0, xi_1, u = v / |v|, t = (xi_2 + 1) / 2 and a, b in {0, 1} along e_ta:
//   d_a u_i = (delta_i,ta - u_i u_ta) / |v|,
//   d_a d_b u_i = -[(d_b u_i) u_ta + u_i (d_b u_ta) + (d_a u_i) u_tb] / |v|;
//   wedge x = (1 - t) a v + t r u: d_a d_b x = t r d_a d_b u,
//     d_a d_2 x = (r d_a u - a e_ta) / 2, d_2 d_2 x = 0;
//   shell x = R(t) u: d_a d_b x = R d_a d_b u, d_a d_2 x = R' d_a u / 2,
//     d_2 d_2 x = R'' u / 4, R' = R^2 (1/r1 - 1/r2), R'' = 2 R R' (1/r1 - 1/r2).
__host__ __device__ inline void block_hessian(const dg_block& B, const double xi[3], double H[3][3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int l = 0; l < 3; ++l)
            for (int m = 0; m < 3; ++m) H[i][l][m] = 0.0;
    if (B.kind == DG_BLOCK_HEX8) {
        for (int c = 0; c < 8; ++c) {
            double f[3], df[3];
            for (int k = 0; k < 3; ++k) {
                const bool hi = (c >> k) & 1;
                f[k] = hi ? 0.5 * (1.0 + xi[k]) : 0.5 * (1.0 - xi[k]);
                df[k] = hi ? 0.5 : -0.5;
            }
            const double w01 = df[0] * df[1] * f[2], w02 = df[0] * f[1] * df[2], w12 = f[0] * df[1] * df[2];
            for (int i = 0; i < 3; ++i) {
                H[i][0][1] += w01 * B.corners[c][i];
                H[i][0][2] += w02 * B.corners[c][i];
                H[i][1][2] += w12 * B.corners[c][i];
            }
        }
        for (int i = 0; i < 3; ++i) {
            H[i][1][0] = H[i][0][1];
            H[i][2][0] = H[i][0][2];
            H[i][2][1] = H[i][1][2];
        }
        return;
    }
    int d, t1, t2;
    double sg;
    wedge_frame(B.face, d, sg, t1, t2);
    double v[3];
    v[d] = sg;
    v[t1] = xi[0];
    v[t2] = xi[1];
    const double len = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const int ta[2] = {t1, t2};
    double u[3], du[2][3], ddu[2][2][3];
    for (int i = 0; i < 3; ++i) u[i] = v[i] / len;
    for (int a = 0; a < 2; ++a)
        for (int i = 0; i < 3; ++i) du[a][i] = ((i == ta[a] ? 1.0 : 0.0) - u[i] * u[ta[a]]) / len;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int i = 0; i < 3; ++i)
                ddu[a][b][i] = -(du[b][i] * u[ta[a]] + u[i] * du[b][ta[a]] + du[a][i] * u[ta[b]]) / len;
    const double t = 0.5 * (xi[2] + 1.0);
    if (B.kind == DG_BLOCK_WEDGE) {
        for (int i = 0; i < 3; ++i) {
            for (int a = 0; a < 2; ++a) {
                for (int b = 0; b < 2; ++b) H[i][a][b] = t * B.r * ddu[a][b][i];
                H[i][a][2] = H[i][2][a] = 0.5 * (B.r * du[a][i] - B.a * (i == ta[a] ? 1.0 : 0.0));
            }
        }
    } else {
        const double k = 1.0 / B.r1 - 1.0 / B.r2;
        const double R = 1.0 / ((1.0 - t) / B.r1 + t / B.r2);
        const double dR = R * R * k, ddR = 2.0 * R * dR * k;
        for (int i = 0; i < 3; ++i) {
            for (int a = 0; a < 2; ++a) {
                for (int b = 0; b < 2; ++b) H[i][a][b] = R * ddu[a][b][i];
                H[i][a][2] = H[i][2][a] = 0.5 * dR * du[a][i];
            }
            H[i][2][2] = 0.25 * ddR * u[i];
        }
    }
}

// Relative orientation of two faces, o = swap | flip1 << 1 | flip2 << 2:
// side A's face coordinates (u, v) (along its tangential axes in increasing
// order) become side B's as (w1, w2) = swap ? (v, u) : (u, v), then w1 and w2
// mirrored where flip1 / flip2 are set.
__host__ __device__ inline void orient_coords(int o, double u, double v, double& b1, double& b2) {
    const double w1 = (o & 1) ? v : u, w2 = (o & 1) ? u : v;
    b1 = (o & 2) ? -w1 : w1;
    b2 = (o & 4) ? -w2 : w2;
}

// The same for cell indices 0..m-1 along each tangential axis.
__host__ __device__ inline void orient_cells(int o, int m, int u, int v, int& b1, int& b2) {
    const int w1 = (o & 1) ? v : u, w2 = (o & 1) ? u : v;
    b1 = (o & 2) ? m - 1 - w1 : w1;
    b2 = (o & 4) ? m - 1 - w2 : w2;
}

}  // namespace dg
