// Geometry precompute on the device, FP64 (Sec. II.A.5):
//  * node coordinates: the block map sampled at each element's LGL nodes
//    (Phi_e linear in the block coordinates, eq. Phi_e); on the single box the
//    geometry is isoparametric (the node coordinates interpolated), on block
//    meshes it is exact (x and J of the block map at every GL point);
//  * volume GL points: J = dx/dxi of the degree-p interpolant, det J, J^-1 and
//    the stiffness metric G_lm = w det J (J^-1)_l . (J^-1)_m of eq. (harald-stiff);
//  * mortar GL points (indexed in side A's face frame): S^m (eq.
//    Surface-Jacobian) and the normal from side A, and per side
//    c_l = (J^-1)_l . n_A (side B evaluated at the same point of its own,
//    possibly turned, face frame), the factors turning reference gradients
//    into the normal derivative; h = 2 J / S per side and point, and the penalty
//    sigma = C p_m^2 / min h (eq. penaltyparameter).
#include "blocks.h"
#include "geom.h"

namespace dg {
namespace {

__device__ inline double lagv(const double* x, int n, int a, double t) {
    double v = 1.0;
    for (int m = 0; m < n; ++m)
        if (m != a) v *= (t - x[m]) / (x[a] - x[m]);
    return v;
}

__device__ inline double lagd(const double* x, int n, int a, double t) {
    double s = 0.0;
    for (int m = 0; m < n; ++m) {
        if (m == a) continue;
        double term = 1.0 / (x[a] - x[m]);
        for (int k = 0; k < n; ++k)
            if (k != a && k != m) term *= (t - x[k]) / (x[a] - x[k]);
        s += term;
    }
    return s;
}

__device__ inline void tangential(int d, int& t1, int& t2) {
    t1 = d == 0 ? 1 : 0;
    t2 = d == 2 ? 1 : 2;
}

__device__ inline double submap(int pos, double s) { return pos == 0 ? s : (pos == 1 ? 0.5 * (s - 1.0) : 0.5 * (s + 1.0)); }

// J[i][l] = d x_i / d xi_l at reference point xi of element e (dense sum over nodes)
__device__ void jacobian_at(const double* X, int n, const double* xl, const double xi[3], double J[3][3],
                            double xphys[3]) {
    double L[3][kMaxN], dL[3][kMaxN];
    for (int d = 0; d < 3; ++d)
        for (int a = 0; a < n; ++a) {
            L[d][a] = lagv(xl, n, a, xi[d]);
            dL[d][a] = lagd(xl, n, a, xi[d]);
        }
    const int n3 = n * n * n;
    for (int i = 0; i < 3; ++i) {
        xphys[i] = 0.0;
        for (int l = 0; l < 3; ++l) J[i][l] = 0.0;
    }
    for (int c = 0; c < n; ++c)
        for (int b = 0; b < n; ++b)
            for (int a = 0; a < n; ++a) {
                const int node = a + n * (b + n * c);
                const double w0 = L[0][a] * L[1][b] * L[2][c];
                const double w1 = dL[0][a] * L[1][b] * L[2][c];
                const double w2 = L[0][a] * dL[1][b] * L[2][c];
                const double w3 = L[0][a] * L[1][b] * dL[2][c];
                for (int i = 0; i < 3; ++i) {
                    const double xv = X[i * n3 + node];
                    xphys[i] += w0 * xv;
                    J[i][0] += w1 * xv;
                    J[i][1] += w2 * xv;
                    J[i][2] += w3 * xv;
                }
            }
}

// Geometry of element e at reference point xi: on block meshes the exact map
// (block map composed with the element's linear map into its block, J scaled
// by 2^-level); on the single box the isoparametric interpolant of the node
// coordinates X.
__device__ void elem_geom(const GeomArgs& g, const double* X, int e, const double xi[3], double J[3][3],
                          double xp[3]) {
    if (g.n_blocks > 0) {
        const int* lf = g.leaves + 4 * e;
        const double inv = 1.0 / (double)(1 << lf[0]);
        double xb[3];
        for (int d = 0; d < 3; ++d) xb[d] = -1.0 + (2.0 * lf[1 + d] + xi[d] + 1.0) * inv;
        block_jacobian(g.blocks[g.block[e]], xb, J, xp);
        for (int i = 0; i < 3; ++i)
            for (int l = 0; l < 3; ++l) J[i][l] *= inv;
        return;
    }
    const int n = g.p[e] + 1;
    jacobian_at(X + 3 * g.dof_off[e], n, g.tab + tab_n(TabIndex::LGLx, n), xi, J, xp);
}

__device__ inline double inv3(const double J[3][3], double Ji[3][3]) {
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    const double r = 1.0 / det;
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * r;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * r;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * r;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * r;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * r;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * r;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * r;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * r;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * r;
    return det;
}

__global__ void node_coords_kernel(GeomArgs g, double* X) {
    const int e = blockIdx.x;
    if (e >= g.n_elems) return;
    const int n = g.p[e] + 1, n3 = n * n * n;
    const int* lf = g.leaves + 4 * e;
    const double* xl = g.tab + tab_n(TabIndex::LGLx, n);
    double lo[3], w[3];
    for (int d = 0; d < 3; ++d) {
        w[d] = (g.hi[d] - g.lo[d]) / (double)(1 << lf[0]);
        lo[d] = g.lo[d] + w[d] * lf[1 + d];
    }
    double* Xe = X + 3 * g.dof_off[e];
    if (g.n_blocks > 0) {   // block reference point of the node, then the block map
        const dg_block& B = g.blocks[g.block[e]];
        const double inv = 1.0 / (double)(1 << lf[0]);
        for (int k = threadIdx.x; k < n3; k += blockDim.x) {
            const int a = k % n, b = (k / n) % n, c = k / (n * n);
            const double xi[3] = {xl[a], xl[b], xl[c]};
            double xb[3], y[3];
            for (int d = 0; d < 3; ++d) xb[d] = -1.0 + (2.0 * lf[1 + d] + xi[d] + 1.0) * inv;
            block_point(B, xb, y);
            for (int d = 0; d < 3; ++d) Xe[d * n3 + k] = y[d];
        }
        return;
    }
    for (int k = threadIdx.x; k < n3; k += blockDim.x) {
        const int a = k % n, b = (k / n) % n, c = k / (n * n);
        const double xi[3] = {xl[a], xl[b], xl[c]};
        double x[3];
        for (int d = 0; d < 3; ++d) x[d] = lo[d] + 0.5 * (xi[d] + 1.0) * w[d];
        double y[3] = {x[0], x[1], x[2]};
        if (g.map_kind == DG_MAP_SINE_WARP) {
            for (int i = 0; i < 3; ++i) {
                const int j = (i + 1) % 3;
                y[i] = x[i] + g.warp_amp * sin(2.0 * M_PI * g.warp_k[i] * x[i]) * sin(2.0 * M_PI * g.warp_k[j] * x[j]);
            }
        }
        for (int d = 0; d < 3; ++d) Xe[d * n3 + k] = y[d];
    }
}

__global__ void volume_geom_kernel(GeomArgs g, const double* X, double* G, double* wdetJ, double* vxyz,
                                   long long n_vqp, int* bad) {
    const int e = blockIdx.x;
    if (e >= g.n_elems) return;
    const int n = g.p[e] + 1, n3 = n * n * n;
    const double* xg = g.tab + tab_n(TabIndex::GLx, n);
    const double* wg = g.tab + tab_n(TabIndex::GLw, n);
    const long long vo = g.vqp_off[e];
    for (int k = threadIdx.x; k < n3; k += blockDim.x) {
        const int i = k % n, j = (k / n) % n, l = k / (n * n);
        const double xi[3] = {xg[i], xg[j], xg[l]};
        double J[3][3], Ji[3][3], xp[3];
        elem_geom(g, X, e, xi, J, xp);
        const double det = inv3(J, Ji);
        if (!(det > 0.0)) atomicExch(bad, 1);
        const double wd = wg[i] * wg[j] * wg[l] * det;
        double* Ge = G + 6 * vo;
        int c = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = a; b < 3; ++b) {
                const double s = Ji[a][0] * Ji[b][0] + Ji[a][1] * Ji[b][1] + Ji[a][2] * Ji[b][2];
                Ge[c * n3 + k] = wd * s;
                ++c;
            }
        wdetJ[vo + k] = wd;
        for (int d = 0; d < 3; ++d) vxyz[d * n_vqp + vo + k] = xp[d];
    }
}

__global__ void mortar_geom_kernel(GeomArgs g, const double* X, const Mortar* mortars, int n_mortars, double C,
                                   double* mg, double* sigma, double* bxyz, long long n_bnd, int* bad) {
    const int mi = blockIdx.x;
    if (mi >= n_mortars) return;
    const Mortar M = mortars[mi];
    const int q = M.q, q2 = q * q;
    const double* sg = g.tab + tab_n(TabIndex::GLx, q);
    const double* wq = g.tab + tab_n(TabIndex::GLw, q);
    __shared__ double hmin[128];
    double my_h = 1e300;
    for (int k = threadIdx.x; k < q2; k += blockDim.x) {
        const int i1 = k % q, i2 = k / q;
        double nA[3];
        {   // side A: normal, surface Jacobian, metric
            const int e = M.eA;
            const int d = M.fA >> 1, s = M.fA & 1;
            int t1, t2;
            tangential(d, t1, t2);
            double xi[3];
            xi[d] = s ? 1.0 : -1.0;
            xi[t1] = submap(M.posA0, sg[i1]);
            xi[t2] = submap(M.posA1, sg[i2]);
            double J[3][3], Ji[3][3], xp[3];
            elem_geom(g, X, e, xi, J, xp);
            const double det = inv3(J, Ji);
            if (!(det > 0.0)) atomicExch(bad, 1);
            const double nrm = sqrt(Ji[d][0] * Ji[d][0] + Ji[d][1] * Ji[d][1] + Ji[d][2] * Ji[d][2]);
            const double S = det * nrm;
            const double sgn = s ? 1.0 : -1.0;
            for (int i = 0; i < 3; ++i) nA[i] = sgn * Ji[d][i] / nrm;
            double* mgm = mg + 7 * M.goff;
            mgm[0 * q2 + k] = wq[i1] * wq[i2] * S;
            for (int l = 0; l < 3; ++l) mgm[(1 + l) * q2 + k] = Ji[l][0] * nA[0] + Ji[l][1] * nA[1] + Ji[l][2] * nA[2];
            my_h = fmin(my_h, 2.0 / nrm);
            if (M.eB < 0) {
                for (int l = 0; l < 3; ++l) mgm[(4 + l) * q2 + k] = 0.0;
                for (int dd = 0; dd < 3; ++dd) bxyz[dd * n_bnd + M.bnd_off + k] = xp[dd];
            }
        }
        if (M.eB >= 0) {
            const int e = M.eB;
            const int d = M.fB >> 1, s = M.fB & 1;
            int t1, t2;
            tangential(d, t1, t2);
            double xi[3], b1, b2;
            orient_coords(M.orient, sg[i1], sg[i2], b1, b2);   // this point in side B's face frame
            xi[d] = s ? 1.0 : -1.0;
            xi[t1] = submap(M.posB0, b1);
            xi[t2] = submap(M.posB1, b2);
            double J[3][3], Ji[3][3], xp[3];
            elem_geom(g, X, e, xi, J, xp);
            const double det = inv3(J, Ji);
            if (!(det > 0.0)) atomicExch(bad, 1);
            const double nrm = sqrt(Ji[d][0] * Ji[d][0] + Ji[d][1] * Ji[d][1] + Ji[d][2] * Ji[d][2]);
            double* mgm = mg + 7 * M.goff;
            for (int l = 0; l < 3; ++l) mgm[(4 + l) * q2 + k] = Ji[l][0] * nA[0] + Ji[l][1] * nA[1] + Ji[l][2] * nA[2];
            my_h = fmin(my_h, 2.0 / nrm);
        }
    }
    hmin[threadIdx.x] = my_h;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) hmin[threadIdx.x] = fmin(hmin[threadIdx.x], hmin[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double pm = q - 1;
        sigma[mi] = C * pm * pm / hmin[0];
    }
}

}  // namespace

cudaError_t launch_node_coords(const GeomArgs& g, double* X, cudaStream_t st) {
    node_coords_kernel<<<g.n_elems, 128, 0, st>>>(g, X);
    return cudaGetLastError();
}

cudaError_t launch_volume_geom(const GeomArgs& g, const double* X, double* G, double* wdetJ, double* vxyz,
                               long long n_vqp, int* bad, cudaStream_t st) {
    volume_geom_kernel<<<g.n_elems, 128, 0, st>>>(g, X, G, wdetJ, vxyz, n_vqp, bad);
    return cudaGetLastError();
}

cudaError_t launch_mortar_geom(const GeomArgs& g, const double* X, const Mortar* mortars, int n_mortars, double C,
                               double* mg, double* sigma, double* bxyz, long long n_bnd, int* bad, cudaStream_t st) {
    if (n_mortars == 0) return cudaSuccess;
    mortar_geom_kernel<<<n_mortars, 128, 0, st>>>(g, X, mortars, n_mortars, C, mg, sigma, bxyz, n_bnd, bad);
    return cudaGetLastError();
}

}  // namespace dg
