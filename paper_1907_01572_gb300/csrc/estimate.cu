// A-posteriori error estimator (Sec. II.D): eta^2(e) of eq. (Eta2_Local) with
// the ingredients of eq. (Eta2_Ingredients) and the weights of eq.
// (Eta2_Integrals), for -Lap u + f u = g with Dirichlet data g_D.
//
// One CTA per element, one volume GL point per thread.  The element residual
// R = f u - g - Lap u needs the exact Laplacian of the mapped polynomial:
// with J = dx/dxi, H the reference Hessian of u and X^k the reference Hessian
// of the coordinate x_k (all polynomials of the element's LGL basis),
//   Hess_x u = J^-T (H - sum_k (du/dx_k) X^k) J^-1.
// Each reference derivative of a nodal field at the GL points is three
// sum-factorised passes with the 1-D matrices of the LGL basis at the GL
// points: values I, first derivatives, and second derivatives (the first
// derivative matrix times the LGL-node derivative matrix, exact because the
// derivative of a degree-p polynomial is held by its LGL values).
// On multi-block meshes the geometry is the exact block map (as in the
// operator): J and X^k come from the map's first and second derivatives at
// the GL points (blocks.h), composed with the element's linear map into its
// block.  With a fiducial grid the integrands stay those of the physical grid
// and the weights (w det J, w S), h_e, h_m and sigma are the fiducial grid's.
// The mortar terms read the trace buffer that an FP64 apply of u leaves
// behind: u and n_A . grad u of both sides at the mortar's GL points; each
// element sums the mortars of its own slots, so every interior mortar counts
// in full for both of its elements and the result needs no atomics.
#include "blocks.h"
#include "estimate.h"

namespace dg {
namespace {

constexpr int kEstThreads = 768;   // >= kMaxN^3 = 729
constexpr int kNV = kMaxN * kMaxN * kMaxN;

// Derivative (d0, d1, d2) of the nodal field F (n^3 values, x fastest) at GL
// point k of this thread (0 when k >= n^3).  Every thread of the CTA calls it.
__device__ double eval_at_point(const double* F, double* T1, double* T2, const double* const* M, int d0, int d1,
                                int d2, int n, int k) {
    const int n2 = n * n, n3 = n2 * n;
    const double* A = M[d0];
    const double* B = M[d1];
    const double* Z = M[d2];
    for (int t = threadIdx.x; t < n3; t += blockDim.x) {
        const int i = t % n, r = t / n;
        double s = 0.0;
        for (int m = 0; m < n; ++m) s += A[i * n + m] * F[m + n * r];
        T1[t] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n3; t += blockDim.x) {
        const int i = t % n, j = (t / n) % n, l = t / n2;
        double s = 0.0;
        for (int m = 0; m < n; ++m) s += B[j * n + m] * T1[i + n * (m + n * l)];
        T2[t] = s;
    }
    __syncthreads();
    double v = 0.0;
    if (k < n3) {
        const int ij = k % n2, l = k / n2;
        for (int m = 0; m < n; ++m) v += Z[l * n + m] * T2[ij + n2 * m];
    }
    __syncthreads();
    return v;
}

// Sum over the CTA, in a fixed order; the result is valid in thread 0.
__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

__global__ void __launch_bounds__(kEstThreads) estimate_kernel(EstimateArgs a, const double* u, const double* g,
                                                               const double* f, const double* gD, double* eta2) {
    const int e = blockIdx.x;
    if (e >= a.n_elems) return;
    const int n = a.p[e] + 1, n2 = n * n, n3 = n2 * n;
    const int k = threadIdx.x;
    __shared__ double F[kNV], T1[kNV], T2[kNV];
    __shared__ double Mx[3][kMaxN * kMaxN];
    __shared__ double red[32];
    const double* I = a.tab + tab_n(TabIndex::I, n);
    const double* D1 = a.tab + tab_n(TabIndex::IDg, n);
    const double* DL = a.tab + tab_n(TabIndex::DL, n);
    const double* wg = a.tab + tab_n(TabIndex::GLw, n);
    for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        const int i = t / n, c = t % n;
        Mx[0][t] = I[t];
        Mx[1][t] = D1[t];
        double s = 0.0;
        for (int b = 0; b < n; ++b) s += D1[i * n + b] * DL[b * n + c];
        Mx[2][t] = s;
    }
    const double* M[3] = {Mx[0], Mx[1], Mx[2]};
    const double* Xe = a.n_blocks > 0 ? nullptr : a.X + 3 * a.dof_off[e];
    const double* ue = u + a.dof_off[e];
    const bool blk = a.n_blocks > 0;

    // element diameter: largest distance between two of the eight vertices
    double he = 0.0;
    double binv = 1.0, bxi0[3] = {0.0, 0.0, 0.0};   // block meshes: xi_block = bxi0 + binv (xi + 1)
    if (blk) {
        const int* lf = a.leaves + 4 * e;
        binv = 1.0 / (double)(1 << lf[0]);
        for (int dd = 0; dd < 3; ++dd) bxi0[dd] = -1.0 + 2.0 * lf[1 + dd] * binv;
    }
    if (threadIdx.x == 0 && blk) {
        const dg_block& BF = a.fblocks[a.block[e]];
        double V[8][3];
        for (int c = 0; c < 8; ++c) {
            double xb[3];
            for (int dd = 0; dd < 3; ++dd) xb[dd] = bxi0[dd] + binv * (((c >> dd) & 1) ? 2.0 : 0.0);
            block_point(BF, xb, V[c]);
        }
        for (int c = 0; c < 8; ++c)
            for (int d = c + 1; d < 8; ++d) {
                const double dx = V[c][0] - V[d][0], dy = V[c][1] - V[d][1], dz = V[c][2] - V[d][2];
                he = fmax(he, sqrt(dx * dx + dy * dy + dz * dz));
            }
    } else if (threadIdx.x == 0) {
        double V[8][3];
        for (int c = 0; c < 8; ++c) {
            const int idx = ((c & 1) ? n - 1 : 0) + n * (((c >> 1) & 1) ? n - 1 : 0) + n2 * (((c >> 2) & 1) ? n - 1 : 0);
            for (int i = 0; i < 3; ++i) V[c][i] = Xe[i * n3 + idx];
        }
        for (int c = 0; c < 8; ++c)
            for (int d = c + 1; d < 8; ++d) {
                const double dx = V[c][0] - V[d][0], dy = V[c][1] - V[d][1], dz = V[c][2] - V[d][2];
                he = fmax(he, sqrt(dx * dx + dy * dy + dz * dz));
            }
    }

    // J_il = d x_i / d xi_l (and, on block meshes, the map's second derivatives Xs and the
    // fiducial Jacobian determinant of the volume weight)
    double J[3][3], Xs[3][3][3], detW = 0.0;
    if (blk) {
        double xp[3], xb[3] = {0.0, 0.0, 0.0};
        const double* xg = a.tab + tab_n(TabIndex::GLx, n);
        if (k < n3) {
            const int ii[3] = {k % n, (k / n) % n, k / n2};
            for (int dd = 0; dd < 3; ++dd) xb[dd] = bxi0[dd] + binv * (xg[ii[dd]] + 1.0);
        }
        const dg_block& B = a.blocks[a.block[e]];
        block_jacobian(B, xb, J, xp);
        block_hessian(B, xb, Xs);
        for (int i = 0; i < 3; ++i)
            for (int l = 0; l < 3; ++l) {
                J[i][l] *= binv;
                for (int m = 0; m < 3; ++m) Xs[i][l][m] *= binv * binv;
            }
        double JF[3][3];
        block_jacobian(a.fblocks[a.block[e]], xb, JF, xp);
        for (int i = 0; i < 3; ++i)
            for (int l = 0; l < 3; ++l) JF[i][l] *= binv;
        detW = JF[0][0] * (JF[1][1] * JF[2][2] - JF[1][2] * JF[2][1]) -
               JF[0][1] * (JF[1][0] * JF[2][2] - JF[1][2] * JF[2][0]) +
               JF[0][2] * (JF[1][0] * JF[2][1] - JF[1][1] * JF[2][0]);
    } else {
        for (int i = 0; i < 3; ++i) {
            for (int t = threadIdx.x; t < n3; t += blockDim.x) F[t] = Xe[i * n3 + t];
            __syncthreads();
            J[i][0] = eval_at_point(F, T1, T2, M, 1, 0, 0, n, k);
            J[i][1] = eval_at_point(F, T1, T2, M, 0, 1, 0, n, k);
            J[i][2] = eval_at_point(F, T1, T2, M, 0, 0, 1, n, k);
        }
    }
    double Ji[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}, det = 1.0;
    if (k < n3) {
        det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
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
    }

    // u, its physical gradient and the reference Hessian; pairs (l, m) in the
    // order 00, 11, 22, 01, 02, 12
    constexpr int kD[6][3] = {{2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
    for (int t = threadIdx.x; t < n3; t += blockDim.x) F[t] = ue[t];
    __syncthreads();
    const double uv = eval_at_point(F, T1, T2, M, 0, 0, 0, n, k);
    double du[3];
    du[0] = eval_at_point(F, T1, T2, M, 1, 0, 0, n, k);
    du[1] = eval_at_point(F, T1, T2, M, 0, 1, 0, n, k);
    du[2] = eval_at_point(F, T1, T2, M, 0, 0, 1, n, k);
    double ux[3];
    for (int i = 0; i < 3; ++i) ux[i] = Ji[0][i] * du[0] + Ji[1][i] * du[1] + Ji[2][i] * du[2];
    double H[6];
    for (int c = 0; c < 6; ++c) H[c] = eval_at_point(F, T1, T2, M, kD[c][0], kD[c][1], kD[c][2], n, k);
    // minus sum_k (du/dx_k) X^k
    if (blk) {
        constexpr int kLM[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
        for (int i = 0; i < 3; ++i)
            for (int c = 0; c < 6; ++c) H[c] -= ux[i] * Xs[i][kLM[c][0]][kLM[c][1]];
    } else {
        for (int i = 0; i < 3; ++i) {
            for (int t = threadIdx.x; t < n3; t += blockDim.x) F[t] = Xe[i * n3 + t];
            __syncthreads();
            for (int c = 0; c < 6; ++c)
                H[c] -= ux[i] * eval_at_point(F, T1, T2, M, kD[c][0], kD[c][1], kD[c][2], n, k);
        }
    }
    double vol = 0.0;
    if (k < n3) {
        double G[3][3];
        for (int l = 0; l < 3; ++l)
            for (int m = 0; m < 3; ++m) G[l][m] = Ji[l][0] * Ji[m][0] + Ji[l][1] * Ji[m][1] + Ji[l][2] * Ji[m][2];
        const double lap = G[0][0] * H[0] + G[1][1] * H[1] + G[2][2] * H[2] +
                           2.0 * (G[0][1] * H[3] + G[0][2] * H[4] + G[1][2] * H[5]);
        const long long vo = a.vqp_off[e];
        const double R = (f ? f[vo + k] : 0.0) * uv - (g ? g[vo + k] : 0.0) - lap;
        const double w = wg[k % n] * wg[(k / n) % n] * wg[k / n2];
        vol = w * (blk ? detW : det) * R * R;
    }
    vol = block_sum(vol, red);

    // mortar terms of the element's slots
    double mort = 0.0;
    for (int s = a.slot_off[e]; s < a.slot_off[e + 1]; ++s) {
        const int mi = a.slot_mortar[s];
        const Mortar Mo = a.mortars[mi];
        const int q2 = Mo.q * Mo.q;
        const double* mg = a.mgW + 7 * Mo.goff;   // w S of the weighting grid
        const double* mt = a.mt + 4 * Mo.goff;
        double s1 = 0.0, s2 = 0.0;
        for (int pt = threadIdx.x; pt < q2; pt += blockDim.x) {
            const double wS = mg[pt];
            if (Mo.eB >= 0) {
                const double j1 = mt[q2 + pt] - mt[3 * q2 + pt];
                const double j2 = mt[pt] - mt[2 * q2 + pt];
                s1 += wS * j1 * j1;
                s2 += wS * j2 * j2;
            } else {
                const double j3 = mt[pt] - (gD ? gD[Mo.bnd_off + pt] : 0.0);
                s2 += wS * j3 * j3;
            }
        }
        s1 = block_sum(s1, red);
        s2 = block_sum(s2, red);
        if (threadIdx.x == 0) {
            const double pm = Mo.q - 1, sig = a.sigW[mi];
            const double hm = a.C * pm * pm / sig;
            mort += (Mo.eB >= 0 ? hm / pm * s1 : 0.0) + sig / hm * pm * pm * s2;
        }
    }
    if (threadIdx.x == 0) {
        const double pe = n - 1;
        eta2[e] = he * he * pe * pe * vol + mort;
    }
}

}  // namespace

cudaError_t launch_estimate(const EstimateArgs& a, const double* u, const double* g, const double* f,
                            const double* gD, double* eta2, cudaStream_t st) {
    if (a.n_elems == 0) return cudaSuccess;
    estimate_kernel<<<a.n_elems, kEstThreads, 0, st>>>(a, u, g, f, gD, eta2);
    return cudaGetLastError();
}

}  // namespace dg
