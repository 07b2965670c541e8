// Zeroth-order term and the puncture equation (Sec. II.E.6 eq. operator_oh,
// Sec. III.B nonlinear terms at GL points, Sec. III.D puncture data).
//
// * Finest level: int f u v is evaluated at the volume GL points with the
//   coefficient c0 = w det J f folded into the apply kernel.
// * Coarse levels: the Galerkin form O^H = (I_h^H)^T O^h I_h^H.  Because the
//   prolongation interpolates exactly (coarse spaces are nested in the fine
//   ones), O^H_ab = sum over the finest descendants' GL points of
//   c0 psi^H_a psi^H_b, with psi^H evaluated at those points.  The kernel sums
//   this per descendant in sum-factorised form (first over the z points for
//   every pair (c, c'), then over x and y per matrix entry).
// * Puncture: 1/alpha = sum_I m_I / (2 r_I); A_ij = sum_I 3/(2 r_I^2)
//   [P_i n_j + P_j n_i - (delta_ij - n_i n_j) P.n] + 3/r_I^3 [n_i w_j + n_j w_i],
//   w = S_I x n (the spin term of eq. Two_Punctures_Aij, its symmetrisation
//   taken as t_(ij) = (t_ij + t_ji) / 2); beta = alpha^7 A_ij A_ij / 8.  Source s(u) = beta (1 + alpha (1 + u))^-7,
//   Jacobian coefficient f(u) = 7 alpha beta (1 + alpha (1 + u))^-8.
// * Power-law source (the constant-density star of Sec. III.C,
//   Lap psi + 2 pi rho psi^5 = 0): s(u) = c u^k, f(u) = -k c u^(k-1), with c
//   given at the GL points; the nonlinear term is evaluated at the GL points
//   after interpolating u there, as the paper describes for that problem.
#include "newton.h"

namespace dg {
namespace {

__device__ inline double lagv(const double* x, int n, int a, double t) {
    double v = 1.0;
    for (int m = 0; m < n; ++m)
        if (m != a) v *= (t - x[m]) / (x[a] - x[m]);
    return v;
}

__global__ void puncture_kernel(const double* vxyz, long long n, PunctureDev P, double* alpha, double* beta) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double x[3] = {vxyz[i], vxyz[n + i], vxyz[2 * n + i]};
        double inv_a = 0.0, A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int I = 0; I < P.n; ++I) {
            double dx[3], r2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                dx[k] = x[k] - P.c[I][k];
                r2 += dx[k] * dx[k];
            }
            const double r = sqrt(r2);
            double nv[3];
            for (int k = 0; k < 3; ++k) nv[k] = dx[k] / r;
            const double Pn = P.P[I][0] * nv[0] + P.P[I][1] * nv[1] + P.P[I][2] * nv[2];
            const double f = 1.5 / r2, fs = 3.0 / (r2 * r);
            const double w[3] = {P.S[I][1] * nv[2] - P.S[I][2] * nv[1], P.S[I][2] * nv[0] - P.S[I][0] * nv[2],
                                 P.S[I][0] * nv[1] - P.S[I][1] * nv[0]};   // S x n
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    A[a][b] += f * (P.P[I][a] * nv[b] + P.P[I][b] * nv[a] - ((a == b ? 1.0 : 0.0) - nv[a] * nv[b]) * Pn) +
                               fs * (nv[a] * w[b] + nv[b] * w[a]);
            inv_a += P.m[I] / (2.0 * r);
        }
        double AA = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) AA += A[a][b] * A[a][b];
        const double al = 1.0 / inv_a;
        const double a2 = al * al, a4 = a2 * a2;
        alpha[i] = al;
        beta[i] = a4 * a2 * al * AA / 8.0;
    }
}

// per element: S = I^T (w det J s(u~)), optional jac = w det J f(u~) at GL points
__global__ void nl_kernel(NlArgs a, const double* u, double* S, double* jac64, float* jac32) {
    const int e = blockIdx.x;
    if (e >= a.n_elems) return;
    const int n = a.p[e] + 1, n2 = n * n, n3 = n2 * n;
    __shared__ double b0[kMaxN * kMaxN * kMaxN], b1[kMaxN * kMaxN * kMaxN];
    const double* I = a.tab + tab_n(TabIndex::I, n);
    const long long vo = a.vqp_off[e], dofo = a.dof_off[e];
    if (n < kMinN || n > kMaxN || vo < 0 || vo + n3 > a.n_vqp) {
        if (threadIdx.x == 0) atomicExch(a.chk, 2);
        return;
    }
    for (int k = threadIdx.x; k < n3; k += blockDim.x) b0[k] = u[dofo + k];
    __syncthreads();
    // u at GL points: three forward passes (x, y, z)
    for (int k = threadIdx.x; k < n3; k += blockDim.x) {
        const int i = k % n, r = k / n;
        double s = 0.0;
        for (int m = 0; m < n; ++m) s += I[i * n + m] * b0[m + n * r];
        b1[k] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n3; k += blockDim.x) {
        const int i = k % n, j = (k / n) % n, l = k / n2;
        double s = 0.0;
        for (int m = 0; m < n; ++m) s += I[j * n + m] * b1[i + n * (m + n * l)];
        b0[k] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n3; k += blockDim.x) {
        const int ij = k % n2, l = k / n2;
        double s = 0.0;
        for (int m = 0; m < n; ++m) s += I[l * n + m] * b0[ij + n2 * m];
        b1[k] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n3; k += blockDim.x) {
        const double wd = a.wdetJ[vo + k];
        double s, jc;
        if (a.kind == kNlPower) {
            const double c = a.alpha[vo + k], uq = b1[k];
            double pk1 = 1.0;                   // u^(k-1)
            for (int q = 1; q < a.power; ++q) pk1 *= uq;
            s = c * pk1 * uq;
            jc = -a.power * c * pk1;            // d(-s)/du: the source grows with u
        } else {
            const double al = a.alpha[vo + k], be = a.beta[vo + k];
            const double base = 1.0 + al * (1.0 + b1[k]);
            const double b2 = base * base, b4 = b2 * b2, b8 = b4 * b4;
            s = be * base / b8;                 // beta base^-7
            jc = 7.0 * al * be / b8;
        }
        if (jac64) {
            jac64[vo + k] = wd * jc;
            jac32[vo + k] = (float)(wd * jc);
        }
        b0[k] = wd * s;
    }
    __syncthreads();
    // lift: three transposed passes
    for (int k = threadIdx.x; k < n3; k += blockDim.x) {
        const int i = k % n, r = k / n;
        double s = 0.0;
        for (int m = 0; m < n; ++m) s += I[m * n + i] * b0[m + n * r];
        b1[k] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n3; k += blockDim.x) {
        const int i = k % n, j = (k / n) % n, l = k / n2;
        double s = 0.0;
        for (int m = 0; m < n; ++m) s += I[m * n + j] * b1[i + n * (m + n * l)];
        b0[k] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n3; k += blockDim.x) {
        const int ij = k % n2, l = k / n2;
        double s = 0.0;
        for (int m = 0; m < n; ++m) s += I[m * n + l] * b0[ij + n2 * m];
        if (S) S[dofo + k] = s;
    }
}

// R = Lu - S - F
__global__ void sub_kernel(const double* Lu, const double* S, const double* F, double* R, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        R[i] = Lu[i] - S[i] - (F ? F[i] : 0.0);
}

// O_H for every coarse element H of one level (block per H, loop over its finest descendants).
__global__ void galerkin_kernel(GalerkinArgs g, const double* c0, double* O64, float* O32) {
    const int H = blockIdx.x;
    if (H >= g.n_coarse) return;
    const int nH = g.pH[H] + 1, nH2 = nH * nH, nH3 = nH2 * nH;
    const long long nent = (long long)nH3 * nH3;
    if (nH < kMinN || nH > kMaxN || g.Ob_off[H] < 0 || g.Ob_off[H] + nent > g.ob_total) {
        if (threadIdx.x == 0) atomicExch(g.chk, 3);
        return;
    }
    double* Oe = O64 + g.Ob_off[H];
    __shared__ double E[3][kMaxN * kMaxN];          // E_d[i][a]
    __shared__ double xlH[kMaxN], xgq[kMaxN];
    extern __shared__ double dyn[];
    double* T1 = dyn;                               // T1[(c, c')][i][j], n_H^2 q^2 <= 9^4
    double* cq = dyn + kMaxN * kMaxN * kMaxN * kMaxN;   // c0 at the descendant's GL points
    for (long long k = threadIdx.x; k < nent; k += blockDim.x) Oe[k] = 0.0;
    if (threadIdx.x < nH) xlH[threadIdx.x] = g.tab[tab_n(TabIndex::LGLx, nH) + threadIdx.x];
    __syncthreads();
    for (int di = g.desc_off[H]; di < g.desc_off[H + 1]; ++di) {
        if (di < 0 || di >= g.n_desc) {
            if (threadIdx.x == 0) atomicExch(g.chk, 4);
            break;
        }
        const int f = g.desc[di];
        const int q = g.pf[f] + 1, q2 = q * q, q3 = q2 * q;
        const long long vo = g.vqp_off_f[f];
        if (q < kMinN || q > kMaxN || vo < 0 || vo + q3 > g.n_vqp_f) {
            if (threadIdx.x == 0) atomicExch(g.chk, 5);
            break;
        }
        if (threadIdx.x < q) xgq[threadIdx.x] = g.tab[tab_n(TabIndex::GLx, q) + threadIdx.x];
        for (int k = threadIdx.x; k < q3; k += blockDim.x) cq[k] = c0[vo + k];
        __syncthreads();
        const double* so = g.map + 6 * (long long)di;   // scale and offset per axis
        for (int k = threadIdx.x; k < 3 * q * nH; k += blockDim.x) {
            const int dd = k / (q * nH), r = k % (q * nH), i = r / nH, a = r % nH;
            E[dd][i * nH + a] = lagv(xlH, nH, a, so[2 * dd] * xgq[i] + so[2 * dd + 1]);
        }
        __syncthreads();
        // T1[(c, c')][i][j] = sum_k c0[i, j, k] Ez[k, c] Ez[k, c']
        for (int k = threadIdx.x; k < nH2 * q2; k += blockDim.x) {
            const int cc = k / q2, ij = k % q2;
            const int c = cc / nH, c2 = cc % nH;
            double s = 0.0;
            for (int kk = 0; kk < q; ++kk) s += cq[ij + q2 * kk] * E[2][kk * nH + c] * E[2][kk * nH + c2];
            T1[k] = s;
        }
        __syncthreads();
        // O[(a, b, c), (a', b', c')] += sum_{i, j} Ex[i,a] Ex[i,a'] Ey[j,b] Ey[j,b'] T1[(c,c')][i][j]
        for (long long k = threadIdx.x; k < nent; k += blockDim.x) {
            const int al = (int)(k / nH3), be = (int)(k % nH3);
            const int a = al % nH, b = (al / nH) % nH, c = al / nH2;
            const int a2 = be % nH, b2 = (be / nH) % nH, c2 = be / nH2;
            const double* t = T1 + (c * nH + c2) * q2;
            double s = 0.0;
            for (int j = 0; j < q; ++j) {
                const double ey = E[1][j * nH + b] * E[1][j * nH + b2];
                double sx = 0.0;
                for (int i = 0; i < q; ++i) sx += E[0][i * nH + a] * E[0][i * nH + a2] * t[i + q * j];
                s += ey * sx;
            }
            Oe[k] += s;
        }
        __syncthreads();
    }
    float* Of = O32 + g.Ob_off[H];
    for (long long k = threadIdx.x; k < nent; k += blockDim.x) Of[k] = (float)Oe[k];
}

inline int grid_for(long long n) {
    long long g = (n + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 2432 ? 2432 : g));
}

}  // namespace

cudaError_t launch_puncture(const double* vxyz, long long n, const PunctureDev& P, double* alpha, double* beta,
                            cudaStream_t st) {
    puncture_kernel<<<grid_for(n), 256, 0, st>>>(vxyz, n, P, alpha, beta);
    return cudaGetLastError();
}

cudaError_t launch_nl(const NlArgs& a, const double* u, double* S, double* jac64, float* jac32, cudaStream_t st) {
    nl_kernel<<<a.n_elems, 128, 0, st>>>(a, u, S, jac64, jac32);
    return cudaGetLastError();
}

cudaError_t launch_sub(const double* Lu, const double* S, const double* F, double* R, long long n, cudaStream_t st) {
    sub_kernel<<<grid_for(n), 256, 0, st>>>(Lu, S, F, R, n);
    return cudaGetLastError();
}

cudaError_t launch_galerkin(const GalerkinArgs& g, const double* c0, double* O64, float* O32, cudaStream_t st) {
    const size_t smem = sizeof(double) * (kMaxN * kMaxN * kMaxN * kMaxN + kMaxN * kMaxN * kMaxN);
    static const cudaError_t attr =   // once per process, thread-safe initialisation
        cudaFuncSetAttribute(galerkin_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess) return attr;
    galerkin_kernel<<<g.n_coarse, 256, smem, st>>>(g, c0, O64, O32);
    return cudaGetLastError();
}

}  // namespace dg
