// Right-hand side of eq. (equationFh2) with Dirichlet data:
//   F_alpha = int_e g psi_alpha  - int_{Gamma_D} g_D n . grad psi_alpha + int_{Gamma_D} sigma g_D psi_alpha,
// volume part by GL quadrature with the interpolation matrix I (Sec. II.A.5),
// boundary part at the boundary mortars' GL points with the side's metric
// factors c = (J^-1) n (so n . grad psi = c . grad_xi psi).
#include "source.h"

namespace dg {
namespace {

__device__ inline void tangential(int d, int& t1, int& t2) {
    t1 = d == 0 ? 1 : 0;
    t2 = d == 2 ? 1 : 2;
}

__global__ void rhs_kernel(RhsArgs a, const double* g, const double* gD, double* F) {
    const int e = blockIdx.x;
    if (e >= a.n_elems) return;
    const int n = a.p[e] + 1, n2 = n * n, n3 = n2 * n;
    __shared__ double b0[kMaxN * kMaxN * kMaxN], b1[kMaxN * kMaxN * kMaxN], Fe[kMaxN * kMaxN * kMaxN];
    const double* I = a.tab + tab_n(TabIndex::I, n);
    const long long vo = a.vqp_off[e];
    for (int k = threadIdx.x; k < n3; k += blockDim.x) b0[k] = g ? a.wdetJ[vo + k] * g[vo + k] : 0.0;
    __syncthreads();
    // F = (I^T x I^T x I^T) b0, one axis at a time
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
        Fe[k] = s;
    }
    __syncthreads();
    if (gD) {
        const int st[3] = {1, n, n2};
        const double* DL = a.tab + tab_n(TabIndex::DL, n);
        for (int s = a.slot_off[e]; s < a.slot_off[e + 1]; ++s) {
            const Mortar M = a.mortars[a.slot_mortar[s]];
            if (M.eB >= 0) continue;
            const int f = a.slot_face[s], d = f >> 1, fn = (f & 1) ? n - 1 : 0;
            int t1, t2;
            tangential(d, t1, t2);
            const int q = M.q, q2 = q * q;
            const double* Im = a.tab + tab_m(TabIndex::Im, n, q, 0);
            const double* Dm = a.tab + tab_m(TabIndex::Dm, n, q, 0);
            const double* mg = a.mg + 7 * M.goff;
            const double sig = a.sigma[a.slot_mortar[s]];
            for (int k = threadIdx.x; k < n2; k += blockDim.x) {
                const int aa = k % n, bb = k / n;
                double fu = 0.0, fd = 0.0;
                for (int pt = 0; pt < q2; ++pt) {
                    const int i1 = pt % q, i2 = pt / q;
                    const double wS = mg[pt], gd = gD[M.bnd_off + pt];
                    const double A = wS * sig * gd, B = -wS * gd;
                    const double c1 = mg[(1 + t1) * q2 + pt], c2 = mg[(1 + t2) * q2 + pt], cd = mg[(1 + d) * q2 + pt];
                    const double I1 = Im[i1 * n + aa], I2 = Im[i2 * n + bb];
                    fu += A * I1 * I2 + B * (c1 * Dm[i1 * n + aa] * I2 + c2 * I1 * Dm[i2 * n + bb]);
                    fd += B * cd * I1 * I2;
                }
                const int base = aa * st[t1] + bb * st[t2];
                Fe[base + fn * st[d]] += fu;
                for (int c = 0; c < n; ++c) Fe[base + c * st[d]] += DL[fn * n + c] * fd;
            }
            __syncthreads();
        }
    }
    for (int k = threadIdx.x; k < n3; k += blockDim.x) F[a.dof_off[e] + k] = Fe[k];
}

__global__ void scale_coef_kernel(const double* wdetJ, const double* coef, double* c64, float* c32, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = wdetJ[i] * coef[i];
        c64[i] = v;
        c32[i] = (float)v;
    }
}

}  // namespace

cudaError_t launch_rhs(const RhsArgs& a, const double* g_qp, const double* gD_qp, double* F, cudaStream_t st) {
    rhs_kernel<<<a.n_elems, 128, 0, st>>>(a, g_qp, gD_qp, F);
    return cudaGetLastError();
}

cudaError_t launch_scale_coef(const double* wdetJ, const double* coef, double* c64, float* c32, long long n,
                              cudaStream_t st) {
    long long g = (n + 255) / 256;
    if (g > 2432) g = 2432;
    if (g < 1) g = 1;
    scale_coef_kernel<<<(int)g, 256, 0, st>>>(wdetJ, coef, c64, c32, n);
    return cudaGetLastError();
}

}  // namespace dg
