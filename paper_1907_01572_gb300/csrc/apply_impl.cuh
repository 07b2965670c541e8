// Matrix-free SIPG operator apply (eq. lh2), one fused element-centric kernel
// per polynomial-degree bucket.
//
// Volume (eq. harald-stiff), sum-factorised with 1-D operators (Sec. II.F.4):
//   u~ = (I x I x I) u            values at the GL points         (3 passes)
//   g_l = Dg_l u~                 reference gradient at GL points (3 passes)
//   f_l = G_lm g_m                G = w det J J^-1 J^-T (stored)
//   z = sum_l Dg_l^T f_l (+ c0 u~ for the zeroth-order term)     (3 passes)
//   y = (I x I x I)^T z                                           (3 passes)
// Faces (consistency, symmetry, penalty integrals of eq. lh2 with the hp
// mortar projection of the mortar figure): for each mortar touching the
// element, both sides' traces u and reference gradients are interpolated to
// the mortar's GL points (sub-face tables for 2:1 faces, degree-change tables
// for p-jumps); with n the element's outward normal,
//   j = u_own - u_nb,  a = {n . grad u},
//   y_alpha += sum_pts wS [ (sigma j - a) psi_alpha - (1/2) j n . grad psi_alpha ]
// (on Dirichlet mortars j = u_own, a = n . grad u_own and the factor 1/2 is 1),
// lifted back through the transposed interpolation and the face-normal row of
// the LGL derivative matrix.  The neighbour's trace and normal derivative are
// read straight from x (its element block, normally an L2 hit), so one launch
// per bucket computes y with no intermediate buffers.
//
// Execution: one warp per element (lanes own pencils of the n^3 tensor grid,
// __syncwarp between phases, no CTA-wide barrier after the table load); one
// persistent CTA per SM strides over the bucket with as many warps as shared
// memory and registers allow; all 1-D tables (FP32: also every mortar
// interpolation / derivative table) sit in shared memory.
#pragma once
#include "apply.h"

namespace dg {
namespace apply_detail {

constexpr int kQ = kMaxN;  // largest mortar q and neighbour n

__device__ inline void tangential(int d, int& t1, int& t2) {
    t1 = d == 0 ? 1 : 0;
    t2 = d == 2 ? 1 : 2;
}

// k -> (k % q, k / q) for the small runtime sizes of the face phase (k < 1024,
// q <= 9): float reciprocal, exact in this range, much cheaper than an integer divide.
__device__ __forceinline__ void split(int k, int q, float qinv, int& r, int& s) {
    s = __float2int_rz((k + 0.5f) * qinv);
    r = k - s * q;
}

// out = M in along direction DIR of an N^3 array held by one warp (TRANS: M^T; ACC: out +=).
template <int N, int DIR, bool TRANS, bool ACC, typename T>
__device__ inline void wpass(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ M, int lane) {
    for (int pid = lane; pid < N * N; pid += 32) {
        int base, stride;
        if (DIR == 0) { base = pid * N; stride = 1; }
        else if (DIR == 1) { base = (pid / N) * N * N + (pid % N); stride = N; }
        else { base = pid; stride = N * N; }
        T v[N];
#pragma unroll
        for (int m = 0; m < N; ++m) v[m] = in[base + m * stride];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            T s = 0;
#pragma unroll
            for (int m = 0; m < N; ++m) s += (TRANS ? M[m * N + i] : M[i * N + m]) * v[m];
            if (ACC) out[base + i * stride] += s;
            else out[base + i * stride] = s;
        }
    }
}

template <int N>
struct Layout {
    static constexpr int N2 = N * N, N3 = N2 * N;
    static constexpr int FACE = 2 * N2 + 2 * kQ * kQ + 6 * kQ * N + 3 * kQ * kQ + 4 * kQ * kQ;
    static constexpr bool ALIAS = 4 * N3 >= FACE;   // face scratch reuses the volume scratch
    static constexpr int WARP = ALIAS ? 6 * N3 : 6 * N3 + FACE;
};

template <int N, typename T>
__global__ void apply_kernel(LevelView<T> L, const int* __restrict__ bucket, int count, const T* __restrict__ x,
                             T* __restrict__ y) {
    using Ly = Layout<N>;
    constexpr int N2 = Ly::N2, N3 = Ly::N3;
    // FP32: every mortar table is staged in shared memory (26.6 KB); FP64 reads
    // them through L1 so that the larger FP64 scratch leaves room for more warps.
    constexpr bool STAGE = sizeof(T) == 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int ftot = STAGE ? L.ft.total : 0;
    T* sFTs = sm;
    const T* sFT = STAGE ? sFTs : L.ftab;
    T* sI = sFTs + ((ftot + 3) & ~3);
    T* sDg = sI + N2;
    T* sDL = sDg + N2;
    const int nwarps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < ftot; k += blockDim.x) sFTs[k] = L.ftab[k];
    for (int k = threadIdx.x; k < N2; k += blockDim.x) {
        sI[k] = L.tab[tab_n(TabIndex::I, N) + k];
        sDg[k] = L.tab[tab_n(TabIndex::Dg, N) + k];
        sDL[k] = L.tab[tab_n(TabIndex::DL, N) + k];
    }
    __syncthreads();
    T* U = sDL + N2 + warp * Ly::WARP;
    T* Y = U + N3;
    T* A = Y + N3;
    T* B = A + N3;
    T* G1 = B + N3;
    T* G3 = G1 + N3;
    T* G2 = Y;  // the y-gradient lives in Y until the backward passes
    T* F = Ly::ALIAS ? A : G3 + N3;
    T* uf = F;
    T* df = uf + N2;
    T* ufn = df + N2;
    T* dfn = ufn + kQ * kQ;
    T* U1o = dfn + kQ * kQ;
    T* DU1o = U1o + kQ * N;
    T* N1o = DU1o + kQ * N;
    T* X1 = N1o + kQ * N;
    T* X2 = X1 + kQ * N;
    T* X3 = X2 + kQ * N;
    T* U1n = X3 + kQ * N;
    T* DU1n = U1n + kQ * kQ;
    T* N1n = DU1n + kQ * kQ;
    T* PA = N1n + kQ * kQ;
    T* PB1 = PA + kQ * kQ;
    T* PB2 = PB1 + kQ * kQ;
    T* PBn = PB2 + kQ * kQ;
    const bool mass = L.c0 != nullptr;
    const int st[3] = {1, N, N2};

    for (int ei = blockIdx.x * nwarps + warp; ei < count; ei += gridDim.x * nwarps) {
        const int e = bucket[ei];
        const long long dofo = L.dof_off[e], vo = L.vqp_off[e];
        for (int k = lane; k < N3; k += 32) U[k] = x[dofo + k];
        __syncwarp();
        // ---- volume ----------------------------------------------------------------
        wpass<N, 0, false, false>(U, A, sI, lane);
        __syncwarp();
        wpass<N, 1, false, false>(A, B, sI, lane);
        __syncwarp();
        wpass<N, 2, false, false>(B, A, sI, lane);  // A = u at GL points
        __syncwarp();
        wpass<N, 0, false, false>(A, G1, sDg, lane);
        wpass<N, 1, false, false>(A, G2, sDg, lane);
        wpass<N, 2, false, false>(A, G3, sDg, lane);
        __syncwarp();
        {
            const T* Ge = L.G + 6 * vo;
            for (int k = lane; k < N3; k += 32) {
                const T g0 = G1[k], g1 = G2[k], g2 = G3[k];
                const T m00 = Ge[k], m01 = Ge[N3 + k], m02 = Ge[2 * N3 + k];
                const T m11 = Ge[3 * N3 + k], m12 = Ge[4 * N3 + k], m22 = Ge[5 * N3 + k];
                G1[k] = m00 * g0 + m01 * g1 + m02 * g2;
                G2[k] = m01 * g0 + m11 * g1 + m12 * g2;
                G3[k] = m02 * g0 + m12 * g1 + m22 * g2;
                if (mass) B[k] = L.c0[vo + k] * A[k];
            }
        }
        __syncwarp();
        if (mass) wpass<N, 0, true, true>(G1, B, sDg, lane);
        else wpass<N, 0, true, false>(G1, B, sDg, lane);
        __syncwarp();
        wpass<N, 1, true, true>(G2, B, sDg, lane);
        __syncwarp();
        wpass<N, 2, true, true>(G3, B, sDg, lane);
        __syncwarp();
        wpass<N, 0, true, false>(B, A, sI, lane);
        __syncwarp();
        wpass<N, 1, true, false>(A, B, sI, lane);
        __syncwarp();
        wpass<N, 2, true, false>(B, Y, sI, lane);
        __syncwarp();
        if (L.Ob != nullptr && L.Ob_off[e] + (long long)N3 * N3 > L.ob_total) {
            if (lane == 0) atomicExch(L.chk, 1);
        } else if (L.Ob != nullptr) {
            const T* Oe = L.Ob + L.Ob_off[e];
            for (int k = lane; k < N3; k += 32) {
                T s = 0;
                for (int j = 0; j < N3; ++j) s += Oe[(long long)j * N3 + k] * U[j];
                Y[k] += s;
            }
            __syncwarp();
        }
        // ---- faces ----------------------------------------------------------------------
        const int s0 = L.slot_off[e], s1 = L.slot_off[e + 1];
        int mi_next = L.slot_mortar[s0];
        Mortar M_next = L.mortars[mi_next];
        for (int si = s0; si < s1; ++si) {
            const int mi = mi_next;
            const Mortar M = M_next;
            if (si + 1 < s1) {   // prefetch the next slot's mortar record
                mi_next = L.slot_mortar[si + 1];
                M_next = L.mortars[mi_next];
            }
            const int f = L.slot_face[si];
            const int side = L.slot_side[si];
            const int q = M.q, q2 = q * q;
            const float qinv = 1.0f / (float)q;
            const T sig = L.sigma[mi];
            int p0, p1, eo, fo, o0, o1;
            if (side == 0) { p0 = M.posA0; p1 = M.posA1; eo = M.eB; fo = M.fB; o0 = M.posB0; o1 = M.posB1; }
            else { p0 = M.posB0; p1 = M.posB1; eo = M.eA; fo = M.fA; o0 = M.posA0; o1 = M.posA1; }
            const int nbN = eo >= 0 ? L.p[eo] + 1 : 2;
            const float nbinv = 1.0f / (float)nbN;
            const int d = f >> 1, fn = (f & 1) ? N - 1 : 0;
            int t1, t2;
            tangential(d, t1, t2);
            // S1: own trace u and d_nu u at own face nodes; the neighbour's from x
            for (int k = lane; k < N2; k += 32) {
                const int a = k % N, b = k / N;
                const int base = a * st[t1] + b * st[t2];
                uf[k] = U[base + fn * st[d]];
                T acc = 0;
#pragma unroll
                for (int c = 0; c < N; ++c) acc += sDL[fn * N + c] * U[base + c * st[d]];
                df[k] = acc;
            }
            if (eo >= 0) {
                const T* xe = x + L.dof_off[eo];
                const int nst[3] = {1, nbN, nbN * nbN};
                const int fno = (fo & 1) ? nbN - 1 : 0;
                const T* DLn = L.tab + tab_n(TabIndex::DL, nbN) + fno * nbN;
                for (int k = lane; k < nbN * nbN; k += 32) {
                    int a, b;
                    split(k, nbN, nbinv, a, b);
                    const int base = a * nst[t1] + b * nst[t2];
                    T acc = 0, fv = 0;
                    for (int c = 0; c < nbN; ++c) {
                        const T v = __ldg(xe + base + c * nst[d]);
                        acc += DLn[c] * v;
                        if (c == fno) fv = v;
                    }
                    ufn[k] = fv;
                    dfn[k] = acc;
                }
            }
            __syncwarp();
            const T* Im1 = sFT + L.ft.off[N - kMinN][q - kMinN][p0];
            const T* Dm1 = Im1 + q * N;
            const T* Im2 = sFT + L.ft.off[N - kMinN][q - kMinN][p1];
            const T* Dm2 = Im2 + q * N;
            // S2: interpolate along the first tangential axis
            for (int k = lane; k < q * N; k += 32) {
                int i1, b;
                split(k, q, qinv, i1, b);
                T su = 0, sd = 0, sn = 0;
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    const T iv = Im1[i1 * N + a], dv = Dm1[i1 * N + a];
                    const T u = uf[a + N * b];
                    su += iv * u;
                    sd += dv * u;
                    sn += iv * df[a + N * b];
                }
                U1o[k] = su;
                DU1o[k] = sd;
                N1o[k] = sn;
            }
            const T* Im1n = nullptr;
            const T* Im2n = nullptr;
            if (eo >= 0) {
                Im1n = sFT + L.ft.off[nbN - kMinN][q - kMinN][o0];
                Im2n = sFT + L.ft.off[nbN - kMinN][q - kMinN][o1];
                const T* Dm1n = Im1n + q * nbN;
                for (int k = lane; k < q * nbN; k += 32) {
                    int i1, b;
                split(k, q, qinv, i1, b);
                    T su = 0, sd = 0, sn = 0;
                    for (int a = 0; a < nbN; ++a) {
                        const T iv = Im1n[i1 * nbN + a], dv = Dm1n[i1 * nbN + a];
                        const T u = ufn[a + nbN * b];
                        su += iv * u;
                        sd += dv * u;
                        sn += iv * dfn[a + nbN * b];
                    }
                    U1n[k] = su;
                    DU1n[k] = sd;
                    N1n[k] = sn;
                }
            }
            __syncwarp();
            // S3: values at the mortar points, numerical flux, lift coefficients
            {
                const T* mg = L.mg + 7 * M.goff;
                const T sgn = side == 0 ? T(1) : T(-1);
                const int oo = side == 0 ? 1 : 4, on = side == 0 ? 4 : 1;
                for (int k = lane; k < q2; k += 32) {
                    int i1, i2;
                split(k, q, qinv, i1, i2);
                    T u = 0, gt1 = 0, gt2 = 0, gn = 0;
#pragma unroll
                    for (int b = 0; b < N; ++b) {
                        const T iv = Im2[i2 * N + b], dv = Dm2[i2 * N + b];
                        const T ub = U1o[i1 + q * b];
                        u += iv * ub;
                        gt1 += iv * DU1o[i1 + q * b];
                        gt2 += dv * ub;
                        gn += iv * N1o[i1 + q * b];
                    }
                    const T wS = mg[k];
                    const T co1 = sgn * mg[(oo + t1) * q2 + k], co2 = sgn * mg[(oo + t2) * q2 + k];
                    const T cod = sgn * mg[(oo + d) * q2 + k];
                    const T dno = co1 * gt1 + co2 * gt2 + cod * gn;
                    T jmp, avg, bc;
                    if (eo >= 0) {
                        const T* Dm2n = Im2n + q * nbN;
                        T un = 0, ht1 = 0, ht2 = 0, hn = 0;
                        for (int b = 0; b < nbN; ++b) {
                            const T iv = Im2n[i2 * nbN + b], dv = Dm2n[i2 * nbN + b];
                            const T ub = U1n[i1 + q * b];
                            un += iv * ub;
                            ht1 += iv * DU1n[i1 + q * b];
                            ht2 += dv * ub;
                            hn += iv * N1n[i1 + q * b];
                        }
                        const T dnn = sgn * (mg[(on + t1) * q2 + k] * ht1 + mg[(on + t2) * q2 + k] * ht2 +
                                             mg[(on + d) * q2 + k] * hn);
                        jmp = u - un;
                        avg = T(0.5) * (dno + dnn);
                        bc = T(-0.5) * wS * jmp;
                    } else {
                        jmp = u;
                        avg = dno;
                        bc = -wS * jmp;
                    }
                    PA[k] = wS * (sig * jmp - avg);
                    PB1[k] = bc * co1;
                    PB2[k] = bc * co2;
                    PBn[k] = bc * cod;
                }
            }
            __syncwarp();
            // S4: transposed interpolation along the second tangential axis
            for (int k = lane; k < q * N; k += 32) {
                int i1, b;
                split(k, q, qinv, i1, b);
                T s1v = 0, s2v = 0, s3v = 0;
                for (int i2 = 0; i2 < q; ++i2) {
                    const T iv = Im2[i2 * N + b], dv = Dm2[i2 * N + b];
                    s1v += iv * PA[i1 + q * i2] + dv * PB2[i1 + q * i2];
                    s2v += iv * PB1[i1 + q * i2];
                    s3v += iv * PBn[i1 + q * i2];
                }
                X1[k] = s1v;
                X2[k] = s2v;
                X3[k] = s3v;
            }
            __syncwarp();
            // S5: transposed interpolation along the first axis and lift into y
            for (int k = lane; k < N2; k += 32) {
                const int a = k % N, b = k / N;
                T fu = 0, fd = 0;
                for (int i1 = 0; i1 < q; ++i1) {
                    const T iv = Im1[i1 * N + a], dv = Dm1[i1 * N + a];
                    fu += iv * X1[i1 + q * b] + dv * X2[i1 + q * b];
                    fd += iv * X3[i1 + q * b];
                }
                const int base = a * st[t1] + b * st[t2];
                Y[base + fn * st[d]] += fu;
#pragma unroll
                for (int c = 0; c < N; ++c) Y[base + c * st[d]] += sDL[fn * N + c] * fd;
            }
            __syncwarp();
        }
        for (int k = lane; k < N3; k += 32) y[dofo + k] = Y[k];
        __syncwarp();
    }
}

inline int& sm_count() {
    static int v = 0;
    return v;
}

template <int N, typename T>
cudaError_t launch_n(const LevelView<T>& L, const BucketInfo& b, const T* x, T* y, cudaStream_t st) {
    using Ly = Layout<N>;
    static int W = 0;
    static size_t smem = 0;
    if (W == 0) {
        // one persistent CTA per SM; warps limited by shared memory (tables staged once per CTA)
        // and by the register file
        const size_t table_vals = (sizeof(T) == 4 ? ((L.ft.total + 3) & ~3) : 0) + 3 * N * N;
        const size_t cap = 220 * 1024;
        cudaError_t err = cudaFuncSetAttribute(apply_kernel<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)cap);
        if (err != cudaSuccess) return err;
        int w = (int)((cap - table_vals * sizeof(T)) / (Ly::WARP * sizeof(T)));
        if (w > 24) w = 24;
        for (; w > 1; --w) {   // largest warp count of which one CTA fits on an SM
            const size_t sm_bytes = (table_vals + (size_t)w * Ly::WARP) * sizeof(T);
            int blocks = 0;
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, apply_kernel<N, T>, w * 32, sm_bytes);
            if (err != cudaSuccess) return err;
            if (blocks >= 1) break;
        }
        W = w;
        smem = (table_vals + (size_t)W * Ly::WARP) * sizeof(T);
    }
    int& g_sm_count = sm_count();
    if (g_sm_count == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (g_sm_count <= 0) g_sm_count = 152;
    }
    int grid = (b.count + W - 1) / W;
    if (grid > g_sm_count) grid = g_sm_count;
    apply_kernel<N, T><<<grid, W * 32, smem, st>>>(L, b.elems, b.count, x, y);
    return cudaGetLastError();
}

}  // namespace apply_detail

template <typename T>
cudaError_t launch_apply(const LevelView<T>& L, const BucketInfo* buckets, const T* x, T* y, cudaStream_t st,
                         int* launches) {
    for (int n = kMinN; n <= kMaxN; ++n) {
        const BucketInfo& b = buckets[n];
        if (b.count == 0) continue;
        cudaError_t err = cudaSuccess;
        switch (n) {
            case 2: err = apply_detail::launch_n<2, T>(L, b, x, y, st); break;
            case 3: err = apply_detail::launch_n<3, T>(L, b, x, y, st); break;
            case 4: err = apply_detail::launch_n<4, T>(L, b, x, y, st); break;
            case 5: err = apply_detail::launch_n<5, T>(L, b, x, y, st); break;
            case 6: err = apply_detail::launch_n<6, T>(L, b, x, y, st); break;
            case 7: err = apply_detail::launch_n<7, T>(L, b, x, y, st); break;
            case 8: err = apply_detail::launch_n<8, T>(L, b, x, y, st); break;
            case 9: err = apply_detail::launch_n<9, T>(L, b, x, y, st); break;
        }
        if (err != cudaSuccess) return err;
        if (launches) ++*launches;
    }
    return cudaSuccess;
}

}  // namespace dg
