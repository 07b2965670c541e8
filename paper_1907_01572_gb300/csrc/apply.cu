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
// read straight from x (its element block), so one launch per bucket computes
// y with no intermediate buffers.
//
// Thread layout: a team of n^2 threads per element (one thread per pencil of
// the tensor grid); E teams per CTA.
#include "apply.h"

namespace dg {
namespace {

__device__ inline void tangential(int d, int& t1, int& t2) {
    t1 = d == 0 ? 1 : 0;
    t2 = d == 2 ? 1 : 2;
}

// out = M in along direction DIR of an N^3 array (TRANS: M^T); ACC: out +=.
template <int N, int DIR, bool TRANS, bool ACC, typename T>
__device__ inline void pass(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ M, int tid) {
    int base, stride;
    if (DIR == 0) { base = tid * N; stride = 1; }
    else if (DIR == 1) { base = (tid / N) * N * N + (tid % N); stride = N; }
    else { base = tid; stride = N * N; }
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

template <int N, typename T>
__global__ void apply_kernel(LevelView<T> L, const int* __restrict__ bucket, int count, int E, int MQ, int MNB,
                             const T* __restrict__ x, T* __restrict__ y) {
    constexpr int N2 = N * N, N3 = N2 * N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    T* sI = sm;
    T* sDg = sI + N2;
    T* sDL = sDg + N2;
    const int face_vals = 2 * N2 + 2 * MNB * MNB + 6 * MQ * N + 3 * MQ * MNB + 4 * MQ * MQ;
    const int team_vals = 6 * N3 + face_vals;
    const int team = threadIdx.x / N2, tid = threadIdx.x - team * N2;
    const int ei = blockIdx.x * E + team;
    const bool has = team < E && ei < count;
    const int e = has ? bucket[ei] : -1;

    for (int k = threadIdx.x; k < N2; k += blockDim.x) {
        sI[k] = L.tab[tab_n(TabIndex::I, N) + k];
        sDg[k] = L.tab[tab_n(TabIndex::Dg, N) + k];
        sDL[k] = L.tab[tab_n(TabIndex::DL, N) + k];
    }
    T* U = sDL + N2 + (has ? team : 0) * team_vals;
    T* A = U + N3;
    T* B = A + N3;
    T* G1 = B + N3;
    T* G2 = G1 + N3;
    T* G3 = G2 + N3;
    T* F = G3 + N3;
    long long dofo = 0, vo = 0;
    if (has) {
        dofo = L.dof_off[e];
        vo = L.vqp_off[e];
        for (int k = tid; k < N3; k += N2) U[k] = x[dofo + k];
    }
    __syncthreads();
    // ---- volume -------------------------------------------------------------
    if (has) pass<N, 0, false, false>(U, A, sI, tid);
    __syncthreads();
    if (has) pass<N, 1, false, false>(A, B, sI, tid);
    __syncthreads();
    if (has) pass<N, 2, false, false>(B, A, sI, tid);
    __syncthreads();
    if (has) {
        pass<N, 0, false, false>(A, G1, sDg, tid);
        pass<N, 1, false, false>(A, G2, sDg, tid);
        pass<N, 2, false, false>(A, G3, sDg, tid);
    }
    __syncthreads();
    const bool mass = L.c0 != nullptr;
    if (has) {
        const T* Ge = L.G + 6 * vo;
        for (int k = tid; k < N3; k += N2) {
            const T g0 = G1[k], g1 = G2[k], g2 = G3[k];
            const T m00 = Ge[k], m01 = Ge[N3 + k], m02 = Ge[2 * N3 + k];
            const T m11 = Ge[3 * N3 + k], m12 = Ge[4 * N3 + k], m22 = Ge[5 * N3 + k];
            G1[k] = m00 * g0 + m01 * g1 + m02 * g2;
            G2[k] = m01 * g0 + m11 * g1 + m12 * g2;
            G3[k] = m02 * g0 + m12 * g1 + m22 * g2;
            if (mass) B[k] = L.c0[vo + k] * A[k];
        }
    }
    __syncthreads();
    if (has) {
        if (mass) pass<N, 0, true, true>(G1, B, sDg, tid);
        else pass<N, 0, true, false>(G1, B, sDg, tid);
    }
    __syncthreads();
    if (has) pass<N, 1, true, true>(G2, B, sDg, tid);
    __syncthreads();
    if (has) pass<N, 2, true, true>(G3, B, sDg, tid);
    __syncthreads();
    if (has) pass<N, 0, true, false>(B, A, sI, tid);
    __syncthreads();
    if (has) pass<N, 1, true, false>(A, G1, sI, tid);
    __syncthreads();
    T* Y = G2;
    if (has) pass<N, 2, true, false>(G1, Y, sI, tid);
    __syncthreads();
    if (has && L.Ob != nullptr) {
        const T* Oe = L.Ob + L.Ob_off[e];
        for (int k = tid; k < N3; k += N2) {
            T s = 0;
            for (int j = 0; j < N3; ++j) s += Oe[(long long)j * N3 + k] * U[j];
            Y[k] += s;
        }
    }
    // ---- faces ----------------------------------------------------------------
    __shared__ int s_nslots;
    if (threadIdx.x == 0) s_nslots = 0;
    __syncthreads();
    int s0 = 0, s1 = 0;
    if (has) {
        s0 = L.slot_off[e];
        s1 = L.slot_off[e + 1];
        if (tid == 0) atomicMax(&s_nslots, s1 - s0);
    }
    __syncthreads();
    const int ns = s_nslots;
    T* uf = F;
    T* df = uf + N2;
    T* ufn = df + N2;
    T* dfn = ufn + MNB * MNB;
    T* U1o = dfn + MNB * MNB;
    T* DU1o = U1o + MQ * N;
    T* N1o = DU1o + MQ * N;
    T* U1n = N1o + MQ * N;
    T* DU1n = U1n + MQ * MNB;
    T* N1n = DU1n + MQ * MNB;
    T* PA = N1n + MQ * MNB;
    T* PB1 = PA + MQ * MQ;
    T* PB2 = PB1 + MQ * MQ;
    T* PBn = PB2 + MQ * MQ;
    T* X1 = PBn + MQ * MQ;
    T* X2 = X1 + MQ * N;
    T* X3 = X2 + MQ * N;
    const int st[3] = {1, N, N2};
    for (int si = 0; si < ns; ++si) {
        const bool act = has && si < s1 - s0;
        int f = 0, side = 0, q = 2, nbN = 2, eo = -1, fo = 0, p0 = 0, p1 = 0, o0 = 0, o1 = 0;
        long long goff = 0;
        T sig = 0;
        if (act) {
            const int mi = L.slot_mortar[s0 + si];
            f = L.slot_face[s0 + si];
            side = L.slot_side[s0 + si];
            const Mortar M = L.mortars[mi];
            q = M.q;
            goff = M.goff;
            sig = L.sigma[mi];
            if (side == 0) { p0 = M.posA0; p1 = M.posA1; eo = M.eB; fo = M.fB; o0 = M.posB0; o1 = M.posB1; }
            else { p0 = M.posB0; p1 = M.posB1; eo = M.eA; fo = M.fA; o0 = M.posA0; o1 = M.posA1; }
            if (eo >= 0) nbN = L.p[eo] + 1;
        }
        const int d = f >> 1, s = f & 1;
        int t1, t2;
        tangential(d, t1, t2);
        const int fn = s ? N - 1 : 0;
        // S1: own trace u and d_nu u at own face LGL nodes; neighbour's from x
        if (act) {
            for (int k = tid; k < N2; k += N2) {
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
                for (int k = tid; k < nbN * nbN; k += N2) {
                    const int a = k % nbN, b = k / nbN;
                    const int base = a * nst[t1] + b * nst[t2];
                    ufn[k] = xe[base + fno * nst[d]];
                    T acc = 0;
                    for (int c = 0; c < nbN; ++c) acc += DLn[c] * xe[base + c * nst[d]];
                    dfn[k] = acc;
                }
            }
        }
        __syncthreads();
        // S2: interpolate along the first tangential axis
        if (act) {
            const T* Im1 = L.tab + tab_m(TabIndex::Im, N, q, p0);
            const T* Dm1 = L.tab + tab_m(TabIndex::Dm, N, q, p0);
            for (int k = tid; k < q * N; k += N2) {
                const int i1 = k % q, b = k / q;
                T su = 0, sd = 0, sn = 0;
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    const T iv = Im1[i1 * N + a], dv = Dm1[i1 * N + a];
                    su += iv * uf[a + N * b];
                    sd += dv * uf[a + N * b];
                    sn += iv * df[a + N * b];
                }
                U1o[k] = su;
                DU1o[k] = sd;
                N1o[k] = sn;
            }
            if (eo >= 0) {
                const T* Im1n = L.tab + tab_m(TabIndex::Im, nbN, q, o0);
                const T* Dm1n = L.tab + tab_m(TabIndex::Dm, nbN, q, o0);
                for (int k = tid; k < q * nbN; k += N2) {
                    const int i1 = k % q, b = k / q;
                    T su = 0, sd = 0, sn = 0;
                    for (int a = 0; a < nbN; ++a) {
                        const T iv = Im1n[i1 * nbN + a], dv = Dm1n[i1 * nbN + a];
                        su += iv * ufn[a + nbN * b];
                        sd += dv * ufn[a + nbN * b];
                        sn += iv * dfn[a + nbN * b];
                    }
                    U1n[k] = su;
                    DU1n[k] = sd;
                    N1n[k] = sn;
                }
            }
        }
        __syncthreads();
        // S3: values at the mortar points, numerical flux, lift coefficients
        if (act) {
            const T* Im2 = L.tab + tab_m(TabIndex::Im, N, q, p1);
            const T* Dm2 = L.tab + tab_m(TabIndex::Dm, N, q, p1);
            const T* Im2n = L.tab + tab_m(TabIndex::Im, nbN, q, o1);
            const T* Dm2n = L.tab + tab_m(TabIndex::Dm, nbN, q, o1);
            const int q2 = q * q;
            const T* mg = L.mg + 7 * goff;
            const T sgn = side == 0 ? T(1) : T(-1);
            for (int k = tid; k < q2; k += N2) {
                const int i1 = k % q, i2 = k / q;
                T u = 0, gt1 = 0, gt2 = 0, gn = 0;
#pragma unroll
                for (int b = 0; b < N; ++b) {
                    const T iv = Im2[i2 * N + b], dv = Dm2[i2 * N + b];
                    u += iv * U1o[i1 + q * b];
                    gt1 += iv * DU1o[i1 + q * b];
                    gt2 += dv * U1o[i1 + q * b];
                    gn += iv * N1o[i1 + q * b];
                }
                const T wS = mg[k];
                T co[3], cn[3];
                for (int l = 0; l < 3; ++l) {
                    co[l] = sgn * mg[(side == 0 ? 1 + l : 4 + l) * q2 + k];
                    cn[l] = sgn * mg[(side == 0 ? 4 + l : 1 + l) * q2 + k];
                }
                const T dno = co[t1] * gt1 + co[t2] * gt2 + co[d] * gn;
                T jmp, avg, bc;
                if (eo >= 0) {
                    T un = 0, ht1 = 0, ht2 = 0, hn = 0;
                    for (int b = 0; b < nbN; ++b) {
                        const T iv = Im2n[i2 * nbN + b], dv = Dm2n[i2 * nbN + b];
                        un += iv * U1n[i1 + q * b];
                        ht1 += iv * DU1n[i1 + q * b];
                        ht2 += dv * U1n[i1 + q * b];
                        hn += iv * N1n[i1 + q * b];
                    }
                    const T dnn = cn[t1] * ht1 + cn[t2] * ht2 + cn[d] * hn;
                    jmp = u - un;
                    avg = T(0.5) * (dno + dnn);
                    bc = T(-0.5) * wS * jmp;
                } else {
                    jmp = u;
                    avg = dno;
                    bc = -wS * jmp;
                }
                PA[k] = wS * (sig * jmp - avg);
                PB1[k] = bc * co[t1];
                PB2[k] = bc * co[t2];
                PBn[k] = bc * co[d];
            }
        }
        __syncthreads();
        // S4: transposed interpolation along the second tangential axis
        if (act) {
            const T* Im2 = L.tab + tab_m(TabIndex::Im, N, q, p1);
            const T* Dm2 = L.tab + tab_m(TabIndex::Dm, N, q, p1);
            for (int k = tid; k < q * N; k += N2) {
                const int i1 = k % q, b = k / q;
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
        }
        __syncthreads();
        // S5: transposed interpolation along the first axis and lift into y
        if (act) {
            const T* Im1 = L.tab + tab_m(TabIndex::Im, N, q, p0);
            const T* Dm1 = L.tab + tab_m(TabIndex::Dm, N, q, p0);
            for (int k = tid; k < N2; k += N2) {
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
        }
        __syncthreads();
    }
    if (has)
        for (int k = tid; k < N3; k += N2) y[dofo + k] = Y[k];
}

template <int N, typename T>
cudaError_t launch_n(const LevelView<T>& L, const BucketInfo& b, const T* x, T* y, cudaStream_t st) {
    constexpr int N2 = N * N, N3 = N2 * N;
    const int MQ = b.max_q, MNB = b.max_nb;
    const int face_vals = 2 * N2 + 2 * MNB * MNB + 6 * MQ * N + 3 * MQ * MNB + 4 * MQ * MQ;
    const size_t team_bytes = sizeof(T) * (6 * N3 + face_vals);
    const size_t budget = 110 * 1024;
    int E = 256 / N2;
    while (E > 1 && 3 * N2 * sizeof(T) + E * team_bytes > budget) --E;
    const size_t smem = 3 * N2 * sizeof(T) + E * team_bytes;
    static bool attr_set[2] = {false, false};
    const int ti = sizeof(T) == 8 ? 0 : 1;
    if (!attr_set[ti]) {
        cudaError_t err = cudaFuncSetAttribute(apply_kernel<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (err != cudaSuccess) return err;
        attr_set[ti] = true;
    }
    const int grid = (b.count + E - 1) / E;
    apply_kernel<N, T><<<grid, E * N2, smem, st>>>(L, b.elems, b.count, E, MQ, MNB, x, y);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_apply(const LevelView<T>& L, const BucketInfo* buckets, const T* x, T* y, cudaStream_t st,
                         int* launches) {
    for (int n = kMinN; n <= kMaxN; ++n) {
        const BucketInfo& b = buckets[n];
        if (b.count == 0) continue;
        cudaError_t err = cudaSuccess;
        switch (n) {
            case 2: err = launch_n<2, T>(L, b, x, y, st); break;
            case 3: err = launch_n<3, T>(L, b, x, y, st); break;
            case 4: err = launch_n<4, T>(L, b, x, y, st); break;
            case 5: err = launch_n<5, T>(L, b, x, y, st); break;
            case 6: err = launch_n<6, T>(L, b, x, y, st); break;
            case 7: err = launch_n<7, T>(L, b, x, y, st); break;
            case 8: err = launch_n<8, T>(L, b, x, y, st); break;
            case 9: err = launch_n<9, T>(L, b, x, y, st); break;
        }
        if (err != cudaSuccess) return err;
        if (launches) ++*launches;
    }
    return cudaSuccess;
}

template cudaError_t launch_apply<double>(const LevelView<double>&, const BucketInfo*, const double*, double*,
                                          cudaStream_t, int*);
template cudaError_t launch_apply<float>(const LevelView<float>&, const BucketInfo*, const float*, float*,
                                         cudaStream_t, int*);

}  // namespace dg
