// Matrix-free SIPG operator apply (eq. lh2) in two element-centric kernels
// per polynomial-degree bucket.
//
// Trace kernel: for every mortar touching the element (Sec. II.A.5, mortar
// figure), the element's own trace u and normal derivative n_A . grad u at the
// mortar's p_m + 1 GL points per direction: the face values and the face-normal
// LGL derivative are interpolated with the sub-face / degree-change tables and
// contracted with c = (J^-1) n_A of this side.  Written to the mortar trace
// buffer MT (per mortar [u_A, dn_A, u_B, dn_B]).
//
// Element kernel (after all trace kernels of the level):
// Volume (eq. harald-stiff), sum-factorised with 1-D operators (Sec. II.F.4):
//   u~ = (I x I x I) u            values at the GL points         (3 passes)
//   g_l = Dg_l u~                 reference gradient at GL points (3 passes)
//   f_l = G_lm g_m                G = w det J J^-1 J^-T (stored)
//   z = sum_l Dg_l^T f_l (+ c0 u~ for the zeroth-order term)     (3 passes)
//   y = (I x I x I)^T z                                           (3 passes)
// Faces (consistency, symmetry and penalty integrals of eq. lh2): with n the
// element's outward normal (= sgn n_A) and both sides' traces from MT,
//   j = u_own - u_nb,  a = {n . grad u} = sgn (dn_A + dn_B) / 2,
//   y_alpha += sum_pts wS [ (sigma j - a) psi_alpha - (1/2) j n . grad psi_alpha ]
// (Dirichlet mortars: j = u_own, a = n . grad u_own, factor 1 instead of 1/2),
// lifted through the transposed mortar tables and the face-normal row of the
// LGL derivative matrix.
//
// Execution: one warp per element (lanes own pencils / face points, __syncwarp
// between phases); persistent CTAs stride over the bucket, sized for the most
// resident warps that shared memory and registers allow; face loops are
// compiled per mortar size q; FP32 stages every mortar table in shared memory
// as (Im, Dm) pairs.  Each element of a bucket has a descriptor (offsets and
// slot range) and each slot a packed record, so one broadcast load and one
// load per lane start an element; the next element's descriptor is loaded
// while the current one runs, and its input and slot records are prefetched
// into L2.  The element's metric terms and per-mortar data are prefetched into
// L2 while the volume passes run, so the face stages mostly hit L2 instead of
// DRAM.  Loops that move global data into shared memory issue all of a lane's
// loads before its stores.  An element's values sit in shared memory with
// padded strides (Strides) so that the pencil passes are free of bank
// conflicts for every N.
#pragma once
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>

#include "apply.h"

namespace dg {
namespace apply_detail {

constexpr int kQ = kMaxN;  // largest mortar q

// Operand load: FP32 / FP64 vectors as stored, BF16 vectors widened to FP32.
template <typename T, typename TX>
__device__ __forceinline__ T ld(const TX* p) {
    if constexpr (sizeof(TX) == 2) return (T)__bfloat162float(*p);
    else return *p;
}

__device__ inline void tangential(int d, int& t1, int& t2) {
    t1 = d == 0 ? 1 : 0;
    t2 = d == 2 ? 1 : 2;
}

// Per-warp arrays start on multiples of four values (16-byte boundaries).
constexpr int r4(int v) { return (v + 3) & ~3; }

// Shared-memory layout of an element's N^3 values: node (a, b, c) at
// a + S1 b + S2 c.  The padding puts the 32 lanes of a pencil pass (one
// x-, y- or z-pencil per lane) into distinct banks where the dense layout
// does not: N = 8 (rows of 9, planes of 72; dense: 8-way conflicts along x,
// 4-way along y) and N = 7 (planes of 52).
template <int N>
struct Strides {
    static constexpr int S1 = N == 8 ? 9 : N;
    static constexpr int S2 = N == 8 ? 72 : (N == 7 ? 52 : N * N);
    static constexpr int SIZE = S2 * N;
};

// Stride of reference direction k (0, 1, 2) in the padded layout; a select
// rather than a table, which a run-time index would put in local memory.
template <int N>
__device__ __forceinline__ int stride_of(int k) {
    return k == 0 ? 1 : (k == 1 ? Strides<N>::S1 : Strides<N>::S2);
}

// Padded shared-memory index of the node with element-blocked index k.
template <int N>
__device__ __forceinline__ int sidx(int k) {
    return k % N + Strides<N>::S1 * ((k / N) % N) + Strides<N>::S2 * (k / (N * N));
}

template <typename T, typename TX>
__device__ __forceinline__ T ld(const TX* p);

// An element's N^3 input values into shared memory (padded layout).  All of
// a lane's global loads are issued before its first shared-memory store: the
// compiler cannot move a load past a store through a generic pointer, so a
// load-store loop would wait for each load in turn.
template <int N, typename T, typename TX>
__device__ __forceinline__ void load_element(const TX* __restrict__ x, T* __restrict__ U, int lane) {
    constexpr int N3 = N * N * N, R = (N3 + 31) / 32;
    T v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int k = lane + 32 * j;
        v[j] = k < N3 ? ld<T>(x + k) : T(0);
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int k = lane + 32 * j;
        if (k < N3) U[sidx<N>(k)] = v[j];
    }
}

// One (Im, Dm) pair of the mortar tables: a single 8- or 16-byte access.
template <typename T>
__device__ __forceinline__ void ld2(const T* p, T& a, T& b) {
    if constexpr (sizeof(T) == 4) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        a = v.x;
        b = v.y;
    } else {
        const double2 v = *reinterpret_cast<const double2*>(p);
        a = v.x;
        b = v.y;
    }
}

// Values of the element's 1-D volume tables in shared memory: I and Dg, each
// followed by its transpose, rows padded to a multiple of four values (a row is
// read with 16-byte accesses, the same address in every lane), then DL (N x N).
__host__ __device__ constexpr int vol_vals(int n) { return 4 * n * r4(n) + r4(n * n); }

template <int N, typename T>
__device__ __forceinline__ void load_row(const T* __restrict__ r, T (&m)[N]) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int j = 0; j < (N + 3) / 4; ++j) {
            const float4 v = reinterpret_cast<const float4*>(r)[j];
            if (4 * j < N) m[4 * j] = v.x;
            if (4 * j + 1 < N) m[4 * j + 1] = v.y;
            if (4 * j + 2 < N) m[4 * j + 2] = v.z;
            if (4 * j + 3 < N) m[4 * j + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < (N + 1) / 2; ++j) {
            const double2 v = reinterpret_cast<const double2*>(r)[j];
            m[2 * j] = v.x;
            if (2 * j + 1 < N) m[2 * j + 1] = v.y;
        }
    }
}

// P pencils per thread (pencil t + j nt): every row of the operator is read
// once and applied to all of them.
template <int N, int DIR, bool ACC, int P, typename T>
__device__ __forceinline__ void pass_rows(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ R,
                                          int t, int nt) {
    constexpr int NP = r4(N);
    constexpr int S1 = Strides<N>::S1, S2 = Strides<N>::S2;
    constexpr int stride = DIR == 0 ? 1 : (DIR == 1 ? S1 : S2);
    T v[P][N];
    int base[P];
    bool ok[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
        const int pid = t + j * nt;
        ok[j] = pid < N * N;
        const int u = pid % N, w = pid / N;   // the pencil's two other coordinates
        base[j] = DIR == 0 ? S1 * u + S2 * w : (DIR == 1 ? u + S2 * w : u + S1 * w);
#pragma unroll
        for (int m = 0; m < N; ++m) v[j][m] = ok[j] ? in[base[j] + m * stride] : T(0);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        T r[N];
        load_row<N>(R + i * NP, r);
#pragma unroll
        for (int j = 0; j < P; ++j) {
            T s = 0;
#pragma unroll
            for (int m = 0; m < N; ++m) s += r[m] * v[j][m];
            if (ok[j]) {
                if (ACC) out[base[j] + i * stride] += s;
                else out[base[j] + i * stride] = s;
            }
        }
    }
}

// out = M in along direction DIR of an N^3 array held by nt threads (TRANS: M^T; ACC: out +=);
// M points at the padded rows of the operator, its transpose follows.
template <int N, int DIR, bool TRANS, bool ACC, typename T>
__device__ inline void wpass(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ M, int t,
                             int nt = 32) {
    const T* R = TRANS ? M + N * r4(N) : M;
    if (nt == 32) {
        pass_rows<N, DIR, ACC, (N * N + 31) / 32>(in, out, R, t, 32);
    } else {
        for (int t0 = t; t0 < N * N; t0 += nt) pass_rows<N, DIR, ACC, 1>(in, out, R, t0, nt);
    }
}

// ---- tensor-core passes (FP32 and BF16-operand applies, N <= 8) -------------
// A pass out[p][i] (+)= sum_m R[i][m] in[p][m] over the element's N^2 pencils p
// is a GEMM (pencils x m) . (m x i): per tile of 16 pencils one
// mma.sync.m16n8k8 TF32 product with K = 8 and 8 output columns (m and i
// zero-padded past N).  Each FP32 operand is split into a TF32 head and a
// TF32 tail (x = hi + lo to about 2^-22), and the product is taken as
// lo_a hi_b + hi_a lo_b + hi_a hi_b (the lo lo term is below FP32 rounding),
// so a pass keeps FP32 accuracy on the tensor pipe.
__device__ __forceinline__ void split_tf32(float x, unsigned& hi, unsigned& lo) {
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
    const float r = x - __uint_as_float(hi);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// B fragments (head and tail) of one operator R (rows R[i][m] padded to
// r4(N), as staged in shared memory): B[k][j] = R[j][k], lane (g, t) =
// (lane / 4, lane % 4) holding B[t][g] and B[t + 4][g].
struct OpFrag {
    unsigned hi[2], lo[2];
};

template <int N>
__device__ __forceinline__ OpFrag op_frag(const float* __restrict__ R, int lane) {
    constexpr int NP = r4(N);
    const int g = lane >> 2, t = lane & 3;
    OpFrag f;
    const float b0 = (g < N && t < N) ? R[g * NP + t] : 0.f;
    const float b1 = (g < N && t + 4 < N) ? R[g * NP + t + 4] : 0.f;
    split_tf32(b0, f.hi[0], f.lo[0]);
    split_tf32(b1, f.hi[1], f.lo[1]);
    return f;
}

// The four volume operators of an element kernel: I, I^T, Dg, Dg^T.
struct VolFrags {
    OpFrag f[4];
};

template <int N>
__device__ __forceinline__ VolFrags vol_frags(const float* sI, const float* sDg, int lane) {
    constexpr int NP = r4(N);
    VolFrags v;
    v.f[0] = op_frag<N>(sI, lane);
    v.f[1] = op_frag<N>(sI + N * NP, lane);
    v.f[2] = op_frag<N>(sDg, lane);
    v.f[3] = op_frag<N>(sDg + N * NP, lane);
    return v;
}

// Shared-memory offset of pencil pid (of N^2) along direction DIR.
template <int N, int DIR>
__device__ __forceinline__ int pencil_base(int pid) {
    constexpr int S1 = Strides<N>::S1, S2 = Strides<N>::S2;
    const int u = pid % N, w = pid / N;
    return DIR == 0 ? S1 * u + S2 * w : (DIR == 1 ? u + S2 * w : u + S1 * w);
}

template <int N, int DIR, bool ACC>
__device__ __forceinline__ void mma_pass(const float* __restrict__ in, float* __restrict__ out, const OpFrag& B,
                                         int lane) {
    constexpr int S1 = Strides<N>::S1, S2 = Strides<N>::S2;
    constexpr int stride = DIR == 0 ? 1 : (DIR == 1 ? S1 : S2);
    constexpr int NN = N * N, TILES = (NN + 15) / 16;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int tile = 0; tile < TILES; ++tile) {
        const int p0 = 16 * tile + g, p1 = p0 + 8;
        const bool v0 = p0 < NN, v1 = p1 < NN;
        const int b0 = pencil_base<N, DIR>(v0 ? p0 : 0), b1 = pencil_base<N, DIR>(v1 ? p1 : 0);
        float a[4];
        a[0] = (v0 && t < N) ? in[b0 + t * stride] : 0.f;
        a[1] = (v1 && t < N) ? in[b1 + t * stride] : 0.f;
        a[2] = (v0 && t + 4 < N) ? in[b0 + (t + 4) * stride] : 0.f;
        a[3] = (v1 && t + 4 < N) ? in[b1 + (t + 4) * stride] : 0.f;
        unsigned ah[4], al[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) split_tf32(a[j], ah[j], al[j]);
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        mma_tf32(d, al, B.hi);
        mma_tf32(d, ah, B.lo);
        mma_tf32(d, ah, B.hi);
        const int i0 = 2 * t, i1 = 2 * t + 1;
        if (v0 && i0 < N) out[b0 + i0 * stride] = ACC ? out[b0 + i0 * stride] + d[0] : d[0];
        if (v0 && i1 < N) out[b0 + i1 * stride] = ACC ? out[b0 + i1 * stride] + d[1] : d[1];
        if (v1 && i0 < N) out[b1 + i0 * stride] = ACC ? out[b1 + i0 * stride] + d[2] : d[2];
        if (v1 && i1 < N) out[b1 + i1 * stride] = ACC ? out[b1 + i1 * stride] + d[3] : d[3];
    }
}

// Volume pass of the warp-per-element kernel: on the tensor pipe for 32-bit
// values and N = 8 (W: 0 I, 1 I^T, 2 Dg, 3 Dg^T), else on the FP32/FP64 pipe.
// Measured on the 32^3 sweep mesh, the tensor passes match the FP32-pipe ones
// in speed; at N = 8 they need fewer registers, at N = 6, 7 more.
template <int N, typename T>
constexpr bool use_mma() {
    return sizeof(T) == 4 && N == 8;
}

template <int N, int DIR, int W, bool ACC, typename T>
__device__ __forceinline__ void vpass(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ M,
                                      const VolFrags& fr, int lane) {
    if constexpr (use_mma<N, T>()) {
        mma_pass<N, DIR, ACC>(in, out, fr.f[W], lane);
    } else {
        wpass<N, DIR, (W & 1) != 0, ACC>(in, out, M, lane);
    }
}

template <typename T>
struct SlotInfo {
    int f, side, p0, p1, q;
    int o;                 // side B across a block interface: orientation of its face frame (blocks.h)
    long long goff;
};

// Index, in the mortar's point order (side A's face frame), of the point at
// (j1, j2) of this side's own Q x Q face grid, as c0 + c1 j1 + c2 j2: the GL
// points are symmetric, so a mirrored axis maps j to Q - 1 - j, and a swap
// exchanges the roles of the two axes.
template <int Q>
struct MortarMap {
    int c0, c1, c2;
    __device__ __forceinline__ explicit MortarMap(int o) {
        const int a1 = (o & 2) ? Q - 1 : 0, b1 = (o & 2) ? -1 : 1;
        const int a2 = (o & 4) ? Q - 1 : 0, b2 = (o & 4) ? -1 : 1;
        if (o & 1) {
            c0 = a2 + Q * a1;
            c1 = Q * b1;
            c2 = b2;
        } else {
            c0 = a1 + Q * a2;
            c1 = b1;
            c2 = Q * b2;
        }
    }
    __device__ __forceinline__ int operator()(int j1, int j2) const { return c0 + c1 * j1 + c2 * j2; }
};

template <typename T>
__device__ __forceinline__ SlotInfo<T> slot_info(const LevelView<T>& L, int si) {
    SlotInfo<T> s;
    const Mortar M = L.mortars[L.slot_mortar[si]];
    s.f = L.slot_face[si];
    s.side = L.slot_side[si];
    s.p0 = s.side == 0 ? M.posA0 : M.posB0;
    s.p1 = s.side == 0 ? M.posA1 : M.posB1;
    s.q = M.q;
    s.o = s.side == 0 ? 0 : M.orient;
    s.goff = M.goff;
    return s;
}

// Own trace at the Q x Q mortar points: u and dn = c^side . grad_xi u (c^side =
// J^-1 n_A, three Q^2 blocks at co).  Mortar tables are (Im, Dm) pairs.  The
// side works on its own face grid; per-point data and the trace buffer are in
// the mortar's point order (side A's frame), reached through MortarMap.
template <int N, int Q, typename T, bool OR = true>
__device__ __forceinline__ void trace_slot(const LevelView<T>& L, const SlotInfo<T>& s, const T* __restrict__ U,
                                           const T* __restrict__ sDL, const T* __restrict__ sFT, T* F,
                                           const T* __restrict__ co, T* __restrict__ mt, int lane) {
    if constexpr (Q < N) {
        return;
    } else {
        constexpr int N2 = N * N, Q2 = Q * Q;
        const int d = s.f >> 1, fn = (s.f & 1) ? N - 1 : 0;
        int t1, t2;
        tangential(d, t1, t2);
        const int sdn = stride_of<N>(d), st1 = stride_of<N>(t1), st2 = stride_of<N>(t2);
        const MortarMap<Q> toA(OR ? s.o : 0);
        // this side's c at the lane's mortar points, loaded first so that they
        // arrive while the two interpolation passes run
        constexpr int QJ = (Q2 + 31) / 32;
        T c1[QJ], c2[QJ], cn[QJ];
#pragma unroll
        for (int j = 0; j < QJ; ++j) {
            const int kk = lane + 32 * j < Q2 ? lane + 32 * j : 0;
            const int kA = OR ? toA(kk % Q, kk / Q) : kk;
            c1[j] = co[t1 * Q2 + kA];
            c2[j] = co[t2 * Q2 + kA];
            cn[j] = co[d * Q2 + kA];
        }
        T* uf = F;                  // u and n . grad_xi u at the N x N face nodes
        T* df = uf + N2;
        T* U1 = df + N2;            // u, d/dt1 u, dn u after the first tangential direction (Q x N)
        T* DU1 = U1 + Q * N;
        T* N1 = DU1 + Q * N;
#pragma unroll
        for (int k0 = 0; k0 < N2; k0 += 32) {   // unrolled: a lane's iterations overlap
            const int k = k0 + lane;
            if (k >= N2) continue;
            const int a = k % N, b = k / N;
            const int base = a * st1 + b * st2;
            T v[N];
#pragma unroll
            for (int c = 0; c < N; ++c) v[c] = U[base + c * sdn];
            T acc = 0;
#pragma unroll
            for (int c = 0; c < N; ++c) acc += sDL[fn * N + c] * v[c];
            uf[k] = fn ? v[N - 1] : v[0];
            df[k] = acc;
        }
        __syncwarp();
        const T* M1 = sFT + L.ft.off[N - kMinN][Q - kMinN][s.p0];
#pragma unroll
        for (int k0 = 0; k0 < Q * N; k0 += 32) {   // unrolled: a lane's iterations overlap
            const int k = k0 + lane;
            if (k >= Q * N) continue;
            const int i1 = k % Q, b = k / Q;
            T su = 0, sd = 0, sn = 0;
#pragma unroll
            for (int a = 0; a < N; ++a) {
                T iv, dv;
                ld2(M1 + 2 * (i1 * N + a), iv, dv);
                const T u = uf[a + N * b], dn = df[a + N * b];
                su += iv * u;
                sd += dv * u;
                sn += iv * dn;
            }
            U1[k] = su;
            DU1[k] = sd;
            N1[k] = sn;
        }
        __syncwarp();
        const T* M2 = sFT + L.ft.off[N - kMinN][Q - kMinN][s.p1];
        T* out = mt + 4 * s.goff + 2 * s.side * Q2;
#pragma unroll
        for (int k0 = 0; k0 < Q2; k0 += 32) {   // unrolled: a lane's iterations overlap
            const int k = k0 + lane;
            if (k >= Q2) continue;
            const int i1 = k % Q, i2 = k / Q, kA = OR ? toA(i1, i2) : k;
            T u = 0, g1 = 0, g2 = 0, gn = 0;
#pragma unroll
            for (int b = 0; b < N; ++b) {
                T iv, dv;
                ld2(M2 + 2 * (i2 * N + b), iv, dv);
                const T ub = U1[i1 + Q * b], dub = DU1[i1 + Q * b], nb = N1[i1 + Q * b];
                u += iv * ub;
                g1 += iv * dub;
                g2 += dv * ub;
                gn += iv * nb;
            }
            out[kA] = u;
            out[Q2 + kA] = c1[k0 / 32] * g1 + c2[k0 / 32] * g2 + cn[k0 / 32] * gn;
        }
        __syncwarp();
    }
}

// Lift of one mortar's flux into Y (the transposed mortar interpolation in
// both tangential directions and the face-normal row of the LGL derivative):
// PA, PB1, PB2, PBn (Q^2 each, consecutive from PA) are the flux factors at
// the mortar points; X holds 3 Q N values of scratch.
template <int N, int Q, typename T>
__device__ __forceinline__ void lift_apply(const LevelView<T>& L, const SlotInfo<T>& s, T* __restrict__ Y,
                                           const T* __restrict__ sDL, const T* __restrict__ sFT,
                                           const T* __restrict__ PA, T* __restrict__ X, int lane) {
    if constexpr (Q < N) {
        return;
    } else {
        constexpr int N2 = N * N, Q2 = Q * Q;
        const int d = s.f >> 1, fn = (s.f & 1) ? N - 1 : 0;
        int t1, t2;
        tangential(d, t1, t2);
        const int sdn = stride_of<N>(d), st1 = stride_of<N>(t1), st2 = stride_of<N>(t2);
        const T* PB1 = PA + Q2;
        const T* PB2 = PB1 + Q2;
        const T* PBn = PB2 + Q2;
        T* X1 = X;
        T* X2 = X1 + Q * N;
        T* X3 = X2 + Q * N;
        const T* M2 = sFT + L.ft.off[N - kMinN][Q - kMinN][s.p1];
#pragma unroll
        for (int k0 = 0; k0 < Q * N; k0 += 32) {   // unrolled: a lane's iterations overlap
            const int k = k0 + lane;
            if (k >= Q * N) continue;
            const int i1 = k % Q, b = k / Q;
            T s1v = 0, s2v = 0, s3v = 0;
#pragma unroll
            for (int i2 = 0; i2 < Q; ++i2) {
                T iv, dv;
                ld2(M2 + 2 * (i2 * N + b), iv, dv);
                s1v += iv * PA[i1 + Q * i2] + dv * PB2[i1 + Q * i2];
                s2v += iv * PB1[i1 + Q * i2];
                s3v += iv * PBn[i1 + Q * i2];
            }
            X1[k] = s1v;
            X2[k] = s2v;
            X3[k] = s3v;
        }
        __syncwarp();
        const T* M1 = sFT + L.ft.off[N - kMinN][Q - kMinN][s.p0];
#pragma unroll
        for (int k0 = 0; k0 < N2; k0 += 32) {   // unrolled: a lane's iterations overlap
            const int k = k0 + lane;
            if (k >= N2) continue;
            const int a = k % N, b = k / N;
            T fu = 0, fd = 0;
#pragma unroll
            for (int i1 = 0; i1 < Q; ++i1) {
                T iv, dv;
                ld2(M1 + 2 * (i1 * N + a), iv, dv);
                fu += iv * X1[i1 + Q * b] + dv * X2[i1 + Q * b];
                fd += iv * X3[i1 + Q * b];
            }
            const int base = a * st1 + b * st2;
            Y[base + fn * sdn] += fu;
#pragma unroll
            for (int c = 0; c < N; ++c) Y[base + c * sdn] += sDL[fn * N + c] * fd;
        }
        __syncwarp();
    }
}

// Flux at the mortar points and lift into Y for one mortar of the element.  Per
// mortar point: surface weight wSp, this side's c (three Q^2 blocks at co) and
// the trace buffer entries m = [u_A, dn_A, u_B, dn_B] (Q^2 each).
template <int N, int Q, typename T, bool OR = true, int BDM = 2>
__device__ __forceinline__ void lift_slot(const LevelView<T>& L, const SlotInfo<T>& s, bool interior, T sig,
                                          T* __restrict__ Y, const T* __restrict__ sDL, const T* __restrict__ sFT,
                                          T* F, const T* __restrict__ wSp, const T* __restrict__ co,
                                          const T* __restrict__ m, int lane) {
    if constexpr (Q < N) {
        return;
    } else {
        constexpr int Q2 = Q * Q;
        const int d = s.f >> 1;
        int t1, t2;
        tangential(d, t1, t2);
        T* PA = F;              // flux factors at the Q x Q mortar points
        T* PB1 = PA + Q2;
        T* PB2 = PB1 + Q2;
        T* PBn = PB2 + Q2;
        T* X1 = PBn + Q2;       // after the second tangential direction (Q x N)
        T* X2 = X1 + Q * N;
        T* X3 = X2 + Q * N;
        const T sgn = s.side == 0 ? T(1) : T(-1);
        const MortarMap<Q> toA(OR ? s.o : 0);
#pragma unroll
        for (int k0 = 0; k0 < Q2; k0 += 32) {   // unrolled: a lane's iterations overlap
            const int k = k0 + lane;
            if (k >= Q2) continue;
            const int kA = OR ? toA(k % Q, k / Q) : k;
            const T wS = wSp[kA];
            T uA = m[kA], dA = m[Q2 + kA];
            T jmp, avg, bc;
            if (interior) {
                T uB = m[2 * Q2 + kA], dB = m[3 * Q2 + kA];
                if (BDM == 1 || (BDM == 2 && L.bdiag)) {   // element diagonal block: the other side's trace is zero
                    if (s.side == 0) uB = dB = T(0);
                    else uA = dA = T(0);
                }
                jmp = sgn * (uA - uB);
                avg = T(0.5) * sgn * (dA + dB);
                bc = T(-0.5) * wS * jmp;
            } else {
                jmp = uA;
                avg = dA;
                bc = -wS * jmp;
            }
            const T b2 = bc * sgn;
            PA[k] = wS * (sig * jmp - avg);
            PB1[k] = b2 * co[t1 * Q2 + kA];
            PB2[k] = b2 * co[t2 * Q2 + kA];
            PBn[k] = b2 * co[d * Q2 + kA];
        }
        __syncwarp();
        lift_apply<N, Q, T>(L, s, Y, sDL, sFT, PA, X1, lane);
    }
}

#define DG_Q_SWITCH(QV, CALL)                                            \
    switch (QV) {                                                        \
        case 2: { constexpr int Q = 2; CALL; break; }                   \
        case 3: { constexpr int Q = 3; CALL; break; }                   \
        case 4: { constexpr int Q = 4; CALL; break; }                   \
        case 5: { constexpr int Q = 5; CALL; break; }                   \
        case 6: { constexpr int Q = 6; CALL; break; }                   \
        case 7: { constexpr int Q = 7; CALL; break; }                   \
        case 8: { constexpr int Q = 8; CALL; break; }                   \
        default: { constexpr int Q = 9; CALL; break; }                  \
    }

// Per-warp shared-memory layout (in values of T) of the warp-per-element kernels.
template <int N>
struct Layout {
    static constexpr int N2 = N * N, N3 = N2 * N, NR = r4(Strides<N>::SIZE);
    static constexpr int TFACE = 2 * N2 + 3 * kQ * N;                 // trace kernel face scratch
    static constexpr int TWARP = NR + TFACE;
    // Element kernel: Y, A, G1, U (the input buffer, dead after the first
    // volume pass, holds the z-gradient); in the face phase A, G1 and U hold
    // the face scratch (flux factors and lift partial sums).
    static constexpr bool UALIAS = true;
    static constexpr int EFACE = 4 * kQ * kQ + 3 * kQ * N;            // element kernel face scratch
    static constexpr int EWARP = r4(NR + (3 * NR > EFACE ? 3 * NR : EFACE));
};

// Values ahead of the per-warp scratch: FP32 mortar tables (staged) and the
// element's 1-D volume tables.
template <int N>
__host__ __device__ constexpr int table_vals(int ftot) {
    return r4(ftot) + vol_vals(N);
}

// One mortar slot of an element, packed so that a warp can hold the records of
// all of an element's slots (one per lane) and broadcast them by shuffles:
// info = face | side << 3 | pos0 << 4 | pos1 << 6 | q << 8 | interior << 12 |
// orientation << 13.
template <typename T>
struct SlotRec {
    int info;
    long long goff;
    T sig;
};

template <typename T>
__device__ __forceinline__ SlotRec<T> load_rec(const LevelView<T>& L, int si) {
    const int mi = L.slot_mortar[si];
    const Mortar M = L.mortars[mi];
    const int f = L.slot_face[si], side = L.slot_side[si];
    const int p0 = side == 0 ? M.posA0 : M.posB0, p1 = side == 0 ? M.posA1 : M.posB1;
    SlotRec<T> r;
    r.info = f | side << 3 | p0 << 4 | p1 << 6 | (int)M.q << 8 | (M.eB >= 0 ? 1 << 12 : 0) |
             (side ? (int)M.orient << 13 : 0);
    r.goff = M.goff;
    r.sig = L.sigma[mi];
    return r;
}

template <typename T>
__device__ __forceinline__ SlotInfo<T> unpack_rec(const SlotRec<T>& r) {
    SlotInfo<T> s;
    s.f = r.info & 7;
    s.side = (r.info >> 3) & 1;
    s.p0 = (r.info >> 4) & 3;
    s.p1 = (r.info >> 6) & 3;
    s.q = (r.info >> 8) & 15;
    s.o = (r.info >> 13) & 7;
    s.goff = r.goff;
    return s;
}

// L2 prefetch of the 128-byte lines holding [p, p + n): lanes lane0, lane0 +
// step, ... take one line each; every address issued lies inside the range.
template <typename T>
__device__ __forceinline__ void prefetch_l2(const T* p, long long n, int lane0, int step) {
    const unsigned long long a0 = (unsigned long long)__cvta_generic_to_global(p), a1 = a0 + n * sizeof(T);
    for (unsigned long long l = (a0 & ~127ull) + 128ull * lane0; l < a1; l += 128ull * step) {
        const unsigned long long a = l < a0 ? a0 : l;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    }
}

// The slot records of one element, lane j holding slot s0 + j: every face is
// covered by one or four mortars (checked when the connectivity is built), so
// an element has 6 to 24 slots.
template <typename T>
struct WarpSlots {
    int s0, s1;
    SlotRec<T> mine;
    __device__ __forceinline__ void load(const LevelView<T>& L, int a, int b, int lane) {
        s0 = a;
        s1 = b;
        if (s0 + lane < s1) {
            const SlotPack<T> sp = L.spack[s0 + lane];
            mine.info = sp.info;
            mine.goff = sp.goff;
            mine.sig = sp.sig;
        } else {
            mine.info = 0;
            mine.goff = 0;
            mine.sig = 0;
        }
    }
    // This lane's slot data into L2 ahead of its use: wS and this side's c, and
    // (lift) the mortar's trace buffer entries.
    __device__ __forceinline__ void prefetch(const LevelView<T>& L, int lane, bool lift) const {
        if (s0 + lane >= s1) return;
        const int q2 = ((mine.info >> 8) & 15) * ((mine.info >> 8) & 15), side = (mine.info >> 3) & 1;
        const T* mg = L.mg + 7 * mine.goff;
        if (lift) prefetch_l2(mg, q2, 0, 1);
        prefetch_l2(mg + (side ? 4 : 1) * q2, 3 * q2, 0, 1);
        if (lift) prefetch_l2(L.mt + 4 * mine.goff, ((mine.info >> 12) & 1) ? 4 * q2 : 2 * q2, 0, 1);
    }
    __device__ __forceinline__ SlotRec<T> get(int si) const {   // warp-uniform si in [s0, s1)
        const int src = si - s0;
        SlotRec<T> r;
        r.info = __shfl_sync(0xffffffffu, mine.info, src);
        r.goff = __shfl_sync(0xffffffffu, mine.goff, src);
        r.sig = __shfl_sync(0xffffffffu, mine.sig, src);
        return r;
    }
};

// Shared-memory preamble common to both kernels: mortar tables (FP32) and the
// element's 1-D volume tables; returns the first per-warp scratch value.
template <int N, typename T>
__device__ __forceinline__ T* load_tables(const LevelView<T>& L, const T*& sFT, const T*& sI, const T*& sDg,
                                          const T*& sDL) {
    constexpr bool STAGE = sizeof(T) == 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int ftot = STAGE ? L.ft.total : 0;
    T* sFTs = sm;
    sFT = STAGE ? sFTs : L.ftab;
    T* sV = sFTs + r4(ftot);
    for (int k = threadIdx.x; k < ftot; k += blockDim.x) sFTs[k] = L.ftab[k];
    constexpr int NP = r4(N);
    const T* tI = L.tab + tab_n(TabIndex::I, N);
    const T* tD = L.tab + tab_n(TabIndex::Dg, N);
    for (int k = threadIdx.x; k < N * NP; k += blockDim.x) {
        const int i = k / NP, m = k % NP;
        const bool in = m < N;
        sV[k] = in ? tI[i * N + m] : T(0);
        sV[N * NP + k] = in ? tI[m * N + i] : T(0);
        sV[2 * N * NP + k] = in ? tD[i * N + m] : T(0);
        sV[3 * N * NP + k] = in ? tD[m * N + i] : T(0);
    }
    for (int k = threadIdx.x; k < N * N; k += blockDim.x) sV[4 * N * NP + k] = L.tab[tab_n(TabIndex::DL, N) + k];
    sI = sV;
    sDg = sV + 2 * N * NP;
    sDL = sV + 4 * N * NP;
    __syncthreads();
    return sV + vol_vals(N);
}

// Warp per element; every element's slot records are fetched once (a lane per
// slot) instead of through a dependent load chain per slot.
template <int N, typename T, typename TX, bool OR = true>
__device__ __forceinline__ void trace_body(const LevelView<T>& L, const ElemDesc* __restrict__ bdesc, int count,
                                           const TX* __restrict__ x, T* __restrict__ mt, int blk, int nblk) {
    using Ly = Layout<N>;
    constexpr int N3 = Ly::N3;
    const T *sFT, *sI, *sDg, *sDL;
    T* wbase = load_tables<N, T>(L, sFT, sI, sDg, sDL);
    const int nwarps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* U = wbase + warp * Ly::TWARP;
    T* F = U + Ly::NR;
    const int stride = nblk * nwarps;
    int ei = blk * nwarps + warp;
    ElemDesc nd{};
    if (ei < count) nd = bdesc[ei];
    for (; ei < count; ei += stride) {
        const ElemDesc d = nd;
        const bool more = ei + stride < count;
        if (more) nd = bdesc[ei + stride];   // the next element's offsets, in flight during this one
        const long long dofo = d.dofo;
        WarpSlots<T> ws;
        ws.load(L, d.s0, d.s1, lane);
        load_element<N, T, TX>(x + dofo, U, lane);
        __syncwarp();
        ws.prefetch(L, lane, false);   // the mortars' c, into L2 ahead of the later slots
        if (more) prefetch_l2(x + nd.dofo, N3, lane, 32);   // the next element's input
        for (int si = ws.s0; si < ws.s1; ++si) {
            const SlotInfo<T> s = unpack_rec(ws.get(si));
            const T* co = L.mg + 7 * s.goff + (s.side == 0 ? 1 : 4) * s.q * s.q;
            DG_Q_SWITCH(s.q, (trace_slot<N, Q, T, OR>(L, s, U, sDL, sFT, F, co, mt, lane)))
        }
    }
}

// OR: the level has mortars whose side B face frame is turned (block meshes);
// without it the mortar-point permutation is compiled out.
template <int N, typename T, typename TX, bool OR>
__global__ void trace_kernel(LevelView<T> L, const ElemDesc* __restrict__ bdesc, int count, const TX* __restrict__ x,
                             T* __restrict__ mt) {
    trace_body<N, T, TX, OR>(L, bdesc, count, x, mt, blockIdx.x, gridDim.x);
}

// BDM: element diagonal blocks only -- 0 never, 1 always, 2 as L.bdiag says.
template <int N, typename T, typename TX, bool OR = true, int BDM = 2>
__device__ __forceinline__ void element_body(const LevelView<T>& L, const ElemDesc* __restrict__ bdesc, int count,
                                             const TX* __restrict__ x, T* __restrict__ y, int blk, int nblk) {
    using Ly = Layout<N>;
    constexpr int N3 = Ly::N3, NR = Ly::NR;
    const T *sFT, *sI, *sDg, *sDL;
    T* wbase = load_tables<N, T>(L, sFT, sI, sDg, sDL);
    const int nwarps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* Y = wbase + warp * Ly::EWARP;
    T* A = Y + NR;
    T* G1 = A + NR;
    T* U = G1 + NR;
    T* G3 = U;
    T* G2 = Y;  // the y-gradient lives in Y until the backward passes
    T* F = A;   // face phase scratch
    const bool mass = L.c0 != nullptr;
    VolFrags fr{};
    if constexpr (use_mma<N, T>()) fr = vol_frags<N>(sI, sDg, lane);
    const int stride = nblk * nwarps;
    int ei = blk * nwarps + warp;
    ElemDesc nd{};
    if (ei < count) nd = bdesc[ei];
    for (; ei < count; ei += stride) {
        const ElemDesc d = nd;
        const bool more = ei + stride < count;
        if (more) nd = bdesc[ei + stride];   // the next element's offsets, in flight during this one
        const int e = d.e;
        const long long dofo = d.dofo, vo = d.vo;
        WarpSlots<T> ws;
        ws.load(L, d.s0, d.s1, lane);
        load_element<N, T, TX>(x + dofo, U, lane);
        prefetch_l2(L.G + 6 * vo, 6 * N3, lane, 32);   // metric terms, needed after 6 passes
        __syncwarp();
        vpass<N, 0, 0, false>(U, A, sI, fr, lane);
        __syncwarp();
        vpass<N, 1, 0, false>(A, G1, sI, fr, lane);
        __syncwarp();
        vpass<N, 2, 0, false>(G1, A, sI, fr, lane);  // A = u at GL points
        ws.prefetch(L, lane, true);   // mortar data, needed after the volume terms
        if (more) {   // the next element's input and slot records
            prefetch_l2(x + nd.dofo, N3, lane, 32);
            prefetch_l2(L.spack + nd.s0, nd.s1 - nd.s0, lane, 32);
        }
        __syncwarp();
        vpass<N, 0, 2, false>(A, G1, sDg, fr, lane);
        vpass<N, 1, 2, false>(A, G2, sDg, fr, lane);
        vpass<N, 2, 2, false>(A, G3, sDg, fr, lane);
        __syncwarp();
        {   // f = G g at the volume GL points (six stored values per point, read once: evict-first)
            const T* Ge = L.G + 6 * vo;
            constexpr int GU = 4;   // points per lane whose metric terms are in flight together
#pragma unroll 1
            for (int k0 = lane; k0 < N3; k0 += 32 * GU) {
                T m[GU][6];
#pragma unroll
                for (int u = 0; u < GU; ++u) {
                    const int k = k0 + 32 * u < N3 ? k0 + 32 * u : k0;
#pragma unroll
                    for (int c = 0; c < 6; ++c) m[u][c] = __ldcs(Ge + c * N3 + k);
                }
#pragma unroll
                for (int u = 0; u < GU; ++u) {
                    const int k = k0 + 32 * u;
                    if (k >= N3) continue;
                    const int s = sidx<N>(k);
                    const T g0 = G1[s], g1 = G2[s], g2 = G3[s];
                    G1[s] = m[u][0] * g0 + m[u][1] * g1 + m[u][2] * g2;
                    G2[s] = m[u][1] * g0 + m[u][3] * g1 + m[u][4] * g2;
                    G3[s] = m[u][2] * g0 + m[u][4] * g1 + m[u][5] * g2;
                    if (mass) A[s] = L.c0[vo + k] * A[s];   // the zeroth-order term, summed into A below
                }
            }
        }
        __syncwarp();
        if (mass) vpass<N, 0, 3, true>(G1, A, sDg, fr, lane);
        else vpass<N, 0, 3, false>(G1, A, sDg, fr, lane);
        __syncwarp();
        vpass<N, 1, 3, true>(G2, A, sDg, fr, lane);
        __syncwarp();
        vpass<N, 2, 3, true>(G3, A, sDg, fr, lane);
        __syncwarp();
        vpass<N, 0, 1, false>(A, G1, sI, fr, lane);
        __syncwarp();
        vpass<N, 1, 1, false>(G1, U, sI, fr, lane);
        __syncwarp();
        vpass<N, 2, 1, false>(U, Y, sI, fr, lane);
        __syncwarp();
        if (L.Ob != nullptr && L.Ob_off[e] + (long long)N3 * N3 > L.ob_total) {
            if (lane == 0) atomicExch(L.chk, 1);
        } else if (L.Ob != nullptr) {
            // (coarse levels only; kept rolled so that its loads do not inflate
            // the register count of the whole kernel)
            const T* Oe = L.Ob + L.Ob_off[e];
#pragma unroll 1
            for (int k = lane; k < N3; k += 32) {
                T s = 0;
#pragma unroll 1
                for (int j = 0; j < N3; ++j)   // u from the input vector when its buffer was reused
                    s += Oe[(long long)j * N3 + k] * (Ly::UALIAS ? ld<T>(x + dofo + j) : U[sidx<N>(j)]);
                Y[sidx<N>(k)] += s;
            }
            __syncwarp();
        }
        for (int si = ws.s0; si < ws.s1; ++si) {
            const SlotRec<T> r = ws.get(si);
            const SlotInfo<T> s = unpack_rec(r);
            const bool interior = (r.info >> 12) & 1;
            const T* mg = L.mg + 7 * s.goff;
            const T* co = mg + (s.side == 0 ? 1 : 4) * s.q * s.q;
            DG_Q_SWITCH(s.q, (lift_slot<N, Q, T, OR, BDM>(L, s, interior, r.sig, Y, sDL, sFT, F, mg, co, L.mt + 4 * s.goff,
                                                 lane)))
        }
        for (int k = lane; k < N3; k += 32) __stcs(y + dofo + k, Y[sidx<N>(k)]);   // written once: evict first
        __syncwarp();
    }
}

// BD: the block-diagonal apply of the Schwarz smoother (compiled apart so that
// the ordinary apply carries no test for it).
// Register budget of the 32-bit element kernels, about what the passes and
// face loops need: left alone, the compiler spends up to twice as many on
// instruction-level parallelism and halves the resident warps.
template <int N, typename T>
constexpr int elem_maxreg() {
    return sizeof(T) == 8 || N > 8 ? 255 : (N <= 3 ? 64 : (N == 4 ? 72 : (N <= 6 ? 96 : 128)));
}

template <int N, typename T, typename TX, bool OR, bool BD = false>
__global__ void __maxnreg__((elem_maxreg<N, T>())) element_kernel(LevelView<T> L, const ElemDesc* __restrict__ bdesc, int count, const TX* __restrict__ x,
                               T* __restrict__ y) {
    element_body<N, T, TX, OR, BD ? 1 : 0>(L, bdesc, count, x, y, blockIdx.x, gridDim.x);
}

// All degree buckets of a level in one launch (used on small levels, where
// latency rather than bandwidth bounds the apply): CTA ranges map to buckets;
// each CTA runs the code compiled for its bucket's degree.
struct FusedBuckets {
    int nb;
    int n[kNumN];
    const int* elems[kNumN];
    const ElemDesc* desc[kNumN];
    int count[kNumN];
    int cta_start[kNumN + 1];
};

#define DG_BODY_SWITCH(NV, CALL)                           \
    switch (NV) {                                          \
        case 2: { constexpr int NN = 2; CALL; break; }     \
        case 3: { constexpr int NN = 3; CALL; break; }     \
        case 4: { constexpr int NN = 4; CALL; break; }     \
        case 5: { constexpr int NN = 5; CALL; break; }     \
        case 6: { constexpr int NN = 6; CALL; break; }     \
        case 7: { constexpr int NN = 7; CALL; break; }     \
        case 8: { constexpr int NN = 8; CALL; break; }     \
        default: { constexpr int NN = 9; CALL; break; }    \
    }

__device__ __forceinline__ int fused_bucket(const FusedBuckets& fb) {
    int b = 0;
    while (b + 1 < fb.nb && (int)blockIdx.x >= fb.cta_start[b + 1]) ++b;
    return b;
}

template <typename T, typename TX>
__global__ void trace_fused(LevelView<T> L, FusedBuckets fb, const TX* __restrict__ x, T* __restrict__ mt) {
    const int b = fused_bucket(fb);
    const int blk = blockIdx.x - fb.cta_start[b], nblk = fb.cta_start[b + 1] - fb.cta_start[b];
    DG_BODY_SWITCH(fb.n[b], (trace_body<NN, T, TX>(L, fb.desc[b], fb.count[b], x, mt, blk, nblk)))
}

template <typename T, typename TX>
__global__ void element_fused(LevelView<T> L, FusedBuckets fb, const TX* __restrict__ x, T* __restrict__ y) {
    const int b = fused_bucket(fb);
    const int blk = blockIdx.x - fb.cta_start[b], nblk = fb.cta_start[b + 1] - fb.cta_start[b];
    DG_BODY_SWITCH(fb.n[b], (element_body<NN, T, TX>(L, fb.desc[b], fb.count[b], x, y, blk, nblk)))
}


// ---- small levels: one CTA per element ------------------------------------------
// The warps of the CTA split the element's mortar slots (each lifts into its own
// accumulator, summed in warp order at the end) and share the volume passes, so
// the latency of one element -- which bounds the apply on levels with few
// elements -- drops several-fold.
constexpr int kCtaWarps = 8;

template <int N>
struct CtaLayout {
    static constexpr int N3 = N * N * N, NR = r4(Strides<N>::SIZE);
    static constexpr int TWARP = Layout<N>::TFACE;                        // per-warp trace scratch
    static constexpr int TSHARED = NR;                                    // U
    static constexpr int EWARP = NR + 4 * kQ * kQ + 3 * kQ * N;           // per-warp lift accumulator + scratch
    static constexpr int ESHARED = 6 * NR;                                // U, Y, A, B, G1, G3
};

template <int N, typename T, typename TX>
__device__ __forceinline__ void trace_body_cta(const LevelView<T>& L, int e, const TX* __restrict__ x,
                                               T* __restrict__ mt) {
    using Ly = CtaLayout<N>;
    const T *sFT, *sI, *sDg, *sDL;
    T* base = load_tables<N, T>(L, sFT, sI, sDg, sDL);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    T* U = base;
    T* F = U + Ly::TSHARED + warp * Ly::TWARP;
    const long long dofo = L.dof_off[e];
    for (int k = threadIdx.x; k < Ly::N3; k += blockDim.x) U[sidx<N>(k)] = ld<T>(x + dofo + k);
    __syncthreads();
    const int s0 = L.slot_off[e], s1 = L.slot_off[e + 1];
    for (int si = s0 + warp; si < s1; si += nw) {
        const SlotInfo<T> s = slot_info(L, si);
        const T* co = L.mg + 7 * s.goff + (s.side == 0 ? 1 : 4) * s.q * s.q;
        DG_Q_SWITCH(s.q, (trace_slot<N, Q, T>(L, s, U, sDL, sFT, F, co, mt, lane)))
    }
}

template <int N, typename T, typename TX>
__device__ __forceinline__ void element_body_cta(const LevelView<T>& L, int e, const TX* __restrict__ x,
                                                 T* __restrict__ y) {
    using Ly = CtaLayout<N>;
    constexpr int N3 = Ly::N3, NR = Ly::NR;
    const T *sFT, *sI, *sDg, *sDL;
    T* base = load_tables<N, T>(L, sFT, sI, sDg, sDL);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    T* U = base;
    T* Y = U + NR;
    T* A = Y + NR;
    T* B = A + NR;
    T* G1 = B + NR;
    T* G3 = G1 + NR;
    T* G2 = Y;
    T* Yw = base + Ly::ESHARED + warp * Ly::EWARP;
    T* F = Yw + NR;
    const long long dofo = L.dof_off[e], vo = L.vqp_off[e];
    const bool mass = L.c0 != nullptr;
    for (int k = tid; k < N3; k += nt) U[sidx<N>(k)] = ld<T>(x + dofo + k);
    __syncthreads();
    wpass<N, 0, false, false>(U, A, sI, tid, nt);
    __syncthreads();
    wpass<N, 1, false, false>(A, B, sI, tid, nt);
    __syncthreads();
    wpass<N, 2, false, false>(B, A, sI, tid, nt);
    __syncthreads();
    wpass<N, 0, false, false>(A, G1, sDg, tid, nt);
    wpass<N, 1, false, false>(A, G2, sDg, tid, nt);
    wpass<N, 2, false, false>(A, G3, sDg, tid, nt);
    __syncthreads();
    {
        const T* Ge = L.G + 6 * vo;
        for (int k = tid; k < N3; k += nt) {
            const int s = sidx<N>(k);
            const T g0 = G1[s], g1 = G2[s], g2 = G3[s];
            const T m00 = __ldcs(Ge + k), m01 = __ldcs(Ge + N3 + k), m02 = __ldcs(Ge + 2 * N3 + k);
            const T m11 = __ldcs(Ge + 3 * N3 + k), m12 = __ldcs(Ge + 4 * N3 + k), m22 = __ldcs(Ge + 5 * N3 + k);
            G1[s] = m00 * g0 + m01 * g1 + m02 * g2;
            G2[s] = m01 * g0 + m11 * g1 + m12 * g2;
            G3[s] = m02 * g0 + m12 * g1 + m22 * g2;
            if (mass) B[s] = L.c0[vo + k] * A[s];
        }
    }
    __syncthreads();
    if (mass) wpass<N, 0, true, true>(G1, B, sDg, tid, nt);
    else wpass<N, 0, true, false>(G1, B, sDg, tid, nt);
    __syncthreads();
    wpass<N, 1, true, true>(G2, B, sDg, tid, nt);
    __syncthreads();
    wpass<N, 2, true, true>(G3, B, sDg, tid, nt);
    __syncthreads();
    wpass<N, 0, true, false>(B, A, sI, tid, nt);
    __syncthreads();
    wpass<N, 1, true, false>(A, B, sI, tid, nt);
    __syncthreads();
    wpass<N, 2, true, false>(B, Y, sI, tid, nt);
    __syncthreads();
    if (L.Ob != nullptr && L.Ob_off[e] + (long long)N3 * N3 > L.ob_total) {
        if (tid == 0) atomicExch(L.chk, 1);
    } else if (L.Ob != nullptr) {
        const T* Oe = L.Ob + L.Ob_off[e];
        for (int k = tid; k < N3; k += nt) {
            T sacc = 0;
            for (int j = 0; j < N3; ++j) sacc += Oe[(long long)j * N3 + k] * U[sidx<N>(j)];
            Y[sidx<N>(k)] += sacc;
        }
    }
    for (int k = lane; k < NR; k += 32) Yw[k] = 0;
    __syncwarp();
    const int s0 = L.slot_off[e], s1 = L.slot_off[e + 1];
    for (int si = s0 + warp; si < s1; si += nw) {
        const int mi = L.slot_mortar[si];
        const SlotInfo<T> s = slot_info(L, si);
        const bool interior = L.mortars[mi].eB >= 0;
        const T sig = L.sigma[mi];
        const T* mg = L.mg + 7 * s.goff;
        const T* co = mg + (s.side == 0 ? 1 : 4) * s.q * s.q;
        DG_Q_SWITCH(s.q, (lift_slot<N, Q, T>(L, s, interior, sig, Yw, sDL, sFT, F, mg, co, L.mt + 4 * s.goff, lane)))
    }
    __syncthreads();
    for (int k = tid; k < N3; k += nt) {
        const int s = sidx<N>(k);
        T acc = Y[s];
        for (int w = 0; w < nw; ++w) acc += base[Ly::ESHARED + w * Ly::EWARP + s];
        __stcs(y + dofo + k, acc);
    }
}

template <typename T, typename TX>
__global__ void trace_cta(LevelView<T> L, FusedBuckets fb, const TX* __restrict__ x, T* __restrict__ mt) {
    const int b = fused_bucket(fb);
    const int e = fb.elems[b][blockIdx.x - fb.cta_start[b]];
    DG_BODY_SWITCH(fb.n[b], (trace_body_cta<NN, T, TX>(L, e, x, mt)))
}

template <typename T, typename TX>
__global__ void element_cta(LevelView<T> L, FusedBuckets fb, const TX* __restrict__ x, T* __restrict__ y) {
    const int b = fused_bucket(fb);
    const int e = fb.elems[b][blockIdx.x - fb.cta_start[b]];
    DG_BODY_SWITCH(fb.n[b], (element_body_cta<NN, T, TX>(L, e, x, y)))
}

// Launch shape of a per-bucket kernel, found once per template instance.  The
// statics below are initialised by the first caller (C++ guarantees that
// this is thread-safe), as the serving loop applies from several threads.
struct LaunchShape {
    cudaError_t err;
    int W, per_sm;
    size_t smem;
};

// Warps per CTA and resident CTAs per SM: the configuration with the most
// resident warps (up to 32 per CTA) that shared memory and registers allow.
template <typename K>
cudaError_t pick_warps(K kernel, size_t table_bytes, size_t warp_bytes, int& W, size_t& smem, int& per_sm) {
    const size_t cap = 220 * 1024;
    cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
    if (err != cudaSuccess) return err;
    int best_w = 1, best_blocks = 1, best_res = 0;
    for (int w = 1; w <= 32; ++w) {
        const size_t bytes = table_bytes + (size_t)w * warp_bytes;
        if (bytes > cap) break;
        int blocks = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, w * 32, bytes);
        if (err != cudaSuccess) return err;
        if (blocks >= 1 && blocks * w >= best_res) {   // ties -> larger CTAs (fewer table copies)
            best_res = blocks * w;
            best_w = w;
            best_blocks = blocks;
        }
    }
    W = best_w;
    per_sm = best_blocks;
    smem = table_bytes + (size_t)W * warp_bytes;
    return cudaSuccess;
}

inline int grid_cap() {
    static const int g = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 152;
    }();
    return g;
}

template <int N, typename T, typename TX, bool OR>
cudaError_t launch_trace(const LevelView<T>& L, const BucketInfo& b, const TX* x, cudaStream_t st) {
    using Ly = Layout<N>;
    static const LaunchShape shp = [&] {   // the mortar tables have the same size in every context
        LaunchShape r{};
        const size_t table_bytes = table_vals<N>(sizeof(T) == 4 ? L.ft.total : 0) * sizeof(T);
        r.err = pick_warps(trace_kernel<N, T, TX, OR>, table_bytes, Ly::TWARP * sizeof(T), r.W, r.smem, r.per_sm);
        return r;
    }();
    if (shp.err != cudaSuccess) return shp.err;
    const int W = shp.W, per_sm = shp.per_sm;
    const size_t smem = shp.smem;
    int grid = (b.count + W - 1) / W;
    if (grid > grid_cap() * per_sm) grid = grid_cap() * per_sm;
    trace_kernel<N, T, TX, OR><<<grid, W * 32, smem, st>>>(L, b.desc, b.count, x, L.mt);
    return cudaGetLastError();
}

template <int N, typename T, typename TX, bool OR, bool BD = false>
cudaError_t launch_element(const LevelView<T>& L, const BucketInfo& b, const TX* x, T* y, cudaStream_t st) {
    using Ly = Layout<N>;
    static const LaunchShape shp = [&] {   // the mortar tables have the same size in every context
        LaunchShape r{};
        const size_t table_bytes = table_vals<N>(sizeof(T) == 4 ? L.ft.total : 0) * sizeof(T);
        r.err = pick_warps(element_kernel<N, T, TX, OR, BD>, table_bytes, Ly::EWARP * sizeof(T), r.W, r.smem, r.per_sm);
        return r;
    }();
    if (shp.err != cudaSuccess) return shp.err;
    const int W = shp.W, per_sm = shp.per_sm;
    const size_t smem = shp.smem;
    int grid = (b.count + W - 1) / W;
    if (grid > grid_cap() * per_sm) grid = grid_cap() * per_sm;
    element_kernel<N, T, TX, OR, BD><<<grid, W * 32, smem, st>>>(L, b.desc, b.count, x, y);
    return cudaGetLastError();
}

#define DG_N_SWITCH(NV, CALL)                              \
    switch (NV) {                                          \
        case 2: { constexpr int NN = 2; CALL; break; }     \
        case 3: { constexpr int NN = 3; CALL; break; }     \
        case 4: { constexpr int NN = 4; CALL; break; }     \
        case 5: { constexpr int NN = 5; CALL; break; }     \
        case 6: { constexpr int NN = 6; CALL; break; }     \
        case 7: { constexpr int NN = 7; CALL; break; }     \
        case 8: { constexpr int NN = 8; CALL; break; }     \
        default: { constexpr int NN = 9; CALL; break; }    \
    }

}  // namespace apply_detail

namespace apply_detail {

constexpr int kFusedWarps = 8;
constexpr int kFusedMaxElems = 8192;   // levels this small use one launch per kernel (warp per element)
constexpr int kCtaMaxElems = 152;      // ... and at most one element per SM: one CTA per element

template <typename T, typename TX>
cudaError_t launch_fused_warp(const LevelView<T>& L, const BucketInfo* buckets, const TX* x, T* y, cudaStream_t st,
                              int* launches) {
    const size_t cap = 220 * 1024;
    const int ftot = sizeof(T) == 4 ? L.ft.total : 0;
    size_t max_tw = 0, max_ew = 0, max_tv = 0;
    for (int n = kMinN; n <= kMaxN; ++n) {
        if (buckets[n].count == 0) continue;
        size_t tw = 0, ew = 0;
        DG_N_SWITCH(n, (tw = Layout<NN>::TWARP, ew = Layout<NN>::EWARP))
        max_tw = std::max(max_tw, tw);
        max_ew = std::max(max_ew, ew);
        max_tv = std::max(max_tv, (size_t)(r4(ftot) + vol_vals(n)));
    }
    if (max_ew == 0) return cudaSuccess;
    int W = kFusedWarps;   // same CTA shape for every bucket; shrink until the largest degree fits
    while (W > 1 && (max_tv + (size_t)W * std::max(max_tw, max_ew)) * sizeof(T) > cap) --W;
    const size_t smem_t = (max_tv + (size_t)W * max_tw) * sizeof(T);
    const size_t smem_e = (max_tv + (size_t)W * max_ew) * sizeof(T);
    FusedBuckets fb{};
    int ctas = 0;
    for (int n = kMinN; n <= kMaxN; ++n) {
        const BucketInfo& b = buckets[n];
        if (b.count == 0) continue;
        fb.n[fb.nb] = n;
        fb.elems[fb.nb] = b.elems;
        fb.desc[fb.nb] = b.desc;
        fb.count[fb.nb] = b.count;
        fb.cta_start[fb.nb] = ctas;
        ctas += (b.count + W - 1) / W;
        ++fb.nb;
    }
    fb.cta_start[fb.nb] = ctas;
    static const cudaError_t attr = [&] {
        cudaError_t e1 = cudaFuncSetAttribute(trace_fused<T, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
        cudaError_t e2 = cudaFuncSetAttribute(element_fused<T, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
        return e1 != cudaSuccess ? e1 : e2;
    }();
    if (attr != cudaSuccess) return attr;
    trace_fused<T, TX><<<ctas, W * 32, smem_t, st>>>(L, fb, x, L.mt);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    element_fused<T, TX><<<ctas, W * 32, smem_e, st>>>(L, fb, x, y);
    err = cudaGetLastError();
    if (launches) *launches += 2;
    return err;
}

template <typename T, typename TX>
cudaError_t launch_fused_cta(const LevelView<T>& L, const BucketInfo* buckets, const TX* x, T* y, cudaStream_t st,
                             int* launches) {
    const size_t cap = 220 * 1024;
    const int ftot = sizeof(T) == 4 ? L.ft.total : 0;
    size_t smem_t = 0, smem_e = 0;
    FusedBuckets fb{};
    int ctas = 0;
    for (int n = kMinN; n <= kMaxN; ++n) {
        const BucketInfo& b = buckets[n];
        if (b.count == 0) continue;
        size_t tsh = 0, tw = 0, esh = 0, ew = 0;
        DG_N_SWITCH(n, (tsh = CtaLayout<NN>::TSHARED, tw = CtaLayout<NN>::TWARP, esh = CtaLayout<NN>::ESHARED,
                        ew = CtaLayout<NN>::EWARP))
        const size_t tv = (size_t)(r4(ftot) + vol_vals(n));
        smem_t = std::max(smem_t, (tv + tsh + kCtaWarps * tw) * sizeof(T));
        smem_e = std::max(smem_e, (tv + esh + kCtaWarps * ew) * sizeof(T));
        fb.n[fb.nb] = n;
        fb.elems[fb.nb] = b.elems;
        fb.desc[fb.nb] = b.desc;
        fb.count[fb.nb] = b.count;
        fb.cta_start[fb.nb] = ctas;
        ctas += b.count;
        ++fb.nb;
    }
    fb.cta_start[fb.nb] = ctas;
    if (ctas == 0) return cudaSuccess;
    if (smem_e > cap || smem_t > cap) return cudaErrorInvalidConfiguration;
    static const cudaError_t attr = [&] {
        cudaError_t e1 = cudaFuncSetAttribute(trace_cta<T, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
        cudaError_t e2 = cudaFuncSetAttribute(element_cta<T, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
        return e1 != cudaSuccess ? e1 : e2;
    }();
    if (attr != cudaSuccess) return attr;
    trace_cta<T, TX><<<ctas, kCtaWarps * 32, smem_t, st>>>(L, fb, x, L.mt);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    element_cta<T, TX><<<ctas, kCtaWarps * 32, smem_e, st>>>(L, fb, x, y);
    err = cudaGetLastError();
    if (launches) *launches += 2;
    return err;
}

}  // namespace apply_detail

template <typename T, typename TX>
cudaError_t launch_path(int path, const LevelView<T>& L, const BucketInfo* buckets, const TX* x, T* y,
                        cudaStream_t st, int* launches, const ApplyStreams* as) {
    if (path == 0) return apply_detail::launch_fused_cta<T, TX>(L, buckets, x, y, st, launches);
    if (path == 1) return apply_detail::launch_fused_warp<T, TX>(L, buckets, x, y, st, launches);
    // Per-bucket launches, largest bucket (elements x n^3) first; plan 3 deals
    // them round robin over the caller's stream and the side streams.
    if (path == 2) as = nullptr;
    int order[kNumN], nb = 0;
    for (int n = kMinN; n <= kMaxN; ++n)
        if (buckets[n].count > 0) order[nb++] = n;
    auto work = [&](int n) { return (long long)buckets[n].count * n * n * n; };
    std::sort(order, order + nb, [&](int a, int b) { return work(a) > work(b); });
    const int ns = as ? std::min(as->n, nb - 1) : 0;
    for (int phase = 0; phase < 2; ++phase) {   // every element's mortar traces, then volume + face lifts
        if (ns > 0) {
            cudaError_t err = cudaEventRecord(as->fork[phase], st);
            for (int i = 0; i < ns && err == cudaSuccess; ++i) err = cudaStreamWaitEvent(as->side[i], as->fork[phase], 0);
            if (err != cudaSuccess) return err;
        }
        for (int j = 0; j < nb; ++j) {
            const int n = order[j], k = j % (ns + 1);
            const cudaStream_t sj = k == 0 ? st : as->side[k - 1];
            const BucketInfo& b = buckets[n];
            cudaError_t err = cudaSuccess;
            if (phase == 0 && L.oriented) {
                DG_N_SWITCH(n, (err = apply_detail::launch_trace<NN, T, TX, true>(L, b, x, sj)))
            } else if (phase == 0) {
                DG_N_SWITCH(n, (err = apply_detail::launch_trace<NN, T, TX, false>(L, b, x, sj)))
            } else if (L.bdiag) {   // block-diagonal apply: the general (turned-interface) form
                DG_N_SWITCH(n, (err = apply_detail::launch_element<NN, T, TX, true, true>(L, b, x, y, sj)))
            } else if (L.oriented) {
                DG_N_SWITCH(n, (err = apply_detail::launch_element<NN, T, TX, true>(L, b, x, y, sj)))
            } else {
                DG_N_SWITCH(n, (err = apply_detail::launch_element<NN, T, TX, false>(L, b, x, y, sj)))
            }
            if (err != cudaSuccess) return err;
            if (launches) ++*launches;
        }
        for (int i = 0; i < ns; ++i) {
            cudaError_t err = cudaEventRecord(as->join[phase][i], as->side[i]);
            if (err == cudaSuccess) err = cudaStreamWaitEvent(st, as->join[phase][i], 0);
            if (err != cudaSuccess) return err;
        }
    }
    return cudaSuccess;
}

// Launch plan of a level: 0 one CTA per element, 1 one warp per element in a
// single launch per kernel, 2 per-degree-bucket launches with occupancy-sized
// CTAs, 3 the same spread over side streams.  With a plan slot and outside
// stream capture the first apply times the candidates (each writes the same
// outputs, in the same order of summation) and keeps the fastest; otherwise a
// size rule picks.  DGELL_APPLY_PLAN=0..3 fixes the plan of every tuned level.
inline int forced_plan() {
    static const int v = [] {
        const char* e = std::getenv("DGELL_APPLY_PLAN");
        return (e && e[0] >= '0' && e[0] <= '3' && e[1] == 0) ? e[0] - '0' : -1;
    }();
    return v;
}

template <typename T, typename TX>
cudaError_t launch_apply_x(const LevelView<T>& L, const BucketInfo* buckets, const TX* x, T* y, cudaStream_t st,
                           int* launches, int* plan, const ApplyStreams* as = nullptr) {
    int path = L.n_elems <= apply_detail::kCtaMaxElems ? 0 : (L.n_elems <= apply_detail::kFusedMaxElems ? 1 : 2);
    if (plan && *plan >= 0) return launch_path<T, TX>(*plan, L, buckets, x, y, st, launches, as);
    if (plan && forced_plan() >= 0) {
        *plan = forced_plan();
        return launch_path<T, TX>(*plan, L, buckets, x, y, st, launches, as);
    }
    unsigned long long key = 1469598103934665603ull;   // FNV-1a over the level shape and precision
    auto mix = [&](unsigned long long v) { key = (key ^ v) * 1099511628211ull; };
    mix(sizeof(T));
    mix(sizeof(TX));
    mix((unsigned long long)L.n_elems);
    for (int n = kMinN; n <= kMaxN; ++n) mix((unsigned long long)buckets[n].count);
    if (plan) {
        const int cached = plan_cache_get(key);
        if (cached >= 0) {
            *plan = cached;
            return launch_path<T, TX>(cached, L, buckets, x, y, st, launches, as);
        }
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (plan && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        int best_path = path;
        const int ncand = (as && as->n > 0) ? 4 : 3;
        for (int cand = 0; cand < ncand; ++cand) {
            cudaError_t err = launch_path<T, TX>(cand, L, buckets, x, y, st, nullptr, as);   // warm-up / validity
            if (err != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            cudaEventRecord(e0, st);
            for (int r = 0; r < 3; ++r) launch_path<T, TX>(cand, L, buckets, x, y, st, nullptr, as);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_path = cand;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        *plan = best_path;
        plan_cache_put(key, best_path);
        path = best_path;
    }
    return launch_path<T, TX>(path, L, buckets, x, y, st, launches, as);
}

template <typename T>
cudaError_t launch_apply(const LevelView<T>& L, const BucketInfo* buckets, const T* x, T* y, cudaStream_t st,
                         int* launches, int* plan, const ApplyStreams* as) {
    return launch_apply_x<T, T>(L, buckets, x, y, st, launches, plan, as);
}

}  // namespace dg
