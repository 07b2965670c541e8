// Vector kernels and device-resident scalar recurrences (see blas.h).
// Reductions: every block sums a fixed grid-stride slice, reduces it in a fixed
// tree order and writes one partial; a single block then sums the partials in
// index order, so repeated runs give bit-identical results.
#include <algorithm>

#include "blas.h"

namespace dg {
namespace {

__device__ inline double block_sum(double v, double* sh) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s) sh[t] += sh[t + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void finalize_kernel(const double* partials, int k, double* out) {
    __shared__ double sh[kRedThreads];
    for (int j = 0; j < k; ++j) {
        double v = 0.0;
        for (int i = threadIdx.x; i < kRedBlocks; i += blockDim.x) v += partials[i * 4 + j];
        const double s = block_sum(v, sh);
        if (threadIdx.x == 0) out[j] = s;
    }
}

template <typename T>
struct DotArgs {
    const T* a[4];
    const T* b[4];
};

template <typename T>
__global__ void dots_kernel(DotArgs<T> args, int k, long long n, double* partials) {
    __shared__ double sh[kRedThreads];
    for (int j = 0; j < k; ++j) {
        double v = 0.0;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
            v += (double)args.a[j][i] * (double)args.b[j][i];
        const double s = block_sum(v, sh);
        if (threadIdx.x == 0) partials[blockIdx.x * 4 + j] = s;
    }
}

__global__ void d2f_kernel(const double* s, float* d, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        d[i] = (float)s[i];
}
__global__ void f2d_kernel(const float* s, double* d, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        d[i] = (double)s[i];
}

template <typename T>
__global__ void residual_init_kernel(const T* b, const T* y, T* r, T* p, long long n, double* partials) {
    __shared__ double sh[kRedThreads];
    double v = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T ri = b[i] - y[i];
        r[i] = ri;
        if (p) p[i] = ri;
        v += (double)ri * (double)ri;
    }
    const double s = block_sum(v, sh);
    if (threadIdx.x == 0) partials[blockIdx.x * 4] = s;
}

__global__ void sm_init_kernel(SmState* s, const double* rr) {
    s->rr = rr[0];
    s->lam = 0.0;
    s->stop = 0;
    s->have_prev = 0;
    s->a = 0.0;
    s->beta = 0.0;
    s->skip = 0;
}

__device__ void alpha_logic(SmState* s, double v) {
    s->pAp = v;
    if (s->stop || !(v > 0.0) || !(s->rr > 0.0) || !isfinite(v)) {
        s->stop = 1;
        s->a = 0.0;
        return;
    }
    s->a = s->rr / v;
}

__global__ void sm_alpha_kernel(SmState* s, const double* pAp) {
    const double v = pAp[0];
    s->pAp = v;
    if (s->stop || !(v > 0.0) || !(s->rr > 0.0) || !isfinite(v)) {
        s->stop = 1;
        s->a = 0.0;
        return;
    }
    s->a = s->rr / v;
}

template <typename T>
__global__ void cg_xr_kernel(const SmState* s, T* x, T* r, const T* p, const T* Ap, long long n, double* partials) {
    __shared__ double sh[kRedThreads];
    const bool stop = s->stop != 0;
    const T a = (T)s->a;
    double v = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (!stop) {
            x[i] += a * p[i];
            const T ri = r[i] - a * Ap[i];
            r[i] = ri;
            v += (double)ri * (double)ri;
        }
    }
    const double sum = block_sum(v, sh);
    if (threadIdx.x == 0) partials[blockIdx.x * 4] = sum;
}

// Gershgorin bound of row k of the Lanczos tridiagonal built from the CG
// coefficients (Alg. 5, eq. tridiag): T_kk = 1/a_k + b_{k-1}/a_{k-1},
// |T_k,k-1| = sqrt(b_{k-1})/a_{k-1}, |T_k,k+1| = sqrt(b_k)/a_k.
__device__ void beta_logic(SmState* s, double rn) {
    if (s->stop) return;
    const double beta = rn / s->rr;
    s->beta = beta;
    s->rr = rn;
    double diag = 1.0 / s->a, left = 0.0;
    if (s->have_prev) {
        diag += s->b_prev / s->a_prev;
        left = sqrt(s->b_prev) / s->a_prev;
    }
    const double lk = diag + left + sqrt(beta) / s->a;
    if (isfinite(lk) && lk > s->lam) s->lam = lk;
    s->a_prev = s->a;
    s->b_prev = beta;
    s->have_prev = 1;
}

// Last block of a grid: sums partials[i * 4] over the grid's blocks in index order.
__device__ bool last_block_sum(double* partials, unsigned* counter, double* sh, double& total) {
    __shared__ bool last;
    __threadfence();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double v = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += ((volatile double*)partials)[i * 4];
    total = block_sum(v, sh);
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

template <typename T>
__global__ void cg_alpha_fused_kernel(SmState* s, const T* p, const T* Ap, long long n, double* partials,
                                      unsigned* counter) {
    __shared__ double sh[kRedThreads];
    double v = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v += (double)p[i] * (double)Ap[i];
    const double b = block_sum(v, sh);
    if (threadIdx.x == 0) partials[blockIdx.x * 4] = b;
    double total;
    if (last_block_sum(partials, counter, sh, total) && threadIdx.x == 0) alpha_logic(s, total);
}

template <typename T>
__global__ void cg_update_fused_kernel(SmState* s, T* x, T* r, const T* p, const T* Ap, long long n,
                                       double* partials, unsigned* counter) {
    __shared__ double sh[kRedThreads];
    const bool stop = s->stop != 0;
    const T a = (T)s->a;
    double v = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (!stop) {
            x[i] += a * p[i];
            const T ri = r[i] - a * Ap[i];
            r[i] = ri;
            v += (double)ri * (double)ri;
        }
    }
    const double b = block_sum(v, sh);
    if (threadIdx.x == 0) partials[blockIdx.x * 4] = b;
    double total;
    if (last_block_sum(partials, counter, sh, total) && threadIdx.x == 0) beta_logic(s, total);
}

__global__ void sm_beta_kernel(SmState* s, const double* rr_new) {
    if (s->stop) return;
    const double rn = rr_new[0];
    const double beta = rn / s->rr;
    s->beta = beta;
    s->rr = rn;
    double diag = 1.0 / s->a, left = 0.0;
    if (s->have_prev) {
        diag += s->b_prev / s->a_prev;
        left = sqrt(s->b_prev) / s->a_prev;
    }
    const double lk = diag + left + sqrt(beta) / s->a;
    if (isfinite(lk) && lk > s->lam) s->lam = lk;
    s->a_prev = s->a;
    s->b_prev = beta;
    s->have_prev = 1;
}

template <typename T>
__global__ void cg_p_kernel(const SmState* s, T* p, const T* r, long long n) {
    if (s->stop) return;
    const T b = (T)s->beta;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = r[i] + b * p[i];
}

// Chebyshev coefficients of Alg. 4 on [lmax/Lambda, lmax], lmax = scale x lam
// (or lmax = fixed, which also becomes the reported lam, when fixed > 0):
// alpha_1 = 1/d, alpha_2 = 2d/(2d^2 - c^2), alpha_k = 1/(d - alpha_{k-1} c^2/4),
// beta_k = alpha_k d - 1, with the update p <- alpha r + beta p.
__global__ void sm_cheb_kernel(SmState* s, int n_cheb, double Lambda, double scale, double fixed) {
    if (fixed > 0.0) s->lam = fixed;
    const double lmax = fixed > 0.0 ? fixed : s->lam * scale;
    if (!(lmax > 0.0) || !isfinite(lmax)) {
        s->skip = 1;
        return;
    }
    s->skip = 0;
    const double lmin = lmax / Lambda;
    const double c = 0.5 * (lmax - lmin), d = 0.5 * (lmax + lmin);
    double a = 0.0;
    for (int k = 1; k <= n_cheb; ++k) {
        if (k == 1) a = 1.0 / d;
        else if (k == 2) a = 2.0 * d / (2.0 * d * d - c * c);
        else a = 1.0 / (d - a * c * c / 4.0);
        s->ca[k - 1] = a;
        s->cb[k - 1] = a * d - 1.0;
    }
}

template <typename T>
__global__ void cheb_kernel(const SmState* s, int k, const T* b, const T* Ax, T* p, T* x, long long n) {
    if (s->skip) return;
    const T a = (T)s->ca[k], be = (T)s->cb[k];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T pi = a * (b[i] - Ax[i]) + be * p[i];
        p[i] = pi;
        x[i] += pi;
    }
}

// Flexible CG scalars (Alg. 2): alpha = v.r, beta = v.w, gamma = v.q_{k-1};
// rho_k = beta (k = 0) or beta - gamma^2 / rho_{k-1}; g = gamma / rho_{k-1};
// c = alpha / rho_k.
__global__ void fcg_scalar_kernel(FcgState* f, const double* dots3, int k) {
    const double al = dots3[0], be = dots3[1], ga = dots3[2];
    f->dots[0] = al;
    f->dots[1] = be;
    f->dots[2] = ga;
    double rho;
    if (k == 0) {
        rho = be;
        f->g = 0.0;
    } else {
        f->g = ga / f->rho;
        rho = be - ga * ga / f->rho;
    }
    if (!(rho > 0.0) || !isfinite(rho)) {
        f->breakdown = 1;
        f->c = 0.0;
        return;
    }
    f->rho = rho;
    f->c = al / rho;
    f->k = k;
}

__global__ void fcg_dq_kernel(const FcgState* f, double* d, double* q, const double* v, const double* w, long long n) {
    if (f->breakdown) return;
    const double g = f->g;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        d[i] = v[i] - g * d[i];
        q[i] = w[i] - g * q[i];
    }
}

__global__ void fcg_update_kernel(const FcgState* f, double* u, double* r, const double* d, const double* q,
                                  long long n, double* partials) {
    __shared__ double sh[kRedThreads];
    const bool brk = f->breakdown != 0;
    const double c = f->c;
    double v = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double ri = r[i];
        if (!brk) {
            u[i] += c * d[i];
            ri -= c * q[i];
            r[i] = ri;
        }
        v += ri * ri;
    }
    const double s = block_sum(v, sh);
    if (threadIdx.x == 0) partials[blockIdx.x * 4] = s;
}

template <typename T>
__global__ void axpby_kernel(T a, const T* x, T b, T* y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}

template <typename T>
__global__ void sub3_kernel(const T* a, const T* b, T* c, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        c[i] = a[i] - b[i];
}

template <typename T>
__global__ void dense_matvec_kernel(const double* M, const T* x, T* y, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += M[(long long)j * n + i] * (double)x[j];
        y[i] = (T)s;
    }
}

// Column-major y = M x: a block of 256 threads owns 32 rows and splits the
// columns into 8 slices (fixed order, so the result is reproducible).
template <typename T>
__global__ void dense_matvec_t_kernel(const T* M, const T* x, T* y, int n) {
    __shared__ T part[8][32];
    const int row = blockIdx.x * 32 + (threadIdx.x & 31);
    const int slice = threadIdx.x >> 5;
    T s = 0;
    if (row < n)
        for (int j = slice; j < n; j += 8) s += M[(long long)j * n + row] * x[j];
    part[slice][threadIdx.x & 31] = s;
    __syncthreads();
    if (slice == 0 && row < n) {
        T t = 0;
        for (int k = 0; k < 8; ++k) t += part[k][threadIdx.x];
        y[row] = t;
    }
}

__global__ void dense_copy_kernel(const double* L, double* D, long long nn) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x)
        D[i] = L[i];
}

__global__ void dense_blocks_kernel(const double* Ob, const long long* Ob_off, const long long* dof_off, const int* p,
                                    int n, double* D) {
    const int e = blockIdx.x;
    const int ne = p[e] + 1, n3 = ne * ne * ne;
    const double* Oe = Ob + Ob_off[e];
    const long long o = dof_off[e];
    for (int k = threadIdx.x; k < n3 * n3; k += blockDim.x) {
        const int j = k / n3, i = k % n3;
        D[(o + j) * n + (o + i)] += Oe[k];
    }
}

__global__ void dense_cast_kernel(const double* D, float* D32, long long nn) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x)
        D32[i] = (float)D[i];
}

inline int grid_for(long long n) {
    long long g = (n + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 4 * 152 * 4 ? 4 * 152 * 4 : g));
}

}  // namespace

template <typename T>
cudaError_t dots(const T* const* a, const T* const* b, int k, long long n, Red red, cudaStream_t st) {
    DotArgs<T> args{};
    for (int j = 0; j < k; ++j) {
        args.a[j] = a[j];
        args.b[j] = b[j];
    }
    dots_kernel<T><<<kRedBlocks, kRedThreads, 0, st>>>(args, k, n, red.partials);
    finalize_kernel<<<1, kRedThreads, 0, st>>>(red.partials, k, red.out);
    return cudaGetLastError();
}
template cudaError_t dots<double>(const double* const*, const double* const*, int, long long, Red, cudaStream_t);
template cudaError_t dots<float>(const float* const*, const float* const*, int, long long, Red, cudaStream_t);

// Penalty sigma of each slot's mortar into the packed slot records.
__global__ void slot_sigma_kernel(SlotPack<double>* s64, SlotPack<float>* s32, const int* slot_mortar,
                                  const double* sigma, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = sigma[slot_mortar[i]];
        s64[i].sig = v;
        s32[i].sig = (float)v;
    }
}

cudaError_t fill_slot_sigma(SlotPack<double>* s64, SlotPack<float>* s32, const int* slot_mortar, const double* sigma,
                            int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    slot_sigma_kernel<<<std::min(1024, (n + 255) / 256), 256, 0, st>>>(s64, s32, slot_mortar, sigma, n);
    return cudaGetLastError();
}

cudaError_t cast_d2f(const double* s, float* d, long long n, cudaStream_t st) {
    d2f_kernel<<<grid_for(n), 256, 0, st>>>(s, d, n);
    return cudaGetLastError();
}
cudaError_t cast_f2d(const float* s, double* d, long long n, cudaStream_t st) {
    f2d_kernel<<<grid_for(n), 256, 0, st>>>(s, d, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t residual_init(const T* b, const T* y, T* r, T* p, long long n, Red red, cudaStream_t st) {
    residual_init_kernel<T><<<kRedBlocks, kRedThreads, 0, st>>>(b, y, r, p, n, red.partials);
    finalize_kernel<<<1, kRedThreads, 0, st>>>(red.partials, 1, red.out);
    return cudaGetLastError();
}
template cudaError_t residual_init<double>(const double*, const double*, double*, double*, long long, Red, cudaStream_t);
template cudaError_t residual_init<float>(const float*, const float*, float*, float*, long long, Red, cudaStream_t);

cudaError_t sm_init(SmState* s, const double* rr, cudaStream_t st) {
    sm_init_kernel<<<1, 1, 0, st>>>(s, rr);
    return cudaGetLastError();
}
template <typename T>
cudaError_t cg_alpha_fused(SmState* s, const T* p, const T* Ap, long long n, Red red, cudaStream_t st) {
    cg_alpha_fused_kernel<T><<<kRedBlocks, kRedThreads, 0, st>>>(s, p, Ap, n, red.partials, red.counter);
    return cudaGetLastError();
}
template cudaError_t cg_alpha_fused<double>(SmState*, const double*, const double*, long long, Red, cudaStream_t);
template cudaError_t cg_alpha_fused<float>(SmState*, const float*, const float*, long long, Red, cudaStream_t);

template <typename T>
cudaError_t cg_update_fused(SmState* s, T* x, T* r, const T* p, const T* Ap, long long n, Red red, cudaStream_t st) {
    cg_update_fused_kernel<T><<<kRedBlocks, kRedThreads, 0, st>>>(s, x, r, p, Ap, n, red.partials, red.counter);
    return cudaGetLastError();
}
template cudaError_t cg_update_fused<double>(SmState*, double*, double*, const double*, const double*, long long, Red,
                                             cudaStream_t);
template cudaError_t cg_update_fused<float>(SmState*, float*, float*, const float*, const float*, long long, Red,
                                            cudaStream_t);

cudaError_t sm_alpha(SmState* s, const double* pAp, cudaStream_t st) {
    sm_alpha_kernel<<<1, 1, 0, st>>>(s, pAp);
    return cudaGetLastError();
}
template <typename T>
cudaError_t cg_xr_update(const SmState* s, T* x, T* r, const T* p, const T* Ap, long long n, Red red, cudaStream_t st) {
    cg_xr_kernel<T><<<kRedBlocks, kRedThreads, 0, st>>>(s, x, r, p, Ap, n, red.partials);
    finalize_kernel<<<1, kRedThreads, 0, st>>>(red.partials, 1, red.out);
    return cudaGetLastError();
}
template cudaError_t cg_xr_update<double>(const SmState*, double*, double*, const double*, const double*, long long, Red, cudaStream_t);
template cudaError_t cg_xr_update<float>(const SmState*, float*, float*, const float*, const float*, long long, Red, cudaStream_t);

cudaError_t sm_beta(SmState* s, const double* rr_new, cudaStream_t st) {
    sm_beta_kernel<<<1, 1, 0, st>>>(s, rr_new);
    return cudaGetLastError();
}
template <typename T>
cudaError_t cg_p_update(const SmState* s, T* p, const T* r, long long n, cudaStream_t st) {
    cg_p_kernel<T><<<grid_for(n), 256, 0, st>>>(s, p, r, n);
    return cudaGetLastError();
}
template cudaError_t cg_p_update<double>(const SmState*, double*, const double*, long long, cudaStream_t);
template cudaError_t cg_p_update<float>(const SmState*, float*, const float*, long long, cudaStream_t);

cudaError_t sm_cheb_coeffs(SmState* s, int n_cheb, double Lambda, double scale, double fixed, cudaStream_t st) {
    sm_cheb_kernel<<<1, 1, 0, st>>>(s, n_cheb, Lambda, scale, fixed);
    return cudaGetLastError();
}
template <typename T>
cudaError_t cheb_step(const SmState* s, int k, const T* b, const T* Ax, T* p, T* x, long long n, cudaStream_t st) {
    cheb_kernel<T><<<grid_for(n), 256, 0, st>>>(s, k, b, Ax, p, x, n);
    return cudaGetLastError();
}
template cudaError_t cheb_step<double>(const SmState*, int, const double*, const double*, double*, double*, long long, cudaStream_t);
template cudaError_t cheb_step<float>(const SmState*, int, const float*, const float*, float*, float*, long long, cudaStream_t);

cudaError_t fcg_scalars(FcgState* f, const double* dots3, int k, cudaStream_t st) {
    fcg_scalar_kernel<<<1, 1, 0, st>>>(f, dots3, k);
    return cudaGetLastError();
}
cudaError_t fcg_dq(const FcgState* f, double* d, double* q, const double* v, const double* w, long long n,
                   cudaStream_t st) {
    fcg_dq_kernel<<<grid_for(n), 256, 0, st>>>(f, d, q, v, w, n);
    return cudaGetLastError();
}
cudaError_t fcg_update(const FcgState* f, double* u, double* r, const double* d, const double* q, long long n,
                       Red red, cudaStream_t st) {
    fcg_update_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(f, u, r, d, q, n, red.partials);
    finalize_kernel<<<1, kRedThreads, 0, st>>>(red.partials, 1, red.out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t axpby(T a, const T* x, T b, T* y, long long n, cudaStream_t st) {
    axpby_kernel<T><<<grid_for(n), 256, 0, st>>>(a, x, b, y, n);
    return cudaGetLastError();
}
template cudaError_t axpby<double>(double, const double*, double, double*, long long, cudaStream_t);
template cudaError_t axpby<float>(float, const float*, float, float*, long long, cudaStream_t);

template <typename T>
cudaError_t sub3(const T* a, const T* b, T* c, long long n, cudaStream_t st) {
    sub3_kernel<T><<<grid_for(n), 256, 0, st>>>(a, b, c, n);
    return cudaGetLastError();
}
template cudaError_t sub3<double>(const double*, const double*, double*, long long, cudaStream_t);
template cudaError_t sub3<float>(const float*, const float*, float*, long long, cudaStream_t);

template <typename T>
cudaError_t dense_matvec(const double* M, const T* x, T* y, int n, cudaStream_t st) {
    dense_matvec_kernel<T><<<(n + 127) / 128, 128, 0, st>>>(M, x, y, n);
    return cudaGetLastError();
}
template cudaError_t dense_matvec<double>(const double*, const double*, double*, int, cudaStream_t);

cudaError_t dense_compose(const double* Lmat, const double* Ob, const long long* Ob_off, const long long* dof_off,
                          const int* p, int n_elems, int n, double* D, float* D32, cudaStream_t st) {
    const long long nn = (long long)n * n;
    dense_copy_kernel<<<grid_for(nn), 256, 0, st>>>(Lmat, D, nn);
    if (Ob) dense_blocks_kernel<<<n_elems, 256, 0, st>>>(Ob, Ob_off, dof_off, p, n, D);
    dense_cast_kernel<<<grid_for(nn), 256, 0, st>>>(D, D32, nn);
    return cudaGetLastError();
}

template <typename T>
cudaError_t dense_matvec_t(const T* M, const T* x, T* y, int n, cudaStream_t st) {
    dense_matvec_t_kernel<T><<<(n + 31) / 32, 256, 0, st>>>(M, x, y, n);
    return cudaGetLastError();
}
template cudaError_t dense_matvec_t<double>(const double*, const double*, double*, int, cudaStream_t);
template cudaError_t dense_matvec_t<float>(const float*, const float*, float*, int, cudaStream_t);
template cudaError_t dense_matvec<float>(const double*, const float*, float*, int, cudaStream_t);


// ---- element-local CG (Schwarz smoother) ------------------------------------------
namespace {

__device__ __forceinline__ double warp_sum(double v) {   // fixed butterfly order
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__global__ void elem_cg_init_kernel(const T* r, T* p, T* dx, const long long* dof_off, int ne, double* es) {
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int e = blockIdx.x * wpb + (threadIdx.x >> 5); e < ne; e += gridDim.x * wpb) {
        const long long a = dof_off[e], b = dof_off[e + 1];
        double s = 0.0;
        for (long long i = a + lane; i < b; i += 32) {
            const T v = r[i];
            p[i] = v;
            dx[i] = T(0);
            s += (double)v * (double)v;
        }
        s = warp_sum(s);
        if (lane == 0) {
            es[3 * e] = s;
            es[3 * e + 1] = 0.0;
            es[3 * e + 2] = s;
        }
    }
}

template <typename T>
__global__ void elem_cg_alpha_kernel(const T* p, const T* Dp, const long long* dof_off, int ne, double* es,
                                     double tol2) {
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int e = blockIdx.x * wpb + (threadIdx.x >> 5); e < ne; e += gridDim.x * wpb) {
        const long long a = dof_off[e], b = dof_off[e + 1];
        double s = 0.0;
        for (long long i = a + lane; i < b; i += 32) s += (double)p[i] * (double)Dp[i];
        s = warp_sum(s);
        if (lane == 0) {
            const double rr = es[3 * e];
            es[3 * e + 1] = (rr > tol2 * es[3 * e + 2] && s > 0.0 && isfinite(s)) ? rr / s : 0.0;
        }
    }
}

template <typename T>
__global__ void elem_cg_update_kernel(T* dx, T* r, T* p, const T* Dp, const long long* dof_off, int ne,
                                      double* es) {
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int e = blockIdx.x * wpb + (threadIdx.x >> 5); e < ne; e += gridDim.x * wpb) {
        const double alpha = es[3 * e + 1];
        if (alpha == 0.0) continue;   // warp-uniform: this element's local solve has stopped
        const long long a = dof_off[e], b = dof_off[e + 1];
        const T al = (T)alpha;
        double s = 0.0;
        for (long long i = a + lane; i < b; i += 32) {
            dx[i] += al * p[i];
            const T v = r[i] - al * Dp[i];
            r[i] = v;
            s += (double)v * (double)v;
        }
        s = warp_sum(s);
        const double rr = es[3 * e];
        const T beta = (T)(rr > 0.0 ? s / rr : 0.0);
        for (long long i = a + lane; i < b; i += 32) p[i] = r[i] + beta * p[i];
        __syncwarp();
        if (lane == 0) es[3 * e] = s;
    }
}

inline int elem_grid(int ne) {
    const int g = (ne + 7) / 8;
    return g < 1 ? 1 : (g > 4 * kRedBlocks ? 4 * kRedBlocks : g);
}

}  // namespace

template <typename T>
cudaError_t elem_cg_init(const T* r, T* p, T* dx, const long long* dof_off, int ne, double* es, cudaStream_t st) {
    elem_cg_init_kernel<T><<<elem_grid(ne), 256, 0, st>>>(r, p, dx, dof_off, ne, es);
    return cudaGetLastError();
}
template <typename T>
cudaError_t elem_cg_alpha(const T* p, const T* Dp, const long long* dof_off, int ne, double* es, double tol2,
                          cudaStream_t st) {
    elem_cg_alpha_kernel<T><<<elem_grid(ne), 256, 0, st>>>(p, Dp, dof_off, ne, es, tol2);
    return cudaGetLastError();
}
template <typename T>
cudaError_t elem_cg_update(T* dx, T* r, T* p, const T* Dp, const long long* dof_off, int ne, double* es,
                           cudaStream_t st) {
    elem_cg_update_kernel<T><<<elem_grid(ne), 256, 0, st>>>(dx, r, p, Dp, dof_off, ne, es);
    return cudaGetLastError();
}
template cudaError_t elem_cg_init<float>(const float*, float*, float*, const long long*, int, double*, cudaStream_t);
template cudaError_t elem_cg_init<double>(const double*, double*, double*, const long long*, int, double*,
                                          cudaStream_t);
template cudaError_t elem_cg_alpha<float>(const float*, const float*, const long long*, int, double*, double,
                                          cudaStream_t);
template cudaError_t elem_cg_alpha<double>(const double*, const double*, const long long*, int, double*, double,
                                           cudaStream_t);
template cudaError_t elem_cg_update<float>(float*, float*, float*, const float*, const long long*, int, double*,
                                           cudaStream_t);
template cudaError_t elem_cg_update<double>(double*, double*, double*, const double*, const long long*, int,
                                            double*, cudaStream_t);

// One CTA per subdomain: its residual entries gathered into shared memory, then
// each thread forms rows of W_s A_s^-1 (R_s r), the inverse read a column at a
// time across the threads.
template <typename T>
__global__ void ovl_local_kernel(const long long* __restrict__ sub_off, const long long* __restrict__ sub_dof,
                                 const T* __restrict__ w, const long long* __restrict__ inv_off,
                                 const T* __restrict__ inv, const T* __restrict__ r, T* __restrict__ u) {
    extern __shared__ unsigned char ovl_smem[];
    T* rs = reinterpret_cast<T*>(ovl_smem);
    const int s = blockIdx.x;
    const long long o = sub_off[s];
    const int m = (int)(sub_off[s + 1] - o);
    for (int j = threadIdx.x; j < m; j += blockDim.x) rs[j] = r[sub_dof[o + j]];
    __syncthreads();
    const T* A = inv + inv_off[s];
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        // four partial sums so that four loads of the (streamed, read-once-per-
        // cycle) inverse are in flight per thread
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        int k = 0;
        for (; k + 4 <= m; k += 4) {
            a0 += __ldcs(A + (long long)k * m + j) * rs[k];
            a1 += __ldcs(A + (long long)(k + 1) * m + j) * rs[k + 1];
            a2 += __ldcs(A + (long long)(k + 2) * m + j) * rs[k + 2];
            a3 += __ldcs(A + (long long)(k + 3) * m + j) * rs[k + 3];
        }
        for (; k < m; ++k) a0 += __ldcs(A + (long long)k * m + j) * rs[k];
        u[o + j] = w[o + j] * ((a0 + a1) + (a2 + a3));
    }
}

template <typename T>
__global__ void ovl_gather_kernel(const long long* __restrict__ cof_off, const long long* __restrict__ cof,
                                  const T* __restrict__ u, T* __restrict__ x, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    T s = 0;
    for (long long c = cof_off[i]; c < cof_off[i + 1]; ++c) s += u[cof[c]];
    x[i] += s;
}

template <typename T>
cudaError_t ovl_local(const long long* sub_off, const long long* sub_dof, const T* w, const long long* inv_off,
                      const T* inv, const T* r, T* u, int n_sub, int max_m, cudaStream_t st) {
    if (n_sub <= 0) return cudaSuccess;
    ovl_local_kernel<T><<<n_sub, 256, (size_t)max_m * sizeof(T), st>>>(sub_off, sub_dof, w, inv_off, inv, r, u);
    return cudaGetLastError();
}
template <typename T>
cudaError_t ovl_gather(const long long* cof_off, const long long* cof, const T* u, T* x, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    ovl_gather_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cof_off, cof, u, x, n);
    return cudaGetLastError();
}
template cudaError_t ovl_local<double>(const long long*, const long long*, const double*, const long long*,
                                       const double*, const double*, double*, int, int, cudaStream_t);
template cudaError_t ovl_local<float>(const long long*, const long long*, const float*, const long long*,
                                      const float*, const float*, float*, int, int, cudaStream_t);
template cudaError_t ovl_gather<double>(const long long*, const long long*, const double*, double*, long long,
                                        cudaStream_t);
template cudaError_t ovl_gather<float>(const long long*, const long long*, const float*, float*, long long,
                                       cudaStream_t);

}  // namespace dg
