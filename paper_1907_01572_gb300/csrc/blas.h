// Vector kernels, deterministic reductions and the device-resident scalar
// recurrences of CG (Alg. 5), Chebyshev (Alg. 4) and flexible CG (Alg. 2).
#pragma once
#include "internal.h"

namespace dg {

constexpr int kRedBlocks = 304;   // 2 x 152 SMs; fixed so that reductions are reproducible
constexpr int kRedThreads = 256;
constexpr int kMaxCheb = 64;

struct SmState {        // smoother scalars (device)
    double rr, rr_new, pAp, a, beta, lam, a_prev, b_prev;
    int stop, have_prev, skip, pad;
    double ca[kMaxCheb], cb[kMaxCheb];
};

struct FcgState {       // flexible-CG scalars (device)
    double dots[4];     // v.r, v.w, v.q, r.r
    double rho, g, c;
    int k, breakdown;
};

struct Red {            // reduction scratch: partials[kRedBlocks * 4] + results[4]
    double* partials;
    double* out;
    unsigned* counter;  // blocks done, for the single-launch (last block) reductions; 0 between launches
};

// out[0..k) = dot products of (a_i, b_i) pairs, T in {float, double}, accumulated in double.
template <typename T>
cudaError_t dots(const T* const* a, const T* const* b, int k, long long n, Red red, cudaStream_t st);

cudaError_t cast_d2f(const double* s, float* d, long long n, cudaStream_t st);
cudaError_t fill_slot_sigma(SlotPack<double>* s64, SlotPack<float>* s32, const int* slot_mortar, const double* sigma,
                            int n, cudaStream_t st);
cudaError_t cast_f2d(const float* s, double* d, long long n, cudaStream_t st);

// r = b - y; p = r (if p); partial r.r into red (then finalize -> out[0])
template <typename T>
cudaError_t residual_init(const T* b, const T* y, T* r, T* p, long long n, Red red, cudaStream_t st);

// CGEIGS pieces
cudaError_t sm_init(SmState* s, const double* rr, cudaStream_t st);
// Fused CG step, two launches plus the p update: (1) p.Ap and alpha, (2) x, r
// update with r.r, beta and the Gershgorin bound; the last block to finish
// sums the per-block partials in index order (same result as dots + finalize).
template <typename T>
cudaError_t cg_alpha_fused(SmState* s, const T* p, const T* Ap, long long n, Red red, cudaStream_t st);
template <typename T>
cudaError_t cg_update_fused(SmState* s, T* x, T* r, const T* p, const T* Ap, long long n, Red red, cudaStream_t st);
cudaError_t sm_alpha(SmState* s, const double* pAp, cudaStream_t st);
template <typename T>
cudaError_t cg_xr_update(const SmState* s, T* x, T* r, const T* p, const T* Ap, long long n, Red red, cudaStream_t st);
cudaError_t sm_beta(SmState* s, const double* rr_new, cudaStream_t st);
template <typename T>
cudaError_t cg_p_update(const SmState* s, T* p, const T* r, long long n, cudaStream_t st);
// Chebyshev
cudaError_t sm_cheb_coeffs(SmState* s, int n_cheb, double Lambda, double scale, double fixed, cudaStream_t st);
template <typename T>
cudaError_t cheb_step(const SmState* s, int k, const T* b, const T* Ax, T* p, T* x, long long n, cudaStream_t st);

// FCG pieces (double vectors)
cudaError_t fcg_scalars(FcgState* f, const double* dots3, int k, cudaStream_t st);
cudaError_t fcg_dq(const FcgState* f, double* d, double* q, const double* v, const double* w, long long n,
                   cudaStream_t st);
cudaError_t fcg_update(const FcgState* f, double* u, double* r, const double* d, const double* q, long long n,
                       Red red, cudaStream_t st);

// Element-local CG on a block-diagonal system (the Schwarz smoother's local
// solves, all elements at once), warp per element, per-element scalars in
// es[3 * e + {0, 1, 2}] = (r.r, alpha, initial r.r):
//   init:   dx = 0, p = r, es = (r.r, 0, r.r)
//   alpha:  alpha_e = r.r / p.Dp, or 0 once r.r <= tol2 * (initial r.r) or p.Dp <= 0
//   update: dx += alpha p, r -= alpha Dp, p = r + (r.r_new / r.r) p
template <typename T>
cudaError_t elem_cg_init(const T* r, T* p, T* dx, const long long* dof_off, int ne, double* es, cudaStream_t st);
template <typename T>
cudaError_t elem_cg_alpha(const T* p, const T* Dp, const long long* dof_off, int ne, double* es, double tol2,
                          cudaStream_t st);
template <typename T>
cudaError_t elem_cg_update(T* dx, T* r, T* p, const T* Dp, const long long* dof_off, int ne, double* es,
                           cudaStream_t st);

// Schwarz smoother with overlapping subdomains (Alg. 6): per subdomain s
// (entries [sub_off[s], sub_off[s+1]), m of them), u = W_s A_s^-1 R_s r with
// the stored inverse (column-major m x m at inv_off[s]); then, per global DOF
// i, x_i += the sum of u over the entries ovl_cof[cof_off[i] .. cof_off[i+1])
// in that order (deterministic).
template <typename T>
cudaError_t ovl_local(const long long* sub_off, const long long* sub_dof, const T* w, const long long* inv_off,
                      const T* inv, const T* r, T* u, int n_sub, int max_m, cudaStream_t st);
template <typename T>
cudaError_t ovl_gather(const long long* cof_off, const long long* cof, const T* u, T* x, long long n, cudaStream_t st);

template <typename T>
cudaError_t axpby(T a, const T* x, T b, T* y, long long n, cudaStream_t st);   // y = a x + b y
template <typename T>
cudaError_t sub3(const T* a, const T* b, T* c, long long n, cudaStream_t st);  // c = a - b

// y = M x, M dense n x n (double, column-major), T vectors
template <typename T>
cudaError_t dense_matvec(const double* M, const T* x, T* y, int n, cudaStream_t st);
// D = L + blockdiag(O_e) (column-major n x n; O_e column-major (n_e^3)^2 at Ob_off[e]),
// D32 = (float) D
cudaError_t dense_compose(const double* Lmat, const double* Ob, const long long* Ob_off, const long long* dof_off,
                          const int* p, int n_elems, int n, double* D, float* D32, cudaStream_t st);
// y = M x with M in the vectors' precision (column-major)
template <typename T>
cudaError_t dense_matvec_t(const T* M, const T* x, T* y, int n, cudaStream_t st);

}  // namespace dg
