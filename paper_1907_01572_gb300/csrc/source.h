// Right-hand side and nonlinear source kernels.
#pragma once
#include "internal.h"

namespace dg {

struct RhsArgs {
    int n_elems;
    const int* p;
    const long long* dof_off;
    const long long* vqp_off;
    const double* wdetJ;
    const int* slot_off;
    const int* slot_mortar;
    const unsigned char* slot_face;
    const Mortar* mortars;
    const double* mg;
    const double* sigma;
    const double* tab;
};

// F = I^T (w det J g) on every element + Dirichlet lifts of g_D (eq. equationFh2).
cudaError_t launch_rhs(const RhsArgs& a, const double* g_qp, const double* gD_qp, double* F, cudaStream_t st);

// out[pt] = w det J * coef[pt]  (volume points; FP64 and FP32 copies)
cudaError_t launch_scale_coef(const double* wdetJ, const double* coef, double* c64, float* c32, long long n,
                              cudaStream_t st);

}  // namespace dg
