// Zeroth-order / Galerkin and puncture kernels.
#pragma once
#include "internal.h"

namespace dg {

struct PunctureDev {
    int n;
    double m[16];
    double c[16][3];
    double P[16][3];
    double S[16][3];
};

enum NlKind { kNlNone = 0, kNlPuncture = 1, kNlPower = 2 };

struct NlArgs {
    int n_elems;
    int kind;                  // kNlPuncture: s = beta (1 + alpha (1 + u))^-7; kNlPower: s = coef u^power
    int power;
    const int* p;
    const long long* dof_off;
    const long long* vqp_off;
    const double* wdetJ;
    const double* alpha;       // puncture: alpha; power: coef
    const double* beta;
    const double* tab;
    long long n_vqp;   // bounds check
    int* chk;
};

struct GalerkinArgs {
    int n_coarse;
    const int* pH;             // coarse degrees
    const long long* Ob_off;   // per coarse element: offset of its (n^3 x n^3) block
    const int* desc_off;       // n_coarse + 1
    const int* desc;           // finest descendants
    const double* map;         // per descendant: (scale, offset) for x, y, z (6 doubles)
    const int* pf;             // finest degrees
    const long long* vqp_off_f;
    const double* tab;
    long long ob_total;    // bounds checks
    long long n_vqp_f;
    int n_desc;
    int* chk;
};

cudaError_t launch_puncture(const double* vxyz, long long n, const PunctureDev& P, double* alpha, double* beta,
                            cudaStream_t st);
// S = I^T (w det J beta (1 + alpha (1 + u))^-7); jac (optional) = w det J 7 alpha beta (...)^-8
cudaError_t launch_nl(const NlArgs& a, const double* u, double* S, double* jac64, float* jac32, cudaStream_t st);
// R = Lu - S - F (F may be NULL)
cudaError_t launch_sub(const double* Lu, const double* S, const double* F, double* R, long long n, cudaStream_t st);
cudaError_t launch_galerkin(const GalerkinArgs& g, const double* c0, double* O64, float* O32, cudaStream_t st);

}  // namespace dg
