// A-posteriori error estimator kernel (Sec. II.D, eqs. Eta2_Ingredients,
// Eta2_Integrals, Eta2_Local), FP64.
#pragma once
#include "internal.h"

namespace dg {

struct EstimateArgs {
    int n_elems;
    const int* p;
    const long long* dof_off;
    const long long* vqp_off;
    const int* slot_off;
    const int* slot_mortar;
    const Mortar* mortars;
    const double* mg;       // per mortar point: w S, c_A (3), c_B (3)
    const double* sigma;    // per mortar
    const double* mt;       // trace buffer of an FP64 apply of u: u_A, dn_A, u_B, dn_B per mortar point
    const double* tab;
    const double* X;        // single box: node coordinates, 3 n^3 per element at 3 dof_off[e]
    double C;               // penalty constant of eq. (penaltyparameter)
    // multi-block meshes: the exact block maps (J and second derivatives at the GL points)
    int n_blocks;           // 0: single box (isoparametric geometry from X)
    const dg_block* blocks; // device
    const int* block;       // device, block of each element
    const int* leaves;      // device, 4 per element
    // fiducial grid (blocks of identical structure): volume weights and h_e from fblocks, mortar
    // weights w S and sigma (hence h_m) from mgW / sigW; without one, fblocks = blocks, mgW = mg,
    // sigW = sigma
    const dg_block* fblocks;
    const double* mgW;
    const double* sigW;
};

// eta2[e] = h_e^2 p_e^2 ||f u - g - Lap u||^2_e + the mortar terms of the element.
// g, f: volume GL point values or NULL (0); gD: Dirichlet mortar point values or NULL (0).
cudaError_t launch_estimate(const EstimateArgs& a, const double* u, const double* g, const double* f,
                            const double* gD, double* eta2, cudaStream_t st);

}  // namespace dg
