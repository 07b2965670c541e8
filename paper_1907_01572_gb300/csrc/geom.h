// Geometry precompute kernels (FP64).
#pragma once
#include "internal.h"

namespace dg {

struct GeomArgs {
    int n_elems;
    const int* leaves;          // device, 4 per element
    const int* p;               // device
    const long long* dof_off;   // device
    const long long* vqp_off;   // device
    const double* tab;          // device FP64 tables
    double lo[3], hi[3];
    int map_kind;
    double warp_amp;
    int warp_k[3];
    int n_blocks;               // 0: the box [lo, hi] with map_kind; else blocks[block[e]]
    const dg_block* blocks;     // device, n_blocks
    const int* block;           // device, per element
};

// X: 3 * n_dofs doubles, element block e at 3*dof_off[e]: [x(n^3), y(n^3), z(n^3)]
cudaError_t launch_node_coords(const GeomArgs& g, double* X, cudaStream_t st);
// G: 6 * n_vqp, wdetJ: n_vqp, vxyz: 3 * n_vqp (SoA)
cudaError_t launch_volume_geom(const GeomArgs& g, const double* X, double* G, double* wdetJ, double* vxyz,
                               long long n_vqp, int* bad, cudaStream_t st);
// mg: 7 * n_mortar_pts, sigma: n_mortars, bxyz: 3 * n_bnd (SoA)
cudaError_t launch_mortar_geom(const GeomArgs& g, const double* X, const Mortar* mortars, int n_mortars, double C,
                               double* mg, double* sigma, double* bxyz, long long n_bnd, int* bad, cudaStream_t st);

}  // namespace dg
