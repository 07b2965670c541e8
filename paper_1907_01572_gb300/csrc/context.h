// Context: device-resident hierarchy, geometry, tables and solver workspaces.
#pragma once
#include <memory>

#include "apply.h"
#include "blas.h"
#include "internal.h"
#include "transfer.h"

namespace dg {

struct Arena {
    std::vector<void*> ptrs;
    size_t bytes = 0;
    bool failed = false;
    template <typename T>
    T* alloc(size_t n) {
        if (n == 0) n = 1;
        void* p = nullptr;
        if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            failed = true;
            return nullptr;
        }
        ptrs.push_back(p);
        bytes += n * sizeof(T);
        return static_cast<T*>(p);
    }
    template <typename T>
    T* upload(const std::vector<T>& v, cudaStream_t st) {
        T* d = alloc<T>(v.size());
        if (d && !v.empty()) cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
        return d;
    }
    void free_all() {
        for (void* p : ptrs) cudaFree(p);
        ptrs.clear();
    }
};

template <typename T>
struct Work {
    T *f = nullptr, *v = nullptr, *r = nullptr, *p = nullptr, *Ap = nullptr, *t = nullptr;
    SmState* sm = nullptr;
    bool ready = false;
};

struct LevelDev {
    LevelHost h;
    int *leaves = nullptr, *p = nullptr, *block = nullptr;
    int oriented = 0;                 // some mortar has a turned side B (block interfaces)
    double* schwarz_es = nullptr;     // element-local CG scalars of the Schwarz smoother (3 per element)
    // Schwarz smoother with overlapping subdomains (one per element): entries
    // [sub_off[s], sub_off[s+1]) hold the subdomain's global DOFs and weights;
    // the inverse of its local operator (column-major, m x m) starts at
    // inv_off[s]; per global DOF, ovl_cof_off / ovl_cof list the entries that
    // hold it (for a fixed-order sum of the local corrections)
    long long *sub_off = nullptr, *sub_dof = nullptr, *inv_off = nullptr;
    long long *ovl_cof_off = nullptr, *ovl_cof = nullptr;
    double *ovl_w64 = nullptr, *ovl_inv64 = nullptr, *ovl_u64 = nullptr;
    float *ovl_w32 = nullptr, *ovl_inv32 = nullptr, *ovl_u32 = nullptr;
    int ovl_max_m = 0;
    long long ovl_version = -1;       // op_version the local inverses belong to
    long long *dof_off = nullptr, *vqp_off = nullptr;
    Mortar* mortars = nullptr;
    int *slot_off = nullptr, *slot_mortar = nullptr;
    unsigned char *slot_face = nullptr, *slot_side = nullptr;
    SlotPack<double>* spack64 = nullptr;
    SlotPack<float>* spack32 = nullptr;
    BucketInfo buckets[kMaxN + 1] = {};
    double *G64 = nullptr, *wdetJ = nullptr, *vxyz = nullptr, *mg64 = nullptr, *sigma64 = nullptr, *bxyz = nullptr;
    float *G32 = nullptr, *mg32 = nullptr, *sigma32 = nullptr;
    double* mt64 = nullptr;           // mortar trace buffers of the apply
    float* mt32 = nullptr;
    double* c0_64 = nullptr;
    float* c0_32 = nullptr;
    double* Ob64 = nullptr;
    float* Ob32 = nullptr;
    long long* Ob_off = nullptr;
    bool z_active = false;            // zeroth-order term (c0 on the finest level, Ob on coarse levels) in use
    double* dense64 = nullptr;        // assembled operator of a small level (column-major), solver use only
    float* dense32 = nullptr;
    double* denseL = nullptr;         // its SIPG (Laplacian) part, built once; + Galerkin blocks -> dense64
    long long dense_version = -1;     // op_version the dense operator was built for
    int plan[3] = {-1, -1, -1};       // tuned apply launch plan per precision (FP64, FP32, BF16 operands)
    // Galerkin structure of a coarse level: finest descendants and their reference maps
    int *g_desc_off = nullptr, *g_desc = nullptr;
    double* g_map = nullptr;
    size_t ob_count = 0;
    // transfer to the next finer level (this level is the coarse side)
    int *child_off = nullptr, *child_id = nullptr, *fine_parent = nullptr;
    unsigned char *child_bits = nullptr, *fine_bits = nullptr;
    Work<double> w64;
    Work<float> w32;
};

}  // namespace dg

struct dg_ctx {
    cudaStream_t st = nullptr;
    double C = 10.0;
    dg_mesh_desc desc{};
    std::vector<dg_block> blocks;   // host copy of the mesh blocks (empty: single box)
    dg::BlockTopo topo;
    dg_block* blocks_dev = nullptr;
    std::vector<dg::LevelDev> lv;   // 0 = coarsest
    dg::Arena arena;
    double* tab64 = nullptr;
    float* tab32 = nullptr;
    double* ftab64 = nullptr;
    float* ftab32 = nullptr;
    dg::FaceTabs ft{};
    dg::Red red{};
    double* red_host = nullptr;     // pinned, 4 doubles
    dg::FcgState* fcg = nullptr;
    double* fcg_vec[6] = {};        // r, v, w, d, q, t (double, finest)
    float* fcg32[2] = {};           // f32 copies of r and v for the mixed-precision V-cycle
    double* coarse_inv = nullptr;   // dense inverse of the level-0 operator
    int coarse_n = 0;
    bool coarse_ready = false;
    long long coarse_version = -1;  // op_version the coarse inverse belongs to
    bool has_zeroth = false;
    // puncture data on the finest level volume points
    double* p_alpha = nullptr;
    double* p_beta = nullptr;
    int nl_kind = 0;                // nonlinear problem for dg_newton_*: 0 none, 1 puncture, 2 power-law source
    int nl_power = 0;
    double* nl_coef = nullptr;      // power-law source coefficient at the finest volume GL points
    double* nl_F = nullptr;         // power-law source: forcing vector (Dirichlet lift), n_dofs
    bool nl_has_F = false;
    double* nw[4] = {};             // Newton work vectors (double, finest): R, du, Lu, S
    bool galerkin_ready = false;
    // CUDA graph of the V-cycle used inside dg_solve (captured once, replayed)
    cudaGraphExec_t vgraph = nullptr;
    int vgraph_prec = -1;
    long long vgraph_epoch = -1;
    long long vgraph_opver = -1;    // operator version the graph's small-level matrices belong to
    long long vgraph_launches = 0;  // kernels in the graph
    dg_mg_opts vgraph_opts{};
    long long epoch = 0;            // bumped whenever kernel arguments of the solver change
    long long op_version = 0;       // bumped whenever operator coefficients change (zeroth-order term)
    long long launches = 0;
    dg::ApplyStreams as{};          // side streams of the per-bucket apply
    // dg_apply_host: copy streams (in, out), per staging slot the events
    // [copied in, applied, copied out], and the device staging slots
    cudaStream_t hst[2] = {};
    cudaEvent_t hev[2][3] = {};
    cudaEvent_t hstart = nullptr;
    void* hstage = nullptr;
    size_t hstage_bytes = 0;
};

namespace dg {
// Kernel arguments of level l in precision T: the level's and the context's
// device pointers (the one definition every apply path uses).
template <typename T>
LevelView<T> level_view(dg_ctx* c, int l);
}  // namespace dg
