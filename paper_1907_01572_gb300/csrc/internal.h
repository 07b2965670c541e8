// Internal data model of libdgell (host + device).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dgell.h"

namespace dg {

constexpr int kMaxN = 9;          // n = p + 1 <= 9 (p <= 8)
constexpr int kMinN = 2;
constexpr int kNumN = kMaxN - kMinN + 1;
constexpr int kTabStride = 81;    // every 1-D table is stored padded to 9 x 9

// ---- 1-D operator tables (Sec. II.F.4: interpolation / derivative operators
// of size (p'+1) x (p+1), kept for every degree pair) -------------------------
// Layout (values of type T, each matrix row-major, padded to 9x9):
//   I  [n]          : I[i][a]  = l_a(x^GL_i)               (LGL -> GL, n x n)
//   Dg [n]          : Dg[i][j] = l^GL_j'(x^GL_i)           (GL collocation derivative)
//   DL [n]          : DL[i][a] = l_a'(x^LGL_i)             (LGL collocation derivative)
//   IDg[n]          : IDg[i][a]= l_a'(x^GL_i)              (derivative at GL points)
//   Im [n][q][pos]  : Im[i][a] = l_a(m_pos(s_i))           (face LGL -> mortar GL, q x n)
//   Dm [n][q][pos]  : Dm[i][a] = l_a'(m_pos(s_i))
//   CI [nH][nh][b]  : CI[i][a] = l^H_a((x^h_i + 2b - 1)/2) (parent -> child half b, nh x nH)
// m_pos: 0 -> s, 1 -> (s - 1)/2, 2 -> (s + 1)/2.
struct TabIndex {
    static constexpr int I = 0;
    static constexpr int Dg = I + kNumN;
    static constexpr int DL = Dg + kNumN;
    static constexpr int IDg = DL + kNumN;
    static constexpr int Im = IDg + kNumN;
    static constexpr int Dm = Im + kNumN * kNumN * 3;
    static constexpr int CI = Dm + kNumN * kNumN * 3;
    static constexpr int LGLx = CI + kNumN * kNumN * 2;   // 1 row: LGL nodes of n
    static constexpr int GLx = LGLx + kNumN;              // GL nodes of q
    static constexpr int GLw = GLx + kNumN;               // GL weights of q
    static constexpr int Count = GLw + kNumN;
};

__host__ __device__ inline int tab_n(int base, int n) { return (base + (n - kMinN)) * kTabStride; }
__host__ __device__ inline int tab_m(int base, int n, int q, int pos) {
    return (base + ((n - kMinN) * kNumN + (q - kMinN)) * 3 + pos) * kTabStride;
}
__host__ __device__ inline int tab_ci(int nH, int nh, int b) {
    return (TabIndex::CI + ((nH - kMinN) * kNumN + (nh - kMinN)) * 2 + b) * kTabStride;
}

void build_tables(std::vector<double>& tab);   // size TabIndex::Count * kTabStride

// Compact mortar tables for the apply kernel's shared memory: for every side
// degree n and mortar q >= n (q = max of both sides' n), sub-face pos 0..2,
// the q x n matrices Im then Dm, packed without padding.
struct FaceTabs {
    int off[kNumN][kNumN][3];   // [n-2][q-2][pos] -> offset of the q*n (Im, Dm) pairs (even); -1 if q < n
    int total;
};
void build_face_tables(const std::vector<double>& tab, std::vector<double>& ftab, FaceTabs& ft);

// ---- mesh ----------------------------------------------------------------------
struct Mortar {            // device record (32 bytes)
    int eA, eB;            // eA: geometry ('-') side = finer / lower index; eB = -1 on the boundary
    unsigned char fA, fB;  // faces (2*dim + side)
    unsigned char posA0, posA1, posB0, posB1;  // sub-face codes along the two tangential axes
    unsigned char q;       // GL points per direction = p_m + 1
    unsigned char orient;  // side B's face frame relative to side A's (blocks.h orient_coords); 0 inside a block
    long long goff;        // offset (in points) into the mortar geometry arrays
    long long bnd_off;     // offset into boundary point arrays (-1 if interior)
};

// Neighbour of each block face: block nb's face nf with relative orientation
// orient (blocks.h), or nb = -1 on the domain boundary.
struct BlockFace {
    int nb = -1, nf = 0, orient = 0;
};
struct BlockTopo {
    int n_blocks = 1;
    std::vector<BlockFace> face;     // 6 per block
};

struct LevelHost {
    std::vector<int> leaves;         // 4 per element
    std::vector<int> block;          // block of each element
    std::vector<int> p;
    std::vector<long long> dof_off;  // n_elems + 1
    std::vector<long long> vqp_off;  // volume GL point offsets, n_elems + 1
    std::vector<Mortar> mortars;
    std::vector<int> slot_off;       // n_elems + 1
    std::vector<int> slot_mortar;
    std::vector<unsigned char> slot_face, slot_side;
    long long n_mortar_pts = 0;
    long long n_bnd_pts = 0;
    // transfer to the next finer level (filled on levels < L):
    //   per coarse element: child count (1 or 8) and children (fine ids) + bits
    std::vector<int> child_off;      // n_elems + 1
    std::vector<int> child_id;
    std::vector<unsigned char> child_bits;   // bit0: x half, bit1: y, bit2: z; 0xFF: carried over
    // per fine element of the next finer level: parent id and bits
    std::vector<int> fine_parent;
    std::vector<unsigned char> fine_bits;
    int n_elems() const { return (int)p.size(); }
    long long n_dofs() const { return dof_off.back(); }
    std::vector<int> buckets[kMaxN + 1];  // element ids by n
};

// Block connectivity from the block maps: faces whose four corners coincide
// are glued, with the orientation under which the corners match.
bool build_block_topology(const dg_block* blocks, int n_blocks, BlockTopo& topo, std::string& err);
// The level-lev cell of block b2 (index c2) across face f of the level-lev cell idx of
// block b, when f lies on b's boundary; false on the domain boundary.
bool block_face_neighbour(const BlockTopo& T, int b, int f, int lev, const int idx[3], int& b2, int c2[3]);
// Builds the finest level's connectivity; returns false with a message on a malformed mesh.
bool build_level_connectivity(LevelHost& L, const BlockTopo& topo, std::string& err);
// Coarsens `fine` into `coarse` (Sec. II.E.3); returns false when no family merges.
bool coarsen_level(const LevelHost& fine, LevelHost& coarse, const BlockTopo& topo, std::string& err);

// ---- device level ------------------------------------------------------------------
// One element of a degree bucket with the offsets its kernels start from
// (one broadcast load instead of a chain of dependent ones).
struct ElemDesc {
    long long dofo, vo;    // DOF and volume GL point offsets
    int e, s0, s1, pad;    // element id, its mortar slots [s0, s1)
};

// One mortar slot (an element's side of a mortar), packed for one load:
// info = face | side << 3 | pos0 << 4 | pos1 << 6 | q << 8 | interior << 12 |
// orientation of side B's face frame << 13; the mortar's point offset and
// penalty sigma in the kernel's precision.
template <typename T>
struct SlotPack {
    int info;
    T sig;
    long long goff;
};

template <typename T>
struct LevelView {         // passed by value to kernels
    int n_elems;
    const int* p;
    const long long* dof_off;
    const long long* vqp_off;
    const T* G;            // 6 * n_vqp: G[6*vqp_off[e] + c*q^3 + pt]
    const T* c0;           // zeroth-order coefficient (w det J f) per volume point or nullptr
    const T* Ob;           // dense Galerkin blocks (coarse levels) or nullptr
    const long long* Ob_off;
    const int* slot_off;
    const int* slot_mortar;
    const unsigned char* slot_face;
    const unsigned char* slot_side;
    const Mortar* mortars;
    const SlotPack<T>* spack;   // per slot, in slot order
    const T* mg;           // 7 * n_mortar_pts: [wS, cA0, cA1, cA2, cB0, cB1, cB2] blocks per mortar
    const T* sigma;        // per mortar
    const T* tab;
    const T* ftab;         // compact mortar tables (FaceTabs layout)
    FaceTabs ft;
    long long ob_total;    // entries of Ob (bounds check)
    int oriented;          // some mortar of the level has a turned side B (Mortar::orient != 0)
    int bdiag;             // apply only the element diagonal blocks (the neighbour's trace taken as 0)
    int* chk;              // self-check flag
    T* mt;                 // mortar trace buffer: 4 * n_mortar_pts ([u_A, dn_A, u_B, dn_B] per mortar)
};

// Self-check support: kernels that index with offsets read from tables check
// them against the buffer sizes, skip the access and record a code here.
int* device_check_flag();          // device pointer to one int (0 = ok)
// Process-wide cache of tuned apply launch plans keyed by level shape and
// precision, so every context with the same level shape uses the same plan
// (and therefore the same summation order) within a process.
int plan_cache_get(unsigned long long key);   // -1 if absent
void plan_cache_put(unsigned long long key, int plan);
bool debug_sync();                 // DGELL_DEBUG_SYNC=1: synchronise and name every checked launch

struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace dg
