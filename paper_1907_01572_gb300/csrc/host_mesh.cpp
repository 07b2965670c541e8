// Host-side mesh tables: mortar set of a multi-block octree mesh (Sec. II.A.1)
// and the multigrid level meshes (Sec. II.E.3).
//
// Mortars: every element face is covered either by the domain boundary, by one
// same-size neighbour, by one coarser neighbour (this face is a quarter of the
// neighbour's face) or by four finer neighbours -- inside a block or across a
// block interface.  One mortar is created per interface piece: on conforming
// faces from the lower-index element, on 2:1 faces from the finer element, on
// the boundary from the owner.  The creating element is side A (the side whose
// map supplies S^m and the normal).  The mortar degree is max(p_A, p_B)
// (mortar figure) with p_m + 1 GL points per direction.  Across a block
// interface side B's face frame is turned against A's; the mortar records the
// orientation, and side B's sub-face position codes refer to B's own frame.
//
// Level meshes: complete sibling families (within a block) are merged into
// their parent (surrogate mesh); a merged parent that would face an element two
// or more levels finer -- in its block or across a block interface -- is split
// again (2:1 rebalancing); the coarse degree is the minimum over the children.
// Coarse elements are numbered in the order in which their first child appears
// on the finer level.
#include <algorithm>
#include <cmath>
#include <unordered_map>
#include <unordered_set>

#include "blocks.h"
#include "internal.h"

namespace dg {
namespace {

constexpr int kMaxLevel = 15;

// block (12 bits) | level (4 bits) | ix, iy, iz (16 bits each)
inline uint64_t key(int b, int L, int i, int j, int k) {
    return ((uint64_t)b << 52) | ((uint64_t)L << 48) | ((uint64_t)i << 32) | ((uint64_t)j << 16) | (uint64_t)k;
}

inline void tangential(int d, int& t1, int& t2) {
    t1 = d == 0 ? 1 : 0;
    t2 = d == 2 ? 1 : 2;
}

// Physical corner (c1, c2) in {0, 1}^2 of block face f.
void face_corner(const dg_block& B, int f, int c1, int c2, double x[3]) {
    const int d = f >> 1;
    int t1, t2;
    tangential(d, t1, t2);
    double xi[3];
    xi[d] = (f & 1) ? 1.0 : -1.0;
    xi[t1] = c1 ? 1.0 : -1.0;
    xi[t2] = c2 ? 1.0 : -1.0;
    block_point(B, xi, x);
}

// Cell of block b' adjacent to face f of the level-lev cell idx of block b
// across the block interface (f on the block boundary); false on the domain
// boundary.
bool across(const BlockTopo& T, int b, int f, int lev, const int idx[3], int& b2, int& f2, int& o, int c2[3]) {
    const BlockFace& bf = T.face[6 * b + f];
    if (bf.nb < 0) return false;
    b2 = bf.nb;
    f2 = bf.nf;
    o = bf.orient;
    const int d = f >> 1, d2 = f2 >> 1, m = 1 << lev;
    int t1, t2, u1, u2;
    tangential(d, t1, t2);
    tangential(d2, u1, u2);
    int w1, w2;
    orient_cells(o, m, idx[t1], idx[t2], w1, w2);
    c2[d2] = (f2 & 1) ? m - 1 : 0;
    c2[u1] = w1;
    c2[u2] = w2;
    return true;
}

}  // namespace

bool block_face_neighbour(const BlockTopo& T, int b, int f, int lev, const int idx[3], int& b2, int c2[3]) {
    int f2 = 0, o = 0;
    return across(T, b, f, lev, idx, b2, f2, o, c2);
}

bool build_block_topology(const dg_block* blocks, int n_blocks, BlockTopo& topo, std::string& err) {
    topo.n_blocks = n_blocks;
    topo.face.assign(6 * (size_t)n_blocks, BlockFace{});
    if (n_blocks <= 1 || blocks == nullptr) return true;
    std::vector<double> C(6 * (size_t)n_blocks * 12);   // 4 corners x 3 per block face
    double scale = 1.0;
    for (int b = 0; b < n_blocks; ++b)
        for (int f = 0; f < 6; ++f)
            for (int c = 0; c < 4; ++c) {
                double* x = &C[((6 * (size_t)b + f) * 4 + c) * 3];
                face_corner(blocks[b], f, c & 1, c >> 1, x);
                for (int i = 0; i < 3; ++i) scale = std::max(scale, std::fabs(x[i]));
            }
    auto close = [&](const double* a, const double* b) {
        const double tol = 1e-9 * std::max(1.0, std::max(std::fabs(a[0]), std::max(std::fabs(a[1]), std::fabs(a[2]))));
        return std::fabs(a[0] - b[0]) <= tol && std::fabs(a[1] - b[1]) <= tol && std::fabs(a[2] - b[2]) <= tol;
    };
    for (int b = 0; b < n_blocks; ++b)
        for (int f = 0; f < 6; ++f) {
            const double* A = &C[(6 * (size_t)b + f) * 12];
            for (int b2 = 0; b2 < n_blocks && topo.face[6 * b + f].nb < 0; ++b2) {
                if (b2 == b) continue;
                for (int f2 = 0; f2 < 6 && topo.face[6 * b + f].nb < 0; ++f2) {
                    const double* Bc = &C[(6 * (size_t)b2 + f2) * 12];
                    for (int o = 0; o < 8; ++o) {
                        bool ok = true;
                        for (int c = 0; c < 4 && ok; ++c) {
                            int w1, w2;
                            orient_cells(o, 2, c & 1, c >> 1, w1, w2);
                            ok = close(A + 3 * c, Bc + 3 * (w1 + 2 * w2));
                        }
                        if (ok) {
                            topo.face[6 * b + f] = BlockFace{b2, f2, o};
                            break;
                        }
                    }
                }
            }
        }
    for (int b = 0; b < n_blocks; ++b)
        for (int f = 0; f < 6; ++f) {
            const BlockFace& bf = topo.face[6 * b + f];
            if (bf.nb < 0) continue;
            const BlockFace& back = topo.face[6 * bf.nb + bf.nf];
            if (back.nb != b || back.nf != f) {
                err = "block faces are glued inconsistently (block " + std::to_string(b) + ")";
                return false;
            }
        }
    return true;
}

bool build_level_connectivity(LevelHost& L, const BlockTopo& T, std::string& err) {
    const int ne = L.n_elems();
    if ((int)L.block.size() != ne) L.block.assign(ne, 0);
    std::unordered_map<uint64_t, int> idx;
    idx.reserve(ne * 2);
    for (int e = 0; e < ne; ++e) {
        const int* lf = &L.leaves[4 * e];
        if (L.block[e] < 0 || L.block[e] >= T.n_blocks) { err = "element block index out of range"; return false; }
        if (lf[0] < 0 || lf[0] > kMaxLevel) { err = "leaf level out of range (0..15)"; return false; }
        int m = 1 << lf[0];
        for (int d = 0; d < 3; ++d)
            if (lf[1 + d] < 0 || lf[1 + d] >= m) { err = "leaf index out of range"; return false; }
        if (L.p[e] < 1 || L.p[e] > kMaxN - 1) { err = "polynomial degree must be in 1..8"; return false; }
        if (!idx.emplace(key(L.block[e], lf[0], lf[1], lf[2], lf[3]), e).second) { err = "duplicate leaf"; return false; }
    }
    L.dof_off.assign(ne + 1, 0);
    L.vqp_off.assign(ne + 1, 0);
    for (int e = 0; e < ne; ++e) {
        long long n = L.p[e] + 1;
        L.dof_off[e + 1] = L.dof_off[e] + n * n * n;
        L.vqp_off[e + 1] = L.vqp_off[e] + n * n * n;
    }
    L.mortars.clear();
    std::vector<std::vector<int>> em(ne * 6);
    long long goff = 0, boff = 0;
    auto not_covered = [&](int e, int f) {
        err = "mesh is not 2:1 balanced or does not tile the blocks (element " + std::to_string(e) + ", face " +
              std::to_string(f) + ")";
        return false;
    };
    for (int e = 0; e < ne; ++e) {
        const int* lf = &L.leaves[4 * e];
        const int lev = lf[0], b = L.block[e];
        for (int f = 0; f < 6; ++f) {
            const int d = f >> 1, s = f & 1;
            int j[3] = {lf[1], lf[2], lf[3]};
            j[d] += s ? 1 : -1;
            Mortar m{};
            m.eA = e;
            m.fA = (unsigned char)f;
            m.posA0 = m.posA1 = 0;
            m.eB = -1;
            m.bnd_off = -1;
            m.orient = 0;
            int pm = L.p[e];
            // the neighbouring region: same block (cell j, face opposite to f) or across the interface
            int nb = b, fB = 2 * d + (1 - s), o = 0, c[3] = {j[0], j[1], j[2]};
            bool boundary = false;
            if (j[d] < 0 || j[d] >= (1 << lev)) {
                const int self[3] = {lf[1], lf[2], lf[3]};
                if (!across(T, b, f, lev, self, nb, fB, o, c)) boundary = true;
            }
            if (boundary) {
                m.bnd_off = boff;
            } else {
                const int dB = fB >> 1, sB = fB & 1;
                int u1, u2;
                tangential(dB, u1, u2);
                auto it = idx.find(key(nb, lev, c[0], c[1], c[2]));
                if (it != idx.end()) {
                    if (it->second < e) continue;
                    m.eB = it->second;
                    m.fB = (unsigned char)fB;
                    m.posB0 = m.posB1 = 0;
                    m.orient = (unsigned char)o;
                } else {
                    auto ic = lev > 0 ? idx.find(key(nb, lev - 1, c[0] >> 1, c[1] >> 1, c[2] >> 1)) : idx.end();
                    if (ic != idx.end()) {
                        m.eB = ic->second;
                        m.fB = (unsigned char)fB;
                        m.posB0 = (unsigned char)(1 + (c[u1] & 1));
                        m.posB1 = (unsigned char)(1 + (c[u2] & 1));
                        m.orient = (unsigned char)o;
                    } else {
                        // must be covered by four finer neighbours (created from their side)
                        for (int q = 0; q < 4; ++q) {
                            int cc[3] = {2 * c[0], 2 * c[1], 2 * c[2]};
                            cc[dB] = 2 * c[dB] + (sB ? 1 : 0);
                            cc[u1] += q & 1;
                            cc[u2] += q >> 1;
                            if (idx.find(key(nb, lev + 1, cc[0], cc[1], cc[2])) == idx.end()) return not_covered(e, f);
                        }
                        continue;
                    }
                }
                pm = std::max(pm, L.p[m.eB]);
            }
            m.q = (unsigned char)(pm + 1);
            m.goff = goff;
            goff += (long long)m.q * m.q;
            if (m.eB < 0) boff += (long long)m.q * m.q;
            L.mortars.push_back(m);
        }
    }
    L.n_mortar_pts = goff;
    L.n_bnd_pts = boff;
    for (int mi = 0; mi < (int)L.mortars.size(); ++mi) {
        const Mortar& m = L.mortars[mi];
        em[m.eA * 6 + m.fA].push_back(mi);
        if (m.eB >= 0) em[m.eB * 6 + m.fB].push_back(mi);
    }
    L.slot_off.assign(ne + 1, 0);
    L.slot_mortar.clear();
    L.slot_face.clear();
    L.slot_side.clear();
    for (int e = 0; e < ne; ++e) {
        for (int f = 0; f < 6; ++f) {
            const auto& v = em[e * 6 + f];
            if (v.size() != 1 && v.size() != 4) {
                err = "face covered by an unexpected number of mortars";
                return false;
            }
            for (int mi : v) {
                L.slot_mortar.push_back(mi);
                L.slot_face.push_back((unsigned char)f);
                L.slot_side.push_back(L.mortars[mi].eA == e ? 0 : 1);
            }
        }
        L.slot_off[e + 1] = (int)L.slot_mortar.size();
    }
    for (int n = 0; n <= kMaxN; ++n) L.buckets[n].clear();
    for (int e = 0; e < ne; ++e) L.buckets[L.p[e] + 1].push_back(e);
    return true;
}

bool coarsen_level(const LevelHost& fine, LevelHost& coarse, const BlockTopo& T, std::string& err) {
    const int ne = fine.n_elems();
    auto blk = [&](int e) { return fine.block.empty() ? 0 : fine.block[e]; };
    std::unordered_map<uint64_t, std::vector<int>> fam;
    for (int e = 0; e < ne; ++e) {
        const int* lf = &fine.leaves[4 * e];
        if (lf[0] == 0) continue;
        fam[key(blk(e), lf[0] - 1, lf[1] >> 1, lf[2] >> 1, lf[3] >> 1)].push_back(e);
    }
    std::unordered_set<uint64_t> merged;
    for (auto& kv : fam)
        if (kv.second.size() == 8) merged.insert(kv.first);
    if (merged.empty()) return false;
    auto parent_of = [&](int e) -> uint64_t {
        const int* lf = &fine.leaves[4 * e];
        return lf[0] == 0 ? ~0ull : key(blk(e), lf[0] - 1, lf[1] >> 1, lf[2] >> 1, lf[3] >> 1);
    };
    int maxL = 0;
    for (int e = 0; e < ne; ++e) maxL = std::max(maxL, fine.leaves[4 * e]);
    while (true) {
        std::unordered_set<uint64_t> cells;
        for (int e = 0; e < ne; ++e) {
            uint64_t P = parent_of(e);
            if (merged.count(P)) cells.insert(P);
            else {
                const int* lf = &fine.leaves[4 * e];
                cells.insert(key(blk(e), lf[0], lf[1], lf[2], lf[3]));
            }
        }
        std::vector<uint64_t> undo;
        for (uint64_t P : merged) {
            const int b = (int)(P >> 52), Lv = (int)((P >> 48) & 0xF);
            const int c0[3] = {(int)((P >> 32) & 0xFFFF), (int)((P >> 16) & 0xFFFF), (int)(P & 0xFFFF)};
            bool bad = false;
            for (int f = 0; f < 6 && !bad; ++f) {
                const int d = f >> 1, sg = (f & 1) ? 1 : -1;
                // the neighbouring cell at level Lv and the face of it that P touches
                int nb = b, fB = 2 * d + (sg < 0 ? 1 : 0), o = 0, c[3] = {c0[0], c0[1], c0[2]};
                c[d] += sg;
                if (c[d] < 0 || c[d] >= (1 << Lv)) {
                    if (!across(T, b, f, Lv, c0, nb, fB, o, c)) continue;
                }
                const int dB = fB >> 1, sB = fB & 1;
                for (int L2 = Lv + 2; L2 <= maxL && !bad; ++L2) {
                    int sh = L2 - Lv, span = 1 << sh;
                    int a0[3], a1[3];
                    for (int t = 0; t < 3; ++t) {
                        a0[t] = c[t] << sh;
                        a1[t] = a0[t] + span;
                    }
                    a0[dB] = (c[dB] << sh) + (sB ? span - 1 : 0);
                    a1[dB] = a0[dB] + 1;
                    for (int x = a0[0]; x < a1[0] && !bad; ++x)
                        for (int y = a0[1]; y < a1[1] && !bad; ++y)
                            for (int z = a0[2]; z < a1[2] && !bad; ++z)
                                if (cells.count(key(nb, L2, x, y, z))) bad = true;
                }
            }
            if (bad) undo.push_back(P);
        }
        if (undo.empty()) break;
        for (auto P : undo) merged.erase(P);
        if (merged.empty()) return false;
    }
    coarse.leaves.clear();
    coarse.block.clear();
    coarse.p.clear();
    coarse.child_off.assign(1, 0);
    coarse.child_id.clear();
    coarse.child_bits.clear();
    coarse.fine_parent.assign(ne, -1);
    coarse.fine_bits.assign(ne, 0xFF);
    std::unordered_map<uint64_t, int> emitted;
    for (int e = 0; e < ne; ++e) {
        uint64_t P = parent_of(e);
        const int* lf = &fine.leaves[4 * e];
        if (merged.count(P)) {
            if (emitted.count(P)) continue;
            int H = (int)coarse.p.size();
            emitted[P] = H;
            std::vector<int> ch = fam[P];
            std::sort(ch.begin(), ch.end());
            int pmin = 99;
            for (int c : ch) {
                const int* cl = &fine.leaves[4 * c];
                unsigned char bits = (unsigned char)((cl[1] & 1) | ((cl[2] & 1) << 1) | ((cl[3] & 1) << 2));
                coarse.child_id.push_back(c);
                coarse.child_bits.push_back(bits);
                coarse.fine_parent[c] = H;
                coarse.fine_bits[c] = bits;
                pmin = std::min(pmin, fine.p[c]);
            }
            coarse.leaves.insert(coarse.leaves.end(), {lf[0] - 1, lf[1] >> 1, lf[2] >> 1, lf[3] >> 1});
            coarse.block.push_back(blk(e));
            coarse.p.push_back(pmin);
        } else {
            int H = (int)coarse.p.size();
            coarse.child_id.push_back(e);
            coarse.child_bits.push_back(0xFF);
            coarse.fine_parent[e] = H;
            coarse.fine_bits[e] = 0xFF;
            coarse.leaves.insert(coarse.leaves.end(), {lf[0], lf[1], lf[2], lf[3]});
            coarse.block.push_back(blk(e));
            coarse.p.push_back(fine.p[e]);
        }
        coarse.child_off.push_back((int)coarse.child_id.size());
    }
    return build_level_connectivity(coarse, T, err);
}

}  // namespace dg
