// Host-side mesh tables: mortar set of an octree mesh (Sec. II.A.1) and the
// multigrid level meshes (Sec. II.E.3).
//
// Mortars: every element face is covered either by the domain boundary, by one
// same-size neighbour, by one coarser neighbour (this face is a quarter of the
// neighbour's face) or by four finer neighbours.  One mortar is created per
// interface piece: on conforming faces from the lower-index element, on 2:1
// faces from the finer element, on the boundary from the owner.  The creating
// element is side A (the side whose map supplies S^m and the normal).  The
// mortar degree is max(p_A, p_B) (mortar figure) with p_m + 1 GL points per
// direction.
//
// Level meshes: complete sibling families are merged into their parent
// (surrogate mesh); a merged parent that would face an element two or more
// levels finer is split again (2:1 rebalancing); the coarse degree is the
// minimum over the children.  Coarse elements are numbered in the order in
// which their first child appears on the finer level.
#include <algorithm>
#include <unordered_map>
#include <unordered_set>

#include "internal.h"

namespace dg {
namespace {

inline uint64_t key(int L, int i, int j, int k) {
    return ((uint64_t)L << 57) | ((uint64_t)i << 38) | ((uint64_t)j << 19) | (uint64_t)k;
}

inline void tangential(int d, int& t1, int& t2) {
    t1 = d == 0 ? 1 : 0;
    t2 = d == 2 ? 1 : 2;
}

}  // namespace

bool build_level_connectivity(LevelHost& L, std::string& err) {
    const int ne = L.n_elems();
    std::unordered_map<uint64_t, int> idx;
    idx.reserve(ne * 2);
    for (int e = 0; e < ne; ++e) {
        const int* lf = &L.leaves[4 * e];
        if (lf[0] < 0 || lf[0] > 18) { err = "leaf level out of range"; return false; }
        int m = 1 << lf[0];
        for (int d = 0; d < 3; ++d)
            if (lf[1 + d] < 0 || lf[1 + d] >= m) { err = "leaf index out of range"; return false; }
        if (L.p[e] < 1 || L.p[e] > kMaxN - 1) { err = "polynomial degree must be in 1..8"; return false; }
        if (!idx.emplace(key(lf[0], lf[1], lf[2], lf[3]), e).second) { err = "duplicate leaf"; return false; }
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
    for (int e = 0; e < ne; ++e) {
        const int* lf = &L.leaves[4 * e];
        const int lev = lf[0];
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
            int pm = L.p[e];
            if (j[d] < 0 || j[d] >= (1 << lev)) {
                m.bnd_off = boff;
            } else {
                auto it = idx.find(key(lev, j[0], j[1], j[2]));
                int t1, t2;
                tangential(d, t1, t2);
                if (it != idx.end()) {
                    if (it->second < e) continue;
                    m.eB = it->second;
                    m.fB = (unsigned char)(2 * d + (1 - s));
                    m.posB0 = m.posB1 = 0;
                } else {
                    auto ic = lev > 0 ? idx.find(key(lev - 1, j[0] >> 1, j[1] >> 1, j[2] >> 1)) : idx.end();
                    if (ic != idx.end()) {
                        m.eB = ic->second;
                        m.fB = (unsigned char)(2 * d + (1 - s));
                        m.posB0 = (unsigned char)(1 + (lf[1 + t1] & 1));
                        m.posB1 = (unsigned char)(1 + (lf[1 + t2] & 1));
                    } else {
                        // must be covered by four finer neighbours (created from their side)
                        for (int b = 0; b < 4; ++b) {
                            int c[3] = {2 * j[0], 2 * j[1], 2 * j[2]};
                            c[d] = 2 * j[d] + (s ? 0 : 1);
                            c[t1] += b & 1;
                            c[t2] += b >> 1;
                            if (idx.find(key(lev + 1, c[0], c[1], c[2])) == idx.end()) {
                                err = "mesh is not 2:1 balanced or does not tile the block (element " +
                                      std::to_string(e) + ", face " + std::to_string(f) + ")";
                                return false;
                            }
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

bool coarsen_level(const LevelHost& fine, LevelHost& coarse, std::string& err) {
    const int ne = fine.n_elems();
    std::unordered_map<uint64_t, std::vector<int>> fam;
    for (int e = 0; e < ne; ++e) {
        const int* lf = &fine.leaves[4 * e];
        if (lf[0] == 0) continue;
        fam[key(lf[0] - 1, lf[1] >> 1, lf[2] >> 1, lf[3] >> 1)].push_back(e);
    }
    std::unordered_set<uint64_t> merged;
    for (auto& kv : fam)
        if (kv.second.size() == 8) merged.insert(kv.first);
    if (merged.empty()) return false;
    auto parent_of = [&](int e) -> uint64_t {
        const int* lf = &fine.leaves[4 * e];
        return lf[0] == 0 ? ~0ull : key(lf[0] - 1, lf[1] >> 1, lf[2] >> 1, lf[3] >> 1);
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
                cells.insert(key(lf[0], lf[1], lf[2], lf[3]));
            }
        }
        std::vector<uint64_t> undo;
        for (uint64_t P : merged) {
            int Lv = (int)(P >> 57), c0[3] = {(int)((P >> 38) & 0x7FFFF), (int)((P >> 19) & 0x7FFFF), (int)(P & 0x7FFFF)};
            bool bad = false;
            for (int d = 0; d < 3 && !bad; ++d)
                for (int sg = -1; sg <= 1 && !bad; sg += 2) {
                    int c[3] = {c0[0], c0[1], c0[2]};
                    c[d] += sg;
                    if (c[d] < 0 || c[d] >= (1 << Lv)) continue;
                    for (int L2 = Lv + 2; L2 <= maxL && !bad; ++L2) {
                        int sh = L2 - Lv, span = 1 << sh;
                        int lo[3] = {c[0] << sh, c[1] << sh, c[2] << sh};
                        int a0[3], a1[3];
                        for (int t = 0; t < 3; ++t) { a0[t] = lo[t]; a1[t] = lo[t] + span; }
                        a0[d] = lo[d] + (sg < 0 ? span - 1 : 0);
                        a1[d] = a0[d] + 1;
                        for (int x = a0[0]; x < a1[0] && !bad; ++x)
                            for (int y = a0[1]; y < a1[1] && !bad; ++y)
                                for (int z = a0[2]; z < a1[2] && !bad; ++z)
                                    if (cells.count(key(L2, x, y, z))) bad = true;
                    }
                }
            if (bad) undo.push_back(P);
        }
        if (undo.empty()) break;
        for (auto P : undo) merged.erase(P);
        if (merged.empty()) return false;
    }
    coarse.leaves.clear();
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
            coarse.p.push_back(pmin);
        } else {
            int H = (int)coarse.p.size();
            coarse.child_id.push_back(e);
            coarse.child_bits.push_back(0xFF);
            coarse.fine_parent[e] = H;
            coarse.fine_bits[e] = 0xFF;
            coarse.leaves.insert(coarse.leaves.end(), {lf[0], lf[1], lf[2], lf[3]});
            coarse.p.push_back(fine.p[e]);
        }
        coarse.child_off.push_back((int)coarse.child_id.size());
    }
    return build_level_connectivity(coarse, err);
}

}  // namespace dg
