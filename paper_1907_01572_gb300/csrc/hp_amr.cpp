// hp-AMR driving strategy (Sec. II.D, Algorithm 4 "smooth-pred") and the
// refinement of a leaf set -- one box or a multi-block mesh -- with 2:1
// balancing, inside blocks and across block interfaces.  Host code.
//
// Marking: the ceil(theta n) largest eta^2 (ties to the lower index) or
// eta^2 > theta * mean (mean summed in element order).  Decision per marked
// element: h when eta^2 exceeds the element's predicted eta^2, else p; the
// predictions are gamma_h 2^-d 2^(-2p) eta^2 for h-children and
// gamma_p eta^2 for p-refined elements.
//
// Balancing: every leaf looks at the cell of its own size across each of its
// six faces (in its own block, or in the neighbouring block's frame through
// the block connectivity the mesh description defines); when the leaf
// covering that cell is two or more levels coarser,
// that leaf is refined.  Repeated until nothing changes, this gives the
// smallest 2:1-balanced refinement of the marked one (finer-side checks find
// every violation, since a violating pair is always seen from its fine side).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.h"

extern "C" int dgi_set_error(int code, const char* msg);

namespace {

constexpr int kMaxLevel = 15;
constexpr int kMaxP = 8;

struct Leaf {
    int b, L, ix, iy, iz, p;
    double pred;
    int parent;
};

// block (12 bits) | level (4 bits) | ix, iy, iz (16 bits each)
uint64_t key_of(int b, int L, int ix, int iy, int iz) {
    return ((uint64_t)b << 52) | ((uint64_t)L << 48) | ((uint64_t)ix << 32) | ((uint64_t)iy << 16) | (uint64_t)iz;
}

void push_children(const Leaf& a, int p, double pred, std::vector<Leaf>& out) {
    for (int c = 0; c < 8; ++c)
        out.push_back(Leaf{a.b, a.L + 1, 2 * a.ix + (c & 1), 2 * a.iy + ((c >> 1) & 1), 2 * a.iz + ((c >> 2) & 1), p,
                           pred, a.parent});
}

// The cell of a's size across face f: in a's block, or across a block
// interface (T set); false on the domain boundary.
bool neighbour_cell(const dg::BlockTopo* T, const Leaf& a, int f, int& b2, int j[3]) {
    j[0] = a.ix;
    j[1] = a.iy;
    j[2] = a.iz;
    j[f >> 1] += (f & 1) ? 1 : -1;
    if (j[f >> 1] >= 0 && j[f >> 1] < (1 << a.L)) {
        b2 = a.b;
        return true;
    }
    if (!T) return false;
    const int idx[3] = {a.ix, a.iy, a.iz};
    return dg::block_face_neighbour(*T, a.b, f, a.L, idx, b2, j);
}

// Input element e with its action: appended to cur (children in place of an
// h-refined element).  Returns DG_OK or an error code (message set).
int push_action(const Leaf& a, int action, std::vector<Leaf>& cur) {
    if (a.L < 0 || a.L > kMaxLevel || a.ix < 0 || a.iy < 0 || a.iz < 0 || a.ix >= (1 << a.L) || a.iy >= (1 << a.L) ||
        a.iz >= (1 << a.L))
        return dgi_set_error(DG_ERR_INVALID, "hp refinement: leaf outside its level's index range");
    if (a.p < 1 || a.p > kMaxP) return dgi_set_error(DG_ERR_INVALID, "hp refinement: degree outside 1..8");
    if (action == DG_AMR_H_REFINE) {
        if (a.L >= kMaxLevel) return dgi_set_error(DG_ERR_INVALID, "hp refinement: h-refinement past level 15");
        push_children(a, a.p, a.pred, cur);
    } else if (action == DG_AMR_P_REFINE) {
        if (a.p >= kMaxP) return dgi_set_error(DG_ERR_INVALID, "hp refinement: degree past 8");
        Leaf b = a;
        b.p = a.p + 1;
        cur.push_back(b);
    } else if (action == DG_AMR_NONE) {
        cur.push_back(a);
    } else {
        return dgi_set_error(DG_ERR_INVALID, "hp refinement: unknown action");
    }
    return DG_OK;
}

// 2:1 balancing: leaves whose face neighbour is two or more levels finer are
// split (children keep the degree and get pred_init) until none is left.
void balance(std::vector<Leaf>& cur, const dg::BlockTopo* T, double pred_init) {
    std::unordered_map<uint64_t, int> at;
    for (;;) {
        at.clear();
        at.reserve(cur.size() * 2);
        for (int i = 0; i < (int)cur.size(); ++i) at[key_of(cur[i].b, cur[i].L, cur[i].ix, cur[i].iy, cur[i].iz)] = i;
        std::vector<char> split(cur.size(), 0);
        bool any = false;
        for (const Leaf& a : cur) {
            for (int f = 0; f < 6; ++f) {
                int b2 = 0, j[3];
                if (!neighbour_cell(T, a, f, b2, j)) continue;   // domain boundary
                for (int l = a.L; l >= 0; --l) {                 // the leaf covering that cell, if not finer
                    const int sh = a.L - l;
                    auto it = at.find(key_of(b2, l, j[0] >> sh, j[1] >> sh, j[2] >> sh));
                    if (it == at.end()) continue;
                    if (l < a.L - 1 && !split[it->second]) {
                        split[it->second] = 1;
                        any = true;
                    }
                    break;
                }
            }
        }
        if (!any) return;
        std::vector<Leaf> nxt;
        nxt.reserve(cur.size() + 8);
        for (size_t i = 0; i < cur.size(); ++i) {
            if (split[i]) push_children(cur[i], cur[i].p, pred_init, nxt);
            else nxt.push_back(cur[i]);
        }
        cur.swap(nxt);
    }
}

int write_out(const std::vector<Leaf>& cur, int max_out, int* n_out, int* leaves_out, int* p_out, int* block_out,
              double* pred_out, int* parent_out) {
    const int total = (int)cur.size();
    *n_out = total;
    if (total > max_out) return dgi_set_error(DG_ERR_INVALID, "hp refinement: output arrays too small (see *n_out)");
    for (int i = 0; i < total; ++i) {
        const Leaf& a = cur[i];
        if (leaves_out) {
            leaves_out[4 * i] = a.L;
            leaves_out[4 * i + 1] = a.ix;
            leaves_out[4 * i + 2] = a.iy;
            leaves_out[4 * i + 3] = a.iz;
        }
        if (p_out) p_out[i] = a.p;
        if (block_out) block_out[i] = a.b;
        if (pred_out) pred_out[i] = a.pred;
        if (parent_out) parent_out[i] = a.parent;
    }
    return DG_OK;
}

}  // namespace

extern "C" int dg_hp_mark(int n, const double* eta2, const double* pred, const int* p, const int* level,
                          const dg_amr_opts* o, int* action, double* pred_next) {
    if (n < 0 || !o || (n > 0 && (!eta2 || !pred || !p || !level || !action || !pred_next)))
        return dgi_set_error(DG_ERR_INVALID, "dg_hp_mark: NULL argument");
    if (o->criterion != DG_MARK_FRACTION && o->criterion != DG_MARK_MEAN)
        return dgi_set_error(DG_ERR_INVALID, "dg_hp_mark: unknown criterion");
    if (o->criterion == DG_MARK_FRACTION ? !(o->theta > 0.0 && o->theta <= 1.0)
                                         : !(o->theta >= 0.0 && std::isfinite(o->theta)))
        return dgi_set_error(DG_ERR_INVALID, "dg_hp_mark: theta outside (0, 1] (fraction) or [0, inf) (mean)");
    const double gh = o->gamma_h > 0 ? o->gamma_h : 0.25;
    const double gp = o->gamma_p > 0 ? o->gamma_p : 0.1;
    const int pmax = o->p_max > 0 ? o->p_max : kMaxP;
    const int lmax = o->level_max > 0 ? o->level_max : kMaxLevel;
    std::vector<char> marked(n, 0);
    if (o->criterion == DG_MARK_FRACTION) {
        const double kd = std::ceil(o->theta * n);   // theta in (0, 1]: 1 <= kd <= n
        const int kk = kd > n ? n : (int)kd;
        std::vector<int> order(n);
        std::iota(order.begin(), order.end(), 0);
        // the kk largest, ties to the lower index: a strict weak order on (-eta2, e)
        auto before = [&](int a, int b) { return eta2[a] > eta2[b] || (eta2[a] == eta2[b] && a < b); };
        std::sort(order.begin(), order.end(), before);
        for (int i = 0; i < kk; ++i) marked[order[i]] = 1;
    } else {
        double s = 0.0;
        for (int e = 0; e < n; ++e) s += eta2[e];
        const double mean = n > 0 ? s / n : 0.0;
        for (int e = 0; e < n; ++e) marked[e] = eta2[e] > o->theta * mean;
    }
    for (int e = 0; e < n; ++e) {
        int a = DG_AMR_NONE;
        if (marked[e]) {
            a = eta2[e] > pred[e] ? DG_AMR_H_REFINE : DG_AMR_P_REFINE;
            if (a == DG_AMR_P_REFINE && p[e] >= pmax) a = DG_AMR_H_REFINE;
            if (a == DG_AMR_H_REFINE && level[e] >= lmax) a = p[e] < pmax ? DG_AMR_P_REFINE : DG_AMR_NONE;
        }
        action[e] = a;
        if (a == DG_AMR_H_REFINE)
            pred_next[e] = gh * std::ldexp(1.0, -3) * std::ldexp(1.0, -2 * p[e]) * eta2[e];
        else if (a == DG_AMR_P_REFINE)
            pred_next[e] = gp * eta2[e];
        else
            pred_next[e] = pred[e];
    }
    return DG_OK;
}

extern "C" int dg_hp_refine(int n, const int* leaves, const int* p, const int* action, const double* pred_next,
                            double pred_init, int max_out, int* n_out, int* leaves_out, int* p_out,
                            double* pred_out, int* parent_out) {
    if (n < 0 || !n_out || (n > 0 && (!leaves || !p || !action || !pred_next)))
        return dgi_set_error(DG_ERR_INVALID, "dg_hp_refine: NULL argument");
    std::vector<Leaf> cur;
    cur.reserve((size_t)n + 16);
    for (int e = 0; e < n; ++e) {
        const Leaf a{0, leaves[4 * e], leaves[4 * e + 1], leaves[4 * e + 2], leaves[4 * e + 3], p[e], pred_next[e], e};
        const int rc = push_action(a, action[e], cur);
        if (rc) return rc;
    }
    balance(cur, nullptr, pred_init);
    return write_out(cur, max_out, n_out, leaves_out, p_out, nullptr, pred_out, parent_out);
}

extern "C" int dg_hp_refine_mesh(const dg_mesh_desc* mesh, const int* action, const double* pred_next, double pred_init,
                                 int max_out, int* n_out, int* leaves_out, int* p_out, int* block_out,
                                 double* pred_out, int* parent_out) {
    if (!mesh || !n_out || mesh->n_elems < 0 ||
        (mesh->n_elems > 0 && (!mesh->leaves || !mesh->p || !action || !pred_next)))
        return dgi_set_error(DG_ERR_INVALID, "dg_hp_refine_mesh: NULL argument");
    const int n = mesh->n_elems, nb = mesh->n_blocks;
    if (nb < 0 || nb > 4096 || (nb > 0 && (!mesh->blocks || !mesh->elem_block)))
        return dgi_set_error(DG_ERR_INVALID, "dg_hp_refine_mesh: bad block description");
    dg::BlockTopo topo;
    std::string err;
    if (nb > 0 && !dg::build_block_topology(mesh->blocks, nb, topo, err))
        return dgi_set_error(DG_ERR_INVALID, err.c_str());
    std::vector<Leaf> cur;
    cur.reserve((size_t)n + 16);
    for (int e = 0; e < n; ++e) {
        const int b = nb > 0 ? mesh->elem_block[e] : 0;
        if (b < 0 || b >= (nb > 0 ? nb : 1)) return dgi_set_error(DG_ERR_INVALID, "dg_hp_refine_mesh: block index out of range");
        const int* lf = mesh->leaves + 4 * e;
        const Leaf a{b, lf[0], lf[1], lf[2], lf[3], mesh->p[e], pred_next[e], e};
        const int rc = push_action(a, action[e], cur);
        if (rc) return rc;
    }
    balance(cur, nb > 0 ? &topo : nullptr, pred_init);
    return write_out(cur, max_out, n_out, leaves_out, p_out, block_out, pred_out, parent_out);
}
