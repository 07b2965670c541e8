// hp-AMR driving strategy (Sec. II.D, Algorithm 4 "smooth-pred") and the
// refinement of a single-box leaf set with 2:1 balancing.  Host code.
//
// Marking: the ceil(theta n) largest eta^2 (ties to the lower index) or
// eta^2 > theta * mean (mean summed in element order).  Decision per marked
// element: h when eta^2 exceeds the element's predicted eta^2, else p; the
// predictions are gamma_h 2^-d 2^(-2p) eta^2 for h-children and
// gamma_p eta^2 for p-refined elements.
//
// Balancing: every leaf looks at the cell of its own size across each of its
// six faces; when the leaf covering that cell is two or more levels coarser,
// that leaf is refined.  Repeated until nothing changes, this gives the
// smallest 2:1-balanced refinement of the marked one (finer-side checks find
// every violation, since a violating pair is always seen from its fine side).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "dgell.h"

extern "C" int dgi_set_error(int code, const char* msg);

namespace {

constexpr int kMaxLevel = 15;
constexpr int kMaxP = 8;

struct Leaf {
    int L, ix, iy, iz, p;
    double pred;
    int parent;
};

uint64_t key_of(int L, int ix, int iy, int iz) {
    return ((uint64_t)L << 48) | ((uint64_t)ix << 32) | ((uint64_t)iy << 16) | (uint64_t)iz;
}

void push_children(const Leaf& a, int p, double pred, std::vector<Leaf>& out) {
    for (int c = 0; c < 8; ++c)
        out.push_back(Leaf{a.L + 1, 2 * a.ix + (c & 1), 2 * a.iy + ((c >> 1) & 1), 2 * a.iz + ((c >> 2) & 1), p, pred,
                           a.parent});
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
        const int L = leaves[4 * e], ix = leaves[4 * e + 1], iy = leaves[4 * e + 2], iz = leaves[4 * e + 3];
        if (L < 0 || L > kMaxLevel || ix < 0 || iy < 0 || iz < 0 || ix >= (1 << L) || iy >= (1 << L) || iz >= (1 << L))
            return dgi_set_error(DG_ERR_INVALID, "dg_hp_refine: leaf outside its level's index range");
        if (p[e] < 1 || p[e] > kMaxP) return dgi_set_error(DG_ERR_INVALID, "dg_hp_refine: degree outside 1..8");
        const Leaf a{L, ix, iy, iz, p[e], pred_next[e], e};
        if (action[e] == DG_AMR_H_REFINE) {
            if (L >= kMaxLevel) return dgi_set_error(DG_ERR_INVALID, "dg_hp_refine: h-refinement past level 15");
            push_children(a, p[e], pred_next[e], cur);
        } else if (action[e] == DG_AMR_P_REFINE) {
            if (p[e] >= kMaxP) return dgi_set_error(DG_ERR_INVALID, "dg_hp_refine: degree past 8");
            Leaf b = a;
            b.p = p[e] + 1;
            cur.push_back(b);
        } else if (action[e] == DG_AMR_NONE) {
            cur.push_back(a);
        } else {
            return dgi_set_error(DG_ERR_INVALID, "dg_hp_refine: unknown action");
        }
    }
    std::unordered_map<uint64_t, int> at;
    for (;;) {
        at.clear();
        at.reserve(cur.size() * 2);
        for (int i = 0; i < (int)cur.size(); ++i) at[key_of(cur[i].L, cur[i].ix, cur[i].iy, cur[i].iz)] = i;
        std::vector<char> split(cur.size(), 0);
        bool any = false;
        for (const Leaf& a : cur) {
            const int m = 1 << a.L;
            for (int f = 0; f < 6; ++f) {
                int j[3] = {a.ix, a.iy, a.iz};
                j[f >> 1] += (f & 1) ? 1 : -1;
                if (j[f >> 1] < 0 || j[f >> 1] >= m) continue;   // domain boundary
                for (int l = a.L; l >= 0; --l) {                 // the leaf covering that cell, if not finer
                    const int sh = a.L - l;
                    auto it = at.find(key_of(l, j[0] >> sh, j[1] >> sh, j[2] >> sh));
                    if (it == at.end()) continue;
                    if (l < a.L - 1 && !split[it->second]) {
                        split[it->second] = 1;
                        any = true;
                    }
                    break;
                }
            }
        }
        if (!any) break;
        std::vector<Leaf> nxt;
        nxt.reserve(cur.size() + 8);
        for (size_t i = 0; i < cur.size(); ++i) {
            if (split[i]) push_children(cur[i], cur[i].p, pred_init, nxt);
            else nxt.push_back(cur[i]);
        }
        cur.swap(nxt);
    }
    const int total = (int)cur.size();
    *n_out = total;
    if (total > max_out) return dgi_set_error(DG_ERR_INVALID, "dg_hp_refine: output arrays too small (see *n_out)");
    for (int i = 0; i < total; ++i) {
        const Leaf& a = cur[i];
        if (leaves_out) {
            leaves_out[4 * i] = a.L;
            leaves_out[4 * i + 1] = a.ix;
            leaves_out[4 * i + 2] = a.iy;
            leaves_out[4 * i + 3] = a.iz;
        }
        if (p_out) p_out[i] = a.p;
        if (pred_out) pred_out[i] = a.pred;
        if (parent_out) parent_out[i] = a.parent;
    }
    return DG_OK;
}
