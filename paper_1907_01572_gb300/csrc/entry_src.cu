// C ABI entry points for right-hand sides, the zeroth-order term (with its
// Galerkin coarse-level form, eq. operator_oh) and the puncture equation
// solved by Newton-Raphson (Alg. 1).
#include <chrono>
#include <cmath>
#include <string>

#include "context.h"
#include "newton.h"
#include "source.h"

using namespace dg;

// shares dg_last_error's buffer (defined in context.cu)
extern "C" int dgi_set_error(int code, const char* msg);

#define CK2(call)                                                                                 \
    do {                                                                                          \
        cudaError_t _e = (call);                                                                  \
        if (_e == cudaSuccess && debug_sync()) _e = cudaDeviceSynchronize();                      \
        if (_e != cudaSuccess)                                                                    \
            return dgi_set_error(DG_ERR_CUDA, (std::string(#call) + ": " + cudaGetErrorString(_e)).c_str()); \
        if (debug_sync()) {                                                                       \
            int _f = 0;                                                                           \
            cudaMemcpy(&_f, device_check_flag(), sizeof(int), cudaMemcpyDeviceToHost);           \
            if (_f) return dgi_set_error(DG_ERR_CUDA, (std::string("self-check ") + std::to_string(_f) + " in " + #call).c_str()); \
        }                                                                                         \
    } while (0)

namespace {

// Finest descendants of every coarse element and the affine maps from their
// reference coordinates to the ancestor's (xi_H = s xi_f + o per axis).
int ensure_galerkin_structure(dg_ctx* c) {
    if (c->galerkin_ready) return DG_OK;
    const int Lt = (int)c->lv.size() - 1;
    const LevelHost& fin = c->lv[Lt].h;
    const int nf = fin.n_elems();
    std::vector<int> anc(nf);
    for (int f = 0; f < nf; ++f) anc[f] = f;
    for (int l = Lt - 1; l >= 0; --l) {
        LevelDev& L = c->lv[l];
        const LevelHost& h = L.h;
        for (int f = 0; f < nf; ++f) anc[f] = h.fine_parent[anc[f]];
        const int nc = h.n_elems();
        std::vector<int> cnt(nc + 1, 0);
        for (int f = 0; f < nf; ++f) cnt[anc[f] + 1]++;
        for (int H = 0; H < nc; ++H) cnt[H + 1] += cnt[H];
        std::vector<int> desc(nf), fill(cnt.begin(), cnt.end() - 1);
        std::vector<double> map(6 * (size_t)nf);
        for (int f = 0; f < nf; ++f) {
            const int H = anc[f];
            const int slot = fill[H]++;
            desc[slot] = f;
            const int* lf = &fin.leaves[4 * f];
            const int* lH = &h.leaves[4 * H];
            const int D = lf[0] - lH[0];
            const double s = std::ldexp(1.0, -D);
            for (int d = 0; d < 3; ++d) {
                map[6 * (size_t)slot + 2 * d] = s;
                map[6 * (size_t)slot + 2 * d + 1] = (2.0 * lf[1 + d] + 1.0) * s - 2.0 * lH[1 + d] - 1.0;
            }
        }
        std::vector<long long> ob_off(nc + 1, 0);
        for (int H = 0; H < nc; ++H) {
            const long long n3 = (long long)(h.p[H] + 1) * (h.p[H] + 1) * (h.p[H] + 1);
            ob_off[H + 1] = ob_off[H] + n3 * n3;
        }
        L.g_desc_off = c->arena.upload(cnt, c->st);
        L.g_desc = c->arena.upload(desc, c->st);
        L.g_map = c->arena.upload(map, c->st);
        L.Ob_off = c->arena.upload(ob_off, c->st);
        L.ob_count = (size_t)ob_off.back();
        L.Ob64 = c->arena.alloc<double>(L.ob_count);
        L.Ob32 = c->arena.alloc<float>(L.ob_count);
        if (c->arena.failed) return dgi_set_error(DG_ERR_OOM, "device allocation failed (Galerkin blocks)");
    }
    LevelDev& F = c->lv[Lt];
    const size_t nv = (size_t)F.h.vqp_off.back();
    if (!F.c0_64) {
        F.c0_64 = c->arena.alloc<double>(nv);
        F.c0_32 = c->arena.alloc<float>(nv);
        if (c->arena.failed) return dgi_set_error(DG_ERR_OOM, "device allocation failed (zeroth-order term)");
    }
    c->galerkin_ready = true;
    return DG_OK;
}

// Coarse-level Galerkin blocks from the finest-level c0 (already in F.c0_64); activates the term.
int build_galerkin(dg_ctx* c) {
    const int Lt = (int)c->lv.size() - 1;
    LevelDev& F = c->lv[Lt];
    for (int l = 0; l < Lt; ++l) {
        LevelDev& L = c->lv[l];
        GalerkinArgs g{};
        g.n_coarse = L.h.n_elems();
        g.pH = L.p;
        g.Ob_off = L.Ob_off;
        g.desc_off = L.g_desc_off;
        g.desc = L.g_desc;
        g.map = L.g_map;
        g.pf = F.p;
        g.vqp_off_f = F.vqp_off;
        g.tab = c->tab64;
        g.ob_total = (long long)L.ob_count;
        g.n_vqp_f = F.h.vqp_off.back();
        g.n_desc = F.h.n_elems();
        g.chk = device_check_flag();
        CK2(launch_galerkin(g, F.c0_64, L.Ob64, L.Ob32, c->st));
        c->launches += 1;
        ++c->op_version;
        if (!L.z_active) ++c->epoch;
        L.z_active = true;
    }
    if (!F.z_active) ++c->epoch;
    F.z_active = true;
    return DG_OK;
}

void set_zeroth_active(dg_ctx* c, bool on) {
    for (auto& L : c->lv) {
        const bool v = on && (L.c0_64 != nullptr || L.Ob64 != nullptr);
        if (v != L.z_active) {
            ++c->epoch;        // kernel arguments of the captured V-cycle change
            ++c->op_version;   // assembled small-level operators are stale
        }
        L.z_active = v;
    }
}

int ensure_newton_work(dg_ctx* c) {
    if (c->nw[0]) return DG_OK;
    const size_t n = (size_t)c->lv.back().h.n_dofs();
    for (int i = 0; i < 4; ++i) c->nw[i] = c->arena.alloc<double>(n);
    if (c->arena.failed) return dgi_set_error(DG_ERR_OOM, "device allocation failed (Newton vectors)");
    return DG_OK;
}

NlArgs nl_args(dg_ctx* c) {
    LevelDev& F = c->lv.back();
    NlArgs a{};
    a.n_elems = F.h.n_elems();
    a.kind = c->nl_kind;
    a.power = c->nl_power;
    a.p = F.p;
    a.dof_off = F.dof_off;
    a.vqp_off = F.vqp_off;
    a.wdetJ = F.wdetJ;
    a.alpha = c->nl_kind == kNlPower ? c->nl_coef : c->p_alpha;
    a.beta = c->p_beta;
    a.tab = c->tab64;
    a.n_vqp = F.h.vqp_off.back();
    a.chk = device_check_flag();
    return a;
}

// R = L u - S(u) (- F for the power-law source) with the zeroth-order term
// off; optionally writes the Jacobian coefficient into the finest c0.
// Returns ||R||_2 in *rn (synchronises).
int nonlinear_residual_impl(dg_ctx* c, const double* u, double* R, bool jac, double* rn) {
    if (c->nl_kind == kNlNone)
        return dgi_set_error(DG_ERR_INVALID, "call dg_puncture_setup or dg_power_source_setup first");
    int rc = ensure_newton_work(c);
    if (rc) return rc;
    const bool was = c->lv.back().z_active;
    set_zeroth_active(c, false);
    rc = dg_apply(c, -1, DG_FP64, u, c->nw[2]);
    if (rc) return rc;
    LevelDev& F = c->lv.back();
    CK2(launch_nl(nl_args(c), u, c->nw[3], jac ? F.c0_64 : nullptr, jac ? F.c0_32 : nullptr, c->st));
    const long long n = F.h.n_dofs();
    CK2(launch_sub(c->nw[2], c->nw[3], c->nl_kind == kNlPower && c->nl_has_F ? c->nl_F : nullptr, R, n, c->st));
    c->launches += 2;
    if (!jac && was) set_zeroth_active(c, true);
    if (rn) {
        const double* a[1] = {R};
        CK2(dots<double>(a, a, 1, n, c->red, c->st));
        CK2(cudaMemcpyAsync(c->red_host, c->red.out, sizeof(double), cudaMemcpyDeviceToHost, c->st));
        CK2(cudaStreamSynchronize(c->st));
        *rn = std::sqrt(c->red_host[0]);
        c->launches += 2;
    }
    return DG_OK;
}

__global__ void negate_kernel(const double* a, double* b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = -a[i];
}

__global__ void axpy_kernel(const double* a, double* b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] += a[i];
}

inline int grid_for(long long n) {
    long long g = (n + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 2432 ? 2432 : g));
}

}  // namespace

extern "C" {

int dg_rhs(dg_ctx* c, const double* g_qp, const double* gD_qp, double* F) {
    if (!c || !F) return dgi_set_error(DG_ERR_INVALID, "NULL argument");
    LevelDev& L = c->lv.back();
    RhsArgs a{};
    a.n_elems = L.h.n_elems();
    a.p = L.p;
    a.dof_off = L.dof_off;
    a.vqp_off = L.vqp_off;
    a.wdetJ = L.wdetJ;
    a.slot_off = L.slot_off;
    a.slot_mortar = L.slot_mortar;
    a.slot_face = L.slot_face;
    a.mortars = L.mortars;
    a.mg = L.mg64;
    a.sigma = L.sigma64;
    a.tab = c->tab64;
    CK2(launch_rhs(a, g_qp, gD_qp, F, c->st));
    c->launches += 1;
    return DG_OK;
}

int dg_set_zeroth_order(dg_ctx* c, const double* coef_qp) {
    if (!c) return dgi_set_error(DG_ERR_INVALID, "NULL context");
    if (!coef_qp) {
        set_zeroth_active(c, false);
        return DG_OK;
    }
    int rc = ensure_galerkin_structure(c);
    if (rc) return rc;
    LevelDev& F = c->lv.back();
    CK2(launch_scale_coef(F.wdetJ, coef_qp, F.c0_64, F.c0_32, F.h.vqp_off.back(), c->st));
    c->launches += 1;
    return build_galerkin(c);
}

int dg_puncture_setup(dg_ctx* c, const dg_puncture_params* prm) {
    if (!c || !prm) return dgi_set_error(DG_ERR_INVALID, "NULL argument");
    if (prm->n < 1 || prm->n > 16) return dgi_set_error(DG_ERR_INVALID, "1..16 punctures");
    PunctureDev P{};
    P.n = prm->n;
    for (int i = 0; i < prm->n; ++i) {
        P.m[i] = prm->m[i];
        for (int k = 0; k < 3; ++k) {
            P.c[i][k] = prm->c[i][k];
            P.P[i][k] = prm->P[i][k];
            P.S[i][k] = prm->S[i][k];
        }
    }
    LevelDev& F = c->lv.back();
    const long long nv = F.h.vqp_off.back();
    if (!c->p_alpha) {
        c->p_alpha = c->arena.alloc<double>(nv);
        c->p_beta = c->arena.alloc<double>(nv);
        if (c->arena.failed) return dgi_set_error(DG_ERR_OOM, "device allocation failed (puncture data)");
    }
    CK2(launch_puncture(F.vxyz, nv, P, c->p_alpha, c->p_beta, c->st));
    c->launches += 1;
    c->nl_kind = kNlPuncture;
    return DG_OK;
}

int dg_power_source_setup(dg_ctx* c, const double* coef_qp, int power, const double* F) {
    if (!c || !coef_qp) return dgi_set_error(DG_ERR_INVALID, "NULL argument");
    if (power < 1 || power > 9) return dgi_set_error(DG_ERR_INVALID, "power must be in 1..9");
    LevelDev& L = c->lv.back();
    const long long nv = L.h.vqp_off.back(), n = L.h.n_dofs();
    if (!c->nl_coef) {
        c->nl_coef = c->arena.alloc<double>(nv);
        c->nl_F = c->arena.alloc<double>(n);
        if (c->arena.failed) return dgi_set_error(DG_ERR_OOM, "device allocation failed (nonlinear source)");
    }
    CK2(cudaMemcpyAsync(c->nl_coef, coef_qp, sizeof(double) * nv, cudaMemcpyDeviceToDevice, c->st));
    if (F) CK2(cudaMemcpyAsync(c->nl_F, F, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st));
    c->nl_has_F = F != nullptr;
    c->nl_power = power;
    c->nl_kind = kNlPower;
    return DG_OK;
}

int dg_puncture_residual(dg_ctx* c, const double* u, double* R) {
    if (!c || !u || !R) return dgi_set_error(DG_ERR_INVALID, "NULL argument");
    if (c->nl_kind != kNlPuncture) return dgi_set_error(DG_ERR_INVALID, "call dg_puncture_setup first");
    return nonlinear_residual_impl(c, u, R, false, nullptr);
}

int dg_nonlinear_residual(dg_ctx* c, const double* u, double* R) {
    if (!c || !u || !R) return dgi_set_error(DG_ERR_INVALID, "NULL argument");
    return nonlinear_residual_impl(c, u, R, false, nullptr);
}

int dg_newton_step(dg_ctx* c, double* u, const dg_solver_opts* o, dg_solve_stats* s, double* rn_out) {
    if (!c || !u) return dgi_set_error(DG_ERR_INVALID, "NULL argument");
    if (c->nl_kind == kNlNone)
        return dgi_set_error(DG_ERR_INVALID, "call dg_puncture_setup or dg_power_source_setup first");
    int rc = ensure_galerkin_structure(c);
    if (rc) return rc;
    if ((rc = ensure_newton_work(c))) return rc;   // c->nw[] must exist before it is passed on
    double rn = 0.0;
    rc = nonlinear_residual_impl(c, u, c->nw[0], true, &rn);   // R(u_k); Jacobian coefficient into c0
    if (rc) return rc;
    if (rn_out) *rn_out = rn;
    if ((rc = build_galerkin(c))) return rc;                    // J_R(u_k) on every level
    const long long n = c->lv.back().h.n_dofs();
    negate_kernel<<<grid_for(n), 256, 0, c->st>>>(c->nw[0], c->nw[0], n);
    CK2(cudaGetLastError() /* negate */);
    CK2(cudaMemsetAsync(c->nw[1], 0, sizeof(double) * n, c->st));
    c->launches += 1;
    rc = dg_solve(c, c->nw[0], c->nw[1], o, s);                 // J du = -R
    if (rc && rc != DG_ERR_NOT_CONVERGED) return rc;
    axpy_kernel<<<grid_for(n), 256, 0, c->st>>>(c->nw[1], u, n);
    CK2(cudaGetLastError() /* newton update */);
    c->launches += 1;
    return rc;
}

int dg_newton_solve(dg_ctx* c, double* u, double tol, int maxn, const dg_solver_opts* o, int* steps,
                    double* rn_out) {
    if (!c || !u) return dgi_set_error(DG_ERR_INVALID, "NULL argument");
    if (c->nl_kind == kNlNone)
        return dgi_set_error(DG_ERR_INVALID, "call dg_puncture_setup or dg_power_source_setup first");
    int k = 0, rc = ensure_newton_work(c);   // c->nw[] must exist before it is passed on
    if (rc) return rc;
    double rn = 0.0;
    while (true) {
        rc = nonlinear_residual_impl(c, u, c->nw[0], false, &rn);
        if (rc) return rc;
        if (!(rn >= tol) || k >= maxn) break;
        dg_solve_stats st{};
        rc = dg_newton_step(c, u, o, &st, nullptr);
        if (rc && rc != DG_ERR_NOT_CONVERGED) return rc;
        ++k;
    }
    if (steps) *steps = k;
    if (rn_out) *rn_out = rn;
    if (!std::isfinite(rn)) return dgi_set_error(DG_ERR_BREAKDOWN, "Newton residual is not finite");
    if (rn >= tol) return dgi_set_error(DG_ERR_NOT_CONVERGED, "Newton reached max steps");
    return DG_OK;
}

}  // extern "C"
