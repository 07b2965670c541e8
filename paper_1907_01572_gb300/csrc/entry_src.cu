// C ABI entry points for right-hand sides, the zeroth-order term and the
// puncture equation (Newton, Alg. 1).
#include <cmath>
#include <string>

#include "context.h"
#include "source.h"

using namespace dg;

// shares dg_last_error's buffer through this setter (defined in context.cu)
extern "C" int dgi_set_error(int code, const char* msg);

#define CK2(call)                                                                          \
    do {                                                                                   \
        cudaError_t _e = (call);                                                           \
        if (_e != cudaSuccess) return dgi_set_error(DG_ERR_CUDA, cudaGetErrorString(_e)); \
    } while (0)

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
    (void)c;
    (void)coef_qp;
    return dgi_set_error(DG_ERR_UNSUPPORTED, "zeroth-order term not built yet");
}

int dg_puncture_setup(dg_ctx* c, const dg_puncture_params* prm) {
    (void)c;
    (void)prm;
    return dgi_set_error(DG_ERR_UNSUPPORTED, "puncture source not built yet");
}

int dg_puncture_residual(dg_ctx* c, const double* u, double* R) {
    (void)c;
    (void)u;
    (void)R;
    return dgi_set_error(DG_ERR_UNSUPPORTED, "puncture source not built yet");
}

int dg_newton_step(dg_ctx* c, double* u, const dg_solver_opts* o, dg_solve_stats* s, double* rn) {
    (void)c;
    (void)u;
    (void)o;
    (void)s;
    (void)rn;
    return dgi_set_error(DG_ERR_UNSUPPORTED, "Newton not built yet");
}

int dg_newton_solve(dg_ctx* c, double* u, double tol, int maxn, const dg_solver_opts* o, int* steps, double* rn) {
    (void)c;
    (void)u;
    (void)tol;
    (void)maxn;
    (void)o;
    (void)steps;
    (void)rn;
    return dgi_set_error(DG_ERR_UNSUPPORTED, "Newton not built yet");
}

}  // extern "C"
