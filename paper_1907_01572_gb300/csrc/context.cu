// C ABI entry points (include/dgell.h): context creation, operator apply,
// smoother (Algs. 4-5), V-cycle (Alg. 3) and flexible CG (Alg. 2).
#include <chrono>
#include <cmath>
#include <cstring>
#include <algorithm>
#include <cstdlib>
#include <string>
#include <thread>
#include <unordered_map>

#include "context.h"
#include "geom.h"
#include "source.h"
#include "estimate.h"

using namespace dg;

namespace dg {
cudaError_t apply_streams_create(ApplyStreams& as) {
    as.n = 0;
    int want = kApplySideDefault;
    if (const char* e = std::getenv("DGELL_APPLY_STREAMS")) want = std::max(0, std::min(kApplySide, std::atoi(e)));
    for (int i = 0; i < want; ++i) {
        cudaError_t err = cudaStreamCreateWithFlags(&as.side[i], cudaStreamNonBlocking);
        if (err != cudaSuccess) return err;
        ++as.n;
    }
    for (int ph = 0; ph < 2; ++ph) {
        cudaError_t err = cudaEventCreateWithFlags(&as.fork[ph], cudaEventDisableTiming);
        for (int i = 0; i < want && err == cudaSuccess; ++i)
            err = cudaEventCreateWithFlags(&as.join[ph][i], cudaEventDisableTiming);
        if (err != cudaSuccess) {
            as.n = 0;   // leave the streams unused
            return err;
        }
    }
    return cudaSuccess;
}

void apply_streams_destroy(ApplyStreams& as) {
    for (int ph = 0; ph < 2; ++ph) {
        if (as.fork[ph]) cudaEventDestroy(as.fork[ph]);
        for (int i = 0; i < kApplySide; ++i)
            if (as.join[ph][i]) cudaEventDestroy(as.join[ph][i]);
    }
    for (int i = 0; i < kApplySide; ++i)
        if (as.side[i]) cudaStreamDestroy(as.side[i]);
    as = ApplyStreams{};
}

template <>
LevelView<double> level_view<double>(dg_ctx* c, int l) {
    LevelDev& L = c->lv[l];
    LevelView<double> v{};
    v.n_elems = L.h.n_elems();
    v.p = L.p;
    v.dof_off = L.dof_off;
    v.vqp_off = L.vqp_off;
    v.G = L.G64;
    v.c0 = L.z_active ? L.c0_64 : nullptr;
    v.Ob = L.z_active ? L.Ob64 : nullptr;
    v.Ob_off = L.Ob_off;
    v.slot_off = L.slot_off;
    v.slot_mortar = L.slot_mortar;
    v.slot_face = L.slot_face;
    v.slot_side = L.slot_side;
    v.mortars = L.mortars;
    v.spack = L.spack64;
    v.mg = L.mg64;
    v.sigma = L.sigma64;
    v.tab = c->tab64;
    v.ftab = c->ftab64;
    v.ft = c->ft;
    v.ob_total = (long long)L.ob_count;
    v.oriented = L.oriented;
    v.chk = device_check_flag();
    v.mt = L.mt64;
    return v;
}

template <>
LevelView<float> level_view<float>(dg_ctx* c, int l) {
    LevelDev& L = c->lv[l];
    LevelView<float> v{};
    v.n_elems = L.h.n_elems();
    v.p = L.p;
    v.dof_off = L.dof_off;
    v.vqp_off = L.vqp_off;
    v.G = L.G32;
    v.c0 = L.z_active ? L.c0_32 : nullptr;
    v.Ob = L.z_active ? L.Ob32 : nullptr;
    v.Ob_off = L.Ob_off;
    v.slot_off = L.slot_off;
    v.slot_mortar = L.slot_mortar;
    v.slot_face = L.slot_face;
    v.slot_side = L.slot_side;
    v.mortars = L.mortars;
    v.spack = L.spack32;
    v.mg = L.mg32;
    v.sigma = L.sigma32;
    v.tab = c->tab32;
    v.ftab = c->ftab32;
    v.ft = c->ft;
    v.ob_total = (long long)L.ob_count;
    v.oriented = L.oriented;
    v.chk = device_check_flag();
    v.mt = L.mt32;
    return v;
}
}  // namespace dg

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t _e = (call);                                                         \
        if (_e == cudaSuccess && debug_sync()) _e = cudaDeviceSynchronize();             \
        if (_e != cudaSuccess) return fail(DG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
        if (debug_sync()) {                                                              \
            int _f = 0;                                                                  \
            cudaMemcpy(&_f, device_check_flag(), sizeof(int), cudaMemcpyDeviceToHost);  \
            if (_f) return fail(DG_ERR_CUDA, "self-check " + std::to_string(_f) + " in " + #call); \
        }                                                                                \
    } while (0)

int resolve_level(dg_ctx* c, int level) {
    if (level < 0) level = (int)c->lv.size() - 1;
    return level;
}

template <typename T>
LevelView<T> view(dg_ctx* c, int l) {
    return level_view<T>(c, l);
}

template <typename T>
const T* tab_of(dg_ctx* c);
template <>
const double* tab_of<double>(dg_ctx* c) { return c->tab64; }
template <>
const float* tab_of<float>(dg_ctx* c) { return c->tab32; }

template <typename T>
Work<T>& work_of(LevelDev& L);
template <>
Work<double>& work_of<double>(LevelDev& L) { return L.w64; }
template <>
Work<float>& work_of<float>(LevelDev& L) { return L.w32; }


template <typename T>
int apply_t(dg_ctx* c, int l, const T* x, T* y) {
    int launches = 0;
    CK(launch_apply<T>(view<T>(c, l), c->lv[l].buckets, x, y, c->st, &launches,
                       &c->lv[l].plan[sizeof(T) == 8 ? 0 : 1], &c->as));
    c->launches += launches;
    return DG_OK;
}

// dg_apply_host: vector r is copied in on hst[0], applied on the context's
// stream and copied out on hst[1]; slot r % 2 of each direction is reused by
// vector r + 2 once its apply (input slot) and its copy out (output slot) have
// finished.  Event waits always refer to the latest record, made earlier in
// host order.
template <typename T>
int apply_host_t(dg_ctx* c, int l, int nvec, const T* hx, T* hy) {
    const long long n = c->lv[l].h.n_dofs();
    const size_t vb = sizeof(T) * (size_t)n;
    if (!c->hst[0]) {
        for (int i = 0; i < 2; ++i) CK(cudaStreamCreateWithFlags(&c->hst[i], cudaStreamNonBlocking));
        for (int s = 0; s < 2; ++s)
            for (int k = 0; k < 3; ++k) CK(cudaEventCreateWithFlags(&c->hev[s][k], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->hstart, cudaEventDisableTiming));
    }
    if (c->hstage_bytes < 4 * vb) {
        CK(cudaStreamSynchronize(c->st));   // earlier calls may still read the old slots
        if (c->hstage) CK(cudaFree(c->hstage));
        c->hstage = nullptr;
        c->hstage_bytes = 0;
        CK(cudaMalloc(&c->hstage, 4 * vb));
        c->hstage_bytes = 4 * vb;
    }
    T* dx[2] = {(T*)c->hstage, (T*)c->hstage + n};
    T* dy[2] = {(T*)c->hstage + 2 * n, (T*)c->hstage + 3 * n};
    CK(cudaEventRecord(c->hstart, c->st));   // the slots' earlier users on the context's stream
    CK(cudaStreamWaitEvent(c->hst[0], c->hstart, 0));
    CK(cudaStreamWaitEvent(c->hst[1], c->hstart, 0));
    for (int r = 0; r < nvec; ++r) {
        const int s = r & 1;
        cudaEvent_t* ev = c->hev[s];   // [copied in, applied, copied out]
        if (r >= 2) CK(cudaStreamWaitEvent(c->hst[0], ev[1], 0));
        CK(cudaMemcpyAsync(dx[s], hx + (size_t)r * n, vb, cudaMemcpyHostToDevice, c->hst[0]));
        CK(cudaEventRecord(ev[0], c->hst[0]));
        CK(cudaStreamWaitEvent(c->st, ev[0], 0));
        if (r >= 2) CK(cudaStreamWaitEvent(c->st, ev[2], 0));
        const int rc = apply_t<T>(c, l, dx[s], dy[s]);
        if (rc != DG_OK) return rc;
        CK(cudaEventRecord(ev[1], c->st));
        CK(cudaStreamWaitEvent(c->hst[1], ev[1], 0));
        CK(cudaMemcpyAsync(hy + (size_t)r * n, dy[s], vb, cudaMemcpyDeviceToHost, c->hst[1]));
        CK(cudaEventRecord(ev[2], c->hst[1]));
    }
    if (nvec > 0) CK(cudaStreamWaitEvent(c->st, c->hev[(nvec - 1) & 1][2], 0));   // copies out are in order
    return DG_OK;
}

// Small coarse levels (at most kDenseMax DOFs): the solver applies the
// assembled operator as a dense matrix-vector product -- one launch instead of
// the latency-bound element pipeline.  The SIPG part is assembled once per
// context, column by column with the matrix-free FP64 apply; the Galerkin
// zeroth-order blocks are added whenever the operator's coefficients change.
// dg_apply itself always stays matrix-free.
constexpr long long kDenseMax = 1024;

int ensure_dense(dg_ctx* c, int l) {
    LevelDev& L = c->lv[l];
    const long long n = L.h.n_dofs();
    if (n > kDenseMax || l == (int)c->lv.size() - 1) return DG_OK;
    if (L.dense64 && L.dense_version == c->op_version) return DG_OK;
    if (!L.denseL) {
        L.denseL = c->arena.alloc<double>((size_t)n * n);
        L.dense64 = c->arena.alloc<double>((size_t)n * n);
        L.dense32 = c->arena.alloc<float>((size_t)n * n);
        if (c->arena.failed) return fail(DG_ERR_OOM, "device allocation failed (small-level operator)");
        double* E = nullptr;
        CK(cudaMalloc(&E, sizeof(double) * n * n));
        std::vector<double> eye((size_t)n * n, 0.0);
        for (long long j = 0; j < n; ++j) eye[(size_t)j * n + j] = 1.0;
        CK(cudaMemcpyAsync(E, eye.data(), sizeof(double) * eye.size(), cudaMemcpyHostToDevice, c->st));
        const bool z = L.z_active;
        L.z_active = false;   // SIPG part only (restored below; not an argument change of any graph)
        for (long long j = 0; j < n; ++j) {
            int rc = apply_t<double>(c, l, E + j * n, L.denseL + j * n);
            if (rc) {
                L.z_active = z;
                cudaFree(E);
                return rc;
            }
        }
        L.z_active = z;
        CK(cudaStreamSynchronize(c->st));
        cudaFree(E);
    }
    const bool blocks = L.z_active && L.Ob64;
    CK(dense_compose(L.denseL, blocks ? L.Ob64 : nullptr, L.Ob_off, L.dof_off, L.p, L.h.n_elems(), (int)n, L.dense64,
                     L.dense32, c->st));
    c->launches += blocks ? 3 : 2;
    L.dense_version = c->op_version;
    return DG_OK;
}

template <typename T>
const T* dense_of(LevelDev& L);
template <>
const double* dense_of<double>(LevelDev& L) { return L.dense64; }
template <>
const float* dense_of<float>(LevelDev& L) { return L.dense32; }

template <typename T>
int solver_apply(dg_ctx* c, int l, const T* x, T* y) {
    LevelDev& L = c->lv[l];
    if (L.dense64 && L.dense_version == c->op_version) {
        CK(dense_matvec_t<T>(dense_of<T>(L), x, y, (int)L.h.n_dofs(), c->st));
        c->launches += 1;
        return DG_OK;
    }
    return apply_t<T>(c, l, x, y);
}

template <typename T>
int ensure_work(dg_ctx* c, int l) {
    Work<T>& W = work_of<T>(c->lv[l]);
    if (W.ready) return DG_OK;
    const size_t n = (size_t)c->lv[l].h.n_dofs();
    W.f = c->arena.alloc<T>(n);
    W.v = c->arena.alloc<T>(n);
    W.r = c->arena.alloc<T>(n);
    W.p = c->arena.alloc<T>(n);
    W.Ap = c->arena.alloc<T>(n);
    W.t = c->arena.alloc<T>(n);
    W.sm = c->arena.alloc<SmState>(1);
    if (c->arena.failed) return fail(DG_ERR_OOM, "device allocation failed (solver workspace)");
    W.ready = true;
    return DG_OK;
}

void cheb_defaults(const dg_cheb_opts* o, int& ne, int& nc, double& Lam, double& scale, double& fixed) {
    fixed = (o && o->lam_fixed > 0) ? o->lam_fixed : 0.0;
    ne = fixed > 0 ? 0 : ((o && o->n_eigs > 0) ? o->n_eigs : 15);
    nc = (o && o->n_cheb > 0) ? o->n_cheb : 15;
    Lam = (o && o->Lambda > 0) ? o->Lambda : 20.0;
    scale = (o && o->lam_scale > 0) ? o->lam_scale : 1.0;
    if (nc > kMaxCheb) nc = kMaxCheb;
}

// Alg. 4 with Alg. 5: smooths J x = b in place on level l.
template <typename T>
int smooth_t(dg_ctx* c, int l, const T* b, T* x, const dg_cheb_opts* o) {
    int rc = ensure_work<T>(c, l);
    if (rc) return rc;
    if ((rc = ensure_dense(c, l))) return rc;
    int ne, nc;
    double Lam, scale, fixed;
    cheb_defaults(o, ne, nc, Lam, scale, fixed);
    Work<T>& W = work_of<T>(c->lv[l]);
    const long long n = c->lv[l].h.n_dofs();
    cudaStream_t st = c->st;
    if ((rc = solver_apply<T>(c, l, x, W.Ap))) return rc;
    CK(residual_init<T>(b, W.Ap, W.r, W.p, n, c->red, st));
    CK(sm_init(W.sm, c->red.out, st));
    c->launches += 3;
    for (int k = 0; k < ne; ++k) {
        if ((rc = solver_apply<T>(c, l, W.p, W.Ap))) return rc;
        CK(cg_alpha_fused<T>(W.sm, W.p, W.Ap, n, c->red, st));
        CK(cg_update_fused<T>(W.sm, x, W.r, W.p, W.Ap, n, c->red, st));
        CK(cg_p_update<T>(W.sm, W.p, W.r, n, st));
        c->launches += 3;
    }
    CK(sm_cheb_coeffs(W.sm, nc, Lam, scale, fixed, st));
    CK(cudaMemsetAsync(W.p, 0, n * sizeof(T), st));
    c->launches += 1;
    for (int k = 0; k < nc; ++k) {
        if ((rc = solver_apply<T>(c, l, x, W.Ap))) return rc;
        CK(cheb_step<T>(W.sm, k, b, W.Ap, W.p, x, n, st));
        c->launches += 1;
    }
    return DG_OK;
}

// y = blockdiag(J_ee) x: the apply with each mortar's other-side trace taken as 0.
template <typename T>
int apply_bdiag_t(dg_ctx* c, int l, const T* x, T* y) {
    int launches = 0;
    LevelView<T> v = view<T>(c, l);
    v.bdiag = 1;
    CK(launch_apply<T>(v, c->lv[l].buckets, x, y, c->st, &launches, &c->lv[l].plan[sizeof(T) == 8 ? 0 : 1],
                       &c->as));
    c->launches += launches;
    return DG_OK;
}

// Alg. 6 (Schwarz smoother) with element subdomains and no overlap: cycles of
// r = b - J x, element-local CG on J_ee dx_e = r_e for all elements at once
// (relative tolerance local_tol, at most local_iters steps), x += omega dx.
template <typename T>
int smooth_schwarz_t(dg_ctx* c, int l, const T* b, T* x, const dg_mg_opts* o) {
    int rc = ensure_work<T>(c, l);
    if (rc) return rc;
    if ((rc = ensure_dense(c, l))) return rc;
    LevelDev& L = c->lv[l];
    const int ne = L.h.n_elems();
    if (!L.schwarz_es) {
        L.schwarz_es = c->arena.alloc<double>(3 * (size_t)ne);
        if (c->arena.failed) return fail(DG_ERR_OOM, "device allocation failed (Schwarz smoother)");
    }
    const int ns = o->n_schwarz > 0 ? o->n_schwarz : 3;
    const int K = o->local_iters > 0 ? o->local_iters : 20;
    const double tol = o->local_tol > 0 ? o->local_tol : 1e-3;
    const double om = o->schwarz_omega > 0 ? o->schwarz_omega : 0.7;
    Work<T>& W = work_of<T>(L);
    const long long n = L.h.n_dofs();
    cudaStream_t st = c->st;
    for (int s = 0; s < ns; ++s) {
        if ((rc = solver_apply<T>(c, l, x, W.Ap))) return rc;
        CK(sub3<T>(b, W.Ap, W.r, n, st));
        CK(elem_cg_init<T>(W.r, W.p, W.t, L.dof_off, ne, L.schwarz_es, st));
        c->launches += 2;
        for (int k = 0; k < K; ++k) {
            if ((rc = apply_bdiag_t<T>(c, l, W.p, W.Ap))) return rc;
            CK(elem_cg_alpha<T>(W.p, W.Ap, L.dof_off, ne, L.schwarz_es, tol * tol, st));
            CK(elem_cg_update<T>(W.t, W.r, W.p, W.Ap, L.dof_off, ne, L.schwarz_es, st));
            c->launches += 2;
        }
        CK(axpby<T>((T)om, W.t, (T)1, x, n, st));
        c->launches += 1;
    }
    return DG_OK;
}

template <typename T>
TransferView<T> tview(dg_ctx* c, int lc) {
    LevelDev& H = c->lv[lc];
    LevelDev& h = c->lv[lc + 1];
    TransferView<T> t{};
    t.n_coarse = H.h.n_elems();
    t.n_fine = h.h.n_elems();
    t.pH = H.p;
    t.ph = h.p;
    t.dofH = H.dof_off;
    t.dofh = h.dof_off;
    t.child_off = H.child_off;
    t.child_id = H.child_id;
    t.child_bits = H.child_bits;
    t.fine_parent = H.fine_parent;
    t.fine_bits = H.fine_bits;
    t.tab = tab_of<T>(c);
    return t;
}

// Inverse of the symmetric part of the column-major n x n matrix h: Cholesky
// L L^T, then the inverse column by column.  False if it is not positive definite.
bool spd_inverse(const std::vector<double>& h, int n, std::vector<double>& inv) {
    std::vector<double> M((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) M[(size_t)i * n + j] = 0.5 * (h[(size_t)i * n + j] + h[(size_t)j * n + i]);
    std::vector<double> Lc((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double s = M[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= Lc[(size_t)j * n + k] * Lc[(size_t)j * n + k];
        if (!(s > 0.0)) return false;
        const double djj = std::sqrt(s);
        Lc[(size_t)j * n + j] = djj;
        for (int i = j + 1; i < n; ++i) {
            double t = M[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= Lc[(size_t)i * n + k] * Lc[(size_t)j * n + k];
            Lc[(size_t)i * n + j] = t / djj;
        }
    }
    inv.assign((size_t)n * n, 0.0);
    std::vector<double> z(n);
    for (int col = 0; col < n; ++col) {
        for (int i = 0; i < n; ++i) {
            double t = (i == col) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) t -= Lc[(size_t)i * n + k] * z[k];
            z[i] = t / Lc[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double t = z[i];
            for (int k = i + 1; k < n; ++k) t -= Lc[(size_t)k * n + i] * inv[(size_t)col * n + k];
            inv[(size_t)col * n + i] = t / Lc[(size_t)i * n + i];
        }
    }
    return true;
}

// coarse-grid solve support: dense inverse of the level-0 operator (FP64),
// assembled column by column with the matrix-free apply.
// Dense inverse of the level-0 operator for the exact coarse solve, rebuilt
// whenever the operator's coefficients change (a new zeroth-order term, e.g.
// every Newton step).
int ensure_coarse_inverse(dg_ctx* c) {
    if (c->coarse_ready && c->coarse_version == c->op_version) return DG_OK;
    const int n = (int)c->lv[0].h.n_dofs();
    if (n > 4096) return fail(DG_ERR_UNSUPPORTED, "coarse Cholesky needs level 0 with at most 4096 dofs");
    double* E = nullptr;
    double* A = nullptr;
    CK(cudaMalloc(&E, sizeof(double) * n * (size_t)n));
    CK(cudaMalloc(&A, sizeof(double) * n * (size_t)n));
    std::vector<double> h((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) h[(size_t)i * n + i] = 1.0;
    CK(cudaMemcpyAsync(E, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, c->st));
    for (int j = 0; j < n; ++j) {
        int rc = apply_t<double>(c, 0, E + (size_t)j * n, A + (size_t)j * n);
        if (rc) return rc;
    }
    CK(cudaMemcpyAsync(h.data(), A, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    cudaFree(E);
    cudaFree(A);
    std::vector<double> inv;
    if (!spd_inverse(h, n, inv)) return fail(DG_ERR_BREAKDOWN, "level-0 operator is not positive definite");
    if (!c->coarse_inv) c->coarse_inv = c->arena.alloc<double>((size_t)n * n);   // level 0's size never changes
    if (!c->coarse_inv) return fail(DG_ERR_OOM, "device allocation failed (coarse inverse)");
    CK(cudaMemcpyAsync(c->coarse_inv, inv.data(), sizeof(double) * inv.size(), cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->coarse_n = n;
    c->coarse_ready = true;
    c->coarse_version = c->op_version;
    return DG_OK;
}

// Alg. 6 with overlapping subdomains (defined below, after the geometry helpers).
template <typename T>
int smooth_overlap_t(dg_ctx* c, int l, const T* b, T* x, const dg_mg_opts* o);

// Alg. 3: v = VCYCLE(f) on the finest level.
template <typename T>
int vcycle_t(dg_ctx* c, const T* f, T* v, const dg_mg_opts* o) {
    const int Lt = (int)c->lv.size() - 1;
    cudaStream_t st = c->st;
    int rc;
    for (int l = 0; l <= Lt; ++l)
        if ((rc = ensure_work<T>(c, l))) return rc;
    if (o && o->coarse == 1 && (rc = ensure_coarse_inverse(c))) return rc;
    const dg_cheb_opts* co = o ? &o->cheb : nullptr;
    auto smooth = [&](int l, const T* b, T* x) {
        if (o && o->smoother == 2) return smooth_overlap_t<T>(c, l, b, x, o);
        return (o && o->smoother == 1) ? smooth_schwarz_t<T>(c, l, b, x, o) : smooth_t<T>(c, l, b, x, co);
    };
    auto F = [&](int l) -> const T* { return l == Lt ? f : work_of<T>(c->lv[l]).f; };
    auto V = [&](int l) -> T* { return l == Lt ? v : work_of<T>(c->lv[l]).v; };
    for (int l = Lt; l >= 1; --l) {
        const long long n = c->lv[l].h.n_dofs();
        Work<T>& W = work_of<T>(c->lv[l]);
        CK(cudaMemsetAsync(V(l), 0, n * sizeof(T), st));
        if ((rc = smooth(l, F(l), V(l)))) return rc;
        if ((rc = solver_apply<T>(c, l, V(l), W.t))) return rc;
        CK(sub3<T>(F(l), W.t, W.r, n, st));
        CK(launch_restrict<T>(tview<T>(c, l - 1), W.r, work_of<T>(c->lv[l - 1]).f, st));
        c->launches += 2;
    }
    {
        const long long n0 = c->lv[0].h.n_dofs();
        if (o && o->coarse == 1) {
            CK(dense_matvec<T>(c->coarse_inv, F(0), V(0), (int)n0, st));
            c->launches += 1;
        } else {
            CK(cudaMemsetAsync(V(0), 0, n0 * sizeof(T), st));
            if ((rc = smooth(0, F(0), V(0)))) return rc;
        }
    }
    for (int l = 1; l <= Lt; ++l) {
        CK(launch_prolong_add<T>(tview<T>(c, l - 1), V(l - 1), V(l), st));
        c->launches += 1;
        if ((rc = smooth(l, F(l), V(l)))) return rc;
    }
    return DG_OK;
}

bool same_opts(const dg_mg_opts& a, const dg_mg_opts* b) {
    const dg_mg_opts z{};
    const dg_mg_opts& bb = b ? *b : z;
    return a.coarse == bb.coarse && a.cheb.n_eigs == bb.cheb.n_eigs && a.cheb.n_cheb == bb.cheb.n_cheb &&
           a.cheb.Lambda == bb.cheb.Lambda && a.cheb.lam_scale == bb.cheb.lam_scale &&
           a.cheb.lam_fixed == bb.cheb.lam_fixed && a.smoother == bb.smoother &&
           a.n_schwarz == bb.n_schwarz && a.local_iters == bb.local_iters && a.local_tol == bb.local_tol &&
           a.schwarz_omega == bb.schwarz_omega;
}

// The V-cycle of one FCG iteration (FP64: r -> v; FP32: fcg32[0] -> fcg32[1]).
// graph_mode 0 on a non-default stream: the first call for a given precision /
// options / argument epoch runs eagerly (allocations, attributes) and then
// captures the same launch sequence into a CUDA graph; later calls replay it.
int vcycle_maybe_graph(dg_ctx* c, int prec, double* r, double* v, const dg_mg_opts* mo, int graph_mode) {
    auto eager = [&]() -> int {
        if (prec == DG_FP32) return vcycle_t<float>(c, c->fcg32[0], c->fcg32[1], mo);
        return vcycle_t<double>(c, r, v, mo);
    };
    if (graph_mode != 0 || c->st == nullptr) return eager();
    if (c->vgraph && c->vgraph_prec == prec && c->vgraph_epoch == c->epoch && c->vgraph_opver == c->op_version &&
        same_opts(c->vgraph_opts, mo)) {
        CK(cudaGraphLaunch(c->vgraph, c->st));
        c->launches += c->vgraph_launches;
        return DG_OK;
    }
    int rc = eager();
    if (rc) return rc;
    if (c->vgraph) {
        cudaGraphExecDestroy(c->vgraph);
        c->vgraph = nullptr;
    }
    const long long before = c->launches;
    CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
    rc = eager();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->st, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(DG_ERR_CUDA, std::string("V-cycle graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->vgraph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->vgraph = nullptr;
        return fail(DG_ERR_CUDA, std::string("V-cycle graph instantiate: ") + cudaGetErrorString(e));
    }
    c->vgraph_launches = c->launches - before;
    c->launches = before;   // captured, not executed
    c->vgraph_prec = prec;
    c->vgraph_epoch = c->epoch;
    c->vgraph_opver = c->op_version;
    c->vgraph_opts = mo ? *mo : dg_mg_opts{};
    return DG_OK;
}

GeomArgs geom_args(dg_ctx* c, const LevelDev& L) {
    GeomArgs g{};
    g.n_elems = L.h.n_elems();
    g.leaves = L.leaves;
    g.p = L.p;
    g.dof_off = L.dof_off;
    g.vqp_off = L.vqp_off;
    g.tab = c->tab64;
    for (int d = 0; d < 3; ++d) {
        g.lo[d] = c->desc.lo[d];
        g.hi[d] = c->desc.hi[d];
        g.warp_k[d] = c->desc.warp_k[d];
    }
    g.map_kind = c->desc.map_kind;
    g.warp_amp = c->desc.warp_amp;
    g.n_blocks = (int)c->blocks.size();
    g.blocks = c->blocks_dev;
    g.block = L.block;
    return g;
}

// ---- Alg. 6 with overlapping subdomains --------------------------------------
// Subdomain of element e_c: its own nodes plus every other element's node at
// the position of one of e_c's boundary nodes (the touching elements'
// coinciding DG nodes: one overlap layer, of zero width).  A node's weight is
// w_h of eq. (schwarz_weight) at vanishing overlap width, evaluated at the
// e_c node it sits on: 1 inside, 1/2 on a face, 1/4 on an edge, 1/8 on a
// corner.  The local operator R_s J R_s^T is read off the level operator's
// element blocks, which are probed with the matrix-free FP64 apply (elements
// three or more faces apart share a probe), and inverted exactly.  Levels with
// one degree and conforming faces only.
struct CellKey {
    long long i, j, k;
    bool operator==(const CellKey& o) const { return i == o.i && j == o.j && k == o.k; }
};
struct CellHash {
    size_t operator()(const CellKey& c) const {
        return (size_t)(c.i * 73856093LL) ^ (size_t)(c.j * 19349663LL) ^ (size_t)(c.k * 83492791LL);
    }
};

int ensure_overlap(dg_ctx* c, int l) {
    LevelDev& L = c->lv[l];
    if (L.ovl_version == c->op_version) return DG_OK;
    const LevelHost& h = L.h;
    const int ne = h.n_elems();
    const int pdeg = h.p[0];
    for (int e = 0; e < ne; ++e)
        if (h.p[e] != pdeg)
            return fail(DG_ERR_UNSUPPORTED, "overlapping Schwarz subdomains need one degree on every element of a level");
    std::vector<std::vector<int>> nbr(ne);
    for (const Mortar& m : h.mortars) {
        if (m.eB < 0) continue;
        if (h.leaves[4 * m.eA] != h.leaves[4 * m.eB])
            return fail(DG_ERR_UNSUPPORTED, "overlapping Schwarz subdomains need conforming faces (no 2:1 faces)");
        nbr[m.eA].push_back(m.eB);
        nbr[m.eB].push_back(m.eA);
    }
    const int n = pdeg + 1, n3 = n * n * n;
    const long long N = h.n_dofs();
    const std::vector<long long>& off = h.dof_off;
    auto elem_of = [&](long long d) { return (int)(std::upper_bound(off.begin(), off.end(), d) - off.begin()) - 1; };
    auto nbound = [&](int k) {
        const int ix[3] = {k % n, (k / n) % n, k / (n * n)};
        int b = 0;
        for (int a = 0; a < 3; ++a) b += (ix[a] == 0 || ix[a] == n - 1);
        return b;
    };
    const bool first = (L.sub_off == nullptr);
    std::vector<long long> sub_off, sub_dof;
    std::vector<double> wts;
    if (first) {
        // node positions
        std::vector<double> X(3 * (size_t)N);
        double* Xd = nullptr;
        CK(cudaMalloc(&Xd, sizeof(double) * 3 * (size_t)N));
        cudaError_t ce = launch_node_coords(geom_args(c, L), Xd, c->st);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(X.data(), Xd, sizeof(double) * X.size(), cudaMemcpyDeviceToHost, c->st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->st);
        cudaFree(Xd);
        if (ce != cudaSuccess) return fail(DG_ERR_CUDA, std::string("overlap subdomains: ") + cudaGetErrorString(ce));
        auto pos = [&](long long d, double P[3]) {
            const int e = elem_of(d);
            const long long k = d - off[e];
            for (int a = 0; a < 3; ++a) P[a] = X[3 * off[e] + a * n3 + k];
        };
        double xmax = 1.0;
        for (double v : X) xmax = std::max(xmax, std::fabs(v));
        const double q = 1e-9 * xmax;   // cell size of the position hash
        auto cell = [&](const double P[3]) {
            return CellKey{(long long)std::floor(P[0] / q), (long long)std::floor(P[1] / q), (long long)std::floor(P[2] / q)};
        };
        std::vector<int> bnd;   // boundary nodes of an element
        for (int k = 0; k < n3; ++k)
            if (nbound(k) > 0) bnd.push_back(k);
        std::unordered_map<CellKey, std::vector<long long>, CellHash> cells;
        for (int e = 0; e < ne; ++e)
            for (int k : bnd) {
                double P[3];
                pos(off[e] + k, P);
                cells[cell(P)].push_back(off[e] + k);
            }
        sub_off.push_back(0);
        for (int e = 0; e < ne; ++e) {
            for (int k = 0; k < n3; ++k) {
                sub_dof.push_back(off[e] + k);
                wts.push_back(std::ldexp(1.0, -nbound(k)));
            }
            std::vector<std::pair<long long, int>> contact;   // (global DOF, e_c node it sits on)
            for (int k : bnd) {
                double P[3];
                pos(off[e] + k, P);
                const double tol = 1e-9 * std::max(1.0, std::sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]));
                const CellKey c0 = cell(P);
                for (int di = -1; di <= 1; ++di)
                    for (int dj = -1; dj <= 1; ++dj)
                        for (int dk = -1; dk <= 1; ++dk) {
                            auto it = cells.find(CellKey{c0.i + di, c0.j + dj, c0.k + dk});
                            if (it == cells.end()) continue;
                            for (long long d : it->second) {
                                if (d >= off[e] && d < off[e] + n3) continue;
                                double Q[3];
                                pos(d, Q);
                                const double dx = Q[0] - P[0], dy = Q[1] - P[1], dz = Q[2] - P[2];
                                if (std::sqrt(dx * dx + dy * dy + dz * dz) <= tol) contact.push_back({d, k});
                            }
                        }
            }
            std::sort(contact.begin(), contact.end());
            for (const auto& ct : contact) {
                sub_dof.push_back(ct.first);
                wts.push_back(std::ldexp(1.0, -nbound(ct.second)));
            }
            sub_off.push_back((long long)sub_dof.size());
        }
    } else {   // the subdomains stay; only the operator changed
        sub_off.resize(ne + 1);
        CK(cudaMemcpyAsync(sub_off.data(), L.sub_off, sizeof(long long) * (ne + 1), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        sub_dof.resize(sub_off.back());
        CK(cudaMemcpyAsync(sub_dof.data(), L.sub_dof, sizeof(long long) * sub_dof.size(), cudaMemcpyDeviceToHost,
                           c->st));
        CK(cudaStreamSynchronize(c->st));
    }
    const long long E = sub_off.back();
    int max_m = 0;
    long long inv_total = 0;
    std::vector<long long> inv_off(ne + 1, 0);
    for (int e = 0; e < ne; ++e) {
        const long long m = sub_off[e + 1] - sub_off[e];
        max_m = std::max(max_m, (int)m);
        inv_off[e + 1] = inv_off[e] + m * m;
    }
    inv_total = inv_off[ne];
    if ((double)inv_total * 12.0 > 8e9)
        return fail(DG_ERR_UNSUPPORTED, "overlapping Schwarz: local inverses would take more than 8 GB");
    // element blocks J(e2, e) for e2 = e and its face neighbours (column-major n3 x n3:
    // row = node of e2, column = node of e), probed colour by colour: a colour holds
    // elements at least three faces apart, so their columns do not overlap
    std::vector<int> color(ne, -1), mark(ne + 1, -1);
    int ncol = 0;
    for (int e = 0; e < ne; ++e) {
        std::vector<char> used;
        auto forbid = [&](int x) {
            if (color[x] >= 0) {
                if ((int)used.size() <= color[x]) used.resize(color[x] + 1, 0);
                used[color[x]] = 1;
            }
        };
        for (int a : nbr[e]) {
            forbid(a);
            for (int b2 : nbr[a]) forbid(b2);
        }
        int cc = 0;
        while (cc < (int)used.size() && used[cc]) ++cc;
        color[e] = cc;
        ncol = std::max(ncol, cc + 1);
    }
    std::unordered_map<long long, size_t> boff;
    size_t nblk = 0;
    for (int e = 0; e < ne; ++e) {
        boff[(long long)e * ne + e] = (nblk++) * (size_t)n3 * n3;
        for (int a : nbr[e]) boff[(long long)a * ne + e] = (nblk++) * (size_t)n3 * n3;
    }
    if ((double)nblk * n3 * n3 * 8.0 > 8e9)
        return fail(DG_ERR_UNSUPPORTED, "overlapping Schwarz: element blocks would take more than 8 GB of host memory");
    std::vector<double> blk(nblk * (size_t)n3 * n3);
    {
        std::vector<std::vector<int>> by_color(ncol);
        for (int e = 0; e < ne; ++e) by_color[color[e]].push_back(e);
        double *xd = nullptr, *yd = nullptr;
        if (cudaMalloc(&xd, sizeof(double) * N) != cudaSuccess || cudaMalloc(&yd, sizeof(double) * N) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(xd);
            return fail(DG_ERR_OOM, "device allocation failed (overlap probes)");
        }
        std::vector<double> xh(N, 0.0), yh(N);
        int rc = DG_OK;
        cudaError_t ce = cudaSuccess;
        for (int cc = 0; cc < ncol && rc == DG_OK && ce == cudaSuccess; ++cc)
            for (int a = 0; a < n3 && rc == DG_OK && ce == cudaSuccess; ++a) {
                for (int e : by_color[cc]) xh[off[e] + a] = 1.0;
                ce = cudaMemcpyAsync(xd, xh.data(), sizeof(double) * N, cudaMemcpyHostToDevice, c->st);
                if (ce == cudaSuccess) rc = apply_t<double>(c, l, xd, yd);
                if (ce == cudaSuccess && rc == DG_OK)
                    ce = cudaMemcpyAsync(yh.data(), yd, sizeof(double) * N, cudaMemcpyDeviceToHost, c->st);
                if (ce == cudaSuccess && rc == DG_OK) ce = cudaStreamSynchronize(c->st);
                for (int e : by_color[cc]) {
                    xh[off[e] + a] = 0.0;
                    auto put = [&](int e2) {
                        double* B = &blk[boff[(long long)e2 * ne + e]];
                        for (int i = 0; i < n3; ++i) B[i + (size_t)a * n3] = yh[off[e2] + i];
                    };
                    put(e);
                    for (int e2 : nbr[e]) put(e2);
                }
            }
        cudaFree(xd);
        cudaFree(yd);
        if (rc != DG_OK) return rc;
        if (ce != cudaSuccess) return fail(DG_ERR_CUDA, std::string("overlap blocks: ") + cudaGetErrorString(ce));
    }
    // local operators and their inverses, subdomains split over the host cores
    std::vector<double> inv(inv_total);
    std::vector<int> bad(ne, 0);
    auto work = [&](int e0, int e1) {
        std::vector<double> A, Ai;
        for (int e = e0; e < e1; ++e) try {
            const long long o = sub_off[e];
            const int m = (int)(sub_off[e + 1] - o);
            std::vector<int> el(m), lo(m);
            for (int j = 0; j < m; ++j) {
                el[j] = elem_of(sub_dof[o + j]);
                lo[j] = (int)(sub_dof[o + j] - off[el[j]]);
            }
            // runs of entries on one element (own nodes first, then contacts by DOF)
            std::vector<int> run0;
            for (int j = 0; j < m; ++j)
                if (j == 0 || el[j] != el[j - 1]) run0.push_back(j);
            run0.push_back(m);
            A.assign((size_t)m * m, 0.0);
            for (size_t rk = 0; rk + 1 < run0.size(); ++rk)
                for (size_t rj = 0; rj + 1 < run0.size(); ++rj) {
                    auto it = boff.find((long long)el[run0[rj]] * ne + el[run0[rk]]);
                    if (it == boff.end()) continue;
                    const double* B = &blk[it->second];
                    for (int k = run0[rk]; k < run0[rk + 1]; ++k)
                        for (int j = run0[rj]; j < run0[rj + 1]; ++j)
                            A[(size_t)k * m + j] = B[lo[j] + (size_t)lo[k] * n3];
                }
            if (!spd_inverse(A, m, Ai)) {
                bad[e] = 1;
                continue;
            }
            std::copy(Ai.begin(), Ai.end(), inv.begin() + inv_off[e]);
        } catch (...) {   // host allocation failure: reported below, never thrown out of the thread
            bad[e] = 2;
        }
    };
    {
        const int nt = std::max(1, std::min((int)std::thread::hardware_concurrency(), 32));
        std::vector<std::thread> th;
        for (int t = 0; t < nt; ++t) {
            const int e0 = (int)((long long)ne * t / nt), e1 = (int)((long long)ne * (t + 1) / nt);
            try {
                th.emplace_back(work, e0, e1);
            } catch (...) {   // no thread to be had: this share runs here
                work(e0, e1);
            }
        }
        for (auto& t : th) t.join();
    }
    for (int e = 0; e < ne; ++e) {
        if (bad[e] == 2) return fail(DG_ERR_OOM, "overlapping Schwarz: host allocation failed");
        if (bad[e]) return fail(DG_ERR_BREAKDOWN, "overlapping Schwarz: a local operator is not positive definite");
    }
    std::vector<float> inv32(inv.begin(), inv.end());
    Arena& Ar = c->arena;
    if (first) {
        // per global DOF, the subdomain entries that hold it, in entry order
        std::vector<long long> cof_off(N + 1, 0), cof(E);
        for (long long t = 0; t < E; ++t) ++cof_off[sub_dof[t] + 1];
        for (long long i = 0; i < N; ++i) cof_off[i + 1] += cof_off[i];
        std::vector<long long> fill(cof_off.begin(), cof_off.end() - 1);
        for (long long t = 0; t < E; ++t) cof[fill[sub_dof[t]]++] = t;
        std::vector<float> w32(wts.begin(), wts.end());
        L.sub_off = Ar.upload(sub_off, c->st);
        L.sub_dof = Ar.upload(sub_dof, c->st);
        L.inv_off = Ar.upload(inv_off, c->st);
        L.ovl_cof_off = Ar.upload(cof_off, c->st);
        L.ovl_cof = Ar.upload(cof, c->st);
        L.ovl_w64 = Ar.upload(wts, c->st);
        L.ovl_w32 = Ar.upload(w32, c->st);
        L.ovl_inv64 = Ar.alloc<double>(inv_total);
        L.ovl_inv32 = Ar.alloc<float>(inv_total);
        L.ovl_u64 = Ar.alloc<double>(E);
        L.ovl_u32 = Ar.alloc<float>(E);
        if (Ar.failed) return fail(DG_ERR_OOM, "device allocation failed (overlapping Schwarz)");
        L.ovl_max_m = max_m;
        CK(cudaStreamSynchronize(c->st));   // the host vectors above go out of scope
    }
    CK(cudaMemcpyAsync(L.ovl_inv64, inv.data(), sizeof(double) * inv.size(), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(L.ovl_inv32, inv32.data(), sizeof(float) * inv32.size(), cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    L.ovl_version = c->op_version;
    return DG_OK;
}

template <typename T>
const T* ovl_w(const LevelDev& L);
template <>
const double* ovl_w<double>(const LevelDev& L) { return L.ovl_w64; }
template <>
const float* ovl_w<float>(const LevelDev& L) { return L.ovl_w32; }
template <typename T>
const T* ovl_inv(const LevelDev& L);
template <>
const double* ovl_inv<double>(const LevelDev& L) { return L.ovl_inv64; }
template <>
const float* ovl_inv<float>(const LevelDev& L) { return L.ovl_inv32; }
template <typename T>
T* ovl_u(LevelDev& L);
template <>
double* ovl_u<double>(LevelDev& L) { return L.ovl_u64; }
template <>
float* ovl_u<float>(LevelDev& L) { return L.ovl_u32; }

// Alg. 6 with overlapping subdomains: n_schwarz cycles of r = b - J x,
// x += sum_s R_s^T W_s (R_s J R_s^T)^-1 R_s r.
template <typename T>
int smooth_overlap_t(dg_ctx* c, int l, const T* b, T* x, const dg_mg_opts* o) {
    int rc = ensure_work<T>(c, l);
    if (rc) return rc;
    if ((rc = ensure_dense(c, l))) return rc;
    if ((rc = ensure_overlap(c, l))) return rc;
    LevelDev& L = c->lv[l];
    const int ns = o->n_schwarz > 0 ? o->n_schwarz : 3;
    Work<T>& W = work_of<T>(L);
    const long long n = L.h.n_dofs();
    cudaStream_t st = c->st;
    for (int s = 0; s < ns; ++s) {
        if ((rc = solver_apply<T>(c, l, x, W.Ap))) return rc;
        CK(sub3<T>(b, W.Ap, W.r, n, st));
        CK(ovl_local<T>(L.sub_off, L.sub_dof, ovl_w<T>(L), L.inv_off, ovl_inv<T>(L), W.r, ovl_u<T>(L), L.h.n_elems(),
                        L.ovl_max_m, st));
        CK(ovl_gather<T>(L.ovl_cof_off, L.ovl_cof, ovl_u<T>(L), x, n, st));
        c->launches += 3;
    }
    return DG_OK;
}

int upload_level(dg_ctx* c, LevelDev& L, int li, std::string& err) {
    Arena& A = c->arena;
    cudaStream_t st = c->st;
    LevelHost& h = L.h;
    L.leaves = A.upload(h.leaves, st);
    L.block = A.upload(h.block, st);
    L.p = A.upload(h.p, st);
    L.dof_off = A.upload(h.dof_off, st);
    L.vqp_off = A.upload(h.vqp_off, st);
    L.mortars = A.upload(h.mortars, st);
    L.oriented = 0;
    for (const Mortar& m : h.mortars)
        if (m.orient) L.oriented = 1;
    L.slot_off = A.upload(h.slot_off, st);
    L.slot_mortar = A.upload(h.slot_mortar, st);
    L.slot_face = A.upload(h.slot_face, st);
    L.slot_side = A.upload(h.slot_side, st);
    for (int n = kMinN; n <= kMaxN; ++n) {
        BucketInfo& b = L.buckets[n];
        b.count = (int)h.buckets[n].size();
        b.elems = b.count ? A.upload(h.buckets[n], st) : nullptr;
        std::vector<ElemDesc> ed;
        for (int e : h.buckets[n]) ed.push_back(ElemDesc{h.dof_off[e], h.vqp_off[e], e, h.slot_off[e], h.slot_off[e + 1], 0});
        b.desc = b.count ? A.upload(ed, st) : nullptr;
        b.max_q = 2;
        b.max_nb = 2;
        for (int e : h.buckets[n])
            for (int s = h.slot_off[e]; s < h.slot_off[e + 1]; ++s) {
                const Mortar& m = h.mortars[h.slot_mortar[s]];
                b.max_q = std::max(b.max_q, (int)m.q);
                const int o = h.slot_side[s] == 0 ? m.eB : m.eA;
                if (o >= 0) b.max_nb = std::max(b.max_nb, h.p[o] + 1);
            }
    }
    if (li + 1 < (int)c->lv.size()) {
        L.child_off = A.upload(h.child_off, st);
        L.child_id = A.upload(h.child_id, st);
        L.child_bits = A.upload(h.child_bits, st);
        L.fine_parent = A.upload(h.fine_parent, st);
        L.fine_bits = A.upload(h.fine_bits, st);
    }
    const long long nv = h.vqp_off.back(), nd = h.n_dofs(), nm = h.n_mortar_pts, nb = h.n_bnd_pts;
    const int nmort = (int)h.mortars.size();
    L.G64 = A.alloc<double>(6 * nv);
    L.wdetJ = A.alloc<double>(nv);
    L.vxyz = A.alloc<double>(3 * nv);
    L.mg64 = A.alloc<double>(7 * nm);
    L.sigma64 = A.alloc<double>(nmort);
    L.bxyz = A.alloc<double>(3 * nb);
    L.G32 = A.alloc<float>(6 * nv);
    L.mg32 = A.alloc<float>(7 * nm);
    L.mt64 = A.alloc<double>(4 * nm);
    L.mt32 = A.alloc<float>(4 * nm);
    L.sigma32 = A.alloc<float>(nmort);
    {   // slot records (sigma filled in after the mortar geometry)
        std::vector<SlotPack<double>> sp(h.slot_mortar.size());
        for (size_t s = 0; s < sp.size(); ++s) {
            const Mortar& m = h.mortars[h.slot_mortar[s]];
            const int side = h.slot_side[s];
            const int p0 = side == 0 ? m.posA0 : m.posB0, p1 = side == 0 ? m.posA1 : m.posB1;
            sp[s].info = h.slot_face[s] | side << 3 | p0 << 4 | p1 << 6 | (int)m.q << 8 | (m.eB >= 0 ? 1 << 12 : 0) |
                         (side ? (int)m.orient << 13 : 0);
            sp[s].sig = 0.0;
            sp[s].goff = m.goff;
        }
        std::vector<SlotPack<float>> sp32(sp.size());
        for (size_t s = 0; s < sp.size(); ++s) sp32[s] = SlotPack<float>{sp[s].info, 0.f, sp[s].goff};
        L.spack64 = A.upload(sp, st);
        L.spack32 = A.upload(sp32, st);
    }
    int* bad = A.alloc<int>(1);
    double* X = nullptr;
    if (A.failed || cudaMalloc(&X, sizeof(double) * 3 * nd) != cudaSuccess) {
        err = "device allocation failed (geometry)";
        return DG_ERR_OOM;
    }
    cudaMemsetAsync(bad, 0, sizeof(int), st);
    const GeomArgs g = geom_args(c, L);
    cudaError_t e1 = launch_node_coords(g, X, st);
    cudaError_t e2 = launch_volume_geom(g, X, L.G64, L.wdetJ, L.vxyz, nv, bad, st);
    cudaError_t e3 = launch_mortar_geom(g, X, L.mortars, nmort, c->C, L.mg64, L.sigma64, L.bxyz, nb, bad, st);
    cudaError_t e4 = cast_d2f(L.G64, L.G32, 6 * nv, st);
    cudaError_t e5 = cast_d2f(L.mg64, L.mg32, 7 * nm, st);
    cudaError_t e6 = cast_d2f(L.sigma64, L.sigma32, nmort, st);
    if (e6 == cudaSuccess) e6 = fill_slot_sigma(L.spack64, L.spack32, L.slot_mortar, L.sigma64, (int)h.slot_mortar.size(), st);
    int hbad = 0;
    cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e7 = cudaStreamSynchronize(st);
    cudaFree(X);
    c->launches += 6;
    for (cudaError_t e : {e1, e2, e3, e4, e5, e6, e7})
        if (e != cudaSuccess) {
            err = std::string("geometry kernels: ") + cudaGetErrorString(e);
            return DG_ERR_CUDA;
        }
    if (hbad) {
        err = "non-positive Jacobian determinant at a GL point (block map folds an element)";
        return DG_ERR_INVALID;
    }
    return DG_OK;
}

bool validate_desc(const dg_mesh_desc* d, std::string& err) {
    if (!d || d->n_elems <= 0 || !d->leaves || !d->p) { err = "mesh description is empty"; return false; }
    if (d->n_blocks < 0) { err = "n_blocks must be >= 0"; return false; }
    if (d->n_blocks == 0) {
        for (int k = 0; k < 3; ++k)
            if (!(d->hi[k] > d->lo[k])) { err = "box must have hi > lo"; return false; }
        if (d->map_kind != DG_MAP_AFFINE && d->map_kind != DG_MAP_SINE_WARP) { err = "unknown map kind"; return false; }
        return true;
    }
    if (d->n_blocks > 4096) { err = "at most 4096 blocks"; return false; }
    if (!d->blocks || !d->elem_block) { err = "blocks and elem_block are required when n_blocks > 0"; return false; }
    for (int b = 0; b < d->n_blocks; ++b) {
        const dg_block& B = d->blocks[b];
        if (B.kind == DG_BLOCK_HEX8) continue;
        if (B.kind != DG_BLOCK_WEDGE && B.kind != DG_BLOCK_SHELL) { err = "unknown block kind"; return false; }
        if (B.face < 0 || B.face > 5) { err = "block face must be 0..5"; return false; }
        if (B.kind == DG_BLOCK_WEDGE && !(B.a > 0 && B.r > B.a)) { err = "wedge needs 0 < a < r"; return false; }
        if (B.kind == DG_BLOCK_SHELL && !(B.r1 > 0 && B.r2 > B.r1)) { err = "shell needs 0 < r1 < r2"; return false; }
    }
    for (int e = 0; e < d->n_elems; ++e)
        if (d->elem_block[e] < 0 || d->elem_block[e] >= d->n_blocks) { err = "element block index out of range"; return false; }
    return true;
}

int build_hierarchy(const dg_mesh_desc* d, std::vector<LevelHost>& levels, BlockTopo& topo, std::string& err) {
    if (!build_block_topology(d->blocks, d->n_blocks > 0 ? d->n_blocks : 1, topo, err)) return DG_ERR_INVALID;
    LevelHost fine;
    fine.leaves.assign(d->leaves, d->leaves + 4 * (size_t)d->n_elems);
    fine.p.assign(d->p, d->p + d->n_elems);
    if (d->n_blocks > 0) fine.block.assign(d->elem_block, d->elem_block + d->n_elems);
    else fine.block.assign(d->n_elems, 0);
    if (!build_level_connectivity(fine, topo, err)) return DG_ERR_INVALID;
    std::vector<LevelHost> fine_first;
    fine_first.push_back(std::move(fine));
    while (true) {
        LevelHost coarse;
        std::string e2;
        if (!coarsen_level(fine_first.back(), coarse, topo, e2)) {
            if (!e2.empty()) { err = e2; return DG_ERR_INVALID; }
            break;
        }
        fine_first.push_back(std::move(coarse));
    }
    levels.assign(fine_first.rbegin(), fine_first.rend());
    return DG_OK;
}

// Boundary tags: values in range, and only Dirichlet on faces that lie on the
// domain boundary (the faces glued to another block ignore their tag).
int check_bc(const dg_mesh_desc* d, const BlockTopo& topo, std::string& err) {
    if (!d->bc) return DG_OK;
    const int nb = d->n_blocks > 0 ? d->n_blocks : 1;
    for (int b = 0; b < nb; ++b)
        for (int f = 0; f < 6; ++f) {
            const int k = d->bc[6 * b + f];
            if (k < DG_BC_DIRICHLET || k > DG_BC_ROBIN) {
                err = "boundary tag out of range";
                return DG_ERR_INVALID;
            }
            if (k != DG_BC_DIRICHLET && topo.face[6 * b + f].nb < 0) {
                err = "Neumann and Robin boundaries are not implemented (Dirichlet only)";
                return DG_ERR_UNSUPPORTED;
            }
        }
    return DG_OK;
}

size_t level_bytes(const LevelHost& h) {
    const size_t nv = h.vqp_off.back(), nd = h.n_dofs(), nm = h.n_mortar_pts;
    size_t b = 0;
    b += nv * (6 * 8 + 8 + 24 + 6 * 4);        // G64, wdetJ, vxyz, G32
    b += nm * 7 * (8 + 4);                     // mortar geometry
    b += nm * 4 * (8 + 4);                     // mortar trace buffers
    b += h.mortars.size() * (sizeof(Mortar) + 12);
    b += h.slot_mortar.size() * 6 + h.n_elems() * 40;
    b += nd * 6 * (8 + 4);                     // solver work vectors, both precisions
    return b;
}

}  // namespace

struct dg_mesh {
    dg_mesh_desc desc{};                // lo, hi, map and warp; array pointers cleared
    std::vector<dg_block> blocks;
    std::vector<LevelHost> levels;      // hierarchy, coarsest first
    BlockTopo topo;
};

extern "C" {

int dgi_set_error(int code, const char* msg) { return fail(code, msg ? msg : ""); }

int dg_mesh_create(const dg_mesh_desc* d, dg_mesh** out) {
    if (!out) return fail(DG_ERR_INVALID, "out is NULL");
    *out = nullptr;
    std::string err;
    if (!validate_desc(d, err)) return fail(DG_ERR_INVALID, err);
    auto m = std::make_unique<dg_mesh>();
    int rc = build_hierarchy(d, m->levels, m->topo, err);
    if (rc) return fail(rc, err);
    if ((rc = check_bc(d, m->topo, err))) return fail(rc, err);
    m->desc = *d;
    m->desc.leaves = nullptr;
    m->desc.p = nullptr;
    m->desc.blocks = nullptr;
    m->desc.elem_block = nullptr;
    m->desc.bc = nullptr;
    if (d->n_blocks > 0) m->blocks.assign(d->blocks, d->blocks + d->n_blocks);
    *out = m.release();
    return DG_OK;
}

void dg_mesh_destroy(dg_mesh* m) { delete m; }

int dg_version(void) { return DGELL_VERSION; }
const char* dg_last_error(void) { return g_err.c_str(); }

int dg_ctx_footprint(const dg_mesh* mesh, const dg_disc_opts* opts, size_t* bytes) {
    (void)opts;
    if (!mesh) return fail(DG_ERR_INVALID, "mesh is NULL");
    const std::vector<LevelHost>& lv = mesh->levels;
    size_t b = 2 * TabIndex::Count * kTabStride * 12;
    for (auto& h : lv) b += level_bytes(h);
    b += lv.back().n_dofs() * 8 * 6;            // FCG vectors
    if (bytes) *bytes = b;
    return DG_OK;
}


int dg_ctx_create(const dg_mesh* mesh, const dg_disc_opts* opts, void* stream, dg_ctx** out) {
    if (!out) return fail(DG_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!mesh) return fail(DG_ERR_INVALID, "mesh is NULL");
    std::string err;
    int rc = DG_OK;
    std::vector<LevelHost> lvh = mesh->levels;
    auto c = std::make_unique<dg_ctx>();
    c->st = (cudaStream_t)stream;
    c->C = (opts && opts->penalty_c > 0) ? opts->penalty_c : 10.0;
    c->desc = mesh->desc;
    c->blocks = mesh->blocks;
    c->topo = mesh->topo;
    std::vector<double> tab;
    build_tables(tab);
    std::vector<float> tabf(tab.begin(), tab.end());
    c->tab64 = c->arena.upload(tab, c->st);
    c->tab32 = c->arena.upload(tabf, c->st);
    std::vector<double> ftab;
    build_face_tables(tab, ftab, c->ft);
    std::vector<float> ftabf(ftab.begin(), ftab.end());
    c->ftab64 = c->arena.upload(ftab, c->st);
    c->ftab32 = c->arena.upload(ftabf, c->st);
    if (!c->blocks.empty()) c->blocks_dev = c->arena.upload(c->blocks, c->st);
    c->red.partials = c->arena.alloc<double>(kRedBlocks * 4);
    c->red.out = c->arena.alloc<double>(4);
    c->red.counter = c->arena.alloc<unsigned>(1);
    if (c->red.counter) cudaMemsetAsync(c->red.counter, 0, sizeof(unsigned), c->st);
    c->fcg = c->arena.alloc<FcgState>(1);
    if (c->arena.failed) {
        c->arena.free_all();
        return fail(DG_ERR_OOM, "device allocation failed");
    }
    if (cudaMallocHost(&c->red_host, 4 * sizeof(double)) != cudaSuccess) {
        c->arena.free_all();
        return fail(DG_ERR_CUDA, "pinned host allocation failed");
    }
    if (apply_streams_create(c->as) != cudaSuccess) {
        cudaGetLastError();
        apply_streams_destroy(c->as);
        c->arena.free_all();
        cudaFreeHost(c->red_host);
        return fail(DG_ERR_CUDA, "stream creation failed");
    }
    c->lv.resize(lvh.size());
    for (size_t l = 0; l < lvh.size(); ++l) c->lv[l].h = std::move(lvh[l]);
    for (size_t l = 0; l < c->lv.size(); ++l) {
        rc = upload_level(c.get(), c->lv[l], (int)l, err);
        if (rc) {
            apply_streams_destroy(c->as);
            c->arena.free_all();
            cudaFreeHost(c->red_host);
            return fail(rc, err);
        }
    }
    *out = c.release();
    return DG_OK;
}

void dg_ctx_destroy(dg_ctx* c) {
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
    else cudaDeviceSynchronize();
    if (c->vgraph) cudaGraphExecDestroy(c->vgraph);
    apply_streams_destroy(c->as);
    for (int i = 0; i < 2; ++i)
        if (c->hst[i]) cudaStreamDestroy(c->hst[i]);
    for (int sl = 0; sl < 2; ++sl)
        for (int k = 0; k < 3; ++k)
            if (c->hev[sl][k]) cudaEventDestroy(c->hev[sl][k]);
    if (c->hstart) cudaEventDestroy(c->hstart);
    if (c->hstage) cudaFree(c->hstage);
    c->arena.free_all();
    if (c->red_host) cudaFreeHost(c->red_host);
    delete c;
}

int dg_level_info_get(dg_ctx* c, int level, dg_level_info* info) {
    if (!c || !info) return fail(DG_ERR_INVALID, "NULL argument");
    level = resolve_level(c, level);
    if (level < 0 || level >= (int)c->lv.size()) return fail(DG_ERR_INVALID, "level out of range");
    const LevelHost& h = c->lv[level].h;
    info->n_levels = (int)c->lv.size();
    info->n_elems = h.n_elems();
    info->n_dofs = h.n_dofs();
    info->n_vol_qp = h.vqp_off.back();
    info->n_bnd_qp = h.n_bnd_pts;
    info->n_mortars = (int)h.mortars.size();
    int mp = 0;
    for (int v : h.p) mp = std::max(mp, v);
    info->max_p = mp;
    info->device_bytes = c->arena.bytes;
    double fl = 0.0;
    for (int e = 0; e < h.n_elems(); ++e) {
        const double n = h.p[e] + 1;
        fl += 24.0 * n * n * n * n + 18.0 * n * n * n;
        for (int si = h.slot_off[e]; si < h.slot_off[e + 1]; ++si) {
            const double q = h.mortars[h.slot_mortar[si]].q;
            fl += 4.0 * n * n * n + 12.0 * q * n * n + 16.0 * q * q * n + 20.0 * q * q;
        }
    }
    info->apply_flops = fl;
    return DG_OK;
}

int dg_level_leaves(dg_ctx* c, int level, int* leaves, int* p, int64_t* dof_off) {
    if (!c) return fail(DG_ERR_INVALID, "NULL context");
    level = resolve_level(c, level);
    if (level < 0 || level >= (int)c->lv.size()) return fail(DG_ERR_INVALID, "level out of range");
    const LevelHost& h = c->lv[level].h;
    if (leaves) std::memcpy(leaves, h.leaves.data(), h.leaves.size() * sizeof(int));
    if (p) std::memcpy(p, h.p.data(), h.p.size() * sizeof(int));
    if (dof_off)
        for (size_t i = 0; i < h.dof_off.size(); ++i) dof_off[i] = h.dof_off[i];
    return DG_OK;
}

int dg_level_blocks(dg_ctx* c, int level, int* elem_block) {
    if (!c || !elem_block) return fail(DG_ERR_INVALID, "NULL argument");
    level = resolve_level(c, level);
    if (level < 0 || level >= (int)c->lv.size()) return fail(DG_ERR_INVALID, "level out of range");
    const LevelHost& h = c->lv[level].h;
    std::memcpy(elem_block, h.block.data(), h.block.size() * sizeof(int));
    return DG_OK;
}

int dg_quadrature_points(dg_ctx* c, int level, double* vol_xyz, double* bnd_xyz) {
    if (!c) return fail(DG_ERR_INVALID, "NULL context");
    level = resolve_level(c, level);
    if (level < 0 || level >= (int)c->lv.size()) return fail(DG_ERR_INVALID, "level out of range");
    LevelDev& L = c->lv[level];
    if (vol_xyz) CK(cudaMemcpyAsync(vol_xyz, L.vxyz, sizeof(double) * 3 * L.h.vqp_off.back(), cudaMemcpyDeviceToDevice, c->st));
    if (bnd_xyz && L.h.n_bnd_pts)
        CK(cudaMemcpyAsync(bnd_xyz, L.bxyz, sizeof(double) * 3 * L.h.n_bnd_pts, cudaMemcpyDeviceToDevice, c->st));
    return DG_OK;
}

int dg_apply(dg_ctx* c, int level, int prec, const void* x, void* y) {
    if (!c || !x || !y) return fail(DG_ERR_INVALID, "NULL argument");
    level = resolve_level(c, level);
    if (level < 0 || level >= (int)c->lv.size()) return fail(DG_ERR_INVALID, "level out of range");
    if (x == y) return fail(DG_ERR_INVALID, "x and y must not alias");
    if (prec == DG_FP64) return apply_t<double>(c, level, (const double*)x, (double*)y);
    if (prec == DG_FP32) return apply_t<float>(c, level, (const float*)x, (float*)y);
    if (prec == DG_BF16) {
        int launches = 0;
        CK(launch_apply_bf16(view<float>(c, level), c->lv[level].buckets, x, (float*)y, c->st, &launches,
                             &c->lv[level].plan[2], &c->as));
        c->launches += launches;
        return DG_OK;
    }
    return fail(DG_ERR_UNSUPPORTED, "precision not implemented");
}

int dg_apply_host(dg_ctx* c, int level, int prec, int nvec, const void* hx, void* hy) {
    if (!c || nvec < 0) return fail(DG_ERR_INVALID, "NULL context or negative nvec");
    if (nvec == 0) return DG_OK;
    if (!hx || !hy) return fail(DG_ERR_INVALID, "NULL argument");
    level = resolve_level(c, level);
    if (level < 0 || level >= (int)c->lv.size()) return fail(DG_ERR_INVALID, "level out of range");
    if (hx == hy) return fail(DG_ERR_INVALID, "hx and hy must not alias");
    if (prec == DG_FP64) return apply_host_t<double>(c, level, nvec, (const double*)hx, (double*)hy);
    if (prec == DG_FP32) return apply_host_t<float>(c, level, nvec, (const float*)hx, (float*)hy);
    return fail(DG_ERR_UNSUPPORTED, "dg_apply_host: precision not implemented");
}

int dg_estimate_fiducial(dg_ctx* c, const dg_block* fiducial, int n_fiducial, const double* u, const double* g_qp,
                         const double* f_qp, const double* gD_qp, double* eta2) {
    if (!c || !u || !eta2) return fail(DG_ERR_INVALID, "NULL argument");
    const int nbk = (int)c->blocks.size();
    if (fiducial) {
        if (nbk == 0) return fail(DG_ERR_INVALID, "a fiducial grid needs a multi-block mesh");
        if (n_fiducial != nbk) return fail(DG_ERR_INVALID, "the fiducial grid must have one block per mesh block");
        for (int b = 0; b < nbk; ++b)
            if (fiducial[b].kind != c->blocks[b].kind ||
                (fiducial[b].kind != DG_BLOCK_HEX8 && fiducial[b].face != c->blocks[b].face))
                return fail(DG_ERR_INVALID, "fiducial block kinds and faces must be the mesh's");
    }
    const int l = (int)c->lv.size() - 1;
    LevelDev& L = c->lv[l];
    const long long nd = L.h.n_dofs(), nm = L.h.n_mortar_pts, nb = L.h.n_bnd_pts;
    const int nmort = (int)L.h.mortars.size();
    if (L.h.n_elems() == 0) return DG_OK;
    // stream-ordered scratch: the apply's output (nd), node coordinates (3 nd, single box) or, with
    // a fiducial grid, its mortar geometry (7 nm + nmort + 3 nb) and blocks
    const size_t nfb = fiducial ? (sizeof(dg_block) * nbk + 7) / 8 : 0;
    const size_t want = (size_t)nd + (nbk == 0 ? 3 * (size_t)nd : 0) +
                        (fiducial ? 7 * (size_t)nm + nmort + 3 * (size_t)nb + nfb + 1 : 0);
    double* S = nullptr;
    CK(cudaMallocAsync((void**)&S, sizeof(double) * want, c->st));
    double* y = S;
    double* X = nbk == 0 ? y + nd : nullptr;
    double *mgF = nullptr, *sigF = nullptr, *bxF = nullptr;
    dg_block* fb = nullptr;
    int* badF = nullptr;
    cudaError_t e = cudaSuccess;
    if (fiducial) {
        mgF = y + nd;
        sigF = mgF + 7 * nm;
        bxF = sigF + nmort;
        fb = reinterpret_cast<dg_block*>(bxF + 3 * nb);
        badF = reinterpret_cast<int*>(reinterpret_cast<double*>(fb) + nfb);
        e = cudaMemcpyAsync(fb, fiducial, sizeof(dg_block) * nbk, cudaMemcpyHostToDevice, c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(badF, 0, sizeof(int), c->st);
        if (e == cudaSuccess) {
            GeomArgs gF = geom_args(c, L);
            gF.blocks = fb;
            e = launch_mortar_geom(gF, nullptr, L.mortars, nmort, c->C, mgF, sigF, bxF, nb, badF, c->st);
            c->launches += 1;
        }
    }
    if (e == cudaSuccess && X) {
        e = launch_node_coords(geom_args(c, L), X, c->st);
        c->launches += 1;
    }
    int rc = e == cudaSuccess ? apply_t<double>(c, l, u, y) : DG_OK;   // fills the trace buffer with u's traces
    if (e == cudaSuccess && rc == DG_OK) {
        EstimateArgs a{};
        a.n_elems = L.h.n_elems();
        a.p = L.p;
        a.dof_off = L.dof_off;
        a.vqp_off = L.vqp_off;
        a.slot_off = L.slot_off;
        a.slot_mortar = L.slot_mortar;
        a.mortars = L.mortars;
        a.mg = L.mg64;
        a.sigma = L.sigma64;
        a.mt = L.mt64;
        a.tab = c->tab64;
        a.X = X;
        a.C = c->C;
        a.n_blocks = nbk;
        a.blocks = c->blocks_dev;
        a.block = L.block;
        a.leaves = L.leaves;
        a.fblocks = fiducial ? fb : c->blocks_dev;
        a.mgW = fiducial ? mgF : L.mg64;
        a.sigW = fiducial ? sigF : L.sigma64;
        e = launch_estimate(a, u, g_qp, f_qp, gD_qp, eta2, c->st);
        c->launches += 1;
    }
    int hbad = 0;
    if (e == cudaSuccess && rc == DG_OK && badF) {
        e = cudaMemcpyAsync(&hbad, badF, sizeof(int), cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    }
    cudaError_t ef = cudaFreeAsync(S, c->st);
    if (e != cudaSuccess) return fail(DG_ERR_CUDA, cudaGetErrorString(e));
    if (rc != DG_OK) return rc;
    if (ef != cudaSuccess) return fail(DG_ERR_CUDA, cudaGetErrorString(ef));
    if (hbad) return fail(DG_ERR_INVALID, "the fiducial grid folds an element (non-positive surface Jacobian)");
    return DG_OK;
}

int dg_estimate(dg_ctx* c, const double* u, const double* g_qp, const double* f_qp, const double* gD_qp,
                double* eta2) {
    return dg_estimate_fiducial(c, nullptr, 0, u, g_qp, f_qp, gD_qp, eta2);
}

int dg_convert(dg_ctx* c, int64_t n, int sp, const void* s, int dp, void* d) {
    if (!c || !s || !d || n < 0) return fail(DG_ERR_INVALID, "bad argument");
    if (sp == DG_FP64 && dp == DG_FP32) CK(cast_d2f((const double*)s, (float*)d, n, c->st));
    else if (sp == DG_FP32 && dp == DG_FP64) CK(cast_f2d((const float*)s, (double*)d, n, c->st));
    else if (sp == dp) CK(cudaMemcpyAsync(d, s, n * (sp == DG_FP64 ? 8 : 4), cudaMemcpyDeviceToDevice, c->st));
    else return fail(DG_ERR_UNSUPPORTED, "conversion not implemented");
    c->launches += 1;
    return DG_OK;
}

int64_t dg_launch_count(dg_ctx* c) { return c ? c->launches : -1; }

int dg_transfer(dg_ctx* c, int lc, int prec, int dir, const void* in, void* out) {
    if (!c || !in || !out) return fail(DG_ERR_INVALID, "NULL argument");
    if (lc < 0 || lc + 1 >= (int)c->lv.size()) return fail(DG_ERR_INVALID, "coarse level out of range");
    if (dir != 0 && dir != 1) return fail(DG_ERR_INVALID, "direction must be 0 or 1");
    if (prec == DG_FP64) {
        if (dir == 0) CK(launch_prolong_add<double>(tview<double>(c, lc), (const double*)in, (double*)out, c->st));
        else CK(launch_restrict<double>(tview<double>(c, lc), (const double*)in, (double*)out, c->st));
    } else if (prec == DG_FP32) {
        if (dir == 0) CK(launch_prolong_add<float>(tview<float>(c, lc), (const float*)in, (float*)out, c->st));
        else CK(launch_restrict<float>(tview<float>(c, lc), (const float*)in, (float*)out, c->st));
    } else {
        return fail(DG_ERR_UNSUPPORTED, "precision not implemented");
    }
    c->launches += 1;
    return DG_OK;
}

int dg_smooth(dg_ctx* c, int level, int prec, const void* b, void* x, const dg_cheb_opts* opts, double* lam_out) {
    if (!c || !b || !x) return fail(DG_ERR_INVALID, "NULL argument");
    level = resolve_level(c, level);
    if (level < 0 || level >= (int)c->lv.size()) return fail(DG_ERR_INVALID, "level out of range");
    int rc;
    if (prec == DG_FP64) rc = smooth_t<double>(c, level, (const double*)b, (double*)x, opts);
    else if (prec == DG_FP32) rc = smooth_t<float>(c, level, (const float*)b, (float*)x, opts);
    else return fail(DG_ERR_UNSUPPORTED, "precision not implemented");
    if (rc) return rc;
    if (lam_out) {
        SmState* sm = prec == DG_FP64 ? c->lv[level].w64.sm : c->lv[level].w32.sm;
        CK(cudaMemcpyAsync(c->red_host, &sm->lam, sizeof(double), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        *lam_out = c->red_host[0];
    }
    return DG_OK;
}

int dg_vcycle(dg_ctx* c, int prec, const void* f, void* v, const dg_mg_opts* opts) {
    if (!c || !f || !v) return fail(DG_ERR_INVALID, "NULL argument");
    if (prec == DG_FP64) return vcycle_t<double>(c, (const double*)f, (double*)v, opts);
    if (prec == DG_FP32) return vcycle_t<float>(c, (const float*)f, (float*)v, opts);
    return fail(DG_ERR_UNSUPPORTED, "precision not implemented");
}

int dg_solve(dg_ctx* c, const double* b, double* x, const dg_solver_opts* o, dg_solve_stats* stats) {
    if (!c || !b || !x) return fail(DG_ERR_INVALID, "NULL argument");
    auto t0 = std::chrono::steady_clock::now();
    const int Lt = (int)c->lv.size() - 1;
    const long long n = c->lv[Lt].h.n_dofs();
    const double tol = (o && o->tol > 0) ? o->tol : 1e-10;
    const int maxit = (o && o->max_iter > 0) ? o->max_iter : 100;
    const int mgp = o ? o->mg_prec : DG_FP64;
    const bool use_mg = o ? o->use_mg != 0 : true;
    const dg_mg_opts* mo = o ? &o->mg : nullptr;
    cudaStream_t st = c->st;
    if (!c->fcg_vec[0]) {
        for (int i = 0; i < 6; ++i) c->fcg_vec[i] = c->arena.alloc<double>(n);
        for (int i = 0; i < 2; ++i) c->fcg32[i] = c->arena.alloc<float>(n);
        if (c->arena.failed) return fail(DG_ERR_OOM, "device allocation failed (FCG vectors)");
    }
    double *r = c->fcg_vec[0], *v = c->fcg_vec[1], *w = c->fcg_vec[2], *d = c->fcg_vec[3], *q = c->fcg_vec[4],
           *t = c->fcg_vec[5];
    int rc;
    auto read_out = [&](int k, double* dst) -> int {
        CK(cudaMemcpyAsync(c->red_host, c->red.out, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int i = 0; i < k; ++i) dst[i] = c->red_host[i];
        return DG_OK;
    };
    // ||b||
    {
        const double* a[1] = {b};
        CK(dots<double>(a, a, 1, n, c->red, st));
    }
    double nb2;
    if ((rc = read_out(1, &nb2))) return rc;
    const double nb = std::sqrt(nb2);
    if ((rc = apply_t<double>(c, Lt, x, t))) return rc;
    CK(residual_init<double>(b, t, r, nullptr, n, c->red, st));
    double rr;
    if ((rc = read_out(1, &rr))) return rc;
    CK(cudaMemsetAsync(c->fcg, 0, sizeof(FcgState), st));
    int k = 0, restarts = 0;
    double rel = nb > 0 ? std::sqrt(rr) / nb : 0.0;
    int status = DG_OK;
    double true_rel = 0.0;
    for (;;) {
        int j = 0;   // iterations since the (re)start
        while (k < maxit && rel >= tol && nb > 0) {
            // v = VCYCLE(r)
            if (!use_mg) {
                CK(cudaMemcpyAsync(v, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
            } else {
                if (mgp == DG_FP32) {
                    CK(cast_d2f(r, c->fcg32[0], n, st));
                    c->launches += 1;
                }
                if ((rc = vcycle_maybe_graph(c, mgp, r, v, mo, o ? o->graph_mode : 0))) return rc;
                if (mgp == DG_FP32) {
                    CK(cast_f2d(c->fcg32[1], v, n, st));
                    c->launches += 1;
                }
            }
            if ((rc = apply_t<double>(c, Lt, v, w))) return rc;
            {
                const double* a[3] = {v, v, v};
                const double* bb[3] = {r, w, q};
                CK(dots<double>(a, bb, j == 0 ? 2 : 3, n, c->red, st));
            }
            CK(fcg_scalars(c->fcg, c->red.out, j, st));
            if (j == 0) {
                CK(cudaMemcpyAsync(d, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(q, w, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
            } else {
                CK(fcg_dq(c->fcg, d, q, v, w, n, st));
            }
            CK(fcg_update(c->fcg, x, r, d, q, n, c->red, st));
            c->launches += 6;
            if ((rc = read_out(1, &rr))) return rc;
            FcgState fs;
            CK(cudaMemcpyAsync(&fs, c->fcg, sizeof(FcgState), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            ++k;
            ++j;
            if (fs.breakdown || !std::isfinite(rr)) {
                status = DG_ERR_BREAKDOWN;
                break;
            }
            rel = std::sqrt(rr) / nb;
        }
        // true residual
        if ((rc = apply_t<double>(c, Lt, x, t))) return rc;
        CK(sub3<double>(b, t, w, n, st));
        {
            const double* a[1] = {w};
            CK(dots<double>(a, a, 1, n, c->red, st));
        }
        double tr2;
        if ((rc = read_out(1, &tr2))) return rc;
        true_rel = nb > 0 ? std::sqrt(tr2) / nb : 0.0;
        // on an ill-conditioned system the recursive residual can drift below the
        // true one: restart FCG from x with r = b - J x (at most 3 times)
        if (status != DG_OK || !(true_rel >= tol) || k >= maxit || restarts >= 3 || nb == 0) break;
        CK(cudaMemcpyAsync(r, w, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemsetAsync(c->fcg, 0, sizeof(FcgState), st));
        rel = true_rel;
        ++restarts;
    }
    if (status == DG_OK && rel >= tol && nb > 0) status = DG_ERR_NOT_CONVERGED;
    if (stats) {
        stats->iterations = k;
        stats->rel_residual = true_rel;
        stats->rel_residual_rec = rel;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        stats->status = status;
    }
    if (status == DG_ERR_BREAKDOWN) return fail(status, "flexible CG breakdown (non-positive rho)");
    if (status == DG_ERR_NOT_CONVERGED) return fail(status, "flexible CG reached max_iter");
    return DG_OK;
}

}  // extern "C"
