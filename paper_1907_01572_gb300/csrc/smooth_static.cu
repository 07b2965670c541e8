// dg_smooth_static: the Chebyshev / CG-eigenvalue smoother of dg_smooth, run
// entirely on a scratch array compiled into this library, so that the call
// itself never allocates device memory.
//
// Who needs it: callers that cannot call cudaMalloc at the time they smooth --
// code running while all free device memory has been handed to a caching
// allocator (PyTorch's, or a serving loop that has admitted requests up to
// the HBM budget), where a fresh cudaMalloc can fail, and latency-sensitive
// loops that cannot accept cudaMalloc's implicit device-wide synchronisation.
//
// The scratch is one file-scope __device__ array (kStaticBytes, below).  Every
// GPU that loads the library reserves it until the process exits.  Host code
// only ever sees a host-side stand-in for the array's name, so the device
// address is looked up once per device with cudaGetSymbolAddress, with that
// device current, on the first call made on that device; make that first
// call before any stream capture.  All calls share the array and it keeps the
// previous call's contents: everything that must start at zero is cleared by
// the call itself, and calls whose GPU work overlaps (different streams or
// threads) race on the array.
#include <mutex>

#include "context.h"

using namespace dg;

extern "C" int dgi_set_error(int code, const char* msg);

namespace {

constexpr long long kStaticMaxDofs = 1LL << 18;   // 262,144 DOFs per level
constexpr size_t kVecBytes = (size_t)kStaticMaxDofs * sizeof(double);
constexpr size_t kStateBytes = (sizeof(SmState) + 255) / 256 * 256;
constexpr size_t kRedBytes = ((size_t)(kRedBlocks * 4 + 4 + 1) * sizeof(double) + 255) / 256 * 256;
constexpr size_t kStaticBytes = 3 * kVecBytes + kStateBytes + kRedBytes;   // ~6.1 MB

static __device__ __align__(256) unsigned char g_smooth_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

int scratch_for_current_device(unsigned char** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return dgi_set_error(DG_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return dgi_set_error(DG_ERR_UNSUPPORTED, "device ordinal too large");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_smooth_scratch);
        if (e != cudaSuccess || !p)
            return dgi_set_error(DG_ERR_CUDA, e != cudaSuccess ? cudaGetErrorString(e) : "null symbol address");
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[dev];
    return DG_OK;
}

#define CKS(call)                                                                          \
    do {                                                                                   \
        cudaError_t _e = (call);                                                           \
        if (_e != cudaSuccess) return dgi_set_error(DG_ERR_CUDA, cudaGetErrorString(_e)); \
    } while (0)

template <typename T>
int smooth_static_t(dg_ctx* c, int l, const T* b, T* x, const dg_cheb_opts* o, unsigned char* base) {
    const double fixed = (o && o->lam_fixed > 0) ? o->lam_fixed : 0.0;
    const int ne = fixed > 0 ? 0 : ((o && o->n_eigs > 0) ? o->n_eigs : 15);
    int nc = (o && o->n_cheb > 0) ? o->n_cheb : 15;
    const double Lam = (o && o->Lambda > 0) ? o->Lambda : 20.0;
    const double scale = (o && o->lam_scale > 0) ? o->lam_scale : 1.0;
    if (nc > kMaxCheb) nc = kMaxCheb;
    const long long n = c->lv[l].h.n_dofs();
    T* r = reinterpret_cast<T*>(base);
    T* p = reinterpret_cast<T*>(base + kVecBytes);
    T* Ap = reinterpret_cast<T*>(base + 2 * kVecBytes);
    SmState* sm = reinterpret_cast<SmState*>(base + 3 * kVecBytes);
    Red red{reinterpret_cast<double*>(base + 3 * kVecBytes + kStateBytes), nullptr, nullptr};
    red.out = red.partials + kRedBlocks * 4;
    red.counter = reinterpret_cast<unsigned*>(red.out + 4);   // each last block resets it; cleared below too
    cudaStream_t st = c->st;
    // The last-block counter must start at zero; a call that stopped early
    // (an error between launches) may have left it non-zero.
    CKS(cudaMemsetAsync(red.counter, 0, sizeof(unsigned), st));
    const LevelView<T> view = level_view<T>(c, l);
    int launches = 0;
    CKS(launch_apply<T>(view, c->lv[l].buckets, x, Ap, st, &launches));
    CKS(residual_init<T>(b, Ap, r, p, n, red, st));
    CKS(sm_init(sm, red.out, st));
    for (int k = 0; k < ne; ++k) {
        CKS(launch_apply<T>(view, c->lv[l].buckets, p, Ap, st, &launches));
        CKS(cg_alpha_fused<T>(sm, p, Ap, n, red, st));
        CKS(cg_update_fused<T>(sm, x, r, p, Ap, n, red, st));
        CKS(cg_p_update<T>(sm, p, r, n, st));
    }
    CKS(sm_cheb_coeffs(sm, nc, Lam, scale, fixed, st));
    CKS(cudaMemsetAsync(p, 0, n * sizeof(T), st));
    for (int k = 0; k < nc; ++k) {
        CKS(launch_apply<T>(view, c->lv[l].buckets, x, Ap, st, &launches));
        CKS(cheb_step<T>(sm, k, b, Ap, p, x, n, st));
    }
    c->launches += launches + 3 + 3 * ne + 1 + nc;
    return DG_OK;
}

}  // namespace

extern "C" int dg_smooth_static(dg_ctx* c, int level, int prec, const void* b, void* x, const dg_cheb_opts* opts,
                                double* lambda_max_out) {
    if (!c || !b || !x) return dgi_set_error(DG_ERR_INVALID, "NULL argument");
    if (level < 0) level = (int)c->lv.size() - 1;
    if (level >= (int)c->lv.size()) return dgi_set_error(DG_ERR_INVALID, "level out of range");
    const long long n = c->lv[level].h.n_dofs();
    if (n > kStaticMaxDofs)
        return dgi_set_error(DG_ERR_INVALID,
                             "dg_smooth_static: the level has more DOFs than the static scratch holds (262144)");
    if (prec != DG_FP64 && prec != DG_FP32) return dgi_set_error(DG_ERR_UNSUPPORTED, "precision not implemented");
    unsigned char* base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc) return rc;
    rc = prec == DG_FP64 ? smooth_static_t<double>(c, level, (const double*)b, (double*)x, opts, base)
                         : smooth_static_t<float>(c, level, (const float*)b, (float*)x, opts, base);
    if (rc) return rc;
    if (lambda_max_out) {
        SmState* sm = reinterpret_cast<SmState*>(base + 3 * kVecBytes);
        CKS(cudaMemcpyAsync(c->red_host, &sm->lam, sizeof(double), cudaMemcpyDeviceToHost, c->st));
        CKS(cudaStreamSynchronize(c->st));
        *lambda_max_out = c->red_host[0];
    }
    return DG_OK;
}
