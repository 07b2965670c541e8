// Inter-mesh operators of Sec. II.E.6.
// Prolongation (eq. psi-interpolation): the coarse polynomial is evaluated at
// the children's LGL nodes, child half b along each axis mapping the child
// coordinate xi to (xi + 2b - 1)/2 of the parent; the 3-D operator is the
// tensor product of three 1-D (n_h x n_H) matrices.  Restriction of weak
// residuals is its transpose (eq. temp-G), summed over the children.
// Elements carried over unchanged between levels are copied.
#include "transfer.h"

namespace dg {
namespace {

template <typename T>
__device__ void rect_pass(const T* in, T* out, const T* M, int dir, int n_out, int n_in, const int din[3], int dout[3],
                          bool trans, int m_cols) {
    // out has dims dout (x fastest), in has dims din; contraction along `dir`
    const int total = dout[0] * dout[1] * dout[2];
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int o[3] = {idx % dout[0], (idx / dout[0]) % dout[1], idx / (dout[0] * dout[1])};
        T s = 0;
        for (int m = 0; m < n_in; ++m) {
            int ii[3] = {o[0], o[1], o[2]};
            ii[dir] = m;
            const T mv = trans ? M[m * m_cols + o[dir]] : M[o[dir] * m_cols + m];
            s += mv * in[ii[0] + din[0] * (ii[1] + din[1] * ii[2])];
        }
        out[idx] = s;
    }
    (void)n_out;
}

template <typename T>
__global__ void prolong_kernel(TransferView<T> t, const T* __restrict__ vH, T* __restrict__ vh) {
    const int c = blockIdx.x;
    if (c >= t.n_fine) return;
    __shared__ T buf[3][kMaxN * kMaxN * kMaxN];
    const int H = t.fine_parent[c];
    const int bits = t.fine_bits[c];
    const int nH = t.pH[H] + 1, nh = t.ph[c] + 1;
    const T* src = vH + t.dofH[H];
    T* dst = vh + t.dofh[c];
    if (bits == 0xFF) {
        for (int k = threadIdx.x; k < nh * nh * nh; k += blockDim.x) dst[k] += src[k];
        return;
    }
    for (int k = threadIdx.x; k < nH * nH * nH; k += blockDim.x) buf[0][k] = src[k];
    __syncthreads();
    const T* Cx = t.tab + tab_ci(nH, nh, bits & 1);
    const T* Cy = t.tab + tab_ci(nH, nh, (bits >> 1) & 1);
    const T* Cz = t.tab + tab_ci(nH, nh, (bits >> 2) & 1);
    int d0[3] = {nH, nH, nH}, d1[3] = {nh, nH, nH}, d2[3] = {nh, nh, nH}, d3[3] = {nh, nh, nh};
    rect_pass(buf[0], buf[1], Cx, 0, nh, nH, d0, d1, false, nH);
    __syncthreads();
    rect_pass(buf[1], buf[2], Cy, 1, nh, nH, d1, d2, false, nH);
    __syncthreads();
    rect_pass(buf[2], buf[0], Cz, 2, nh, nH, d2, d3, false, nH);
    __syncthreads();
    for (int k = threadIdx.x; k < nh * nh * nh; k += blockDim.x) dst[k] += buf[0][k];
}

template <typename T>
__global__ void restrict_kernel(TransferView<T> t, const T* __restrict__ rh, T* __restrict__ fH) {
    const int H = blockIdx.x;
    if (H >= t.n_coarse) return;
    __shared__ T buf[3][kMaxN * kMaxN * kMaxN];
    __shared__ T acc[kMaxN * kMaxN * kMaxN];
    const int nH = t.pH[H] + 1;
    const int n3H = nH * nH * nH;
    for (int k = threadIdx.x; k < n3H; k += blockDim.x) acc[k] = 0;
    __syncthreads();
    for (int ci = t.child_off[H]; ci < t.child_off[H + 1]; ++ci) {
        const int c = t.child_id[ci];
        const int bits = t.child_bits[ci];
        const int nh = t.ph[c] + 1;
        const T* src = rh + t.dofh[c];
        if (bits == 0xFF) {
            for (int k = threadIdx.x; k < n3H; k += blockDim.x) acc[k] += src[k];
            __syncthreads();
            continue;
        }
        for (int k = threadIdx.x; k < nh * nh * nh; k += blockDim.x) buf[0][k] = src[k];
        __syncthreads();
        const T* Cx = t.tab + tab_ci(nH, nh, bits & 1);
        const T* Cy = t.tab + tab_ci(nH, nh, (bits >> 1) & 1);
        const T* Cz = t.tab + tab_ci(nH, nh, (bits >> 2) & 1);
        int d0[3] = {nh, nh, nh}, d1[3] = {nH, nh, nh}, d2[3] = {nH, nH, nh}, d3[3] = {nH, nH, nH};
        rect_pass(buf[0], buf[1], Cx, 0, nH, nh, d0, d1, true, nH);
        __syncthreads();
        rect_pass(buf[1], buf[2], Cy, 1, nH, nh, d1, d2, true, nH);
        __syncthreads();
        rect_pass(buf[2], buf[0], Cz, 2, nH, nh, d2, d3, true, nH);
        __syncthreads();
        for (int k = threadIdx.x; k < n3H; k += blockDim.x) acc[k] += buf[0][k];
        __syncthreads();
    }
    T* dst = fH + t.dofH[H];
    for (int k = threadIdx.x; k < n3H; k += blockDim.x) dst[k] = acc[k];
}

}  // namespace

template <typename T>
cudaError_t launch_prolong_add(const TransferView<T>& t, const T* vH, T* vh, cudaStream_t st) {
    prolong_kernel<T><<<t.n_fine, 128, 0, st>>>(t, vH, vh);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_restrict(const TransferView<T>& t, const T* rh, T* fH, cudaStream_t st) {
    restrict_kernel<T><<<t.n_coarse, 128, 0, st>>>(t, rh, fH);
    return cudaGetLastError();
}
template cudaError_t launch_prolong_add<double>(const TransferView<double>&, const double*, double*, cudaStream_t);
template cudaError_t launch_prolong_add<float>(const TransferView<float>&, const float*, float*, cudaStream_t);
template cudaError_t launch_restrict<double>(const TransferView<double>&, const double*, double*, cudaStream_t);
template cudaError_t launch_restrict<float>(const TransferView<float>&, const float*, float*, cudaStream_t);

}  // namespace dg
