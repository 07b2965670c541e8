// Prolongation / restriction launchers.
#pragma once
#include "internal.h"

namespace dg {

template <typename T>
struct TransferView {      // between coarse level l-1 (H) and fine level l (h)
    int n_coarse, n_fine;
    const int* pH;
    const int* ph;
    const long long* dofH;
    const long long* dofh;
    const int* child_off;      // coarse: n_coarse + 1
    const int* child_id;
    const unsigned char* child_bits;
    const int* fine_parent;    // fine: n_fine
    const unsigned char* fine_bits;
    const T* tab;
};

// vh += I_h^H vH
template <typename T>
cudaError_t launch_prolong_add(const TransferView<T>& t, const T* vH, T* vh, cudaStream_t st);
// fH = (I_h^H)^T rh
template <typename T>
cudaError_t launch_restrict(const TransferView<T>& t, const T* rh, T* fH, cudaStream_t st);

}  // namespace dg
