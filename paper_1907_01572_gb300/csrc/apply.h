// Operator-apply launcher.
#pragma once
#include "internal.h"

namespace dg {

struct BucketInfo {        // elements of one degree on one level
    const int* elems;      // device element ids
    int count;
    int max_q;             // largest mortar q among the bucket's slots
    int max_nb;            // largest neighbour n among the bucket's slots
};

// y = L x on one level; buckets indexed by n (2..9).  launches: incremented per kernel launch.
// plan: the level's launch-plan slot (-1 = not tuned yet; tuned on first use) or nullptr.
template <typename T>
cudaError_t launch_apply(const LevelView<T>& L, const BucketInfo* buckets, const T* x, T* y, cudaStream_t st,
                         int* launches, int* plan = nullptr);

// BF16 operand x (2-byte bfloat16 values), FP32 arithmetic and FP32 y.
cudaError_t launch_apply_bf16(const LevelView<float>& L, const BucketInfo* buckets, const void* x, float* y,
                              cudaStream_t st, int* launches, int* plan = nullptr);

}  // namespace dg
