// Operator-apply launcher.
#pragma once
#include "internal.h"

namespace dg {

struct BucketInfo {        // elements of one degree on one level
    const int* elems;      // device element ids
    const ElemDesc* desc;  // device, per element of the bucket
    int count;
    int max_q;             // largest mortar q among the bucket's slots
    int max_nb;            // largest neighbour n among the bucket's slots
};

// Side streams on which per-degree bucket kernels run next to those on the
// caller's stream, so that one bucket's last elements overlap the next
// bucket's first (fork and join by events; capturable into CUDA graphs).
constexpr int kApplySide = 5;          // capacity (DGELL_APPLY_STREAMS=k, k <= 5, uses k)
constexpr int kApplySideDefault = 1;   // two-way overlap measured fastest on the 32^3 sweep mesh
struct ApplyStreams {
    int n = 0;                                   // side streams in use (0: the caller's stream only)
    cudaStream_t side[kApplySide] = {};
    cudaEvent_t fork[2] = {};                    // trace phase, element phase
    cudaEvent_t join[2][kApplySide] = {};
};
cudaError_t apply_streams_create(ApplyStreams& as);
void apply_streams_destroy(ApplyStreams& as);

// y = L x on one level; buckets indexed by n (2..9).  launches: incremented per kernel launch.
// plan: the level's launch-plan slot (-1 = not tuned yet; tuned on first use) or nullptr.
// as: side streams for the per-bucket launch plan, or nullptr.
template <typename T>
cudaError_t launch_apply(const LevelView<T>& L, const BucketInfo* buckets, const T* x, T* y, cudaStream_t st,
                         int* launches, int* plan = nullptr, const ApplyStreams* as = nullptr);

// BF16 operand x (2-byte bfloat16 values), FP32 arithmetic and FP32 y.
cudaError_t launch_apply_bf16(const LevelView<float>& L, const BucketInfo* buckets, const void* x, float* y,
                              cudaStream_t st, int* launches, int* plan = nullptr,
                              const ApplyStreams* as = nullptr);

}  // namespace dg
