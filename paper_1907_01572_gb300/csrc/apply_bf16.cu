// BF16-operand instantiation of the operator apply (apply_impl.cuh): the input
// vector is read as bfloat16 and widened to FP32; all arithmetic, geometry and
// tables are FP32; y is FP32.
#include "apply_impl.cuh"

namespace dg {
cudaError_t launch_apply_bf16(const LevelView<float>& L, const BucketInfo* buckets, const void* x, float* y,
                              cudaStream_t st, int* launches, int* plan, const ApplyStreams* as) {
    return launch_apply_x<float, __nv_bfloat16>(L, buckets, static_cast<const __nv_bfloat16*>(x), y, st, launches,
                                                plan, as);
}
}  // namespace dg
