// FP32 instantiation of the operator apply (apply_impl.cuh).
#include "apply_impl.cuh"

namespace dg {
template cudaError_t launch_apply<float>(const LevelView<float>&, const BucketInfo*, const float*, float*,
                                         cudaStream_t, int*, int*, const ApplyStreams*);
}  // namespace dg
