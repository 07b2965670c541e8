// FP64 instantiation of the operator apply (apply_impl.cuh).
#include "apply_impl.cuh"

namespace dg {
template cudaError_t launch_apply<double>(const LevelView<double>&, const BucketInfo*, const double*, double*,
                                          cudaStream_t, int*, int*, const ApplyStreams*);
}  // namespace dg
