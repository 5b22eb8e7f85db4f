// Hop kernels of one precision and direction (see hop_kernels.cuh).
#include "hop_kernels.cuh"

namespace dwf {
template cudaError_t hop_launch_pd<DWF_F16, false>(const HopArgs &, int, int, int, cudaStream_t);
template cudaError_t hop_batch_launch_pd<DWF_F16, false>(const HopArgs *, int, const HopArgs &, int, int, cudaStream_t);
}  // namespace dwf
