// Forward kernels, FP32, 3D (one translation unit per precision and dimension, so
// that the library builds in parallel).
#include "sf_forward.cuh"

namespace sf {

template cudaError_t launch_forward_nd<float, 3>(const FwdArgs<float> &, int, size_t, cudaStream_t);

}  // namespace sf
