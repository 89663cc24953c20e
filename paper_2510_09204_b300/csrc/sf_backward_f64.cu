// Backward kernels and launch entry for FP64 arithmetic.
#include "sf_backward.cuh"

namespace sf {

template cudaError_t launch_backward_nd<double, 2>(const BwdArgs<double> &, int, size_t, cudaStream_t);
template cudaError_t launch_backward_nd<double, 3>(const BwdArgs<double> &, int, size_t, cudaStream_t);

cudaError_t launch_backward(const BwdArgs<double> &a, int threads, size_t smem, cudaStream_t s)
{
    return launch_backward_t(a, threads, smem, s);
}

}  // namespace sf
