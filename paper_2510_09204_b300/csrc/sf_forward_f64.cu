// Forward kernels and launch entry for FP64 arithmetic.
#include "sf_forward.cuh"

namespace sf {

template cudaError_t launch_forward_nd<double, 2>(const FwdArgs<double> &, int, size_t, cudaStream_t);
template cudaError_t launch_forward_nd<double, 3>(const FwdArgs<double> &, int, size_t, cudaStream_t);

cudaError_t launch_forward(const FwdArgs<double> &a, int threads, size_t smem, cudaStream_t s)
{
    return launch_forward_t(a, threads, smem, s);
}

}  // namespace sf
