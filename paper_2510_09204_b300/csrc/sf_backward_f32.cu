// Backward launch entry for FP32 arithmetic (the kernels are instantiated per dimension).
#include "sf_backward.cuh"

namespace sf {

cudaError_t launch_backward(const BwdArgs<float> &a, int threads, size_t smem, cudaStream_t s)
{
    return launch_backward_t(a, threads, smem, s);
}

}  // namespace sf
