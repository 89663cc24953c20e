// Forward launch entry for FP32 arithmetic (the kernels are instantiated per dimension).
#include "sf_forward.cuh"

namespace sf {

cudaError_t launch_forward(const FwdArgs<float> &a, int threads, size_t smem, cudaStream_t s)
{
    return launch_forward_t(a, threads, smem, s);
}

}  // namespace sf
