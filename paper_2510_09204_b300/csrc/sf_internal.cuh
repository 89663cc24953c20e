// Internal device structures of the SF solver library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sf.h"

namespace sf {

constexpr int kMaxThreads = 512;
constexpr int kIPT = 8;            // (robot, timestep) items a thread keeps in registers per chunk
constexpr int kRedDoubles = 100;   // block-reduction scratch (3 x 32 warps + 3 results)

// One instance as the kernels see it.  Offsets are in elements of T.
template <typename T>
struct Inst {
    int n, n_obs, H, dyn;
    int N;        // n * n_xi coefficients per axis
    int shape;    // index into the shape table
    int hc;       // timesteps per chunk in the forward kernel
    int pad_;
    T ia2, ib2;   // diagonal of M_r^-2: 1/a^2 (x, y), 1/b^2 (z)
    T a, b;
    T pmin[3], pmax[3];
    int64_t off_xi, off_bnd, off_obs, off_oab;
};

// One distinct (n, n_obs, H) shape: basis and xi_bar-step operators.
struct Shape {
    int n, n_obs, H, N;
    int64_t off_W;    // H x n_xi
    int64_t off_P;    // N x N, P_eta (symmetric)
    int64_t off_Pb;   // N x 2n, P_b (columns: robot-major (start, goal))
    int64_t off_S;    // structured form: P_dev, P_mean, B_dev, B_mean (n_xi x n_xi, n_xi x 2 each)
};

template <typename T>
struct FwdArgs {
    int nd, nxi, iters, n_inst;
    int p_smem;       // 1: P_eta of each instance staged in shared memory
    int proj;         // SF_PROJ_DENSE / SF_PROJ_STRUCTURED
    T rho;
    double tol;
    const Inst<T> *inst;
    const int *order;           // instance order (largest first), n_inst entries
    const Shape *shapes;
    const T *W, *P, *Pb, *Sx;   // shape pools
    const T *xc, *x0, *l0;      // candidate, initial iterate (nullable)
    const T *bnd, *obs, *oab;   // instance data
    T *xo, *lo;                 // outputs (lo nullable)
    double *resid;              // [n_inst][SF_NRES] (nullable)
    int32_t *its;               // [n_inst] (nullable)
    float *hist;                // [n_inst][iters] (nullable)
    T *ck_x, *ck_l;             // checkpoints: slot-major, packed like xi (nullable)
    int ck_every;
    int64_t ck_slot;            // elements per checkpoint slot (= packed xi length)
    int32_t *status;            // [n_inst]
};

template <typename T>
struct ResArgs {
    int nd, nxi, n_inst;
    double tol;
    const Inst<T> *inst;
    const Shape *shapes;
    const T *W;
    const T *x;                 // coefficients to evaluate (packed xi)
    const T *obs, *oab;
    double *resid;              // [n_inst][SF_NRES]
    int32_t *its;
    int iters;                  // iteration count of the solve (its fix-up)
    int32_t *status;
    int64_t smem_doubles;       // dynamic shared memory of the launch, in doubles
};

// ---- launchers (defined in the .cu files) ---------------------------------
cudaError_t launch_forward(const FwdArgs<double> &a, int grid, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_forward(const FwdArgs<float> &a, int grid, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_residual(const ResArgs<double> &a, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_residual(const ResArgs<float> &a, int threads, size_t smem, cudaStream_t s);
cudaError_t forward_smem_limit(size_t bytes);

// FP64 factorisation of every shape (sf_factor.cu).  W64/P64/Pb64/S64 are pools laid out by
// Shape offsets; info[s] receives 0 or a failing pivot index + 1.
cudaError_t factor_shapes(const Shape *shapes_dev, int n_shapes, const Shape *shapes_host, int nxi,
                          double rho, double *W64, double *P64, double *Pb64, double *S64,
                          double *scratch, int64_t scratch_elems, int *info, cudaStream_t s);
cudaError_t convert_pool(const double *src, float *dst, int64_t n, cudaStream_t s);

}  // namespace sf
