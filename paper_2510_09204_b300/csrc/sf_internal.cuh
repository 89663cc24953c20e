// Internal device structures of the SF solver library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sf.h"

namespace sf {

constexpr int kMaxThreads = 1024;    // largest CTA of any kernel (FP32 forward)
constexpr int kDefaultThreads = 512;
// Largest CTA of the forward kernel for element size esz: FP64 keeps 128 registers per thread.
__host__ __device__ constexpr int max_threads(int esz) { return esz == 8 ? 512 : 1024; }
constexpr int kMaxCluster = 8;     // CTAs per instance (portable cluster size)
constexpr int kMaxGroupCluster = 16;   // CTAs of a cluster that serves several instances (non-portable size)
constexpr int kRedDoubles = 100;   // block-reduction scratch of the residual kernel

// One instance as the kernels see it.  Offsets are in elements of T.
template <typename T>
struct Inst {
    int n, n_obs, H, dyn;
    int N;        // n * n_xi coefficients per axis
    int shape;    // index into the shape table
    int hc;       // timesteps per chunk of one CTA's share of the horizon (forward kernel)
    int pad_;
    T ia2, ib2;   // diagonal of M_r^-2: 1/a^2 (x, y), 1/b^2 (z)
    T a, b;
    T pmin[3], pmax[3];
    int64_t off_xi, off_bnd, off_obs, off_oab;
};

// One distinct (n, n_obs, H) shape: basis and xi_bar-step operators.
struct Shape {
    int n, n_obs, H, N;
    int nbc;          // boundary rows per robot and axis: 2 (start, goal) or 3 (+ initial velocity)
    int pad_;
    double vsc;       // scale of the velocity row: p'(0) = vsc (xi_1 - xi_0), vsc = (n_xi - 1) / ((H - 1) dt)
    int64_t off_W;    // H x n_xi
    int64_t off_P;    // N x N, P_eta (symmetric)
    int64_t off_Pb;   // N x nbc n, P_b (columns: robot-major (start, goal[, velocity]))
    int64_t off_S;    // structured form: P_dev, P_mean (n_xi x n_xi), B_dev, B_mean (n_xi x nbc), cost block
};

// Layout of a shape's Kronecker record: P_dev, P_mean, B_dev, B_mean, then the per-robot
// cost block (n_xi x n_xi).
__host__ __device__ inline int64_t kron_cost_off(int nxi, int nbc) { return 2 * (int64_t)nxi * nxi + 2 * (int64_t)nbc * nxi; }
__host__ __device__ inline int64_t kron_len(int nxi, int nbc) { return kron_cost_off(nxi, nbc) + (int64_t)nxi * nxi; }

// Boundary row s of one robot (eq. boundary_con) at coefficient c: the basis at tau = 0
// (start, s = 0) and tau = 1 (goal, s = 1), and the initial velocity p'(0) (s = 2), which
// for the Bernstein basis is vsc (xi_1 - xi_0).
__host__ __device__ inline double a0_row(const double *Ws, int nxi, int H, int s, int c, double vsc)
{
    if (s == 2) return c == 1 ? vsc : c == 0 ? -vsc : 0.0;
    return Ws[(s ? H - 1 : 0) * nxi + c];
}

// ---- tensor-core projection (dense P_eta on tcgen05) -----------------------------
// Modes: 0 none (SIMT), 1 TF32, 2 BF16, 3 BF16 x3 (hi*hi + hi*lo + lo*hi).
__host__ __device__ inline int tc_mode_of(int precision)
{
    return precision == SF_TF32 ? 1 : precision == SF_BF16 ? 2 : precision == SF_BF16X3 ? 3 : 0;
}
__host__ __device__ inline int tc_es(int mode) { return mode == 1 ? 4 : 2; }          // operand bytes
__host__ __device__ inline int tc_kc(int mode) { return 128 / tc_es(mode); }          // K per 128-byte chunk row
__host__ __device__ inline int tc_nk(int mode, int N) { return (N + tc_kc(mode) - 1) / tc_kc(mode); }
__host__ __device__ inline int tc_na(int mode) { return mode == 3 ? 2 : 1; }          // A (and B) parts
__host__ __device__ inline int tc_ntiles(int N, int C) { return (((N + C - 1) / C) + 127) / 128; }
constexpr int kTcChunkBytes = 128 * 128;   // one 128-row x 128-byte A chunk
constexpr uint32_t kWaitLimit = 1u << 20;   // polls of a bounded mbarrier wait (tens of ms)

// ---- batched tensor-core projection (instance groups) ------------------------------
// G instances of one shape share a cluster of G x C CTAs (C per instance for the rows).
// Each CTA of the cluster keeps Lb = ceil(N / (G C)) rows of P_eta in tensor memory as
// BF16 (with BF16 x3 the low parts in lanes 64..127 beneath the high parts in 0..63), and
// one product multiplies them by the right-hand sides of all G instances (G n_d <= 16
// columns of B: the BF16 high parts; with BF16 x3 the low parts in columns 16..31 of the
// same operand, so one MMA of N = 32 takes both).
__host__ __device__ inline int tcb_kpad(int N) { return (N + 15) / 16 * 16; }              // K padded to the MMA's 16
__host__ __device__ inline int64_t tcb_bbytes(int N) { return 16 * (int64_t)tcb_kpad(N) * 2; }   // 16 columns of B
__host__ __device__ inline int tcb_dcol(int N) { return (tcb_kpad(N) / 2 + 31) / 32 * 32; }   // accumulator column
__host__ __device__ inline uint32_t tcb_tmem_cols(int N)
{
    uint32_t c = 32;
    while (c < (uint32_t)(tcb_dcol(N) + 32)) c <<= 1;
    return c;
}
__host__ __device__ inline int tcb_rows(int N, int CC) { return (N + CC - 1) / CC; }

// A ring stages of a CTA: every chunk of its rows when they stay resident in shared
// memory for the whole launch (res), else two stages that stream from global memory.
__host__ __device__ inline int tc_stages(int mode, int N, int C, int res)
{
    return res ? tc_ntiles(N, C) * tc_nk(mode, N) : 2;
}

// Bytes at the front of shared memory for the tensor-core path: the A ring, the B
// operand, slack after B (so any misread of a descriptor stays inside the allocation),
// and the mbarriers / tensor-memory address.
__host__ __device__ inline int64_t tc_smem_bytes(int mode, int N, int stages)
{
    if (!mode) return 0;
    if (stages < 0)   // instance groups: B (high and low parts), the low lanes' staging, barriers
        return tc_na(mode) * tcb_bbytes(N) + 64 * 16 * 4 + 1024 + 128;
    const int64_t kpad = (int64_t)tc_nk(mode, N) * tc_kc(mode);
    const int64_t b = 16 * kpad * tc_es(mode);
    return (int64_t)stages * kTcChunkBytes * tc_na(mode) + b * tc_na(mode) + b + 1024 + 128;
}

// Shared-memory carve of the forward kernel, in elements of T.  Every region starts on a
// 32-byte boundary.  Host and kernel both call forward_carve, so they cannot disagree.
struct FwdCarve {
    int64_t W, xb, lam, xc, v, gp, dl, dd, rr, wtw, pb, Rb, ob, bd, db, bf, sx, red, Ps, bb, os, lp, lo, lc, total;
};

// Candidate lists of the culled row loops: per robot, the partners and obstacles whose
// bounding boxes over the chunk come within reach, padded to a multiple of four.
__host__ __device__ inline int cull_lp(int n) { return (n + 3) / 4 * 4 + 4; }          // partner list stride
__host__ __device__ inline int cull_lo(int nobs) { return (nobs + 3) / 4 * 4 + 4; }    // obstacle list stride

// Timesteps of the horizon one CTA of a C-CTA cluster owns at most (CTA r owns
// [r H / C, (r + 1) H / C)).
__host__ __device__ inline int cta_rows(int H, int C) { return (H + C - 1) / C; }

__host__ __device__ inline int64_t carve_round(int64_t cnt, int esz)
{
    const int64_t q = 32 / esz;
    return (cnt + q - 1) / q * q;
}

// nd, nxi: dimension and coefficients; wrows: rows of the basis a CTA keeps (its share
// of the horizon, ceil(H / C)); n, nobs: instance sizes; hc: timesteps per chunk;
// p_rows: rows of P_eta staged in shared memory (0: read from global memory); tc_mode,
// tc_st: tensor-core projection mode and A ring stages.
__host__ __device__ inline FwdCarve forward_carve(int nd, int nxi, int wrows, int n, int nobs, int hc, int p_rows, int esz,
                                                  int tc_mode = 0, int tc_st = 2, int cull = 0)
{
    const int64_t N = (int64_t)n * nxi, NN = nd * N, ndp = nd == 2 ? 2 : 4;
    FwdCarve c;
    int64_t o = (tc_smem_bytes(tc_mode, (int)N, tc_st) + 127) / 128 * 128 / esz;   // tensor-core buffers first
    c.W = o;   o += carve_round((int64_t)wrows * nxi, esz);            // this CTA's rows of W
    c.xb = o;  o += carve_round(NN, esz);
    c.lam = o; o += carve_round(NN, esz);
    c.xc = o;  o += carve_round(NN, esz);
    c.v = o;   o += carve_round(NN, esz);
    c.gp = o;  o += 2 * carve_round(NN + 4 + 3 * 32, esz);        // partial g + per-warp stats, two buffers
    c.dl = o;  o += carve_round(NN, esz);                         // projection rows of this CTA
    c.dd = o;  o += carve_round(NN, esz);                         // projection output
    c.rr = o;  o += carve_round(tc_mode ? NN : 0, esz);           // refinement residual (tensor cores)
    c.wtw = o; o += carve_round(tc_mode ? (int64_t)nxi * nxi + nd * nxi : 0, esz);   // W'W and robot sums
    const int64_t npad = (n + 3) / 4 * 4, opad = (nobs + 3) / 4 * 4;
    c.pb = o;  o += carve_round((npad + 4) * hc * ndp, esz);      // positions [i][k] as vectors (+ far dummies)
    c.Rb = o;  o += carve_round((int64_t)nd * n * hc, esz);       // row sums R [ax][i][k]
    c.ob = o;  o += carve_round((opad + 4) * 8, esz);             // obstacle records (+ dummies)
    c.bd = o;  o += carve_round((int64_t)nd * n * 3, esz);        // b (up to three rows per robot and axis)
    c.db = o;  o += carve_round((int64_t)nd * n * 3, esz);        // b - A xi_bar^0
    c.bf = o;  o += carve_round((int64_t)nd * n * 3, esz);        // values of the coefficients A fixes
    c.sx = o;  o += carve_round(3 * (int64_t)nxi * nxi + 6 * nxi + 2 * (int64_t)nd * nxi + 3 * nd, esz);
    c.red = o; o += carve_round(4 * 32, esz);
    c.Ps = o;  o += carve_round((int64_t)p_rows * N, esz);
    // culling, per segment of at most 32 timesteps: boxes [ax][lo, hi][segment][robot |
    // dynamic obstacle], obstacle columns [x, y, z, a_o^2, kz_o][m] (both read one entry
    // per lane), lists [segment][robot] (16-bit), counts
    const int64_t ns = (hc + 31) / 32;                            // culling segments of a chunk
    c.bb = o;  o += carve_round(cull ? ns * (n + nobs) * nd * 2 : 0, esz);
    c.os = o;  o += carve_round(cull ? (int64_t)nobs * 5 : 0, esz);
    c.lp = o;  o += carve_round(cull ? (ns * n * cull_lp(n) * 2 + esz - 1) / esz : 0, esz);
    c.lo = o;  o += carve_round(cull ? (ns * n * cull_lo(nobs) * 2 + esz - 1) / esz : 0, esz);
    c.lc = o;  o += carve_round(cull ? (ns * n * 2 * 4 + esz - 1) / esz : 0, esz);
    c.total = o;
    return c;
}

// The adjoint kernel's carve: the forward carve followed by the adjoint state
// (dL/dxi_bar, dL/dlambda, dL/dxi_cand) and R* in the vector layout of the positions.
struct BwdCarve {
    FwdCarve f;
    int64_t xs, ls, cs, xn, xz, xq, lq, Rs, total;
};

__host__ __device__ inline BwdCarve backward_carve(int nd, int nxi, int wrows, int n, int nobs, int hc, int p_rows, int esz,
                                                   int tc_mode = 0, int tc_st = 2, int cull = 0)
{
    BwdCarve b;
    b.f = forward_carve(nd, nxi, wrows, n, nobs, hc, p_rows, esz, tc_mode, tc_st, cull);
    const int64_t NN = (int64_t)nd * n * nxi, npad = (n + 3) / 4 * 4, ndp = nd == 2 ? 2 : 4;
    int64_t o = b.f.total;
    b.xs = o; o += carve_round(NN, esz);
    b.ls = o; o += carve_round(NN, esz);
    b.cs = o; o += carve_round(NN, esz);
    b.xn = o; o += carve_round(NN, esz);
    b.xz = o; o += carve_round(NN, esz);
    b.xq = o; o += carve_round(NN, esz);   // z^{l+1} of the reverse step (fixed-point loss seed)
    b.lq = o; o += carve_round(NN, esz);
    b.Rs = o; o += carve_round((npad + 4) * hc * ndp, esz);
    b.total = o;
    return b;
}

template <typename T>
struct FwdArgs {
    int nd, nxi, iters, n_inst;
    int nbc;          // boundary rows per robot and axis (every shape of the handle)
    int csize;        // CTAs per instance (thread-block cluster), 1..kMaxCluster
    int tcb;          // instances per cluster of the batched tensor-core projection (0: one per cluster)
    int p_rows;       // rows of P_eta per CTA staged in shared memory (dense; 0 = global)
    int tc_mode;      // tensor-core projection: 0 none, 1 TF32, 2 BF16, 3 BF16 x3
    int tc_res;       // the CTA's projector chunks stay resident in shared memory
    int cull;         // row loops over per-chunk candidate lists (bounding-box culling)
    int early;        // an instance stops after the iteration whose iterate met the tolerance
    int cost;         // SF_COST_PROJECTION or SF_COST_SMOOTHNESS (per-robot cost block Q1)
    uint32_t wait_budget;   // polls of the tensor-core pipeline's waits (0 only in tests)
    int n_refine;     // refinement passes of the tensor-core projection
    const unsigned char *tcA;   // arranged P_eta chunks for the current cluster size
    const int64_t *tc_off;      // byte offset of each shape's chunks in tcA
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
    int ck_final;               // slot that receives the final iterate
    int64_t ck_slot;            // elements per checkpoint slot (= packed xi length)
    int32_t *status;            // [n_inst]
};

template <typename T>
struct BwdArgs {
    FwdArgs<T> f;               // instance data, operators, checkpoints, iteration count
    const T *gxo, *glo;         // seeds dL/dxi_bar^L, dL/dlambda^L (nullable)
    const double *grp2;         // dL/d||r_p(xi_bar^L)||^2 per instance (nullable)
    const double *gfp;          // dL/d(sum_l ||z^{l+1} - z^l||^2) per instance (nullable)
    T *gxc, *gx0, *gl0;         // dL/dxi_cand, dL/dxi_bar^0, dL/dlambda^0 (gx0, gl0 nullable)
    T *seg;                     // recomputed iterates (xi_bar, then lambda) of a segment, per instance and CTA
    int x0_null;                // the solve started from xi_bar^0 = xi_cand
};

template <typename T>
struct ResArgs {
    int nd, nxi, n_inst;
    double tol;
    const Inst<T> *inst;
    const Shape *shapes;
    const double *W;            // the FP64 basis, whatever the solve precision
    const T *x;                 // coefficients to evaluate (packed xi)
    const T *obs, *oab;
    double *resid;              // [n_inst][stride]
    int stride;                 // doubles per instance in resid (SF_NRES; 4 for sf_metrics)
    int32_t *its;
    int iters;                  // iteration count of the solve (its fix-up)
    int32_t *status;
    int64_t smem_doubles;       // dynamic shared memory of the launch, in doubles
    int csize;                  // CTAs per instance (thread-block cluster)
    int its_fixup;              // update SF_RES_ITERS (a solve's residual check; not for metrics)
};

// ---- launchers (defined in the .cu files) ---------------------------------
// Launch geometry shared by every entry point that runs the forward kernel.
struct Plan {
    int csize = 1;        // CTAs per instance
    int tcb = 0;          // instances per cluster of the batched tensor-core projection (0: off)
    int threads = kDefaultThreads;
    int p_rows = 0;       // rows of P_eta staged per CTA (dense projection), 0 = read from global
    int tc_res = 0;       // tensor-core projector chunks resident in shared memory
    int cull = 0;         // culled row loops (the candidate lists fit in shared memory)
    size_t smem_fwd = 0;  // dynamic shared memory of the forward launch
    size_t smem_res = 0;  // and of the residual launch
    size_t smem_bwd = 0;  // and of the adjoint launch (0: does not fit)
};

// Chooses the cluster size (csize_req > 0 forces it), each instance's timestep chunk
// hc_out[i] and the shared-memory sizes.  Returns SF_OK or SF_EUNSUPPORTED when an
// instance cannot fit in `optin` bytes of shared memory.
int plan_forward(int nd, int nxi, int esz, int proj, int n_inst, const int *n, const int *nobs, const int *H,
                 int num_sms, int optin, int csize_req, int threads, Plan *out, int *hc_out, int tc_mode = 0,
                 int cull_req = 1, int need_bwd = 0, int tcb_req = 0);

// The A ring stages argument of the carves for a launch (-1: instance groups)
__host__ __device__ inline int tc_stage_arg(int tc_mode, int tcb, int N, int C, int res)
{
    return tcb ? -1 : tc_stages(tc_mode, N, C, res);
}

// Arranges every shape's P_eta (FP64 pool) into the tensor-core chunk layout for cluster
// size C: per shape [C][tiles][K chunks][128 x 128 bytes] (x 2 for the BF16 x3 low part).
cudaError_t arrange_tc(const Shape *shapes_dev, int n_shapes, const Shape *shapes_host, const double *P64,
                       const int64_t *tc_off_dev, const int64_t *tc_off_host, int mode, int C, unsigned char *out,
                       cudaStream_t s);
int64_t tc_pool_bytes(int mode, int N, int C);
cudaError_t basis_dd(const Shape *shapes_dev, int n_shapes, int nxi, double dt, double *Wdd, cudaStream_t s);
cudaError_t shape_metrics(const Inst<double> *inst, const Shape *shapes, int n_inst, int nd, int nxi, const double *W,
                          const double *Wdd, const double *x, double *out, cudaStream_t s);
cudaError_t shape_metrics(const Inst<float> *inst, const Shape *shapes, int n_inst, int nd, int nxi, const double *W,
                          const double *Wdd, const float *x, double *out, cudaStream_t s);

// Both launch n_inst clusters of a.csize CTAs (one cluster per instance).
cudaError_t launch_forward(const FwdArgs<double> &a, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_forward(const FwdArgs<float> &a, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_residual(const ResArgs<double> &a, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_residual(const ResArgs<float> &a, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_backward(const BwdArgs<double> &a, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_backward(const BwdArgs<float> &a, int threads, size_t smem, cudaStream_t s);

// Shared memory (doubles) the residual kernel needs for one instance at a chunk of hc timesteps.
__host__ __device__ inline int64_t residual_doubles(int nd, int nxi, int wrows, int n, int nobs, int hc)
{
    const int64_t N = (int64_t)n * nxi;
    return carve_round((int64_t)wrows * nxi, 8) + carve_round(nd * N, 8) + carve_round((int64_t)n * hc * (nd == 2 ? 2 : 4), 8) +
           carve_round((int64_t)nobs * 8, 8) + kRedDoubles;
}

// FP64 factorisation of every shape (sf_factor.cu): the dense KKT inverse (dense), or for
// structured handles the Kronecker blocks from the n_xi-size systems with the dense
// operators assembled from them.  W64/P64/Pb64/S64 are pools laid out by
// Shape offsets; info[s] receives 0 or a failing pivot index + 1.
cudaError_t factor_shapes(const Shape *shapes_dev, int n_shapes, const Shape *shapes_host, int nxi,
                          double rho, int cost, double dt, double *W64, double *P64, double *Pb64, double *S64,
                          double *scratch, int64_t scratch_elems, int *info, cudaStream_t s, bool dense);
cudaError_t convert_pool(const double *src, float *dst, int64_t n, cudaStream_t s);

}  // namespace sf
