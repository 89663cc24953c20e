// sf_solve_noalloc: the FP32 structured-projection solve for one shared shape, with
// every piece of working memory in one fixed array compiled into the library, for
// callers that may not allocate device memory while they run (see include/sf.h).
//
// The array holds the instance table, the shape record, the Bernstein basis, the
// Kronecker blocks of the projection (P_dev, P_mean, B_dev, B_mean, computed here in
// FP64 by the same routine as a handle's factorisation) and the status words.  One
// set-up kernel writes all of it from arguments passed by value, so no host memory is
// read after the call returns; the forward and residual kernels are the library's
// ordinary ones, given pointers into this array.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "sf_internal.cuh"
#include "sf_kron.cuh"

namespace {

constexpr int kNaMaxInst = SF_NOALLOC_MAX_INST;
constexpr int kNaMaxH = SF_NOALLOC_MAX_H;
constexpr int kNaMaxXi = 32;
constexpr int kNaBlocks = 3 * kNaMaxXi * kNaMaxXi + 4 * kNaMaxXi;   // Kronecker record with two boundary rows
constexpr int kNaMaxDevices = 64;

struct NaScratch {
    sf::Inst<float> inst[kNaMaxInst];
    sf::Shape shape;
    int32_t status[kNaMaxInst];
    double W64[kNaMaxH * kNaMaxXi];
    double S64[kNaBlocks];
    float W32[kNaMaxH * kNaMaxXi];
    float S32[kNaBlocks];
};

// The fixed working memory (about 450 KB per device).  Host code must not pass this
// name to a kernel: on the host it is only a stand-in; its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NaScratch)];

// Device addresses of the array, looked up once per device under the mutex.
std::mutex g_mu;
void *g_addr[kNaMaxDevices];
bool g_ready[kNaMaxDevices];

// One call's set-up, passed by value (a captured launch carries its own copy).
struct NaSetup {
    sf_shape s;
    int nd, nxi, n_inst, hc;
    double rho;
};

// Instance table, shape record, basis and Kronecker blocks (FP64, then FP32 copies),
// status words cleared.  One CTA.  A singular KKT system (a zero pivot) leaves NaN
// blocks, so every iterate and residual of the call is NaN, and sets SF_EINVAL in the
// status words.
__global__ void k_na_setup(NaScratch *S, NaSetup u)
{
    __shared__ sf::KronSmem sm;
    const int tid = threadIdx.x, nt = blockDim.x, nxi = u.nxi, nd = u.nd, H = u.s.H, deg = nxi - 1;
    const int64_t N = (int64_t)u.s.n * nxi;
    const int64_t per_xi = nd * N, per_bnd = (int64_t)nd * u.s.n * 2;
    const int64_t per_obs = (int64_t)u.s.n_obs * (u.s.dyn_obs ? H : 1) * nd, per_oab = (int64_t)u.s.n_obs * 2;
    for (int i = tid; i < u.n_inst; i += nt) {
        sf::Inst<float> x;
        memset(&x, 0, sizeof(x));
        x.n = u.s.n;
        x.n_obs = u.s.n_obs;
        x.H = H;
        x.dyn = u.s.dyn_obs;
        x.N = (int)N;
        x.shape = 0;
        x.hc = u.hc;
        x.a = (float)u.s.a;
        x.b = (float)u.s.b;
        x.ia2 = (float)(1.0 / (u.s.a * u.s.a));
        x.ib2 = (float)(1.0 / (u.s.b * u.s.b));
        for (int ax = 0; ax < 3; ++ax) {
            x.pmin[ax] = (float)(ax < nd ? u.s.p_min[ax] : 0.0);
            x.pmax[ax] = (float)(ax < nd ? u.s.p_max[ax] : 0.0);
        }
        x.off_xi = i * per_xi;
        x.off_bnd = i * per_bnd;
        x.off_obs = i * per_obs;
        x.off_oab = i * per_oab;
        S->inst[i] = x;
        S->status[i] = SF_OK;
    }
    sf::Shape sh;
    memset(&sh, 0, sizeof(sh));
    sh.n = u.s.n;
    sh.n_obs = u.s.n_obs;
    sh.H = H;
    sh.N = (int)N;
    sh.nbc = 2;
    if (tid == 0) S->shape = sh;
    for (int e = tid; e < H * nxi; e += nt) {
        const int k = e / nxi, c = e % nxi;
        const double tau = (double)k / (double)(H - 1);
        double bin = 1.0;
        for (int q = 1; q <= c; ++q) bin = bin * (double)(deg - c + q) / (double)q;
        S->W64[e] = bin * pow(tau, (double)c) * pow(1.0 - tau, (double)(deg - c));
    }
    double *Cb = S->S64 + sf::kron_cost_off(nxi, 2);   // the projection cost's identity block
    for (int e = tid; e < nxi * nxi; e += nt) Cb[e] = (e / nxi == e % nxi) ? 1.0 : 0.0;
    __syncthreads();
    const int bad = sf::kron_kkt_blocks(sh, nxi, u.rho, S->W64, Cb, S->S64, sm);
    for (int e = tid; e < H * nxi; e += nt) S->W32[e] = (float)S->W64[e];
    const int nb = (int)sf::kron_len(nxi, 2);
    for (int e = tid; e < nb; e += nt) S->S32[e] = bad ? nanf("") : (float)S->S64[e];
    if (bad)
        for (int i = tid; i < u.n_inst; i += nt) S->status[i] = SF_EINVAL;
}

}  // namespace

extern "C" int sf_solve_noalloc(int32_t n_d, int32_t n_xi, double rho, const sf_shape *shape, int32_t n_inst,
                                const float *bnd, const float *obs_c, const float *obs_ab, const float *xi_cand,
                                int32_t iters, float *xi_out, float *lam_out, double *resid_out, void *stream)
{
    using namespace sf;
    if (!shape || !bnd || !xi_cand || !xi_out) return SF_EINVAL;
    if (n_d < 2 || n_d > 3 || n_xi < 4 || !(rho > 0.0) || !isfinite(rho) || n_inst < 1 || iters < 0) return SF_EINVAL;
    const sf_shape s = *shape;
    if (s.n < 1 || s.n > 256 || s.n_obs < 0 || s.n_obs > 4096 || s.H < 2) return SF_EINVAL;
    if (!(s.a > 0.0) || !(s.b > 0.0) || !isfinite(s.a) || !isfinite(s.b) || (s.dyn_obs != 0 && s.dyn_obs != 1))
        return SF_EINVAL;
    for (int ax = 0; ax < n_d; ++ax)
        if (!isfinite(s.p_min[ax]) || !isfinite(s.p_max[ax]) || !(s.p_min[ax] <= s.p_max[ax])) return SF_EINVAL;
    if (s.n_obs > 0 && (!obs_c || !obs_ab)) return SF_EINVAL;
    if (n_inst > kNaMaxInst || s.H > kNaMaxH || n_xi > kNaMaxXi) return SF_ETOOBIG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return SF_ECUDA;
    NaScratch *S;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_ready[dev]) {
            if (cudaGetSymbolAddress(&g_addr[dev], g_noalloc_scratch) != cudaSuccess) return SF_ECUDA;
            g_ready[dev] = true;
        }
        S = static_cast<NaScratch *>(g_addr[dev]);  // device address: pointer arithmetic only
    }
    cudaStream_t st = (cudaStream_t)stream;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return SF_ECUDA;

    // launch geometry of the forward kernel (structured projection, FP32)
    int num_sms = 0;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SF_ECUDA;
    const int nd = n_d, nxi = n_xi;
    Plan plan;
    int hc = 1;
    {
        int vn = s.n, vo = s.n_obs, vH = s.H;
        // every instance has the same shape: plan one and reuse it
        if (plan_forward(nd, nxi, (int)sizeof(float), SF_PROJ_STRUCTURED, 1, &vn, &vo, &vH,
                         std::max(1, num_sms / n_inst), optin, 0, kDefaultThreads, &plan, &hc) != SF_OK)
            return SF_ETOOBIG;
    }
    const int threads = plan.threads;

    NaSetup u;
    memset(&u, 0, sizeof(u));
    u.s = s;
    u.nd = nd;
    u.nxi = nxi;
    u.n_inst = n_inst;
    u.hc = hc;
    u.rho = rho;
    k_na_setup<<<1, 256, 0, st>>>(S, u);
    if (cudaGetLastError() != cudaSuccess) return SF_ECUDA;

    FwdArgs<float> a;
    memset(&a, 0, sizeof(a));
    a.nd = nd;
    a.nxi = nxi;
    a.nbc = 2;
    a.iters = iters;
    a.n_inst = n_inst;
    a.csize = plan.csize;
    a.p_rows = 0;
    a.cull = plan.cull;
    a.wait_budget = kWaitLimit;
    a.proj = SF_PROJ_STRUCTURED;
    a.rho = (float)rho;
    a.tol = 1e-3;
    a.inst = S->inst;
    a.order = nullptr;
    a.shapes = &S->shape;
    a.W = S->W32;
    a.Sx = S->S32;
    a.xc = xi_cand;
    a.bnd = bnd;
    a.obs = obs_c;
    a.oab = obs_ab;
    a.xo = xi_out;
    a.lo = lam_out;
    a.resid = resid_out;
    a.status = S->status;
    if (launch_forward(a, threads, plan.smem_fwd, st) != cudaSuccess) return SF_ECUDA;
    if (resid_out) {
        ResArgs<float> r;
        memset(&r, 0, sizeof(r));
        r.nd = nd;
        r.nxi = nxi;
        r.n_inst = n_inst;
        r.tol = 1e-3;
        r.inst = S->inst;
        r.shapes = &S->shape;
        r.W = S->W64;
        r.x = xi_out;
        r.obs = obs_c;
        r.oab = obs_ab;
        r.resid = resid_out;
        r.stride = SF_NRES;
        r.iters = iters;
        r.status = S->status;
        r.smem_doubles = (int64_t)(plan.smem_res / sizeof(double));
        r.csize = plan.csize;
        r.its_fixup = 1;
        if (launch_residual(r, std::min(threads, 512), plan.smem_res, st) != cudaSuccess) return SF_ECUDA;
    }
    return SF_OK;
}
