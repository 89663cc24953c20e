// sf_solve_noalloc: the FP32 structured-projection solve for one shared shape, with
// every piece of working memory in one fixed array compiled into the library, for
// callers that may not allocate device memory while they run (see include/sf.h).
//
// The array holds the instance table, the shape record, the Bernstein basis, the
// Kronecker blocks of the projection (P_dev, P_mean, B_dev, B_mean, computed here in
// FP64 from the two n_xi x n_xi constrained inverses) and the status words.  The
// forward and residual kernels are the library's ordinary ones, given pointers into
// this array.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "sf_internal.cuh"

namespace {

constexpr int kNaMaxInst = SF_NOALLOC_MAX_INST;
constexpr int kNaMaxH = SF_NOALLOC_MAX_H;
constexpr int kNaMaxXi = 32;
constexpr int kNaBlocks = 2 * kNaMaxXi * kNaMaxXi + 4 * kNaMaxXi;
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

void *g_addr[kNaMaxDevices];
bool g_ready[kNaMaxDevices];
sf::Inst<float> g_inst_host[kNaMaxInst];
sf::Shape g_shape_host;

constexpr int kKkt = kNaMaxXi + 2;

// Basis and Kronecker blocks of one shape, FP64 then FP32 copies.  One CTA.
// P_dev / P_mean are the x-blocks of the inverse of [[I + rho c W'W, A0'], [A0, 0]]
// for c = n + n_obs + 2 and c = n_obs + 2 (A0 = rows 0 and H-1 of W); B_dev / B_mean
// are its (x, b) blocks.  Gauss-Jordan elimination with partial pivoting.
__global__ void k_na_operators(NaScratch *S, int nxi, int H, int n, int n_obs, double rho)
{
    __shared__ double wtw[kNaMaxXi * kNaMaxXi];
    __shared__ double K[kKkt * kKkt];
    __shared__ double X[kKkt * kKkt];
    __shared__ int piv;
    const int tid = threadIdx.x, nt = blockDim.x, deg = nxi - 1, m = nxi + 2;
    for (int e = tid; e < H * nxi; e += nt) {
        const int k = e / nxi, c = e % nxi;
        const double tau = (double)k / (double)(H - 1);
        double bin = 1.0;
        for (int q = 1; q <= c; ++q) bin = bin * (double)(deg - c + q) / (double)q;
        S->W64[e] = bin * pow(tau, (double)c) * pow(1.0 - tau, (double)(deg - c));
    }
    __syncthreads();
    for (int e = tid; e < nxi * nxi; e += nt) {
        const int u = e / nxi, v = e % nxi;
        double s = 0.0;
        for (int k = 0; k < H; ++k) s += S->W64[k * nxi + u] * S->W64[k * nxi + v];
        wtw[e] = s;
    }
    for (int pass = 0; pass < 2; ++pass) {
        const double c = pass == 0 ? (double)(n + n_obs + 2) : (double)(n_obs + 2);
        __syncthreads();
        for (int e = tid; e < m * m; e += nt) {
            const int r = e / m, q = e % m;
            double v;
            if (r < nxi && q < nxi) v = (r == q ? 1.0 : 0.0) + rho * c * wtw[r * nxi + q];
            else if (r < nxi) v = S->W64[(q == nxi ? 0 : H - 1) * nxi + r];
            else if (q < nxi) v = S->W64[(r == nxi ? 0 : H - 1) * nxi + q];
            else v = 0.0;
            K[e] = v;
            X[e] = r == q ? 1.0 : 0.0;
        }
        for (int p = 0; p < m; ++p) {
            __syncthreads();
            if (tid == 0) {
                int best = p;
                for (int r = p + 1; r < m; ++r)
                    if (fabs(K[r * m + p]) > fabs(K[best * m + p])) best = r;
                piv = best;
            }
            __syncthreads();
            const int b = piv;
            if (b != p)
                for (int q = tid; q < m; q += nt) {
                    double t = K[p * m + q]; K[p * m + q] = K[b * m + q]; K[b * m + q] = t;
                    t = X[p * m + q]; X[p * m + q] = X[b * m + q]; X[b * m + q] = t;
                }
            __syncthreads();
            const double d = K[p * m + p];
            __syncthreads();
            for (int q = tid; q < m; q += nt) {
                K[p * m + q] /= d;
                X[p * m + q] /= d;
            }
            __syncthreads();
            for (int e = tid; e < m * m; e += nt) {
                const int r = e / m, q = e % m;
                if (r == p) continue;
                const double f = K[r * m + p];
                if (q != p) K[r * m + q] -= f * K[p * m + q];
                X[r * m + q] -= f * X[p * m + q];
            }
            __syncthreads();
            for (int r = tid; r < m; r += nt)
                if (r != p) K[r * m + p] = 0.0;
        }
        __syncthreads();
        double *Pout = S->S64 + pass * nxi * nxi;
        double *Bout = S->S64 + 2 * nxi * nxi + pass * 2 * nxi;
        for (int e = tid; e < nxi * nxi; e += nt) Pout[e] = X[(e / nxi) * m + e % nxi];
        for (int e = tid; e < nxi * 2; e += nt) Bout[e] = X[(e / 2) * m + nxi + e % 2];
    }
    __syncthreads();
    for (int e = tid; e < H * nxi; e += nt) S->W32[e] = (float)S->W64[e];
    for (int e = tid; e < 2 * nxi * nxi + 4 * nxi; e += nt) S->S32[e] = (float)S->S64[e];
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
    if (!g_ready[dev]) {
        if (cudaGetSymbolAddress(&g_addr[dev], g_noalloc_scratch) != cudaSuccess) return SF_ECUDA;
        g_ready[dev] = true;
    }
    NaScratch *S = static_cast<NaScratch *>(g_addr[dev]);  // device address: pointer arithmetic only
    cudaStream_t st = (cudaStream_t)stream;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return SF_ECUDA;

    // launch geometry of the forward kernel (structured projection, FP32)
    int num_sms = 0;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SF_ECUDA;
    const int nd = n_d, nxi = n_xi, N = s.n * nxi;
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

    // instance table and shape record, written into the fixed array
    const int64_t per_xi = (int64_t)nd * s.n * nxi, per_bnd = (int64_t)nd * s.n * 2;
    const int64_t per_obs = (int64_t)s.n_obs * (s.dyn_obs ? s.H : 1) * nd, per_oab = (int64_t)s.n_obs * 2;
    for (int i = 0; i < n_inst; ++i) {
        Inst<float> &x = g_inst_host[i];
        memset(&x, 0, sizeof(x));
        x.n = s.n;
        x.n_obs = s.n_obs;
        x.H = s.H;
        x.dyn = s.dyn_obs;
        x.N = N;
        x.shape = 0;
        x.hc = hc;
        x.a = (float)s.a;
        x.b = (float)s.b;
        x.ia2 = (float)(1.0 / (s.a * s.a));
        x.ib2 = (float)(1.0 / (s.b * s.b));
        for (int ax = 0; ax < 3; ++ax) {
            x.pmin[ax] = (float)(ax < nd ? s.p_min[ax] : 0.0);
            x.pmax[ax] = (float)(ax < nd ? s.p_max[ax] : 0.0);
        }
        x.off_xi = i * per_xi;
        x.off_bnd = i * per_bnd;
        x.off_obs = i * per_obs;
        x.off_oab = i * per_oab;
    }
    memset(&g_shape_host, 0, sizeof(g_shape_host));
    g_shape_host.n = s.n;
    g_shape_host.n_obs = s.n_obs;
    g_shape_host.H = s.H;
    g_shape_host.N = N;
    // pageable host sources: each copy has read its source when the call returns
    if (cudaMemcpyAsync(S->inst, g_inst_host, sizeof(Inst<float>) * n_inst, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(&S->shape, &g_shape_host, sizeof(Shape), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(S->status, 0, sizeof(int32_t) * n_inst, st) != cudaSuccess)
        return SF_ECUDA;
    k_na_operators<<<1, 256, 0, st>>>(S, nxi, s.H, s.n, s.n_obs, rho);
    if (cudaGetLastError() != cudaSuccess) return SF_ECUDA;

    FwdArgs<float> a;
    memset(&a, 0, sizeof(a));
    a.nd = nd;
    a.nxi = nxi;
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
