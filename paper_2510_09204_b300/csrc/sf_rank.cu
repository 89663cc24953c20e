// Candidate ranking around the SF: trajectory metrics and per-group selection.
//
// The paper's pipeline samples many candidates per problem, keeps the few with the
// least constraint violation, refines them with the SF and returns the feasible one of
// least smoothness cost (Sec. V, the three stages of the planning pipeline).  Its quality
// metrics are the path length and the smoothness cost, the sum over timesteps of
// ||p''||^2 averaged across robots (Sec. V, Metrics).
#include <vector>

#include "sf_internal.cuh"

namespace sf {

// Second time derivative of the basis per shape, t_k = k dt: d (d - 1) / T^2 times the
// second difference of the degree-(d - 2) Bernstein polynomials, T = (H - 1) dt.
__global__ void k_basis_dd(const Shape *sh, int nxi, double dt, double *Wdd)
{
    const Shape S = sh[blockIdx.x];
    double *o = Wdd + S.off_W;
    const int deg = nxi - 1, H = S.H;
    const double T = (double)(H - 1) * dt, scale = (double)deg * (double)(deg - 1) / (T * T);
    for (int e = threadIdx.x; e < H * nxi; e += blockDim.x) {
        const int k = e / nxi, c = e % nxi;
        const double tau = (double)k / (double)(H - 1);
        double v = 0.0;
        for (int j = c - 2; j <= c; ++j) {
            if (j < 0 || j > deg - 2) continue;
            double bin = 1.0;
            for (int t = 1; t <= j; ++t) bin = bin * (double)(deg - 2 - j + t) / (double)t;
            v += (j == c - 1 ? -2.0 : 1.0) * bin * pow(tau, (double)j) * pow(1.0 - tau, (double)(deg - 2 - j));
        }
        o[e] = scale * v;
    }
}

cudaError_t basis_dd(const Shape *shapes_dev, int n_shapes, int nxi, double dt, double *Wdd, cudaStream_t s)
{
    k_basis_dd<<<n_shapes, 256, 0, s>>>(shapes_dev, nxi, dt, Wdd);
    return cudaGetLastError();
}

// One CTA per instance: out[ii][2] = smoothness (1/n) sum_i sum_k ||p''_{i|k}||^2,
// out[ii][3] = path length (1/n) sum_i sum_k ||p_{i|k+1} - p_{i|k}||, in FP64 with the FP64
// bases.  Each thread owns fixed (robot, timestep) items; the block sum is taken in a
// fixed order, so the result does not depend on scheduling.
template <typename T>
__global__ void k_shape_metrics(const Inst<T> *inst, const Shape *shapes, int nd, int nxi, const double *W,
                                const double *Wdd, const T *x, double *out)
{
    const int ii = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const Inst<T> I = inst[ii];
    const Shape S = shapes[I.shape];
    const int n = I.n, H = I.H;
    const double *Ws = W + S.off_W, *Wd = Wdd + S.off_W;
    const T *xi = x + I.off_xi;
    double sm = 0.0, pl = 0.0;
    for (int e = tid; e < n * H; e += nt) {
        const int i = e / H, k = e - i * H;
        double acc2 = 0.0, step2 = 0.0;
        for (int ax = 0; ax < nd; ++ax) {
            const T *xr = xi + ((int64_t)ax * n + i) * nxi;
            double a = 0.0, p0 = 0.0, p1 = 0.0;
            for (int c = 0; c < nxi; ++c) {
                const double xc = (double)xr[c];
                a += Wd[k * nxi + c] * xc;
                p0 += Ws[k * nxi + c] * xc;
                if (k + 1 < H) p1 += Ws[(k + 1) * nxi + c] * xc;
            }
            acc2 += a * a;
            step2 += (p1 - p0) * (p1 - p0);
        }
        sm += acc2;
        if (k + 1 < H) pl += sqrt(step2);
    }
    __shared__ double red[2][32];
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        sm += __shfl_xor_sync(0xffffffffu, sm, o);
        pl += __shfl_xor_sync(0xffffffffu, pl, o);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = sm;
        red[1][tid >> 5] = pl;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (nt >> 5); ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        out[(int64_t)ii * 4 + 2] = a / n;
        out[(int64_t)ii * 4 + 3] = b / n;
    }
}

cudaError_t shape_metrics(const Inst<double> *inst, const Shape *shapes, int n_inst, int nd, int nxi, const double *W,
                          const double *Wdd, const double *x, double *out, cudaStream_t s)
{
    k_shape_metrics<double><<<n_inst, 256, 0, s>>>(inst, shapes, nd, nxi, W, Wdd, x, out);
    return cudaGetLastError();
}
cudaError_t shape_metrics(const Inst<float> *inst, const Shape *shapes, int n_inst, int nd, int nxi, const double *W,
                          const double *Wdd, const float *x, double *out, cudaStream_t s)
{
    k_shape_metrics<float><<<n_inst, 256, 0, s>>>(inst, shapes, nd, nxi, W, Wdd, x, out);
    return cudaGetLastError();
}

// Per group (one CTA): the k best candidates in order.  A candidate is feasible when its
// primary score is <= threshold; feasible ones come first, ordered by the secondary score
// (or the primary when there is none), then the rest by the primary score; ties go to the
// lower index.  k rounds of a block-wide arg-min over the candidates not yet taken.
constexpr int kSelMax = 4096;

struct Key {
    int feas;      // 0 feasible, 1 not
    double v;
    int idx;
};

__device__ __forceinline__ bool key_less(const Key &a, const Key &b)
{
    if (a.feas != b.feas) return a.feas < b.feas;
    if (a.v != b.v) return a.v < b.v;
    return a.idx < b.idx;
}

__global__ void k_select(const int64_t *goff, const int *gsize, const double *primary, const double *secondary,
                         double threshold, int k, int *out)
{
    const int g = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int m = gsize[g];
    const double *p = primary + goff[g];
    const double *q = secondary ? secondary + goff[g] : nullptr;
    __shared__ unsigned char taken[kSelMax];
    __shared__ Key best[32];
    for (int j = tid; j < m; j += nt) taken[j] = 0;
    __syncthreads();
    for (int r = 0; r < k; ++r) {
        Key mine{2, 0.0, 0x7fffffff};
        for (int j = tid; j < m; j += nt) {
            if (taken[j]) continue;
            const double pv = p[j];
            // NaN scores sort last (never feasible, after every finite value)
            const bool ok = pv <= threshold;
            Key c{ok ? 0 : 1, ok ? (q ? q[j] : pv) : pv, j};
            if (!(c.v == c.v)) { c.feas = 2; c.v = 0.0; }
            if (key_less(c, mine)) mine = c;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            Key other;
            other.feas = __shfl_xor_sync(0xffffffffu, mine.feas, o);
            other.v = __shfl_xor_sync(0xffffffffu, mine.v, o);
            other.idx = __shfl_xor_sync(0xffffffffu, mine.idx, o);
            if (key_less(other, mine)) mine = other;
        }
        if ((tid & 31) == 0) best[tid >> 5] = mine;
        __syncthreads();
        if (tid == 0) {
            Key b = best[0];
            for (int w = 1; w < (nt >> 5); ++w)
                if (key_less(best[w], b)) b = best[w];
            const bool any = b.idx < m;
            out[(int64_t)g * k + r] = any ? b.idx : -1;
            if (any) taken[b.idx] = 1;
        }
        __syncthreads();
    }
}

}  // namespace sf

using namespace sf;

extern "C" int sf_select(int32_t n_groups, const int32_t *group_size, const double *primary, const double *secondary,
                         double threshold, int32_t k, int32_t *out_idx, void *stream)
{
    if (n_groups < 1 || !group_size || !primary || !out_idx || k < 1 || k > kSelMax) return SF_EINVAL;
    std::vector<int64_t> off(n_groups);
    std::vector<int> sz(n_groups);
    int64_t o = 0;
    for (int g = 0; g < n_groups; ++g) {
        if (group_size[g] < 0 || group_size[g] > kSelMax) return SF_EINVAL;
        off[g] = o;
        sz[g] = group_size[g];
        o += group_size[g];
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *scr = nullptr;
    const size_t b64 = sizeof(int64_t) * n_groups, b32 = sizeof(int) * n_groups;
    if (cudaMallocAsync((void **)&scr, b64 + b32 + 16, st) != cudaSuccess) return SF_ENOMEM;
    int rc = SF_OK;
    // pageable sources: each copy has read its host buffer when the call returns
    if (cudaMemcpyAsync(scr, off.data(), b64, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(scr + b64, sz.data(), b32, cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = SF_ECUDA;
    if (rc == SF_OK) {
        k_select<<<n_groups, 256, 0, st>>>((const int64_t *)scr, (const int *)(scr + b64), primary, secondary,
                                           threshold, k, out_idx);
        if (cudaGetLastError() != cudaSuccess) rc = SF_ECUDA;
    }
    cudaFreeAsync(scr, st);
    return rc;
}
