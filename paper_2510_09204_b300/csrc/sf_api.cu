// C ABI of the SF solver: handle, validation, shape registry, factorisation and
// launches.  See include/sf.h for the contract of every call.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sf_internal.cuh"

using namespace sf;

namespace {

// NVTX range around a host entry point (visible in nsys / ncu timelines).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Simulated allocation failure for tests of the unwinding paths (no device fault): the
// environment variable SF_TEST_FAIL_ALLOC = k makes the (k+1)-th device allocation of
// the next sf_create on this thread fail as out of memory.  Unset: -1, no effect.
thread_local int t_fail_countdown = -1;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t alloc(size_t b)
    {
        bytes = b;
        if (b == 0) return cudaSuccess;
        if (t_fail_countdown == 0) {
            bytes = 0;
            return cudaErrorMemoryAllocation;
        }
        if (t_fail_countdown > 0) --t_fail_countdown;
        return cudaMalloc(&p, b);
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
};

struct SolveRecord {
    bool valid = false;
    const void *bnd = nullptr, *obs = nullptr, *oab = nullptr;
    const void *xc = nullptr, *x0 = nullptr, *l0 = nullptr;
    int iters = 0;
};

}  // namespace

struct sf_handle {
    sf_desc d{};
    std::vector<sf_shape> shp;
    int esz = 8;                       // sizeof(T)
    int nbc = 2;                       // boundary rows per robot and axis (3 with the initial velocity)
    int n_shapes = 0;
    std::vector<int> inst_shape;
    std::vector<Shape> shapes_h;
    std::vector<int64_t> off[4];       // SF_LAYOUT_* offsets, n_inst + 1 each
    std::vector<int> order;
    std::vector<int> hc;
    // device memory
    DevBuf inst_dev, shapes_dev, order_dev, status_dev;
    DevBuf W64, P64, Pb64, S64;        // FP64 factors
    DevBuf Wt, Pt, Pbt, St;            // in T (aliases of the FP64 pools when T = double)
    DevBuf ck_x, ck_l;
    DevBuf seg;                        // adjoint: recomputed iterates of a checkpoint segment
    DevBuf Wdd64;                      // second time derivative of the basis (metrics; dt > 0)
    DevBuf tcA, tcoff;                 // tensor-core chunks of P_eta for the current cluster size
    int tc_mode = 0, tc_c = 0;
    int cull_req = 1;                  // culled row loops (sf_set_option SF_OPT_CULL)
    int tcb_req = 1;                   // batched tensor-core projection when eligible (SF_OPT_TC_BATCH)
    int test_timeout = 0;              // SF_OPT_TEST_TIMEOUT: zero polling budget
    int early = 0;                     // SF_OPT_EARLY_EXIT
    int n_slots = 0;
    int64_t xi_total = 0;
    // launch configuration
    Plan plan;
    int smem_optin = 0;
    int num_sms = 0;
    SolveRecord last;
    cudaStream_t last_stream = nullptr;
    bool profile = false;
    cudaEvent_t ev[2 * SF_NKT] = {};
    bool ev_used[SF_NKT] = {};
};

// Geometry chosen by sf_autotune, keyed by the batch's shape signature.
static std::mutex g_tune_mu;
static std::map<std::vector<int64_t>, std::pair<int, int>> g_tune_cache;

static std::vector<int64_t> tune_key(const sf_desc &d, const std::vector<sf_shape> &shp)
{
    std::vector<int64_t> k = {d.n_d, d.n_xi, d.precision, d.proj, d.n_inst, d.ckpt_every > 0, d.n_bc == 3};
    for (const sf_shape &s : shp) {
        k.push_back(s.n);
        k.push_back(s.n_obs);
        k.push_back(s.H);
        k.push_back(s.dyn_obs);
    }
    return k;
}

static int plan_with_groups(const sf_handle *h, int B, const int *vn, const int *vo, const int *vH, int cluster,
                            int threads, Plan *p, int *hc);

static int cuda_status(cudaError_t e) { return e == cudaSuccess ? SF_OK : (e == cudaErrorMemoryAllocation ? SF_ENOMEM : SF_ECUDA); }

#define SF_TRY(expr)                                  \
    do {                                              \
        cudaError_t e_ = (expr);                      \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)


// Instances per cluster of the batched tensor-core projection for C CTAs per instance: the
// largest G >= 2 that divides the batch, with G C <= 16 CTAs, G n_d <= 16 MMA columns, at
// most 64 rows of P_eta per CTA, G n_d Lb <= n_d N (the rows fit the CTA's projection
// buffer) and the operator in tensor memory; 0 when none (BF16 and BF16 x3 with every
// instance of one shape only).
static int tcb_groups(int nd, int nxi, int esz, int tc_mode, int n_inst, const int *n, const int *nobs, const int *H, int C)
{
    if (esz != 4 || (tc_mode != 2 && tc_mode != 3) || n_inst < 2) return 0;
    for (int i = 1; i < n_inst; ++i)
        if (n[i] != n[0] || nobs[i] != nobs[0] || H[i] != H[0]) return 0;
    const int N = n[0] * nxi;
    if (tcb_tmem_cols(N) > 512) return 0;
    for (int G = std::min(n_inst, std::min(kMaxGroupCluster / C, 16 / nd)); G >= 2; --G) {
        const int Lb = tcb_rows(N, G * C);
        if (n_inst % G == 0 && Lb <= 64 && G * nd * Lb <= nd * N) return G;
    }
    return 0;
}

int sf::plan_forward(int nd, int nxi, int esz, int proj, int n_inst, const int *n, const int *nobs, const int *H,
                     int num_sms, int optin, int csize_req, int threads, Plan *out, int *hc_out, int tc_mode,
                     int cull_req, int need_bwd, int tcb_req)
{
    if (proj != SF_PROJ_DENSE) tc_mode = 0;
    Plan p;
    p.threads = threads;
    int minH = H[0];
    for (int i = 1; i < n_inst; ++i) minH = std::min(minH, H[i]);
    int C = csize_req > 0 ? csize_req : std::max(1, num_sms / std::max(1, n_inst));
    C = std::max(1, std::min(std::min(C, kMaxCluster), minH));
    p.csize = C;
    const int tcb = tcb_req ? tcb_groups(nd, nxi, esz, tc_mode, n_inst, n, nobs, H, C) : 0;
    p.tcb = tcb;
    const int st2 = tcb ? -1 : 2;   // the carves' A ring argument: two streaming stages, or groups
    // culled row loops when the candidate lists fit beside a chunk of at least 8 timesteps
    // (in the adjoint's carve too when the handle keeps checkpoints)
    int cull = cull_req ? 1 : 0;
    for (int i = 0; i < n_inst && cull; ++i) {
        const int h8 = std::min((H[i] + C - 1) / C, 8);
        const int64_t fb = forward_carve(nd, nxi, cta_rows(H[i], C), n[i], nobs[i], h8, 0, esz, tc_mode, st2, 1).total;
        const int64_t bb = need_bwd ? backward_carve(nd, nxi, cta_rows(H[i], C), n[i], nobs[i], h8, 0, esz, tc_mode, st2, 1).total : 0;
        const size_t b = (size_t)std::max(fb, bb) * esz;
        if (b > (size_t)optin || n[i] > 65535 - 8 || nobs[i] > 65535 - 8) cull = 0;
    }
    p.cull = cull;
    size_t need = 0, need_r = 0;
    int maxL = 0;
    bool res_ok = tc_mode != 0 && !tcb;
    std::vector<int> hc_res(n_inst, 1);
    for (int i = 0; i < n_inst; ++i) {
        const int own = (H[i] + C - 1) / C;
        int hc = own;
        if (tc_mode && !tcb && tc_ntiles(n[i] * nxi, C) > 8) return SF_EUNSUPPORTED;   // 8 x 128 rows per CTA at most
        // the forward's carve, or the larger adjoint carve when the handle keeps checkpoints
        auto bytes = [&](int h, int rows) {
            const int64_t f = forward_carve(nd, nxi, cta_rows(H[i], C), n[i], nobs[i], h, rows, esz, tc_mode, st2, cull).total;
            const int64_t b = need_bwd ? backward_carve(nd, nxi, cta_rows(H[i], C), n[i], nobs[i], h, rows, esz, tc_mode, st2, cull).total : 0;
            return (size_t)std::max(f, b) * esz;
        };
        while (hc > 1 && bytes(hc, 0) > (size_t)optin) --hc;
        if (bytes(hc, 0) > (size_t)optin) return SF_EUNSUPPORTED;
        if (tc_mode && !tcb) {   // resident projector chunks, if they fit with a chunk of at least 8 timesteps
            const int st = tc_stages(tc_mode, n[i] * nxi, C, 1);
            int hr = own;
            auto rbytes = [&](int h) {
                return (size_t)std::max(forward_carve(nd, nxi, cta_rows(H[i], C), n[i], nobs[i], h, 0, esz, tc_mode, st, cull).total,
                                        backward_carve(nd, nxi, cta_rows(H[i], C), n[i], nobs[i], h, 0, esz, tc_mode, st, cull).total) * esz;
            };
            while (hr > 1 && rbytes(hr) > (size_t)optin) --hr;
            if (rbytes(hr) > (size_t)optin || hr < std::min(own, 8)) res_ok = false;
            hc_res[i] = hr;
        }
        hc_out[i] = hc;
        need = std::max(need, bytes(hc, 0));
        maxL = std::max(maxL, (n[i] * nxi + C - 1) / C);
        // the residual check stages the obstacle records when they fit, else reads them from
        // global memory (it decides the same way from the shared memory it is given)
        const int wr = cta_rows(H[i], C);
        const int nob = residual_doubles(nd, nxi, wr, n[i], nobs[i], 1) * (int64_t)sizeof(double) <= optin ? nobs[i] : 0;
        if (residual_doubles(nd, nxi, wr, n[i], nob, 1) * (int64_t)sizeof(double) > optin) return SF_EUNSUPPORTED;
        need_r = std::max(need_r, (size_t)residual_doubles(nd, nxi, wr, n[i], nob, own) * sizeof(double));
    }
    if (proj == SF_PROJ_DENSE && !tc_mode) {
        size_t with_p = 0;
        for (int i = 0; i < n_inst; ++i) {
            with_p = std::max(with_p, (size_t)forward_carve(nd, nxi, cta_rows(H[i], C), n[i], nobs[i], hc_out[i], maxL, esz, 0, 2, cull).total * esz);
            if (need_bwd)
                with_p = std::max(with_p, (size_t)backward_carve(nd, nxi, cta_rows(H[i], C), n[i], nobs[i], hc_out[i], maxL, esz, 0, 2, cull).total * esz);
        }
        if (with_p <= (size_t)optin) {
            p.p_rows = maxL;
            need = with_p;
        }
    }
    if (res_ok) {
        p.tc_res = 1;
        need = 0;
        for (int i = 0; i < n_inst; ++i) {
            hc_out[i] = hc_res[i];
            need = std::max(need, (size_t)forward_carve(nd, nxi, cta_rows(H[i], C), n[i], nobs[i], hc_out[i], 0, esz, tc_mode,
                                                        tc_stages(tc_mode, n[i] * nxi, C, 1), cull).total * esz);
        }
    }
    p.smem_fwd = need;
    p.smem_res = std::min((size_t)optin, need_r);
    size_t need_b = 0;
    for (int i = 0; i < n_inst; ++i)
        need_b = std::max(need_b, (size_t)backward_carve(nd, nxi, cta_rows(H[i], C), n[i], nobs[i], hc_out[i], p.p_rows, esz, tc_mode,
                                                         tc_stage_arg(tc_mode, tcb, n[i] * nxi, C, p.tc_res), cull).total * esz);
    p.smem_bwd = need_b <= (size_t)optin ? need_b : 0;
    *out = p;
    return SF_OK;
}

static int validate(const sf_desc *d)
{
    if (!d || !d->shapes) return SF_EINVAL;
    if (d->n_d < 2 || d->n_d > 3 || d->n_xi < 4 || d->n_xi > 32) return SF_EINVAL;
    if (!(d->rho > 0.0) || !isfinite(d->rho) || d->n_inst < 1) return SF_EINVAL;
    if (d->precision < SF_FP64 || d->precision > SF_BF16) return SF_EINVAL;
    if (d->proj != SF_PROJ_DENSE && d->proj != SF_PROJ_STRUCTURED) return SF_EINVAL;
    if (d->max_iters < 0 || d->ckpt_every < 0 || d->n_refine < 0 || d->n_refine > 8 || !(d->tol >= 0.0)) return SF_EINVAL;
    if (d->cost != SF_COST_PROJECTION && d->cost != SF_COST_SMOOTHNESS) return SF_EINVAL;
    if (d->cost == SF_COST_SMOOTHNESS && (!(d->dt > 0.0) || !isfinite(d->dt) || d->n_xi < 3)) return SF_EINVAL;
    if (d->n_bc != 0 && d->n_bc != 2 && d->n_bc != 3) return SF_EINVAL;
    if (d->n_bc == 3 && (!(d->dt > 0.0) || !isfinite(d->dt) || d->n_xi < 5)) return SF_EINVAL;
    for (int i = 0; i < d->n_inst; ++i) {
        const sf_shape &s = d->shapes[i];
        if (s.n < 1 || s.n > 256 || s.n_obs < 0 || s.n_obs > 4096 || s.H < 2 || s.H > 4096) return SF_EINVAL;
        if (!(s.a > 0.0) || !(s.b > 0.0) || !isfinite(s.a) || !isfinite(s.b)) return SF_EINVAL;
        if (s.dyn_obs != 0 && s.dyn_obs != 1) return SF_EINVAL;
        for (int ax = 0; ax < d->n_d; ++ax)
            if (!isfinite(s.p_min[ax]) || !isfinite(s.p_max[ax]) || !(s.p_min[ax] <= s.p_max[ax])) return SF_EINVAL;
    }
    return SF_OK;
}

template <typename T>
static int upload_instances(sf_handle *h)
{
    const int nd = h->d.n_d;
    std::vector<Inst<T>> I(h->d.n_inst);
    for (int i = 0; i < h->d.n_inst; ++i) {
        const sf_shape &s = h->shp[i];
        Inst<T> &x = I[i];
        memset(&x, 0, sizeof(x));
        x.n = s.n;
        x.n_obs = s.n_obs;
        x.H = s.H;
        x.dyn = s.dyn_obs;
        x.N = s.n * h->d.n_xi;
        x.shape = h->inst_shape[i];
        x.hc = h->hc[i];
        x.a = (T)s.a;
        x.b = (T)s.b;
        x.ia2 = (T)(1.0 / (s.a * s.a));
        x.ib2 = (T)(1.0 / (s.b * s.b));
        for (int ax = 0; ax < 3; ++ax) {
            x.pmin[ax] = (T)(ax < nd ? s.p_min[ax] : 0.0);
            x.pmax[ax] = (T)(ax < nd ? s.p_max[ax] : 0.0);
        }
        x.off_xi = h->off[SF_LAYOUT_XI][i];
        x.off_bnd = h->off[SF_LAYOUT_BND][i];
        x.off_obs = h->off[SF_LAYOUT_OBS][i];
        x.off_oab = h->off[SF_LAYOUT_OBS_AB][i];
    }
    if (!h->inst_dev.p) SF_TRY(h->inst_dev.alloc(sizeof(Inst<T>) * I.size()));
    SF_TRY(cudaMemcpy(h->inst_dev.p, I.data(), sizeof(Inst<T>) * I.size(), cudaMemcpyHostToDevice));
    return SF_OK;
}

static void destroy_all(sf_handle *h)
{
    for (int k = 0; k < 2 * SF_NKT; ++k)
        if (h->ev[k]) {
            cudaEventDestroy(h->ev[k]);
            h->ev[k] = nullptr;
        }
    DevBuf *bufs[] = {&h->inst_dev, &h->shapes_dev, &h->order_dev, &h->status_dev, &h->W64, &h->P64,
                      &h->Pb64, &h->S64, &h->ck_x, &h->ck_l, &h->seg, &h->tcA, &h->tcoff, &h->Wdd64};
    if (h->esz == 4) {
        h->Wt.release();
        h->Pt.release();
        h->Pbt.release();
        h->St.release();
    }
    for (DevBuf *b : bufs) b->release();
}

// Bytes of the adjoint's segment scratch: per cluster CTA, a segment of recomputed
// iterates and their multipliers.
static size_t seg_bytes_of(const sf_handle *h)
{
    return (size_t)h->xi_total * h->plan.csize * h->d.ckpt_every * 2 * h->esz;
}

// Sizes the adjoint's segment scratch for the current plan, so that sf_solve_backward
// never allocates and can be captured in a CUDA graph.  Only grows.
static int ensure_seg(sf_handle *h)
{
    if (h->d.ckpt_every <= 0) return SF_OK;
    const size_t need = seg_bytes_of(h);
    if (h->seg.bytes >= need) return SF_OK;
    SF_TRY(cudaDeviceSynchronize());
    h->seg.release();
    SF_TRY(h->seg.alloc(need));
    return SF_OK;
}

// Event records are skipped while the stream is being captured into a graph.
static bool capturing(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// (Re)builds the tensor-core chunk pool for the plan's cluster size.
static int build_tc_pool(sf_handle *h, cudaStream_t st)
{
    if (!h->tc_mode || h->tc_c == h->plan.csize) return SF_OK;
    const int C = h->plan.csize;
    std::vector<int64_t> off(h->n_shapes);
    int64_t tot = 0;
    for (int i = 0; i < h->n_shapes; ++i) {
        off[i] = tot;
        tot += tc_pool_bytes(h->tc_mode, h->shapes_h[i].N, C);
    }
    SF_TRY(cudaStreamSynchronize(st));
    h->tcA.release();
    if (!h->tcoff.p) SF_TRY(h->tcoff.alloc(sizeof(int64_t) * h->n_shapes));
    SF_TRY(h->tcA.alloc((size_t)tot));
    SF_TRY(cudaMemcpy(h->tcoff.p, off.data(), sizeof(int64_t) * h->n_shapes, cudaMemcpyHostToDevice));
    SF_TRY(arrange_tc((const Shape *)h->shapes_dev.p, h->n_shapes, h->shapes_h.data(), (const double *)h->P64.p,
                      (const int64_t *)h->tcoff.p, off.data(), h->tc_mode, C, (unsigned char *)h->tcA.p, st));
    SF_TRY(cudaStreamSynchronize(st));
    h->tc_c = C;
    return SF_OK;
}

extern "C" int sf_create(const sf_desc *desc, sf_handle **out)
{
    NvtxRange nv("sf_create");
    {
        const char *fa = getenv("SF_TEST_FAIL_ALLOC");
        t_fail_countdown = fa ? atoi(fa) : -1;
    }
    struct CountdownOff {
        ~CountdownOff() { t_fail_countdown = -1; }
    } countdown_off;
    if (!out) return SF_EINVAL;
    *out = nullptr;
    int rc = validate(desc);
    if (rc) return rc;
    sf_handle *h = new (std::nothrow) sf_handle();
    if (!h) return SF_ENOMEM;
    h->d = *desc;
    h->shp.assign(desc->shapes, desc->shapes + desc->n_inst);
    h->d.shapes = nullptr;
    h->esz = desc->precision == SF_FP64 ? 8 : 4;
    h->nbc = desc->n_bc == 3 ? 3 : 2;
    h->tc_mode = desc->proj == SF_PROJ_DENSE ? tc_mode_of(desc->precision) : 0;
    const int nd = desc->n_d, nxi = desc->n_xi, B = desc->n_inst;
    cudaStream_t st = (cudaStream_t)desc->stream;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { delete h; return SF_ECUDA; }
    cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);

    // layouts
    for (int k = 0; k < 4; ++k) h->off[k].assign(B + 1, 0);
    for (int i = 0; i < B; ++i) {
        const sf_shape &s = h->shp[i];
        h->off[SF_LAYOUT_XI][i + 1] = h->off[SF_LAYOUT_XI][i] + (int64_t)nd * s.n * nxi;
        h->off[SF_LAYOUT_BND][i + 1] = h->off[SF_LAYOUT_BND][i] + (int64_t)nd * s.n * h->nbc;
        h->off[SF_LAYOUT_OBS][i + 1] = h->off[SF_LAYOUT_OBS][i] + (int64_t)s.n_obs * (s.dyn_obs ? s.H : 1) * nd;
        h->off[SF_LAYOUT_OBS_AB][i + 1] = h->off[SF_LAYOUT_OBS_AB][i] + (int64_t)s.n_obs * 2;
    }
    h->xi_total = h->off[SF_LAYOUT_XI][B];

    // distinct shapes
    std::map<std::tuple<int, int, int>, int> key;
    h->inst_shape.resize(B);
    int64_t oW = 0, oP = 0, oPb = 0, oS = 0;
    for (int i = 0; i < B; ++i) {
        const sf_shape &s = h->shp[i];
        auto k = std::make_tuple(s.n, s.n_obs, s.H);
        auto it = key.find(k);
        if (it == key.end()) {
            Shape S;
            S.n = s.n;
            S.n_obs = s.n_obs;
            S.H = s.H;
            S.N = s.n * nxi;
            S.nbc = h->nbc;
            S.pad_ = 0;
            S.vsc = h->nbc == 3 ? (double)(nxi - 1) / ((double)(s.H - 1) * desc->dt) : 0.0;
            S.off_W = oW;
            S.off_P = oP;
            S.off_Pb = oPb;
            S.off_S = oS;
            oW += (int64_t)s.H * nxi;
            oP += (int64_t)S.N * S.N;
            oPb += (int64_t)S.N * h->nbc * s.n;
            oS += kron_len(nxi, h->nbc);   // Kronecker blocks + cost block
            it = key.emplace(k, (int)h->shapes_h.size()).first;
            h->shapes_h.push_back(S);
        }
        h->inst_shape[i] = it->second;
    }
    h->n_shapes = (int)h->shapes_h.size();

    // launch geometry: cluster size, chunk of timesteps per instance, shared memory
    {
        std::vector<int> vn(B), vo(B), vH(B);
        for (int i = 0; i < B; ++i) {
            vn[i] = h->shp[i].n;
            vo[i] = h->shp[i].n_obs;
            vH[i] = h->shp[i].H;
        }
        h->hc.resize(B);
        int c0 = 0, t0 = kDefaultThreads;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(tune_key(h->d, h->shp));
            if (it != g_tune_cache.end()) {
                c0 = it->second.first;
                t0 = it->second.second;
            }
        }
        int prc = plan_with_groups(h, B, vn.data(), vo.data(), vH.data(), c0, t0, &h->plan, h->hc.data());
        if (prc && c0) prc = plan_with_groups(h, B, vn.data(), vo.data(), vH.data(), 0, kDefaultThreads, &h->plan, h->hc.data());
        if (prc) { destroy_all(h); delete h; return prc; }
    }

    // instance order: largest work first
    h->order.resize(B);
    for (int i = 0; i < B; ++i) h->order[i] = i;
    std::stable_sort(h->order.begin(), h->order.end(), [&](int x, int y) {
        auto cost = [&](int i) {
            const sf_shape &s = h->shp[i];
            return (double)s.H * ((double)s.n * (s.n - 1) + (double)s.n * s.n_obs);
        };
        return cost(x) > cost(y);
    });

    // device allocations
    int r;
    if ((r = cuda_status(h->shapes_dev.alloc(sizeof(Shape) * h->n_shapes))) ||
        (r = cuda_status(h->order_dev.alloc(sizeof(int) * B))) ||
        (r = cuda_status(h->status_dev.alloc(sizeof(int32_t) * B))) ||
        (r = cuda_status(h->W64.alloc(sizeof(double) * oW))) ||
        (r = cuda_status(h->P64.alloc(sizeof(double) * oP))) ||
        (r = cuda_status(h->Pb64.alloc(sizeof(double) * oPb))) ||
        (r = cuda_status(h->S64.alloc(sizeof(double) * oS)))) {
        destroy_all(h);
        delete h;
        return r;
    }
    if ((r = cuda_status(cudaMemcpy(h->shapes_dev.p, h->shapes_h.data(), sizeof(Shape) * h->n_shapes, cudaMemcpyHostToDevice))) ||
        (r = cuda_status(cudaMemcpy(h->order_dev.p, h->order.data(), sizeof(int) * B, cudaMemcpyHostToDevice))) ||
        (r = cuda_status(cudaMemset(h->status_dev.p, 0, sizeof(int32_t) * B)))) {
        destroy_all(h);
        delete h;
        return r;
    }
    r = h->esz == 8 ? upload_instances<double>(h) : upload_instances<float>(h);
    if (r) { destroy_all(h); delete h; return r; }

    // FP64 factorisation on the GPU
    {
        DevBuf scratch, info;
        if ((r = cuda_status(scratch.alloc(sizeof(double) * 3 * std::max<int64_t>(oP, 1)))) ||
            (r = cuda_status(info.alloc(sizeof(int) * h->n_shapes)))) {
            scratch.release();
            info.release();
            destroy_all(h);
            delete h;
            return r;
        }
        cudaMemsetAsync(info.p, 0, sizeof(int) * h->n_shapes, st);
        cudaError_t e = factor_shapes((const Shape *)h->shapes_dev.p, h->n_shapes, h->shapes_h.data(), nxi,
                                      desc->rho, desc->cost, desc->dt, (double *)h->W64.p, (double *)h->P64.p,
                                      (double *)h->Pb64.p,
                                      (double *)h->S64.p, (double *)scratch.p, 3 * oP, (int *)info.p, st, desc->proj == SF_PROJ_DENSE);
        std::vector<int> inf(h->n_shapes, 0);
        if (e == cudaSuccess && desc->dt > 0.0 && isfinite(desc->dt)) {   // basis'' for sf_metrics
            e = h->Wdd64.alloc(sizeof(double) * oW);
            if (e == cudaSuccess) e = basis_dd((const Shape *)h->shapes_dev.p, h->n_shapes, nxi, desc->dt,
                                               (double *)h->Wdd64.p, st);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = cudaMemcpy(inf.data(), info.p, sizeof(int) * h->n_shapes, cudaMemcpyDeviceToHost);
        scratch.release();
        info.release();
        if (e != cudaSuccess) { destroy_all(h); delete h; return cuda_status(e); }
        for (int v : inf)
            if (v) { destroy_all(h); delete h; return SF_EINVAL; }
    }
    if (h->esz == 8) {
        h->Wt = h->W64;
        h->Pt = h->P64;
        h->Pbt = h->Pb64;
        h->St = h->S64;
    } else {
        if ((r = cuda_status(h->Wt.alloc(sizeof(float) * oW))) || (r = cuda_status(h->Pt.alloc(sizeof(float) * oP))) ||
            (r = cuda_status(h->Pbt.alloc(sizeof(float) * oPb))) || (r = cuda_status(h->St.alloc(sizeof(float) * oS)))) {
            destroy_all(h);
            delete h;
            return r;
        }
        convert_pool((double *)h->W64.p, (float *)h->Wt.p, oW, st);
        convert_pool((double *)h->P64.p, (float *)h->Pt.p, oP, st);
        convert_pool((double *)h->Pb64.p, (float *)h->Pbt.p, oPb, st);
        convert_pool((double *)h->S64.p, (float *)h->St.p, oS, st);
        if ((r = cuda_status(cudaStreamSynchronize(st)))) { destroy_all(h); delete h; return r; }
    }
    if ((r = build_tc_pool(h, st))) { destroy_all(h); delete h; return r; }
    // checkpoints
    if (desc->ckpt_every > 0) {
        h->n_slots = desc->max_iters / desc->ckpt_every + 2;   // every c-th iterate, then the final one
        size_t b = (size_t)h->n_slots * h->xi_total * h->esz;
        if ((r = cuda_status(h->ck_x.alloc(b))) || (r = cuda_status(h->ck_l.alloc(b)))) {
            destroy_all(h);
            delete h;
            return r;
        }
    }
    if ((r = ensure_seg(h))) { destroy_all(h); delete h; return r; }
    *out = h;
    return SF_OK;
}

extern "C" int sf_destroy(sf_handle *h)
{
    if (!h) return SF_EINVAL;
    cudaDeviceSynchronize();
    destroy_all(h);
    delete h;
    return SF_OK;
}

extern "C" int sf_layout(const sf_handle *h, int32_t kind, int64_t *offsets)
{
    if (!h || !offsets || kind < 0 || kind > 3) return SF_EINVAL;
    memcpy(offsets, h->off[kind].data(), sizeof(int64_t) * (h->d.n_inst + 1));
    return SF_OK;
}

// The forward kernel's arguments for one solve (also the adjoint's view of that solve).
template <typename T>
static FwdArgs<T> fwd_args(const sf_handle *h, const void *bnd, const void *obs, const void *oab, const void *xc,
                           const void *x0, const void *l0, int iters)
{
    FwdArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.nd = h->d.n_d;
    a.nxi = h->d.n_xi;
    a.nbc = h->nbc;
    a.iters = iters;
    a.n_inst = h->d.n_inst;
    a.csize = h->plan.csize;
    a.p_rows = h->plan.p_rows;
    a.proj = h->d.proj;
    a.rho = (T)h->d.rho;
    a.tol = h->d.tol;
    a.inst = (const Inst<T> *)h->inst_dev.p;
    a.order = (const int *)h->order_dev.p;
    a.shapes = (const Shape *)h->shapes_dev.p;
    a.W = (const T *)h->Wt.p;
    a.P = (const T *)h->Pt.p;
    a.Pb = (const T *)h->Pbt.p;
    a.Sx = (const T *)h->St.p;
    a.xc = (const T *)xc;
    a.x0 = (const T *)x0;
    a.l0 = (const T *)l0;
    a.bnd = (const T *)bnd;
    a.obs = (const T *)obs;
    a.oab = (const T *)oab;
    a.status = (int32_t *)h->status_dev.p;
    a.tc_mode = h->tc_mode;
    a.tc_res = h->plan.tc_res;
    a.tcb = h->plan.tcb;
    a.cost = h->d.cost;
    a.wait_budget = h->test_timeout ? 0u : kWaitLimit;
    a.early = h->early && h->d.ckpt_every == 0 && !h->plan.tcb;
    a.cull = h->plan.cull;
    a.n_refine = h->tc_mode ? h->d.n_refine : 0;
    a.tcA = (const unsigned char *)h->tcA.p;
    a.tc_off = (const int64_t *)h->tcoff.p;
    if (h->d.ckpt_every > 0) {
        a.ck_x = (T *)h->ck_x.p;
        a.ck_l = (T *)h->ck_l.p;
        a.ck_every = h->d.ckpt_every;
        a.ck_final = h->n_slots - 1;
        a.ck_slot = h->xi_total;
    }
    return a;
}

template <typename T>
static int solve_t(sf_handle *h, const sf_instance_data *data, const void *xc, const void *x0, const void *l0,
                   int iters, void *xo, void *lo, double *resid, int32_t *its, cudaStream_t st)
{
    FwdArgs<T> a = fwd_args<T>(h, data->bnd, data->obs_c, data->obs_ab, xc, x0, l0, iters);
    a.xo = (T *)xo;
    a.lo = (T *)lo;
    a.resid = resid;
    a.its = its;
    const bool prof = h->profile && !capturing(st);
    if (prof)
        for (int k = 0; k < SF_NKT; ++k) h->ev_used[k] = false;
    if (prof) SF_TRY(cudaEventRecord(h->ev[0], st));
    SF_TRY(launch_forward(a, h->plan.threads, h->plan.smem_fwd, st));
    if (prof) {
        SF_TRY(cudaEventRecord(h->ev[1], st));
        h->ev_used[SF_KT_FORWARD] = true;
    }
    if (resid) {
        ResArgs<T> r;
        memset(&r, 0, sizeof(r));
        r.nd = a.nd;
        r.nxi = a.nxi;
        r.n_inst = a.n_inst;
        r.tol = a.tol;
        r.inst = a.inst;
        r.shapes = a.shapes;
        r.W = (const double *)h->W64.p;
        r.x = (const T *)xo;
        r.obs = a.obs;
        r.oab = a.oab;
        r.resid = resid;
        r.stride = SF_NRES;
        r.its = its;
        r.iters = iters;
        r.status = a.status;
        r.smem_doubles = (int64_t)(h->plan.smem_res / sizeof(double));
        r.csize = h->plan.csize;
        r.its_fixup = 1;
        if (prof) SF_TRY(cudaEventRecord(h->ev[2], st));
        SF_TRY(launch_residual(r, std::min(h->plan.threads, 512), h->plan.smem_res, st));
        if (prof) {
            SF_TRY(cudaEventRecord(h->ev[3], st));
            h->ev_used[SF_KT_RESIDUAL] = true;
        }
    }
    return SF_OK;
}

extern "C" int sf_solve(sf_handle *h, const sf_instance_data *data, const void *xi_cand, const void *xi0,
                        const void *lam0, int32_t iters, void *xi_out, void *lam_out, double *resid_out,
                        int32_t *iters_to_tol, void *stream)
{
    NvtxRange nv("sf_solve");
    if (!h || !data || !xi_cand || !xi_out || !data->bnd) return SF_EINVAL;
    if (iters < 0 || iters > h->d.max_iters) return SF_EINVAL;
    bool any_obs = h->off[SF_LAYOUT_OBS][h->d.n_inst] > 0;
    if (any_obs && (!data->obs_c || !data->obs_ab)) return SF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = h->esz == 8 ? solve_t<double>(h, data, xi_cand, xi0, lam0, iters, xi_out, lam_out, resid_out, iters_to_tol, st)
                         : solve_t<float>(h, data, xi_cand, xi0, lam0, iters, xi_out, lam_out, resid_out, iters_to_tol, st);
    if (rc) return rc;
    h->last_stream = st;
    h->last.valid = h->d.ckpt_every > 0;
    h->last.bnd = data->bnd;
    h->last.obs = data->obs_c;
    h->last.oab = data->obs_ab;
    h->last.xc = xi_cand;
    h->last.x0 = xi0;
    h->last.l0 = lam0;
    h->last.iters = iters;
    return SF_OK;
}

extern "C" int sf_solve_backward(sf_handle *h, const void *g_xi_out, const void *g_lam_out, const double *g_rp2,
                                 const double *g_fp, void *g_xi_cand, void *g_xi0, void *g_lam0, void *stream)
{
    NvtxRange nv("sf_solve_backward");
    if (!h || !g_xi_cand) return SF_EINVAL;
    if (!h->last.valid) return SF_ESTATE;
    if (!h->plan.smem_bwd) return SF_EUNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    if (h->seg.bytes < seg_bytes_of(h)) return SF_ESTATE;   // sized whenever the plan changes
    const bool prof = h->profile && !capturing(st);
    const SolveRecord &R = h->last;
    int rc;
    auto go = [&](auto tag) -> int {
        using T = decltype(tag);
        BwdArgs<T> b;
        memset(&b, 0, sizeof(b));
        b.f = fwd_args<T>(h, R.bnd, R.obs, R.oab, R.xc, R.x0, R.l0, R.iters);
        b.gxo = (const T *)g_xi_out;
        b.glo = (const T *)g_lam_out;
        b.grp2 = g_rp2;
        b.gfp = g_fp;
        b.gxc = (T *)g_xi_cand;
        b.gx0 = (T *)g_xi0;
        b.gl0 = (T *)g_lam0;
        b.seg = (T *)h->seg.p;
        b.x0_null = R.x0 == nullptr;
        if (prof) SF_TRY(cudaEventRecord(h->ev[2 * SF_KT_BACKWARD], st));
        SF_TRY(launch_backward(b, h->plan.threads, h->plan.smem_bwd, st));
        if (prof) {
            SF_TRY(cudaEventRecord(h->ev[2 * SF_KT_BACKWARD + 1], st));
            h->ev_used[SF_KT_BACKWARD] = true;
        }
        return SF_OK;
    };
    rc = h->esz == 8 ? go(double(0)) : go(float(0));
    if (rc) return rc;
    h->last_stream = st;
    return SF_OK;
}

// An empty kernel that only occupies what a CTA of the solver occupies (its threads and
// shared memory), for asking whether a cluster of that many CTAs can be resident at once.
__global__ void k_cluster_probe() {}

// True when a cluster of cdim CTAs of `threads` threads and `smem` bytes of shared memory
// each fits on the device (clusters above 8 CTAs are a non-portable size that the device
// may not offer).
static bool cluster_fits(int cdim, int threads, size_t smem)
{
    if (cdim <= kMaxCluster) return true;
    if (cudaFuncSetAttribute(k_cluster_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_cluster_probe, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cdim, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cdim;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_cluster_probe, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n >= 1;
}

// Plans with instance groups when they are asked for, eligible and fit on the device,
// else without them.
static int plan_with_groups(const sf_handle *h, int B, const int *vn, const int *vo, const int *vH, int cluster,
                            int threads, Plan *p, int *hc)
{
    int rc = plan_forward(h->d.n_d, h->d.n_xi, h->esz, h->d.proj, B, vn, vo, vH, h->num_sms, h->smem_optin, cluster,
                          threads, p, hc, h->tc_mode, h->cull_req, h->d.ckpt_every > 0, h->tcb_req);
    if (rc == SF_OK && p->tcb) {
        // tcgen05.alloc waits while the SM lacks free columns, so the CTAs that can share an
        // SM must not ask for more than its 512 together (else two CTAs of one cluster could
        // wait on each other): the shared-memory request bounds the CTAs per SM.
        int dev = 0, smem_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        const int per_sm = 512 / (int)tcb_tmem_cols(vn[0] * h->d.n_xi);
        const size_t floor_b = (size_t)smem_sm / (size_t)(per_sm + 1) + 1;
        p->smem_fwd = std::max(p->smem_fwd, floor_b);
        if (p->smem_bwd) p->smem_bwd = std::max(p->smem_bwd, floor_b);
        if (smem_sm <= 0 || p->smem_fwd > (size_t)h->smem_optin || p->smem_bwd > (size_t)h->smem_optin ||
            !cluster_fits(p->tcb * p->csize, p->threads, std::max(p->smem_fwd, p->smem_bwd)))
            rc = plan_forward(h->d.n_d, h->d.n_xi, h->esz, h->d.proj, B, vn, vo, vH, h->num_sms, h->smem_optin, cluster,
                              threads, p, hc, h->tc_mode, h->cull_req, h->d.ckpt_every > 0, 0);
    }
    return rc;
}

extern "C" int sf_set_launch(sf_handle *h, int32_t cluster, int32_t threads)
{
    if (!h || cluster < 0 || cluster > kMaxCluster || threads < 0 || threads > max_threads(h->esz) || threads % 32 ||
        (threads > 0 && threads < 64))
        return SF_EINVAL;
    const int B = h->d.n_inst;
    std::vector<int> vn(B), vo(B), vH(B), hc(B);
    for (int i = 0; i < B; ++i) {
        vn[i] = h->shp[i].n;
        vo[i] = h->shp[i].n_obs;
        vH[i] = h->shp[i].H;
    }
    Plan p;
    int rc = plan_with_groups(h, B, vn.data(), vo.data(), vH.data(), cluster, threads ? threads : kDefaultThreads, &p,
                              hc.data());
    if (rc) return rc;
    SF_TRY(cudaDeviceSynchronize());
    h->plan = p;
    h->hc = hc;
    if ((rc = build_tc_pool(h, (cudaStream_t)0))) return rc;
    if ((rc = ensure_seg(h))) return rc;
    return h->esz == 8 ? upload_instances<double>(h) : upload_instances<float>(h);
}

extern "C" int sf_autotune(sf_handle *h, const sf_instance_data *data, const void *xi_cand, int32_t iters,
                           int32_t reps, void *stream, int32_t *best_cluster, int32_t *best_threads, float *best_ms)
{
    NvtxRange nv("sf_autotune");
    if (!h || !data || !xi_cand || iters < 1 || iters > h->d.max_iters || reps < 1) return SF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)h->xi_total * h->esz;
    const bool bwd = h->d.ckpt_every > 0;   // a differentiable handle: time forward + adjoint
    DevBuf xo, lo, gxo, gxc;
    int r;
    if ((r = cuda_status(xo.alloc(bytes))) || (r = cuda_status(lo.alloc(bytes))) ||
        (bwd && ((r = cuda_status(gxo.alloc(bytes))) || (r = cuda_status(gxc.alloc(bytes)))))) {
        xo.release();
        lo.release();
        gxo.release();
        gxc.release();
        return r;
    }
    if (bwd && (r = cuda_status(cudaMemsetAsync(gxo.p, 0, bytes, st)))) {
        xo.release();
        lo.release();
        gxo.release();
        gxc.release();
        return r;
    }
    const Plan keep = h->plan;
    const std::vector<int> keep_hc = h->hc;
    const bool keep_prof = h->profile;
    h->profile = false;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const SolveRecord keep_last = h->last;
    int bc = keep.csize, bt = keep.threads;
    float bms = 1e30f;
    const int clusters[] = {1, 2, 4, 8}, threads[] = {128, 256, 512, 1024};
    for (int c : clusters)
        for (int t : threads) {
            if (t > max_threads(h->esz)) continue;
            if (sf_set_launch(h, c, t) != SF_OK) continue;
            float best = 1e30f;
            bool ok = true;
            for (int q = 0; q <= reps && ok; ++q) {   // the first run warms up
                cudaEventRecord(e0, st);
                ok = sf_solve(h, data, xi_cand, nullptr, nullptr, iters, xo.p, lo.p, nullptr, nullptr, st) == SF_OK;
                if (ok && bwd)
                    ok = sf_solve_backward(h, gxo.p, nullptr, nullptr, nullptr, gxc.p, nullptr, nullptr, st) == SF_OK;
                cudaEventRecord(e1, st);
                if (ok && cudaEventSynchronize(e1) == cudaSuccess && q > 0) {
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    best = std::min(best, ms);
                }
            }
            if (ok && best < bms) {
                bms = best;
                bc = c;
                bt = t;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    xo.release();
    lo.release();
    gxo.release();
    gxc.release();
    h->profile = keep_prof;
    h->last = keep_last;
    r = sf_set_launch(h, bc, bt);
    if (r) {
        h->plan = keep;
        h->hc = keep_hc;
        return r;
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[tune_key(h->d, h->shp)] = std::make_pair(bc, bt);
    }
    if (best_cluster) *best_cluster = bc;
    if (best_threads) *best_threads = bt;
    if (best_ms) *best_ms = bms;
    return SF_OK;
}

extern "C" int sf_get_launch(const sf_handle *h, int32_t *cluster, int32_t *threads, int32_t *p_rows)
{
    if (!h) return SF_EINVAL;
    if (cluster) *cluster = h->plan.csize;
    if (threads) *threads = h->plan.threads;
    if (p_rows) *p_rows = h->plan.p_rows;
    return SF_OK;
}

extern "C" int sf_metrics(sf_handle *h, const sf_instance_data *data, const void *xi, double *out, void *stream)
{
    NvtxRange nv("sf_metrics");
    if (!h || !data || !xi || !out || !data->bnd) return SF_EINVAL;
    if (!h->Wdd64.p) return SF_EINVAL;   // the handle was created without a time step
    const bool any_obs = h->off[SF_LAYOUT_OBS][h->d.n_inst] > 0;
    if (any_obs && (!data->obs_c || !data->obs_ab)) return SF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    auto go = [&](auto tag) -> int {
        using T = decltype(tag);
        ResArgs<T> r;
        memset(&r, 0, sizeof(r));
        r.nd = h->d.n_d;
        r.nxi = h->d.n_xi;
        r.n_inst = h->d.n_inst;
        r.tol = h->d.tol;
        r.inst = (const Inst<T> *)h->inst_dev.p;
        r.shapes = (const Shape *)h->shapes_dev.p;
        r.W = (const double *)h->W64.p;
        r.x = (const T *)xi;
        r.obs = (const T *)data->obs_c;
        r.oab = (const T *)data->obs_ab;
        r.resid = out;
        r.stride = 4;   // sf_metrics' [n_inst][4] output
        r.status = (int32_t *)h->status_dev.p;
        r.smem_doubles = (int64_t)(h->plan.smem_res / sizeof(double));
        r.csize = h->plan.csize;
        r.its_fixup = 0;
        SF_TRY(launch_residual(r, std::min(h->plan.threads, 512), h->plan.smem_res, st));
        SF_TRY(shape_metrics(r.inst, r.shapes, h->d.n_inst, h->d.n_d, h->d.n_xi, (const double *)h->W64.p,
                             (const double *)h->Wdd64.p, (const T *)xi, out, st));
        return SF_OK;
    };
    return h->esz == 8 ? go(double(0)) : go(float(0));
}

extern "C" int sf_set_option(sf_handle *h, int32_t option, int32_t value)
{
    if (!h) return SF_EINVAL;
    if (option == SF_OPT_TEST_TIMEOUT) {
        if (value != 0 && value != 1) return SF_EINVAL;
        h->test_timeout = value;
        return SF_OK;
    }
    if (option == SF_OPT_CULL) {
        if (value != 0 && value != 1) return SF_EINVAL;
        const int keep = h->cull_req;
        h->cull_req = value;
        const int rc = sf_set_launch(h, h->plan.csize, h->plan.threads);
        if (rc) h->cull_req = keep;
        return rc;
    }
    if (option == SF_OPT_EARLY_EXIT) {
        if (value != 0 && value != 1) return SF_EINVAL;
        if (value && h->d.ckpt_every > 0) return SF_EUNSUPPORTED;   // the adjoint needs every iteration
        h->early = value;
        return SF_OK;
    }
    if (option == SF_OPT_TC_BATCH) {
        if (value != 0 && value != 1) return SF_EINVAL;
        const int keep = h->tcb_req;
        h->tcb_req = value;
        const int rc = sf_set_launch(h, h->plan.csize, h->plan.threads);
        if (rc) h->tcb_req = keep;
        return rc;
    }
    return SF_EINVAL;
}

extern "C" int sf_get_option(const sf_handle *h, int32_t option, int32_t *value)
{
    if (!h || !value) return SF_EINVAL;
    if (option == SF_OPT_CULL) {
        *value = h->plan.cull;
        return SF_OK;
    }
    if (option == SF_OPT_TEST_TIMEOUT) {
        *value = h->test_timeout;
        return SF_OK;
    }
    if (option == SF_OPT_TC_RESIDENT) {
        *value = h->plan.tc_res;
        return SF_OK;
    }
    if (option == SF_OPT_TC_BATCH) {
        *value = h->plan.tcb;
        return SF_OK;
    }
    if (option == SF_OPT_EARLY_EXIT) {
        *value = h->early && !h->plan.tcb;
        return SF_OK;
    }
    return SF_EINVAL;
}

extern "C" int sf_profile(sf_handle *h, int32_t enable)
{
    if (!h) return SF_EINVAL;
    if (enable && !h->ev[0])
        for (int k = 0; k < 2 * SF_NKT; ++k) SF_TRY(cudaEventCreate(&h->ev[k]));
    h->profile = enable != 0;
    return SF_OK;
}

extern "C" int sf_kernel_times(sf_handle *h, float *ms_out)
{
    if (!h || !ms_out) return SF_EINVAL;
    if (!h->ev[0]) return SF_ESTATE;
    for (int k = 0; k < SF_NKT; ++k) {
        ms_out[k] = 0.0f;
        if (h->ev_used[k]) {
            SF_TRY(cudaEventSynchronize(h->ev[2 * k + 1]));
            SF_TRY(cudaEventElapsedTime(&ms_out[k], h->ev[2 * k], h->ev[2 * k + 1]));
        }
    }
    return SF_OK;
}

extern "C" int sf_get_status(sf_handle *h, int32_t *per_instance_status)
{
    if (!h || !per_instance_status) return SF_EINVAL;
    SF_TRY(cudaDeviceSynchronize());
    SF_TRY(cudaMemcpy(per_instance_status, h->status_dev.p, sizeof(int32_t) * h->d.n_inst, cudaMemcpyDeviceToHost));
    SF_TRY(cudaMemset(h->status_dev.p, 0, sizeof(int32_t) * h->d.n_inst));
    return SF_OK;
}

extern "C" int sf_shape_operator(const sf_handle *h, int32_t inst, int32_t which, double *host_out)
{
    if (!h || !host_out || inst < 0 || inst >= h->d.n_inst || which < 0 || which > 3) return SF_EINVAL;
    const Shape &S = h->shapes_h[h->inst_shape[inst]];
    const int nxi = h->d.n_xi;
    const double *src;
    size_t cnt;
    switch (which) {
    case 0: src = (const double *)h->W64.p + S.off_W; cnt = (size_t)S.H * nxi; break;
    case 1: src = (const double *)h->P64.p + S.off_P; cnt = (size_t)S.N * S.N; break;
    case 2: src = (const double *)h->Pb64.p + S.off_Pb; cnt = (size_t)S.N * S.nbc * S.n; break;
    default: src = (const double *)h->S64.p + S.off_S; cnt = (size_t)kron_len(nxi, S.nbc); break;
    }
    SF_TRY(cudaDeviceSynchronize());
    SF_TRY(cudaMemcpy(host_out, src, sizeof(double) * cnt, cudaMemcpyDeviceToHost));
    return SF_OK;
}

extern "C" const char *sf_strerror(int32_t code)
{
    switch (code) {
    case SF_OK: return "ok";
    case SF_EINVAL: return "invalid argument";
    case SF_ESHAPE: return "inconsistent shapes";
    case SF_ECUDA: return "CUDA runtime error";
    case SF_ENOMEM: return "out of memory";
    case SF_ETIMEOUT: return "bounded device wait ran out";
    case SF_ENONFINITE: return "non-finite value in an iterate";
    case SF_ESTATE: return "call order violated";
    case SF_EUNSUPPORTED: return "option not supported";
    case SF_ETOOBIG: return "size beyond the fixed limits of sf_solve_noalloc";
    case SF_EBOUNDS: return "device-side bounds check failed";
    default: return "unknown status";
    }
}

extern "C" int32_t sf_version(void) { return 200; }
