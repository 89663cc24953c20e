// FP64 residual check of a solve (its own translation unit).
#include "sf_iter.cuh"

namespace sf {

// FP64 residual of packed coefficients x (reading of eq. primal_residual):
// ||r_p||_2 and the max row residual in metres, whatever the solve precision.
// One cluster per instance, CTA r evaluating its share of the timesteps.
template <typename T, int ND>
__global__ void __launch_bounds__(512) k_residual(ResArgs<T> A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    double *sm = reinterpret_cast<double *>(smem_raw);
    cg::cluster_group cl = cg::this_cluster();
    const int tid = threadIdx.x, nt = blockDim.x, nxi = A.nxi;
    const int C = A.csize, cr = (int)cl.block_rank();
    const int ii = blockIdx.x / C;
    const Inst<T> I = A.inst[ii];
    const Shape S = A.shapes[I.shape];
    const int n = I.n, H = I.H, nobs = I.n_obs, NN = ND * I.N;
    const int k_lo = (int)((int64_t)cr * H / C), k_hi = (int)((int64_t)(cr + 1) * H / C);
    const int wrows = cta_rows(H, C);   // this CTA's rows of W
    // obstacle records staged in shared memory when they fit beside a one-step chunk, else
    // read from global memory in the row loop (the same for every CTA of the cluster)
    const bool staged = residual_doubles(ND, nxi, wrows, n, nobs, 1) <= A.smem_doubles;
    const int nob = staged ? nobs : 0;
    const int64_t fixed = residual_doubles(ND, nxi, wrows, n, nob, 0);
    int hc = (int)((A.smem_doubles - fixed) / ((int64_t)n * NDP<ND>::v));
    // the same hc in every CTA of the cluster, so every CTA's carve (and the partial sums
    // that peers read through distributed shared memory) sits at the same offsets
    hc = max(1, min(hc, H));
    while (hc > 1 && residual_doubles(ND, nxi, wrows, n, nob, hc) > A.smem_doubles) --hc;
    // carve in doubles, every region on a 32-byte boundary (mirrors residual_doubles)
    // W holds rows [k_lo, k_hi), addressed by the absolute timestep through Wk
    double *W = sm, *xb = W + carve_round((int64_t)wrows * nxi, 8);
    double *Wk = W - (int64_t)k_lo * nxi;
    Vec<double, NDP<ND>::v> *P = reinterpret_cast<Vec<double, NDP<ND>::v> *>(xb + carve_round(NN, 8));
    double *ob = reinterpret_cast<double *>(P) + carve_round((int64_t)n * hc * NDP<ND>::v, 8);
    double *red = ob + carve_round((int64_t)nob * 8, 8);
    Inst<double> Id;
    Id.n = n; Id.n_obs = nobs; Id.H = H; Id.dyn = I.dyn; Id.N = I.N; Id.hc = hc;
    Id.a = (double)I.a; Id.b = (double)I.b;
    Id.ia2 = 1.0 / (Id.a * Id.a); Id.ib2 = 1.0 / (Id.b * Id.b);
    for (int ax = 0; ax < 3; ++ax) { Id.pmin[ax] = (double)I.pmin[ax]; Id.pmax[ax] = (double)I.pmax[ax]; }
    for (int e = k_lo * nxi + tid; e < k_hi * nxi; e += nt) Wk[e] = A.W[S.off_W + e];
    for (int e = tid; e < NN; e += nt) xb[e] = (double)A.x[I.off_xi + e];
    // record of obstacle m: centre (static), a_o^2, a_o^2 / b_o^2, 1 / a_o^2, a_o, b_o
    auto record = [&](int m, double *o) {
        const double ao = (double)A.oab[I.off_oab + 2 * m], bo = (double)A.oab[I.off_oab + 2 * m + 1];
        for (int ax = 0; ax < 3; ++ax) o[ax] = (!I.dyn && ax < ND) ? (double)A.obs[I.off_obs + (int64_t)m * ND + ax] : 0.0;
        o[3] = ao * ao;
        o[4] = (ao * ao) / (bo * bo);
        o[5] = 1.0 / (ao * ao);
        o[6] = ao;
        o[7] = bo;
    };
    for (int m = tid; m < nob; m += nt) record(m, ob + 8 * m);
    // dynamic obstacle centres are read from global memory in the row loop; convert on the fly
    double rp2 = 0.0, mx2 = 0.0;
    const double a2 = Id.a * Id.a, kz = a2 * Id.ib2;
    for (int k0 = k_lo; k0 < k_hi; k0 += hc) {
        const int hcc = min(hc, k_hi - k0);
        __syncthreads();
        for (int e = tid; e < n * hcc; e += nt) {
            const int i = e / hcc, kl = e - i * hcc;
            Vec<double, NDP<ND>::v> p;
            for (int ax = 0; ax < NDP<ND>::v; ++ax) p.v[ax] = 0.0;
            for (int ax = 0; ax < ND; ++ax) {
                double s = 0.0;
                for (int c = 0; c < nxi; ++c) s += Wk[(k0 + kl) * nxi + c] * xb[(ax * n + i) * nxi + c];
                p.v[ax] = s;
            }
            P[i * hcc + kl] = p;
        }
        __syncthreads();
        for (int e = tid; e < n * hcc; e += nt) {
            const int i = e / hcc, kl = e - i * hcc, k = k0 + kl;
            const Vec<double, NDP<ND>::v> pi = P[i * hcc + kl];
            double R[ND], tie[ND];
            for (int ax = 0; ax < ND; ++ax) { R[ax] = 0.0; tie[ax] = 0.0; }
            if (ND == 2) tie[0] = -Id.a; else tie[ND - 1] = -Id.b;
            for (int j = i + 1; j < n; ++j) {
                const Vec<double, NDP<ND>::v> pj = P[j * hcc + kl];
                double d[ND];
                for (int ax = 0; ax < ND; ++ax) d[ax] = pi.v[ax] - pj.v[ax];
                const double q = qdist<double, ND>(d, kz);
                if (q <= a2) row_active<double, ND>(d, q, Id.ia2, tie, R, rp2, mx2, true);
            }
            // field j of obstacle m's record, from shared memory or computed from global memory
            auto obstacles = [&](auto field) {
                for (int m = 0; m < nobs; ++m) {
                    double d[ND];
                    if (I.dyn) {
                        const T *c = A.obs + I.off_obs + ((int64_t)m * H + k) * ND;
                        for (int ax = 0; ax < ND; ++ax) d[ax] = pi.v[ax] - (double)c[ax];
                    } else {
                        for (int ax = 0; ax < ND; ++ax) d[ax] = pi.v[ax] - field(m, ax);
                    }
                    double q = d[0] * d[0] + d[1] * d[1];
                    if (ND == 3) q += field(m, 4) * d[ND - 1] * d[ND - 1];
                    if (q <= field(m, 3)) {
                        double t2[ND];
                        for (int ax = 0; ax < ND; ++ax) t2[ax] = 0.0;
                        if (ND == 2) t2[0] = -field(m, 6); else t2[ND - 1] = -field(m, 7);
                        row_active<double, ND>(d, q, field(m, 5), t2, R, rp2, mx2, true);
                    }
                }
            };
            if (staged) {
                obstacles([&](int m, int j) { return ob[8 * m + j]; });
            } else {
                obstacles([&](int m, int j) {
                    double o[8];
                    record(m, o);
                    return o[j];
                });
            }
            for (int ax = 0; ax < ND; ++ax) {
                const double u = pi.v[ax] - Id.pmax[ax], l = Id.pmin[ax] - pi.v[ax];
                if (u > 0.0) { rp2 += u * u; mx2 = fmax(mx2, u * u); }
                if (l > 0.0) { rp2 += l * l; mx2 = fmax(mx2, l * l); }
            }
        }
    }
    block_reduce3_to<double>(rp2, mx2, 0.0, red);
    cl.sync();
    if (cr == 0 && tid == 0) {
        double s_rp2 = 0.0, s_mx2 = 0.0;
        for (int q = 0; q < C; ++q) {
            const double *rr = cl.map_shared_rank(red, q);
            s_rp2 += rr[96];
            s_mx2 = fmax(s_mx2, rr[97]);
        }
        const double mx = sqrt(s_mx2);
        A.resid[(int64_t)ii * A.stride + SF_RES_RP] = sqrt(s_rp2);
        A.resid[(int64_t)ii * A.stride + SF_RES_MAX] = mx;
        const double itv = A.its_fixup ? A.resid[(int64_t)ii * A.stride + SF_RES_ITERS] : 0.0;
        if (itv < 0.0 && mx <= A.tol) {
            A.resid[(int64_t)ii * A.stride + SF_RES_ITERS] = (double)A.iters;
            if (A.its) A.its[ii] = A.iters;
        }
        if (!isfinite(s_rp2)) A.status[ii] = SF_ENONFINITE;
    }
    cl.sync();
}

template <typename T>
static cudaError_t launch_residual_t(const ResArgs<T> &a, int threads, size_t smem, cudaStream_t s)
{
    if (a.n_inst < 1 || a.csize < 1 || a.csize > kMaxCluster) return cudaErrorInvalidValue;
    if (a.nd == 2) return launch_cluster(k_residual<T, 2>, a, a.n_inst, a.csize, 1, threads, smem, s);
    return launch_cluster(k_residual<T, 3>, a, a.n_inst, a.csize, 1, threads, smem, s);
}

cudaError_t launch_residual(const ResArgs<double> &a, int threads, size_t smem, cudaStream_t s)
{
    return launch_residual_t(a, threads, smem, s);
}
cudaError_t launch_residual(const ResArgs<float> &a, int threads, size_t smem, cudaStream_t s)
{
    return launch_residual_t(a, threads, smem, s);
}

}  // namespace sf
