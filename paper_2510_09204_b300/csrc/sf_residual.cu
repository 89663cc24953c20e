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
    const int64_t fixed = residual_doubles(ND, nxi, H, n, nobs, 0);
    int hc = (int)((A.smem_doubles - fixed) / ((int64_t)n * NDP<ND>::v));
    // the same hc in every CTA of the cluster, so every CTA's carve (and the partial sums
    // that peers read through distributed shared memory) sits at the same offsets
    hc = max(1, min(hc, H));
    while (hc > 1 && residual_doubles(ND, nxi, H, n, nobs, hc) > A.smem_doubles) --hc;
    // carve in doubles, every region on a 32-byte boundary (mirrors residual_doubles)
    double *W = sm, *xb = W + carve_round((int64_t)H * nxi, 8);
    Vec<double, NDP<ND>::v> *P = reinterpret_cast<Vec<double, NDP<ND>::v> *>(xb + carve_round(NN, 8));
    double *ob = reinterpret_cast<double *>(P) + carve_round((int64_t)n * hc * NDP<ND>::v, 8);
    double *red = ob + carve_round((int64_t)nobs * 8, 8);
    Inst<double> Id;
    Id.n = n; Id.n_obs = nobs; Id.H = H; Id.dyn = I.dyn; Id.N = I.N; Id.hc = hc;
    Id.a = (double)I.a; Id.b = (double)I.b;
    Id.ia2 = 1.0 / (Id.a * Id.a); Id.ib2 = 1.0 / (Id.b * Id.b);
    for (int ax = 0; ax < 3; ++ax) { Id.pmin[ax] = (double)I.pmin[ax]; Id.pmax[ax] = (double)I.pmax[ax]; }
    for (int e = tid; e < H * nxi; e += nt) W[e] = A.W[S.off_W + e];
    for (int e = tid; e < NN; e += nt) xb[e] = (double)A.x[I.off_xi + e];
    for (int m = tid; m < nobs; m += nt) {
        const double ao = (double)A.oab[I.off_oab + 2 * m], bo = (double)A.oab[I.off_oab + 2 * m + 1];
        double *o = ob + 8 * m;
        for (int ax = 0; ax < 3; ++ax) o[ax] = (!I.dyn && ax < ND) ? (double)A.obs[I.off_obs + (int64_t)m * ND + ax] : 0.0;
        o[3] = ao * ao;
        o[4] = (ao * ao) / (bo * bo);
        o[5] = 1.0 / (ao * ao);
        o[6] = ao;
        o[7] = bo;
    }
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
                for (int c = 0; c < nxi; ++c) s += W[(k0 + kl) * nxi + c] * xb[(ax * n + i) * nxi + c];
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
            for (int m = 0; m < nobs; ++m) {
                const double *o = ob + 8 * m;
                double d[ND];
                if (I.dyn) {
                    const T *c = A.obs + I.off_obs + ((int64_t)m * H + k) * ND;
                    for (int ax = 0; ax < ND; ++ax) d[ax] = pi.v[ax] - (double)c[ax];
                } else {
                    for (int ax = 0; ax < ND; ++ax) d[ax] = pi.v[ax] - o[ax];
                }
                double q = d[0] * d[0] + d[1] * d[1];
                if (ND == 3) q += o[4] * d[ND - 1] * d[ND - 1];
                if (q <= o[3]) {
                    double t2[ND];
                    for (int ax = 0; ax < ND; ++ax) t2[ax] = 0.0;
                    if (ND == 2) t2[0] = -o[6]; else t2[ND - 1] = -o[7];
                    row_active<double, ND>(d, q, o[5], t2, R, rp2, mx2, true);
                }
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
        A.resid[(int64_t)ii * SF_NRES + SF_RES_RP] = sqrt(s_rp2);
        A.resid[(int64_t)ii * SF_NRES + SF_RES_MAX] = mx;
        const double itv = A.its_fixup ? A.resid[(int64_t)ii * SF_NRES + SF_RES_ITERS] : 0.0;
        if (itv < 0.0 && mx <= A.tol) {
            A.resid[(int64_t)ii * SF_NRES + SF_RES_ITERS] = (double)A.iters;
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
    if (a.nd == 2) return launch_cluster(k_residual<T, 2>, a, a.n_inst, a.csize, threads, smem, s);
    return launch_cluster(k_residual<T, 3>, a, a.n_inst, a.csize, threads, smem, s);
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
