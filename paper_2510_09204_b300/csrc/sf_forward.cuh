// Persistent SF forward kernel.  Each instance is owned by one thread-block
// cluster of C CTAs that runs every iteration of T (eq. fixed_point) with the
// iterate, multipliers, candidate, basis and positions in shared memory.  CTA r
// of the cluster owns a contiguous share of the horizon's timesteps; the only
// exchange per iteration is the all-reduce of g = F'r_1 + G'r_2 through
// distributed shared memory (and, for the dense projection, the gather of the
// projected rows).  Every CTA then holds the same xi_bar and lambda.
//
// Per iteration, from (xi_bar, lambda):
//   positions   p = W xi_bar for this CTA's timesteps          (eq. poly)
//   rows        per (robot i, timestep k): every partner j and obstacle m gives a
//               line of sight Delta; the alpha/beta/d closed forms give e and the
//               row residual r_1 = Delta - e, summed with the sign of the incidence
//               row (F'); the box adds r_2 = max(0, p - p_max) - max(0, p_min - p) (G')
//                                                              (eqs. alpha_step..s_step)
//   g           = W' R over the cluster                       (structure of F, G)
//   lambda'     = lambda - rho g                                (eq. lambda_step)
//   xi_bar'     = xi_bar + P_eta (xi - xi_bar + lambda' - rho g) [+ P_b (b - A xi_bar)]
//                                                              (eq. xi_step)
// The xi_bar step is applied in correction form: with eta the paper's right-hand side
// and H = I + rho F'F + rho G'G, eta - H xi_bar = xi - xi_bar + lambda' - rho g and
// P_eta H + P_b A = I, so this equals P_eta eta + P_b b.
// The alpha/beta/d steps in algebraic form: with q = ||M^-1 Delta||, e = Delta when
// q >= 1 and e = Delta / q otherwise; Delta = 0 gives e = (a, 0) in 2D and (0, 0, b)
// in 3D for the row's own orientation (atan2(0, 0) = 0).
#pragma once
#include "sf_iter.cuh"

namespace sf {

template <typename T, int ND, int MAXT, bool TC, int NXI, int MODE>
__global__ void __launch_bounds__(MAXT) k_forward(FwdArgs<T> A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    cg::cluster_group cl = cg::this_cluster();
    // C CTAs per instance; with instance groups a cluster of G C CTAs serves G instances
    const int C = A.csize, G = A.tcb > 0 ? A.tcb : 1, CC = G * C, crc = (int)cl.block_rank();
    const int grp = crc / C, cr = crc - grp * C;
    const int w = (blockIdx.x / CC) * G + grp;
    const int ii = A.order ? A.order[w] : w;
    const Inst<T> I0 = A.inst[ii];
    const FwdCarve cv = forward_carve(ND, NXI > 0 ? NXI : A.nxi, cta_rows(I0.H, A.csize), I0.n, I0.n_obs, I0.hc, A.p_rows, (int)sizeof(T), A.tc_mode,
                                    tc_stage_arg(A.tc_mode, A.tcb, I0.n * A.nxi, A.csize, A.tc_res), A.cull);
#ifdef SF_BOUNDS_CHECK
    {   // the carve must fit the launch's dynamic shared memory (the same in every CTA)
        uint32_t dsm;
        asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsm));
        if ((uint64_t)cv.total * sizeof(T) > dsm) {
            if (threadIdx.x == 0) A.status[ii] = SF_EBOUNDS;
            return;
        }
    }
#endif
    Cta<T, ND, TC, NXI, MODE> X;
    X.init(A, smem_raw, cv, ii, cr, C);
    X.set_group(grp, G, crc, CC);
    X.load_constants(A, A.p_rows);
    X.tc_setup(A, smem_raw);
    const int tid = X.tid, nt = X.nt, NN = X.NN;
    const int64_t off = X.I.off_xi;
    const T *x0g = A.x0 ? A.x0 + off : A.xc + off;
    for (int e = tid; e < NN; e += nt) {
        X.xb[e] = x0g[e];
        X.lam[e] = A.l0 ? A.l0[off + e] : T(0);
    }
    X.boundary_gap();

    __shared__ int s_stop;   // early exit: the instance met the tolerance (set by the statistics warp)
    if (tid == 0) s_stop = 0;
    int its_tol = -1;
    T fp = T(0), fp_prev = T(0);
    double fp_sum = 0.0;   // sum over the iterations of ||z^{l+1} - z^l||^2
    bool bad = false;
    for (int it = 0; it <= A.iters; ++it) {
        const bool last = it == A.iters;   // the final pass only reduces the last fixed-point step
        T *gme = X.gp + (it & 1) * X.gstride;
        T rp2 = T(0), mx2 = T(0);
        if (!last) {
            if (cr == 0 && A.ck_every > 0 && it % A.ck_every == 0) {
                const int64_t base = (int64_t)(it / A.ck_every) * A.ck_slot + off;
                for (int e = tid; e < NN; e += nt) {
                    A.ck_x[base + e] = X.xb[e];
                    A.ck_l[base + e] = X.lam[e];
                }
            }
            X.rows_and_g(gme, rp2, mx2);
        }
        // per-warp partial stats (this iteration's rows, the previous iteration's step) into
        // gme[NN + 4 + 3 w ..]; after the cluster barrier one warp reduces them (off the
        // critical path: the CTA's last warp, after its share of the g gather in update())
        X.warp_partials(gme, rp2, mx2, fp);
        cl.sync();
        auto stats = [&]() {
            T s_rp2, s_mx2, s_fp;
            X.cluster_stats(cl, gme, s_rp2, s_mx2, s_fp);
            if ((tid & 31) == 0) {
                if (it > 0) {
                    fp_prev = s_fp;
                    fp_sum += (double)s_fp;
                    if (!isfinite(fp_prev)) bad = true;
                }
                if (!last) {
                    if (!isfinite(s_rp2)) bad = true;
                    const T mxr = sqrt(s_mx2);
                    if (its_tol < 0 && (double)mxr <= A.tol) {
                        its_tol = it;
                        if (A.early) s_stop = 1;   // every CTA of the instance takes the same decision
                    }
                    if (A.hist && cr == 0) A.hist[(int64_t)ii * A.iters + it] = (float)mxr;
                }
            }
        };
        if (last) {
            if (tid >> 5 == (nt >> 5) - 1) stats();
            break;
        }
        fp = X.update(cl, gme, X.need_b && it == 0, stats);
        if (s_stop) break;   // written before update()'s barrier; the output is the next iterate
    }
    const bool stat_thread = tid == nt - 32;   // lane 0 of the last warp holds the statistics
    if (cr == 0) {
        for (int e = tid; e < NN; e += nt) {
            A.xo[off + e] = X.xb[e];
            if (A.lo) A.lo[off + e] = X.lam[e];
        }
        if (A.ck_every > 0) {   // the final iterate, for the adjoint's residual seed
            const int64_t base = (int64_t)A.ck_final * A.ck_slot + off;
            for (int e = tid; e < NN; e += nt) {
                A.ck_x[base + e] = X.xb[e];
                A.ck_l[base + e] = X.lam[e];
            }
        }
        if (stat_thread) {
            if (A.resid) {
                A.resid[(int64_t)ii * SF_NRES + SF_RES_FP] = sqrt((double)fp_prev);
                A.resid[(int64_t)ii * SF_NRES + SF_RES_ITERS] = (double)its_tol;
                A.resid[(int64_t)ii * SF_NRES + SF_RES_FPSUM] = fp_sum;
            }
            if (A.its) A.its[ii] = its_tol;
            if (bad) A.status[ii] = SF_ENONFINITE;
        }
    }
#ifdef SF_BOUNDS_CHECK
    if (__syncthreads_or(X.oob) && tid == 0) A.status[ii] = SF_EBOUNDS;
#endif
    if (tid == 0 && X.tc_timed_out()) A.status[ii] = SF_ETIMEOUT;
    X.tc_teardown();
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

// The default configuration runs a kernel with its choices fixed at compile time (the
// code of the other choices compiled away): FP32, n_xi = 11, culled rows, the projection
// cost, and the structured (MODE 1) or dense (MODE 2) projection; the trajectory
// optimiser's default (the smoothness cost, structured) runs MODE 3.  Every other
// combination runs the generic kernel, whose choices are runtime flags.
template <typename T, int ND, int MAXT, bool TC>
static cudaError_t go_forward(const FwdArgs<T> &a, int nxi, int ni, int cs, int threads, size_t smem, cudaStream_t s)
{
    constexpr bool f32 = sizeof(T) == 4;
    const auto &f = a;
    if (f32 && nxi == 11 && f.nbc == 2 && f.cull && f.cost == SF_COST_PROJECTION) {
        if (f.proj == SF_PROJ_DENSE)
            return launch_cluster(k_forward<T, ND, MAXT, TC, f32 ? 11 : 0, f32 ? 2 : 0>, a, ni, cs, a.tcb, threads, smem, s);
        if (!TC) return launch_cluster(k_forward<T, ND, MAXT, TC, f32 ? 11 : 0, f32 ? 1 : 0>, a, ni, cs, a.tcb, threads, smem, s);
    }
    if (f32 && !TC && nxi == 11 && f.nbc == 2 && f.cull && f.cost == SF_COST_SMOOTHNESS && f.proj == SF_PROJ_STRUCTURED)
        return launch_cluster(k_forward<T, ND, MAXT, TC, f32 ? 11 : 0, f32 ? 3 : 0>, a, ni, cs, a.tcb, threads, smem, s);
    return launch_cluster(k_forward<T, ND, MAXT, TC, 0, 0>, a, ni, cs, a.tcb, threads, smem, s);
}

// Launch for one dimension: tensor-core projection or not, 512- or 1024-thread CTAs.
template <typename T, int ND>
cudaError_t launch_forward_nd(const FwdArgs<T> &a, int threads, size_t smem, cudaStream_t s)
{
    constexpr int big = sizeof(T) == 8 ? 512 : 1024;
    constexpr bool tcok = sizeof(T) == 4;
    const int ni = a.n_inst, cs = a.csize, nx = a.nxi;
    if (a.tc_mode && tcok) {
        if (threads > 512) return go_forward<T, ND, big, tcok>(a, nx, ni, cs, threads, smem, s);
        return go_forward<T, ND, 512, tcok>(a, nx, ni, cs, threads, smem, s);
    }
    if (threads > 512) return go_forward<T, ND, big, false>(a, nx, ni, cs, threads, smem, s);
    return go_forward<T, ND, 512, false>(a, nx, ni, cs, threads, smem, s);
}

// Each (precision, dimension) is instantiated in a translation unit of its own.
extern template cudaError_t launch_forward_nd<float, 2>(const FwdArgs<float> &, int, size_t, cudaStream_t);
extern template cudaError_t launch_forward_nd<float, 3>(const FwdArgs<float> &, int, size_t, cudaStream_t);
extern template cudaError_t launch_forward_nd<double, 2>(const FwdArgs<double> &, int, size_t, cudaStream_t);
extern template cudaError_t launch_forward_nd<double, 3>(const FwdArgs<double> &, int, size_t, cudaStream_t);

template <typename T>
static cudaError_t launch_forward_t(const FwdArgs<T> &a, int threads, size_t smem, cudaStream_t s)
{
    if (a.n_inst < 1 || a.csize < 1 || a.csize > kMaxCluster) return cudaErrorInvalidValue;
    if (threads > max_threads((int)sizeof(T))) return cudaErrorInvalidValue;
    if (a.nd == 2) return launch_forward_nd<T, 2>(a, threads, smem, s);
    return launch_forward_nd<T, 3>(a, threads, smem, s);
}

}  // namespace sf
