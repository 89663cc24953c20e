// Hand-written adjoint of the unrolled SF iterations (the differentiable chain of T
// in Fig. unroll_learning and Sec. IV-B): the vector-Jacobian product with respect to
// the candidate xi and the initialisation (xi_bar^0, lambda^0).
//
// One thread-block cluster per instance, the same timestep split as the forward
// kernel.  The forward kept (xi_bar, lambda) every c iterations; segments are
// processed from the last to the first: the segment's iterates are recomputed with
// the forward's own code (stored per CTA in global scratch) and then reversed.
//
// Adjoint of one iteration l in correction form, xi_bar' = xi_bar + P_eta v +
// P_b (b - A xi_bar) with v = xi - xi_bar + lambda - 2 rho g (projection cost; the
// smoothness cost has -Q1 xi_bar per robot in place of xi - xi_bar) and lambda' =
// lambda - rho g, g = W'R(p), p = W xi_bar, from (xi_bar'*, lambda'*):
//   x*  = xi_bar'* with the coefficients A fixes cleared (they are overwritten by b)
//   v*  = P_eta x*                        (P_eta symmetric)
//   xi*      += v* (projection only),   lambda* = lambda'* + v*,   g* = -rho lambda'* - 2 rho v*
//   R*  = W g*;  p* = sum over active rows of J' (R*_i - R*_j) (pairs; J even, r_1 odd),
//                J' R*_i (obstacles), mask R*_i (box)
//   xi_bar*  = x* - v* (- Q1 v* per robot, smoothness) + W' p*
//              [- A' P_b' x* at l = 0: xi_bar^0 enters through b - A xi_bar^0]
// with J = dr_1/dDelta = (1 - s) I + s^3 Delta (M^-2 Delta)' on active rows and 0 on
// inactive ones (derivative conventions of the kinks: the clamped branch counts as
// active, Delta = 0 has zero derivative).
//
// The self-supervised loss of eq. NN_loss adds w sum_l ||z^{l+1} - z^l||^2 (z = (xi_bar,
// lambda), w = gfp per instance): reverse step l adds 2 w (z^{l+1} - z^l) to the adjoint
// of z^{l+1} before the step and subtracts it from the adjoint of z^l after it, so each
// step needs only its own pair of iterates (z^{l+1} carried in xq, lq from the step
// before; lambda of the recomputed iterates kept beside them in the segment scratch).
#pragma once
#include "sf_iter.cuh"

namespace sf {

template <typename T, int ND, int MAXT, bool TC, int NXI, int MODE>
__global__ void __launch_bounds__(MAXT) k_backward(BwdArgs<T> B)
{
    using VP = Vec<T, NDP<ND>::v>;
    const FwdArgs<T> &A = B.f;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    cg::cluster_group cl = cg::this_cluster();
    // C CTAs per instance; with instance groups a cluster of G C CTAs serves G instances
    const int C = A.csize, G = A.tcb > 0 ? A.tcb : 1, CC = G * C, crc = (int)cl.block_rank();
    const int grp = crc / C, cr = crc - grp * C;
    const int w = (blockIdx.x / CC) * G + grp;
    const int ii = A.order ? A.order[w] : w;
    const Inst<T> I0 = A.inst[ii];
    const BwdCarve cv = backward_carve(ND, NXI > 0 ? NXI : A.nxi, cta_rows(I0.H, A.csize), I0.n, I0.n_obs, I0.hc, A.p_rows, (int)sizeof(T), A.tc_mode,
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
    X.init(A, smem_raw, cv.f, ii, cr, C);
    X.set_group(grp, G, crc, CC);
    X.load_constants(A, A.p_rows);
    X.tc_setup(A, smem_raw);
    T *sm = reinterpret_cast<T *>(smem_raw);
    T *xs = sm + cv.xs, *ls = sm + cv.ls, *cs = sm + cv.cs, *xn = sm + cv.xn;
    T *xz = sm + cv.xz;   // xs with the end coefficients cleared: the next reverse step's x*
    T *xq = sm + cv.xq, *lq = sm + cv.lq;   // z^{l+1} of the reverse step (fixed-point seed)
    VP *Rs = reinterpret_cast<VP *>(sm + cv.Rs);
    const int tid = X.tid, nt = X.nt, NN = X.NN, nxi = X.nxi, N = X.N, n = X.n;
    const int64_t off = X.I.off_xi;
    const T rho = X.rho;
    for (int e = tid; e < NN; e += nt) {
        xs[e] = B.gxo ? B.gxo[off + e] : T(0);
        ls[e] = B.glo ? B.glo[off + e] : T(0);
        cs[e] = T(0);
    }
    const int Lit = A.iters, ce = A.ck_every;
    T *seg = B.seg + (off * C + (int64_t)cr * NN) * ce * 2;   // this CTA's copy of a segment's iterates
    T *segl = seg + (int64_t)ce * NN;                          // and of their multipliers
    int step = 0;                                         // parity of the all-reduce buffer
    const T wfp = B.gfp ? T(B.gfp[ii]) : T(0);            // weight of the fixed-point loss
    const bool fps = wfp != T(0);                         // block-uniform
    const bool need_l = ce > 1 || fps;                    // lambda of each iterate is read

    // seed from dL/d||r_p(xi_bar^L)||^2: gradient w r_1-weighted rows (w = 2 dL/d||r_p||^2);
    // with instance groups every instance of the cluster takes this branch (its barriers)
    // whenever the seed array is given, whatever its own weight
    const T wseed = B.grp2 ? T(2.0 * B.grp2[ii]) : T(0);
    if (wseed != T(0) || (G > 1 && B.grp2)) {
        for (int e = tid; e < NN; e += nt) X.xb[e] = A.ck_x[(int64_t)A.ck_final * A.ck_slot + off + e];
        T *gme = X.gp + (step & 1) * X.gstride;
        ++step;
        for (int e = tid; e < NN; e += nt) gme[e] = T(0);
        for (int k0 = X.k_lo; k0 < X.k_hi; k0 += X.hc) {
            const int hcc = min(X.hc, X.k_hi - k0);
            __syncthreads();
            X.begin_chunk();
            X.positions(k0, hcc, X.xb);
            X.sync_lists();
            X.cull_lists(k0, hcc);
            X.rows_adjoint(k0, hcc, Rs, wseed, true);
            __syncthreads();
            X.wt_acc(k0, hcc, X.Rb, gme);
        }
        cl.sync();
        for (int e = tid; e < NN; e += nt) {
            xs[e] += X.csum(cl, gme, e);
        }
    }
    for (int e = tid; e < NN; e += nt) {
        const int c = e - (e / nxi) * nxi;
        xz[e] = X.fixed_c(c) ? T(0) : xs[e];
        if (fps) {
            xq[e] = A.ck_x[(int64_t)A.ck_final * A.ck_slot + off + e];
            lq[e] = A.ck_l[(int64_t)A.ck_final * A.ck_slot + off + e];
        }
    }

    const int S = ce > 0 ? (Lit + ce - 1) / ce : 0;
    // The next segment's checkpoint is fetched into registers while the current segment
    // runs (lambda only when the segment has iterations to recompute).
    constexpr int kPF = 4;
    T pfx[kPF], pfl[kPF];
    auto fetch = [&](int sg) {
        const bool wl = need_l;
#pragma unroll
        for (int q = 0; q < kPF; ++q) {
            const int e = tid + q * nt;
            if (e < NN) {
                pfx[q] = A.ck_x[(int64_t)sg * A.ck_slot + off + e];
                if (wl) pfl[q] = A.ck_l[(int64_t)sg * A.ck_slot + off + e];
            }
        }
    };
    if (S > 0) fetch(S - 1);
    for (int sg = S - 1; sg >= 0; --sg) {
        const int l0 = sg * ce, l1 = min(Lit, l0 + ce);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kPF; ++q) {
            const int e = tid + q * nt;
            if (e < NN) {
                X.xb[e] = pfx[q];
                if (need_l) X.lam[e] = pfl[q];
            }
        }
        for (int e = tid + kPF * nt; e < NN; e += nt) {
            X.xb[e] = A.ck_x[(int64_t)sg * A.ck_slot + off + e];
            if (need_l) X.lam[e] = A.ck_l[(int64_t)sg * A.ck_slot + off + e];
        }
        if (sg > 0) fetch(sg - 1);
        if (sg == 0) X.boundary_gap();   // b - A xi_bar^0 for the first step's P_b term
        // recompute the segment's iterates x^l0 .. x^(l1-1) with the forward's code (the
        // reverse sweep needs the iterate each step started from, so x^l1 is not computed;
        // x^(l1-1) stays in xb, the earlier ones go to the segment scratch; with a checkpoint
        // every iteration nothing is recomputed)
        for (int l = l0; l + 1 < l1; ++l) {
            for (int e = tid; e < NN; e += nt) {
                seg[(int64_t)(l - l0) * NN + e] = X.xb[e];
                if (fps) segl[(int64_t)(l - l0) * NN + e] = X.lam[e];
            }
            T *gme = X.gp + (step & 1) * X.gstride;
            ++step;
            T rp2 = T(0), mx2 = T(0);
            X.rows_and_g(gme, rp2, mx2);
            cl.sync();
            X.update(cl, gme, X.need_b && l == 0);
        }
        if (fps)   // lambda of the segment's last iterate (the reverse step uses X.lam as scratch)
            for (int e = tid; e < NN; e += nt) segl[(int64_t)(l1 - 1 - l0) * NN + e] = X.lam[e];
        // reverse through the segment
        for (int l = l1 - 1; l >= l0; --l) {
            const T *xl = l + 1 == l1 ? X.xb : seg + (int64_t)(l - l0) * NN;
            const T *ll = segl + (int64_t)(l - l0) * NN;   // lambda^l (fixed-point seed only)
            T *vs = X.dd, *gs = X.lam;
            if (fps)   // the fixed-point term's share of z^{l+1}: + 2 w (z^{l+1} - z^l)
                for (int e = tid; e < NN; e += nt) {
                    const int c = e - (e / nxi) * nxi;
                    const T x = xs[e] + T(2) * wfp * (xq[e] - xl[e]);
                    xs[e] = x;
                    xz[e] = X.fixed_c(c) ? T(0) : x;
                    ls[e] += T(2) * wfp * (lq[e] - ll[e]);
                }
            __syncthreads();   // xz of the previous step's gather (or the seed) complete
            X.project(cl, xz, vs, false);
            if (X.smooth) __syncthreads();   // the cost block mixes a row's coefficients
            for (int e = tid; e < NN; e += nt) {
                const T vst = vs[e];
                gs[e] = -rho * ls[e] - T(2) * rho * vst;
                if (X.smooth) {   // d v / d xi_bar = -Q1 (symmetric); the candidate does not enter
                    const int r = e / nxi, c = e - r * nxi;
                    T qv = T(0);
                    for (int k = 0; k < nxi; ++k) qv += X.Qc[c * nxi + k] * vs[r * nxi + k];
                    xn[e] = xz[e] - qv;
                } else {          // d v / d xi_bar = -I, d v / d xi = I
                    xn[e] = xz[e] - vst;
                    cs[e] += vst;
                }
                ls[e] += vst;
            }
            if (l == 0) {   // - A' P_b' x*: xi_bar^0 enters through b - A xi_bar^0
                const int nbc = X.nbc, m = nbc * n;
                T *t = X.v;   // P_b' x* per (axis, robot, boundary row); v is free in the reverse sweep
                __syncthreads();
                for (int q2 = tid; q2 < ND * m; q2 += nt) {
                    const int ax = q2 / m, q = q2 - ax * m;
                    T s = T(0);
                    for (int r = 0; r < N; ++r) s += X.Pbg[(int64_t)r * m + q] * xz[ax * N + r];
                    t[q2] = s;
                }
                __syncthreads();
                for (int r = tid; r < ND * n; r += nt) {   // A' row by row: e_0, e_{n_xi - 1}, vsc (e_1 - e_0)
                    const T *tr = t + (int64_t)r * nbc;
                    T *x = xn + (int64_t)r * nxi;
                    x[0] -= tr[0];
                    x[nxi - 1] -= tr[1];
                    if (nbc == 3) {
                        x[1] -= X.vsc * tr[2];
                        x[0] += X.vsc * tr[2];
                    }
                }
            }
            T *gme = X.gp + (step & 1) * X.gstride;
            ++step;
            for (int e = tid; e < NN; e += nt) gme[e] = T(0);
            for (int k0 = X.k_lo; k0 < X.k_hi; k0 += X.hc) {
                const int hcc = min(X.hc, X.k_hi - k0);
                __syncthreads();
                X.begin_chunk();
                X.positions2(k0, hcc, xl, gs, Rs);
                X.sync_lists();
                X.cull_lists(k0, hcc);
                X.rows_adjoint(k0, hcc, Rs, T(0), false);
                __syncthreads();
                X.wt_acc(k0, hcc, X.Rb, gme);
            }
            cl.sync();
            for (int e = tid; e < NN; e += nt) {
                T x = xn[e] + X.csum(cl, gme, e);
                if (fps) {   // and its share of z^l: - 2 w (z^{l+1} - z^l); z^l becomes the next z^{l+1}
                    x -= T(2) * wfp * (xq[e] - xl[e]);
                    ls[e] -= T(2) * wfp * (lq[e] - ll[e]);
                    xq[e] = xl[e];
                    lq[e] = ll[e];
                }
                const int c = e - (e / nxi) * nxi;
                xs[e] = x;
                xz[e] = X.fixed_c(c) ? T(0) : x;
            }
        }
    }
    if (cr == 0) {
        for (int e = tid; e < NN; e += nt) {
            B.gxc[off + e] = cs[e] + (B.x0_null ? xs[e] : T(0));
            if (B.gx0) B.gx0[off + e] = xs[e];
            if (B.gl0) B.gl0[off + e] = ls[e];
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
static cudaError_t go_backward(const BwdArgs<T> &a, int nxi, int ni, int cs, int threads, size_t smem, cudaStream_t s)
{
    constexpr bool f32 = sizeof(T) == 4;
    const auto &f = a.f;
    if (f32 && nxi == 11 && f.nbc == 2 && f.cull && f.cost == SF_COST_PROJECTION) {
        if (f.proj == SF_PROJ_DENSE)
            return launch_cluster(k_backward<T, ND, MAXT, TC, f32 ? 11 : 0, f32 ? 2 : 0>, a, ni, cs, a.f.tcb, threads, smem, s);
        if (!TC) return launch_cluster(k_backward<T, ND, MAXT, TC, f32 ? 11 : 0, f32 ? 1 : 0>, a, ni, cs, a.f.tcb, threads, smem, s);
    }
    if (f32 && !TC && nxi == 11 && f.nbc == 2 && f.cull && f.cost == SF_COST_SMOOTHNESS && f.proj == SF_PROJ_STRUCTURED)
        return launch_cluster(k_backward<T, ND, MAXT, TC, f32 ? 11 : 0, f32 ? 3 : 0>, a, ni, cs, a.f.tcb, threads, smem, s);
    return launch_cluster(k_backward<T, ND, MAXT, TC, 0, 0>, a, ni, cs, a.f.tcb, threads, smem, s);
}

// Launch for one dimension: tensor-core projection or not, 512- or 1024-thread CTAs.
template <typename T, int ND>
cudaError_t launch_backward_nd(const BwdArgs<T> &a, int threads, size_t smem, cudaStream_t s)
{
    const FwdArgs<T> &f = a.f;
    constexpr int big = sizeof(T) == 8 ? 512 : 1024;
    constexpr bool tcok = sizeof(T) == 4;
    const int ni = f.n_inst, cs = f.csize, nx = f.nxi;
    if (f.tc_mode && tcok) {
        if (threads > 512) return go_backward<T, ND, big, tcok>(a, nx, ni, cs, threads, smem, s);
        return go_backward<T, ND, 512, tcok>(a, nx, ni, cs, threads, smem, s);
    }
    if (threads > 512) return go_backward<T, ND, big, false>(a, nx, ni, cs, threads, smem, s);
    return go_backward<T, ND, 512, false>(a, nx, ni, cs, threads, smem, s);
}

// Each (precision, dimension) is instantiated in a translation unit of its own.
extern template cudaError_t launch_backward_nd<float, 2>(const BwdArgs<float> &, int, size_t, cudaStream_t);
extern template cudaError_t launch_backward_nd<float, 3>(const BwdArgs<float> &, int, size_t, cudaStream_t);
extern template cudaError_t launch_backward_nd<double, 2>(const BwdArgs<double> &, int, size_t, cudaStream_t);
extern template cudaError_t launch_backward_nd<double, 3>(const BwdArgs<double> &, int, size_t, cudaStream_t);

template <typename T>
static cudaError_t launch_backward_t(const BwdArgs<T> &a, int threads, size_t smem, cudaStream_t s)
{
    const FwdArgs<T> &f = a.f;
    if (f.n_inst < 1 || f.csize < 1 || f.csize > kMaxCluster) return cudaErrorInvalidValue;
    if (threads > max_threads((int)sizeof(T))) return cudaErrorInvalidValue;
    if (f.nd == 2) return launch_backward_nd<T, 2>(a, threads, smem, s);
    return launch_backward_nd<T, 3>(a, threads, smem, s);
}

}  // namespace sf
