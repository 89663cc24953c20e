// Device pieces of one SF iteration shared by the forward and the adjoint kernels.
//
// An instance is owned by a thread-block cluster of C CTAs; CTA r takes a contiguous
// share [k_lo, k_hi) of the H timesteps and keeps a full copy of the iterate.  The
// phases of an iteration (positions, constraint rows, the W' aggregation, the
// cluster all-reduce through distributed shared memory, the multiplier step and the
// projection) are methods of Cta so that the adjoint kernel recomputes checkpoint
// segments with exactly the forward's arithmetic.
#pragma once
#include <cooperative_groups.h>
#include <math.h>

#include <cuda_bf16.h>

#include "sf_internal.cuh"
#include "sf_tc.cuh"

namespace sf {

namespace cg = cooperative_groups;


template <typename T> __device__ __forceinline__ T rsq(T x);
template <> __device__ __forceinline__ float rsq<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsq<double>(double x) { return 1.0 / sqrt(x); }

template <typename T, int K>
struct alignas(K * sizeof(T) >= 16 ? 16 : K * sizeof(T)) Vec {
    T v[K];
};

template <int ND> struct NDP { static constexpr int v = ND == 2 ? 2 : 4; };

// Far-away stand-ins: padded robots sit at +kFar, lanes without an item at -kFar, so
// every distance test against them fails without a bounds check.
template <typename T> struct Far { static constexpr T v = T(1e15); };

// An active row (q <= a^2): r_1 = Delta (1 - 1/||M^-1 Delta||), or the tie value tie
// when Delta = 0.  Adds r_1 to R, its squared norm to rp2 (if count) and to the max.
template <typename T, int ND>
__device__ __forceinline__ void row_active(const T (&d)[ND], T q, T ia2, const T (&tie)[ND], T (&R)[ND], T &rp2,
                                           T &mx2, bool count)
{
    T r1[ND];
    if (q > T(0)) {
        const T f = T(1) - rsq(q * ia2);
#pragma unroll
        for (int ax = 0; ax < ND; ++ax) r1[ax] = d[ax] * f;
    } else {
#pragma unroll
        for (int ax = 0; ax < ND; ++ax) r1[ax] = tie[ax];
    }
    T nn = T(0);
#pragma unroll
    for (int ax = 0; ax < ND; ++ax) {
        R[ax] += r1[ax];
        nn += r1[ax] * r1[ax];
    }
    if (count) rp2 += nn;
    mx2 = fmax(mx2, nn);
}

// Transposed Jacobian of an active row (q > 0): with s = 1/||M^-1 d||,
// r_1(d) = d (1 - s) and dr_1/dd = (1 - s) I + s^3 d (M^-2 d)'.  Adds J' y to out.
// mode 0: y given; mode 1: y = w r_1(d) (gradient of w ||r_1||^2 / 2, times 2 by the caller).
template <typename T, int ND>
__device__ __forceinline__ void row_adjoint(const T (&d)[ND], T q, T ia2, T ib2, const T (&y_in)[ND], T w, bool seed,
                                            T (&out)[ND])
{
    if (!(q > T(0))) return;   // Delta = 0: the row's e is constant there (zero derivative)
    const T s = rsq(q * ia2), f = T(1) - s;
    T y[ND];
#pragma unroll
    for (int ax = 0; ax < ND; ++ax) y[ax] = seed ? w * d[ax] * f : y_in[ax];
    T dy = T(0);
#pragma unroll
    for (int ax = 0; ax < ND; ++ax) dy += d[ax] * y[ax];
    const T s3dy = s * s * s * dy;
#pragma unroll
    for (int ax = 0; ax < ND; ++ax) out[ax] += f * y[ax] + s3dy * d[ax] * (ax == 2 ? ib2 : ia2);
}

// e / d for 0 <= e < 2^22 and 1 <= d < 2^22 without an integer division: e times the
// rounded reciprocal of d is within 2^22 * 2^-23 < 1 of the quotient, so its truncation
// is off by at most one, which the remainder test corrects.
struct FDiv {
    int d;
    float r;
    __device__ __forceinline__ void set(int dd)
    {
        d = dd;
        r = 1.0f / (float)dd;
    }
    __device__ __forceinline__ int q(int e) const
    {
        const int x = __float2int_rz((float)e * r);
        const int m = e - x * d;
        return x + (m >= d ? 1 : 0) - (m < 0 ? 1 : 0);
    }
};

// squared scaled distance: dx^2 + dy^2 + kz dz^2 with kz = a^2 / b^2
template <typename T, int ND>
__device__ __forceinline__ T qdist(const T (&d)[ND], T kz)
{
    T q = d[0] * d[0] + d[1] * d[1];
    if (ND == 3) q += kz * d[ND - 1] * d[ND - 1];
    return q;
}

// Warp then block reduction of (sum, max, sum) into red[96..98] (the result is valid
// after the caller's next barrier).
template <typename T>
__device__ __forceinline__ void block_reduce3_to(T a, T b, T c, T *red)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    if (l == 0) {
        red[w] = a;
        red[32 + w] = b;
        red[64 + w] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        T x = T(0), y = T(0), z = T(0);
        for (int q = 0; q < nw; ++q) {
            x += red[q];
            y = fmax(y, red[32 + q]);
            z += red[64 + q];
        }
        red[96] = x;
        red[97] = y;
        red[98] = z;
    }
}

// TC: compile in the tensor-core projection (FP32 only); other instantiations stay lean.
// NXI > 0: the coefficient count fixed at compile time (loops over it unroll, divisions by
// it become multiplications); 0: taken from the arguments.  MODE 0: the projection form,
// culling and cost are runtime flags; MODE 1 / 2: fixed to culled rows with the
// projection cost and the structured (1) or dense (2) projection; MODE 3: culled rows, the
// structured projection and the smoothness cost (the trajectory optimiser).
template <typename T, int ND, bool TC = false, int NXI = 0, int MODE = 0>
struct Cta {
    using VP = Vec<T, NDP<ND>::v>;
    int tid, nt, C, cr, nxi, n, npad, H, N, NN, nobs, opad, hc, k_lo, k_hi, L, r_lo, r_hi, ii;
    bool dense;
    T rho, invn;
    Inst<T> I;
    Shape S;
    T *W, *xb, *lam, *xc, *v, *gp, *dl, *dd, *rr, *wtw, *Rb, *ob, *bd, *db, *bf, *sx, *red, *Ps;
    int n_refine, n_obs_;
    int nbc;          // boundary rows per robot and axis (2, or 3 with the initial velocity)
    T vsc;            // velocity row p'(0) = vsc (xi_1 - xi_0)
    VP *P;
    const T *Prow, *Pbg, *obs_g;
    int64_t gstride;
    T *Pdev, *Pdif, *Bdev, *Bdif, *mv, *pm, *mb;
    T *Qc;            // per-robot cost block of the smoothness cost (n_xi x n_xi)
    int smooth;       // the trajectory optimiser's smoothness cost instead of the projection
    int need_b;
    // culled row loops: boxes, candidate lists (partners, obstacles) and their counts
    T *bbx, *osa;
    unsigned short *lpl, *lol;
    int *lcn;
    int cull, LPs, LOs, NBX;
    FDiv fn, fN, fL;  // divisions by n, N and L
    int lv, need;     // lists valid for the current chunk; rebuild asked (block-uniform)
    int oob;          // a bounds check failed in this thread (builds with SF_BOUNDS_CHECK)
    bool esc;         // this thread saw a position outside its robot's inflated box
    T cdel;           // inflation of the robots' boxes
    // tensor-core projection (FP32 kernels, dense mode)
    int tcm, tc_nK, tc_nT, tc_na, tc_es, tc_bbytes, tc_sbo_b, tc_res;
    uint32_t wbud;             // polls of a pipeline wait; the teardown's drain always uses kWaitLimit
    unsigned char *tc_ring, *tc_B;
    uint64_t *tc_bar;          // full[2], empty[2], done
    int *tc_flag;              // sticky failure flag
    uint32_t *tc_slot;         // tensor-memory address written by tcgen05.alloc
    // per ring stage s: full-barrier phases waited (fw), loads issued (ld), MMA commits (ec);
    // scalars, not arrays, so that a runtime stage index keeps the object in registers
    uint32_t tmem_base, tmem_cols, tc_done, tc_seen, tc_fw0, tc_fw1, tc_ld0, tc_ld1, tc_ec0, tc_ec1;
    const unsigned char *tc_src;
    // instance groups (batched tensor-core projection): gb is the cluster rank of this
    // instance's first CTA (0 outside groups), crc this CTA's rank among the cluster's CC
    // CTAs, G the instances per cluster, grp this instance's group; the CTA keeps rows
    // [tb_rl, tb_rh) of P_eta (Lb per CTA) in tensor memory
    int gb, CC, crc, G, grp, tcb, Lb, tb_rl, tb_rh, tb_kp, tb_dcol;
    unsigned char *tb_Bh;
    float *tb_stage;
    FDiv fLb;

    __device__ __forceinline__ void init(const FwdArgs<T> &A, unsigned char *smem_raw, const FwdCarve &cv, int inst, int rank, int csize)
    {
        T *sm = reinterpret_cast<T *>(smem_raw);
        tid = threadIdx.x;
        nt = blockDim.x;
        C = csize;
        cr = rank;
        ii = inst;
        nxi = NXI > 0 ? NXI : A.nxi;   // a compile-time constant in the specialised kernels
        I = A.inst[ii];
        S = A.shapes[I.shape];
        n = I.n;
        npad = (n + 3) & ~3;
        H = I.H;
        N = I.N;
        NN = ND * N;
        nobs = I.n_obs;
        opad = (nobs + 3) & ~3;
        hc = I.hc;
        rho = A.rho;
        invn = T(1) / T(n);
        dense = MODE == 2 ? true : (MODE == 1 || MODE == 3) ? false : A.proj == SF_PROJ_DENSE;
        k_lo = (int)((int64_t)cr * H / C);
        k_hi = (int)((int64_t)(cr + 1) * H / C);
        L = (N + C - 1) / C;
        r_lo = min(N, cr * L);
        r_hi = min(N, r_lo + L);
        // this CTA's rows [k_lo, k_hi) of W, addressed by the absolute timestep: W[k * nxi + c]
        W = sm + cv.W - (int64_t)k_lo * nxi;
        xb = sm + cv.xb; lam = sm + cv.lam; xc = sm + cv.xc; v = sm + cv.v;
        gp = sm + cv.gp; dl = sm + cv.dl; dd = sm + cv.dd; rr = sm + cv.rr; wtw = sm + cv.wtw;
        Rb = sm + cv.Rb; ob = sm + cv.ob;
        n_refine = A.n_refine;
        n_obs_ = I.n_obs;
        cull = MODE ? 1 : A.cull;
        bbx = sm + cv.bb;
        osa = sm + cv.os;
        lpl = reinterpret_cast<unsigned short *>(sm + cv.lp);
        lol = reinterpret_cast<unsigned short *>(sm + cv.lo);
        lcn = reinterpret_cast<int *>(sm + cv.lc);
        LPs = cull_lp(n);
        LOs = cull_lo(nobs);
        NBX = n + nobs;
        fn.set(n);
        fN.set(N);
        fL.set(L);
        lv = 0;
        need = 0;
        oob = 0;
        esc = false;
        cdel = T(0.5) * fmax(I.a, I.b);
        bd = sm + cv.bd; db = sm + cv.db; bf = sm + cv.bf; sx = sm + cv.sx; red = sm + cv.red; Ps = sm + cv.Ps;
        nbc = MODE ? 2 : S.nbc;   // the compile-time modes serve the two-row boundary only
        vsc = T(S.vsc);
        P = reinterpret_cast<VP *>(sm + cv.pb);
        gstride = carve_round(NN + 4 + 3 * 32, (int)sizeof(T));
        Pbg = A.Pb + S.off_Pb;
        obs_g = A.obs + I.off_obs;
        Pdev = sx; Pdif = sx + nxi * nxi; Bdev = sx + 2 * nxi * nxi; Bdif = Bdev + nbc * nxi;
        mv = Bdif + nbc * nxi; pm = mv + ND * nxi; mb = pm + ND * nxi;
        Qc = mb + 3 * ND;
        smooth = MODE == 3 ? 1 : MODE ? 0 : A.cost == SF_COST_SMOOTHNESS;
        Prow = nullptr;
        need_b = 0;
        tcm = 0;
        gb = 0;
        CC = C;
        crc = cr;
        G = 1;
        grp = 0;
        tcb = 0;
    }

    // This CTA serves instance group g of a cluster of ccount CTAs (ngroups instances, C
    // CTAs each) as cluster rank crank.
    __device__ __forceinline__ void set_group(int g, int ngroups, int crank, int ccount)
    {
        gb = g * C;
        grp = g;
        G = ngroups;
        crc = crank;
        CC = ccount;
    }

    // Tensor-core projection set-up: barriers, the zeroed B operand and a tensor-memory
    // accumulator of 16 columns per 128-row tile.  All threads call it.
    __device__ __forceinline__ void tc_setup(const FwdArgs<T> &A, unsigned char *smem_raw)
    {
        if constexpr (TC && sizeof(T) == 4) {
            tcm = dense ? A.tc_mode : 0;
            if (!tcm) return;
            if (A.tcb) {
                tcb_setup(A, smem_raw);
                return;
            }
            tc_es = sf::tc_es(tcm);
            tc_nK = tc_nk(tcm, N);
            tc_nT = tc_ntiles(N, C);
            tc_na = sf::tc_na(tcm);
            const int kpad = tc_nK * tc_kc(tcm);
            tc_bbytes = 16 * kpad * tc_es;
            tc_sbo_b = (kpad * tc_es / 16) * 128;
            tc_res = A.tc_res;
            wbud = A.wait_budget;
            tc_ring = smem_raw;
            tc_B = tc_ring + (int64_t)tc_stages(tcm, N, C, tc_res) * kTcChunkBytes * tc_na;
            unsigned char *bars = tc_B + (int64_t)tc_bbytes * tc_na + tc_bbytes + 1024;
            tc_bar = reinterpret_cast<uint64_t *>(bars);
            tc_flag = reinterpret_cast<int *>(bars + 40);
            tc_slot = reinterpret_cast<uint32_t *>(bars + 44);
            tc_src = A.tcA + A.tc_off[I.shape] + (int64_t)cr * tc_nT * tc_nK * tc_na * kTcChunkBytes;
            for (int e = tid; e < tc_bbytes * tc_na / 4; e += nt) reinterpret_cast<uint32_t *>(tc_B)[e] = 0u;
            for (int e = tid; e < nxi * nxi; e += nt) {   // W'W for the refinement's Hessian products
                const int u = e / nxi, vv = e - u * nxi;
                float acc = 0.f;
                const T *Wg = A.W + S.off_W;   // every row: shared memory holds this CTA's only
                for (int k = 0; k < H; ++k) acc += Wg[k * nxi + u] * Wg[k * nxi + vv];
                wtw[e] = acc;
            }
            tc_fw0 = tc_fw1 = tc_ld0 = tc_ld1 = tc_ec0 = tc_ec1 = 0;
            if (tid == 0) {
                for (int b = 0; b < 5; ++b) tc::mbar_init(tc_bar + b, 1);
                *tc_flag = 0;
                tc::fence_barrier_init();
                if (tc_res) {   // every chunk of this CTA's rows, once, on barrier 0
                    const int items = tc_nT * tc_nK;
                    const uint32_t stage_bytes = (uint32_t)(tc_na * kTcChunkBytes);
                    tc::mbar_arrive_expect_tx(tc_bar, (uint32_t)items * stage_bytes);
                    for (int w = 0; w < items; ++w)
                        tc::bulk_g2s(tc_ring + (int64_t)w * stage_bytes, tc_src + (int64_t)w * stage_bytes, stage_bytes,
                                     tc_bar);
                    tc_ld0 = 1;
                    if (tc::mbar_wait(tc_bar, 0, wbud)) tc_fw0 = 1;
                    else *tc_flag = 1;
                }
            }
            tmem_cols = 32;
            while (tmem_cols < (uint32_t)(16 * tc_nT)) tmem_cols <<= 1;
            if ((tid >> 5) == 0) {
                tc::tmem_alloc(tc_slot, tmem_cols);
                tc::tmem_relinquish();
            }
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            tmem_base = *tc_slot;
            tc_done = tc_seen = 0;
        }
    }

    // Releases the tensor memory after waiting (bounded) for copies still in flight.
    __device__ __forceinline__ void tc_teardown()
    {
        if constexpr (TC && sizeof(T) == 4) {
            if (!tcm) return;
            if (tid == 0) {
                while (tc_fw0 < tc_ld0 && tc::mbar_wait(tc_bar + 0, tc_fw0 & 1, kWaitLimit)) ++tc_fw0;
                while (tc_fw1 < tc_ld1 && tc::mbar_wait(tc_bar + 1, tc_fw1 & 1, kWaitLimit)) ++tc_fw1;
                // an MMA commit whose completion a timed-out wait did not observe
                while (tc_seen < tc_done && tc::mbar_wait(tc_bar + 4, tc_seen & 1, kWaitLimit)) ++tc_seen;
            }
            tc::fence_before_sync();
            __syncthreads();
            if ((tid >> 5) == 0) tc::tmem_dealloc(tmem_base, tmem_cols);
        }
    }


    // Coefficient c of a robot is fixed by A (eq. boundary_con): the first and last (start
    // and goal of the Bernstein basis) and, with the velocity row, the second.
    __device__ __forceinline__ bool fixed_c(int c) const { return c == 0 || c == nxi - 1 || (nbc == 3 && c == 1); }

    // Basis, candidate, boundary values, obstacle records and projection operators.
    __device__ __forceinline__ void load_constants(const FwdArgs<T> &A, int p_rows)
    {
        const T *Wg = A.W + S.off_W;
        for (int e = k_lo * nxi + tid; e < k_hi * nxi; e += nt) W[e] = Wg[e];
        const T *xcg = A.xc + I.off_xi;
        for (int e = tid; e < NN; e += nt) xc[e] = xcg[e];
        for (int e = tid; e < ND * n * nbc; e += nt) bd[e] = A.bnd[I.off_bnd + e];
        // the values A xi = b fixes, per (axis, robot) r: coefficient 0 (start), 1 (start +
        // v_0 / vsc, with the velocity row) and n_xi - 1 (goal)
        for (int r = tid; r < ND * n; r += nt) {
            const T *b = A.bnd + I.off_bnd + (int64_t)r * nbc;
            bf[3 * r] = b[0];
            bf[3 * r + 1] = nbc == 3 ? b[0] + b[2] / vsc : T(0);
            bf[3 * r + 2] = b[1];
        }
        for (int m = nobs + tid; m < opad + 4; m += nt) {   // padding records: far away, zero radius
            T *o = ob + 8 * m;
            for (int q = 0; q < 8; ++q) o[q] = T(0);
            for (int ax = 0; ax < ND; ++ax) o[ax] = Far<T>::v;
            o[4] = T(1);
        }
        for (int m = tid; m < nobs; m += nt) {
            const T ao = A.oab[I.off_oab + 2 * m], bo = A.oab[I.off_oab + 2 * m + 1];
            T *o = ob + 8 * m;
            for (int ax = 0; ax < 3; ++ax) o[ax] = (!I.dyn && ax < ND) ? A.obs[I.off_obs + (int64_t)m * ND + ax] : T(0);
            o[3] = ao * ao;                 // compare d_x^2 + d_y^2 + kz_o d_z^2 with a_o^2
            o[4] = (ao * ao) / (bo * bo);   // kz_o
            o[5] = T(1) / (ao * ao);
            o[6] = ao;
            o[7] = bo;
            if (cull) {
                for (int ax = 0; ax < 3; ++ax) osa[ax * nobs + m] = o[ax];
                osa[3 * nobs + m] = o[3];
                osa[4 * nobs + m] = o[4];
            }
        }
        const T *Pg = A.P + S.off_P;
        if (dense && p_rows > 0)
            for (int e = tid; e < (r_hi - r_lo) * N; e += nt) Ps[e] = Pg[(int64_t)r_lo * N + e];
        Prow = (dense && p_rows > 0) ? Ps - (int64_t)r_lo * N : Pg;   // Prow[r * N + c], r in [r_lo, r_hi)
        if (smooth) {
            const T *Cg = A.Sx + S.off_S + kron_cost_off(nxi, nbc);
            for (int e = tid; e < nxi * nxi; e += nt) Qc[e] = Cg[e];
        }
        if (!dense) {
            const T *Sg = A.Sx + S.off_S;
            for (int e = tid; e < nxi * nxi; e += nt) {
                Pdev[e] = Sg[e];
                Pdif[e] = Sg[nxi * nxi + e] - Sg[e];
            }
            for (int e = tid; e < nbc * nxi; e += nt) {
                Bdev[e] = Sg[2 * nxi * nxi + e];
                Bdif[e] = Sg[2 * nxi * nxi + nbc * nxi + e] - Sg[2 * nxi * nxi + e];
            }
        }
    }

    // b - A xi_bar for the current xb (nonzero only when it misses the boundary values);
    // sets need_b (block-uniform) and the robot means mb for the structured form.
    __device__ __forceinline__ void boundary_gap()
    {
        __syncthreads();
        int nb = 0;
        for (int e = tid; e < ND * n * nbc; e += nt) {
            const int r = e / nbc, s = e - r * nbc;
            const T *x = xb + r * nxi;
            const T ax = s == 0 ? x[0] : s == 1 ? x[nxi - 1] : vsc * (x[1] - x[0]);
            db[e] = bd[e] - ax;
            if (db[e] != T(0)) nb = 1;
        }
        need_b = __syncthreads_or(nb);
        if (need_b && !dense)
            for (int e = tid; e < ND * nbc; e += nt) {
                const int ax = e / nbc, s = e - ax * nbc;
                T acc = T(0);
                for (int i = 0; i < n; ++i) acc += db[(ax * n + i) * nbc + s];
                mb[e] = acc * invn;
            }
        __syncthreads();
    }

    // sum_c wr[c] xr[c] with three partial sums (the order every position is formed in)
    __device__ __forceinline__ T wdot(const T *wr, const T *xr) const
    {
        T s0 = T(0), s1 = T(0), s2 = T(0);
        int c = 0;
        for (; c + 2 < nxi; c += 3) {
            s0 += wr[c] * xr[c];
            s1 += wr[c + 1] * xr[c + 1];
            s2 += wr[c + 2] * xr[c + 2];
        }
        for (; c < nxi; ++c) s0 += wr[c] * xr[c];
        return (s0 + s1) + s2;
    }

    // out[i][kl] = (sum_c W[k0 + kl][c] coeff[ax][i][c])_ax (vector layout, one (i, kl) per
    // thread, every axis from one load of the basis row).  chk: also note in esc whether a
    // value leaves its robot's inflated box.
    __device__ __forceinline__ void wvec(int k0, int hcc, const T *coeff, VP *out, bool chk = false)
    {
        const int S = seg_len(hcc), ns = nseg_of(hcc);
        FDiv fh, fS;
        fh.set(hcc);
        fS.set(S);
        for (int e = tid; e < n * hcc; e += nt) {
            const int i = fh.q(e), kl = e - i * hcc;
            const T *wr = W + (k0 + kl) * nxi;
            VP p;
#pragma unroll
            for (int ax = 0; ax < NDP<ND>::v; ++ax) p.v[ax] = T(0);
#pragma unroll
            for (int ax = 0; ax < ND; ++ax) p.v[ax] = wdot(wr, coeff + (ax * n + i) * nxi);
            out[i * hcc + kl] = p;
            if (chk) {
                const int sg = fS.q(kl);
#pragma unroll
                for (int ax = 0; ax < ND; ++ax)
                    if (!(p.v[ax] >= bbx[((2 * ax) * ns + sg) * NBX + i] && p.v[ax] <= bbx[((2 * ax + 1) * ns + sg) * NBX + i]))
                        esc = true;
            }
        }
    }

    // wvec of c1 into out1 (with the escape check when chk) and of c2 into out2 in one pass
    // over the items: the adjoint needs both products for every chunk, and they share the
    // basis rows and the index arithmetic.  The same sums as two wvec calls.
    __device__ __forceinline__ void wvec2(int k0, int hcc, const T *c1, VP *out1, const T *c2, VP *out2, bool chk)
    {
        const int S = seg_len(hcc), ns = nseg_of(hcc);
        FDiv fh, fS;
        fh.set(hcc);
        fS.set(S);
        for (int e = tid; e < n * hcc; e += nt) {
            const int i = fh.q(e), kl = e - i * hcc;
            const T *wr = W + (k0 + kl) * nxi;
            VP p, q;
#pragma unroll
            for (int ax = 0; ax < NDP<ND>::v; ++ax) p.v[ax] = q.v[ax] = T(0);
#pragma unroll
            for (int ax = 0; ax < ND; ++ax) {
                p.v[ax] = wdot(wr, c1 + (ax * n + i) * nxi);
                q.v[ax] = wdot(wr, c2 + (ax * n + i) * nxi);
            }
            out1[i * hcc + kl] = p;
            out2[i * hcc + kl] = q;
            if (chk) {
                const int sg = fS.q(kl);
#pragma unroll
                for (int ax = 0; ax < ND; ++ax)
                    if (!(p.v[ax] >= bbx[((2 * ax) * ns + sg) * NBX + i] && p.v[ax] <= bbx[((2 * ax + 1) * ns + sg) * NBX + i]))
                        esc = true;
            }
        }
    }

    // Segments of a chunk for the culling boxes: at most 32 timesteps each.
    __device__ __forceinline__ static int nseg_of(int hcc) { return (hcc + 31) >> 5; }
    __device__ __forceinline__ static int seg_len(int hcc) { return (hcc + nseg_of(hcc) - 1) / nseg_of(hcc); }

    // Call before positions() of each chunk: lists of another chunk are not reused.
    __device__ __forceinline__ void begin_chunk()
    {
        if (k_hi - k_lo > hc) lv = 0;
    }

    // The barrier after positions(); with culling it also decides (block-uniformly)
    // whether the candidate lists must be rebuilt: none yet, or a position left its box.
    __device__ __forceinline__ void sync_lists()
    {
        if (cull) {
            need = __syncthreads_or(esc || !lv);
            esc = false;
        } else {
            __syncthreads();
        }
    }

    // positions of coeff for the chunk, robots padded with far stand-ins
    __device__ __forceinline__ void positions(int k0, int hcc, const T *coeff)
    {
        wvec(k0, hcc, coeff, P, cull && lv);
        for (int e = n * hcc + tid; e < (npad + 4) * hcc; e += nt) {
            VP p;
#pragma unroll
            for (int ax = 0; ax < NDP<ND>::v; ++ax) p.v[ax] = Far<T>::v;
            P[e] = p;
        }
    }

    // positions() of coeff together with W c2 into out2 (the adjoint's R* = W g*)
    __device__ __forceinline__ void positions2(int k0, int hcc, const T *coeff, const T *c2, VP *out2)
    {
        wvec2(k0, hcc, coeff, P, c2, out2, cull && lv);
        for (int e = n * hcc + tid; e < (npad + 4) * hcc; e += nt) {
            VP p;
#pragma unroll
            for (int ax = 0; ax < NDP<ND>::v; ++ax) p.v[ax] = Far<T>::v;
            P[e] = p;
        }
    }

    // wt_acc for a chunk of exactly HCC timesteps: the same sums in the same order, with the
    // loop fully unrolled (all loads issued ahead of the multiply-adds)
    template <int HCC>
    __device__ __forceinline__ void wt_acc_fixed(int k0, const T *src, T *dst)
    {
        for (int e = tid; e < NN; e += nt) {
            const int r = e / NXI, c = e - r * NXI;
            const T *rr = src + r * HCC;
            const T *wc = W + k0 * NXI + c;
            T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
#pragma unroll
            for (int kl = 0; kl + 3 < HCC; kl += 4) {
                s0 += wc[kl * NXI] * rr[kl];
                s1 += wc[(kl + 1) * NXI] * rr[kl + 1];
                s2 += wc[(kl + 2) * NXI] * rr[kl + 2];
                s3 += wc[(kl + 3) * NXI] * rr[kl + 3];
            }
#pragma unroll
            for (int kl = HCC & ~3; kl < HCC; ++kl) s0 += wc[kl * NXI] * rr[kl];
            dst[e] += (s0 + s1) + (s2 + s3);
        }
    }

    // dst[ax][i][c] += sum_kl W[k0 + kl][c] src[ax][i][kl]
    __device__ __forceinline__ void wt_acc(int k0, int hcc, const T *src, T *dst)
    {
        if constexpr (NXI > 0) {
            if (hcc == 25) {   // a quarter of a 100-step horizon, the common chunk
                wt_acc_fixed<25>(k0, src, dst);
                return;
            }
        }
        for (int e = tid; e < NN; e += nt) {
            const int r = e / nxi, c = e - r * nxi;
            const T *rr = src + r * hcc;
            const T *wc = W + k0 * nxi + c;
            T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
            int kl = 0;
            for (; kl + 3 < hcc; kl += 4) {
                s0 += wc[kl * nxi] * rr[kl];
                s1 += wc[(kl + 1) * nxi] * rr[kl + 1];
                s2 += wc[(kl + 2) * nxi] * rr[kl + 2];
                s3 += wc[(kl + 3) * nxi] * rr[kl + 3];
            }
            for (; kl < hcc; ++kl) s0 += wc[kl * nxi] * rr[kl];
            dst[e] += (s0 + s1) + (s2 + s3);
        }
    }

    // Candidate lists of the chunk [k0, k0 + hcc), rebuilt after sync_lists() asked for it.
    // The chunk is cut into segments of at most 32 timesteps.  Per segment, each robot's
    // bounding box over the segment, inflated by cdel on every axis, and each dynamic
    // obstacle's box; then per (segment, robot), in ascending order, the partners j != i
    // and obstacles m whose boxes come within the activity threshold (relative margin
    // 1e-5).  While every position stays inside its robot's inflated box (checked by
    // positions()), a row that is not listed is inactive at every timestep of its segment:
    // the culled loops add the same terms in the same order as the full ones.  Lists are
    // padded to a multiple of four with the far stand-ins npad (robots) and opad
    // (obstacles).  Ends with a barrier when it rebuilds.
    __device__ __forceinline__ void cull_lists(int k0, int hcc)
    {
        if (!cull || !need) return;
        const int lane = tid & 31, wp = tid >> 5, nw = nt >> 5;
        const int nbox = n + (I.dyn ? nobs : 0), ns = nseg_of(hcc), S = seg_len(hcc);
        // boxes: groups of 8 lanes per (segment, box), lane s8 taking timesteps s8, s8 + 8, ...
        const int tasks = ns * nbox;
        for (int base = wp * 4; base < tasks; base += nw * 4) {   // warp-uniform: full-mask shuffles
            const int t = base + (lane >> 3), s8 = lane & 7;
            const int sg = t / nbox, b = t - sg * nbox;
            const int kb = sg * S, ke = min(hcc, kb + S);
            T lo[ND], hi[ND];
#pragma unroll
            for (int ax = 0; ax < ND; ++ax) {
                lo[ax] = T(1e30);
                hi[ax] = T(-1e30);
            }
            if (t < tasks)
                for (int kl = kb + s8; kl < ke; kl += 8) {
                    T x[ND];
                    if (b < n) {
                        const VP pv = P[b * hcc + kl];
#pragma unroll
                        for (int ax = 0; ax < ND; ++ax) x[ax] = pv.v[ax];
                    } else {
                        const T *c = obs_g + ((int64_t)(b - n) * H + k0 + kl) * ND;
#pragma unroll
                        for (int ax = 0; ax < ND; ++ax) x[ax] = c[ax];
                    }
#pragma unroll
                    for (int ax = 0; ax < ND; ++ax) {
                        lo[ax] = fmin(lo[ax], x[ax]);
                        hi[ax] = fmax(hi[ax], x[ax]);
                    }
                }
#pragma unroll
            for (int o = 4; o; o >>= 1)
#pragma unroll
                for (int ax = 0; ax < ND; ++ax) {
                    lo[ax] = fmin(lo[ax], __shfl_xor_sync(0xffffffffu, lo[ax], o));
                    hi[ax] = fmax(hi[ax], __shfl_xor_sync(0xffffffffu, hi[ax], o));
                }
            if (s8 == 0 && t < tasks) {
                const T dl = b < n ? cdel : T(0);
#pragma unroll
                for (int ax = 0; ax < ND; ++ax) {
                    bbx[((2 * ax) * ns + sg) * NBX + b] = lo[ax] - dl;
                    bbx[((2 * ax + 1) * ns + sg) * NBX + b] = hi[ax] + dl;
                }
            }
        }
        __syncthreads();
        const T a2c = I.a * I.a * T(1.00001), kz = (I.a * I.a) * I.ib2;
        for (int task = wp; task < ns * n; task += nw) {
            const int sg = task / n, i = task - sg * n;
            const T *bl = bbx + sg * NBX, *bh = bbx + (ns + sg) * NBX;   // axis ax at + 2 ax ns NBX
            T lo[ND], hi[ND];
#pragma unroll
            for (int ax = 0; ax < ND; ++ax) {
                lo[ax] = bl[2 * ax * ns * NBX + i];
                hi[ax] = bh[2 * ax * ns * NBX + i];
            }
            unsigned short *L = lpl + task * LPs;
            int cp = 0;
            for (int j0 = 0; j0 < n; j0 += 32) {
                const int j = j0 + lane;
                bool c = false;
                if (j < n && j != i) {
                    T g[ND];
#pragma unroll
                    for (int ax = 0; ax < ND; ++ax)
                        g[ax] = fmax(T(0), fmax(bl[2 * ax * ns * NBX + j] - hi[ax], lo[ax] - bh[2 * ax * ns * NBX + j]));
                    c = qdist<T, ND>(g, kz) <= a2c;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, c);
                const int at = cp + __popc(bal & ((1u << lane) - 1u));
                if (c && in_bounds(at < LPs)) L[at] = (unsigned short)j;
                cp += __popc(bal);
            }
            for (int u = cp + lane; u < ((cp + 3) & ~3); u += 32)
                if (in_bounds(u < LPs)) L[u] = (unsigned short)npad;
            unsigned short *M = lol + task * LOs;
            int co = 0;
            for (int m0 = 0; m0 < nobs; m0 += 32) {
                const int m = m0 + lane;
                bool c = false;
                if (m < nobs) {
                    T g[ND];
#pragma unroll
                    for (int ax = 0; ax < ND; ++ax) {
                        T cl, ch;
                        if (I.dyn) {
                            cl = bl[2 * ax * ns * NBX + n + m];
                            ch = bh[2 * ax * ns * NBX + n + m];
                        } else {
                            cl = ch = osa[ax * nobs + m];
                        }
                        g[ax] = fmax(T(0), fmax(cl - hi[ax], lo[ax] - ch));
                    }
                    T q = g[0] * g[0] + g[1] * g[1];
                    if (ND == 3) q += osa[4 * nobs + m] * g[ND - 1] * g[ND - 1];
                    c = q <= osa[3 * nobs + m] * T(1.00001);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, c);
                const int at = co + __popc(bal & ((1u << lane) - 1u));
                if (c && in_bounds(at < LOs)) M[at] = (unsigned short)m;
                co += __popc(bal);
            }
            for (int u = co + lane; u < ((co + 3) & ~3); u += 32)
                if (in_bounds(u < LOs)) M[u] = (unsigned short)opad;
            if (lane == 0) {
                lcn[2 * task] = cp;
                lcn[2 * task + 1] = co;
            }
        }
        __syncthreads();
        lv = 1;
    }

    // Four partner (or obstacle) indices of block b of robot i's loop: the full loop's
    // b*4 .. b*4+3, or the culled loop's list entries (far stand-ins past the count).  With
    // SF_BOUNDS_CHECK an index outside [0, stand_in + 4) is recorded and replaced by the
    // stand-in.
    __device__ __forceinline__ void block_ids(const unsigned short *list, int cnt, int b4, int stand_in, int (&id)[4])
    {
        if (b4 < cnt) {
            const ushort4 q = *reinterpret_cast<const ushort4 *>(list + b4);
            id[0] = q.x; id[1] = q.y; id[2] = q.z; id[3] = q.w;
        } else {
            id[0] = id[1] = id[2] = id[3] = stand_in;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (!in_bounds((unsigned)id[u] < (unsigned)(stand_in + 4))) id[u] = stand_in;
    }

    // true when c holds; with SF_BOUNDS_CHECK a false c is recorded in oob (the kernel
    // reports SF_EBOUNDS for the instance) and the caller skips the access.  Without it the
    // check compiles away.
    __device__ __forceinline__ bool in_bounds(bool c)
    {
#ifdef SF_BOUNDS_CHECK
        if (!c) oob = 1;
        return c;
#else
        (void)c;
        return true;
#endif
    }

    // Rows of the items (i, k) of one chunk: R written to Rb[ax][i][kl].  Partners and
    // obstacles are tested four at a time; the warp votes once per block of four and takes
    // the rare active-row path only when one of its lanes needs it.
    __device__ __forceinline__ void rows(int k0, int hcc, T &rp2, T &mx2)
    {
        const int items = n * hcc, segS = seg_len(hcc);
        FDiv fh, fS;
        fh.set(hcc);
        fS.set(segS);
        const T a2 = I.a * I.a, ia2 = I.ia2, kz = (I.a * I.a) * I.ib2;
        T tie_f[ND], tie_b[ND];   // r_1 of a coincident pair seen from the row's first / second robot
#pragma unroll
        for (int ax = 0; ax < ND; ++ax) tie_f[ax] = tie_b[ax] = T(0);
        if (ND == 2) { tie_f[0] = -I.a; tie_b[0] = I.a; }
        else { tie_f[ND - 1] = -I.b; tie_b[ND - 1] = I.b; }
        for (int e0 = 0; e0 < items; e0 += nt) {
            const int e = e0 + tid;
            const bool valid = e < items;
            if (__all_sync(0xffffffffu, !valid)) continue;   // a whole warp without items skips the round
            const int ee = valid ? e : 0;
            const int i = fh.q(ee), kl = ee - i * hcc, k = k0 + kl;
            VP pi = P[i * hcc + kl];
            if (!valid)
#pragma unroll
                for (int ax = 0; ax < ND; ++ax) pi.v[ax] = -Far<T>::v;
            T R[ND];
#pragma unroll
            for (int ax = 0; ax < ND; ++ax) R[ax] = T(0);
            const int task = fS.q(kl) * n + i;   // culling lists of (segment, robot)
            const int cp4 = cull ? (lcn[2 * task] + 3) & ~3 : 0, co4 = cull ? (lcn[2 * task + 1] + 3) & ~3 : 0;
            const int jend = cull ? __reduce_max_sync(0xffffffffu, cp4) : npad;
            const int mend = cull ? __reduce_max_sync(0xffffffffu, co4) : opad;
            // robot pairs: the row of pair (min(i,j), max(i,j)); j == i (q = 0) is excluded in
            // the slow path
            for (int j0 = 0; j0 < jend; j0 += 4) {
                int jj[4];
                if (cull) block_ids(lpl + task * LPs, cp4, j0, npad, jj);
                else { jj[0] = j0; jj[1] = j0 + 1; jj[2] = j0 + 2; jj[3] = j0 + 3; }
                T d[4][ND], q[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const VP pj = P[jj[u] * hcc + kl];
#pragma unroll
                    for (int ax = 0; ax < ND; ++ax) d[u][ax] = pi.v[ax] - pj.v[ax];
                    q[u] = qdist<T, ND>(d[u], kz);
                }
                const bool any = (q[0] <= a2) | (q[1] <= a2) | (q[2] <= a2) | (q[3] <= a2);
                if (__any_sync(0xffffffffu, any)) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int j = jj[u];
                        if (q[u] <= a2 && j != i) {
                            if (j > i) row_active<T, ND>(d[u], q[u], ia2, tie_f, R, rp2, mx2, true);
                            else row_active<T, ND>(d[u], q[u], ia2, tie_b, R, rp2, mx2, false);
                        }
                    }
                }
            }
            // obstacles
            for (int m0 = 0; m0 < mend; m0 += 4) {
                int mm[4];
                if (cull) block_ids(lol + task * LOs, co4, m0, opad, mm);
                else { mm[0] = m0; mm[1] = m0 + 1; mm[2] = m0 + 2; mm[3] = m0 + 3; }
                T d[4][ND], q[4], lim[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int m = mm[u];
                    const Vec<T, 4> r0 = reinterpret_cast<const Vec<T, 4> *>(ob)[2 * m];
                    if (I.dyn && m < nobs) {
                        const T *c = obs_g + ((int64_t)m * H + k) * ND;
#pragma unroll
                        for (int ax = 0; ax < ND; ++ax) d[u][ax] = pi.v[ax] - c[ax];
                    } else {
#pragma unroll
                        for (int ax = 0; ax < ND; ++ax) d[u][ax] = pi.v[ax] - r0.v[ax];
                    }
                    q[u] = d[u][0] * d[u][0] + d[u][1] * d[u][1];
                    if (ND == 3) q[u] += ob[8 * m + 4] * d[u][ND - 1] * d[u][ND - 1];
                    lim[u] = r0.v[3];
                }
                const bool any = (q[0] <= lim[0]) | (q[1] <= lim[1]) | (q[2] <= lim[2]) | (q[3] <= lim[3]);
                if (__any_sync(0xffffffffu, any)) {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (q[u] <= lim[u]) {
                            const int m = mm[u];
                            T tie[ND];
#pragma unroll
                            for (int ax = 0; ax < ND; ++ax) tie[ax] = T(0);
                            if (ND == 2) tie[0] = -ob[8 * m + 6]; else tie[ND - 1] = -ob[8 * m + 7];
                            row_active<T, ND>(d[u], q[u], ob[8 * m + 5], tie, R, rp2, mx2, true);
                        }
                }
            }
            if (!valid) continue;
            // workspace box (G rows: upper side p <= p_max, lower side -p <= -p_min)
#pragma unroll
            for (int ax = 0; ax < ND; ++ax) {
                const T u = pi.v[ax] - I.pmax[ax];
                const T l = I.pmin[ax] - pi.v[ax];
                if (u > T(0)) {
                    R[ax] += u;
                    rp2 += u * u;
                    mx2 = fmax(mx2, u * u);
                }
                if (l > T(0)) {
                    R[ax] -= l;
                    rp2 += l * l;
                    mx2 = fmax(mx2, l * l);
                }
            }
#pragma unroll
            for (int ax = 0; ax < ND; ++ax) Rb[(ax * n + i) * hcc + kl] = R[ax];
        }
    }

    // Adjoint of rows(): with R* (vector layout Rs[i][kl]) the adjoint of R, writes
    // p* = sum over active rows of J' (R*_i - R*_j) (pairs), J' R*_i (obstacles) and the
    // box mask times R*_i, to Rb[ax][i][kl].  seed instead differentiates
    // seed_w / 2 * ||r_p||^2: y = seed_w r_1 on every active row and seed_w (u+ - l+) on the box
    // (Rs is not read; seed_w = 0 gives zeros).
    __device__ __forceinline__ void rows_adjoint(int k0, int hcc, const VP *Rs, T seed_w, bool seed)
    {
        const int items = n * hcc, segS = seg_len(hcc);
        FDiv fh, fS;
        fh.set(hcc);
        fS.set(segS);
        const T a2 = I.a * I.a, ia2 = I.ia2, ib2 = I.ib2, kz = (I.a * I.a) * I.ib2;
        for (int e0 = 0; e0 < items; e0 += nt) {
            const int e = e0 + tid;
            const bool valid = e < items;
            if (__all_sync(0xffffffffu, !valid)) continue;
            const int ee = valid ? e : 0;
            const int i = fh.q(ee), kl = ee - i * hcc, k = k0 + kl;
            VP pi = P[i * hcc + kl];
            if (!valid)
#pragma unroll
                for (int ax = 0; ax < ND; ++ax) pi.v[ax] = -Far<T>::v;
            T Ri[ND], ps[ND];
#pragma unroll
            for (int ax = 0; ax < ND; ++ax) {
                Ri[ax] = seed ? T(0) : Rs[i * hcc + kl].v[ax];
                ps[ax] = T(0);
            }
            const int task = fS.q(kl) * n + i;   // culling lists of (segment, robot)
            const int cp4 = cull ? (lcn[2 * task] + 3) & ~3 : 0, co4 = cull ? (lcn[2 * task + 1] + 3) & ~3 : 0;
            const int jend = cull ? __reduce_max_sync(0xffffffffu, cp4) : npad;
            const int mend = cull ? __reduce_max_sync(0xffffffffu, co4) : opad;
            for (int j0 = 0; j0 < jend; j0 += 4) {
                int jj[4];
                if (cull) block_ids(lpl + task * LPs, cp4, j0, npad, jj);
                else { jj[0] = j0; jj[1] = j0 + 1; jj[2] = j0 + 2; jj[3] = j0 + 3; }
                T d[4][ND], q[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const VP pj = P[jj[u] * hcc + kl];
#pragma unroll
                    for (int ax = 0; ax < ND; ++ax) d[u][ax] = pi.v[ax] - pj.v[ax];
                    q[u] = qdist<T, ND>(d[u], kz);
                }
                const bool any = (q[0] <= a2) | (q[1] <= a2) | (q[2] <= a2) | (q[3] <= a2);
                if (__any_sync(0xffffffffu, any)) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int j = jj[u];
                        if (q[u] <= a2 && j != i) {
                            T y[ND];
#pragma unroll
                            for (int ax = 0; ax < ND; ++ax) y[ax] = seed ? T(0) : Ri[ax] - Rs[j * hcc + kl].v[ax];
                            row_adjoint<T, ND>(d[u], q[u], ia2, ib2, y, seed_w, seed, ps);
                        }
                    }
                }
            }
            for (int m0 = 0; m0 < mend; m0 += 4) {
                int mm[4];
                if (cull) block_ids(lol + task * LOs, co4, m0, opad, mm);
                else { mm[0] = m0; mm[1] = m0 + 1; mm[2] = m0 + 2; mm[3] = m0 + 3; }
                T d[4][ND], q[4], lim[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int m = mm[u];
                    const Vec<T, 4> r0 = reinterpret_cast<const Vec<T, 4> *>(ob)[2 * m];
                    if (I.dyn && m < nobs) {
                        const T *c = obs_g + ((int64_t)m * H + k) * ND;
#pragma unroll
                        for (int ax = 0; ax < ND; ++ax) d[u][ax] = pi.v[ax] - c[ax];
                    } else {
#pragma unroll
                        for (int ax = 0; ax < ND; ++ax) d[u][ax] = pi.v[ax] - r0.v[ax];
                    }
                    q[u] = d[u][0] * d[u][0] + d[u][1] * d[u][1];
                    if (ND == 3) q[u] += ob[8 * m + 4] * d[u][ND - 1] * d[u][ND - 1];
                    lim[u] = r0.v[3];
                }
                const bool any = (q[0] <= lim[0]) | (q[1] <= lim[1]) | (q[2] <= lim[2]) | (q[3] <= lim[3]);
                if (__any_sync(0xffffffffu, any)) {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (q[u] <= lim[u]) {
                            const int m = mm[u];
                            const T iao = ob[8 * m + 5], ibo = ob[8 * m + 4] * ob[8 * m + 5];
                            row_adjoint<T, ND>(d[u], q[u], iao, ibo, Ri, seed_w, seed, ps);
                        }
                }
            }
            if (!valid) continue;
#pragma unroll
            for (int ax = 0; ax < ND; ++ax) {
                const T u = pi.v[ax] - I.pmax[ax];
                const T l = I.pmin[ax] - pi.v[ax];
                if (seed) {
                    if (u > T(0)) ps[ax] += seed_w * u;
                    if (l > T(0)) ps[ax] -= seed_w * l;
                } else {
                    if (u > T(0)) ps[ax] += Ri[ax];
                    if (l > T(0)) ps[ax] += Ri[ax];
                }
            }
#pragma unroll
            for (int ax = 0; ax < ND; ++ax) Rb[(ax * n + i) * hcc + kl] = ps[ax];
        }
    }

    // Rows [r_lo, r_hi) of P_eta src on the tensor cores into dl: B = src (axes as rows,
    // converted to TF32 / BF16 [+ BF16 residual]); the CTA's A chunks stream through a
    // two-stage ring by bulk copies; one thread issues tcgen05.mma into tensor memory;
    // warps 0-3 read the 128-row tiles back.  A wait that runs out sets the sticky flag
    // and the instance's status; the control flow of every thread stays the same.
    __device__ __forceinline__ void tc_rows(const T *src, bool corr_b)
    {
        if constexpr (TC && sizeof(T) == 4) {
            const int es = tc_es, na = tc_na;
            for (int e = tid; e < ND * N; e += nt) {
                const int ax = e / N, c = e - ax * N;
                const float x = src[ax * N + c];
                const int off = ((c * es) >> 4) * 128 + ax * 16 + ((c * es) & 15);
                if (tcm == 1) {
                    *reinterpret_cast<float *>(tc_B + off) = tc::to_tf32(x);
                } else {
                    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                    *reinterpret_cast<__nv_bfloat16 *>(tc_B + off) = hi;
                    if (na == 2)
                        *reinterpret_cast<__nv_bfloat16 *>(tc_B + tc_bbytes + off) =
                            __float2bfloat16_rn(x - __bfloat162float(hi));
                }
            }
            tc::fence_async_shared();
            __syncthreads();
            const bool failed = *tc_flag != 0;
            if (!failed && tid == 0) {
                const int items = tc_nT * tc_nK;
                const uint32_t stage_bytes = (uint32_t)(na * kTcChunkBytes);
                const uint32_t idesc = tc::instr_desc(tcm == 1 ? 2u : 1u, 128, 16);
                const uint32_t ring0 = tc::smem_u32(tc_ring), b0 = tc::smem_u32(tc_B);
                bool bad = false;
                // one k-chunk of one 128-row tile: 4 MMAs of K = 32 bytes (x3 for BF16 x3)
                auto issue = [&](uint32_t a_hi, int t, int kc) {
                    const uint32_t d_tmem = tmem_base + 16u * t, a_lo = a_hi + kTcChunkBytes;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint64_t ad = tc::smem_desc(a_hi + 256u * j, 128, 1024);
                        const uint32_t boff = (uint32_t)((kc * 8 + 2 * j) * 128);
                        const uint64_t bd_ = tc::smem_desc(b0 + boff, 128, tc_sbo_b);
                        const uint32_t acc = (kc > 0 || j > 0) ? 1u : 0u;
                        if (tcm == 1) {
                            tc::mma_tf32(d_tmem, ad, bd_, idesc, acc);
                        } else {
                            tc::mma_bf16(d_tmem, ad, bd_, idesc, acc);
                            if (na == 2) {
                                const uint64_t bl = tc::smem_desc(b0 + tc_bbytes + boff, 128, tc_sbo_b);
                                const uint64_t al = tc::smem_desc(a_lo + 256u * j, 128, 1024);
                                tc::mma_bf16(d_tmem, ad, bl, idesc, 1u);
                                tc::mma_bf16(d_tmem, al, bd_, idesc, 1u);
                            }
                        }
                    }
                };
                if (tc_res) {   // resident chunks: no waits between the MMAs
                    tc::fence_after_sync();
                    for (int w = 0; w < items; ++w) {
                        const int t = w / tc_nK;
                        issue(ring0 + (uint32_t)w * stage_bytes, t, w - t * tc_nK);
                    }
                }
                for (int w = 0; w < items && w < 2 && !tc_res; ++w) {
                    tc::mbar_arrive_expect_tx(tc_bar + w, stage_bytes);
                    tc::bulk_g2s(tc_ring + w * stage_bytes, tc_src + (int64_t)w * stage_bytes, stage_bytes, tc_bar + w);
                    if (w) ++tc_ld1; else ++tc_ld0;
                }
                for (int w = 0; w < items && !tc_res; ++w) {
                    const int st = w & 1;
                    const uint32_t fw = st ? tc_fw1 : tc_fw0;
                    if (!tc::mbar_wait(tc_bar + st, fw & 1, wbud)) {
                        bad = true;
                        break;
                    }
                    if (st) ++tc_fw1; else ++tc_fw0;
                    tc::fence_after_sync();
                    const int t = w / tc_nK;
                    issue(ring0 + st * stage_bytes, t, w - t * tc_nK);
                    tc::mma_commit(tc_bar + 2 + st);
                    if (st) ++tc_ec1; else ++tc_ec0;
                    if (w + 2 < items) {
                        const uint32_t ec = st ? tc_ec1 : tc_ec0;
                        if (!tc::mbar_wait(tc_bar + 2 + st, (ec - 1) & 1, wbud)) {
                            bad = true;
                            break;
                        }
                        tc::mbar_arrive_expect_tx(tc_bar + st, stage_bytes);
                        tc::bulk_g2s(tc_ring + st * stage_bytes, tc_src + (int64_t)(w + 2) * stage_bytes, stage_bytes,
                                     tc_bar + st);
                        if (st) ++tc_ld1; else ++tc_ld0;
                    }
                }
                tc::mma_commit(tc_bar + 4);
                if (bad) *tc_flag = 1;
            }
            bool ok = !failed;
            if (!failed) {
                ok = tc::mbar_wait(tc_bar + 4, tc_done & 1, wbud);
                ++tc_done;
                if (ok) tc_seen = tc_done;
            }
            ok = __all_sync(0xffffffffu, ok);   // tcgen05.ld below is warp-collective
            if (!ok && (tid & 31) == 0) *tc_flag = 1;   // later calls skip the tensor cores
            tc::fence_after_sync();
            const int wp = tid >> 5, lane = tid & 31;
            if (wp < 4) {
                for (int t = 0; t < tc_nT; ++t) {
                    float dv[4] = {0.f, 0.f, 0.f, 0.f};
                    if (ok) tc::tmem_ld_x4(tmem_base + ((uint32_t)(32 * wp) << 16) + 16u * t, dv);
                    const int row = r_lo + 128 * t + 32 * wp + lane;
                    if (row < r_hi) {
#pragma unroll
                        for (int ax = 0; ax < ND; ++ax) {
                            T a = (T)dv[ax];
                            if (corr_b)
                                for (int q = 0; q < nbc * n; ++q)
                                    a += Pbg[(int64_t)row * nbc * n + q] * db[ax * n * nbc + q];
                            dl[ax * N + row] = a;
                        }
                    }
                }
            }
            tc::fence_before_sync();
            __syncthreads();
        }
    }

    // Instance-group set-up: B (high and low BF16 parts, zeroed once: the K padding and the
    // unused columns must hold finite values), W'W for the refinement, the commit barrier,
    // tensor memory, and this CTA's rows of P_eta written into it: row r of [tb_rl, tb_rh)
    // in lane r (BF16 high part) and, with BF16 x3, lane 64 + r (the low part, the
    // remainder rounded to BF16), two K elements per 32-bit column.  All threads call it.
    __device__ __forceinline__ void tcb_setup(const FwdArgs<T> &A, unsigned char *smem_raw)
    {
        if constexpr (TC && sizeof(T) == 4) {
            tcb = 1;
            tc_na = sf::tc_na(tcm);
            wbud = A.wait_budget;
            Lb = tcb_rows(N, CC);
            fLb.set(Lb);
            tb_rl = min(N, crc * Lb);
            tb_rh = min(N, tb_rl + Lb);
            tb_kp = tcb_kpad(N);
            tb_dcol = tcb_dcol(N);
            const int64_t bb = tcb_bbytes(N);
            tb_Bh = smem_raw;
            tb_stage = reinterpret_cast<float *>(smem_raw + tc_na * bb);
            unsigned char *bars = smem_raw + tc_na * bb + 64 * 16 * 4;
            tc_bar = reinterpret_cast<uint64_t *>(bars);
            tc_flag = reinterpret_cast<int *>(bars + 40);
            tc_slot = reinterpret_cast<uint32_t *>(bars + 44);
            for (int e = tid; e < (int)(tc_na * bb / 4); e += nt) reinterpret_cast<uint32_t *>(smem_raw)[e] = 0u;
            for (int e = tid; e < nxi * nxi; e += nt) {   // W'W for the refinement's Hessian products
                const int u = e / nxi, vv = e - u * nxi;
                float acc = 0.f;
                const T *Wg = A.W + S.off_W;
                for (int k = 0; k < H; ++k) acc += Wg[k * nxi + u] * Wg[k * nxi + vv];
                wtw[e] = acc;
            }
            tc_fw0 = tc_fw1 = tc_ld0 = tc_ld1 = tc_ec0 = tc_ec1 = 0;
            if (tid == 0) {
                for (int b = 0; b < 5; ++b) tc::mbar_init(tc_bar + b, 1);
                *tc_flag = 0;
                tc::fence_barrier_init();
            }
            tmem_cols = tcb_tmem_cols(N);
            if ((tid >> 5) == 0) {
                tc::tmem_alloc(tc_slot, tmem_cols);
                tc::tmem_relinquish();
            }
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            tmem_base = *tc_slot;
            if (tid < 128) {   // warps 0-3: each writes its own quarter of the lanes
                const int lane = tid, row = lane & 63, grow = tb_rl + row;
                const bool lo = lane >= 64, valid = grow < tb_rh && (!lo || tc_na == 2);
                const T *Pr = A.P + S.off_P + (int64_t)(valid ? grow : 0) * N;
                const uint32_t taddr = tmem_base + ((uint32_t)(lane & ~31) << 16);
                for (int j = 0; j < tb_kp / 2; j += 32) {   // 32 columns = 64 K elements per store
                    uint32_t v[32];
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        uint32_t h2 = 0u;
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const int k = 2 * (j + c) + q;
                            const float p = (valid && k < N) ? (float)Pr[k] : 0.f;
                            const __nv_bfloat16 hi = __float2bfloat16_rn(p);
                            const __nv_bfloat16 part = lo ? __float2bfloat16_rn(p - __bfloat162float(hi)) : hi;
                            h2 |= (uint32_t)__bfloat16_as_ushort(part) << (16 * q);
                        }
                        v[c] = h2;
                    }
                    tc::tmem_st_x32(taddr + (uint32_t)j, v);
                }
                tc::tmem_wait_st();
            }
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            tc_done = tc_seen = 0;
        }
    }

    // One batched product: for every instance g of the cluster, rows [tb_rl, tb_rh) of
    // P~ src_g into dl[(g n_d + ax) Lb + r - tb_rl].  src is every CTA's own instance's
    // vector (all CTAs of an instance hold the same values); the CTA reads instance g's from
    // the CTA of group g with its own in-group rank.  Begins and ends with a cluster
    // barrier (the sources complete; every CTA's rows complete).  A wait that runs out sets
    // the sticky flag; the control flow of every thread stays the same.  hi_b: B as its BF16
    // high parts only (a refinement's residual, already 2^-16 of the right-hand side, needs
    // no more: its product then carries about 2^-24 of the result's size).
    __device__ __forceinline__ void tcb_product(cg::cluster_group &cl, const T *src, bool hi_b = false)
    {
        if constexpr (TC && sizeof(T) == 4) {
            cl.sync();
            const int SBO = tb_kp * 16;   // bytes between groups of 8 B columns
            const int na = hi_b ? 1 : tc_na, lo_off = 2 * SBO;   // the low parts: columns 16.. (two groups on)
            // the sources as 16-byte remote loads, kU of them in flight per thread before any
            // is converted (src is 32-byte aligned and padded to 8 floats, so the last vector
            // stays inside it)
            constexpr int kU = 4;
            if ((N & 3) == 0) {   // four consecutive k of one axis per vector: 8-byte stores
                // a warp takes 8 columns x 4 vectors (the columns fastest: its stores fall in
                // distinct banks but for a two-way overlap of the vectors 0 and 2)
                const int NV = N >> 2, ncol = G * ND, cb = (ncol + 7) >> 3, qb = (NV + 3) >> 2, tot = 32 * cb * qb;
                for (int b0 = tid; b0 < tot; b0 += nt * kU) {
                    float4 x4[kU];
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        const int t = b0 + u * nt, blk = t >> 5, gc = (blk % cb) * 8 + (t & 7),
                                  q = (blk / cb) * 4 + ((t >> 3) & 3);
                        if (t < tot && gc < ncol && q < NV) {
                            const int g = gc / ND, ax = gc - g * ND;
                            x4[u] = reinterpret_cast<const float4 *>(cl.map_shared_rank(src, g * C + cr))[ax * NV + q];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        const int t = b0 + u * nt, blk = t >> 5, gc = (blk % cb) * 8 + (t & 7),
                                  q = (blk / cb) * 4 + ((t >> 3) & 3), k0 = 4 * q;   // gc = g n_d + ax: the B column
                        if (t >= tot || gc >= ncol || q >= NV) continue;
                        const int off = (gc >> 3) * SBO + (k0 >> 3) * 128 + (gc & 7) * 16 + (k0 & 7) * 2;
                        const __nv_bfloat162 h01 = __floats2bfloat162_rn(x4[u].x, x4[u].y);
                        const __nv_bfloat162 h23 = __floats2bfloat162_rn(x4[u].z, x4[u].w);
                        uint2 hv;
                        hv.x = *reinterpret_cast<const uint32_t *>(&h01);
                        hv.y = *reinterpret_cast<const uint32_t *>(&h23);
                        *reinterpret_cast<uint2 *>(tb_Bh + off) = hv;
                        if (na == 2) {
                            const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
                            const __nv_bfloat162 l01 = __floats2bfloat162_rn(x4[u].x - f01.x, x4[u].y - f01.y);
                            const __nv_bfloat162 l23 = __floats2bfloat162_rn(x4[u].z - f23.x, x4[u].w - f23.y);
                            uint2 lv;
                            lv.x = *reinterpret_cast<const uint32_t *>(&l01);
                            lv.y = *reinterpret_cast<const uint32_t *>(&l23);
                            *reinterpret_cast<uint2 *>(tb_Bh + lo_off + off) = lv;
                        }
                    }
                }
            } else {
                for (int e = tid; e < G * NN; e += nt) {
                    const int g = e / NN, rem = e - g * NN, ax = fN.q(rem), k = rem - ax * N, col = g * ND + ax;
                    const float x = (float)cl.map_shared_rank(src, g * C + cr)[rem];
                    const int off = (col >> 3) * SBO + (k >> 3) * 128 + (col & 7) * 16 + (k & 7) * 2;
                    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                    *reinterpret_cast<__nv_bfloat16 *>(tb_Bh + off) = hi;
                    if (na == 2)
                        *reinterpret_cast<__nv_bfloat16 *>(tb_Bh + lo_off + off) = __float2bfloat16_rn(x - __bfloat162float(hi));
                }
            }
            tc::fence_async_shared();
            __syncthreads();
            const bool failed = *tc_flag != 0;
            if (!failed && tid == 0) {
                tc::fence_after_sync();
                const uint32_t idesc = tc::instr_desc(1u, 128, na == 2 ? 32 : 16);
                const uint32_t bh = tc::smem_u32(tb_Bh), d = tmem_base + (uint32_t)tb_dcol;
                for (int j = 0; j < tb_kp / 16; ++j)   // K = 16 per MMA: 8 columns of A, 256 bytes of B
                    tc::mma_bf16_ta(d, tmem_base + 8u * j, tc::smem_desc(bh + 256u * j, 128, SBO), idesc, j > 0 ? 1u : 0u);
                tc::mma_commit(tc_bar + 4);
            }
            bool ok = !failed;
            if (!failed) {
                ok = tc::mbar_wait(tc_bar + 4, tc_done & 1, wbud);
                ++tc_done;
                if (ok) tc_seen = tc_done;
            }
            ok = __all_sync(0xffffffffu, ok);   // tcgen05.ld below is warp-collective
            if (!ok && (tid & 31) == 0) *tc_flag = 1;
            tc::fence_after_sync();
            // D: lanes 0..63 hold A's high parts' rows, 64..127 its low parts' (BF16 x3);
            // columns 0..15 the products with B's high parts, 16..31 with its low parts
            const int wp = tid >> 5, rows = tb_rh - tb_rl, ncol = G * ND, la = tc_na;
            float dv[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) dv[q] = 0.f;
            if (wp < 4 && ok) {
                const uint32_t ta = tmem_base + ((uint32_t)(32 * wp) << 16) + (uint32_t)tb_dcol;
                tc::tmem_ld_x16(ta, dv);
                if (na == 2) {
                    float dl2[16];
                    tc::tmem_ld_x16(ta + 16u, dl2);
#pragma unroll
                    for (int q = 0; q < 16; ++q) dv[q] += dl2[q];
                }
            }
            if (la == 2 && (wp == 2 || wp == 3))   // A's low parts' rows, tid - 64; [column][row]
                for (int q = 0; q < 16; ++q) tb_stage[q * 64 + tid - 64] = dv[q];
            __syncthreads();
            if (wp < 2 && tid < rows)
                for (int q = 0; q < ncol; ++q) dl[q * Lb + tid] = (T)(dv[q] + (la == 2 ? tb_stage[q * 64 + tid] : 0.f));
            tc::fence_before_sync();
            cl.sync();
        }
    }

    // dst = this instance's P~ src (rows gathered from the CTAs of the cluster that own
    // them), then P_b (b - A xi_bar) when corr_b, then n_refine passes of
    // dst += P~ (src - H dst).  Ends with a barrier: every element of dst is valid for
    // every thread.
    __device__ __forceinline__ void tcb_project(cg::cluster_group &cl, const T *src, T *dst, bool corr_b)
    {
        if constexpr (TC && sizeof(T) == 4) {
            auto gather = [&](bool add) {
                if ((N & 3) == 0 && (Lb & 3) == 0) {   // four rows of one owner per 16-byte remote load
                    constexpr int kU = 4;
                    const int tot = NN >> 2;
                    for (int b0 = tid; b0 < tot; b0 += nt * kU) {
                        float4 x4[kU];
#pragma unroll
                        for (int u = 0; u < kU; ++u) {
                            const int idx = b0 + u * nt;
                            if (idx < tot) {
                                const int e = 4 * idx, ax = fN.q(e), row = e - ax * N, own = fLb.q(row);
                                x4[u] = *reinterpret_cast<const float4 *>(cl.map_shared_rank(dl, own) + (grp * ND + ax) * Lb +
                                                                          row - own * Lb);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < kU; ++u) {
                            const int idx = b0 + u * nt;
                            if (idx >= tot) continue;
                            float4 *o = reinterpret_cast<float4 *>(dst) + idx;
                            if (add) {
                                float4 y = *o;
                                y.x += x4[u].x; y.y += x4[u].y; y.z += x4[u].z; y.w += x4[u].w;
                                *o = y;
                            } else {
                                *o = x4[u];
                            }
                        }
                    }
                    return;
                }
                for (int e = tid; e < NN; e += nt) {
                    const int ax = fN.q(e), row = e - ax * N, own = fLb.q(row);
                    const T x = cl.map_shared_rank(dl, own)[(grp * ND + ax) * Lb + row - own * Lb];
                    dst[e] = add ? dst[e] + x : x;
                }
            };
            tcb_product(cl, src);
            gather(false);
            __syncthreads();
            if (corr_b) {   // the first step from an iterate that misses A xi = b
                const int m = nbc * n;
                for (int e = tid; e < NN; e += nt) {
                    const int ax = fN.q(e), row = e - ax * N;
                    T a = T(0);
                    for (int q = 0; q < m; ++q) a += Pbg[(int64_t)row * m + q] * db[ax * n * nbc + q];
                    dst[e] += a;
                }
            }
            for (int pass = 0; pass < n_refine; ++pass) {
                __syncthreads();
                refine_residual(src, dst);
                __syncthreads();
                tcb_product(cl, rr, true);
                gather(true);
            }
            __syncthreads();   // the vector gathers write elements other threads own
        }
    }

    // true when a bounded wait of the tensor-core pipeline ran out in this CTA
    __device__ __forceinline__ bool tc_timed_out() const
    {
        if constexpr (TC && sizeof(T) == 4) return tcm && *tc_flag != 0;
        return false;
    }

    // The refinement residual rr = src - H dst on the coefficients A leaves free, in FP32
    // through H = I (x) C + rho ((n + n_obs + 2) I - 11') (x) W'W, C the cost block (the
    // Kronecker structure of eq. batch_comp's matrix).  Barriers between its two phases only.
    __device__ __forceinline__ void refine_residual(const T *src, const T *dst)
    {
        T *sums = wtw + nxi * nxi;   // [ND][nxi] robot sums of dst
        const int lane = tid & 31, nw = nt >> 5;
        for (int pq = tid >> 5; pq < ND * nxi; pq += nw) {
            const int ax = pq / nxi, c = pq - ax * nxi;
            T sacc = T(0);
            for (int i = lane; i < n; i += 32) sacc += dst[(ax * n + i) * nxi + c];
#pragma unroll
            for (int o = 16; o; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
            if (lane == 0) sums[pq] = sacc;
        }
        __syncthreads();
        const T cn = T(n + n_obs_ + 2);
        for (int e = tid; e < NN; e += nt) {
            const int r = e / nxi, u = e - r * nxi, ax = fn.q(r);
            T hv = T(0), cd = smooth ? T(0) : dst[e];   // C dst: identity or the smoothness block
            for (int c = 0; c < nxi; ++c) {
                hv += wtw[u * nxi + c] * (cn * dst[r * nxi + c] - sums[ax * nxi + c]);
                if (smooth) cd += Qc[u * nxi + c] * dst[r * nxi + c];
            }
            const T res = src[e] - (cd + rho * hv);
            rr[e] = fixed_c(u) ? T(0) : res;
        }
    }

    // dst = P_eta src (+ P_b db when corr_b); dst[e] is valid for the elements e this
    // thread owns (e = tid + j nt).  src and dst must differ from each other and from dl.
    __device__ __forceinline__ void project(cg::cluster_group &cl, const T *src, T *dst, bool corr_b)
    {
        if (TC && dense && tcm && tcb) {
            tcb_project(cl, src, dst, corr_b);
        } else if (TC && dense && tcm) {
            tc_rows(src, corr_b);
            cl.sync();
            for (int e = tid; e < NN; e += nt) {
                const int row = e - fN.q(e) * N;
                dst[e] = cl.map_shared_rank(dl, gb + fL.q(row))[e];
            }
            // refinement: dst += P~ (src - H dst) on the interior coefficients, the residual in
            // FP32 through H = I (x) C + rho ((n + n_obs + 2) I - 11') (x) W'W, C the cost block
            for (int pass = 0; pass < n_refine; ++pass) {
                __syncthreads();
                refine_residual(src, dst);
                __syncthreads();
                tc_rows(rr, false);
                cl.sync();
                for (int e = tid; e < NN; e += nt) {
                    const int row = e - fN.q(e) * N;
                    dst[e] += cl.map_shared_rank(dl, gb + fL.q(row))[e];
                }
            }
        } else if (dense) {
            // rows [r_lo, r_hi) of P_eta src: 8 lanes per row, interleaved columns; the trip
            // count is the same for every thread, so whole warps take part in the shuffles
            const int seg = 8, rows = r_hi - r_lo;
            for (int t0 = 0; t0 < rows * seg; t0 += nt) {
                const int t = t0 + tid;
                const bool act = t < rows * seg;
                const int r = r_lo + t / seg, s = t % seg;
                T acc[ND];
#pragma unroll
                for (int ax = 0; ax < ND; ++ax) acc[ax] = T(0);
                if (act) {
                    const T *pr = Prow + (int64_t)r * N;
                    for (int c = s; c < N; c += seg) {
                        const T pv = pr[c];
#pragma unroll
                        for (int ax = 0; ax < ND; ++ax) acc[ax] += pv * src[ax * N + c];
                    }
                    if (corr_b)
                        for (int q = s; q < nbc * n; q += seg) {
                            const T pbq = Pbg[(int64_t)r * nbc * n + q];
#pragma unroll
                            for (int ax = 0; ax < ND; ++ax) acc[ax] += pbq * db[ax * n * nbc + q];
                        }
                }
#pragma unroll
                for (int ax = 0; ax < ND; ++ax) {
                    T a = acc[ax];
                    a += __shfl_xor_sync(0xffffffffu, a, 4);
                    a += __shfl_xor_sync(0xffffffffu, a, 2);
                    a += __shfl_xor_sync(0xffffffffu, a, 1);
                    if (act && s == 0) dl[ax * N + r] = a;
                }
            }
            cl.sync();
            for (int e = tid; e < NN; e += nt) {
                const int row = e - fN.q(e) * N;
                dst[e] = cl.map_shared_rank(dl, gb + fL.q(row))[e];
            }
        } else {
            // Kronecker form, per axis with robot mean m of src:
            //   dst_i = P_dev src_i + (P_mean - P_dev) m   (+ the same with B for b - A xi_bar)
            // robot means: one thread per (axis, coefficient), four independent partial sums
            // (shorter than a warp's shuffle reduction for tens of robots)
            for (int pq = tid; pq < ND * nxi; pq += nt) {
                const int ax = pq / nxi, c = pq - ax * nxi;
                const T *sp = src + ax * n * nxi + c;
                T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
                int i = 0;
                for (; i + 3 < n; i += 4) {
                    s0 += sp[i * nxi];
                    s1 += sp[(i + 1) * nxi];
                    s2 += sp[(i + 2) * nxi];
                    s3 += sp[(i + 3) * nxi];
                }
                for (; i < n; ++i) s0 += sp[i * nxi];
                mv[pq] = ((s0 + s1) + (s2 + s3)) * invn;
            }
            __syncthreads();
            for (int e = tid; e < ND * nxi; e += nt) {
                const int ax = e / nxi, u = e - ax * nxi;
                T s = T(0);
                for (int c = 0; c < nxi; ++c) s += Pdif[u * nxi + c] * mv[ax * nxi + c];
                if (corr_b)
                    for (int q = 0; q < nbc; ++q) s += Bdif[u * nbc + q] * mb[ax * nbc + q];
                pm[e] = s;
            }
            __syncthreads();
            for (int e = tid; e < NN; e += nt) {
                const int r = e / nxi, u = e - r * nxi, ax = fn.q(r);
                const T *vr = src + r * nxi;
                const T *pu = Pdev + u * nxi;
                T s0 = pm[ax * nxi + u], s1 = T(0);
                int c = 0;
                for (; c + 1 < nxi; c += 2) {
                    s0 += pu[c] * vr[c];
                    s1 += pu[c + 1] * vr[c + 1];
                }
                if (c < nxi) s0 += pu[c] * vr[c];
                if (corr_b)
                    for (int q = 0; q < nbc; ++q) s1 += Bdev[u * nbc + q] * db[r * nbc + q];
                dst[e] = s0 + s1;
            }
        }
    }

    // First half of an iteration of T: rows of this CTA's timesteps, partial g into gme.
    __device__ __forceinline__ void rows_and_g(T *gme, T &rp2, T &mx2)
    {
        for (int e = tid; e < NN; e += nt) gme[e] = T(0);
        for (int k0 = k_lo; k0 < k_hi; k0 += hc) {
            const int hcc = min(hc, k_hi - k0);
            __syncthreads();
            begin_chunk();
            positions(k0, hcc, xb);
            sync_lists();
            cull_lists(k0, hcc);
            rows(k0, hcc, rp2, mx2);
            __syncthreads();
            wt_acc(k0, hcc, Rb, gme);
        }
    }

    // Minus the cost's gradient at xi_bar, element e: xi - xi_bar (projection) or
    // -(Q1 xi_bar_row)_c (smoothness cost, the same block for every robot).
    __device__ __forceinline__ T cost_term(int e) const
    {
        if (!smooth) return xc[e] - xb[e];
        const int r = e / nxi, c = e - r * nxi;
        const T *q = Qc + c * nxi, *x = xb + r * nxi;
        T s = T(0);
        for (int k = 0; k < nxi; ++k) s += q[k] * x[k];
        return -s;
    }

    // update() without side work (the adjoint's recomputation of the iterates)
    __device__ __forceinline__ T update(cg::cluster_group &cl, const T *gme, bool corr_b)
    {
        return update(cl, gme, corr_b, [] {});
    }

    // Sum over this instance's C CTAs of buf[e] (their copies in distributed shared memory),
    // in rank order: every remote load is issued before the first addition, so the C
    // round trips overlap; the same bits in every CTA.
    __device__ __forceinline__ T csum(cg::cluster_group &cl, const T *buf, int e) const
    {
        T x[kMaxCluster];
#pragma unroll
        for (int q = 0; q < kMaxCluster; ++q)
            if (q < C) x[q] = cl.map_shared_rank(buf, gb + q)[e];
        T s = T(0);
#pragma unroll
        for (int q = 0; q < kMaxCluster; ++q)
            if (q < C) s += x[q];
        return s;
    }

    // Per-warp partial statistics into gme[NN + 4 + 3 w + (0, 1, 2)]: sum of rp2, max of mx2,
    // sum of fp over the warp's lanes.
    __device__ __forceinline__ void warp_partials(T *gme, T rp2, T mx2, T fp) const
    {
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            rp2 += __shfl_xor_sync(0xffffffffu, rp2, o);
            mx2 = fmax(mx2, __shfl_xor_sync(0xffffffffu, mx2, o));
            fp += __shfl_xor_sync(0xffffffffu, fp, o);
        }
        if ((tid & 31) == 0) {
            T *g = gme + NN + 4 + 3 * (tid >> 5);
            g[0] = rp2;
            g[1] = mx2;
            g[2] = fp;
        }
    }

    // Cluster statistics from every CTA's per-warp partials (after the cluster barrier that
    // follows warp_partials): the sum of rp2 and the max of mx2 over the cluster, the sum of
    // fp over this CTA (each CTA updates the whole iterate).  Called by one full warp, in a
    // fixed order; the results are valid in every lane.
    __device__ __forceinline__ void cluster_stats(cg::cluster_group &cl, const T *gme, T &s_rp2, T &s_mx2,
                                                  T &s_fp) const
    {
        const int lane = tid & 31, nw = nt >> 5;
        T a = T(0), b = T(0), c = T(0);
        for (int idx = lane; idx < C * nw; idx += 32) {
            const int q = idx / nw, w = idx - q * nw;
            const T *g = cl.map_shared_rank(gme, gb + q) + NN + 4 + 3 * w;
            a += g[0];
            b = fmax(b, g[1]);
            if (q == cr) c += g[2];
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        s_rp2 = a;
        s_mx2 = b;
        s_fp = c;
    }

    // Second half, after the cluster barrier: g = sum over the cluster of gme (fixed order,
    // the same bits in every CTA), lambda step, correction projection, xi_bar update.
    // Returns this thread's share of ||z^{l+1} - z^l||^2.
    // side(): work for the CTA's last warp after its share of the g gather (the cluster
    // statistics of the forward), overlapped with the other warps' gathers.
    template <typename F>
    __device__ __forceinline__ T update(cg::cluster_group &cl, const T *gme, bool corr_b, F &&side)
    {
        T fp = T(0);
        for (int e = tid; e < NN; e += nt) {
            const T gg = csum(cl, gme, e);
            const T ln = lam[e] - rho * gg;
            const T dlam = ln - lam[e];
            fp += dlam * dlam;
            v[e] = cost_term(e) + ln - rho * gg;
            lam[e] = ln;
        }
        if (tid >> 5 == (nt >> 5) - 1) side();
        __syncthreads();
        project(cl, v, dd, corr_b);
        for (int e = tid; e < NN; e += nt) {
            const int r = e / nxi, c = e - r * nxi;
            T xn = xb[e] + dd[e];
            if (c == 0) xn = bf[3 * r];                  // A xi_bar = b holds exactly
            else if (c == nxi - 1) xn = bf[3 * r + 2];
            else if (nbc == 3 && c == 1) xn = bf[3 * r + 1];
            const T dx = xn - xb[e];
            fp += dx * dx;
            xb[e] = xn;
        }
        return fp;
    }
};

// Launches n_inst instances of csize CTAs each of `kernel` with `smem` bytes of dynamic
// shared memory, in clusters of group instances (group csize CTAs; above 8 a non-portable
// cluster size).
template <typename K, typename Arg>
inline cudaError_t launch_cluster(K kernel, const Arg &a, int n_inst, int csize, int group, int threads, size_t smem,
                                  cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int cdim = csize * (group > 1 ? group : 1);
    if (cdim > kMaxCluster) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_inst * csize), 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cdim;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

}  // namespace sf
