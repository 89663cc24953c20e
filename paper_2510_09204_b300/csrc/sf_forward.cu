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
#include <cooperative_groups.h>
#include <math.h>

#include "sf_internal.cuh"

namespace cg = cooperative_groups;

namespace sf {

template <typename T> __device__ __forceinline__ T rsq(T x);
template <> __device__ __forceinline__ float rsq<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsq<double>(double x) { return 1.0 / sqrt(x); }

template <typename T, int K>
struct alignas(K * sizeof(T) >= 16 ? 16 : K * sizeof(T)) Vec {
    T v[K];
};

template <int ND> struct NDP { static constexpr int v = ND == 2 ? 2 : 4; };

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

// squared scaled distance: dx^2 + dy^2 + kz dz^2 with kz = a^2 / b^2
template <typename T, int ND>
__device__ __forceinline__ T qdist(const T (&d)[ND], T kz)
{
    T q = d[0] * d[0] + d[1] * d[1];
    if (ND == 3) q += kz * d[ND - 1] * d[ND - 1];
    return q;
}

// Far-away stand-ins: padded robots sit at +kFar, lanes without an item at -kFar, so
// every distance test against them fails without a bounds check.
template <typename T> struct Far { static constexpr T v = T(1e15); };

// Rows of the items (i, k) of one chunk: positions P[i][kl] (vectors; robots padded to a
// multiple of 4 with far dummies), obstacle records ob[m] = (c_x, c_y, [c_z,] a_o^2, kz_o,
// 1/a_o^2, a_o, b_o) padded the same way; R is written to Rb[ax][i][kl].  Partners and
// obstacles are tested four at a time (independent loads and tests); the warp votes once
// per block and takes the rare active-row path only when one of its lanes needs it.
template <typename T, int ND>
__device__ __forceinline__ void rows_chunk(const Inst<T> &I, const Vec<T, NDP<ND>::v> *P, const T *ob,
                                           const T *obs_g, T *Rb, int k0, int hcc, T &rp2, T &mx2)
{
    using VP = Vec<T, NDP<ND>::v>;
    const int n = I.n, nobs = I.n_obs, items = n * hcc;
    const int npad = (n + 3) & ~3, opad = (nobs + 3) & ~3;
    const T a2 = I.a * I.a, ia2 = I.ia2, kz = (I.a * I.a) * I.ib2;
    T tie_f[ND], tie_b[ND];   // r_1 of a coincident pair seen from the row's first / second robot
#pragma unroll
    for (int ax = 0; ax < ND; ++ax) tie_f[ax] = tie_b[ax] = T(0);
    if (ND == 2) { tie_f[0] = -I.a; tie_b[0] = I.a; }
    else { tie_f[ND - 1] = -I.b; tie_b[ND - 1] = I.b; }
    for (int e0 = 0; e0 < items; e0 += blockDim.x) {
        const int e = e0 + threadIdx.x;
        const bool valid = e < items;
        if (__all_sync(0xffffffffu, !valid)) continue;   // a whole warp without items skips the round
        const int ee = valid ? e : 0;
        const int i = ee / hcc, kl = ee - i * hcc, k = k0 + kl;
        VP pi = P[i * hcc + kl];
        if (!valid)
#pragma unroll
            for (int ax = 0; ax < ND; ++ax) pi.v[ax] = -Far<T>::v;
        T R[ND];
#pragma unroll
        for (int ax = 0; ax < ND; ++ax) R[ax] = T(0);
        // robot pairs: the row of pair (min(i,j), max(i,j)); j == i (q = 0) is sorted out in
        // the slow path
        for (int j0 = 0; j0 < npad; j0 += 4) {
            T d[4][ND], q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const VP pj = P[(j0 + u) * hcc + kl];
#pragma unroll
                for (int ax = 0; ax < ND; ++ax) d[u][ax] = pi.v[ax] - pj.v[ax];
                q[u] = qdist<T, ND>(d[u], kz);
            }
            const bool any = (q[0] <= a2) | (q[1] <= a2) | (q[2] <= a2) | (q[3] <= a2);
            if (__any_sync(0xffffffffu, any)) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = j0 + u;
                    if (q[u] <= a2 && j != i) {
                        if (j > i) row_active<T, ND>(d[u], q[u], ia2, tie_f, R, rp2, mx2, true);
                        else row_active<T, ND>(d[u], q[u], ia2, tie_b, R, rp2, mx2, false);
                    }
                }
            }
        }
        // obstacles
        for (int m0 = 0; m0 < opad; m0 += 4) {
            T d[4][ND], q[4], lim[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int m = m0 + u;
                const Vec<T, 4> r0 = reinterpret_cast<const Vec<T, 4> *>(ob)[2 * m];
                if (I.dyn && m < nobs) {
                    const T *c = obs_g + ((int64_t)m * I.H + k) * ND;
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
                        const int m = m0 + u;
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

// Warp then block reduction of (sum, max, sum) into red[0..2] (all threads participate;
// the result is valid after the caller's next barrier).
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

// MAXT: the launch bound this instantiation is compiled for (512 or, FP32 only, 1024).
template <typename T, int ND, int MAXT>
__global__ void __launch_bounds__(MAXT) k_forward(FwdArgs<T> A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    cg::cluster_group cl = cg::this_cluster();
    const int tid = threadIdx.x, nt = blockDim.x;
    const int C = A.csize, cr = (int)cl.block_rank();
    const int nxi = A.nxi;
    const int w = blockIdx.x / C;
    const int ii = A.order ? A.order[w] : w;
    const Inst<T> I = A.inst[ii];
    const Shape S = A.shapes[I.shape];
    const int n = I.n, H = I.H, N = I.N, nobs = I.n_obs, hc = I.hc;
    const int NN = ND * N;
    const T rho = A.rho;
    const bool dense = A.proj == SF_PROJ_DENSE;
    const T invn = T(1) / T(n);
    // this CTA's timesteps and projection rows
    const int k_lo = (int)((int64_t)cr * H / C), k_hi = (int)((int64_t)(cr + 1) * H / C);
    const int L = (N + C - 1) / C, r_lo = min(N, cr * L), r_hi = min(N, r_lo + L);
    const FwdCarve cv = forward_carve(ND, nxi, H, n, nobs, hc, A.p_rows, (int)sizeof(T));
    T *W = sm + cv.W, *xb = sm + cv.xb, *lam = sm + cv.lam, *xc = sm + cv.xc, *v = sm + cv.v;
    T *gp = sm + cv.gp, *dl = sm + cv.dl, *Rb = sm + cv.Rb, *ob = sm + cv.ob, *bd = sm + cv.bd;
    T *db = sm + cv.db, *sx = sm + cv.sx, *red = sm + cv.red, *Ps = sm + cv.Ps;
    Vec<T, NDP<ND>::v> *P = reinterpret_cast<Vec<T, NDP<ND>::v> *>(sm + cv.pb);
    const int64_t gstride = carve_round(NN + 4, (int)sizeof(T));
    // ---- load
    const T *Wg = A.W + S.off_W;
    for (int e = tid; e < H * nxi; e += nt) W[e] = Wg[e];
    const T *xcg = A.xc + I.off_xi;
    const T *x0g = A.x0 ? A.x0 + I.off_xi : xcg;
    for (int e = tid; e < NN; e += nt) {
        xc[e] = xcg[e];
        xb[e] = x0g[e];
        lam[e] = A.l0 ? A.l0[I.off_xi + e] : T(0);
    }
    for (int e = tid; e < ND * n * 2; e += nt) bd[e] = A.bnd[I.off_bnd + e];
    for (int m = nobs + tid; m < ((nobs + 3) & ~3); m += nt) {   // padding records: far away, zero radius
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
    }
    const T *Pg = A.P + S.off_P;
    const T *Pbg = A.Pb + S.off_Pb;
    if (dense && A.p_rows > 0)
        for (int e = tid; e < (r_hi - r_lo) * N; e += nt) Ps[e] = Pg[(int64_t)r_lo * N + e];
    const T *Prow = (dense && A.p_rows > 0) ? Ps - (int64_t)r_lo * N : Pg;   // Prow[r * N + c], r in [r_lo, r_hi)
    // structured blocks: P_dev, P_mean - P_dev, B_dev, B_mean - B_dev, then mv, pm, mb
    T *Pdev = sx, *Pdif = sx + nxi * nxi, *Bdev = sx + 2 * nxi * nxi, *Bdif = Bdev + 2 * nxi;
    T *mv = Bdif + 2 * nxi, *pm = mv + ND * nxi, *mb = pm + ND * nxi;
    if (!dense) {
        const T *Sg = A.Sx + S.off_S;
        for (int e = tid; e < nxi * nxi; e += nt) {
            Pdev[e] = Sg[e];
            Pdif[e] = Sg[nxi * nxi + e] - Sg[e];
        }
        for (int e = tid; e < 2 * nxi; e += nt) {
            Bdev[e] = Sg[2 * nxi * nxi + e];
            Bdif[e] = Sg[2 * nxi * nxi + 2 * nxi + e] - Sg[2 * nxi * nxi + e];
        }
    }
    __syncthreads();
    // b - A xi_bar^0: nonzero only when the initial iterate misses the boundary values
    int need_b = 0;
    for (int e = tid; e < ND * n * 2; e += nt) {
        const int r = e >> 1, s = e & 1;
        db[e] = bd[e] - xb[r * nxi + (s ? nxi - 1 : 0)];
        if (db[e] != T(0)) need_b = 1;
    }
    need_b = __syncthreads_or(need_b);
    if (need_b && !dense)
        for (int e = tid; e < ND * 2; e += nt) {
            const int ax = e >> 1, s = e & 1;
            T acc = T(0);
            for (int i = 0; i < n; ++i) acc += db[(ax * n + i) * 2 + s];
            mb[e] = acc * invn;
        }

    int its_tol = -1;
    T fp = T(0), fp_prev = T(0);
    T gstat[3] = {T(0), T(0), T(0)};
    bool bad = false;
    for (int it = 0; it <= A.iters; ++it) {
        const bool last = it == A.iters;   // the final pass only reduces the last fixed-point step
        T *gme = gp + (it & 1) * gstride;
        T rp2 = T(0), mx2 = T(0);
        if (!last) {
            if (cr == 0 && A.ck_every > 0 && it % A.ck_every == 0) {
                const int64_t base = (int64_t)(it / A.ck_every) * A.ck_slot + I.off_xi;
                for (int e = tid; e < NN; e += nt) {
                    A.ck_x[base + e] = xb[e];
                    A.ck_l[base + e] = lam[e];
                }
            }
            for (int e = tid; e < NN; e += nt) gme[e] = T(0);
            for (int k0 = k_lo; k0 < k_hi; k0 += hc) {
                const int hcc = min(hc, k_hi - k0);
                __syncthreads();
                // p[ax][i][k] = sum_c W[k][c] xi_bar[ax][i][c], one (axis, robot, timestep) per thread
                T *Ps_ = reinterpret_cast<T *>(P);
                for (int e = tid; e < ND * n * hcc; e += nt) {
                    const int r = e / hcc, kl = e - r * hcc, ax = r / n, i = r - ax * n;
                    const T *wr = W + (k0 + kl) * nxi;
                    const T *xr = xb + r * nxi;
                    T s0 = T(0), s1 = T(0), s2 = T(0);
                    int c = 0;
                    for (; c + 2 < nxi; c += 3) {
                        s0 += wr[c] * xr[c];
                        s1 += wr[c + 1] * xr[c + 1];
                        s2 += wr[c + 2] * xr[c + 2];
                    }
                    for (; c < nxi; ++c) s0 += wr[c] * xr[c];
                    Ps_[(i * hcc + kl) * NDP<ND>::v + ax] = (s0 + s1) + s2;
                }
                for (int e = n * hcc + tid; e < ((n + 3) & ~3) * hcc; e += nt) {   // padding robots
                    Vec<T, NDP<ND>::v> p;
#pragma unroll
                    for (int ax = 0; ax < NDP<ND>::v; ++ax) p.v[ax] = Far<T>::v;
                    P[e] = p;
                }
                __syncthreads();
                rows_chunk<T, ND>(I, P, ob, A.obs + I.off_obs, Rb, k0, hcc, rp2, mx2);
                __syncthreads();
                for (int e = tid; e < NN; e += nt) {
                    const int r = e / nxi, c = e - r * nxi;
                    const T *rr = Rb + r * hcc;
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
                    gme[e] += (s0 + s1) + (s2 + s3);
                }
            }
        }
        // per-CTA stats (this iteration's rows, the previous iteration's step) -> gme[NN..]
        block_reduce3_to<T>(rp2, mx2, fp, red);
        __syncthreads();
        if (tid == 0) {
            gme[NN] = red[96];
            gme[NN + 1] = red[97];
            gme[NN + 2] = red[98];
        }
        cl.sync();
        if (tid == 0) {
            T s_rp2 = T(0), s_mx2 = T(0);
            for (int q = 0; q < C; ++q) {
                const T *rg = cl.map_shared_rank(gme, q);
                s_rp2 += rg[NN];
                s_mx2 = fmax(s_mx2, rg[NN + 1]);
            }
            gstat[0] = s_rp2;
            gstat[1] = s_mx2;
            gstat[2] = gme[NN + 2];
            if (it > 0) {
                fp_prev = gme[NN + 2];
                if (!isfinite(fp_prev)) bad = true;
            }
            if (!last) {
                if (!isfinite(s_rp2)) bad = true;
                const T mxr = sqrt(s_mx2);
                if (its_tol < 0 && (double)mxr <= A.tol) its_tol = it;
                if (A.hist && cr == 0) A.hist[(int64_t)ii * A.iters + it] = (float)mxr;
            }
        }
        if (last) break;
        // g over the cluster (fixed order: the same bits in every CTA), lambda step, correction
        fp = T(0);
        for (int e = tid; e < NN; e += nt) {
            T gg = T(0);
            for (int q = 0; q < C; ++q) gg += cl.map_shared_rank(gme, q)[e];
            const T ln = lam[e] - rho * gg;
            const T dlam = ln - lam[e];
            fp += dlam * dlam;
            v[e] = xc[e] - xb[e] + ln - rho * gg;
            lam[e] = ln;
        }
        __syncthreads();
        const bool corr_b = need_b && it == 0;
        if (dense) {
            // rows [r_lo, r_hi) of P_eta v: 8 lanes per row, interleaved columns
            const int seg = 8, rows = r_hi - r_lo;
            // the trip count is the same for every thread, so whole warps take part in the shuffles
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
                        for (int ax = 0; ax < ND; ++ax) acc[ax] += pv * v[ax * N + c];
                    }
                    if (corr_b)
                        for (int q = s; q < 2 * n; q += seg) {
                            const T pbq = Pbg[(int64_t)r * 2 * n + q];
#pragma unroll
                            for (int ax = 0; ax < ND; ++ax) acc[ax] += pbq * db[(ax * n + (q >> 1)) * 2 + (q & 1)];
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
                const int r = e / nxi, c = e - r * nxi, row = e - (e / N) * N;
                const T *src = cl.map_shared_rank(dl, row / L);
                T xn = xb[e] + src[e];
                if (c == 0) xn = bd[r * 2];                  // A xi_bar = b holds exactly
                else if (c == nxi - 1) xn = bd[r * 2 + 1];
                const T dx = xn - xb[e];
                fp += dx * dx;
                xb[e] = xn;
            }
        } else {
            // Kronecker form, per axis with robot mean m of v:
            //   delta_i = P_dev v_i + (P_mean - P_dev) m   (+ the same with B for b - A xi_bar)
            {   // robot means, one warp per (axis, coefficient), lanes over robots
                const int lane = tid & 31, nw = nt >> 5;
                for (int pq = tid >> 5; pq < ND * nxi; pq += nw) {
                    const int ax = pq / nxi, c = pq - ax * nxi;
                    T s = T(0);
                    for (int i = lane; i < n; i += 32) s += v[(ax * n + i) * nxi + c];
#pragma unroll
                    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                    if (lane == 0) mv[pq] = s * invn;
                }
            }
            __syncthreads();
            for (int e = tid; e < ND * nxi; e += nt) {
                const int ax = e / nxi, u = e - ax * nxi;
                T s = T(0);
                for (int c = 0; c < nxi; ++c) s += Pdif[u * nxi + c] * mv[ax * nxi + c];
                if (corr_b) s += Bdif[u * 2] * mb[ax * 2] + Bdif[u * 2 + 1] * mb[ax * 2 + 1];
                pm[e] = s;
            }
            __syncthreads();
            for (int e = tid; e < NN; e += nt) {
                const int r = e / nxi, u = e - r * nxi, ax = r / n;
                const T *vr = v + r * nxi;
                const T *pu = Pdev + u * nxi;
                T s0 = pm[ax * nxi + u], s1 = T(0);
                int c = 0;
                for (; c + 1 < nxi; c += 2) {
                    s0 += pu[c] * vr[c];
                    s1 += pu[c + 1] * vr[c + 1];
                }
                if (c < nxi) s0 += pu[c] * vr[c];
                if (corr_b) s1 += Bdev[u * 2] * db[r * 2] + Bdev[u * 2 + 1] * db[r * 2 + 1];
                T xn = xb[e] + (s0 + s1);
                if (u == 0) xn = bd[r * 2];
                else if (u == nxi - 1) xn = bd[r * 2 + 1];
                const T dx = xn - xb[e];
                fp += dx * dx;
                xb[e] = xn;
            }
        }
    }
    if (cr == 0) {
        for (int e = tid; e < NN; e += nt) {
            A.xo[I.off_xi + e] = xb[e];
            if (A.lo) A.lo[I.off_xi + e] = lam[e];
        }
        if (A.ck_every > 0 && A.iters % A.ck_every == 0) {
            const int64_t base = (int64_t)(A.iters / A.ck_every) * A.ck_slot + I.off_xi;
            for (int e = tid; e < NN; e += nt) {
                A.ck_x[base + e] = xb[e];
                A.ck_l[base + e] = lam[e];
            }
        }
        if (tid == 0) {
            if (A.resid) {
                A.resid[(int64_t)ii * SF_NRES + SF_RES_FP] = sqrt((double)fp_prev);
                A.resid[(int64_t)ii * SF_NRES + SF_RES_ITERS] = (double)its_tol;
            }
            if (A.its) A.its[ii] = its_tol;
            if (bad) A.status[ii] = SF_ENONFINITE;
        }
    }
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

// ---------------------------------------------------------------------------
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
    for (int e = tid; e < H * nxi; e += nt) W[e] = (double)A.W[S.off_W + e];
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
        const double itv = A.resid[(int64_t)ii * SF_NRES + SF_RES_ITERS];
        if (itv < 0.0 && mx <= A.tol) {
            A.resid[(int64_t)ii * SF_NRES + SF_RES_ITERS] = (double)A.iters;
            if (A.its) A.its[ii] = A.iters;
        }
        if (!isfinite(s_rp2)) A.status[ii] = SF_ENONFINITE;
    }
    cl.sync();
}

template <typename K, typename Arg>
static cudaError_t launch_cluster(K kernel, const Arg &a, int n_inst, int csize, int threads, size_t smem,
                                  cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_inst * csize), 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

template <typename T>
static cudaError_t launch_forward_t(const FwdArgs<T> &a, int threads, size_t smem, cudaStream_t s)
{
    if (a.n_inst < 1 || a.csize < 1 || a.csize > kMaxCluster) return cudaErrorInvalidValue;
    if (threads > max_threads((int)sizeof(T))) return cudaErrorInvalidValue;
    constexpr int big = sizeof(T) == 8 ? 512 : 1024;
    if (threads > 512) {
        if (a.nd == 2) return launch_cluster(k_forward<T, 2, big>, a, a.n_inst, a.csize, threads, smem, s);
        return launch_cluster(k_forward<T, 3, big>, a, a.n_inst, a.csize, threads, smem, s);
    }
    if (a.nd == 2) return launch_cluster(k_forward<T, 2, 512>, a, a.n_inst, a.csize, threads, smem, s);
    return launch_cluster(k_forward<T, 3, 512>, a, a.n_inst, a.csize, threads, smem, s);
}

cudaError_t launch_forward(const FwdArgs<double> &a, int threads, size_t smem, cudaStream_t s)
{
    return launch_forward_t(a, threads, smem, s);
}
cudaError_t launch_forward(const FwdArgs<float> &a, int threads, size_t smem, cudaStream_t s)
{
    return launch_forward_t(a, threads, smem, s);
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
