// Persistent SF forward kernel: every iteration of T (eq. fixed_point) for one
// instance runs inside one CTA, with the iterate, multipliers, candidate, basis,
// positions and (when it fits) the projection operator resident in shared
// memory.  Instances are taken from a largest-first order.
//
// Per iteration, from the current iterate (xi_bar, lambda):
//   positions   p = W xi_bar                               (eq. poly)
//   rows        per (robot i, timestep k): for every partner j and obstacle m the
//               alpha/beta/d closed forms give e; the row residual r_1 = Delta - e is
//               accumulated with the sign of the incidence row (F'), plus the box
//               residual r_2 = max(0, p - p_max) - max(0, p_min - p) (G')
//                                                          (eqs. alpha_step..s_step)
//   g           = W' R = F'r_1 + G'r_2                      (Appendix, structure of F, G)
//   lambda'     = lambda - rho g                            (eq. lambda_step)
//   xi_bar'     = xi_bar + P_eta (xi - xi_bar + lambda' - rho g) [+ P_b (b - A xi_bar)]
//                                                          (eq. xi_step, see below)
// The xi_bar step is applied in correction form: with eta the paper's right-hand
// side and H = I + rho F'F + rho G'G, eta - H xi_bar = xi - xi_bar + lambda' - rho g,
// and P_eta H + P_b A = I, so P_eta eta + P_b b equals the line above exactly.
// The alpha/beta/d steps use the algebraic form of the closed forms: for a row
// with line of sight Delta and q = ||M^-1 Delta||, e = Delta when q >= 1 and
// e = Delta / q otherwise (the scaled radial point on the spheroid); Delta = 0
// maps to e = (a, 0) in 2D and (0, 0, b) in 3D (atan2(0, 0) = 0).
#include <math.h>

#include "sf_internal.cuh"

namespace sf {

template <typename T> __device__ __forceinline__ T rsq(T x);
template <> __device__ __forceinline__ float rsq<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsq<double>(double x) { return 1.0 / sqrt(x); }

// One constraint row: adds sg * r_1 to R, the squared norm to rp2 (if count) and the
// norm to the running max.
template <typename T, int ND>
__device__ __forceinline__ void add_row(const T (&d)[ND], T ia2, T ib2, T ra, T rb, T sg, T (&R)[ND],
                                        T &rp2, T &mx, bool count)
{
    T q2 = (d[0] * d[0] + d[1] * d[1]) * ia2;
    if (ND == 3) q2 += d[ND - 1] * d[ND - 1] * ib2;
    if (q2 <= T(1)) {
        T r1[ND];
        if (q2 > T(0)) {
            const T f = T(1) - rsq(q2);
#pragma unroll
            for (int ax = 0; ax < ND; ++ax) r1[ax] = d[ax] * f;
        } else {
#pragma unroll
            for (int ax = 0; ax < ND; ++ax) r1[ax] = T(0);
            if (ND == 2) r1[0] = -ra; else r1[ND - 1] = -rb;
        }
        T nn = T(0);
#pragma unroll
        for (int ax = 0; ax < ND; ++ax) {
            R[ax] += sg * r1[ax];
            nn += r1[ax] * r1[ax];
        }
        if (count) rp2 += nn;
        mx = fmax(mx, sqrt(nn));
    }
}

// (sum, max, sum) block reduction in double; every thread receives the result.
__device__ __forceinline__ void block_reduce3(double &a, double &b, double &c, double *red)
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
        double x = 0.0, y = 0.0, z = 0.0;
        for (int q = 0; q < nw; ++q) {
            x += red[q];
            y = fmax(y, red[32 + q]);
            z += red[64 + q];
        }
        red[96] = x;
        red[97] = y;
        red[98] = z;
    }
    __syncthreads();
    a = red[96];
    b = red[97];
    c = red[98];
}

// Residual stats and R for the items of one timestep chunk [k0, k0 + hcc).
// pb holds positions [ND][n][hcc]; on return R (registers) has been written over pb.
template <typename T, int ND>
__device__ __forceinline__ void rows_chunk(const Inst<T> &I, const T *pb_in, T *pb,
                                           const T *__restrict__ ob, const T *__restrict__ obs_g, int k0,
                                           int hcc, T &rp2, T &mx)
{
    const int n = I.n, nobs = I.n_obs, tid = threadIdx.x, nt = blockDim.x;
    T R[kIPT][ND];
#pragma unroll
    for (int q = 0; q < kIPT; ++q) {
#pragma unroll
        for (int ax = 0; ax < ND; ++ax) R[q][ax] = T(0);
        const int item = tid + q * nt;
        if (item < n * hcc) {
            const int i = item / hcc, kl = item - (item / hcc) * hcc, k = k0 + kl;
            T pi[ND];
#pragma unroll
            for (int ax = 0; ax < ND; ++ax) pi[ax] = pb_in[(ax * n + i) * hcc + kl];
            // robot pairs (F_r rows): orientation of row (min(i,j), max(i,j))
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                const T sg = j > i ? T(1) : T(-1);
                T d[ND];
#pragma unroll
                for (int ax = 0; ax < ND; ++ax) d[ax] = sg * (pi[ax] - pb_in[(ax * n + j) * hcc + kl]);
                add_row<T, ND>(d, I.ia2, I.ib2, I.a, I.b, sg, R[q], rp2, mx, j > i);
            }
            // obstacles (F_o rows)
            for (int m = 0; m < nobs; ++m) {
                const T *o = ob + m * (ND + 4);
                T d[ND];
                if (I.dyn) {
                    const T *c = obs_g + ((int64_t)m * I.H + k) * ND;
#pragma unroll
                    for (int ax = 0; ax < ND; ++ax) d[ax] = pi[ax] - c[ax];
                } else {
#pragma unroll
                    for (int ax = 0; ax < ND; ++ax) d[ax] = pi[ax] - o[ax];
                }
                add_row<T, ND>(d, o[ND], o[ND + 1], o[ND + 2], o[ND + 3], T(1), R[q], rp2, mx, true);
            }
            // workspace box (G rows, upper then lower side)
#pragma unroll
            for (int ax = 0; ax < ND; ++ax) {
                const T u = pi[ax] - I.pmax[ax];
                const T l = I.pmin[ax] - pi[ax];
                if (u > T(0)) {
                    R[q][ax] += u;
                    rp2 += u * u;
                    mx = fmax(mx, u);
                }
                if (l > T(0)) {
                    R[q][ax] -= l;
                    rp2 += l * l;
                    mx = fmax(mx, l);
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kIPT; ++q) {
        const int item = tid + q * nt;
        if (item < n * hcc) {
            const int i = item / hcc, kl = item - (item / hcc) * hcc;
#pragma unroll
            for (int ax = 0; ax < ND; ++ax) pb[(ax * n + i) * hcc + kl] = R[q][ax];
        }
    }
}

template <typename T, int ND>
__global__ void __launch_bounds__(kMaxThreads) k_forward(FwdArgs<T> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nxi = A.nxi;
    for (int w = blockIdx.x; w < A.n_inst; w += gridDim.x) {
        const int ii = A.order ? A.order[w] : w;
        const Inst<T> I = A.inst[ii];
        const Shape S = A.shapes[I.shape];
        const int n = I.n, H = I.H, N = I.N, nobs = I.n_obs, hc = I.hc;
        const int NN = ND * N;
        const T rho = A.rho;
        // ---- shared-memory carve (sizes mirror forward_smem_bytes on the host)
        T *W = sm;
        T *xb = W + H * nxi;
        T *lam = xb + NN;
        T *xc = lam + NN;
        T *g = xc + NN;
        T *v = g + NN;
        T *pb = v + NN;
        T *ob = pb + ND * n * hc;
        T *bd = ob + nobs * (ND + 4);
        T *sx = bd + ND * n * 2;
        T *endT = sx + (A.proj == SF_PROJ_STRUCTURED ? 2 * nxi * nxi + 4 * nxi + ND * nxi * 2 : 0);
        size_t off = (size_t)((unsigned char *)endT - smem_raw);
        off = (off + 15) & ~(size_t)15;
        double *red = reinterpret_cast<double *>(smem_raw + off);
        T *Ps = reinterpret_cast<T *>(red + kRedDoubles);
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
        for (int m = tid; m < nobs; m += nt) {
            const T ao = A.oab[I.off_oab + 2 * m], bo = A.oab[I.off_oab + 2 * m + 1];
            T *o = ob + m * (ND + 4);
            if (!I.dyn)
                for (int ax = 0; ax < ND; ++ax) o[ax] = A.obs[I.off_obs + (int64_t)m * ND + ax];
            o[ND] = T(1) / (ao * ao);
            o[ND + 1] = T(1) / (bo * bo);
            o[ND + 2] = ao;
            o[ND + 3] = bo;
        }
        const T *Pg = A.P + S.off_P;
        const T *Pbg = A.Pb + S.off_Pb;
        if (A.p_smem && A.proj == SF_PROJ_DENSE)
            for (int e = tid; e < N * N; e += nt) Ps[e] = Pg[e];
        if (A.proj == SF_PROJ_STRUCTURED)
            for (int e = tid; e < 2 * nxi * nxi + 4 * nxi; e += nt) sx[e] = A.Sx[S.off_S + e];
        const T *Pm = (A.p_smem && A.proj == SF_PROJ_DENSE) ? Ps : Pg;
        __syncthreads();
        // boundary mismatch of the initial iterate: P_b (b - A xi_bar^0) joins the first step
        int need_b = 0;
        for (int e = tid; e < ND * n * 2; e += nt) {
            const int r = e >> 1, s = e & 1;
            if (xb[r * nxi + (s ? nxi - 1 : 0)] != bd[e]) need_b = 1;
        }
        need_b = __syncthreads_or(need_b);

        int its_tol = -1;
        double fp_last = 0.0;
        int bad = 0;
        for (int it = 0; it < A.iters; ++it) {
            if (A.ck_every > 0 && it % A.ck_every == 0) {
                const int64_t base = (int64_t)(it / A.ck_every) * A.ck_slot + I.off_xi;
                for (int e = tid; e < NN; e += nt) {
                    A.ck_x[base + e] = xb[e];
                    A.ck_l[base + e] = lam[e];
                }
            }
            for (int e = tid; e < NN; e += nt) g[e] = T(0);
            T rp2 = T(0), mx = T(0);
            for (int k0 = 0; k0 < H; k0 += hc) {
                const int hcc = min(hc, H - k0);
                __syncthreads();
                for (int e = tid; e < ND * n * hcc; e += nt) {
                    const int r = e / hcc, kl = e - r * hcc;
                    const T *wr = W + (k0 + kl) * nxi;
                    const T *xr = xb + r * nxi;
                    T s = T(0);
                    for (int c = 0; c < nxi; ++c) s += wr[c] * xr[c];
                    pb[r * hcc + kl] = s;
                }
                __syncthreads();
                rows_chunk<T, ND>(I, pb, pb, ob, A.obs + I.off_obs, k0, hcc, rp2, mx);
                __syncthreads();
                for (int e = tid; e < NN; e += nt) {
                    const int r = e / nxi, c = e - r * nxi;
                    const T *rr = pb + r * hcc;
                    T s = T(0);
                    for (int kl = 0; kl < hcc; ++kl) s += W[(k0 + kl) * nxi + c] * rr[kl];
                    g[e] += s;
                }
            }
            __syncthreads();
            T fp = T(0);
            for (int e = tid; e < NN; e += nt) {
                const T gg = g[e];
                const T ln = lam[e] - rho * gg;
                const T dl = ln - lam[e];
                fp += dl * dl;
                v[e] = xc[e] - xb[e] + ln - rho * gg;
                lam[e] = ln;
            }
            __syncthreads();
            // ---- projection: delta = P_eta v (+ P_b (b - A xi_bar) on the first step) -> g
            const bool corr_b = need_b && it == 0;
            if (A.proj == SF_PROJ_DENSE) {
                for (int r = tid; r < N; r += nt) {
                    T acc[ND];
#pragma unroll
                    for (int ax = 0; ax < ND; ++ax) acc[ax] = T(0);
                    for (int c = 0; c < N; ++c) {
                        const T pv = Pm[(int64_t)c * N + r];
#pragma unroll
                        for (int ax = 0; ax < ND; ++ax) acc[ax] += pv * v[ax * N + c];
                    }
                    if (corr_b) {
                        for (int q = 0; q < 2 * n; ++q) {
                            const T pbq = Pbg[(int64_t)r * 2 * n + q];
                            const int i = q >> 1, s = q & 1;
#pragma unroll
                            for (int ax = 0; ax < ND; ++ax)
                                acc[ax] += pbq * (bd[(ax * n + i) * 2 + s] - xb[(ax * n + i) * nxi + (s ? nxi - 1 : 0)]);
                        }
                    }
#pragma unroll
                    for (int ax = 0; ax < ND; ++ax) g[ax * N + r] = acc[ax];
                }
            } else {
                // Kronecker form: per axis, with mean m over robots,
                //   delta_i = P_dev (v_i - m) + P_mean m   (+ the same with B for b - A xi_bar)
                T *mv = sx + 2 * nxi * nxi + 4 * nxi;   // [ND][nxi] robot means of v
                T *mb = mv + ND * nxi;                    // [ND][2] robot means of b - A xi_bar
                for (int e = tid; e < ND * nxi; e += nt) {
                    const int ax = e / nxi, c = e - ax * nxi;
                    T s = T(0);
                    for (int i = 0; i < n; ++i) s += v[(ax * n + i) * nxi + c];
                    mv[e] = s / T(n);
                }
                if (corr_b)
                    for (int e = tid; e < ND * 2; e += nt) {
                        const int ax = e >> 1, s = e & 1;
                        T acc = T(0);
                        for (int i = 0; i < n; ++i)
                            acc += bd[(ax * n + i) * 2 + s] - xb[(ax * n + i) * nxi + (s ? nxi - 1 : 0)];
                        mb[e] = acc / T(n);
                    }
                __syncthreads();
                const T *Pdev = sx, *Pmean = sx + nxi * nxi, *Bdev = sx + 2 * nxi * nxi, *Bmean = Bdev + 2 * nxi;
                for (int e = tid; e < NN; e += nt) {
                    const int r = e / nxi, u = e - r * nxi, ax = r / n;
                    const T *vr = v + r * nxi;
                    const T *m = mv + ax * nxi;
                    T acc = T(0);
                    for (int c = 0; c < nxi; ++c) acc += Pdev[u * nxi + c] * (vr[c] - m[c]) + Pmean[u * nxi + c] * m[c];
                    if (corr_b) {
                        for (int s = 0; s < 2; ++s) {
                            const T db = bd[r * 2 + s] - xb[r * nxi + (s ? nxi - 1 : 0)];
                            acc += Bdev[u * 2 + s] * (db - mb[ax * 2 + s]) + Bmean[u * 2 + s] * mb[ax * 2 + s];
                        }
                    }
                    g[e] = acc;
                }
            }
            __syncthreads();
            for (int e = tid; e < NN; e += nt) {
                const int r = e / nxi, c = e - r * nxi;
                T xn = xb[e] + g[e];
                if (c == 0) xn = bd[r * 2];                 // A xi_bar = b holds exactly
                else if (c == nxi - 1) xn = bd[r * 2 + 1];
                const T dx = xn - xb[e];
                fp += dx * dx;
                xb[e] = xn;
            }
            double s_rp2 = (double)rp2, s_mx = (double)mx, s_fp = (double)fp;
            block_reduce3(s_rp2, s_mx, s_fp, red);
            if (!isfinite(s_fp) || !isfinite(s_rp2)) bad = 1;
            if (its_tol < 0 && s_mx <= A.tol) its_tol = it;
            fp_last = s_fp;
            if (A.hist && tid == 0) A.hist[(int64_t)ii * A.iters + it] = (float)s_mx;
        }
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
                A.resid[(int64_t)ii * SF_NRES + SF_RES_FP] = sqrt(fp_last);
                A.resid[(int64_t)ii * SF_NRES + SF_RES_ITERS] = (double)its_tol;
            }
            if (A.its) A.its[ii] = its_tol;
            if (bad) A.status[ii] = SF_ENONFINITE;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// FP64 residual of packed coefficients x (reading of eq. primal_residual):
// ||r_p||_2 and the max row residual in metres.  One CTA per instance; the same
// row algebra as the forward kernel, in double whatever the solve precision.
template <typename T, int ND>
__global__ void __launch_bounds__(kMaxThreads) k_residual(ResArgs<T> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *sm = reinterpret_cast<double *>(smem_raw);
    const int tid = threadIdx.x, nt = blockDim.x, nxi = A.nxi;
    const int ii = blockIdx.x;
    const Inst<T> I = A.inst[ii];
    const Shape S = A.shapes[I.shape];
    const int n = I.n, H = I.H, nobs = I.n_obs;
    const int64_t fixed = (int64_t)H * nxi + (int64_t)ND * I.N + (int64_t)nobs * (ND + 4) + kRedDoubles;
    int hc = (int)((A.smem_doubles - fixed) / (ND * n));
    hc = hc < 1 ? 1 : (hc > H ? H : hc);
    double *W = sm;
    double *xb = W + H * nxi;
    double *pb = xb + ND * I.N;
    double *ob = pb + ND * n * hc;
    double *red = ob + nobs * (ND + 4);
    Inst<double> Id;
    Id.n = n; Id.n_obs = nobs; Id.H = H; Id.dyn = I.dyn; Id.N = I.N; Id.hc = hc;
    Id.ia2 = (double)I.ia2; Id.ib2 = (double)I.ib2; Id.a = (double)I.a; Id.b = (double)I.b;
    for (int ax = 0; ax < 3; ++ax) { Id.pmin[ax] = (double)I.pmin[ax]; Id.pmax[ax] = (double)I.pmax[ax]; }
    for (int e = tid; e < H * nxi; e += nt) W[e] = (double)A.W[S.off_W + e];
    for (int e = tid; e < ND * I.N; e += nt) xb[e] = (double)A.x[I.off_xi + e];
    for (int m = tid; m < nobs; m += nt) {
        const double ao = (double)A.oab[I.off_oab + 2 * m], bo = (double)A.oab[I.off_oab + 2 * m + 1];
        double *o = ob + m * (ND + 4);
        if (!I.dyn)
            for (int ax = 0; ax < ND; ++ax) o[ax] = (double)A.obs[I.off_obs + (int64_t)m * ND + ax];
        o[ND] = 1.0 / (ao * ao);
        o[ND + 1] = 1.0 / (bo * bo);
        o[ND + 2] = ao;
        o[ND + 3] = bo;
    }
    __syncthreads();
    double rp2 = 0.0, mx = 0.0;
    for (int k0 = 0; k0 < H; k0 += hc) {
        const int hcc = min(hc, H - k0);
        __syncthreads();
        for (int e = tid; e < ND * n * hcc; e += nt) {
            const int r = e / hcc, kl = e - r * hcc;
            double s = 0.0;
            for (int c = 0; c < nxi; ++c) s += W[(k0 + kl) * nxi + c] * xb[r * nxi + c];
            pb[r * hcc + kl] = s;
        }
        __syncthreads();
        // rows_chunk writes R over its position buffer; evaluate into registers only here
        const int items = n * hcc;
        for (int item = tid; item < items; item += nt) {
            const int i = item / hcc, kl = item - i * hcc, k = k0 + kl;
            double pi[ND];
            for (int ax = 0; ax < ND; ++ax) pi[ax] = pb[(ax * n + i) * hcc + kl];
            double R[ND];
            for (int ax = 0; ax < ND; ++ax) R[ax] = 0.0;
            for (int j = i + 1; j < n; ++j) {
                double d[ND];
                for (int ax = 0; ax < ND; ++ax) d[ax] = pi[ax] - pb[(ax * n + j) * hcc + kl];
                add_row<double, ND>(d, Id.ia2, Id.ib2, Id.a, Id.b, 1.0, R, rp2, mx, true);
            }
            for (int m = 0; m < nobs; ++m) {
                const double *o = ob + m * (ND + 4);
                double d[ND];
                if (I.dyn) {
                    const T *c = A.obs + I.off_obs + ((int64_t)m * H + k) * ND;
                    for (int ax = 0; ax < ND; ++ax) d[ax] = pi[ax] - (double)c[ax];
                } else {
                    for (int ax = 0; ax < ND; ++ax) d[ax] = pi[ax] - o[ax];
                }
                add_row<double, ND>(d, o[ND], o[ND + 1], o[ND + 2], o[ND + 3], 1.0, R, rp2, mx, true);
            }
            for (int ax = 0; ax < ND; ++ax) {
                const double u = pi[ax] - Id.pmax[ax], l = Id.pmin[ax] - pi[ax];
                if (u > 0.0) { rp2 += u * u; mx = fmax(mx, u); }
                if (l > 0.0) { rp2 += l * l; mx = fmax(mx, l); }
            }
        }
    }
    double dummy = 0.0;
    block_reduce3(rp2, mx, dummy, red);
    if (tid == 0) {
        A.resid[(int64_t)ii * SF_NRES + SF_RES_RP] = sqrt(rp2);
        A.resid[(int64_t)ii * SF_NRES + SF_RES_MAX] = mx;
        double it = A.resid[(int64_t)ii * SF_NRES + SF_RES_ITERS];
        if (it < 0.0 && mx <= A.tol) {
            A.resid[(int64_t)ii * SF_NRES + SF_RES_ITERS] = (double)A.iters;
            if (A.its) A.its[ii] = A.iters;
        }
        if (!isfinite(rp2)) A.status[ii] = SF_ENONFINITE;
    }
}

template <typename T>
static cudaError_t launch_forward_t(const FwdArgs<T> &a, int grid, int threads, size_t smem, cudaStream_t s)
{
    if (a.nd == 2) {
        cudaFuncSetAttribute(k_forward<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_forward<T, 2><<<grid, threads, smem, s>>>(a);
    } else {
        cudaFuncSetAttribute(k_forward<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_forward<T, 3><<<grid, threads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_forward(const FwdArgs<double> &a, int grid, int threads, size_t smem, cudaStream_t s)
{
    return launch_forward_t(a, grid, threads, smem, s);
}
cudaError_t launch_forward(const FwdArgs<float> &a, int grid, int threads, size_t smem, cudaStream_t s)
{
    return launch_forward_t(a, grid, threads, smem, s);
}

template <typename T>
static cudaError_t launch_residual_t(const ResArgs<T> &a, int threads, size_t smem, cudaStream_t s)
{
    if (a.nd == 2) {
        cudaFuncSetAttribute(k_residual<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_residual<T, 2><<<a.n_inst, threads, smem, s>>>(a);
    } else {
        cudaFuncSetAttribute(k_residual<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_residual<T, 3><<<a.n_inst, threads, smem, s>>>(a);
    }
    return cudaGetLastError();
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
