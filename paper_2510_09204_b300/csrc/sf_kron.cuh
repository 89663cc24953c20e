// The Kronecker blocks of one shape's xi_bar-step operator (Appendix, M and eta of
// eq. xi_step, in the structured form), shared by the handle factorisation and the
// allocation-free entry point.
//
// The Hessian I_n (x) C + rho ((n + n_obs + 2) I - 11') (x) W'W has eigenvalue
// n + n_obs + 2 of its robot factor on the deviation from the robot mean and n_obs + 2
// on the mean, and A = I_n (x) A0 commutes with that split, so P_dev / P_mean and
// B_dev / B_mean are the (x, x) and (x, b) blocks of the inverse of
// [[C + rho c W'W, A0'], [A0, 0]] (A0: the nbc boundary rows of one robot) for the two
// values of c.
#pragma once
#include "sf_internal.cuh"

namespace sf {

constexpr int kKronMax = 32 + 3;   // n_xi + boundary rows

// Shared memory of kron_kkt_blocks.
struct KronSmem {
    double wtw[32 * 32];
    double K[kKronMax * kKronMax], X[kKronMax * kKronMax];
    int piv, bad;
};

// All threads of one CTA call it.  Ws: the shape's basis [H][nxi]; Cb: the per-robot cost
// block [nxi][nxi]; out: P_dev, P_mean [nxi][nxi], B_dev, B_mean [nxi][nbc], back to back.
// Gauss-Jordan elimination with partial pivoting; returns 0, or the first zero pivot + 1
// (the blocks are then not written).
__device__ inline int kron_kkt_blocks(const Shape &S, int nxi, double rho, const double *Ws, const double *Cb,
                                      double *out, KronSmem &sm)
{
    const int tid = threadIdx.x, nt = blockDim.x, nbc = S.nbc, m = nxi + nbc, H = S.H;
    double *wtw = sm.wtw, *K = sm.K, *X = sm.X;
    if (tid == 0) sm.bad = 0;
    for (int e = tid; e < nxi * nxi; e += nt) {
        const int u = e / nxi, v = e % nxi;
        double acc = 0.0;
        for (int k = 0; k < H; ++k) acc += Ws[k * nxi + u] * Ws[k * nxi + v];
        wtw[e] = acc;
    }
    for (int pass = 0; pass < 2; ++pass) {
        const double c = pass == 0 ? (double)(S.n + S.n_obs + 2) : (double)(S.n_obs + 2);
        __syncthreads();
        for (int e = tid; e < m * m; e += nt) {
            const int r = e / m, q = e % m;
            double val;
            if (r < nxi && q < nxi) val = Cb[r * nxi + q] + rho * c * wtw[r * nxi + q];
            else if (r < nxi) val = a0_row(Ws, nxi, H, q - nxi, r, S.vsc);
            else if (q < nxi) val = a0_row(Ws, nxi, H, r - nxi, q, S.vsc);
            else val = 0.0;
            K[e] = val;
            X[e] = r == q ? 1.0 : 0.0;
        }
        for (int p = 0; p < m; ++p) {
            __syncthreads();
            if (tid == 0) {
                int best = p;
                for (int r = p + 1; r < m; ++r)
                    if (fabs(K[r * m + p]) > fabs(K[best * m + p])) best = r;
                sm.piv = best;
                if (!(fabs(K[best * m + p]) > 0.0) && !sm.bad) sm.bad = p + 1;
            }
            __syncthreads();
            if (sm.bad) break;
            const int b = sm.piv;
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
            // eliminate column p from the other rows; column p itself is read by every
            // update, so it is cleared only after a barrier
            for (int e = tid; e < m * m; e += nt) {
                const int r = e / m, q = e % m;
                if (r == p || q == p) continue;
                K[r * m + q] -= K[r * m + p] * K[p * m + q];
            }
            for (int e = tid; e < m * m; e += nt) {
                const int r = e / m, q = e % m;
                if (r == p) continue;
                X[r * m + q] -= K[r * m + p] * X[p * m + q];
            }
            __syncthreads();
            for (int r = tid; r < m; r += nt)
                if (r != p) K[r * m + p] = 0.0;
        }
        __syncthreads();
        if (sm.bad) break;
        double *Po = out + pass * nxi * nxi, *Bo = out + 2 * nxi * nxi + pass * nbc * nxi;
        for (int e = tid; e < nxi * nxi; e += nt) Po[e] = X[(e / nxi) * m + e % nxi];
        for (int e = tid; e < nxi * nbc; e += nt) Bo[e] = X[(e / nbc) * m + nxi + e % nbc];
    }
    __syncthreads();
    return sm.bad;
}

}  // namespace sf
