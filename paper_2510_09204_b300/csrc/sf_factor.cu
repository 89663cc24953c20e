// FP64 factorisation of the xi_bar-step operator, once per (n, n_obs, H) shape.
//
// The xi_bar step (Appendix, eq. xi_step) is the equality-constrained QP
//   argmin_x 1/2 x'Hx - eta'x  s.t.  A x = b,   H = I + rho F'F + rho G'G,
// whose matrix does not depend on the candidate, so it is factored once and
// stored (the Appendix's remark on refactorisation: only rho or the horizon
// change it).  With F_r = D (x) W (pair incidence), F_o = I (x) stack(W) and
// the two-sided box G = [I (x) W; -I (x) W], the Hessian is
//   H = I_N + rho ((n + n_obs + 2) I_n - 1 1') (x) W'W,
// assembled here from that identity and then factored densely:
//   H = L L' (Cholesky), Hinv = L^-T L^-1, Y = Hinv A', S = A Y (Schur
//   complement), P_b = Y S^-1, P_eta = Hinv - P_b Y'.
// so that argmin = P_eta eta + P_b b.  Every step runs in FP64 on the GPU.
#include <cuda_bf16.h>
#include <math.h>

#include "sf_internal.cuh"
#include "sf_kron.cuh"
#include "sf_tc.cuh"

#include <algorithm>

namespace sf {

// Bernstein basis W[k][c] = C(deg, c) tau^c (1 - tau)^(deg - c), tau = k / (H - 1)
__global__ void k_basis(const Shape *sh, int nxi, double *W)
{
    const Shape S = sh[blockIdx.x];
    double *Ws = W + S.off_W;
    const int deg = nxi - 1;
    for (int e = threadIdx.x; e < S.H * nxi; e += blockDim.x) {
        const int k = e / nxi, c = e % nxi;
        const double tau = (double)k / (double)(S.H - 1);
        double bin = 1.0;
        for (int q = 1; q <= c; ++q) bin = bin * (double)(deg - c + q) / (double)q;
        Ws[e] = bin * pow(tau, (double)c) * pow(1.0 - tau, (double)(deg - c));
    }
}

// Per-robot block of the cost's Hessian, into the shape's Kronecker record after the
// projection blocks: the identity (projection cost) or Q1 = Wdd' Wdd (smoothness cost,
// eq. cost), Wdd the second time derivative of the basis at t_k = k dt: d (d - 1) / T^2
// times the second difference of the degree-(d - 2) Bernstein polynomials, T = (H-1) dt.
__global__ void k_cost_block(const Shape *sh, int nxi, int cost, double dt, double *Sx)
{
    const Shape S = sh[blockIdx.x];
    double *Cb = Sx + S.off_S + kron_cost_off(nxi, S.nbc);
    const int deg = nxi - 1, H = S.H;
    const double T = (double)(H - 1) * dt, scale = (double)deg * (double)(deg - 1) / (T * T);
    for (int e = threadIdx.x; e < nxi * nxi; e += blockDim.x) {
        const int u = e / nxi, v = e % nxi;
        if (cost == SF_COST_PROJECTION) {
            Cb[e] = u == v ? 1.0 : 0.0;
            continue;
        }
        double q = 0.0;
        for (int k = 0; k < H; ++k) {
            const double tau = (double)k / (double)(H - 1);
            double du = 0.0, dv = 0.0;
            for (int j = 0; j <= deg - 2; ++j) {
                double bin = 1.0;
                for (int t = 1; t <= j; ++t) bin = bin * (double)(deg - 2 - j + t) / (double)t;
                const double b = bin * pow(tau, (double)j) * pow(1.0 - tau, (double)(deg - 2 - j));
                // B_c'' gets + b for j = c - 2 and j = c, - 2 b for j = c - 1
                if (j == u - 2 || j == u) du += b;
                if (j == u - 1) du -= 2.0 * b;
                if (j == v - 2 || j == v) dv += b;
                if (j == v - 1) dv -= 2.0 * b;
            }
            q += (scale * du) * (scale * dv);
        }
        Cb[e] = q;
    }
}

__global__ void k_build_H(const Shape *sh, int nxi, double rho, const double *W, const double *Sx, double *Hs)
{
    const Shape S = sh[blockIdx.y];
    const int N = S.N;
    double *Hm = Hs + S.off_P;
    const double *Ws = W + S.off_W;
    const double *Cb = Sx + S.off_S + kron_cost_off(nxi, S.nbc);   // per-robot cost block
    const double cdiag = (double)(S.n + S.n_obs + 2);
    const int64_t tot = (int64_t)N * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / N), c = (int)(e % N);
        const int i = r / nxi, u = r % nxi, j = c / nxi, v = c % nxi;
        double wtw = 0.0;
        for (int k = 0; k < S.H; ++k) wtw += Ws[k * nxi + u] * Ws[k * nxi + v];
        const double lap = (i == j ? cdiag : 0.0) - 1.0;
        Hm[e] = (i == j ? Cb[u * nxi + v] : 0.0) + rho * lap * wtw;
    }
}

// Right-looking Cholesky, one CTA per shape, in place (lower triangle).  info = 0 or pivot + 1.
__global__ void k_cholesky(const Shape *sh, double *Hs, int *info)
{
    const Shape S = sh[blockIdx.x];
    const int N = S.N, tid = threadIdx.x, nt = blockDim.x;
    double *A = Hs + S.off_P;
    __shared__ double piv;
    __shared__ int bad;
    if (tid == 0) bad = 0;
    for (int j = 0; j < N; ++j) {
        __syncthreads();
        if (tid == 0) {
            double d = A[(int64_t)j * N + j];
            if (!(d > 0.0)) {
                if (!bad) bad = j + 1;
                d = 1.0;
            }
            piv = sqrt(d);
            A[(int64_t)j * N + j] = piv;
        }
        __syncthreads();
        const double p = piv;
        for (int i = j + 1 + tid; i < N; i += nt) A[(int64_t)i * N + j] /= p;
        __syncthreads();
        const int m = N - j - 1;
        const int64_t tot = (int64_t)m * m;
        for (int64_t t = tid; t < tot; t += nt) {
            const int ii = (int)(t / m), kk = (int)(t % m);
            if (kk <= ii) {
                const int i = j + 1 + ii, k = j + 1 + kk;
                A[(int64_t)i * N + k] -= A[(int64_t)i * N + j] * A[(int64_t)k * N + j];
            }
        }
    }
    __syncthreads();
    for (int64_t t = tid; t < (int64_t)N * N; t += nt) {
        const int i = (int)(t / N), k = (int)(t % N);
        if (k > i) A[t] = 0.0;
    }
    if (tid == 0) info[blockIdx.x] = bad;
}

// Hinv = (L L')^-1, one thread per column: forward then backward substitution.
__global__ void k_chol_inverse(const Shape *sh, const double *Ls_pool, double *X_pool)
{
    const Shape S = sh[blockIdx.y];
    const int N = S.N;
    if (blockIdx.x * blockDim.x >= N) return;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N) return;
    const double *L = Ls_pool + S.off_P;
    double *X = X_pool + S.off_P;
    for (int i = 0; i < N; ++i) {
        double s = (i == q) ? 1.0 : 0.0;
        for (int k = 0; k < i; ++k) s -= L[(int64_t)i * N + k] * X[(int64_t)k * N + q];
        X[(int64_t)i * N + q] = s / L[(int64_t)i * N + i];
    }
    for (int i = N - 1; i >= 0; --i) {
        double s = X[(int64_t)i * N + q];
        for (int k = i + 1; k < N; ++k) s -= L[(int64_t)k * N + i] * X[(int64_t)k * N + q];
        X[(int64_t)i * N + q] = s / L[(int64_t)i * N + i];
    }
}

// Per shape (one CTA): Y = Hinv A', S = A Y, Cholesky of S, Sinv, P_b = Y Sinv, with A's
// row q = nbc i + s the boundary row s of robot i (a0_row).
// Y goes to Ypool (N x nbc n), S / Sinv to Spool ((nbc n)^2 each, within the N^2 slot).
__global__ void k_schur(const Shape *sh, int nxi, const double *W, const double *Hinv, double *Ypool,
                        double *Spool, double *Pb, int *info)
{
    const Shape S = sh[blockIdx.x];
    const int N = S.N, n = S.n, nbc = S.nbc, m = nbc * n, tid = threadIdx.x, nt = blockDim.x;
    const double *Ws = W + S.off_W;
    const double *Hi = Hinv + S.off_P;
    double *Y = Ypool + S.off_P;
    double *Sm = Spool + S.off_P;
    double *Si = Sm + (int64_t)m * m;
    double *B = Pb + S.off_Pb;
    for (int64_t e = tid; e < (int64_t)N * m; e += nt) {
        const int r = (int)(e / m), q = (int)(e % m), i = q / nbc, s = q % nbc;
        double acc = 0.0;
        for (int c = 0; c < nxi; ++c) acc += Hi[(int64_t)r * N + i * nxi + c] * a0_row(Ws, nxi, S.H, s, c, S.vsc);
        Y[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < m * m; e += nt) {
        const int q = e / m, q2 = e % m, i = q / nbc, s = q % nbc;
        double acc = 0.0;
        for (int c = 0; c < nxi; ++c) acc += a0_row(Ws, nxi, S.H, s, c, S.vsc) * Y[(int64_t)(i * nxi + c) * m + q2];
        Sm[e] = acc;
    }
    // Cholesky of S (m <= 2 * 64 * ... small), then Sinv column by column
    __shared__ double piv;
    __shared__ int bad;
    if (tid == 0) bad = 0;
    for (int j = 0; j < m; ++j) {
        __syncthreads();
        if (tid == 0) {
            double d = Sm[j * m + j];
            if (!(d > 0.0)) {
                if (!bad) bad = N + j + 1;
                d = 1.0;
            }
            piv = sqrt(d);
            Sm[j * m + j] = piv;
        }
        __syncthreads();
        for (int i = j + 1 + tid; i < m; i += nt) Sm[i * m + j] /= piv;
        __syncthreads();
        const int mm = m - j - 1;
        for (int t = tid; t < mm * mm; t += nt) {
            const int ii = t / mm, kk = t % mm;
            if (kk <= ii) Sm[(j + 1 + ii) * m + j + 1 + kk] -= Sm[(j + 1 + ii) * m + j] * Sm[(j + 1 + kk) * m + j];
        }
    }
    __syncthreads();
    for (int q = tid; q < m; q += nt) {
        for (int i = 0; i < m; ++i) {
            double s = (i == q) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= Sm[i * m + k] * Si[k * m + q];
            Si[i * m + q] = s / Sm[i * m + i];
        }
        for (int i = m - 1; i >= 0; --i) {
            double s = Si[i * m + q];
            for (int k = i + 1; k < m; ++k) s -= Sm[k * m + i] * Si[k * m + q];
            Si[i * m + q] = s / Sm[i * m + i];
        }
    }
    __syncthreads();
    for (int64_t e = tid; e < (int64_t)N * m; e += nt) {
        const int r = (int)(e / m), q = (int)(e % m);
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc += Y[(int64_t)r * m + k] * Si[k * m + q];
        B[e] = acc;
    }
    if (tid == 0 && bad && !info[blockIdx.x]) info[blockIdx.x] = bad;
}

// P_eta = Hinv - P_b Y'   (in place over Hinv)
__global__ void k_peta(const Shape *sh, const double *Ypool, const double *Pb, double *P)
{
    const Shape S = sh[blockIdx.y];
    const int N = S.N, m = S.nbc * S.n;
    const double *Y = Ypool + S.off_P;
    const double *B = Pb + S.off_Pb;
    double *Pe = P + S.off_P;
    const int64_t tot = (int64_t)N * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / N), c = (int)(e % N);
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc += B[(int64_t)r * m + k] * Y[(int64_t)c * m + k];
        Pe[e] -= acc;
    }
}

// Kronecker blocks of the dense operators: P_eta = (I - Q) (x) P_dev + Q (x) P_mean with
// Q = 11'/n, read off robot blocks (0,0) and (0,1); the same for P_b with B_dev, B_mean.
// Layout per shape at off_S: P_dev [nxi][nxi], P_mean [nxi][nxi], B_dev [nxi][nbc], B_mean [nxi][nbc].
__global__ void k_structured(const Shape *sh, int nxi, const double *P, const double *Pb, double *Sx)
{
    const Shape S = sh[blockIdx.x];
    const int N = S.N, n = S.n, nbc = S.nbc, m = nbc * n;
    const double *Pe = P + S.off_P;
    const double *B = Pb + S.off_Pb;
    double *o = Sx + S.off_S;
    for (int e = threadIdx.x; e < nxi * nxi; e += blockDim.x) {
        const int u = e / nxi, v = e % nxi;
        const double d0 = Pe[(int64_t)u * N + v];
        const double d1 = n > 1 ? Pe[(int64_t)u * N + nxi + v] : 0.0;
        o[e] = n > 1 ? d0 - d1 : d0;
        o[nxi * nxi + e] = d0 + (n - 1) * d1;
    }
    for (int e = threadIdx.x; e < nxi * nbc; e += blockDim.x) {
        const int u = e / nbc, s = e % nbc;
        const double d0 = B[(int64_t)u * m + s];
        const double d1 = n > 1 ? B[(int64_t)u * m + nbc + s] : 0.0;
        o[2 * nxi * nxi + e] = n > 1 ? d0 - d1 : d0;
        o[2 * nxi * nxi + nbc * nxi + e] = d0 + (n - 1) * d1;
    }
}

// The Kronecker blocks directly, without the dense factorisation (handles that project in
// the structured form): kron_kkt_blocks per shape, one CTA each; info = 0 or pivot + 1.
__global__ void k_kron_blocks(const Shape *sh, int nxi, double rho, const double *W, double *Sx, int *info)
{
    __shared__ KronSmem sm;
    const Shape S = sh[blockIdx.x];
    const int bad = kron_kkt_blocks(S, nxi, rho, W + S.off_W, Sx + S.off_S + kron_cost_off(nxi, S.nbc), Sx + S.off_S, sm);
    if (threadIdx.x == 0 && bad) info[blockIdx.x] = bad;
}

// Dense P_eta = (I - Q) (x) P_dev + Q (x) P_mean and P_b likewise (columns robot-major
// (start, goal[, velocity])), from the blocks: for the operator queries and the adjoint's
// P_b term.
__global__ void k_kron_assemble(const Shape *sh, int nxi, const double *Sx, double *P, double *Pb)
{
    const Shape S = sh[blockIdx.y];
    const int N = S.N, n = S.n, nbc = S.nbc, m2 = nbc * n;
    const double *Pd = Sx + S.off_S, *Pm = Pd + nxi * nxi, *Bd = Pd + 2 * nxi * nxi, *Bm = Bd + nbc * nxi;
    const double inv_n = 1.0 / (double)n;
    const int64_t totP = (int64_t)N * N, totB = (int64_t)N * m2;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < totP + totB; e += (int64_t)gridDim.x * blockDim.x) {
        if (e < totP) {
            const int r = (int)(e / N), c = (int)(e % N), i = r / nxi, u = r % nxi, j = c / nxi, v = c % nxi;
            const double dv = Pd[u * nxi + v];
            P[S.off_P + e] = (i == j ? dv : 0.0) + (Pm[u * nxi + v] - dv) * inv_n;
        } else {
            const int64_t f = e - totP;
            const int r = (int)(f / m2), q = (int)(f % m2), i = r / nxi, u = r % nxi, j = q / nbc, sd = q % nbc;
            const double dv = Bd[u * nbc + sd];
            Pb[S.off_Pb + f] = (i == j ? dv : 0.0) + (Bm[u * nbc + sd] - dv) * inv_n;
        }
    }
}

__global__ void k_convert(const double *src, float *dst, int64_t n)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = (float)src[e];
}

cudaError_t convert_pool(const double *src, float *dst, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int grid = (int)((n + 255) / 256);
    if (grid > 4096) grid = 4096;
    k_convert<<<grid, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

int64_t tc_pool_bytes(int mode, int N, int C)
{
    if (!mode) return 0;
    return (int64_t)C * tc_ntiles(N, C) * tc_nk(mode, N) * tc_na(mode) * kTcChunkBytes;
}

// One element of the tensor-core chunk layout per thread: CTA rank cr takes rows
// [cr L, cr L + L) of P_eta (L = ceil(N / C)) in 128-row tiles; each tile is split into
// K chunks of 128 bytes per row, stored as core matrices [16 row groups][8 K groups][8][16 B].
__global__ void k_arrange_tc(const Shape *sh, const double *P64, const int64_t *tc_off, int mode, int C,
                             unsigned char *out)
{
    const Shape S = sh[blockIdx.y];
    const int N = S.N, L = (N + C - 1) / C, nT = tc_ntiles(N, C), nK = tc_nk(mode, N), na = tc_na(mode);
    const int es = tc_es(mode), KC = tc_kc(mode);
    const int64_t tot = (int64_t)C * nT * nK * 128 * KC;
    unsigned char *base = out + tc_off[blockIdx.y];
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t rest = idx;
        const int kk = (int)(rest % KC); rest /= KC;
        const int i = (int)(rest % 128); rest /= 128;
        const int kc = (int)(rest % nK); rest /= nK;
        const int t = (int)(rest % nT);
        const int cr = (int)(rest / nT);
        const int r = cr * L + 128 * t + i, c = kc * KC + kk, rhi = min(N, (cr + 1) * L);
        const double val = (r < rhi && c < N) ? P64[S.off_P + (int64_t)r * N + c] : 0.0;
        unsigned char *blk = base + ((((int64_t)cr * nT + t) * nK + kc) * na) * kTcChunkBytes;
        const int within = ((i >> 3) * 8 + ((kk * es) >> 4)) * 128 + (i & 7) * 16 + ((kk * es) & 15);
        if (mode == 1) {
            *reinterpret_cast<float *>(blk + within) = tc::to_tf32((float)val);
        } else {
            const __nv_bfloat16 hi = __float2bfloat16_rn((float)val);
            *reinterpret_cast<__nv_bfloat16 *>(blk + within) = hi;
            if (na == 2)
                *reinterpret_cast<__nv_bfloat16 *>(blk + kTcChunkBytes + within) =
                    __float2bfloat16_rn((float)(val - (double)__bfloat162float(hi)));
        }
    }
}

cudaError_t arrange_tc(const Shape *shapes_dev, int n_shapes, const Shape *shapes_host, const double *P64,
                       const int64_t *tc_off_dev, const int64_t *tc_off_host, int mode, int C, unsigned char *out,
                       cudaStream_t s)
{
    (void)tc_off_host;
    if (!mode || n_shapes < 1) return cudaSuccess;
    int64_t most = 0;
    for (int i = 0; i < n_shapes; ++i) {
        const int N = shapes_host[i].N;
        most = std::max<int64_t>(most, (int64_t)C * tc_ntiles(N, C) * tc_nk(mode, N) * 128 * tc_kc(mode));
    }
    const int64_t blocks = std::min<int64_t>(4096, (most + 255) / 256);
    k_arrange_tc<<<dim3((unsigned)blocks, n_shapes), 256, 0, s>>>(shapes_dev, P64, tc_off_dev, mode, C, out);
    return cudaGetLastError();
}

cudaError_t factor_shapes(const Shape *shapes_dev, int n_shapes, const Shape *shapes_host, int nxi,
                          double rho, int cost, double dt, double *W64, double *P64, double *Pb64, double *S64,
                          double *scratch, int64_t scratch_elems, int *info, cudaStream_t s, bool dense)
{
    if (!dense) {   // structured handles: the Kronecker blocks directly, dense forms assembled
        int maxN = 0;
        int64_t most = 0;
        for (int i = 0; i < n_shapes; ++i) {
            maxN = std::max(maxN, shapes_host[i].N);
            most = std::max<int64_t>(most, (int64_t)shapes_host[i].N * (shapes_host[i].N + shapes_host[i].nbc * shapes_host[i].n));
        }
        k_basis<<<n_shapes, 256, 0, s>>>(shapes_dev, nxi, W64);
        k_cost_block<<<n_shapes, 128, 0, s>>>(shapes_dev, nxi, cost, dt, S64);
        k_kron_blocks<<<n_shapes, 128, 0, s>>>(shapes_dev, nxi, rho, W64, S64, info);
        const int64_t blocks = (most + 255) / 256;
        k_kron_assemble<<<dim3((unsigned)(blocks > 1024 ? 1024 : blocks), n_shapes), 256, 0, s>>>(shapes_dev, nxi, S64,
                                                                                               P64, Pb64);
        (void)maxN;
        return cudaGetLastError();
    }
    // scratch holds three pools laid out like P64: L (Cholesky), Y, S
    (void)scratch_elems;
    int maxN = 0;
    int64_t poolP = 0;
    for (int i = 0; i < n_shapes; ++i) {
        if (shapes_host[i].N > maxN) maxN = shapes_host[i].N;
        int64_t end = shapes_host[i].off_P + (int64_t)shapes_host[i].N * shapes_host[i].N;
        if (end > poolP) poolP = end;
    }
    double *Lp = scratch, *Yp = scratch + poolP, *Sp = scratch + 2 * poolP;
    k_basis<<<n_shapes, 256, 0, s>>>(shapes_dev, nxi, W64);
    k_cost_block<<<n_shapes, 128, 0, s>>>(shapes_dev, nxi, cost, dt, S64);
    const int64_t hblocks = ((int64_t)maxN * maxN + 255) / 256;
    dim3 gH((unsigned)(hblocks > 1024 ? 1024 : hblocks), n_shapes);
    k_build_H<<<gH, 256, 0, s>>>(shapes_dev, nxi, rho, W64, S64, Lp);
    k_cholesky<<<n_shapes, 1024, 0, s>>>(shapes_dev, Lp, info);
    dim3 gI((maxN + 31) / 32, n_shapes);
    k_chol_inverse<<<gI, 32, 0, s>>>(shapes_dev, Lp, P64);
    k_schur<<<n_shapes, 256, 0, s>>>(shapes_dev, nxi, W64, P64, Yp, Sp, Pb64, info);
    k_peta<<<gH, 256, 0, s>>>(shapes_dev, Yp, Pb64, P64);
    k_structured<<<n_shapes, 128, 0, s>>>(shapes_dev, nxi, P64, Pb64, S64);
    return cudaGetLastError();
}

}  // namespace sf
