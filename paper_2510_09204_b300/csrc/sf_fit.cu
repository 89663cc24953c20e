// sf_fit_positions: least-squares Bernstein coefficients of sampled trajectories with the
// end coefficients pinned to the first and last sample (eq. poly: p = W xi; the boundary
// rows A xi = b fix coefficients 0 and n_xi - 1, which the Bernstein basis interpolates).
// A helper for building candidates from sampled positions, not part of the solve.
//
// For a row p[0..H) (one robot, one axis): xi_0 = p_0, xi_{m+1} = p_{H-1} (m = n_xi - 2)
// and the interior xi_1..m minimises ||W_int xi_int - (p - w_0 p_0 - w_last p_{H-1})||^2,
// so xi_int = F r with F = (W_int' W_int)^-1 W_int' (m x H), formed once per distinct H
// in FP64 by Gauss-Jordan elimination of the m x m normal matrix.
#include <algorithm>
#include <map>
#include <vector>

#include "sf_internal.cuh"

namespace sf {

constexpr int kFitMaxXi = 32;

// One CTA per distinct horizon: W (H x nxi), then F (m x H) into Fop + off.
__global__ void k_fit_operator(const int *Hs, const int64_t *offs, int nxi, double *Fop, double *Wop,
                               const int64_t *woffs, int *info)
{
    const int H = Hs[blockIdx.x], m = nxi - 2, deg = nxi - 1;
    double *F = Fop + offs[blockIdx.x];
    double *W = Wop + woffs[blockIdx.x];
    __shared__ double Nm[kFitMaxXi][2 * kFitMaxXi];   // [normal matrix | identity]
    __shared__ int bad;
    for (int e = threadIdx.x; e < H * nxi; e += blockDim.x) {
        const int k = e / nxi, c = e - k * nxi;
        const double tau = (double)k / (double)(H - 1);
        double bin = 1.0;
        for (int q = 1; q <= c; ++q) bin = bin * (double)(deg - c + q) / (double)q;
        W[e] = bin * pow(tau, (double)c) * pow(1.0 - tau, (double)(deg - c));
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int u = e / m, v = e - u * m;
        double s = 0.0;
        for (int k = 0; k < H; ++k) s += W[k * nxi + 1 + u] * W[k * nxi + 1 + v];
        Nm[u][v] = s;
        Nm[u][m + v] = u == v ? 1.0 : 0.0;
    }
    __syncthreads();
    // Gauss-Jordan with partial pivoting (the normal matrix is SPD for H >= n_xi)
    for (int col = 0; col < m; ++col) {
        if (threadIdx.x == 0) {
            int piv = col;
            for (int r = col + 1; r < m; ++r)
                if (fabs(Nm[r][col]) > fabs(Nm[piv][col])) piv = r;
            if (!(fabs(Nm[piv][col]) > 1e-300)) bad = 1;
            if (piv != col)
                for (int q = 0; q < 2 * m; ++q) {
                    const double t = Nm[col][q];
                    Nm[col][q] = Nm[piv][q];
                    Nm[piv][q] = t;
                }
        }
        __syncthreads();
        if (bad) break;
        const double d = Nm[col][col];
        __syncthreads();
        for (int q = threadIdx.x; q < 2 * m; q += blockDim.x) Nm[col][q] /= d;
        __syncthreads();
        // eliminate the column from the other rows; the column itself is read by every
        // update, so it is cleared only after a barrier
        for (int e = threadIdx.x; e < m * 2 * m; e += blockDim.x) {
            const int r = e / (2 * m), q = e - r * 2 * m;
            if (r != col && q != col) Nm[r][q] -= Nm[r][col] * Nm[col][q];
        }
        __syncthreads();
        for (int r = threadIdx.x; r < m; r += blockDim.x)
            if (r != col) Nm[r][col] = 0.0;
        __syncthreads();
    }
    if (bad) {
        if (threadIdx.x == 0) info[blockIdx.x] = 1;
        return;
    }
    // F = N^-1 W_int'
    for (int e = threadIdx.x; e < m * H; e += blockDim.x) {
        const int u = e / H, k = e - u * H;
        double s = 0.0;
        for (int v = 0; v < m; ++v) s += Nm[u][m + v] * W[k * nxi + 1 + v];
        F[e] = s;
    }
}

// One warp per (instance, axis, robot) row.
__global__ void k_fit_apply(int rows_total, const int64_t *row_inst, const int *inst_H, const int *inst_op,
                            const int64_t *pos_off, const int64_t *xi_off, const int64_t *row_first, int nxi,
                            const double *Fop, const int64_t *offs, const double *Wop, const int64_t *woffs,
                            const double *pos, double *xi)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= rows_total) return;
    const int k = (int)row_inst[row];
    const int H = inst_H[k], op = inst_op[k], m = nxi - 2;
    const int64_t r = row - row_first[k];
    const double *p = pos + pos_off[k] + r * H;
    const double *F = Fop + offs[op];
    const double *W = Wop + woffs[op];
    const double p0 = p[0], p1 = p[H - 1];
    double acc[kFitMaxXi - 2];
#pragma unroll
    for (int u = 0; u < kFitMaxXi - 2; ++u) acc[u] = 0.0;
    for (int t = lane; t < H; t += 32) {
        const double rr = p[t] - W[t * nxi] * p0 - W[t * nxi + nxi - 1] * p1;
#pragma unroll
        for (int u = 0; u < kFitMaxXi - 2; ++u)
            if (u < m) acc[u] += F[(int64_t)u * H + t] * rr;
    }
#pragma unroll
    for (int u = 0; u < kFitMaxXi - 2; ++u) {
        if (u >= m) break;
        double s = acc[u];
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        acc[u] = s;
    }
    if (lane == 0) {
        double *x = xi + xi_off[k] + r * nxi;
        x[0] = p0;
        for (int u = 0; u < m; ++u) x[1 + u] = acc[u];
        x[nxi - 1] = p1;
    }
}

}  // namespace sf

using namespace sf;

extern "C" int sf_fit_positions(int32_t n_d, int32_t n_xi, int32_t n_inst, const int32_t *n, const int32_t *H,
                                const double *pos, double *xi_out, void *stream)
{
    if (n_d < 2 || n_d > 3 || n_xi < 3 || n_xi > kFitMaxXi || n_inst < 1 || !n || !H || !pos || !xi_out)
        return SF_EINVAL;
    for (int k = 0; k < n_inst; ++k)
        if (n[k] < 1 || H[k] < n_xi || H[k] > 1 << 20) return SF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    // distinct horizons, instance offsets, row table
    std::map<int, int> hidx;
    std::vector<int> hs, inst_H(n_inst), inst_op(n_inst);
    std::vector<int64_t> offs, woffs, pos_off(n_inst), xi_off(n_inst), row_first(n_inst), row_inst;
    int64_t fo = 0, wo = 0, po = 0, xo = 0;
    for (int k = 0; k < n_inst; ++k) {
        auto it = hidx.find(H[k]);
        if (it == hidx.end()) {
            it = hidx.emplace(H[k], (int)hs.size()).first;
            hs.push_back(H[k]);
            offs.push_back(fo);
            woffs.push_back(wo);
            fo += (int64_t)(n_xi - 2) * H[k];
            wo += (int64_t)H[k] * n_xi;
        }
        inst_H[k] = H[k];
        inst_op[k] = it->second;
        pos_off[k] = po;
        xi_off[k] = xo;
        row_first[k] = (int64_t)row_inst.size();
        for (int r = 0; r < n_d * n[k]; ++r) row_inst.push_back(k);
        po += (int64_t)n_d * n[k] * H[k];
        xo += (int64_t)n_d * n[k] * n_xi;
    }
    const int nh = (int)hs.size();
    const int64_t rows = (int64_t)row_inst.size();
    // one stream-ordered scratch block: operators, basis, tables
    const size_t b_F = sizeof(double) * std::max<int64_t>(fo, 1), b_W = sizeof(double) * wo;
    const size_t b_i64 = sizeof(int64_t) * (2 * nh + 3 * n_inst + rows), b_i32 = sizeof(int) * (nh + 2 * n_inst + nh);
    unsigned char *scr = nullptr;
    if (cudaMallocAsync((void **)&scr, b_F + b_W + b_i64 + b_i32 + 64, st) != cudaSuccess) return SF_ENOMEM;
    double *Fop = (double *)scr, *Wop = (double *)(scr + b_F);
    int64_t *d64 = (int64_t *)(scr + b_F + b_W);
    int64_t *d_offs = d64, *d_woffs = d64 + nh, *d_pos_off = d64 + 2 * nh, *d_xi_off = d_pos_off + n_inst,
            *d_row_first = d_xi_off + n_inst, *d_row_inst = d_row_first + n_inst;
    int *d32 = (int *)(scr + b_F + b_W + b_i64);
    int *d_hs = d32, *d_inst_H = d32 + nh, *d_inst_op = d_inst_H + n_inst, *d_info = d_inst_op + n_inst;
    std::vector<int64_t> h64(2 * nh + 3 * n_inst + rows);
    std::copy(offs.begin(), offs.end(), h64.begin());
    std::copy(woffs.begin(), woffs.end(), h64.begin() + nh);
    std::copy(pos_off.begin(), pos_off.end(), h64.begin() + 2 * nh);
    std::copy(xi_off.begin(), xi_off.end(), h64.begin() + 2 * nh + n_inst);
    std::copy(row_first.begin(), row_first.end(), h64.begin() + 2 * nh + 2 * n_inst);
    std::copy(row_inst.begin(), row_inst.end(), h64.begin() + 2 * nh + 3 * n_inst);
    std::vector<int> h32(nh + 2 * n_inst + nh, 0);
    std::copy(hs.begin(), hs.end(), h32.begin());
    std::copy(inst_H.begin(), inst_H.end(), h32.begin() + nh);
    std::copy(inst_op.begin(), inst_op.end(), h32.begin() + nh + n_inst);
    int rc = SF_OK;
    std::vector<int> info(nh, 0);
    // pageable sources: each copy has read its host buffer when the call returns
    if (cudaMemcpyAsync(d64, h64.data(), b_i64, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d32, h32.data(), b_i32, cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = SF_ECUDA;
    if (rc == SF_OK) {
        k_fit_operator<<<nh, 256, 0, st>>>(d_hs, d_offs, n_xi, Fop, Wop, d_woffs, d_info);
        const int wpb = 8;
        k_fit_apply<<<(unsigned)((rows + wpb - 1) / wpb), 32 * wpb, 0, st>>>(
            (int)rows, d_row_inst, d_inst_H, d_inst_op, d_pos_off, d_xi_off, d_row_first, n_xi, Fop, d_offs, Wop,
            d_woffs, pos, xi_out);
        if (cudaGetLastError() != cudaSuccess) rc = SF_ECUDA;
    }
    if (rc == SF_OK && cudaMemcpyAsync(info.data(), d_info, sizeof(int) * nh, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = SF_ECUDA;
    cudaFreeAsync(scr, st);
    if (rc == SF_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = SF_ECUDA;
    if (rc == SF_OK)
        for (int v : info)
            if (v) rc = SF_EINVAL;
    return rc;
}
