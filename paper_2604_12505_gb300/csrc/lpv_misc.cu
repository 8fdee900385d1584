// lpv_misc.cu -- LPV kernels off the tensor cores: gradient reduction, Adam,
// data statistics, and the FP64 least-squares initialisation.
#include <cuda_runtime.h>

#include "lpv_common.cuh"
#include "lpv_launch.h"

namespace lpv {

// One thread per padded weight: sum of the warp partials in fixed order (FP64).
__global__ void reduce_kernel(const float* __restrict__ gpart, int n_warps, const double* __restrict__ loss_part,
                              const float* __restrict__ Wp, Dims d, double sigma2, double n_samples,
                              float* __restrict__ grad, double* __restrict__ loss, double* __restrict__ loss_hist,
                              int it)
{
    __shared__ double red[kWN / 32];
    const int idx = threadIdx.x;
    const int o = idx / (kFB * kMaxKT), col = idx % (kFB * kMaxKT);
    double gsum = 0.0;
    for (int w = 0; w < n_warps; ++w) gsum += (double)gpart[(size_t)w * kWN + idx];
    const double wv = (double)Wp[idx];
    const bool tr = trainable(d, o, col);
    grad[idx] = tr ? (float)(gsum + sigma2 * wv) : 0.f;
    double sq = tr ? wv * wv : 0.0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, s);
    if ((idx & 31) == 0) red[idx >> 5] = sq;
    __syncthreads();
    if (idx == 0) {
        double w2 = 0.0, ls = 0.0;
        for (int j = 0; j < kWN / 32; ++j) w2 += red[j];
        for (int w = 0; w < n_warps; ++w) ls += loss_part[w];
        const double L = ls / n_samples + 0.5 * sigma2 * w2;
        if (loss) *loss = L;
        if (loss_hist) loss_hist[it] = L;
    }
}

// Adam (Kingma and Ba) on the trainable weights; c1 = 1/(1-b1^t), c2 = 1/(1-b2^t).
__global__ void adam_kernel(float* __restrict__ Wp, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ grad, Dims d, float lr, float b1, float b2, float eps, float c1,
                            float c2)
{
    const int idx = threadIdx.x;
    const int o = idx / (kFB * kMaxKT), col = idx % (kFB * kMaxKT);
    if (!trainable(d, o, col)) {
        Wp[idx] = 0.f;
        return;
    }
    const float gv = grad[idx];
    const float mm = b1 * m[idx] + (1.f - b1) * gv;
    const float vv = b2 * v[idx] + (1.f - b2) * gv * gv;
    m[idx] = mm;
    v[idx] = vv;
    Wp[idx] -= lr * (mm * c1) / (sqrtf(vv * c2) + eps);
}

// Channel sums over n rows (FP64); block partials, then a fixed-order sum.
__global__ void stats_kernel(const float* __restrict__ u, const float* __restrict__ y, const float* __restrict__ p,
                             long long n, int nu, int ny, int np, double* __restrict__ part)
{
    const int nch = nu + ny + 2 * np;
    double acc[32];
    for (int c = 0; c < nch; ++c) acc[c] = 0.0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        for (int c = 0; c < nu; ++c) {
            const double x = u[r * nu + c];
            acc[c] += x * x;
        }
        for (int c = 0; c < ny; ++c) {
            const double x = y[r * ny + c];
            acc[nu + c] += x * x;
        }
        for (int c = 0; c < np; ++c) {
            const double x = p[r * np + c];
            acc[nu + ny + c] += x;
            acc[nu + ny + np + c] += x * x;
        }
    }
    __shared__ double sh[32][33];
    for (int c = 0; c < nch; ++c) {
        double v = acc[c];
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) v += __shfl_down_sync(0xffffffffu, v, s);
        if ((threadIdx.x & 31) == 0) sh[c][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < nch) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[threadIdx.x][w];
        part[blockIdx.x * 32 + threadIdx.x] = v;
    }
}

__global__ void stats_final_kernel(const double* __restrict__ part, int n_blocks, int nch, double* __restrict__ stats)
{
    const int c = threadIdx.x;
    if (c >= nch) return;
    double v = 0.0;
    for (int b = 0; b < n_blocks; ++b) v += part[b * 32 + c];
    stats[c] = v;
}

// ---------------------------------------------------------------------------
// FP64 least squares of the MIMO ARX model on normalised data
// ---------------------------------------------------------------------------
constexpr int kGramBlocks = 152;
constexpr int kGramRows = 32;   // rows staged per pass

// Extended row e = [y_{k-1}..y_{k-na}, u_{k-1}..u_{k-na}, y_k] (n_ext entries).
__device__ __forceinline__ double ext_entry(const float* __restrict__ u, const float* __restrict__ y, const Dims& d,
                                            int na, long long base, int k, int T, int j)
{
    const int nreg_y = na * d.ny, nreg = na * (d.ny + d.nu);
    if (j < nreg_y) {
        const int lag = 1 + j / d.ny, c = j % d.ny;
        return (double)y[(base + k - lag) * d.ny + c] * (double)d.inv_sy[c];
    }
    if (j < nreg) {
        const int jj = j - nreg_y, lag = 1 + jj / d.nu, c = jj % d.nu;
        return (double)u[(base + k - lag) * d.nu + c] * (double)d.inv_su[c];
    }
    const int c = j - nreg;
    return (double)y[(base + k) * d.ny + c] * (double)d.inv_sy[c];
}

// One thread per entry (i, j) of the n_ext x n_ext Gram matrix.
__global__ void __launch_bounds__(1024) gram_kernel(const float* __restrict__ u, const float* __restrict__ y,
                                                    int n_traj, int T, Dims d, int na, double* __restrict__ part)
{
    __shared__ double rows[kGramRows][33];
    const int n_ext = na * (d.ny + d.nu) + d.ny;
    const int i = threadIdx.x / n_ext, j = threadIdx.x % n_ext;
    const bool own = threadIdx.x < n_ext * n_ext;
    const long long per = (long long)(T - na);
    const long long n_rows = per * n_traj;
    double acc = 0.0;
    for (long long r0 = (long long)blockIdx.x * kGramRows; r0 < n_rows; r0 += (long long)gridDim.x * kGramRows) {
        __syncthreads();
        for (int q = threadIdx.x; q < kGramRows * n_ext; q += blockDim.x) {
            const int rl = q / n_ext, jj = q % n_ext;
            const long long r = r0 + rl;
            double v = 0.0;
            if (r < n_rows) {
                const long long b = r / per;
                const int k = (int)(r % per) + na;
                v = ext_entry(u, y, d, na, b * T, k, T, jj);
            }
            rows[rl][jj] = v;
        }
        __syncthreads();
        if (own)
            for (int rl = 0; rl < kGramRows; ++rl) acc += rows[rl][i] * rows[rl][j];
    }
    if (own) part[(size_t)blockIdx.x * 1024 + threadIdx.x] = acc;
}

// Fixed-order sum of the block partials, Cholesky solve of the normal
// equations (FP64, one thread), observer-canonical M_0 into Wp.
__global__ void ls_solve_kernel(const double* __restrict__ part, int n_blocks, Dims d, int na,
                                double* __restrict__ theta, float* __restrict__ Wp, int* __restrict__ status)
{
    __shared__ double E[32][33];
    const int n_ext = na * (d.ny + d.nu) + d.ny, nreg = na * (d.ny + d.nu);
    const int idx = threadIdx.x;
    if (idx < n_ext * n_ext) {
        double s = 0.0;
        for (int b = 0; b < n_blocks; ++b) s += part[(size_t)b * 1024 + idx];
        E[idx / n_ext][idx % n_ext] = s;
    }
    for (int q = idx; q < kWN; q += blockDim.x) Wp[q] = 0.f;
    __syncthreads();
    if (idx != 0) return;
    // Cholesky G = L L^T in place (lower triangle of E[0..nreg)[0..nreg))
    for (int c = 0; c < nreg; ++c) {
        double s = E[c][c];
        for (int k = 0; k < c; ++k) s -= E[c][k] * E[c][k];
        if (!(s > 0.0)) {
            *status = 1;
            return;
        }
        const double lc = sqrt(s);
        E[c][c] = lc;
        for (int r = c + 1; r < nreg; ++r) {
            double t = E[r][c];
            for (int k = 0; k < c; ++k) t -= E[r][k] * E[c][k];
            E[r][c] = t / lc;
        }
    }
    // solve L L^T theta = Phi^T Y for each output (column nreg + q of E)
    for (int q = 0; q < d.ny; ++q) {
        double z[32];
        for (int r = 0; r < nreg; ++r) {
            double t = E[r][nreg + q];
            for (int k = 0; k < r; ++k) t -= E[r][k] * z[k];
            z[r] = t / E[r][r];
        }
        for (int r = nreg - 1; r >= 0; --r) {
            double t = z[r];
            for (int k = r + 1; k < nreg; ++k) t -= E[k][r] * z[k];
            z[r] = t / E[r][r];
        }
        for (int r = 0; r < nreg; ++r) theta[r * d.ny + q] = z[r];
    }
    // observer-canonical form: x^j_{k+1} = A_j y_k + x^{j+1}_k + B_j u_k, y_k = x^1_k
    constexpr int ld = kFB * kMaxKT;
    for (int j = 0; j < na; ++j)
        for (int q = 0; q < d.ny; ++q) {
            const int o = j * d.ny + q;
            for (int c = 0; c < d.ny; ++c) Wp[o * ld + c] = (float)theta[(j * d.ny + c) * d.ny + q];
            if (j + 1 < na) Wp[o * ld + (j + 1) * d.ny + q] = 1.f;
            for (int c = 0; c < d.nu; ++c) Wp[o * ld + d.nx + c] = (float)theta[(na * d.ny + j * d.nu + c) * d.ny + q];
        }
    for (int q = 0; q < d.ny; ++q) Wp[(d.nx + q) * ld + q] = 1.f;
    *status = 0;
}

// ---------------------------------------------------------------------------
cudaError_t launch_reduce(const float* gpart, int n_warps, const double* loss_part, const float* Wp, const Dims& d,
                          double sigma2, double n_samples, float* grad, double* loss, double* loss_hist, int it,
                          cudaStream_t st)
{
    reduce_kernel<<<1, kWN, 0, st>>>(gpart, n_warps, loss_part, Wp, d, sigma2, n_samples, grad, loss, loss_hist, it);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* Wp, float* m, float* v, const float* grad, const Dims& d, float lr, float b1, float b2,
                        float eps, float c1, float c2, cudaStream_t st)
{
    adam_kernel<<<1, kWN, 0, st>>>(Wp, m, v, grad, d, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_stats(const float* u, const float* y, const float* p, long long n, int nu, int ny, int np,
                         double* part, double* stats, cudaStream_t st)
{
    stats_kernel<<<256, 256, 0, st>>>(u, y, p, n, nu, ny, np, part);
    stats_final_kernel<<<1, 32, 0, st>>>(part, 256, nu + ny + 2 * np, stats);
    return cudaGetLastError();
}

int gram_blocks() { return kGramBlocks; }

cudaError_t launch_gram(const float* u, const float* y, int n_traj, int T, const Dims& d, int na, double* part,
                        cudaStream_t st)
{
    gram_kernel<<<kGramBlocks, 1024, 0, st>>>(u, y, n_traj, T, d, na, part);
    return cudaGetLastError();
}

cudaError_t launch_ls_solve(const double* part, const Dims& d, int na, double* theta, float* Wp, int* status,
                            cudaStream_t st)
{
    ls_solve_kernel<<<1, 1024, 0, st>>>(part, kGramBlocks, d, na, theta, Wp, status);
    return cudaGetLastError();
}

}  // namespace lpv
