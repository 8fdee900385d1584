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

constexpr double kRejectFactor = 10.0;

// Adam (Kingma and Ba) on the trainable weights; c1 = 1/(1-b1^t), c2 = 1/(1-b2^t),
// step lr * lr_scale.  Wb, mb, vb hold the last accepted iterate and its
// updated moments, acc_loss its loss.  The current iterate is accepted when its
// loss is at most kRejectFactor times acc_loss (so never when it is not
// finite); otherwise the step is rejected: the weights go back to Wb and the
// same Adam direction is retried with half the step (lr_scale halves and
// stays halved).
__global__ void adam_kernel(float* __restrict__ Wp, float* __restrict__ m, float* __restrict__ v,
                            float* __restrict__ Wb, float* __restrict__ mb, float* __restrict__ vb,
                            float* __restrict__ lr_scale, double* __restrict__ acc_loss,
                            const float* __restrict__ grad, const double* __restrict__ loss, Dims d, float lr,
                            float b1, float b2, float eps, float c1, float c2)
{
    const int idx = threadIdx.x;
    const double L = *loss;
    const bool good = L <= kRejectFactor * *acc_loss;
    float sc = *lr_scale;
    __syncthreads();
    if (!good) {
        sc *= 0.5f;
        if (idx == 0) *lr_scale = sc;
    } else if (idx == 0) {
        *acc_loss = L;
    }
    const int o = idx / (kFB * kMaxKT), col = idx % (kFB * kMaxKT);
    if (!trainable(d, o, col)) {
        Wp[idx] = 0.f;
        return;
    }
    float mm, vv, w;
    if (good) {
        const float gv = grad[idx];
        mm = b1 * m[idx] + (1.f - b1) * gv;
        vv = b2 * v[idx] + (1.f - b2) * gv * gv;
        w = Wp[idx];
        Wb[idx] = w;
        mb[idx] = mm;
        vb[idx] = vv;
    } else {
        mm = mb[idx];
        vv = vb[idx];
        w = Wb[idx];
    }
    m[idx] = mm;
    v[idx] = vv;
    Wp[idx] = w - lr * sc * (mm * c1) / (sqrtf(vv * c2) + eps);
}

// Channel sums over n rows (FP64) and the range of each scheduling channel;
// block partials (stride kStatStride: sums at 0.., min at 32.., max at 32 + np..),
// then a fixed-order combination.
constexpr int kStatStride = 64;

__global__ void stats_kernel(const float* __restrict__ u, const float* __restrict__ y, const float* __restrict__ p,
                             long long n, int nu, int ny, int np, double* __restrict__ part)
{
    const int nch = nu + ny + 2 * np;
    double acc[32];
    float lo[2] = {INFINITY, INFINITY}, hi[2] = {-INFINITY, -INFINITY};
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
            const float xf = p[r * np + c];
            const double x = xf;
            acc[nu + ny + c] += x;
            acc[nu + ny + np + c] += x * x;
            lo[c] = fminf(lo[c], xf);
            hi[c] = fmaxf(hi[c], xf);
        }
    }
    __shared__ double sh[36][33];
    for (int c = 0; c < nch; ++c) {
        double v = acc[c];
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) v += __shfl_down_sync(0xffffffffu, v, s);
        if ((threadIdx.x & 31) == 0) sh[c][threadIdx.x >> 5] = v;
    }
    for (int c = 0; c < np; ++c) {
        float a = lo[c], b = hi[c];
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            a = fminf(a, __shfl_down_sync(0xffffffffu, a, s));
            b = fmaxf(b, __shfl_down_sync(0xffffffffu, b, s));
        }
        if ((threadIdx.x & 31) == 0) {
            sh[32 + c][threadIdx.x >> 5] = a;
            sh[32 + np + c][threadIdx.x >> 5] = b;
        }
    }
    __syncthreads();
    const int nw = (int)(blockDim.x >> 5);
    if (threadIdx.x < nch) {
        double v = 0.0;
        for (int w = 0; w < nw; ++w) v += sh[threadIdx.x][w];
        part[blockIdx.x * kStatStride + threadIdx.x] = v;
    } else if (threadIdx.x >= 32 && threadIdx.x < 32 + 2 * np) {
        const bool is_lo = threadIdx.x < 32 + np;
        double v = sh[threadIdx.x][0];
        for (int w = 1; w < nw; ++w) v = is_lo ? fmin(v, sh[threadIdx.x][w]) : fmax(v, sh[threadIdx.x][w]);
        part[blockIdx.x * kStatStride + threadIdx.x] = v;
    }
}

__global__ void stats_final_kernel(const double* __restrict__ part, int n_blocks, int nch, int np,
                                   double* __restrict__ stats)
{
    const int c = threadIdx.x;
    if (c < nch) {
        double v = 0.0;
        for (int b = 0; b < n_blocks; ++b) v += part[b * kStatStride + c];
        stats[c] = v;
    } else if (c >= 32 && c < 32 + 2 * np) {
        const bool is_lo = c < 32 + np;
        double v = part[c];
        for (int b = 1; b < n_blocks; ++b)
            v = is_lo ? fmin(v, part[b * kStatStride + c]) : fmax(v, part[b * kStatStride + c]);
        stats[c] = v;
    }
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

// Cholesky G = L L^T of the leading nreg x nreg block of E (in place, lower
// triangle) and the solves L L^T theta = Phi^T Y for each output (column
// nreg + q of E).  One thread; returns false if G is not positive definite.
__device__ bool cholesky_solve(double (*E)[33], int nreg, int ny, double* th)
{
    for (int c = 0; c < nreg; ++c) {
        double s = E[c][c];
        for (int k = 0; k < c; ++k) s -= E[c][k] * E[c][k];
        if (!(s > 0.0)) return false;
        const double lc = sqrt(s);
        E[c][c] = lc;
        for (int r = c + 1; r < nreg; ++r) {
            double t = E[r][c];
            for (int k = 0; k < c; ++k) t -= E[r][k] * E[c][k];
            E[r][c] = t / lc;
        }
    }
    for (int q = 0; q < ny; ++q) {
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
        for (int r = 0; r < nreg; ++r) th[r * ny + q] = z[r];
    }
    return true;
}

typedef double Mat16[16][17];

// C (m x n) = op(A) (m x kk) op(B) (kk x n) in shared memory; C may alias A or
// B (every product is read before any is written).  All threads call it.
__device__ void bmm(Mat16& C, const Mat16& A, bool ta, const Mat16& B, bool tb, int m, int n, int kk)
{
    const int idx = threadIdx.x;
    double t = 0.0;
    if (idx < m * n) {
        const int r = idx / n, c = idx % n;
        for (int k = 0; k < kk; ++k) t += (ta ? A[k][r] : A[r][k]) * (tb ? B[c][k] : B[k][c]);
    }
    __syncthreads();
    if (idx < m * n) C[idx / n][idx % n] = t;
    __syncthreads();
}

// In-place lower Cholesky factor of (X + reg * trace(X) * I), upper part zeroed.
// One thread; false if the matrix is not positive definite.
__device__ bool chol_reg(Mat16& X, int n, double reg)
{
    double tr = 0.0;
    for (int i = 0; i < n; ++i) tr += X[i][i];
    for (int i = 0; i < n; ++i) X[i][i] += reg * tr;
    for (int c = 0; c < n; ++c) {
        double s = X[c][c];
        for (int k = 0; k < c; ++k) s -= X[c][k] * X[c][k];
        if (!(s > 0.0)) return false;
        const double lc = sqrt(s);
        X[c][c] = lc;
        for (int r = c + 1; r < n; ++r) {
            double t = X[r][c];
            for (int k = 0; k < c; ++k) t -= X[r][k] * X[c][k];
            X[r][c] = t / lc;
        }
        for (int r = 0; r < c; ++r) X[r][c] = 0.0;
    }
    return true;
}

// One-sided Jacobi SVD (Hestenes): G (n x n) is replaced by U, V receives V and
// sv the singular values of G = U diag(sv) V^T, in decreasing order.  One thread.
__device__ void jacobi_svd(Mat16& G, Mat16& V, double* sv, int n)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p + 1 < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = 0; i < n; ++i) {
                    al += G[i][p] * G[i][p];
                    be += G[i][q] * G[i][q];
                    ga += G[i][p] * G[i][q];
                }
                if (!(fabs(ga) > 1e-15 * sqrt(al * be))) continue;
                off = fmax(off, fabs(ga) / sqrt(al * be));
                const double ze = (be - al) / (2.0 * ga);
                const double t = copysign(1.0, ze) / (fabs(ze) + sqrt(1.0 + ze * ze));
                const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int i = 0; i < n; ++i) {
                    const double gp = G[i][p], gq = G[i][q];
                    G[i][p] = c * gp - s * gq;
                    G[i][q] = s * gp + c * gq;
                    const double vp = V[i][p], vq = V[i][q];
                    V[i][p] = c * vp - s * vq;
                    V[i][q] = s * vp + c * vq;
                }
            }
        if (off < 1e-15) break;
    }
    for (int j = 0; j < n; ++j) {
        double t = 0.0;
        for (int i = 0; i < n; ++i) t += G[i][j] * G[i][j];
        sv[j] = sqrt(t);
    }
    for (int j = 0; j < n; ++j) {  // selection sort, decreasing
        int b = j;
        for (int k = j + 1; k < n; ++k)
            if (sv[k] > sv[b]) b = k;
        if (b != j) {
            const double t = sv[j];
            sv[j] = sv[b];
            sv[b] = t;
            for (int i = 0; i < n; ++i) {
                double u = G[i][j];
                G[i][j] = G[i][b];
                G[i][b] = u;
                u = V[i][j];
                V[i][j] = V[i][b];
                V[i][b] = u;
            }
        }
    }
    for (int j = 0; j < n; ++j) {
        const double inv = sv[j] > 0.0 ? 1.0 / sv[j] : 0.0;
        for (int i = 0; i < n; ++i) G[i][j] *= inv;
    }
}

constexpr int kSquarings = 40;
constexpr int kSmith = 30;        // Gramian series summed over 2^30 terms
constexpr double kGramReg = 1e-12;

// Least-squares start: sums the Gram partials, solves the normal equations
// (one thread), estimates the spectral radius of the observer-canonical state
// matrix by Gelfand's formula rho = lim ||A^(2^s)||^(1/2^s) with Frobenius-
// normalised squarings (nx^2 threads), scales its roots into |z| <= rho_max,
// and writes M_0 as the balanced realisation of that model: Gramians by Smith
// doubling P <- P + A^(2^j) P A^(2^j)^T, Cholesky factors, Jacobi SVD of
// Lq^T Lp (states by decreasing Hankel singular value, each column of C signed
// so that its largest-magnitude entry is positive).  Without a stable
// scaled model (rho_max outside (0, 1)) or with singular Gramians, M_0 stays
// in observer-canonical form.
__global__ void ls_solve_kernel(const double* __restrict__ part, int n_blocks, Dims d, int na, double rho_max,
                                double* __restrict__ theta, float* __restrict__ Wp, int* __restrict__ status,
                                double* __restrict__ rho_out)
{
    __shared__ double E[32][33];
    __shared__ double th[32 * 16];
    __shared__ double S[2][16][17];
    __shared__ double red[256];
    __shared__ double nrm_s;
    __shared__ int ok;
    __shared__ Mat16 Am, Bm, Cm, P, Q, G, Vm, Tm, Ti, Tmp;
    __shared__ double sv[16];
    const int n_ext = na * (d.ny + d.nu) + d.ny, nreg = na * (d.ny + d.nu);
    const int idx = threadIdx.x;
    if (idx < n_ext * n_ext) {
        double s = 0.0;
        for (int b = 0; b < n_blocks; ++b) s += part[(size_t)b * 1024 + idx];
        E[idx / n_ext][idx % n_ext] = s;
    }
    for (int q = idx; q < kWN; q += blockDim.x) Wp[q] = 0.f;
    __syncthreads();
    if (idx == 0) ok = cholesky_solve(E, nreg, d.ny, th) ? 1 : 0;
    __syncthreads();
    if (!ok) {
        if (idx == 0) *status = 1;
        return;
    }
    for (int q = idx; q < nreg * d.ny; q += blockDim.x) theta[q] = th[q];
    // state matrix: block row j holds A_{j+1} in block column 0 and I in block column j+1
    const int nx = na * d.ny, nn = nx * nx;
    const int r = idx / nx, c = idx % nx;
    if (idx < nn) {
        const int j = r / d.ny, q = r % d.ny;
        double v = 0.0;
        if (c < d.ny) v = th[(j * d.ny + c) * d.ny + q];
        else if (c == (j + 1) * d.ny + q) v = 1.0;
        S[0][r][c] = v;
    }
    __syncthreads();
    double logr = 0.0;
    bool zero = false;
    int cur = 0;
    for (int s = 0; s <= kSquarings; ++s) {
        if (s > 0) {
            if (idx < nn) {
                double t = 0.0;
                for (int k = 0; k < nx; ++k) t += S[cur][r][k] * S[cur][k][c];
                S[cur ^ 1][r][c] = t;
            }
            cur ^= 1;
            __syncthreads();
        }
        if (idx < 256) red[idx] = idx < nn ? S[cur][r][c] * S[cur][r][c] : 0.0;
        __syncthreads();
        if (idx == 0) {
            double t = 0.0;
            for (int i = 0; i < nn; ++i) t += red[i];
            nrm_s = sqrt(t);
        }
        __syncthreads();
        const double nrm = nrm_s;
        if (!(nrm > 0.0)) {  // nilpotent: rho = 0
            zero = true;
            break;
        }
        logr += ldexp(log(nrm), -s);
        if (idx < nn) S[cur][r][c] /= nrm;
        __syncthreads();
    }
    const double rho = zero ? 0.0 : exp(logr);
    const double lam = (rho_max > 0.0 && rho > rho_max) ? rho_max / rho : 1.0;
    if (idx == 0 && rho_out) *rho_out = rho;
    // scaled observer-canonical form: x^j_{k+1} = A_j y_k + x^{j+1}_k + B_j u_k, y_k = x^1_k
    const int nu = d.nu, ny = d.ny;
    if (idx < nx * 16) {
        const int rr = idx / 16, cc = idx % 16, j = rr / ny, q = rr % ny;
        const double f = pow(lam, (double)(j + 1));
        double a = 0.0, bb = 0.0;
        if (cc < nx) {
            if (cc < ny) a = f * th[(j * ny + cc) * ny + q];
            else if (cc == (j + 1) * ny + q) a = 1.0;
        }
        if (cc < nu) bb = f * th[(na * ny + j * nu + cc) * ny + q];
        Am[rr][cc] = a;
        Bm[rr][cc] = bb;
    }
    if (idx < ny * 16) {
        const int q = idx / 16, cc = idx % 16;
        Cm[q][cc] = cc == q ? 1.0 : 0.0;
    }
    __syncthreads();
    const bool stable = rho_max > 0.0 && rho_max < 1.0 && rho * lam < 1.0;
    if (stable) {
        // controllability Gramian P = sum_k A^k B B^T A^kT (Tm holds A^(2^j))
        bmm(P, Bm, false, Bm, true, nx, nx, nu);
        if (idx < nx * nx) Tm[idx / nx][idx % nx] = Am[idx / nx][idx % nx];
        __syncthreads();
        for (int j = 0; j < kSmith; ++j) {
            bmm(Tmp, Tm, false, P, false, nx, nx, nx);
            bmm(Tmp, Tmp, false, Tm, true, nx, nx, nx);
            if (idx < nx * nx) P[idx / nx][idx % nx] += Tmp[idx / nx][idx % nx];
            __syncthreads();
            bmm(Tm, Tm, false, Tm, false, nx, nx, nx);
        }
        // observability Gramian Q = sum_k A^kT C^T C A^k
        bmm(Q, Cm, true, Cm, false, nx, nx, ny);
        if (idx < nx * nx) Tm[idx / nx][idx % nx] = Am[idx % nx][idx / nx];
        __syncthreads();
        for (int j = 0; j < kSmith; ++j) {
            bmm(Tmp, Tm, false, Q, false, nx, nx, nx);
            bmm(Tmp, Tmp, false, Tm, true, nx, nx, nx);
            if (idx < nx * nx) Q[idx / nx][idx % nx] += Tmp[idx / nx][idx % nx];
            __syncthreads();
            bmm(Tm, Tm, false, Tm, false, nx, nx, nx);
        }
        if (idx == 0) ok = (chol_reg(P, nx, kGramReg) && chol_reg(Q, nx, kGramReg)) ? 1 : 0;
        __syncthreads();
    }
    if (stable && ok) {
        bmm(G, Q, true, P, false, nx, nx, nx);  // Lq^T Lp
        if (idx == 0) {
            jacobi_svd(G, Vm, sv, nx);
            ok = sv[nx - 1] > 0.0 ? 1 : 0;
        }
        __syncthreads();
    }
    if (stable && ok) {
        bmm(Tm, P, false, Vm, false, nx, nx, nx);  // T = Lp V S^-1/2
        bmm(Ti, G, true, Q, true, nx, nx, nx);     // T^-1 = S^-1/2 U^T Lq^T
        if (idx < nx * nx) {
            const int rr = idx / nx, cc = idx % nx;
            Tm[rr][cc] *= rsqrt(sv[cc]);
            Ti[rr][cc] *= rsqrt(sv[rr]);
        }
        __syncthreads();
        bmm(Tmp, Am, false, Tm, false, nx, nx, nx);
        bmm(Am, Ti, false, Tmp, false, nx, nx, nx);
        bmm(Bm, Ti, false, Bm, false, nx, nu, nx);
        bmm(Cm, Cm, false, Tm, false, ny, nx, nx);
        if (idx < nx) {  // sign of state idx: largest-magnitude entry of column idx of C positive
            int best = 0;
            for (int q = 1; q < ny; ++q)
                if (fabs(Cm[q][idx]) > fabs(Cm[best][idx])) best = q;
            sv[idx] = Cm[best][idx] < 0.0 ? -1.0 : 1.0;
        }
        __syncthreads();
        if (idx < nx * 16) {
            const int rr = idx / 16, cc = idx % 16;
            if (cc < nx) Am[rr][cc] *= sv[rr] * sv[cc];
            if (cc < nu) Bm[rr][cc] *= sv[rr];
        }
        if (idx < ny * nx) Cm[idx / nx][idx % nx] *= sv[idx % nx];
        __syncthreads();
    }
    constexpr int ld = kFB * kMaxKT;
    if (idx < nx * nx) Wp[(idx / nx) * ld + idx % nx] = (float)Am[idx / nx][idx % nx];
    if (idx < nx * nu) Wp[(idx / nu) * ld + nx + idx % nu] = (float)Bm[idx / nu][idx % nu];
    if (idx < ny * nx) Wp[(nx + idx / nx) * ld + idx % nx] = (float)Cm[idx / nx][idx % nx];
    if (idx == 0) *status = 0;
}

// ---------------------------------------------------------------------------
cudaError_t launch_reduce(const float* gpart, int n_warps, const double* loss_part, const float* Wp, const Dims& d,
                          double sigma2, double n_samples, float* grad, double* loss, double* loss_hist, int it,
                          cudaStream_t st)
{
    reduce_kernel<<<1, kWN, 0, st>>>(gpart, n_warps, loss_part, Wp, d, sigma2, n_samples, grad, loss, loss_hist, it);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* Wp, float* m, float* v, float* Wb, float* mb, float* vb, float* lr_scale,
                        double* acc_loss, const float* grad, const double* loss, const Dims& d, float lr, float b1,
                        float b2, float eps, float c1, float c2, cudaStream_t st)
{
    adam_kernel<<<1, kWN, 0, st>>>(Wp, m, v, Wb, mb, vb, lr_scale, acc_loss, grad, loss, d, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_stats(const float* u, const float* y, const float* p, long long n, int nu, int ny, int np,
                         double* part, double* stats, cudaStream_t st)
{
    stats_kernel<<<256, 256, 0, st>>>(u, y, p, n, nu, ny, np, part);
    stats_final_kernel<<<1, kStatStride, 0, st>>>(part, 256, nu + ny + 2 * np, np, stats);
    return cudaGetLastError();
}

int gram_blocks() { return kGramBlocks; }

cudaError_t launch_gram(const float* u, const float* y, int n_traj, int T, const Dims& d, int na, double* part,
                        cudaStream_t st)
{
    gram_kernel<<<kGramBlocks, 1024, 0, st>>>(u, y, n_traj, T, d, na, part);
    return cudaGetLastError();
}

cudaError_t launch_ls_solve(const double* part, const Dims& d, int na, double rho_max, double* theta, float* Wp,
                            int* status, double* rho_out, cudaStream_t st)
{
    ls_solve_kernel<<<1, 1024, 0, st>>>(part, kGramBlocks, d, na, rho_max, theta, Wp, status, rho_out);
    return cudaGetLastError();
}

}  // namespace lpv

namespace lpv {

// ---------------------------------------------------------------------------
// L-BFGS (Nocedal and Wright, Algorithm 7.4) on the trainable weights: FP64
// master weights, gradient and curvature pairs; one block of kWN threads
// (one per padded weight), fixed-order FP64 block reductions.
// ---------------------------------------------------------------------------
namespace {

__device__ double block_dot(double v, double* red)
{
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_down_sync(0xffffffffu, v, s);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kWN / 32; ++w) t += red[w];
    return t;  // every thread
}

}  // namespace

__global__ void lbfgs_init_kernel(const float* __restrict__ Wp, const float* __restrict__ grad, Dims d, LbfgsDev L)
{
    const int i = threadIdx.x;
    const bool tr = trainable(d, i / (kFB * kMaxKT), i % (kFB * kMaxKT));
    L.W[i] = tr ? (double)Wp[i] : 0.0;
    L.g[i] = tr ? (double)grad[i] : 0.0;
    if (i == 0) {
        L.count[0] = 0;
        L.count[1] = 0;
    }
}

// d = -H g by the two-loop recursion over the stored pairs (newest first),
// H_0 = (s.y / y.y) I of the newest pair; falls back to d = -g (and clears the
// history) when that is not a descent direction.  Writes g.d and g.g.
__global__ void lbfgs_dir_kernel(LbfgsDev L)
{
    __shared__ double red[kWN / 32];
    __shared__ double alpha[kLbfgsM];
    const int i = threadIdx.x;
    const int n = L.count[0], next = L.count[1];
    double q = L.g[i];
    for (int k = 0; k < n; ++k) {
        const int j = (next - 1 - k + kLbfgsM) % kLbfgsM;
        const double a = L.rho[j] * block_dot(L.S[j * kWN + i] * q, red);
        if (i == 0) alpha[j] = a;
        q -= a * L.Y[j * kWN + i];
    }
    double gamma = 1.0;
    if (n > 0) {
        const int j = (next - 1 + kLbfgsM) % kLbfgsM;
        const double yy = block_dot(L.Y[j * kWN + i] * L.Y[j * kWN + i], red);
        gamma = yy > 0.0 ? 1.0 / (L.rho[j] * yy) : 1.0;
    }
    __syncthreads();
    double r = gamma * q;
    for (int k = n - 1; k >= 0; --k) {
        const int j = (next - 1 - k + kLbfgsM) % kLbfgsM;
        const double b = L.rho[j] * block_dot(L.Y[j * kWN + i] * r, red);
        r += L.S[j * kWN + i] * (alpha[j] - b);
    }
    const double gi = L.g[i];
    const double gd = -block_dot(gi * r, red);
    const double gg = block_dot(gi * gi, red);
    if (gd < 0.0) {
        L.d[i] = -r;
        if (i == 0) L.gd[0] = gd;
    } else {
        L.d[i] = -gi;
        if (i == 0) {
            L.gd[0] = -gg;
            L.count[0] = 0;
        }
    }
    if (i == 0) L.gd[1] = gg;
}

// Wp = W + step d on the trainable entries (the trial point).
__global__ void lbfgs_try_kernel(float* __restrict__ Wp, Dims d, LbfgsDev L, double step)
{
    const int i = threadIdx.x;
    const bool tr = trainable(d, i / (kFB * kMaxKT), i % (kFB * kMaxKT));
    Wp[i] = tr ? (float)(L.W[i] + step * L.d[i]) : 0.f;
}

// Accepts the trial point: s = step d, y = g_new - g; the pair is stored when
// s.y > 0 (curvature condition), then W and g move to the new point.
__global__ void lbfgs_accept_kernel(const float* __restrict__ grad, Dims d, LbfgsDev L, double step)
{
    __shared__ double red[kWN / 32];
    const int i = threadIdx.x;
    const bool tr = trainable(d, i / (kFB * kMaxKT), i % (kFB * kMaxKT));
    const double gn = tr ? (double)grad[i] : 0.0;
    const double s = step * L.d[i], y = gn - L.g[i];
    const double sy = block_dot(s * y, red);
    const double yy = block_dot(y * y, red);
    const int next = L.count[1];
    __syncthreads();
    if (sy > 1e-12 * yy && sy > 0.0) {
        L.S[next * kWN + i] = s;
        L.Y[next * kWN + i] = y;
        if (i == 0) {
            L.rho[next] = 1.0 / sy;
            L.count[0] = min(L.count[0] + 1, kLbfgsM);
            L.count[1] = (next + 1) % kLbfgsM;
        }
    }
    L.W[i] += s;
    L.g[i] = gn;
}

cudaError_t launch_lbfgs_init(const float* Wp, const float* grad, const Dims& d, const LbfgsDev& L, cudaStream_t st)
{
    lbfgs_init_kernel<<<1, kWN, 0, st>>>(Wp, grad, d, L);
    return cudaGetLastError();
}

cudaError_t launch_lbfgs_dir(const LbfgsDev& L, cudaStream_t st)
{
    lbfgs_dir_kernel<<<1, kWN, 0, st>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_lbfgs_try(float* Wp, const Dims& d, const LbfgsDev& L, double step, cudaStream_t st)
{
    lbfgs_try_kernel<<<1, kWN, 0, st>>>(Wp, d, L, step);
    return cudaGetLastError();
}

cudaError_t launch_lbfgs_accept(const float* grad, const Dims& d, const LbfgsDev& L, double step, cudaStream_t st)
{
    lbfgs_accept_kernel<<<1, kWN, 0, st>>>(grad, d, L, step);
    return cudaGetLastError();
}

}  // namespace lpv
