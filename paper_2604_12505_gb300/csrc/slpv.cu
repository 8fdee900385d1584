// slpv.cu -- the self-scheduled LPV surrogate of the identification study
// (Section 4, Eqs. 24-27; Section 5.3.2) behind the C ABI of include/slpv.h:
// free-run loss and its gradient by backpropagation through time, Adam, the
// free run of the augmented model and its closed loop with the PD law of
// Eq. 28.
//
// One thread carries one trajectory.  The state (nx <= 8), the scheduling
// network (two layers of four tanh neurons) and the 7 x 7 matrices of the
// paper's model are far below a tensor-core tile, and every step depends on
// the previous one, so the work is FP32 FMA chains with the parameters
// broadcast from shared memory.  The gradient kernel accumulates each
// thread's gradient in its own shared-memory column ([parameter][thread],
// conflict-free) and sums the columns in a fixed order in FP64, so results
// are deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/slpv.h"

namespace sph {
int set_last_error(int code, const char* msg);
}

namespace slpvk {

constexpr int NU = 3, NY = 3, NH = 4;
constexpr int kThreads = 64;  // trajectories per block of the gradient kernel

// Offsets of the blocks of theta (see include/slpv.h).
template <int NX>
struct Lay {
    static constexpr int NZ = NX + NU, NO = NX + NY, NM = NO * NZ;
    static constexpr int M0 = 0, M1 = NM, W1 = 2 * NM, B1 = W1 + NH * NZ, W2 = B1 + NH, B2 = W2 + NH * NH;
    static constexpr int W3 = B2 + NH, B3 = W3 + NH, N = B3 + 1;
};

inline int n_params(int nx)
{
    const int nz = nx + NU, no = nx + NY;
    return 2 * no * nz + NH * nz + NH + NH * NH + NH + NH + 1;
}

// Training stages: which entries of theta move (never the D blocks).
enum { kStageAll = 0, kStageLti = 1, kStageScheduling = 2 };

// Whether theta[q] is trained in `stage`: all entries, M_0 only (the LTI
// stage), or M_1 and the network only (M_0 held).
__host__ __device__ inline bool trainable(int q, int nx, int stage)
{
    const int nz = nx + NU, nm = (nx + NY) * nz;
    if (q < 2 * nm) {
        if (stage == kStageLti && q >= nm) return false;
        if (stage == kStageScheduling && q < nm) return false;
        const int r = (q % nm) / nz, j = (q % nm) % nz;
        return !(r >= nx && j >= nx);
    }
    return stage != kStageLti;
}

// Scheduling map eta(z) = w3 . tanh(W2 tanh(W1 z + b1) + b2) + b3.
template <int NX>
__device__ __forceinline__ float eta(const float* th, const float* z, float* h1, float* h2)
{
    using Q = Lay<NX>;
#pragma unroll
    for (int i = 0; i < NH; ++i) {
        float a = th[Q::B1 + i];
#pragma unroll
        for (int j = 0; j < Q::NZ; ++j) a = fmaf(th[Q::W1 + i * Q::NZ + j], z[j], a);
        h1[i] = tanhf(a);
    }
#pragma unroll
    for (int i = 0; i < NH; ++i) {
        float a = th[Q::B2 + i];
#pragma unroll
        for (int j = 0; j < NH; ++j) a = fmaf(th[Q::W2 + i * NH + j], h1[j], a);
        h2[i] = tanhf(a);
    }
    float p = th[Q::B3];
#pragma unroll
    for (int i = 0; i < NH; ++i) p = fmaf(th[Q::W3 + i], h2[i], p);
    return p;
}

// o = (M_0 + p M_1) z = [x_{k+1}; y_k] (Eqs. 24, 25).
template <int NX>
__device__ __forceinline__ void mz(const float* th, float p, const float* z, float* o)
{
    using Q = Lay<NX>;
#pragma unroll
    for (int r = 0; r < Q::NO; ++r) {
        float a = 0.f;
#pragma unroll
        for (int j = 0; j < Q::NZ; ++j) a = fmaf(fmaf(p, th[Q::M1 + r * Q::NZ + j], th[Q::M0 + r * Q::NZ + j]), z[j], a);
        o[r] = a;
    }
}

// ---------------------------------------------------------------------------
// Loss and gradient: per block, partial sums part[block][0..N) (gradient of
// the data term, already divided by the sample count) and part[block][N]
// (sum of squared normalised errors).
// ---------------------------------------------------------------------------
template <int NX>
__global__ void __launch_bounds__(kThreads) grad_kernel(const float* __restrict__ theta, const float* __restrict__ u,
                                                        const float* __restrict__ y, const float* __restrict__ scales,
                                                        int n_traj, int T, float inv_n, int want_grad,
                                                        float* __restrict__ xh, double* __restrict__ part)
{
    using Q = Lay<NX>;
    extern __shared__ float4 shm4[];
    float* th = reinterpret_cast<float*>(shm4);
    float* acc = th + ((Q::N + 3) & ~3);                            // [N][kThreads]
    double* lbuf = reinterpret_cast<double*>(acc + Q::N * kThreads);  // [kThreads]
    const int tid = threadIdx.x;
    for (int i = tid; i < Q::N; i += kThreads) th[i] = theta[i];
    if (want_grad)
        for (int i = tid; i < Q::N * kThreads; i += kThreads) acc[i] = 0.f;
    __syncthreads();
    const int tr = blockIdx.x * kThreads + tid;
    double lsum = 0.0;
    if (tr < n_traj) {
        float isu[NU], isy[NY];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            isu[c] = 1.0f / scales[c];
            isy[c] = 1.0f / scales[3 + c];
        }
        const float* ut = u + (size_t)tr * T * NU;
        const float* yt = y + (size_t)tr * T * NY;
        float x[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) x[i] = 0.f;
        for (int k = 0; k < T; ++k) {
            if (want_grad) {
#pragma unroll
                for (int i = 0; i < NX; ++i) xh[((size_t)k * n_traj + tr) * NX + i] = x[i];
            }
            float z[Q::NZ], h1[NH], h2[NH], o[Q::NO];
#pragma unroll
            for (int i = 0; i < NX; ++i) z[i] = x[i];
#pragma unroll
            for (int c = 0; c < NU; ++c) z[NX + c] = ut[NU * k + c] * isu[c];
            const float p = eta<NX>(th, z, h1, h2);
            mz<NX>(th, p, z, o);
            float e2 = 0.f;
#pragma unroll
            for (int c = 0; c < NY; ++c) {
                const float r = o[NX + c] - yt[NY * k + c] * isy[c];
                e2 = fmaf(r, r, e2);
            }
            lsum += (double)e2;
#pragma unroll
            for (int i = 0; i < NX; ++i) x[i] = o[i];
        }
        if (want_grad) {
            float lam[NX];  // dJ / dx_{k+1}
#pragma unroll
            for (int i = 0; i < NX; ++i) lam[i] = 0.f;
            float* my = acc + tid;
            for (int k = T - 1; k >= 0; --k) {
                float z[Q::NZ], h1[NH], h2[NH], o[Q::NO], a[Q::NO];
#pragma unroll
                for (int i = 0; i < NX; ++i) z[i] = xh[((size_t)k * n_traj + tr) * NX + i];
#pragma unroll
                for (int c = 0; c < NU; ++c) z[NX + c] = ut[NU * k + c] * isu[c];
                const float p = eta<NX>(th, z, h1, h2);
                mz<NX>(th, p, z, o);
#pragma unroll
                for (int i = 0; i < NX; ++i) a[i] = lam[i];
#pragma unroll
                for (int c = 0; c < NY; ++c) a[NX + c] = 2.0f * (o[NX + c] - yt[NY * k + c] * isy[c]) * inv_n;
                // M_0 and M_1 (outer product a z^T, scaled by p for M_1); s = dJ/dp
                float s = 0.f;
#pragma unroll
                for (int r = 0; r < Q::NO; ++r) {
                    float m1z = 0.f;
#pragma unroll
                    for (int j = 0; j < Q::NZ; ++j) {
                        const int q = r * Q::NZ + j;
                        const float az = a[r] * z[j];
                        my[(Q::M0 + q) * kThreads] += az;
                        my[(Q::M1 + q) * kThreads] += p * az;
                        m1z = fmaf(th[Q::M1 + q], z[j], m1z);
                    }
                    s = fmaf(a[r], m1z, s);
                }
                // back through the scheduling network
                float d2[NH], d1[NH];
#pragma unroll
                for (int i = 0; i < NH; ++i) {
                    my[(Q::W3 + i) * kThreads] += s * h2[i];
                    d2[i] = s * th[Q::W3 + i] * (1.0f - h2[i] * h2[i]);
                    my[(Q::B2 + i) * kThreads] += d2[i];
                }
                my[Q::B3 * kThreads] += s;
#pragma unroll
                for (int i = 0; i < NH; ++i) {
                    float b = 0.f;
#pragma unroll
                    for (int j = 0; j < NH; ++j) {
                        my[(Q::W2 + i * NH + j) * kThreads] += d2[i] * h1[j];
                        b = fmaf(th[Q::W2 + j * NH + i], d2[j], b);
                    }
                    d1[i] = b * (1.0f - h1[i] * h1[i]);
                    my[(Q::B1 + i) * kThreads] += d1[i];
                }
#pragma unroll
                for (int i = 0; i < NH; ++i)
#pragma unroll
                    for (int j = 0; j < Q::NZ; ++j) my[(Q::W1 + i * Q::NZ + j) * kThreads] += d1[i] * z[j];
                // dJ/dx_k = (M^T a + W1^T d1)[0..nx)
#pragma unroll
                for (int j = 0; j < NX; ++j) {
                    float v = 0.f;
#pragma unroll
                    for (int r = 0; r < Q::NO; ++r)
                        v = fmaf(fmaf(p, th[Q::M1 + r * Q::NZ + j], th[Q::M0 + r * Q::NZ + j]), a[r], v);
#pragma unroll
                    for (int i = 0; i < NH; ++i) v = fmaf(th[Q::W1 + i * Q::NZ + j], d1[i], v);
                    lam[j] = v;
                }
            }
        }
    }
    lbuf[tid] = lsum;
    __syncthreads();
    double* pb = part + (size_t)blockIdx.x * (Q::N + 1);
    if (want_grad) {
        for (int q = tid; q < Q::N; q += kThreads) {
            double s = 0.0;
            for (int t = 0; t < kThreads; ++t) s += (double)acc[q * kThreads + t];
            pb[q] = s;
        }
    }
    if (tid == 0) {
        double s = 0.0;
        for (int t = 0; t < kThreads; ++t) s += lbuf[t];
        pb[Q::N] = s;
    }
}

// Sums the block partials in block order, adds the l2 term, masks the fixed
// entries: loss = sum_sq * inv_n + sigma2/2 |theta|^2, grad = sum + sigma2 theta.
__global__ void final_kernel(const double* __restrict__ part, int nblk, int N, int nx, const float* __restrict__ theta,
                             float sigma2, double inv_n, int want_grad, int stage, double* __restrict__ loss,
                             float* __restrict__ grad)
{
    __shared__ double sq[512];
    const int q = threadIdx.x;
    double t2 = 0.0;
    if (q < N) {
        const double th = (double)theta[q];
        t2 = th * th;
        if (want_grad) {
            double g = 0.0;
            for (int b = 0; b < nblk; ++b) g += part[(size_t)b * (N + 1) + q];
            g += (double)sigma2 * th;
            grad[q] = trainable(q, nx, stage) ? (float)g : 0.f;
        }
    }
    sq[q] = t2;
    __syncthreads();
    if (q == 0) {
        double s = 0.0, r = 0.0;
        for (int i = 0; i < N; ++i) r += sq[i];
        for (int b = 0; b < nblk; ++b) s += part[(size_t)b * (N + 1) + N];
        *loss = s * inv_n + 0.5 * (double)sigma2 * r;
    }
}

// ---------------------------------------------------------------------------
// Adam with step rejection (one block, one thread per entry of theta)
// ---------------------------------------------------------------------------
struct AdamDev {
    float *th, *m, *v, *thb, *lr_scale;
    double* acc_loss;
    int* t;
};

__global__ void adam_kernel(AdamDev A, const float* __restrict__ grad, const double* __restrict__ loss,
                            double* __restrict__ hist, int it, int N, float lr)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const int q = threadIdx.x;
    const double L = *loss, La = *A.acc_loss;
    const int t0 = *A.t;
    float sc = *A.lr_scale;
    const bool ok = isfinite(L) && (La < 0.0 || L <= 10.0 * La);
    if (q == 0 && hist) hist[it] = L;
    __syncthreads();
    if (ok) {  // the iterate is accepted: it becomes the fall-back point, then one Adam step
        const int t = t0 + 1;
        if (q < N) {
            A.thb[q] = A.th[q];
            const float g = grad[q];
            const float m = b1 * A.m[q] + (1.0f - b1) * g;
            const float v = b2 * A.v[q] + (1.0f - b2) * g * g;
            A.m[q] = m;
            A.v[q] = v;
            const float mh = m / (1.0f - powf(b1, (float)t)), vh = v / (1.0f - powf(b2, (float)t));
            A.th[q] -= lr * sc * mh / (sqrtf(vh) + eps);
        }
        if (q == 0) {
            *A.t = t;
            *A.acc_loss = L;
        }
    } else if (t0 > 0) {  // back to the fall-back point, the same step at half the size
        sc *= 0.5f;
        if (q < N) {
            const float mh = A.m[q] / (1.0f - powf(b1, (float)t0)), vh = A.v[q] / (1.0f - powf(b2, (float)t0));
            A.th[q] = A.thb[q] - lr * sc * mh / (sqrtf(vh) + eps);
        }
        if (q == 0) *A.lr_scale = sc;
    }
}

// ---------------------------------------------------------------------------
// L-BFGS (one block, one thread per entry of theta; FP64 state)
// ---------------------------------------------------------------------------
constexpr int kLM = 10;   // curvature pairs kept
constexpr int kLT = 320;  // threads: at least n_theta (315 for nx = 8)

struct LbDev {
    double *W, *g, *d, *S, *Y, *rho, *gd;
    int* count;  // [0] pairs held, [1] next slot
    int N;
};

__device__ double block_dot(double v, double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kLT / 32; ++w) t += red[w];
    return t;  // every thread, fixed order
}

// W = theta, g = grad (zero on fixed entries), no pairs.
__global__ void lb_init_kernel(const float* __restrict__ th, const float* __restrict__ grad, LbDev L)
{
    const int i = threadIdx.x;
    L.W[i] = i < L.N ? (double)th[i] : 0.0;
    L.g[i] = i < L.N ? (double)grad[i] : 0.0;
    if (i == 0) L.count[0] = L.count[1] = 0;
}

// d = -H g by the two-loop recursion (newest pair first), H_0 = (s.y / y.y) I
// of the newest pair; d = -g (history cleared) when that is no descent
// direction.  gd[0] = g.d, gd[1] = g.g.
__global__ void lb_dir_kernel(LbDev L)
{
    __shared__ double red[kLT / 32];
    __shared__ double alpha[kLM];
    const int i = threadIdx.x;
    const int n = L.count[0], next = L.count[1];
    double q = L.g[i];
    for (int k = 0; k < n; ++k) {
        const int j = (next - 1 - k + kLM) % kLM;
        const double a = L.rho[j] * block_dot(L.S[j * kLT + i] * q, red);
        if (i == 0) alpha[j] = a;
        q -= a * L.Y[j * kLT + i];
    }
    double gamma = 1.0;
    if (n > 0) {
        const int j = (next - 1 + kLM) % kLM;
        const double yy = block_dot(L.Y[j * kLT + i] * L.Y[j * kLT + i], red);
        gamma = yy > 0.0 ? 1.0 / (L.rho[j] * yy) : 1.0;
    }
    __syncthreads();
    double r = gamma * q;
    for (int k = n - 1; k >= 0; --k) {
        const int j = (next - 1 - k + kLM) % kLM;
        const double b = L.rho[j] * block_dot(L.Y[j * kLT + i] * r, red);
        r += L.S[j * kLT + i] * (alpha[j] - b);
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

// theta = W + step d (the trial point; fixed entries have d = 0).
__global__ void lb_try_kernel(float* __restrict__ th, LbDev L, double step)
{
    const int i = threadIdx.x;
    if (i < L.N) th[i] = (float)(L.W[i] + step * L.d[i]);
}

// Accepts the trial point: s = step d, y = g_new - g, stored when s.y > 0.
__global__ void lb_accept_kernel(const float* __restrict__ grad, LbDev L, double step)
{
    __shared__ double red[kLT / 32];
    const int i = threadIdx.x;
    const double gn = i < L.N ? (double)grad[i] : 0.0;
    const double s = step * L.d[i], y = gn - L.g[i];
    const double sy = block_dot(s * y, red);
    const double yy = block_dot(y * y, red);
    const int next = L.count[1];
    __syncthreads();
    if (sy > 1e-12 * yy && sy > 0.0) {
        L.S[next * kLT + i] = s;
        L.Y[next * kLT + i] = y;
        if (i == 0) {
            L.rho[next] = 1.0 / sy;
            L.count[0] = min(L.count[0] + 1, kLM);
            L.count[1] = (next + 1) % kLM;
        }
    }
    L.W[i] += s;
    L.g[i] = gn;
}

// ---------------------------------------------------------------------------
// Free run of the augmented model (velocities and positions, physical units)
// ---------------------------------------------------------------------------
template <int NX>
__global__ void predict_kernel(const float* __restrict__ theta, const float* __restrict__ scales,
                               const float* __restrict__ u, int n_traj, int T, float Ts, float* __restrict__ vel,
                               float* __restrict__ pos)
{
    using Q = Lay<NX>;
    __shared__ float th[Q::N];
    for (int i = threadIdx.x; i < Q::N; i += blockDim.x) th[i] = theta[i];
    __syncthreads();
    const int tr = blockIdx.x * blockDim.x + threadIdx.x;
    if (tr >= n_traj) return;
    float isu[NU], sy[NY], x[NX], e[NY] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        isu[c] = 1.0f / scales[c];
        sy[c] = scales[3 + c];
    }
#pragma unroll
    for (int i = 0; i < NX; ++i) x[i] = 0.f;
    for (int k = 0; k < T; ++k) {
        float z[Q::NZ], h1[NH], h2[NH], o[Q::NO];
#pragma unroll
        for (int i = 0; i < NX; ++i) z[i] = x[i];
        const size_t row = ((size_t)tr * T + k) * 3;
#pragma unroll
        for (int c = 0; c < NU; ++c) z[NX + c] = u[row + c] * isu[c];
        const float p = eta<NX>(th, z, h1, h2);
        mz<NX>(th, p, z, o);
#pragma unroll
        for (int c = 0; c < NY; ++c) {
            const float v = o[NX + c] * sy[c];
            if (vel) vel[row + c] = v;
            if (pos) pos[row + c] = e[c];
            e[c] = fmaf(Ts, v, e[c]);
        }
#pragma unroll
        for (int i = 0; i < NX; ++i) x[i] = o[i];
    }
}

// ---------------------------------------------------------------------------
// Closed loop with the PD law of Eq. 28 (one thread per run)
// ---------------------------------------------------------------------------
template <int NX>
__global__ void closed_loop_kernel(const float* __restrict__ theta, const float* __restrict__ scales, int B, int T,
                                   const double* __restrict__ F, const double* __restrict__ tau,
                                   const double* __restrict__ ref, float Ts, float J, float w, float xi,
                                   float* __restrict__ out)
{
    using Q = Lay<NX>;
    __shared__ float th[Q::N];
    for (int i = threadIdx.x; i < Q::N; i += blockDim.x) th[i] = theta[i];
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float isu[NU], sy[NY], x[NX], e[NY] = {0.f, 0.f, 0.f}, un[NU] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        isu[c] = 1.0f / scales[c];
        sy[c] = scales[3 + c];
    }
#pragma unroll
    for (int i = 0; i < NX; ++i) x[i] = 0.f;
    const float kp = J * w * w, kd = 2.0f * xi * J * w;
    for (int k = 0; k < T; ++k) {
        float z[Q::NZ], h1[NH], h2[NH], o[Q::NO];
        // the sample: thetadot from the scheduling of the held input
#pragma unroll
        for (int i = 0; i < NX; ++i) z[i] = x[i];
#pragma unroll
        for (int c = 0; c < NU; ++c) z[NX + c] = un[c];
        float p = eta<NX>(th, z, h1, h2);
        float wd = 0.f;
#pragma unroll
        for (int j = 0; j < Q::NZ; ++j)
            wd = fmaf(fmaf(p, th[Q::M1 + (NX + 2) * Q::NZ + j], th[Q::M0 + (NX + 2) * Q::NZ + j]), z[j], wd);
        wd *= sy[2];
        const size_t bk = (size_t)b * T + k;
        const float tc = kp * ((float)ref[bk] - e[2]) - kd * wd;
        un[0] = (float)F[2 * bk] * isu[0];
        un[1] = (float)F[2 * bk + 1] * isu[1];
        un[2] = ((float)tau[bk] + tc) * isu[2];
#pragma unroll
        for (int c = 0; c < NU; ++c) z[NX + c] = un[c];
        p = eta<NX>(th, z, h1, h2);
        mz<NX>(th, p, z, o);
        float* ob = out + bk * 6;
#pragma unroll
        for (int c = 0; c < NY; ++c) {
            const float v = o[NX + c] * sy[c];
            ob[c] = e[c];
            ob[3 + c] = v;
            e[c] = fmaf(Ts, v, e[c]);
        }
#pragma unroll
        for (int i = 0; i < NX; ++i) x[i] = o[i];
    }
}

// ---------------------------------------------------------------------------
// Data scales: root mean square per channel (fixed-order FP64 sums)
// ---------------------------------------------------------------------------
constexpr int kStatBlocks = 152, kStatThreads = 256;

__global__ void stats_kernel(const float* __restrict__ u, const float* __restrict__ y, long long n,
                             double* __restrict__ part)
{
    __shared__ double s[6][kStatThreads];
    double a[6] = {0, 0, 0, 0, 0, 0};
    for (long long i = blockIdx.x * (long long)kStatThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kStatThreads) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double uu = u[3 * i + c], yy = y[3 * i + c];
            a[c] += uu * uu;
            a[3 + c] += yy * yy;
        }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) s[c][threadIdx.x] = a[c];
    __syncthreads();
    if (threadIdx.x < 6) {
        double t = 0.0;
        for (int i = 0; i < kStatThreads; ++i) t += s[threadIdx.x][i];
        part[blockIdx.x * 6 + threadIdx.x] = t;
    }
}

__global__ void stats_final_kernel(const double* __restrict__ part, int nblk, long long n, float* __restrict__ scales)
{
    const int c = threadIdx.x;
    if (c >= 6) return;
    double t = 0.0;
    for (int b = 0; b < nblk; ++b) t += part[b * 6 + c];
    scales[c] = (float)sqrt(t / (double)n);
}

// ---------------------------------------------------------------------------
// Least-squares LTI start: y_{k+1} = A1 y_k + B1 u_k over all samples
// (normalised), normal equations G = sum phi phi^T, R = sum phi t^T with
// phi = [y_k; u_k], t = y_{k+1}; per-block FP64 partials, fixed-order sums.
// ---------------------------------------------------------------------------
constexpr int kLsThreads = 128;
constexpr int kLsVals = 36 + 18;  // G (6 x 6) and R (6 x 3)

__global__ void ls_gram_kernel(const float* __restrict__ u, const float* __restrict__ y,
                               const float* __restrict__ scales, int n_traj, int T, double* __restrict__ part)
{
    __shared__ double red[kLsThreads];
    double acc[kLsVals];
#pragma unroll
    for (int i = 0; i < kLsVals; ++i) acc[i] = 0.0;
    const long long n = (long long)n_traj * (T - 1);
    for (long long s = blockIdx.x * (long long)kLsThreads + threadIdx.x; s < n; s += (long long)gridDim.x * kLsThreads) {
        const int tr = (int)(s / (T - 1)), k = (int)(s % (T - 1));
        const size_t r0 = ((size_t)tr * T + k) * 3, r1 = r0 + 3;
        double ph[6], t[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ph[c] = (double)y[r0 + c] / (double)scales[3 + c];
            ph[3 + c] = (double)u[r0 + c] / (double)scales[c];
            t[c] = (double)y[r1 + c] / (double)scales[3 + c];
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) {
#pragma unroll
            for (int j = 0; j < 6; ++j) acc[i * 6 + j] = fma(ph[i], ph[j], acc[i * 6 + j]);
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[36 + i * 3 + c] = fma(ph[i], t[c], acc[36 + i * 3 + c]);
        }
    }
    for (int v = 0; v < kLsVals; ++v) {  // block sums in thread order
        red[threadIdx.x] = acc[v];
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int i = 0; i < kLsThreads; ++i) t += red[i];
            part[blockIdx.x * kLsVals + v] = t;
        }
        __syncthreads();
    }
}

// Sums the partials, solves (G + 1e-12 tr(G)/6 I) Theta = R by Cholesky and
// writes theta: A_0 = [[A1, 0], [0, 0]], B_0 = [[B1], [0]], C_0 = [I, 0], the
// rest zero.
template <int NX>
__global__ void ls_solve_kernel(const double* __restrict__ part, int nblk, float* __restrict__ theta,
                                int* __restrict__ status)
{
    using Q = Lay<NX>;
    for (int i = threadIdx.x; i < Q::N; i += blockDim.x) theta[i] = 0.f;
    __syncthreads();
    if (threadIdx.x != 0) return;
    double G[36], R[18];
    for (int v = 0; v < kLsVals; ++v) {
        double t = 0.0;
        for (int b = 0; b < nblk; ++b) t += part[b * kLsVals + v];
        if (v < 36) G[v] = t; else R[v - 36] = t;
    }
    double tr = 0.0;
    for (int i = 0; i < 6; ++i) tr += G[i * 6 + i];
    for (int i = 0; i < 6; ++i) G[i * 6 + i] += 1e-12 * tr / 6.0;
    // Cholesky G = L L^T in place (lower triangle)
    for (int j = 0; j < 6; ++j) {
        double d = G[j * 6 + j];
        for (int k = 0; k < j; ++k) d -= G[j * 6 + k] * G[j * 6 + k];
        if (!(d > 0.0)) {
            *status = 1;
            return;
        }
        d = sqrt(d);
        G[j * 6 + j] = d;
        for (int i = j + 1; i < 6; ++i) {
            double s = G[i * 6 + j];
            for (int k = 0; k < j; ++k) s -= G[i * 6 + k] * G[j * 6 + k];
            G[i * 6 + j] = s / d;
        }
    }
    double X[18];
    for (int c = 0; c < 3; ++c) {  // L z = r, L^T x = z
        double z[6];
        for (int i = 0; i < 6; ++i) {
            double s = R[i * 3 + c];
            for (int k = 0; k < i; ++k) s -= G[i * 6 + k] * z[k];
            z[i] = s / G[i * 6 + i];
        }
        for (int i = 5; i >= 0; --i) {
            double s = z[i];
            for (int k = i + 1; k < 6; ++k) s -= G[k * 6 + i] * X[k * 3 + c];
            X[i * 3 + c] = s / G[i * 6 + i];
        }
    }
    // y_{k+1}[c] = sum_i X[i][c] phi[i]: A1[c][j] = X[j][c], B1[c][j] = X[3 + j][c]
    for (int c = 0; c < 3; ++c) {
        for (int j = 0; j < 3; ++j) {
            theta[Q::M0 + c * Q::NZ + j] = (float)X[j * 3 + c];
            theta[Q::M0 + c * Q::NZ + NX + j] = (float)X[(3 + j) * 3 + c];
        }
        theta[Q::M0 + (NX + c) * Q::NZ + c] = 1.0f;
    }
    *status = 0;
}

}  // namespace slpvk

using namespace slpvk;

struct slpv_model {
    slpv_config cfg{};
    int N = 0;
    float *th = nullptr, *m = nullptr, *v = nullptr, *thb = nullptr, *lr_scale = nullptr, *grad = nullptr;
    float* scales = nullptr;
    double *acc_loss = nullptr, *loss = nullptr;
    int* t = nullptr;
    double* part = nullptr;
    size_t part_cap = 0;
    float* xh = nullptr;
    size_t xh_cap = 0;
    double* spart = nullptr;
    double* lb = nullptr;  // L-BFGS state, allocated on first use
    int* lb_count = nullptr;
};

namespace {

#define SCK(call)                                                                                        \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) return sph::set_last_error(SPH_E_CUDA, (std::string(#call ": ") +        \
                                                                       cudaGetErrorString(e_)).c_str()); \
    } while (0)

int inval(const char* msg) { return sph::set_last_error(SPH_E_INVAL, msg); }

bool nx_ok(int nx) { return nx == 2 || nx == 4 || nx == 6 || nx == 8; }

template <class F>
cudaError_t by_nx(int nx, F&& f)
{
    switch (nx) {
    case 2: return f(std::integral_constant<int, 2>{});
    case 4: return f(std::integral_constant<int, 4>{});
    case 6: return f(std::integral_constant<int, 6>{});
    case 8: return f(std::integral_constant<int, 8>{});
    default: return cudaErrorInvalidValue;
    }
}

size_t grad_smem(int N) { return (size_t)((N + 3) & ~3) * 4 + (size_t)N * kThreads * 4 + kThreads * 8; }

// Ensures the per-call buffers (block partials, state history) are large enough.
int reserve(slpv_model* m, int n_traj, int T, bool grad)
{
    const size_t nblk = (size_t)(n_traj + kThreads - 1) / kThreads;
    const size_t pneed = nblk * (m->N + 1);
    if (pneed > m->part_cap) {
        cudaFree(m->part);
        m->part = nullptr;
        m->part_cap = 0;
        SCK(cudaMalloc(&m->part, pneed * sizeof(double)));
        m->part_cap = pneed;
    }
    const size_t xneed = grad ? (size_t)n_traj * T * m->cfg.nx : 0;
    if (xneed > m->xh_cap) {
        cudaFree(m->xh);
        m->xh = nullptr;
        m->xh_cap = 0;
        cudaError_t e = cudaMalloc(&m->xh, xneed * sizeof(float));
        if (e != cudaSuccess) return sph::set_last_error(SPH_E_NOMEM, "slpv: state history allocation failed");
        m->xh_cap = xneed;
    }
    return SPH_OK;
}

// Launches the loss (and gradient) into m->loss / grad_out.
int loss_grad_launch(slpv_model* m, const float* u, const float* y, int n_traj, int T, int stage, float* grad_out,
                     cudaStream_t st)
{
    const bool want = grad_out != nullptr;
    int rc = reserve(m, n_traj, T, want);
    if (rc) return rc;
    const int nblk = (n_traj + kThreads - 1) / kThreads;
    const float inv_n = (float)(1.0 / ((double)n_traj * T));
    const size_t smem = grad_smem(m->N);
    cudaError_t e = by_nx(m->cfg.nx, [&](auto c) {
        constexpr int NX = decltype(c)::value;
        cudaError_t a = cudaFuncSetAttribute(grad_kernel<NX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (a != cudaSuccess) return a;
        grad_kernel<NX><<<nblk, kThreads, smem, st>>>(m->th, u, y, m->scales, n_traj, T, inv_n, want ? 1 : 0, m->xh,
                                                      m->part);
        return cudaGetLastError();
    });
    SCK(e);
    final_kernel<<<1, 512, 0, st>>>(m->part, nblk, m->N, m->cfg.nx, m->th, m->cfg.sigma2, 1.0 / ((double)n_traj * T),
                                    want ? 1 : 0, stage, m->loss, grad_out);
    SCK(cudaGetLastError());
    return SPH_OK;
}

int check_data(const slpv_model* m, const void* u, int n_traj, int T)
{
    if (!m || !u || n_traj < 1 || T < 1) return inval("slpv: NULL pointer or empty data");
    return SPH_OK;
}

}  // namespace

extern "C" {

int slpv_n_params(int32_t nx, int32_t* n_theta)
{
    if (!n_theta || !nx_ok(nx)) return inval("slpv_n_params: nx must be 2, 4, 6 or 8");
    *n_theta = n_params(nx);
    return SPH_OK;
}

int slpv_destroy(slpv_model* m)
{
    if (!m) return SPH_OK;
    cudaFree(m->th);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->thb);
    cudaFree(m->lr_scale);
    cudaFree(m->grad);
    cudaFree(m->scales);
    cudaFree(m->acc_loss);
    cudaFree(m->loss);
    cudaFree(m->t);
    cudaFree(m->part);
    cudaFree(m->xh);
    cudaFree(m->spart);
    cudaFree(m->lb);
    cudaFree(m->lb_count);
    delete m;
    return SPH_OK;
}

int slpv_create(const slpv_config* cfg, slpv_model** out)
{
    if (!cfg || !out) return inval("slpv_create: NULL pointer");
    *out = nullptr;
    if (!nx_ok(cfg->nx) || !(cfg->sigma2 >= 0.0f)) return inval("slpv_create: nx must be 2, 4, 6 or 8, sigma2 >= 0");
    slpv_model* m = new slpv_model;
    m->cfg = *cfg;
    m->N = n_params(cfg->nx);
    const size_t nb = (size_t)m->N * sizeof(float);
    bool ok = cudaMalloc(&m->th, nb) == cudaSuccess && cudaMalloc(&m->m, nb) == cudaSuccess &&
              cudaMalloc(&m->v, nb) == cudaSuccess && cudaMalloc(&m->thb, nb) == cudaSuccess &&
              cudaMalloc(&m->grad, nb) == cudaSuccess && cudaMalloc(&m->lr_scale, sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->scales, 6 * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->acc_loss, sizeof(double)) == cudaSuccess &&
              cudaMalloc(&m->loss, sizeof(double)) == cudaSuccess && cudaMalloc(&m->t, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&m->spart, kStatBlocks * 6 * sizeof(double)) == cudaSuccess;
    if (!ok) {
        slpv_destroy(m);
        return sph::set_last_error(SPH_E_NOMEM, "slpv_create: cudaMalloc failed");
    }
    const float one[6] = {1, 1, 1, 1, 1, 1};
    if (cudaMemset(m->th, 0, nb) != cudaSuccess ||
        cudaMemcpy(m->scales, one, sizeof(one), cudaMemcpyHostToDevice) != cudaSuccess) {
        slpv_destroy(m);
        return sph::set_last_error(SPH_E_CUDA, "slpv_create: initialisation failed");
    }
    *out = m;
    return SPH_OK;
}

int slpv_set_params(slpv_model* m, const float* theta, const float* scales)
{
    if (!m) return inval("slpv_set_params: NULL model");
    if (theta) {
        std::vector<float> h(theta, theta + m->N);
        for (int q = 0; q < m->N; ++q)
            if (q < 2 * (m->cfg.nx + NY) * (m->cfg.nx + NU) && !trainable(q, m->cfg.nx, kStageAll)) h[q] = 0.f;
        SCK(cudaMemcpy(m->th, h.data(), m->N * sizeof(float), cudaMemcpyHostToDevice));
    }
    if (scales) {
        for (int c = 0; c < 6; ++c)
            if (!(scales[c] > 0.0f) || !std::isfinite(scales[c])) return inval("slpv_set_params: scales must be > 0");
        SCK(cudaMemcpy(m->scales, scales, 6 * sizeof(float), cudaMemcpyHostToDevice));
    }
    return SPH_OK;
}

int slpv_get_params(const slpv_model* m, float* theta, float* scales)
{
    if (!m) return inval("slpv_get_params: NULL model");
    if (theta) SCK(cudaMemcpy(theta, m->th, m->N * sizeof(float), cudaMemcpyDeviceToHost));
    if (scales) SCK(cudaMemcpy(scales, m->scales, 6 * sizeof(float), cudaMemcpyDeviceToHost));
    return SPH_OK;
}

int slpv_normalize(slpv_model* m, const float* u, const float* y, int32_t n_traj, int32_t T, void* stream)
{
    int rc = check_data(m, u, n_traj, T);
    if (rc) return rc;
    if (!y) return inval("slpv_normalize: NULL y");
    cudaStream_t st = (cudaStream_t)stream;
    const long long n = (long long)n_traj * T;
    stats_kernel<<<kStatBlocks, kStatThreads, 0, st>>>(u, y, n, m->spart);
    stats_final_kernel<<<1, 32, 0, st>>>(m->spart, kStatBlocks, n, m->scales);
    SCK(cudaGetLastError());
    float h[6];
    SCK(cudaMemcpyAsync(h, m->scales, sizeof(h), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    for (int c = 0; c < 6; ++c)
        if (!(h[c] > 0.0f) || !std::isfinite(h[c])) return inval("slpv_normalize: a channel is identically zero");
    return SPH_OK;
}

int slpv_loss_grad(slpv_model* m, const float* u, const float* y, int32_t n_traj, int32_t T, int32_t stage,
                   double* loss_out, float* grad_out, void* stream)
{
    int rc = check_data(m, u, n_traj, T);
    if (rc) return rc;
    if (!y || !loss_out) return inval("slpv_loss_grad: NULL y or loss_out");
    if (stage < 0 || stage > 2) return inval("slpv_loss_grad: stage must be 0, 1 or 2");
    cudaStream_t st = (cudaStream_t)stream;
    rc = loss_grad_launch(m, u, y, n_traj, T, stage, grad_out, st);
    if (rc) return rc;
    SCK(cudaMemcpyAsync(loss_out, m->loss, sizeof(double), cudaMemcpyDeviceToDevice, st));
    return SPH_OK;
}

int slpv_train(slpv_model* m, const float* u, const float* y, int32_t n_traj, int32_t T, int32_t iters, float lr,
               int32_t stage, double* loss_hist, void* stream)
{
    int rc = check_data(m, u, n_traj, T);
    if (rc) return rc;
    if (!y || iters < 0 || !(lr > 0.0f)) return inval("slpv_train: NULL y, iters < 0 or lr <= 0");
    if (stage < 0 || stage > 2) return inval("slpv_train: stage must be 0, 1 or 2");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nb = (size_t)m->N * sizeof(float);
    const float one = 1.0f;
    const double neg = -1.0;
    SCK(cudaMemsetAsync(m->m, 0, nb, st));
    SCK(cudaMemsetAsync(m->v, 0, nb, st));
    SCK(cudaMemsetAsync(m->t, 0, sizeof(int), st));
    SCK(cudaMemcpyAsync(m->thb, m->th, nb, cudaMemcpyDeviceToDevice, st));
    SCK(cudaMemcpyAsync(m->lr_scale, &one, sizeof(float), cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(m->acc_loss, &neg, sizeof(double), cudaMemcpyHostToDevice, st));
    const int threads = ((m->N + 31) / 32) * 32;
    AdamDev A{m->th, m->m, m->v, m->thb, m->lr_scale, m->acc_loss, m->t};
    for (int it = 0; it < iters; ++it) {
        rc = loss_grad_launch(m, u, y, n_traj, T, stage, m->grad, st);
        if (rc) return rc;
        adam_kernel<<<1, threads, 0, st>>>(A, m->grad, m->loss, loss_hist, it, m->N, lr);
        SCK(cudaGetLastError());
    }
    // end on the last accepted iterate
    SCK(cudaMemcpyAsync(m->th, m->thb, nb, cudaMemcpyDeviceToDevice, st));
    return SPH_OK;
}

int slpv_lbfgs(slpv_model* m, const float* u, const float* y, int32_t n_traj, int32_t T, int32_t iters,
               int32_t stage, double* loss_hist, void* stream)
{
    int rc = check_data(m, u, n_traj, T);
    if (rc) return rc;
    if (!y || iters < 0) return inval("slpv_lbfgs: NULL y or iters < 0");
    if (stage < 0 || stage > 2) return inval("slpv_lbfgs: stage must be 0, 1 or 2");
    cudaStream_t st = (cudaStream_t)stream;
    if (!m->lb) {
        const size_t n = (size_t)kLT * (3 + 2 * kLM) + kLM + 2;
        if (cudaMalloc(&m->lb, n * sizeof(double)) != cudaSuccess || cudaMalloc(&m->lb_count, 2 * sizeof(int)) != cudaSuccess)
            return sph::set_last_error(SPH_E_NOMEM, "slpv_lbfgs: cudaMalloc failed");
        SCK(cudaMemset(m->lb, 0, n * sizeof(double)));
    }
    LbDev L;
    L.W = m->lb;
    L.g = L.W + kLT;
    L.d = L.g + kLT;
    L.S = L.d + kLT;
    L.Y = L.S + (size_t)kLM * kLT;
    L.rho = L.Y + (size_t)kLM * kLT;
    L.gd = L.rho + kLM;
    L.count = m->lb_count;
    L.N = m->N;
    auto eval = [&](bool grad, double* f) -> int {
        int r = loss_grad_launch(m, u, y, n_traj, T, stage, grad ? m->grad : nullptr, st);
        if (r) return r;
        SCK(cudaMemcpyAsync(f, m->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        SCK(cudaStreamSynchronize(st));
        return SPH_OK;
    };
    double f = 0.0;
    if ((rc = eval(true, &f))) return rc;
    if (!std::isfinite(f)) return sph::set_last_error(SPH_E_DIVERGED, "slpv_lbfgs: the loss at the start is not finite");
    lb_init_kernel<<<1, kLT, 0, st>>>(m->th, m->grad, L);
    SCK(cudaGetLastError());
    constexpr double kArmijo = 1e-4;
    int it = 0;
    for (; it < iters; ++it) {
        lb_dir_kernel<<<1, kLT, 0, st>>>(L);
        SCK(cudaGetLastError());
        double gd[2];
        int cnt[2];
        SCK(cudaMemcpyAsync(gd, L.gd, sizeof(gd), cudaMemcpyDeviceToHost, st));
        SCK(cudaMemcpyAsync(cnt, L.count, sizeof(cnt), cudaMemcpyDeviceToHost, st));
        SCK(cudaStreamSynchronize(st));
        if (!(gd[0] < 0.0)) break;  // stationary
        double step = cnt[0] > 0 ? 1.0 : std::min(1.0, 0.01 / std::sqrt(gd[1]));  // after a reset: 0.01 in theta
        bool ok = false;
        double fn = 0.0;
        for (int tries = 0; tries < 40; ++tries) {
            lb_try_kernel<<<1, kLT, 0, st>>>(m->th, L, step);
            SCK(cudaGetLastError());
            if ((rc = eval(false, &fn))) return rc;
            if (std::isfinite(fn) && fn <= f + kArmijo * step * gd[0]) {
                ok = true;
                break;
            }
            step *= 0.5;
        }
        if (!ok) {  // no decrease along d: back to the last accepted point
            lb_try_kernel<<<1, kLT, 0, st>>>(m->th, L, 0.0);
            SCK(cudaGetLastError());
            break;
        }
        if ((rc = eval(true, &fn))) return rc;
        lb_accept_kernel<<<1, kLT, 0, st>>>(m->grad, L, step);
        SCK(cudaGetLastError());
        f = fn;
        if (loss_hist) loss_hist[it] = f;
    }
    if (loss_hist)
        for (int k = it; k < iters; ++k) loss_hist[k] = f;
    SCK(cudaStreamSynchronize(st));
    return SPH_OK;
}

int slpv_init_ls(slpv_model* m, const float* u, const float* y, int32_t n_traj, int32_t T, void* stream)
{
    int rc = check_data(m, u, n_traj, T);
    if (rc) return rc;
    if (!y || T < 2) return inval("slpv_init_ls: NULL y or T < 2");
    if (m->cfg.nx < 3) return inval("slpv_init_ls: the start needs nx >= 3 (the velocities are states)");
    cudaStream_t st = (cudaStream_t)stream;
    constexpr int nblk = 152;
    double* part = nullptr;
    int* status = nullptr;
    SCK(cudaMalloc(&part, (size_t)nblk * kLsVals * sizeof(double)));
    cudaError_t e = cudaMalloc(&status, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(part);
        return sph::set_last_error(SPH_E_NOMEM, "slpv_init_ls: cudaMalloc failed");
    }
    ls_gram_kernel<<<nblk, kLsThreads, 0, st>>>(u, y, m->scales, n_traj, T, part);
    e = by_nx(m->cfg.nx, [&](auto c) {
        constexpr int NX = decltype(c)::value;
        ls_solve_kernel<NX><<<1, 128, 0, st>>>(part, nblk, m->th, status);
        return cudaGetLastError();
    });
    int hs = 1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(part);
    cudaFree(status);
    SCK(e);
    if (hs != 0) return sph::set_last_error(SPH_E_DIVERGED, "slpv_init_ls: the normal equations are singular");
    return SPH_OK;
}

int slpv_predict(const slpv_model* m, const float* u, int32_t n_traj, int32_t T, double Ts, float* vel_out,
                 float* pos_out, void* stream)
{
    int rc = check_data(m, u, n_traj, T);
    if (rc) return rc;
    if (!(Ts > 0.0)) return inval("slpv_predict: Ts must be > 0");
    cudaStream_t st = (cudaStream_t)stream;
    const int threads = 128, blocks = (n_traj + threads - 1) / threads;
    SCK(by_nx(m->cfg.nx, [&](auto c) {
        constexpr int NX = decltype(c)::value;
        predict_kernel<NX><<<blocks, threads, 0, st>>>(m->th, m->scales, u, n_traj, T, (float)Ts, vel_out, pos_out);
        return cudaGetLastError();
    }));
    return SPH_OK;
}

int slpv_simulate(const slpv_model* m, int32_t B, int32_t T, const double* F, const double* tau,
                  const double* theta_ref, double Ts, double J, double omega, double xi, float* out, void* stream)
{
    if (!m || !F || !tau || !theta_ref || !out || B < 1 || T < 1) return inval("slpv_simulate: NULL pointer or empty");
    if (!(Ts > 0.0) || !(J > 0.0)) return inval("slpv_simulate: Ts and J must be > 0");
    cudaStream_t st = (cudaStream_t)stream;
    const int threads = 128, blocks = (B + threads - 1) / threads;
    SCK(by_nx(m->cfg.nx, [&](auto c) {
        constexpr int NX = decltype(c)::value;
        closed_loop_kernel<NX><<<blocks, threads, 0, st>>>(m->th, m->scales, B, T, F, tau, theta_ref, (float)Ts,
                                                           (float)J, (float)omega, (float)xi, out);
        return cudaGetLastError();
    }));
    return SPH_OK;
}

}  // extern "C"
