// lpv_kernels.cu -- tensor-core kernels of the LPV surrogate (Section 4).
//
// One warp carries 16 trajectories through the recurrence
//     [x_{k+1}; y_k] = W w_k,   w_k = [z_k; p_1 z_k; p_2 z_k],  z_k = [x_k; u_k; 0]
// as one mma.sync.m16n8k16 (BF16 in, FP32 accumulate) product per 16x16x8
// tile.  Each operand is split into two BF16 halves (v = hi + lo) and the
// product is hi*hi + hi*lo + lo*hi, which keeps about 16 significant bits
// per half: a recurrent state rounded to plain BF16 every step would drift.
//
// Register layouts (PTX m16n8k16, groupID g = lane / 4, t = lane % 4):
//   A 16x16: rows g, g+8; columns 2t, 2t+1, 2t+8, 2t+9
//   D 16x8 : rows g, g+8; columns 2t, 2t+1 (of the n-tile)
// With features ordered [x (n_x), u (n_u), 0...] in each 16-column block and
// outputs ordered [x_next (n_x), y (n_y), 0...], the accumulator of n-tiles
// 0 and 1 holds exactly the entries of the next step's first A block that
// this thread owns, and the scheduled blocks p_i z are thread-local scalings:
// the recurrence runs without shuffles.  The backward pass uses the same
// identity for the adjoint; the weight gradient sum_k G_k^T w_k is one more
// MMA whose operands are transposed through a per-warp shared-memory tile.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lpv_common.cuh"
#include "lpv_launch.h"

namespace lpv {

constexpr int kPrefetch = 4;  // steps of inputs in flight in the recurrences

__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// (v0, v1) -> packed bf16x2 (v0 in the low half), split into hi and lo parts.
__device__ __forceinline__ void split2(float v0, float v1, uint32_t& hi, uint32_t& lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// A fragment from the 8 values s[] a thread owns (see layout above).
__device__ __forceinline__ void afrag(const float* s, uint32_t* hi, uint32_t* lo)
{
    split2(s[0], s[1], hi[0], lo[0]);
    split2(s[2], s[3], hi[1], lo[1]);
    split2(s[4], s[5], hi[2], lo[2]);
    split2(s[6], s[7], hi[3], lo[3]);
}

// Column and row (0: g, 1: g + 8) of the thread's value s[i].
__device__ __forceinline__ int scol(int i, int t) { return ((i < 4) ? 2 * t : 8 + 2 * t) + (i & 1); }
__device__ __forceinline__ int srow(int i) { return (i >> 1) & 1; }

// d[8] += A[kt] B for the split operands: three independent accumulation
// chains (hi.hi, hi.lo, lo.hi) over the k-tiles, summed at the end.
template <int NKT>
__device__ __forceinline__ void mma_split(float* d, const uint32_t (*ahi)[4], const uint32_t (*alo)[4],
                                          const uint32_t (*bhi)[2][2], const uint32_t (*blo)[2][2], int nkt)
{
    float c1[8] = {0, 0, 0, 0, 0, 0, 0, 0}, c2[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int kt = 0; kt < NKT; ++kt) {
        if (kt >= nkt) break;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            mma16816(d + 4 * nt, ahi[kt], bhi[kt][nt][0], bhi[kt][nt][1]);
            mma16816(c1 + 4 * nt, ahi[kt], blo[kt][nt][0], blo[kt][nt][1]);
            mma16816(c2 + 4 * nt, alo[kt], bhi[kt][nt][0], bhi[kt][nt][1]);
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) d[i] += c1[i] + c2[i];
}

}  // namespace lpv

namespace lpv {

// B fragments of the forward product D[row][o] = sum_f w[row][f] Wp[o][f].
__device__ __forceinline__ void load_fwd_frags(const float* __restrict__ Wp, uint32_t (*bhi)[2][2],
                                               uint32_t (*blo)[2][2], int nkt, int g, int t)
{
#pragma unroll
    for (int kt = 0; kt < kMaxKT; ++kt) {
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const float* w = Wp + (nt * 8 + g) * (kFB * kMaxKT) + kt * kFB;
            if (kt < nkt) {
                split2(w[2 * t], w[2 * t + 1], bhi[kt][nt][0], blo[kt][nt][0]);
                split2(w[8 + 2 * t], w[9 + 2 * t], bhi[kt][nt][1], blo[kt][nt][1]);
            } else {
                bhi[kt][nt][0] = bhi[kt][nt][1] = blo[kt][nt][0] = blo[kt][nt][1] = 0u;
            }
        }
    }
}

// Scheduling variables of the thread's two trajectories at step k, normalised.
__device__ __forceinline__ void load_p(const Dims& d, const float* __restrict__ p, int r, bool valid, int T, int k,
                                       float* pp)
{
    const size_t o = ((size_t)r * T + k) * d.np;
    pp[0] = (valid && d.np > 0) ? (p[o] - d.pm[0]) * d.inv_ps[0] : 0.f;
    pp[1] = (valid && d.np > 1) ? (p[o + 1] - d.pm[1]) * d.inv_ps[1] : 0.f;
}

// Inputs of one step that a thread owns: the scheduling of its two
// trajectories and its feature (u) and output (y) columns, normalised.
struct StepIn {
    float p0[2], p1[2];
    float uz[8];  // u part of z at the thread's 8 columns (0 elsewhere)
    float yv[8];  // y at the thread's output columns (0 elsewhere; loss only)
};

template <bool WANT_Y>
__device__ __forceinline__ void load_step(const Dims& d, const float* __restrict__ u, const float* __restrict__ p,
                                          const float* __restrict__ y, int r0, int r1, bool v0, bool v1, int T, int k,
                                          int t, StepIn& in)
{
    load_p(d, p, r0, v0, T, k, in.p0);
    load_p(d, p, r1, v1, T, k, in.p1);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int c = scol(i, t);
        const int r = srow(i) ? r1 : r0;
        const bool v = srow(i) ? v1 : v0;
        in.uz[i] = (v && c >= d.nx && c < d.nx + d.nu)
                       ? u[((size_t)r * T + k) * d.nu + (c - d.nx)] * d.inv_su[c - d.nx] : 0.f;
        in.yv[i] = (WANT_Y && v && c >= d.nx && c < d.nx + d.ny)
                       ? y[((size_t)r * T + k) * d.ny + (c - d.nx)] * d.inv_sy[c - d.nx] : 0.f;
    }
}

// Free-run simulation of 16 trajectories per warp.  MODE 0 writes the
// prediction (physical units); MODE 1 accumulates the squared error of the
// normalised outputs and records, per step, x_k and dJ/dy_k for the
// backward pass in hist[traj][k][16] (state columns, then output columns).
// The inputs of steps k + 1 .. k + kPrefetch are in flight while step k's products run.
template <int MODE>
__global__ void __launch_bounds__(128) fwd_kernel(const float* __restrict__ Wp, Dims d, const float* __restrict__ u,
                                                  const float* __restrict__ p, const float* __restrict__ y, int n_traj,
                                                  int T, float* __restrict__ y_out, float* __restrict__ hist,
                                                  double* __restrict__ loss_part, float grad_scale)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int r0 = wid * 16 + g, r1 = r0 + 8;
    const bool v0 = r0 < n_traj, v1 = r1 < n_traj;
    uint32_t bhi[kMaxKT][2][2], blo[kMaxKT][2][2];
    load_fwd_frags(Wp, bhi, blo, d.nkt, g, t);
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // x_0 = 0
    float lsum_f = 0.f;                     // widened to FP64 once, after the loop
    // a ring of the inputs of the next kPrefetch steps: the loads of step
    // k + kPrefetch are issued when step k starts, so a step waits on no
    // global load issued less than kPrefetch steps before it
    StepIn ring[kPrefetch];
#pragma unroll
    for (int i = 0; i < kPrefetch; ++i)
        load_step<MODE == 1>(d, u, p, y, r0, r1, v0, v1, T, i < T ? i : T - 1, t, ring[i]);
    for (int k0 = 0; k0 < T; k0 += kPrefetch) {
#pragma unroll
    for (int i = 0; i < kPrefetch; ++i) {
        const int k = k0 + i;
        if (k >= T) break;
        const StepIn cur = ring[i];
        load_step<MODE == 1>(d, u, p, y, r0, r1, v0, v1, T, k + kPrefetch < T ? k + kPrefetch : T - 1, t, ring[i]);
        float z[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) z[i] = (scol(i, t) < d.nx) ? s[i] : cur.uz[i];
        uint32_t ahi[kMaxKT][4], alo[kMaxKT][4];
        afrag(z, ahi[0], alo[0]);
#pragma unroll
        for (int kt = 1; kt < kMaxKT; ++kt) {
            float zs[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) zs[i] = z[i] * (srow(i) ? cur.p1[kt - 1] : cur.p0[kt - 1]);
            afrag(zs, ahi[kt], alo[kt]);
        }
        float D[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        mma_split<kMaxKT>(D, ahi, alo, bhi, blo, d.nkt);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c = scol(i, t);
            const int r = srow(i) ? r1 : r0;
            const bool v = srow(i) ? v1 : v0;
            if (c < d.nx) {
                if (MODE == 1 && v) hist[((size_t)r * T + k) * 16 + c] = s[i];
            } else if (c < d.nx + d.ny && v) {
                const int q = c - d.nx;
                if (MODE == 0) {
                    y_out[((size_t)r * T + k) * d.ny + q] = D[i] * d.sy[q];
                } else {
                    const float res = D[i] - cur.yv[i];
                    lsum_f = fmaf(res, res, lsum_f);
                    hist[((size_t)r * T + k) * 16 + c] = grad_scale * res;
                }
            }
            s[i] = (c < d.nx) ? D[i] : 0.f;
        }
    }
    }
    if (MODE == 1) {
        double lsum = (double)lsum_f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
        if (lane == 0) loss_part[wid] = lsum;
    }
}

template __global__ void fwd_kernel<0>(const float*, Dims, const float*, const float*, const float*, int, int, float*,
                                       float*, double*, float);
template __global__ void fwd_kernel<1>(const float*, Dims, const float*, const float*, const float*, int, int, float*,
                                       float*, double*, float);

// B fragments of the adjoint product gw[row][f] = sum_o G[row][o] Wp[o][f]
// (k = output o, n = feature f; six n-tiles cover the 48 padded features).
__device__ __forceinline__ void load_bwd_frags(const float* __restrict__ Wp, uint32_t (*bhi)[2], uint32_t (*blo)[2],
                                               int g, int t)
{
    constexpr int ld = kFB * kMaxKT;
#pragma unroll
    for (int nt = 0; nt < 6; ++nt) {
        const int f = nt * 8 + g;
        split2(Wp[(2 * t) * ld + f], Wp[(2 * t + 1) * ld + f], bhi[nt][0], blo[nt][0]);
        split2(Wp[(8 + 2 * t) * ld + f], Wp[(9 + 2 * t) * ld + f], bhi[nt][1], blo[nt][1]);
    }
}

// Backpropagation through time for 16 trajectories per warp, k = T-1 .. 0:
//   G_k = [lambda_{k+1}; dJ/dy_k],  gw_k = G_k W,
//   lambda_k = gw_k[x] + sum_i p_{k,i} gw_k[block i, x],
//   dJ/dW += G_k^T w_k  (tensor cores, operands transposed in shared memory).
// Each warp writes its partial gradient gpart[warp][16][48].
constexpr int kBwdWarps = 4;

__global__ void __launch_bounds__(32 * kBwdWarps) bwd_kernel(const float* __restrict__ Wp, Dims d,
                                                             const float* __restrict__ u, const float* __restrict__ p,
                                                             int n_traj, int T, const float* __restrict__ hist,
                                                             float* __restrict__ gpart)
{
    __shared__ float sG[kBwdWarps][16][17];
    __shared__ float sZ[kBwdWarps][16][kFB * kMaxKT + 1];
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, wl = threadIdx.x >> 5;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int r0 = wid * 16 + g, r1 = r0 + 8;
    const bool v0 = r0 < n_traj, v1 = r1 < n_traj;
    uint32_t bhi[6][2], blo[6][2];
    load_bwd_frags(Wp, bhi, blo, g, t);
    float lam[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // lambda_T = 0
    float gacc[6][4];
#pragma unroll
    for (int nt = 0; nt < 6; ++nt) gacc[nt][0] = gacc[nt][1] = gacc[nt][2] = gacc[nt][3] = 0.f;
    // step inputs: scheduling, recorded history (x_k | dJ/dy_k) and u
    auto fetch = [&](int k, float* pa0, float* pa1, float* hv, float* uz) {
        load_p(d, p, r0, v0, T, k, pa0);
        load_p(d, p, r1, v1, T, k, pa1);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c = scol(i, t);
            const int r = srow(i) ? r1 : r0;
            const bool v = srow(i) ? v1 : v0;
            hv[i] = (v && c < d.nx + d.ny) ? hist[((size_t)r * T + k) * 16 + c] : 0.f;
            uz[i] = (v && c >= d.nx && c < d.nx + d.nu)
                        ? u[((size_t)r * T + k) * d.nu + (c - d.nx)] * d.inv_su[c - d.nx] : 0.f;
        }
    };
    // a ring of the inputs of the next kPrefetch steps (backwards in k), as in
    // the forward pass
    float rp0[kPrefetch][2], rp1[kPrefetch][2], rhv[kPrefetch][8], ruz[kPrefetch][8];
#pragma unroll
    for (int i = 0; i < kPrefetch; ++i) fetch(T - 1 - i >= 0 ? T - 1 - i : 0, rp0[i], rp1[i], rhv[i], ruz[i]);
    for (int k0 = T - 1; k0 >= 0; k0 -= kPrefetch) {
#pragma unroll
    for (int ri = 0; ri < kPrefetch; ++ri) {
        const int k = k0 - ri;
        if (k < 0) break;
        float chv[8], cuz[8];
        const float pp0[2] = {rp0[ri][0], rp0[ri][1]}, pp1[2] = {rp1[ri][0], rp1[ri][1]};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            chv[i] = rhv[ri][i];
            cuz[i] = ruz[ri][i];
        }
        fetch(k - kPrefetch >= 0 ? k - kPrefetch : 0, rp0[ri], rp1[ri], rhv[ri], ruz[ri]);
        float G[8], z[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c = scol(i, t);
            G[i] = (c < d.nx) ? lam[i] : chv[i];
            z[i] = (c < d.nx) ? chv[i] : cuz[i];  // x_k, u_k, 0
        }
        // gw = G W
        uint32_t ghi[4], glo[4];
        afrag(G, ghi, glo);
        float gw[6][4];
#pragma unroll
        for (int nt = 0; nt < 6; ++nt) {
            float c1[4] = {0, 0, 0, 0}, c2[4] = {0, 0, 0, 0};
            gw[nt][0] = gw[nt][1] = gw[nt][2] = gw[nt][3] = 0.f;
            mma16816(gw[nt], ghi, bhi[nt][0], bhi[nt][1]);
            mma16816(c1, ghi, blo[nt][0], blo[nt][1]);
            mma16816(c2, glo, bhi[nt][0], bhi[nt][1]);
#pragma unroll
            for (int q = 0; q < 4; ++q) gw[nt][q] += c1[q] + c2[q];
        }
        // lambda_k
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c = scol(i, t);
            const int nt0 = (i < 4) ? 0 : 1, q = i & 3;
            const float* pr = srow(i) ? pp1 : pp0;
            float l = gw[nt0][q];
            if (d.np > 0) l += pr[0] * gw[nt0 + 2][q];
            if (d.np > 1) l += pr[1] * gw[nt0 + 4][q];
            lam[i] = (c < d.nx) ? l : 0.f;
        }
        // dJ/dW += G^T w: stage G and w in shared memory, read them transposed
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c = scol(i, t), rl = srow(i) ? g + 8 : g;
            const float* pr = srow(i) ? pp1 : pp0;
            sG[wl][rl][c] = G[i];
            sZ[wl][rl][c] = z[i];
            sZ[wl][rl][kFB + c] = d.np > 0 ? z[i] * pr[0] : 0.f;
            sZ[wl][rl][2 * kFB + c] = d.np > 1 ? z[i] * pr[1] : 0.f;
        }
        __syncwarp();
        float a[8] = {sG[wl][2 * t][g],     sG[wl][2 * t + 1][g],     sG[wl][2 * t][g + 8],     sG[wl][2 * t + 1][g + 8],
                      sG[wl][2 * t + 8][g], sG[wl][2 * t + 9][g],     sG[wl][2 * t + 8][g + 8], sG[wl][2 * t + 9][g + 8]};
        uint32_t ahi[4], alo[4];
        afrag(a, ahi, alo);
#pragma unroll
        for (int nt = 0; nt < 6; ++nt) {
            const int f = nt * 8 + g;
            uint32_t b0h, b0l, b1h, b1l;
            split2(sZ[wl][2 * t][f], sZ[wl][2 * t + 1][f], b0h, b0l);
            split2(sZ[wl][2 * t + 8][f], sZ[wl][2 * t + 9][f], b1h, b1l);
            mma16816(gacc[nt], ahi, b0h, b1h);
            mma16816(gacc[nt], ahi, b0l, b1l);
            mma16816(gacc[nt], alo, b0h, b1h);
        }
        __syncwarp();
    }
    }
    // gacc[nt]: (o = g, f = 8 nt + 2t), (g, +1), (g + 8, 2t), (g + 8, 2t + 1)
    float* out = gpart + (size_t)wid * kWN;
    constexpr int ld = kFB * kMaxKT;
#pragma unroll
    for (int nt = 0; nt < 6; ++nt) {
        const int f = nt * 8 + 2 * t;
        out[g * ld + f] = gacc[nt][0];
        out[g * ld + f + 1] = gacc[nt][1];
        out[(g + 8) * ld + f] = gacc[nt][2];
        out[(g + 8) * ld + f + 1] = gacc[nt][3];
    }
}

// Value D[i] of the lane owning output column c of row rsel (0: g, 1: g + 8).
__device__ __forceinline__ float quad_get(const float* D, int c, int rsel, int g)
{
    const int tc = (c < 8) ? (c >> 1) : ((c - 8) >> 1);
    const int ic = ((c < 8) ? 0 : 4) + (c & 1) + 2 * rsel;
    float v = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        if (j == ic) v = D[j];
    return __shfl_sync(0xffffffffu, v, g * 4 + tc);
}

struct BodyPar {
    float inv_m, inv_J, dt;      // substep dt = Ts / n_sub
    float n, n_half;             // n_sub and n_sub (n_sub + 1) / 2
    float kp, kd;                // PD gains J w^2 and 2 xi J w
};

// Closed loop of 16 runs per warp (Sections 5.1.1, 5.4): per period the PD
// torque (Eq. 28, zero-order hold), the surrogate step with p = [fill,
// thetadot], and n_sub kick-then-drift substeps of the body under the held
// forces, summed in closed form: v += n dt a, x += n dt v + dt^2 a n(n+1)/2.
// The body state (FP32) is replicated in the four lanes of each row group.
__global__ void __launch_bounds__(128, 4) closed_loop_kernel(const float* __restrict__ Wp, Dims d, int B, int T,
                                                          const double* __restrict__ F, const double* __restrict__ tau,
                                                          const double* __restrict__ ref,
                                                          const double* __restrict__ fill, BodyPar bp,
                                                          double* __restrict__ out)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int rr[2] = {wid * 16 + g, wid * 16 + g + 8};
    const bool vv[2] = {rr[0] < B, rr[1] < B};
    uint32_t bhi[kMaxKT][2][2], blo[kMaxKT][2][2];
    load_fwd_frags(Wp, bhi, blo, d.nkt, g, t);
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    float bs[2][6] = {{0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 0, 0}};  // r_x r_y theta v_x v_y omega
    const float fl[2] = {vv[0] ? (float)fill[rr[0]] : 0.f, vv[1] ? (float)fill[rr[1]] : 0.f};
    // inputs of a period (F_x, F_y, tau, theta_ref) for the two rows; those of
    // period k + 1 are loaded while period k runs
    auto fetch = [&](int k, float (*in)[4]) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const size_t o = (size_t)rr[q] * T + k;
            in[q][0] = vv[q] ? (float)F[2 * o] : 0.f;
            in[q][1] = vv[q] ? (float)F[2 * o + 1] : 0.f;
            in[q][2] = vv[q] ? (float)tau[o] : 0.f;
            in[q][3] = vv[q] ? (float)ref[o] : 0.f;
        }
    };
    float cin[2][4];
    fetch(0, cin);
    for (int k = 0; k < T; ++k) {
        float nin[2][4];
        fetch(k + 1 < T ? k + 1 : k, nin);
        float uu[2][3], pp[2][2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const size_t o = (size_t)rr[q] * T + k;
            if (vv[q] && t == 0) {
#pragma unroll
                for (int j = 0; j < 6; ++j) out[o * 6 + j] = bs[q][j];
            }
            const float tc = vv[q] ? bp.kp * (cin[q][3] - bs[q][2]) - bp.kd * bs[q][5] : 0.f;
            uu[q][0] = cin[q][0];
            uu[q][1] = cin[q][1];
            uu[q][2] = vv[q] ? cin[q][2] + tc : 0.f;
            // scheduling clamped to the range it was identified on
            pp[q][0] = d.np > 0 ? (fminf(fmaxf(fl[q], d.plo[0]), d.phi[0]) - d.pm[0]) * d.inv_ps[0] : 0.f;
            pp[q][1] = d.np > 1 ? (fminf(fmaxf(bs[q][5], d.plo[1]), d.phi[1]) - d.pm[1]) * d.inv_ps[1] : 0.f;
        }
        float z[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c = scol(i, t), q = srow(i);
            z[i] = (c < d.nx) ? s[i] : (c < d.nx + d.nu) ? uu[q][c - d.nx] * d.inv_su[c - d.nx] : 0.f;
        }
        uint32_t ahi[kMaxKT][4], alo[kMaxKT][4];
        afrag(z, ahi[0], alo[0]);
#pragma unroll
        for (int kt = 1; kt < kMaxKT; ++kt) {
            float zs[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) zs[i] = z[i] * pp[srow(i)][kt - 1];
            afrag(zs, ahi[kt], alo[kt]);
        }
        float D[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        mma_split<kMaxKT>(D, ahi, alo, bhi, blo, d.nkt);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            // sloshing loads: the first three outputs, in physical units
            const float Fx = quad_get(D, d.nx, q, g) * d.sy[0];
            const float Fy = quad_get(D, d.nx + 1, q, g) * d.sy[1];
            const float Tb = quad_get(D, d.nx + 2, q, g) * d.sy[2];
            const float ax = (uu[q][0] + Fx) * bp.inv_m, ay = (uu[q][1] + Fy) * bp.inv_m;
            const float aw = (uu[q][2] + Tb) * bp.inv_J;
            const float ndt = bp.n * bp.dt, hdt2 = bp.n_half * bp.dt * bp.dt;
            bs[q][0] += ndt * bs[q][3] + hdt2 * ax;
            bs[q][1] += ndt * bs[q][4] + hdt2 * ay;
            bs[q][2] += ndt * bs[q][5] + hdt2 * aw;
            bs[q][3] += ndt * ax;
            bs[q][4] += ndt * ay;
            bs[q][5] += ndt * aw;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) s[i] = (scol(i, t) < d.nx) ? D[i] : 0.f;
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int j = 0; j < 4; ++j) cin[q][j] = nin[q][j];
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_forward(int mode, const float* Wp, const Dims& d, const float* u, const float* p, const float* y,
                           int n_traj, int T, float* y_out, float* hist, double* loss_part, float grad_scale,
                           cudaStream_t st)
{
    const int warps = warps_for(n_traj), blocks = (warps + 3) / 4;
    if (mode == 0)
        fwd_kernel<0><<<blocks, 128, 0, st>>>(Wp, d, u, p, y, n_traj, T, y_out, hist, loss_part, grad_scale);
    else
        fwd_kernel<1><<<blocks, 128, 0, st>>>(Wp, d, u, p, y, n_traj, T, y_out, hist, loss_part, grad_scale);
    return cudaGetLastError();
}

cudaError_t launch_backward(const float* Wp, const Dims& d, const float* u, const float* p, int n_traj, int T,
                            const float* hist, float* gpart, cudaStream_t st)
{
    const int warps = warps_for(n_traj), blocks = (warps + kBwdWarps - 1) / kBwdWarps;
    bwd_kernel<<<blocks, 32 * kBwdWarps, 0, st>>>(Wp, d, u, p, n_traj, T, hist, gpart);
    return cudaGetLastError();
}

cudaError_t launch_closed_loop(const float* Wp, const Dims& d, int B, int T, const double* F, const double* tau,
                               const double* ref, const double* fill, const BodyParHost& h, double* out,
                               cudaStream_t st)
{
    const int warps = warps_for(B), blocks = (warps + 3) / 4;
    BodyPar bp{h.inv_m, h.inv_J, h.dt, h.n, h.n_half, h.kp, h.kd};
    closed_loop_kernel<<<blocks, 128, 0, st>>>(Wp, d, B, T, F, tau, ref, fill, bp, out);
    return cudaGetLastError();
}

}  // namespace lpv
