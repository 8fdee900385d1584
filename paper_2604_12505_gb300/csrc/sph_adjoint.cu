// sph_adjoint.cu -- reverse-mode (adjoint) derivative of one SPH step.
//
// The step (Algorithm 1 + symplectic Euler, Section 3.4) is differentiated
// with the neighbour set of the step frozen, as the forward-mode tangent is.
// For a state before the step (x, v, body) and the adjoint of the state after
// it (x', v', body') plus the adjoints of the step's samples, one reverse step
// produces the adjoint of the state before it and of the step's input u:
//
//   body (kick then drift)   rdot_bar_t = rdot'_bar + dt r'_bar,  F_bar = dt / M rdot_bar_t
//                            (theta likewise with J);  u_bar = (F_bar, T_bar) of the integration
//   fluid (kick then drift)  v_bar = v'_bar + dt x'_bar,  a_bar = dt v_bar,  x_bar = x'_bar
//   force pass (Eqs. 10, 12) for each fluid pair the accelerations contribute
//                            m s_ij (a_bar_i - a_bar_j) . d_ij, symmetric in i and j, so each
//                            particle differentiates it in its own variables over its
//                            neighbours (a gather, like the forward pass)
//   ghost pairs (Eqs. 16-20) f (a_bar_i / m - F_bar) . d - T_bar f (arm x d): into x_bar, v_bar,
//                            q_bar, rho_bar and, through the ghost kinematics (Eq. 21), the body
//   EOS (Eq. 11)             rho_bar += q_bar (k / rho^2 - 2 q / rho),  q = P / rho^2
//   density pass (Eq. 14)    x_bar_i += m (rho_bar_i + rho_bar_j) (dW/dr / r) d_ij, ghosts likewise
//
// Body terms are summed per tile in compensated two-float FP32 and per tank
// in fixed order, so the result is deterministic.  One CTA per tile of 4x4
// cells, staged like the forward pass.
#include <cuda_runtime.h>

#include "sph_common.cuh"
#include "sph_launch.h"
#include "sph_tile.cuh"

namespace sph {

namespace {

constexpr int kAdjCode = 3;  // 4x4 tiles
constexpr int kAdjTX = 4, kAdjTY = 4;

__device__ __forceinline__ F2 shfl_down_f2a(F2 v, int o)
{
    return F2{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}

// Fixed-order block sum of six components (compensated two-float); the
// result is valid in thread 0.
template <int THREADS>
__device__ void block_sum6(F2 (&v)[6])
{
    __shared__ F2 sc[THREADS / 32][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < 6; ++c) v[c] = f2_add(v[c], shfl_down_f2a(v[c], o));
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 6; ++c) sc[warp][c] = v[c];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < THREADS / 32; ++w)
#pragma unroll
            for (int c = 0; c < 6; ++c) v[c] = f2_add(v[c], sc[w][c]);
}

// Per-tile partial of the six body-adjoint components (r_x, r_y, theta,
// rdot_x, rdot_y, thetadot), as (hi, lo) pairs.
template <int THREADS>
__device__ void store_part6(const float (&a)[6], float* out)
{
    F2 v[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) v[c] = F2{a[c], 0.f};
    block_sum6<THREADS>(v);
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            out[2 * c] = v[c].hi;
            out[2 * c + 1] = v[c].lo;
        }
}

}  // namespace

// Body integration adjoint and the step's sample adjoints, one thread per tank (FP64).
__global__ void adj_body_pre_kernel(SimDev S, AdjDev A)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= S.B) return;
    const TankDev& T = S.tank[b];
    const double* bb = A.bbar + 6 * b;
    const double dt = T.dt_d;
    // r' = r + dt rdot', rdot' = rdot + dt (F_b + u) / M (theta likewise)
    const double rdx = bb[3] + dt * bb[0], rdy = bb[4] + dt * bb[1], wd = bb[5] + dt * bb[2];
    double Fx = dt / T.m_body * rdx, Fy = dt / T.m_body * rdy, Tq = dt / T.J_body * wd;
    if (A.ubar) {
        double* ub = A.ubar + b * A.ubar_stride + 3ll * A.k;
        ub[0] = Fx;
        ub[1] = Fy;
        ub[2] = Tq;
    }
    double part[6] = {bb[0], bb[1], bb[2], rdx, rdy, wd};
    float cx = 0.f, cy = 0.f;
    if (A.row >= 0 && A.ybar) {  // samples of this step: body state, F_b, T_b, fluid centre of mass
        const double* y = A.ybar + b * A.ybar_stride + (long long)A.row * SPH_NY;
        for (int q = 0; q < 6; ++q) part[q] += y[q];
        Fx += y[6];
        Fy += y[7];
        Tq += y[8];
        if (T.n_f) {
            cx = (float)(y[9] / T.n_f);
            cy = (float)(y[10] / T.n_f);
        }
    }
    for (int q = 0; q < 6; ++q) A.bbar_part[6 * b + q] = part[q];
    float* fb = A.fbar + 8 * b;
    fb[0] = (float)Fx;
    fb[1] = (float)Fy;
    fb[2] = (float)Tq;
    fb[3] = cx;
    fb[4] = cy;
}

// Adjoint of the force pass, the EOS and the kick-then-drift of the fluid.
template <int TX, int TY>
__global__ void __launch_bounds__(Shape<TX, TY>::THREADS) adj_force_kernel(SimDev S, AdjDev A)
{
    using Sh = Shape<TX, TY>;
    __shared__ Stage<TX, TY, true, false> sm;
    __shared__ float2 sab[Sh::MAXS];  // acceleration adjoint of each staged particle
    const int4 td = S.tiles[blockIdx.x];
    const int tank = td.x;
    const TankDev T = S.tank[tank];
    const int buf = (int)(S.run->step & 1);
    float bacc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (stage_tile<TX, TY, true, false>(S, T, buf, td.y, td.z, sm)) {
        const float dt = T.dt;
        const int total = sm.start[Sh::NC];
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            const float4 a = A.in[sm.pid[e]];
            sab[e] = make_float2(dt * (a.z + dt * a.x), dt * (a.w + dt * a.y));
        }
        __syncthreads();
        const BodyDev& b = S.body[tank];
        const float bc = b.fc, bs = b.fs, brx = b.frx, bry = b.fry, om = b.fw;
        const float* fb = A.fbar + 8 * tank;
        const float Fbx = fb[0], Fby = fb[1], Tbb = fb[2], cmx = fb[3], cmy = fb[4];
        const float m = T.m, mm = T.m * T.m;
        const int n_own = sm.own_row[TY];
        for (int t = threadIdx.x; t < n_own; t += blockDim.x) {
            const int e = own_index(t, sm);
            const float4 pi = sm.pv[e];
            const float2 li = sm.plo[e];
            const float2 ri = sm.rho[e];
            const int id = sm.pid[e];
            const float4 ain = A.in[id];
            const float2 ai = sab[e];
            float xbx = ain.x + cmx, xby = ain.y + cmy;                   // x_bar = x'_bar (+ centre of mass)
            float vbx = ain.z + dt * ain.x, vby = ain.w + dt * ain.y;     // v_bar = v'_bar + dt x'_bar
            float qb = 0.f, rb = 0.f;
            auto pair = [&](int j) {
                const float4 pj = sm.pv[j];
                const float2 d = sep_ff(pi, li, pj, sm.plo[j]);
                const float dx = d.x, dy = d.y;
                const float r2 = dist2(dx, dy);
                if (!(r2 > 0.f)) return;
                const float2 rj = sm.rho[j];
                const float inv_r = rsqrtf(r2), r = r2 * inv_r;
                const float G = dw_cubic_over_r(T, r, inv_r);           // (dW/dr) / r
                const float Gp = dG_cubic_dr(T, r, inv_r, G);           // dG/dr
                const float Bs = ri.x + rj.x, C = r2 + T.epsh2;
                const float ux = pi.z - pj.z, uy = pi.w - pj.w;
                const float vr = ux * dx + uy * dy;
                const float iBC = 1.0f / (Bs * C);
                const float V = T.visc_a * vr * iBC;                     // Eq. 12 factor
                const float S0 = -(ri.y + rj.y) + V;                     // Eq. 10 + 12 bracket
                const float dax = ai.x - sab[j].x, day = ai.y - sab[j].y;
                const float c = dax * dx + day * dy;
                const float mcG = m * c * G;
                qb -= mcG;
                rb -= mcG * V / Bs;
                const float kv = mcG * T.visc_a * iBC;
                vbx += kv * dx;
                vby += kv * dy;
                const float k1 = m * S0 * G, k2 = m * c * S0 * Gp * inv_r;
                const float k3 = m * c * G * T.visc_a * iBC, k4 = 2.0f * vr / C;
                xbx += k1 * dax + k2 * dx + k3 * (ux - k4 * dx);
                xby += k1 * day + k2 * dy + k3 * (uy - k4 * dy);
            };
            if (!for_recorded_neighbours<Sh::MAXOWN>(S, blockIdx.x, t, pair)) {
                const int c = sm.cell[e];
#pragma unroll
                for (int dyc = -1; dyc <= 1; ++dyc) {
                    const int a = sm.start[c + dyc * Sh::SX - 1], zz = sm.start[c + dyc * Sh::SX + 2];
                    for (int j = a; j < zz; ++j) {
                        const float2 d = sep_ff(pi, li, sm.pv[j], sm.plo[j]);
                        if (j != e && dist2(d.x, d.y) < T.R2) pair(j);
                    }
                }
            }
            for_ghosts(S, T, pi.x, pi.y, bc, bs, brx, bry, [&](int g) {
                const float4 gp = S.gpos[g];
                const float2 sg = sep_fg(pi, li, gp);
                const float dx = sg.x, dy = sg.y;
                const float r2 = dist2(dx, dy);
                if (!(r2 < T.h2) || !(r2 > 0.f)) return;
                const float4 gv = S.gvel[g];                             // (v_g, arm)
                const float inv_r = rsqrtf(r2), r = r2 * inv_r;
                const float d = T.h - r;
                const float Gs = T.cdS * d * d * inv_r;                  // (dW_s/dr) / r
                const float Gsp = -T.cdS * d * (T.h + r) * inv_r * inv_r; // dGs/dr
                const float Cp = T.gp_sign * 2.0f * mm;
                const float qg = T.gp_clamp ? fmaxf(ri.y, 0.f) : ri.y;   // clamped P_i / rho_i^2
                const float fp = Cp * qg * Gs;                           // Eq. 16
                const float ux = pi.z - gv.x, uy = pi.w - gv.y;
                const float vr = ux * dx + uy * dy;
                const float C = r2 + T.epsh2;
                const float cv = mm * T.beta2 / ((ri.x + ri.x) * C);
                const float mv = fminf(vr, 0.f);
                const float fv = cv * mv * Gs;                           // Eq. 18
                const float f = fp + fv;
                const float ex = ai.x * T.inv_m - Fbx, ey = ai.y * T.inv_m - Fby;
                const float cross = gv.z * dy - gv.w * dx;               // (arm x d)_z
                const float kap = ex * dx + ey * dy - Tbb * cross;
                if (qg == ri.y) qb += kap * Cp * Gs;
                rb -= kap * fv / ri.x;
                const float neg = (vr < 0.f) ? 1.0f : 0.0f;
                const float kvi = kap * neg * cv * Gs;
                vbx += kvi * dx;
                vby += kvi * dy;
                const float kd = Cp * qg * Gsp * inv_r + cv * mv * (Gsp * inv_r - 2.0f * Gs / C);
                const float dfx = kd * dx + neg * cv * Gs * ux, dfy = kd * dy + neg * cv * Gs * uy;
                const float dbx = kap * dfx + f * (ex + Tbb * gv.w), dby = kap * dfy + f * (ey - Tbb * gv.z);
                xbx += dbx;
                xby += dby;
                // Eq. 21: g_w = r + arm, v_g = rdot + thetadot z x arm, arm = R(theta) g_B
                const float gwx = -dbx, gwy = -dby;                      // ghost position adjoint
                const float vgx = -kvi * dx, vgy = -kvi * dy;            // ghost velocity adjoint
                bacc[0] += gwx;
                bacc[1] += gwy;
                bacc[2] += gwy * gv.z - gwx * gv.w - om * (vgx * gv.z + vgy * gv.w) + Tbb * f * (dx * gv.z + dy * gv.w);
                bacc[3] += vgx;
                bacc[4] += vgy;
                bacc[5] += vgy * gv.z - vgx * gv.w;
            });
            A.out[id] = make_float4(xbx, xby, vbx, vby);
            A.rhobar[id] = rb + qb * (T.k / (ri.x * ri.x) - 2.0f * ri.y / ri.x);  // Eq. 11 with q = P / rho^2
        }
    }
    store_part6<Sh::THREADS>(bacc, A.part + (size_t)blockIdx.x * 12);
}

// Adjoint of the density pass (Eq. 14) with the density adjoint of the EOS.
template <int TX, int TY>
__global__ void __launch_bounds__(Shape<TX, TY>::THREADS) adj_density_kernel(SimDev S, AdjDev A)
{
    using Sh = Shape<TX, TY>;
    __shared__ Stage<TX, TY, false, false> sm;
    __shared__ float srb[Sh::MAXS];  // density adjoint of each staged particle
    const int4 td = S.tiles[blockIdx.x];
    const int tank = td.x;
    const TankDev T = S.tank[tank];
    const int buf = (int)(S.run->step & 1);
    float bacc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (stage_tile<TX, TY, false, false>(S, T, buf, td.y, td.z, sm)) {
        const int total = sm.start[Sh::NC];
        for (int e = threadIdx.x; e < total; e += blockDim.x) srb[e] = A.rhobar[sm.pid[e]];
        __syncthreads();
        const BodyDev& b = S.body[tank];
        const float bc = b.fc, bs = b.fs, brx = b.frx, bry = b.fry;
        const float m = T.m, mg = T.m * T.gamma1;
        const int n_own = sm.own_row[TY];
        for (int t = threadIdx.x; t < n_own; t += blockDim.x) {
            const int e = own_index(t, sm);
            const float4 pi = sm.pv[e];
            const float2 li = sm.plo[e];
            const float rbi = srb[e];
            float xbx = 0.f, xby = 0.f;
            auto pair = [&](int j) {
                const float4 pj = sm.pv[j];
                const float2 d = sep_ff(pi, li, pj, sm.plo[j]);
                const float dx = d.x, dy = d.y;
                const float r2 = dist2(dx, dy);
                if (!(r2 > 0.f)) return;
                const float inv_r = rsqrtf(r2), r = r2 * inv_r;
                const float k = m * (rbi + srb[j]) * dw_cubic_over_r(T, r, inv_r);
                xbx += k * dx;
                xby += k * dy;
            };
            if (!for_recorded_neighbours<Sh::MAXOWN>(S, blockIdx.x, t, pair)) {
                const int c = sm.cell[e];
#pragma unroll
                for (int dyc = -1; dyc <= 1; ++dyc) {
                    const int a = sm.start[c + dyc * Sh::SX - 1], zz = sm.start[c + dyc * Sh::SX + 2];
                    for (int j = a; j < zz; ++j) {
                        const float2 d = sep_ff(pi, li, sm.pv[j], sm.plo[j]);
                        if (j != e && dist2(d.x, d.y) < T.R2) pair(j);
                    }
                }
            }
            for_ghosts(S, T, pi.x, pi.y, bc, bs, brx, bry, [&](int g) {
                const float4 gp = S.gpos[g];
                const float2 d = sep_fg(pi, li, gp);
                const float dx = d.x, dy = d.y;
                const float r2 = dist2(dx, dy);
                if (!(r2 < T.R2) || !(r2 > 0.f)) return;
                const float4 gv = S.gvel[g];
                const float inv_r = rsqrtf(r2), r = r2 * inv_r;
                const float k = mg * rbi * dw_cubic_over_r(T, r, inv_r);
                xbx += k * dx;
                xby += k * dy;
                const float gwx = -k * dx, gwy = -k * dy;  // ghost position adjoint, Eq. 21
                bacc[0] += gwx;
                bacc[1] += gwy;
                bacc[2] += gwy * gv.z - gwx * gv.w;
            });
            const int id = sm.pid[e];
            float4 o = A.out[id];
            o.x += xbx;
            o.y += xby;
            A.out[id] = o;
        }
    }
    store_part6<Sh::THREADS>(bacc, A.part + ((size_t)A.max_tiles + blockIdx.x) * 12);
}

// Body adjoint of the state before the step: the integration part plus the
// ghost terms of both passes, summed over the tank's tiles in fixed order.
__global__ void __launch_bounds__(128) adj_body_post_kernel(SimDev S, AdjDev A)
{
    const int b = blockIdx.x;
    const int t0 = S.tile_tank_first[b], t1 = S.tile_tank_first[b + 1];
    F2 v[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) v[c] = F2{0.f, 0.f};
    for (int p = 0; p < 2; ++p)
        for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
            const float* P = A.part + ((size_t)p * A.max_tiles + t) * 12;
#pragma unroll
            for (int c = 0; c < 6; ++c) v[c] = f2_add(v[c], F2{P[2 * c], P[2 * c + 1]});
        }
    block_sum6<128>(v);
    if (threadIdx.x == 0)
        for (int c = 0; c < 6; ++c) A.bbar[6 * b + c] = A.bbar_part[6 * b + c] + ((double)v[c].hi + (double)v[c].lo);
}

__global__ void set_step_kernel(RunDev* run, long long step)
{
    run->step = step;
    run->step0 = step;
    run->tanks_done = 0;
    run->next_buf = (int)(step & 1);
}

cudaError_t launch_set_step(RunDev* run, long long step, cudaStream_t st)
{
    set_step_kernel<<<1, 1, 0, st>>>(run, step);
    return cudaGetLastError();
}

int adjoint_tile_code() { return kAdjCode; }

// One reverse step on the state set in the grid (S built for the 4x4 tiles).
cudaError_t launch_adjoint_step(const SimDev& S, const AdjDev& A, int n_tiles, cudaStream_t st)
{
    using Sh = Shape<kAdjTX, kAdjTY>;
    adj_body_pre_kernel<<<(S.B + 127) / 128, 128, 0, st>>>(S, A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    EvalOut E{};
    e = launch_phase(S, E, 0, kAdjCode, n_tiles, 0, st, false);  // primal density pass of this state
    if (e != cudaSuccess) return e;
    adj_force_kernel<kAdjTX, kAdjTY><<<n_tiles, Sh::THREADS, 0, st>>>(S, A);
    adj_density_kernel<kAdjTX, kAdjTY><<<n_tiles, Sh::THREADS, 0, st>>>(S, A);
    adj_body_post_kernel<<<S.B, 128, 0, st>>>(S, A);
    return cudaGetLastError();
}

}  // namespace sph
