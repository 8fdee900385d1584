// sph_kernels.cu -- the per-step kernels of the SPH sloshing simulator.
//
// One inner step (Algorithm 1 + symplectic Euler, Section 3.4) is two
// launches over all tanks of a batch, chained by programmatic dependent
// launch (each kernel lets its successor be scheduled at once and waits for
// its predecessor only before touching data the predecessor writes):
//   density_kernel  Eq. 21 for the ghosts each particle meets (two-float
//                   arithmetic on the FP32 pipe), Eqs. 14 and 11 (+ the
//                   continuity sum): one CTA per tile of TX x TY grid cells;
//                   the tile plus a one-cell halo is staged in shared memory,
//                   each cell ordered by x (then particle index), and every own
//                   particle sums over its 3x3 cells, each row clipped in x to
//                   the part that can lie within the support.
//   force_kernel    Eqs. 10, 12 (fluid pairs), 16-19 (ghost pairs), the fluid
//                   acceleration of Algorithm 1, kick-then-drift of the fluid,
//                   and the re-binning of the moved particle into the other
//                   grid buffer.  Per-tile compensated force/torque partials;
//                   the last CTA of a tank reduces them in fixed order,
//                   assembles them in FP64 and integrates the FP64 body
//                   (Eq. 20), samples outputs and runs the PD law (Eq. 28).
// No warp-wide FP64 arithmetic runs in the tile kernels: this GPU's FP64
// pipe issues a warp instruction in about 16 cycles per SM.
#include <algorithm>
#include <cfloat>
#include <climits>

#include "sph_common.cuh"
#include "sph_launch.h"
#include <type_traits>
#include "sph_tile.cuh"

namespace sph {

// ---------------------------------------------------------------------------
// Density pass: Eqs. 14, 11 (+ continuity sum)
// ---------------------------------------------------------------------------
// TAN: also the forward-mode tangent d rho (Eq. 14 differentiated along the
// tangent of positions and of the body pose) and d(P / rho^2).
template <int TX, int TY, bool TAN>
__global__ void __launch_bounds__(Shape<TX, TY>::THREADS, TAN ? 1 : Shape<TX, TY>::DENSITY_MIN_CTAS)
    density_kernel(SimDev S, EvalOut E, int eval, int chained)
{
    using Sh = Shape<TX, TY>;
    __shared__ Stage<TX, TY, false, TAN> sm;
    __shared__ GhostStage<!TAN> gs;
    const int4 td = S.tiles[blockIdx.x];
    const TankDev T = S.tank[td.x];  // by value: the constants live in registers
    const int cx0 = td.y, cy0 = td.z;
    // chained (a step after a step of the same sequence): the staging and the
    // fluid part of Eq. 14 read only what the previous force pass wrote, and
    // that pass completed before the body update passed its dependency, so
    // they run before this pass's dependency on the body update (through L2:
    // the staging loads bypass L1); the ghosts wait for the body
    const bool early = !TAN && chained;
    int buf;
    if (early) {
        buf = __ldcg(&S.run->next_buf);
    } else {
        pdl_wait();
        buf = (int)(S.run->step & 1);
    }
    const int nbuf = buf ^ 1;

    // clear the other buffer's counts of the own cells (it is re-filled by the force pass)
    for (int c = threadIdx.x; c < TX * TY; c += blockDim.x) {
        int ix = cx0 + c % TX, iy = cy0 + c / TX;
        if (ix < T.G && iy < T.G) S.count[nbuf][T.cell_base + iy * T.G + ix] = 0;
    }
    const bool staged = stage_tile<TX, TY, false, TAN>(S, T, buf, cx0, cy0, sm);
    save_stage(sm, staged, stage_record<TX, TY>(S, blockIdx.x));
    const int n_own = staged ? sm.own_row[TY] : 0;
    if (n_own == 0) {
        // a CTA that leaves without its dependency must not let the pass end
        // before the body update: the first CTA always waits (the force pass,
        // which depends on this one, reads what the body update writes)
        if (early && blockIdx.x == 0) pdl_wait();
        return;
    }

    const bool want_drho = eval && E.drho;
    // the fluid part of own particle t: Sf (Eq. 14's fluid sum), Df (the
    // fluid part of the continuity sum, evaluation only) and, in the tangent
    // variant, dRf; the neighbour record for the force pass
    auto fluid_part = [&](int t, float& Sf, float& Df, float& dRf) {
        const int e = own_index(t, sm);
        const float4 pi = sm.pv[e];
        const float2 li = sm.plo[e];
        const int c = sm.cell[e];
        Sf = 0.f;
        Df = 0.f;
        dRf = 0.f;
        float4 ti = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (TAN) ti = sm.tpv[e];
        // the fluid neighbours found here (staged index, r < 2h, j != i) are
        // recorded for the force pass, which stages the tile identically: per
        // stencil row, its last candidate zl and a mask of the candidates
        // zl - k that are neighbours (a row of more than kNbrRowBits
        // candidates is not recorded, and the force pass scans the stencil)
        const bool rec = t < Sh::MAXOWN;
        const size_t rec_at = (size_t)blockIdx.x * (3 * Sh::MAXOWN) + t;
        int nn = 0;
        bool wide = false;
        const float xlo = pi.x - T.clip, xhi = pi.x + T.clip;
        // each cell is sorted by x: of the row's left cell only the suffix
        // with x >= x_i - clip, of its right cell only the prefix with
        // x < x_i + clip can lie within the support (clip = 2h (1 + 1e-3)
        // keeps every FP32 decision r^2 < (2h)^2 inside the range).
        // Branch-free candidate loop: the support test r^2 < (2h)^2 splits
        // almost every warp, so the kernel value is computed for every
        // candidate and selected by the test.  For q = r / h,
        // f(q) = (2 - q)^3 - 4 max(1 - q, 0)^3 is Eq. 22's bracket on [0, 2)
        // (W = sigma / h^2 f); r = r^2 rsqrt(max(r^2, FLT_MIN)) is exactly 0
        // for the particle itself, giving W(0) = 4 sigma / h^2.  The tangent
        // variant runs the same arithmetic, so its primal equals the step's.
        // the candidate loop in two copies, with and without the continuity
        // sum (an evaluation output), so that the step's copy carries no
        // branch on it
        auto rows = [&](auto drho_tag) {
            constexpr bool want_drho = decltype(drho_tag)::value;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const int cl = c + dy * Sh::SX - 1;
                const int a = lower_x(sm, sm.start[cl], sm.start[cl + 1], xlo);
                const int z = lower_x(sm, sm.start[cl + 2], sm.start[cl + 3], xhi);
                wide |= z - a > kNbrRowBits;
                unsigned int bits = 0u;  // candidate j at bit z - 1 - j (the row's last candidate at bit 0)
#pragma unroll 2
                for (int j = a; j < z; ++j) {
                    const float4 pj = sm.pv[j];
                    const float2 d = sep_ff(pi, li, pj, sm.plo[j]);
                    const float ddx = d.x, ddy = d.y;
                    const float r2 = dist2(ddx, ddy);
                    const bool in = r2 < T.R2;
                    const float inv_r = rsqrtf(fmaxf(r2, FLT_MIN));
                    const float q = r2 * inv_r * T.inv_h;
                    const float qa = 2.0f - q, qb = fmaxf(1.0f - q, 0.0f);
                    const float f = fmaf(-4.0f * qb * qb, qb, qa * qa * qa);
                    Sf += in ? f : 0.0f;
                    const bool nb = in && (dy != 0 || j != e);  // the particle itself lies in its own row
                    bits = 2u * bits + (nb ? 1u : 0u);
                    const bool nd = nb && r2 > 0.f;
                    if (want_drho || TAN) {
                        const float gW = T.cdW * fmaf(12.0f * qb, qb, -3.0f * qa * qa) * inv_r;  // (dW/dr) / r
                        if (want_drho) Df += nd ? ((pi.z - pj.z) * ddx + (pi.w - pj.w) * ddy) * gW : 0.0f;
                        if constexpr (TAN) {
                            const float4 tj = sm.tpv[j];
                            dRf += nd ? (ddx * (ti.x - tj.x) + ddy * (ti.y - tj.y)) * gW : 0.0f;
                        }
                    }
                }
                nn += __popc(bits);
                if (rec) {
                    S.nbm[rec_at + (dy + 1) * Sh::MAXOWN] = bits;
                    S.nba[rec_at + (dy + 1) * Sh::MAXOWN] = (unsigned short)(z - 1);
                }
            }
        };
        if (want_drho) rows(std::integral_constant<bool, true>{});
        else rows(std::integral_constant<bool, false>{});
        Sf = __fmul_rn(Sf, T.cW);  // rounded here in every variant (no contraction with the ghost sum)
        if (rec) S.nbn[blockIdx.x * Sh::MAXOWN + t] = wide ? kNbrNone : (unsigned char)nn;
    };

    // after the body update: the ghosts of Eqs. 14 and 21, then rho and P
    const BodyDev& b = S.body[td.x];
    int gmode = kGhostsGlobal;  // the tangent variant visits the ghosts through global memory
    float bc = 0.f, bs = 0.f, brx = 0.f, bry = 0.f, fw = 0.f;
    GhostFrame fr{};
    float t_rx = 0.f, t_ry = 0.f, t_th = 0.f, t_vx = 0.f, t_vy = 0.f, t_w = 0.f;
    auto body_frame = [&]() {
        if constexpr (!TAN) gmode = stage_ghosts<true>(S, T, b, sm, n_own, gs);
        bc = b.fc;
        bs = b.fs;
        brx = b.frx;
        bry = b.fry;
        fr = ghost_frame(b);
        fw = fr.fw;
        if constexpr (TAN) {
            t_rx = b.ftr[0];
            t_ry = b.ftr[1];
            t_th = b.ftth;
            t_vx = b.ftv[0];
            t_vy = b.ftv[1];
            t_w = b.ftw;
        }
    };
    auto ghost_part = [&](int t, float Sf, float Df, float dRf) {
        const int e = own_index(t, sm);
        const float4 pi = sm.pv[e];
        const float2 li = sm.plo[e];
        float dRg = 0.f;
        float4 ti = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (TAN) ti = sm.tpv[e];
        float Sg = 0.f, Dg = 0.f;
        int ng2 = 0;
        // one ghost within reach: gp = (x_hi, y_hi, x_lo, y_lo) world position,
        // gv = (v_x, v_y, arm_x, arm_y) (Eq. 21), (tgx, tgy) its position tangent
        auto ghost = [&](const float4 gp, const float4 gv, float tgx, float tgy) {
            const float2 d = sep_fg(pi, li, gp);
            const float ddx = d.x, ddy = d.y;
            const float r2 = dist2(ddx, ddy);
            if (r2 < T.R2) {
                ++ng2;
                const float inv_r = rsqrtf(r2);
                const float r = r2 * inv_r;
                Sg += (r2 > 0.f) ? w_cubic(T, r) : T.cW * 4.0f;
                if (want_drho && r2 > 0.f)
                    Dg += ((pi.z - gv.x) * ddx + (pi.w - gv.y) * ddy) * dw_cubic_over_r(T, r, inv_r);
                if constexpr (TAN) {
                    if (r2 > 0.f) dRg += (ddx * (ti.x - tgx) + ddy * (ti.y - tgy)) * dw_cubic_over_r(T, r, inv_r);
                }
            }
        };
        if (gmode == kGhostsStaged) {
            if constexpr (!TAN)
                for_staged_ghosts(T, gs, pi.x, pi.y, bc, bs, brx, bry, T.clip,
                                  [&](int, int sg) { ghost(gs.gp[sg], gs.gv[sg], 0.f, 0.f); });
        } else if (gmode == kGhostsGlobal) {
            // Eq. 21 per visit, stored for the force pass and the adjoint
            for_ghosts(S, T, pi.x, pi.y, bc, bs, brx, bry, [&](int g) {
                float4 gp, gv;
                ghost_world(fr, __ldg(S.gB + g), gp, gv);
                S.gpos[g] = gp;
                S.gvel[g] = gv;
                float tgx = 0.f, tgy = 0.f;
                if constexpr (TAN) {  // d r_g = d r + d theta z x arm, d v_g likewise (Eq. 21)
                    const float armx = gv.z, army = gv.w;
                    tgx = t_rx - t_th * army;
                    tgy = t_ry + t_th * armx;
                    S.tgh[g] = make_float4(tgx, tgy, t_vx - t_w * army - fw * t_th * armx,
                                           t_vy + t_w * armx - fw * t_th * army);
                }
                ghost(gp, gv, tgx, tgy);
            });
        }
        // explicit roundings, so that the variants (fluid sums through shared
        // memory or in registers) take the same arithmetic
        const float rho = __fmul_rn(T.m, __fmaf_rn(T.gamma1, Sg, Sf));       // Eq. 14
        const float P = __fmul_rn(T.k, __fsub_rn(rho, T.rho0));               // Eq. 11
        const float pr2 = __fdiv_rn(P, __fmul_rn(rho, rho));
        S.rhoP[sm.slot[e]] = make_float2(rho, pr2);
        if constexpr (TAN) {  // d rho, and d(P/rho^2) = d rho (k / rho^2 - 2 P / rho^3)
            const float trh = T.m * (dRf + T.gamma1 * dRg);
            S.trho[sm.slot[e]] = make_float2(trh, trh * (T.k / (rho * rho) - 2.0f * pr2 / rho));
        }
        if (eval) {
            const int id = sm.pid[e];
            if (E.rho) E.rho[id] = rho;
            if (E.drho) E.drho[id] = T.m * (Df + T.gamma1 * Dg);
            if (E.nbr) E.nbr[3 * id + 1] = ng2;
        }
    };

    if constexpr (TAN) {
        body_frame();
        for (int t = threadIdx.x; t < n_own; t += blockDim.x) {
            float Sf, Df, dRf;
            fluid_part(t, Sf, Df, dRf);
            ghost_part(t, Sf, Df, dRf);
        }
    } else {
        // the fluid sums wait in the staging scratch (key_in, pid_in: free
        // once the tile is staged), each read back by the thread that wrote it
        for (int t = threadIdx.x; t < n_own; t += blockDim.x) {
            float Sf, Df, dRf;
            fluid_part(t, Sf, Df, dRf);
            sm.key_in[t] = __float_as_uint(Sf);
            sm.pid_in[t] = __float_as_int(Df);
        }
        if (early) pdl_wait();
        body_frame();
        for (int t = threadIdx.x; t < n_own; t += blockDim.x)
            ghost_part(t, __uint_as_float(sm.key_in[t]), __int_as_float(sm.pid_in[t]), 0.f);
    }
    // the successor's CTAs may be placed once every CTA of this pass is past
    // its particle loop (or has exited): placed earlier, they would wait in
    // griddepcontrol.wait on SM slots that tiles of this pass still need
    pdl_trigger();
}

// ---------------------------------------------------------------------------
// Block reductions (fixed order: deterministic)
// ---------------------------------------------------------------------------
__device__ __forceinline__ F2 shfl_f2(F2 v)
{
    return F2{__shfl_sync(0xffffffffu, v.hi, 0), __shfl_sync(0xffffffffu, v.lo, 0)};
}

__device__ __forceinline__ F2 shfl_down_f2(F2 v, int o)
{
    return F2{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}

struct Red {
    F2 fx, fy, t, cx, cy;
    unsigned long long pairs;
};

// Sums over a warp (result valid in lane 0).  Only the parts flagged by the
// uniform switches are reduced.
__device__ __forceinline__ Red warp_reduce(Red r, bool forces, bool com, int first = 16)
{
#pragma unroll
    for (int o = first; o > 0; o >>= 1) {
        if (forces) {
            r.fx = f2_add(r.fx, shfl_down_f2(r.fx, o));
            r.fy = f2_add(r.fy, shfl_down_f2(r.fy, o));
            r.t = f2_add(r.t, shfl_down_f2(r.t, o));
        }
        if (com) {
            r.cx = f2_add(r.cx, shfl_down_f2(r.cx, o));
            r.cy = f2_add(r.cy, shfl_down_f2(r.cy, o));
        }
        r.pairs += __shfl_down_sync(0xffffffffu, r.pairs, o);
    }
    return r;
}

// Sums over the block (result valid in thread 0): each warp's sum, then the
// warps' sums by a fixed shuffle tree in warp 0 (blockDim a power-of-two
// multiple of 32).
__device__ Red block_reduce(Red r, bool forces, bool com, Red* scratch /* one per warp */)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    r = warp_reduce(r, forces, com);
    __syncthreads();
    if (lane == 0) scratch[warp] = r;
    __syncthreads();
    if (warp == 0 && nw > 1) {
        const F2 z{0.f, 0.f};
        r = lane < nw ? scratch[lane] : Red{z, z, z, z, z, 0ull};
        r = warp_reduce(r, forces, com, nw >> 1);
    }
    return r;
}

// Sum of partials [p0, p1) by the whole block in fixed order: thread t adds
// p0 + t, p0 + t + blockDim.x, ... in that order, then the block tree (result
// in thread 0).
__device__ Red block_reduce_partials(const TilePartial* P, int p0, int p1, bool com, Red* scratch)
{
    const F2 z{0.f, 0.f};
    Red r{z, z, z, z, z, 0ull};
    for (int i = p0 + (int)threadIdx.x; i < p1; i += blockDim.x) {
        const float4 a = __ldcg(&P[i].a), b = __ldcg(&P[i].b);
        const int4 c = __ldcg(&P[i].c);
        r.fx = f2_add(r.fx, F2{a.x, a.y});
        r.fy = f2_add(r.fy, F2{a.z, a.w});
        r.t = f2_add(r.t, F2{b.x, b.y});
        if (com) {
            r.cx = f2_add(r.cx, F2{b.z, b.w});
            r.cy = f2_add(r.cy, F2{__int_as_float(c.x), __int_as_float(c.y)});
        }
        r.pairs += (unsigned long long)(unsigned)c.z;
    }
    return block_reduce(r, true, com, scratch);
}

__device__ __forceinline__ void store_partial(TilePartial* P, const Red& r, int wall)
{
    P->a = make_float4(r.fx.hi, r.fx.lo, r.fy.hi, r.fy.lo);
    P->b = make_float4(r.t.hi, r.t.lo, r.cx.hi, r.cx.lo);
    P->c = make_int4(__float_as_int(r.cy.hi), __float_as_int(r.cy.lo), (int)r.pairs, wall);
}

// Sum of partials [p0, p1) by one warp in fixed order: lane-strided, then a
// shuffle tree (result in lane 0).  *wall receives whether any of them saw a
// ghost pair (all lanes).
__device__ Red warp_reduce_partials(const TilePartial* P, int p0, int p1, bool com, int* wall)
{
    const F2 z{0.f, 0.f};
    Red r{z, z, z, z, z, 0ull};
    int w = 0;
    for (int i = p0 + (int)(threadIdx.x & 31); i < p1; i += 32) {
        const float4 a = __ldcg(&P[i].a), b = __ldcg(&P[i].b);
        const int4 c = __ldcg(&P[i].c);
        r.fx = f2_add(r.fx, F2{a.x, a.y});
        r.fy = f2_add(r.fy, F2{a.z, a.w});
        r.t = f2_add(r.t, F2{b.x, b.y});
        if (com) {
            r.cx = f2_add(r.cx, F2{b.z, b.w});
            r.cy = f2_add(r.cy, F2{__int_as_float(c.x), __int_as_float(c.y)});
        }
        r.pairs += (unsigned long long)(unsigned)c.z;
        w |= c.w;
    }
    *wall = __any_sync(0xffffffffu, w);
    return warp_reduce(r, true, com);
}

// ---------------------------------------------------------------------------
// Body update by the last CTA of a tank (Eq. 20, Eq. 28, outputs)
// ---------------------------------------------------------------------------
// Runs in warp 0 of the CTA that finished the tank's reduction, with the
// reduced fluid force, torque and position sums as FP64 totals.  The FP64 pipe
// of this GPU is narrow and every global access on the serial path costs an
// L2 round trip, so warp 0 of every CTA loads the values the update reads
// (finalize_preload) right after the grid dependency resolves, while the tile
// is staged; the body is updated in registers and stored once, and the masses
// enter as reciprocals.
//
// finalize_preload: lane l of warp 0 holds one value (as a double or as the
// bits of one): the body's r, theta, rdot, thetadot, cos, sin (l < 8, the
// leading doubles of BodyDev), the held control torque (8), the input of this
// step (9..11), the controller's J, omega, xi (12..14), the reference angle of
// this sample (15), the controller / held-tank switches (16), the sample
// output pointer (17), the call's first step (18), the sample stride (19) and
// the step (20).
__device__ __forceinline__ double finalize_preload(const SimDev& S, const TankDev& T, int tank)
{
    const int lane = (int)(threadIdx.x & 31);
    const RunDev* run = S.run;
    const BodyDev* bp = S.body + tank;
    const long long step = run->step, step0 = run->step0;
    const long long k = step - step0;
    double pre = 0.0;
    if (lane < 8) {
        pre = reinterpret_cast<const double*>(bp)[lane];
    } else if (lane == 8) {
        pre = bp->tau_c;
    } else if (lane < 12) {
        const double* up = run->u;
        if (up) pre = up[tank * run->u_tank_stride + 3 * k + (lane - 9)];
    } else if (lane == 12) {
        pre = run->ctrl_J;
    } else if (lane == 13) {
        pre = run->ctrl_w;
    } else if (lane == 14) {
        pre = run->ctrl_xi;
    } else if (lane == 15) {
        const long long oe = T.outer_every;
        const double* ref = run->theta_ref;
        if (ref && (step % oe) == 0) pre = ref[tank * run->ref_stride + (step / oe - (step0 + oe - 1) / oe)];
    } else if (lane == 16) {
        pre = __longlong_as_double((long long)(run->ctrl_on ? 1 : 0) | (long long)(run->body_fixed ? 2 : 0));
    } else if (lane == 17) {
        pre = __longlong_as_double((long long)run->y);
    } else if (lane == 18) {
        pre = __longlong_as_double(step0);
    } else if (lane == 19) {
        pre = __longlong_as_double(run->y_tank_stride);
    } else if (lane == 20) {
        pre = __longlong_as_double(step);
    }
    return pre;
}

// cos and sin of theta + dtheta from those of theta: for |dtheta| <= 1e-2 the
// angle-addition formulas with Taylor series of cos and sin of dtheta (their
// first omitted terms are below 1e-16 relative) and one Newton step that
// keeps cos^2 + sin^2 at 1; otherwise FP64 sincos of the new angle.  The
// dependent FP64 chain is a quarter of sincos's, and it is on the serial
// path of every step.
__device__ __forceinline__ void rotate(double dth, double th_new, double& c, double& s)
{
    if (fabs(dth) > 1e-2) {
        sincos(th_new, &s, &c);
        return;
    }
    const double d2 = dth * dth;
    const double cd = 1.0 - d2 * (0.5 - d2 * (1.0 / 24.0 - d2 * (1.0 / 720.0)));
    const double sd = dth * (1.0 - d2 * (1.0 / 6.0 - d2 * (1.0 / 120.0 - d2 * (1.0 / 5040.0))));
    const double c1 = c * cd - s * sd, s1 = s * cd + c * sd;
    const double f = 1.5 - 0.5 * (c1 * c1 + s1 * s1);
    c = c1 * f;
    s = s1 * f;
}

// The value at position `lane` of the list (0 past its end): nested selects,
// so the lanes of a warp pick different values without diverging.
__device__ __forceinline__ double pick(int, int) { return 0.0; }
template <class... R>
__device__ __forceinline__ double pick(int lane, int i, double x, R... rest)
{
    return lane == i ? x : pick(lane, i + 1, rest...);
}

// Fx, Fy, Tq: fluid force and torque on the body (Eq. 20); Cx, Cy: sums of the
// particle positions (sample steps only).  add_pairs: pair interactions of the
// pass still to be added to the tank's count (the tiles of the step pass add
// theirs themselves).  tr: tangent of the reduced sums (TAN only).
// Every lane of warp 0 computes the same FP64 body update (one warp
// instruction costs the same for one lane as for all), and the lanes then
// convert and store one field each, so the stores of the body record, its
// FP32 forms and the sample are one short parallel step.
__device__ void tank_finalize(const SimDev& S, const TankDev& T, int tank, int eval, const EvalOut& E, int nbuf,
                              long long step, bool sample, bool tan, double Fx, double Fy, double Tq, double Cx,
                              double Cy, unsigned long long add_pairs, const Red& tr, double pre)
{
    RunDev* run = S.run;
    BodyDev* bp = S.body + tank;
    const int lane = (int)(threadIdx.x & 31);
    double rx = __shfl_sync(0xffffffffu, pre, 0), ry = __shfl_sync(0xffffffffu, pre, 1);
    double th = __shfl_sync(0xffffffffu, pre, 2), vx = __shfl_sync(0xffffffffu, pre, 3);
    double vy = __shfl_sync(0xffffffffu, pre, 4), w = __shfl_sync(0xffffffffu, pre, 5);
    double c = __shfl_sync(0xffffffffu, pre, 6), sn = __shfl_sync(0xffffffffu, pre, 7);
    double tau_c = __shfl_sync(0xffffffffu, pre, 8);
    const double ux = __shfl_sync(0xffffffffu, pre, 9), uy = __shfl_sync(0xffffffffu, pre, 10);
    const double ut = __shfl_sync(0xffffffffu, pre, 11);
    const double cJ = __shfl_sync(0xffffffffu, pre, 12), cw = __shfl_sync(0xffffffffu, pre, 13);
    const double cxi = __shfl_sync(0xffffffffu, pre, 14), ref = __shfl_sync(0xffffffffu, pre, 15);
    const long long sw = __double_as_longlong(__shfl_sync(0xffffffffu, pre, 16));
    double* const yout = (double*)__double_as_longlong(__shfl_sync(0xffffffffu, pre, 17));
    const long long step0 = __double_as_longlong(__shfl_sync(0xffffffffu, pre, 18));
    const long long ystride = __double_as_longlong(__shfl_sync(0xffffffffu, pre, 19));
    const long long k = step - step0;
    const bool ctrl_on = (sw & 1) != 0, body_fixed = (sw & 2) != 0;

    // FP64 from here on: assembly of the body state.  The serial chain runs
    // in lane 0 alone: on this GPU's narrow FP64 pipe a warp instruction costs
    // in proportion to its active lanes.
    if (sample) {
        const long long oe = T.outer_every;
        const long long row = step / oe - (step0 + oe - 1) / oe;
        if (ctrl_on) {  // Eq. 28 under zero-order hold
            if (lane == 0) {
                const double Jc = cJ > 0.0 ? cJ : T.J_body;
                tau_c = Jc * cw * cw * (ref - th) - 2.0 * cxi * Jc * cw * w;
                bp->tau_c = tau_c;
            }
        }
        if (yout && lane < SPH_NY) {
            double v = pick(lane, 0, rx, ry, th, vx, vy, w, Fx, Fy, Tq);
            if (lane == 9) v = T.n_f ? Cx / T.n_f : 0.0;
            if (lane == 10) v = T.n_f ? Cy / T.n_f : 0.0;
            yout[tank * ystride + row * SPH_NY + lane] = v;
        }
    }
    if (tan && !eval && lane == 0) {  // tangent of Eq. 20 and of the kick-then-drift body step
        const double dFx = (double)tr.fx.hi + (double)tr.fx.lo;
        const double dFy = (double)tr.fy.hi + (double)tr.fy.lo;
        const double dTq = (double)tr.t.hi + (double)tr.t.lo;
        double dux = 0.0, duy = 0.0, dut = 0.0;
        if (run->du) {
            const double* du = run->du + tank * run->u_tank_stride + 3 * k;
            dux = du[0];
            duy = du[1];
            dut = du[2];
        }
        BodyDev& b = *bp;
        if (sample && run->dy) {
            const long long oe = T.outer_every;
            const long long row = step / oe - (step0 + oe - 1) / oe;
            double* y = run->dy + tank * run->y_tank_stride + row * SPH_NY;
            y[0] = b.tr[0];
            y[1] = b.tr[1];
            y[2] = b.tth;
            y[3] = b.tv[0];
            y[4] = b.tv[1];
            y[5] = b.tw;
            y[6] = dFx;
            y[7] = dFy;
            y[8] = dTq;
            y[9] = T.n_f ? ((double)tr.cx.hi + (double)tr.cx.lo) / T.n_f : 0.0;
            y[10] = T.n_f ? ((double)tr.cy.hi + (double)tr.cy.lo) / T.n_f : 0.0;
        }
        if (!body_fixed) {
            b.tv[0] += T.dt_d * (dFx + dux) * T.inv_m_body;
            b.tv[1] += T.dt_d * (dFy + duy) * T.inv_m_body;
            b.tw += T.dt_d * (dTq + dut) * T.inv_J_body;
            b.tr[0] += T.dt_d * b.tv[0];
            b.tr[1] += T.dt_d * b.tv[1];
            b.tth += T.dt_d * b.tw;
        }
        b.ftr[0] = (float)b.tr[0];
        b.ftr[1] = (float)b.tr[1];
        b.ftth = (float)b.tth;
        b.ftv[0] = (float)b.tv[0];
        b.ftv[1] = (float)b.tv[1];
        b.ftw = (float)b.tw;
    }
    if (tan && eval && E.dbody && lane == 0) {  // tangent of the evaluation's body outputs (no controller)
        const double dFx = (double)tr.fx.hi + (double)tr.fx.lo;
        const double dFy = (double)tr.fy.hi + (double)tr.fy.lo;
        const double dTq = (double)tr.t.hi + (double)tr.t.lo;
        double dux = 0.0, duy = 0.0, dut = 0.0;
        if (run->du) {
            const double* du = run->du + tank * run->u_tank_stride + 3 * k;
            dux = du[0];
            duy = du[1];
            dut = du[2];
        }
        double* o = E.dbody + 6 * tank;
        o[0] = dFx;
        o[1] = dFy;
        o[2] = dTq;
        o[3] = (dFx + dux) * T.inv_m_body;
        o[4] = (dFy + duy) * T.inv_m_body;
        o[5] = (dTq + dut) * T.inv_J_body;
    }
    double ax = 0.0, ay = 0.0, aw = 0.0;
    if (lane == 0) {
        const double tau = ut + (ctrl_on ? tau_c : 0.0);
        ax = (Fx + ux) * T.inv_m_body;
        ay = (Fy + uy) * T.inv_m_body;
        aw = (Tq + tau) * T.inv_J_body;
        if (!eval && !body_fixed) {
            vx += T.dt_d * ax;  // kick then drift (Section 3.4)
            vy += T.dt_d * ay;
            w += T.dt_d * aw;
            rx += T.dt_d * vx;
            ry += T.dt_d * vy;
            const double dth = T.dt_d * w;
            th += dth;
            rotate(dth, th, c, sn);
        }
    }
    if (eval) {
        ax = __shfl_sync(0xffffffffu, ax, 0);
        ay = __shfl_sync(0xffffffffu, ay, 0);
        aw = __shfl_sync(0xffffffffu, aw, 0);
        if (E.body && lane < 6) E.body[6 * tank + lane] = pick(lane, 0, Fx, Fy, Tq, ax, ay, aw);
    } else {
        if (lane < 2) bp->anchor[nbuf][lane] = lane ? ry : rx;  // the state before the step (unchanged in lanes 1..)
        rx = __shfl_sync(0xffffffffu, rx, 0);
        ry = __shfl_sync(0xffffffffu, ry, 0);
        th = __shfl_sync(0xffffffffu, th, 0);
        vx = __shfl_sync(0xffffffffu, vx, 0);
        vy = __shfl_sync(0xffffffffu, vy, 0);
        w = __shfl_sync(0xffffffffu, w, 0);
        c = __shfl_sync(0xffffffffu, c, 0);
        sn = __shfl_sync(0xffffffffu, sn, 0);
        // the leading doubles of BodyDev: r, theta, rdot, thetadot, cos, sin
        if (!body_fixed && lane < 8) reinterpret_cast<double*>(bp)[lane] = pick(lane, 0, rx, ry, th, vx, vy, w, c, sn);
        // FP32 forms: two-float splits (lanes 0-3: dc, ds, drx, dry), rounded
        // values (lanes 4-9: fc, fs, frx, fry, fo_next; lanes 10-12: fvx, fvy, fw)
        if (lane < 13) {
            double d = pick(lane, 0, c, sn, rx, ry, c, sn, rx, ry, rx, ry, vx, vy, w);
            if (lane == 8 || lane == 9) d -= T.W;
            const float hi = (float)d;
            if (lane < 4) (&bp->dc)[lane] = make_float2(hi, (float)(d - (double)hi));
            else if (lane < 10) (&bp->fc)[lane - 4] = hi;
            else (&bp->fvx)[lane - 10] = hi;
        }
        if (lane == 0) bp->pairs += add_pairs;
    }
    if (lane != 0) return;
    bp->done = 0;
    if (S.B == 1) {  // the only tank: its step is the pass's (visible when the kernel completes)
        if (!eval) run->step = step + 1;
        return;
    }
    fence_acq_rel();
    const unsigned prev = atomicAdd(&run->tanks_done, 1u);
    if (prev == (unsigned)S.B - 1) {
        if (!eval) run->step = step + 1;
        run->tanks_done = 0;
    }
}

// Adds a two-float sum to a fixed-point body accumulator (an integer
// reduction: the total does not depend on the order of the tiles).
__device__ __forceinline__ void fix_add(unsigned long long* a, F2 v)
{
    const long long q = __float2ll_rn(v.hi * kFixScale) + __float2ll_rn(v.lo * kFixScale);
    atomicAdd(a, (unsigned long long)q);
}
// ---------------------------------------------------------------------------
// Force pass: Eqs. 10, 12, 16-19, Algorithm 1, symplectic Euler, re-binning
// ---------------------------------------------------------------------------
// TAN: also the forward-mode tangent of the accelerations, of the step and of
// the body force/torque, along the tangent staged with the particles.
template <int TX, int TY, bool TAN>
__global__ void __launch_bounds__(Shape<TX, TY>::THREADS, TAN ? 1 : Shape<TX, TY>::FORCE_MIN_CTAS)
    force_kernel(SimDev S, EvalOut E, int eval)
{
    using Sh = Shape<TX, TY>;
    __shared__ Stage<TX, TY, true, TAN> sm;
    __shared__ GhostStage<!TAN> gs;
    __shared__ Red scratch[32];
    __shared__ int is_last;
    // the successor is the body update, a few warps: placed at once, it
    // prepares its update during this pass (the tangent variant's successor
    // is the next density pass, placed after the loop as there)
    if constexpr (!TAN) pdl_trigger();
    const int4 td = S.tiles[blockIdx.x];
    const int tank = td.x;
    const TankDev T = S.tank[tank];  // by value: the constants live in registers
    const int cx0 = td.y, cy0 = td.z;
    pdl_wait();
    const long long step = S.run->step;
    const int buf = (int)(step & 1), nbuf = buf ^ 1;
    // the buffer the next density pass stages from, readable before its grid
    // dependency once this pass has completed
    if (!eval && blockIdx.x == 0 && threadIdx.x == 0) S.run->next_buf = nbuf;
    const bool sample = !eval && (step % T.outer_every) == 0;
    const float damp = 1.0f - S.run->damping;

    const F2 z{0.f, 0.f};
    Red acc{z, z, z, z, z, 0ull};
    Red tacc{z, z, z, z, z, 0ull};
    int flags = 0, wall = 0, own = 0;
    if (stage_from_record<TX, TY, TAN>(S, tank, buf, stage_record<TX, TY>(S, blockIdx.x), sm)) {
        const BodyDev& b = S.body[tank];
        const int n_own = sm.own_row[TY];
        own = n_own;
        int gmode = kGhostsGlobal;  // the tangent variant visits the ghosts through global memory
        if constexpr (!TAN) gmode = n_own > 0 ? stage_ghosts<false>(S, T, b, sm, n_own, gs) : kGhostsNone;
        const float bc = b.fc, bs = b.fs, brx = b.frx, bry = b.fry;
        const float ox = b.fo_next[0], oy = b.fo_next[1];  // origin of the next grid
        const float mm = T.m * T.m;
        float wfx = 0.f, wfy = 0.f, wt = 0.f, cxs = 0.f, cys = 0.f;
        float twfx = 0.f, twfy = 0.f, twt = 0.f, tcxs = 0.f, tcys = 0.f;
        const float t_th = TAN ? b.ftth : 0.f;
        for (int t = threadIdx.x; t < n_own; t += blockDim.x) {
            const int e = own_index(t, sm);
            const float4 pi = sm.pv[e];
            const float2 li = sm.plo[e];
            const float2 ri = sm.rho[e];
            const int c = sm.cell[e];
            float ax = 0.f, ay = 0.f, tax = 0.f, tay = 0.f;
            float4 ti = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 tri = make_float2(0.f, 0.f);
            if constexpr (TAN) {
                ti = sm.tpv[e];
                tri = sm.trho[e];
            }
            int nff = 0;
            // one fluid pair, r < 2h, j != i: Eqs. 10 and 12
            auto pair = [&](int j) {
                const float4 pj = sm.pv[j];
                const float2 d = sep_ff(pi, li, pj, sm.plo[j]);
                const float ddx = d.x, ddy = d.y;
                const float r2 = dist2(ddx, ddy);
                if (r2 > 0.f) {
                    const float2 rj = sm.rho[j];
                    const float inv_r = rsqrtf(r2);
                    const float r = r2 * inv_r;
                    const float gW = dw_cubic_over_r(T, r, inv_r);
                    const float press = -(ri.y + rj.y);                                  // Eq. 10
                    const float vr = (pi.z - pj.z) * ddx + (pi.w - pj.w) * ddy;
                    const float visc = __fdividef(T.visc_a * vr, (ri.x + rj.x) * (r2 + T.epsh2));  // Eq. 12
                    const float s = T.m * (press + visc) * gW;
                    ax = fmaf(s, ddx, ax);
                    ay = fmaf(s, ddy, ay);
                    if constexpr (TAN) {  // d(s d) = ds d + s dd
                        const float4 tj = sm.tpv[j];
                        const float2 trj = sm.trho[j];
                        const float tdx = ti.x - tj.x, tdy = ti.y - tj.y;
                        const float rd = ddx * tdx + ddy * tdy;                          // d . dd
                        const float tG = dG_cubic_dr(T, r, inv_r, gW) * rd * inv_r;
                        const float B = ri.x + rj.x, Cc = r2 + T.epsh2;
                        const float tA = (ti.z - tj.z) * ddx + (ti.w - tj.w) * ddy + (pi.z - pj.z) * tdx +
                                         (pi.w - pj.w) * tdy;
                        const float tvisc = __fdividef(T.visc_a, B * Cc) *
                                            (tA - vr * (__fdividef(tri.x + trj.x, B) + __fdividef(2.0f * rd, Cc)));
                        const float ts = T.m * ((-(tri.y + trj.y) + tvisc) * gW + (press + visc) * tG);
                        tax += ts * ddx + s * tdx;
                        tay += ts * ddy + s * tdy;
                    }
                }
            };
            // the neighbours recorded by the density pass (no candidate tests)
            if (for_recorded_neighbours<Sh::MAXOWN>(S, blockIdx.x, t, [&](int j) { ++nff; pair(j); })) {
            } else {              // not recorded: scan the 3x3 cells
#pragma unroll
                for (int dy = -1; dy <= 1; ++dy) {
                    const int a = sm.start[c + dy * Sh::SX - 1], zz = sm.start[c + dy * Sh::SX + 2];
                    for (int j = a; j < zz; ++j) {
                        const float2 d = sep_ff(pi, li, sm.pv[j], sm.plo[j]);
                        if (j != e && dist2(d.x, d.y) < T.R2) {
                            ++nff;
                            pair(j);
                        }
                    }
                }
            }
            int nfg = 0;
            // P_i / rho_i^2 in Eq. 16: clamped at zero when the wall only pushes
            const float qg = T.gp_clamp ? fmaxf(ri.y, 0.f) : ri.y;
            // one ghost: gp its world position (x_hi, y_hi, x_lo, y_lo), load_gv()
            // its (v_x, v_y, arm_x, arm_y), read only for a pair within reach
            auto ghost = [&](int g, const float4 gp, auto&& load_gv) {
                const float2 d = sep_fg(pi, li, gp);
                const float ddx = d.x, ddy = d.y;
                const float r2 = dist2(ddx, ddy);
                if (r2 < T.h2) {
                    ++nfg;
                    if (r2 > 0.f) {
                        const float4 gv = load_gv();
                        const float inv_r = rsqrtf(r2);
                        const float r = r2 * inv_r;
                        const float d = T.h - r;
                        const float gWs = T.cdS * d * d * inv_r;                         // (dW_s3/dr)/r
                        const float fp = T.gp_sign * 2.0f * mm * qg * gWs;              // Eq. 16
                        const float vr = (pi.z - gv.x) * ddx + (pi.w - gv.y) * ddy;
                        const float fv = __fdividef(mm * T.beta2 * fminf(vr, 0.f), (ri.x + ri.x) * (r2 + T.epsh2)) * gWs;  // Eq. 18
                        const float f = fp + fv;
                        const float fx = f * ddx, fy = f * ddy;
                        ax = fmaf(fx, T.inv_m, ax);
                        ay = fmaf(fy, T.inv_m, ay);
                        wfx -= fx;                                                       // Eqs. 17, 19
                        wfy -= fy;
                        wt -= gv.z * fy - gv.w * fx;                                     // Eq. 20 torque
                        if constexpr (TAN) {
                            const float4 tg = __ldg(S.tgh + g);                           // (d r_g, d v_g)
                            const float tdx = ti.x - tg.x, tdy = ti.y - tg.y;
                            const float rd = ddx * tdx + ddy * tdy;
                            const float tGs = -T.cdS * d * (T.h + r) * inv_r * inv_r * rd * inv_r;  // d(Gs)
                            const float tfp = T.gp_sign * 2.0f * mm * (qg == ri.y ? tri.y : 0.f);
                            float tcv = 0.f;
                            if (vr < 0.f) {
                                const float Cc = r2 + T.epsh2;
                                const float tA = (ti.z - tg.z) * ddx + (ti.w - tg.w) * ddy + (pi.z - gv.x) * tdx +
                                                 (pi.w - gv.y) * tdy;
                                tcv = __fdividef(mm * T.beta2, (ri.x + ri.x) * Cc) *
                                      (tA - vr * (__fdividef(tri.x, ri.x) + __fdividef(2.0f * rd, Cc)));
                            }
                            const float cf = T.gp_sign * 2.0f * mm * qg +                 // fp + fv without Gs
                                             __fdividef(mm * T.beta2 * fminf(vr, 0.f), (ri.x + ri.x) * (r2 + T.epsh2));
                            const float tf = (tfp + tcv) * gWs + cf * tGs;
                            const float tfx = tf * ddx + f * tdx, tfy = tf * ddy + f * tdy;
                            tax = fmaf(tfx, T.inv_m, tax);
                            tay = fmaf(tfy, T.inv_m, tay);
                            twfx -= tfx;
                            twfy -= tfy;
                            // d(arm x f) with d arm = d theta z x arm
                            twt -= (-t_th * gv.w) * fy + gv.z * tfy - ((t_th * gv.z) * fx + gv.w * tfx);
                        }
                    }
                }
            };
            if (gmode == kGhostsStaged) {
                if constexpr (!TAN)
                    for_staged_ghosts(T, gs, pi.x, pi.y, bc, bs, brx, bry, T.hclip,
                                      [&](int g, int sg) { ghost(g, gs.gp[sg], [&] { return gs.gv[sg]; }); });
            } else if (gmode == kGhostsGlobal) {
                for_ghosts(S, T, pi.x, pi.y, bc, bs, brx, bry,
                           [&](int g) { ghost(g, __ldg(S.gpos + g), [&] { return __ldg(S.gvel + g); }); });
            }
            wall |= (nfg > 0);
            acc.pairs += (unsigned long long)(nff + nfg);
            cxs += pi.x;
            cys += pi.y;
            tcxs += ti.x;
            tcys += ti.y;
            ax += T.grav_x;
            ay += T.grav_y;
            const int id = sm.pid[e];
            if (eval) {
                if (E.acc) {
                    E.acc[2 * id] = ax;
                    E.acc[2 * id + 1] = ay;
                }
                if constexpr (TAN) {
                    if (E.dacc) {
                        E.dacc[2 * id] = tax;
                        E.dacc[2 * id + 1] = tay;
                    }
                }
                if (E.nbr) {
                    E.nbr[3 * id] = nff;
                    E.nbr[3 * id + 2] = nfg;
                }
                if (E.keys) E.keys[id] = (cy0 - 1 + c / Sh::SX) * T.G + (cx0 - 1 + c % Sh::SX);
            } else {
                // kick then drift (Section 3.4) on the two-float state, then bin
                // into the next grid: v' = (v + dt a)(1 - c), x' = x + dt v'
                const float2 vl = sm.vlo[e];
                float2 kx = two_sum(pi.z, fmaf(T.dt, ax, vl.x)), ky = two_sum(pi.w, fmaf(T.dt, ay, vl.y));
                if (damp != 1.0f) {  // relaxation: scale the two-float velocity
                    const float hx = kx.x * damp, hy = ky.x * damp;
                    kx = two_sum(hx, fmaf(kx.x, damp, -hx) + kx.y * damp);
                    ky = two_sum(hy, fmaf(ky.x, damp, -hy) + ky.y * damp);
                }
                const float2 dx2 = two_sum(pi.x, fmaf(T.dt, kx.x, fmaf(T.dt, kx.y, li.x)));
                const float2 dy2 = two_sum(pi.y, fmaf(T.dt, ky.x, fmaf(T.dt, ky.y, li.y)));
                const float vx = kx.x, vy = ky.x, x = dx2.x, y = dy2.x;
                if (!(isfinite(x) && isfinite(y) && isfinite(vx) && isfinite(vy))) flags |= SPH_FLAG_NAN;
                bool out = false;
                const int ccx = cell_coord(x, ox, T.inv_cell, T.G, &out);
                const int ccy = cell_coord(y, oy, T.inv_cell, T.G, &out);
                const float ex = x - (ox + T.Wf), ey = y - (oy + T.Wf);   // from the next grid's centre
                if (out || fmaf(ex, ex, ey * ey) > T.cover2) flags |= SPH_FLAG_ESCAPED;
                const int cell = T.cell_base + ccy * T.G + ccx;
                const int slot = atomicAdd(&S.count[nbuf][cell], 1);
                if ((unsigned)slot < (unsigned)kCap) {
                    S.pv[nbuf][cell * kCap + slot] = make_float4(x, y, vx, vy);
                    S.lo[nbuf][cell * kCap + slot] = make_float4(dx2.y, dy2.y, kx.y, ky.y);
                    S.pid[nbuf][cell * kCap + slot] = id;
                    if constexpr (TAN) {  // tangent of kick then drift, binned with the particle
                        const float tvx = fmaf(T.dt, tax, ti.z) * damp, tvy = fmaf(T.dt, tay, ti.w) * damp;
                        S.tpv[nbuf][cell * kCap + slot] = make_float4(fmaf(T.dt, tvx, ti.x), fmaf(T.dt, tvy, ti.y),
                                                                      tvx, tvy);
                    }
                } else {
                    flags |= SPH_FLAG_CELL_FULL;
                }
            }
        }
        acc.fx = F2{wfx, 0.f};
        acc.fy = F2{wfy, 0.f};
        acc.t = F2{wt, 0.f};
        acc.cx = F2{cxs, 0.f};
        acc.cy = F2{cys, 0.f};
        tacc.fx = F2{twfx, 0.f};
        tacc.fy = F2{twfy, 0.f};
        tacc.t = F2{twt, 0.f};
        tacc.cx = F2{tcxs, 0.f};
        tacc.cy = F2{tcys, 0.f};
    }
    if constexpr (TAN) pdl_trigger();  // past the particle loop (see the density pass)
    if (flags) atomicOr(&S.body[tank].flags, flags);
    if constexpr (!TAN) {
        // The tile's sums go into the tank's fixed-point accumulators by
        // integer atomics (order-independent, so every run, and a tank run
        // alone or in a batch, gets the same bits); the body kernel that
        // follows this pass reads them.  A tile without own particles adds
        // nothing.
        if (own == 0) return;  // uniform over the block
        BodyDev* bp = S.body + tank;
        const int lane = (int)(threadIdx.x & 31);
        const bool any_wall = __syncthreads_or(wall) != 0;
        const Red r = block_reduce(acc, any_wall, sample, scratch);
        if (threadIdx.x >= 32) return;
        // lane q adds component q (F_x, F_y, T on wall tiles; the position
        // sums on sample steps), lane 5 the pair count
        const F2 fx = shfl_f2(r.fx), fy = shfl_f2(r.fy), tq = shfl_f2(r.t), cx = shfl_f2(r.cx), cy = shfl_f2(r.cy);
        const unsigned long long pairs = __shfl_sync(0xffffffffu, r.pairs, 0);
        const F2 mine = lane == 0 ? fx : lane == 1 ? fy : lane == 2 ? tq : lane == 3 ? cx : cy;
        if ((lane < 3 && any_wall) || (lane >= 3 && lane < 5 && sample)) fix_add(&bp->acc[lane], mine);
        if (lane == 5 && !eval && pairs) atomicAdd(&bp->pairs, pairs);
        return;
    } else {
        // what the body update reads, in flight during the tile's reduction
        // (only the tank's last tile uses it)
        double pre = 0.0;
        if (threadIdx.x < 32) pre = finalize_preload(S, T, tank);
        const int t0 = S.tile_tank_first[tank], t1 = S.tile_tank_first[tank + 1];
        const bool any_wall = __syncthreads_or(wall) != 0;
        Red r = block_reduce(acc, any_wall, sample, scratch);
        // Tangent variant: fixed-order reduction of the tile partials (the
        // tangent's scale is the caller's, unsuited to a fixed point).  One
        // level when the tank's last tile can fetch them with at most
        // kOneLevelLoads loads per thread: the last tile (by a counter of
        // finished tiles) sums them with the whole block.  Otherwise two
        // levels: the last tile of each group of kTileGroup tiles sums the
        // group, the last group of the tank sums the groups.
        Red tr = block_reduce(tacc, any_wall, sample, scratch);
        // called by all of warp 0 with the sums valid in lane 0: every lane
        // of the body update needs them
        auto finish = [&](const Red& rt, const Red& trt) {
            auto all = [](F2 v) { return __shfl_sync(0xffffffffu, (double)v.hi + (double)v.lo, 0); };
            tank_finalize(S, T, tank, eval, E, nbuf, step, sample, true, all(rt.fx), all(rt.fy), all(rt.t),
                          all(rt.cx), all(rt.cy), rt.pairs, trt, pre);
        };
        if (t1 - t0 <= kOneLevelLoads * (int)blockDim.x) {
            if (threadIdx.x == 0) {
                store_partial(S.partials + blockIdx.x, r, any_wall ? 1 : 0);
                store_partial(S.tpartials + blockIdx.x, tr, any_wall ? 1 : 0);
                fence_acq_rel();
                is_last = (atomicAdd(&S.body[tank].done, 1u) == (unsigned)(t1 - t0 - 1));
            }
            __syncthreads();
            if (!is_last) return;
            fence_acq_rel();
            const Red rt = block_reduce_partials(S.partials, t0, t1, sample, scratch);
            const Red trt = block_reduce_partials(S.tpartials, t0, t1, sample, scratch);
            if (threadIdx.x < 32) finish(rt, trt);
            return;
        }
        const int gi = (blockIdx.x - t0) / kTileGroup;
        const int gt0 = t0 + gi * kTileGroup, gt1 = min(gt0 + kTileGroup, t1);
        const int g = S.group_first[tank] + gi;
        if (threadIdx.x == 0) {
            store_partial(S.partials + blockIdx.x, r, any_wall ? 1 : 0);
            store_partial(S.tpartials + blockIdx.x, tr, any_wall ? 1 : 0);
            fence_acq_rel();
            is_last = (atomicAdd(&S.gdone[g], 1u) == (unsigned)(gt1 - gt0 - 1));
        }
        __syncthreads();
        if (!is_last || threadIdx.x >= 32) return;  // warp 0 of the group's last tile goes on
        fence_acq_rel();
        int wall_g;
        r = warp_reduce_partials(S.partials, gt0, gt1, sample, &wall_g);
        tr = warp_reduce_partials(S.tpartials, gt0, gt1, sample, &wall_g);
        unsigned prev = 0;
        if (threadIdx.x == 0) {
            store_partial(S.gpartials + g, r, wall_g);
            store_partial(S.tgpartials + g, tr, wall_g);
            S.gdone[g] = 0;
            fence_acq_rel();
            prev = atomicAdd(&S.body[tank].done, 1u);
        }
        const unsigned n_groups = (unsigned)(S.group_first[tank + 1] - S.group_first[tank]);
        if (__shfl_sync(0xffffffffu, prev, 0) != n_groups - 1) return;
        fence_acq_rel();
        int wall_t;
        const Red rt = warp_reduce_partials(S.gpartials, S.group_first[tank], S.group_first[tank + 1], sample, &wall_t);
        const Red trt = warp_reduce_partials(S.tgpartials, S.group_first[tank], S.group_first[tank + 1], sample, &wall_t);
        finish(rt, trt);
    }
}

// ---------------------------------------------------------------------------
// Body update after the force pass (Eq. 20, Eq. 28, outputs): one warp per tank
// ---------------------------------------------------------------------------
// The kernel boundary after the force pass takes the place of a counter of
// finished tiles: when the grid dependency resolves, every tile's sums are in
// the tank's accumulators.  The previous body update and the call's run
// record were complete before this kernel could be placed, so each warp does
// everything that does not depend on this step's fluid force before the
// dependency.  Kick then drift (Section 3.4) is affine in the fluid force and
// torque: v' = v + dt (F + u) / M = A + B F, r' = r + dt v' = A' + B' F, and
// likewise theta', thetadot' in T_b.  Lane l holds the coefficients of output
// l, so after the dependency each output is one FP64 FMA (FP64 latency on this
// GPU is 65 cycles per dependent operation), cos and sin of the new angle a
// rotation by dtheta, and the lanes convert and store their own outputs.
// Multiplication is reassociated against the oracle's sequence: the results
// differ from it in the last bits only.
constexpr int kBodyWarps = 4;  // tanks per CTA

__device__ __forceinline__ double sel3(int i, double a, double b, double c) { return i == 0 ? a : (i == 1 ? b : c); }

__global__ void __launch_bounds__(32 * kBodyWarps) body_kernel(SimDev S, EvalOut E, int eval)
{
    const int tank = blockIdx.x * kBodyWarps + (int)(threadIdx.x >> 5);
    const int lane = (int)(threadIdx.x & 31);
    if (tank >= S.B) return;  // a whole warp
    const TankDev T = S.tank[tank];
    RunDev* run = S.run;
    BodyDev* bp = S.body + tank;
    const double pre = finalize_preload(S, T, tank);
    const double rx = __shfl_sync(0xffffffffu, pre, 0), ry = __shfl_sync(0xffffffffu, pre, 1);
    const double th = __shfl_sync(0xffffffffu, pre, 2), vx = __shfl_sync(0xffffffffu, pre, 3);
    const double vy = __shfl_sync(0xffffffffu, pre, 4), w = __shfl_sync(0xffffffffu, pre, 5);
    double c = __shfl_sync(0xffffffffu, pre, 6), sn = __shfl_sync(0xffffffffu, pre, 7);
    double tau_c = __shfl_sync(0xffffffffu, pre, 8);
    const double ux = __shfl_sync(0xffffffffu, pre, 9), uy = __shfl_sync(0xffffffffu, pre, 10);
    const double ut = __shfl_sync(0xffffffffu, pre, 11);
    const double cJ = __shfl_sync(0xffffffffu, pre, 12), cw = __shfl_sync(0xffffffffu, pre, 13);
    const double cxi = __shfl_sync(0xffffffffu, pre, 14), ref = __shfl_sync(0xffffffffu, pre, 15);
    const long long sw = __double_as_longlong(__shfl_sync(0xffffffffu, pre, 16));
    double* const yout = (double*)__double_as_longlong(__shfl_sync(0xffffffffu, pre, 17));
    const long long step0 = __double_as_longlong(__shfl_sync(0xffffffffu, pre, 18));
    const long long ystride = __double_as_longlong(__shfl_sync(0xffffffffu, pre, 19));
    const long long step = __double_as_longlong(__shfl_sync(0xffffffffu, pre, 20));
    const bool ctrl_on = (sw & 1) != 0, body_fixed = (sw & 2) != 0;
    const bool sample = !eval && (step % T.outer_every) == 0;
    const int nbuf = (int)(step & 1) ^ 1;
    double* y = nullptr;
    if (sample) {
        const long long oe = T.outer_every;
        y = yout ? yout + tank * ystride + (step / oe - (step0 + oe - 1) / oe) * SPH_NY : nullptr;
        if (ctrl_on) {  // Eq. 28 under zero-order hold, from the state before the step
            const double Jc = cJ > 0.0 ? cJ : T.J_body;
            tau_c = Jc * cw * cw * (ref - th) - 2.0 * cxi * Jc * cw * w;
            if (lane == 0) bp->tau_c = tau_c;
        }
        if (y && lane < 6) y[lane] = pick(lane, 0, rx, ry, th, vx, vy, w);
    }
    const double tau = ut + (ctrl_on ? tau_c : 0.0);
    // output l = A + B F_which: 0..5 r', theta', rdot', thetadot'; 6, 7 r' - W
    // (the origin of the next grid); in an evaluation 0..5 are F_b, T_b and
    // the accelerations of Eq. 20
    const double dt = T.dt_d, im = T.inv_m_body, iJ = T.inv_J_body;
    const int comp = lane % 3;  // F_x, F_y or T_b for lanes 0..7 (0, 1, 2, 0, 1, 2, 0, 1)
    const int k = lane < 8 ? lane : 0;
    double A, B;
    if (eval) {
        const double u3 = sel3(comp, ux, uy, tau), i3 = comp == 2 ? iJ : im;
        A = k < 3 ? 0.0 : u3 * i3;
        B = k < 3 ? 1.0 : i3;
    } else if (body_fixed) {
        A = pick(k, 0, rx, ry, th, vx, vy, w, rx - T.W, ry - T.W);
        B = 0.0;
    } else {
        const double x0 = sel3(comp, rx, ry, th), v0 = sel3(comp, vx, vy, w);
        const double u3 = sel3(comp, ux, uy, tau), i3 = comp == 2 ? iJ : im;
        const double Av = v0 + dt * (u3 * i3), Bv = dt * i3;  // velocity
        const bool vel = (k >= 3 && k <= 5);
        A = vel ? Av : x0 + dt * Av - (k >= 6 ? T.W : 0.0);
        B = vel ? Bv : dt * Bv;
    }
    // rotation of (cos, sin) by dtheta = dt thetadot' = Ad + Bd T_b, with
    // (cos, sin) first brought back to unit norm (off the dependent chain)
    double Ad = 0.0, Bd = 0.0;
    if (!eval && !body_fixed) {
        Ad = dt * (w + dt * (tau * iJ));
        Bd = dt * dt * iJ;
        const double f = 1.5 - 0.5 * (c * c + sn * sn);
        c *= f;
        sn *= f;
    }
    const double X = lane == 9 ? sn : c, Yr = lane == 9 ? c : -sn;  // lane 8: cos', lane 9: sin'

    pdl_wait();
    // the next density pass may be placed now: every tile of the force pass
    // has finished, so its CTAs take no SM slot that this step still needs
    pdl_trigger();
    double vq = 0.0;
    if (lane < 5) {  // each lane converts its own sum
        vq = (double)(long long)__ldcg(&bp->acc[lane]) * kFixUnit;
        bp->acc[lane] = 0ull;  // cleared for the next force pass
    }
    const double Fx = __shfl_sync(0xffffffffu, vq, 0), Fy = __shfl_sync(0xffffffffu, vq, 1);
    const double Tq = __shfl_sync(0xffffffffu, vq, 2), Cx = __shfl_sync(0xffffffffu, vq, 3);
    const double Cy = __shfl_sync(0xffffffffu, vq, 4);
    const double lin = fma(B, sel3(comp, Fx, Fy, Tq), A);
    double v = lin;
    if (!eval && !body_fixed) {
        const double d = fma(Bd, Tq, Ad), d2 = d * d;
        double cd, sd;
        if (fabs(d) <= 1e-4) {  // first omitted terms d^4 / 24, d^5 / 120 below 1e-16 relative
            cd = fma(-0.5, d2, 1.0);
            sd = fma(d * d2, -1.0 / 6.0, d);
        } else if (fabs(d) <= 1e-2) {
            cd = 1.0 - d2 * (0.5 - d2 * (1.0 / 24.0 - d2 * (1.0 / 720.0)));
            sd = d * (1.0 - d2 * (1.0 / 6.0 - d2 * (1.0 / 120.0 - d2 * (1.0 / 5040.0))));
        } else {
            double s1, c1;
            sincos(d, &s1, &c1);
            cd = c1;
            sd = s1;
        }
        if (lane == 8 || lane == 9) v = fma(X, cd, Yr * sd);
    } else if (lane == 8 || lane == 9) {
        v = X;  // unchanged angle
    }
    if (sample && y && lane >= 6 && lane < SPH_NY) {
        double o = sel3(lane - 6, Fx, Fy, Tq);
        if (lane == 9) o = T.n_f ? Cx / T.n_f : 0.0;
        if (lane == 10) o = T.n_f ? Cy / T.n_f : 0.0;
        y[lane] = o;
    }
    if (eval) {
        if (E.body && lane < 6) E.body[6 * tank + lane] = v;
    } else {
        if (lane < 2) bp->anchor[nbuf][lane] = lane ? ry : rx;  // the state before the step
        // the leading doubles of BodyDev: r, theta, rdot, thetadot (lanes 0-5), cos, sin (lanes 8, 9)
        if (!body_fixed && (lane < 6 || lane == 8 || lane == 9)) reinterpret_cast<double*>(bp)[lane < 6 ? lane : lane - 2] = v;
        // FP32 forms: two-float splits (dc, ds from lanes 8, 9; drx, dry from
        // 0, 1), rounded values (fc, fs; frx, fry; fo_next from 6, 7; fvx, fvy, fw from 3-5)
        const float hi = (float)v;
        const float lo = (float)(v - (double)hi);
        if (lane == 8 || lane == 9) {
            (&bp->dc)[lane - 8] = make_float2(hi, lo);
            (&bp->fc)[lane - 8] = hi;
        } else if (lane < 2) {
            (&bp->drx)[lane] = make_float2(hi, lo);
            (&bp->frx)[lane] = hi;
        } else if (lane == 6 || lane == 7) {
            bp->fo_next[lane - 6] = hi;
        } else if (lane >= 3 && lane < 6) {
            (&bp->fvx)[lane - 3] = hi;
        }
    }
    if (lane != 0) return;
    if (S.B == 1) {  // the only tank: its step is the pass's (visible when the kernel completes)
        if (!eval) run->step = step + 1;
        return;
    }
    fence_acq_rel();
    const unsigned prev = atomicAdd(&run->tanks_done, 1u);
    if (prev == (unsigned)S.B - 1) {
        if (!eval) run->step = step + 1;
        run->tanks_done = 0;
    }
}

// ---------------------------------------------------------------------------
// State transfer and bookkeeping kernels
// ---------------------------------------------------------------------------

// Bins flat particles [N, 4] (tanks concatenated) into grid buffer `buf`,
// anchored at each tank's stored anchor for that buffer.
__global__ void bin_flat_kernel(SimDev S, const float4* __restrict__ xv, const float4* __restrict__ lo,
                                const int* __restrict__ part_tank, int n, int buf)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int t = part_tank[i];
    const TankDev& T = S.tank[t];
    const BodyDev& b = S.body[t];
    const float4 p = xv[i];
    const float ox = (float)(b.anchor[buf][0] - T.W), oy = (float)(b.anchor[buf][1] - T.W);
    bool out = false;
    const int cx = cell_coord(p.x, ox, T.inv_cell, T.G, &out), cy = cell_coord(p.y, oy, T.inv_cell, T.G, &out);
    const float ex = p.x - (ox + T.Wf), ey = p.y - (oy + T.Wf);
    int flags = (out || fmaf(ex, ex, ey * ey) > T.cover2) ? SPH_FLAG_ESCAPED : 0;
    if (!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w))) flags |= SPH_FLAG_NAN;
    const int cell = T.cell_base + cy * T.G + cx;
    const int slot = atomicAdd(&S.count[buf][cell], 1);
    if ((unsigned)slot < (unsigned)kCap) {
        S.pv[buf][cell * kCap + slot] = p;
        S.lo[buf][cell * kCap + slot] = lo ? lo[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        S.pid[buf][cell * kCap + slot] = i;
    } else {
        flags |= SPH_FLAG_CELL_FULL;
    }
    if (flags) atomicOr(&S.body[t].flags, flags);
}

// Writes the body state [B, 6] and derived quantities; anchors buffer `buf`.
__global__ void set_body_kernel(SimDev S, const double* __restrict__ body, int buf)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S.B) return;
    BodyDev& b = S.body[t];
    const TankDev& T = S.tank[t];
    const double* s = body + 6 * t;
    b.r[0] = s[0];
    b.r[1] = s[1];
    b.th = s[2];
    b.v[0] = s[3];
    b.v[1] = s[4];
    b.w = s[5];
    sincos(b.th, &b.s, &b.c);
    b.anchor[buf][0] = s[0];
    b.anchor[buf][1] = s[1];
    b.tau_c = 0.0;
    b.done = 0;
    for (int q = 0; q < 5; ++q) b.acc[q] = 0ull;
    b.dc = df_split(b.c);
    b.ds = df_split(b.s);
    b.drx = df_split(b.r[0]);
    b.dry = df_split(b.r[1]);
    b.fvx = (float)b.v[0];
    b.fvy = (float)b.v[1];
    b.fw = (float)b.w;
    b.fc = (float)b.c;
    b.fs = (float)b.s;
    b.frx = (float)b.r[0];
    b.fry = (float)b.r[1];
    b.fo_next[0] = (float)(b.r[0] - T.W);
    b.fo_next[1] = (float)(b.r[1] - T.W);
}

__global__ void get_body_kernel(SimDev S, double* __restrict__ body)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S.B) return;
    const BodyDev& b = S.body[t];
    double* o = body + 6 * t;
    o[0] = b.r[0];
    o[1] = b.r[1];
    o[2] = b.th;
    o[3] = b.v[0];
    o[4] = b.v[1];
    o[5] = b.w;
}

// One warp per cell: scatter the occupied slots of buffer `buf` to [N, 4]
// (the hi parts of the state; its lo parts to lo when given).
__global__ void gather_state_kernel(SimDev S, float4* __restrict__ xv, float4* __restrict__ lo, int n_cells_total,
                                    int buf)
{
    const int cell = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (cell >= n_cells_total) return;
    const int n = min(S.count[buf][cell], kCap);
    if (lane < n) {
        const int gs = cell * kCap + lane;
        const int id = S.pid[buf][gs];
        if (xv) xv[id] = S.pv[buf][gs];
        if (lo) lo[id] = S.lo[buf][gs];
    }
}

// Tangent state transfer: one warp per cell; a particle's tangent lives in
// the slot of the particle itself.  xv == NULL sets a zero tangent.
__global__ void scatter_tangent_kernel(SimDev S, const float4* __restrict__ txv, int n_cells_total, int buf)
{
    const int cell = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (cell >= n_cells_total) return;
    const int n = min(S.count[buf][cell], kCap);
    if (lane < n) {
        const int gs = cell * kCap + lane;
        S.tpv[buf][gs] = txv ? txv[S.pid[buf][gs]] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__global__ void gather_tangent_kernel(SimDev S, float4* __restrict__ txv, int n_cells_total, int buf)
{
    const int cell = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (cell >= n_cells_total) return;
    const int n = min(S.count[buf][cell], kCap);
    if (lane < n) {
        const int gs = cell * kCap + lane;
        txv[S.pid[buf][gs]] = S.tpv[buf][gs];
    }
}

// Body tangent [B, 6] in (NULL: zero) / out.
__global__ void body_tangent_kernel(SimDev S, const double* __restrict__ in, double* __restrict__ out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= S.B) return;
    BodyDev& b = S.body[t];
    if (out) {
        double* o = out + 6 * t;
        o[0] = b.tr[0];
        o[1] = b.tr[1];
        o[2] = b.tth;
        o[3] = b.tv[0];
        o[4] = b.tv[1];
        o[5] = b.tw;
        return;
    }
    const double* s = in ? in + 6 * t : nullptr;
    b.tr[0] = s ? s[0] : 0.0;
    b.tr[1] = s ? s[1] : 0.0;
    b.tth = s ? s[2] : 0.0;
    b.tv[0] = s ? s[3] : 0.0;
    b.tv[1] = s ? s[4] : 0.0;
    b.tw = s ? s[5] : 0.0;
    b.ftr[0] = (float)b.tr[0];
    b.ftr[1] = (float)b.tr[1];
    b.ftth = (float)b.tth;
    b.ftv[0] = (float)b.tv[0];
    b.ftv[1] = (float)b.tv[1];
    b.ftw = (float)b.tw;
}

__global__ void set_run_kernel(RunDev* run, RunDev desc)
{
    desc.step = run->step;
    desc.step0 = run->step;
    desc.tanks_done = 0;
    desc.next_buf = (int)(run->step & 1);
    *run = desc;
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------
template <typename... KArgs, typename... Args>
static cudaError_t launch(void (*k)(KArgs...), int grid, int block, cudaStream_t st, bool pdl, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

template <int TX, int TY>
static cudaError_t launch_tile_phase(const SimDev& S, const EvalOut& E, int eval, int n_tiles, int phase,
                                     cudaStream_t st, bool pdl, bool tan, bool chained)
{
    using Sh = Shape<TX, TY>;
    if (tan) {
        if constexpr (TX * TY <= 32) {  // the tangent staging of 8x8 tiles exceeds static shared memory
            if (phase == 0) return launch(density_kernel<TX, TY, true>, n_tiles, Sh::THREADS, st, pdl, S, E, eval, 0);
            if (phase == 2) return cudaSuccess;  // the tangent force pass updates the body itself
            return launch(force_kernel<TX, TY, true>, n_tiles, Sh::THREADS, st, pdl, S, E, eval);
        } else {
            return cudaErrorInvalidValue;
        }
    }
    if (phase == 0)
        return launch(density_kernel<TX, TY, false>, n_tiles, Sh::THREADS, st, pdl, S, E, eval, (pdl && chained) ? 1 : 0);
    if (phase == 1) return launch(force_kernel<TX, TY, false>, n_tiles, Sh::THREADS, st, pdl, S, E, eval);
    return launch(body_kernel, (S.B + kBodyWarps - 1) / kBodyWarps, 32 * kBodyWarps, st, pdl, S, E, eval);
}

template <int TX, int TY>
static size_t record_bytes(int n_tiles)
{
    return (size_t)n_tiles * sizeof(StageRec<TX, TY>);
}

size_t stage_record_bytes(const int* n_tiles)
{
    size_t b = record_bytes<2, 2>(n_tiles[1]);
    b = std::max(b, record_bytes<4, 2>(n_tiles[2]));
    b = std::max(b, record_bytes<4, 4>(n_tiles[3]));
    b = std::max(b, record_bytes<8, 4>(n_tiles[4]));
    return std::max(b, record_bytes<8, 8>(n_tiles[5]));
}

void tile_dims(int code, int* tx, int* ty)
{
    static const int T[SPH_TILE_COUNT][2] = {{2, 2}, {4, 2}, {4, 4}, {8, 4}, {8, 8}};
    *tx = T[code - 1][0];
    *ty = T[code - 1][1];
}

// phase 0: density pass, 1: force pass, 2: body update (none in the tangent variant)
cudaError_t launch_phase(const SimDev& S, const EvalOut& E, int eval, int tile_code, int n_tiles, int phase,
                         cudaStream_t st, bool pdl, bool tan, bool chained)
{
    switch (tile_code) {
    case 1: return launch_tile_phase<2, 2>(S, E, eval, n_tiles, phase, st, pdl, tan, chained);
    case 2: return launch_tile_phase<4, 2>(S, E, eval, n_tiles, phase, st, pdl, tan, chained);
    case 3: return launch_tile_phase<4, 4>(S, E, eval, n_tiles, phase, st, pdl, tan, chained);
    case 4: return launch_tile_phase<8, 4>(S, E, eval, n_tiles, phase, st, pdl, tan, chained);
    case 5: return launch_tile_phase<8, 8>(S, E, eval, n_tiles, phase, st, pdl, tan, chained);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step(const SimDev& S, const EvalOut& E, int eval, int tile_code, int n_tiles, cudaStream_t st,
                        bool pdl, bool tan, bool chained)
{
    for (int ph = 0; ph < 3; ++ph) {
        cudaError_t e = launch_phase(S, E, eval, tile_code, n_tiles, ph, st, pdl, tan, chained);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_bin_flat(const SimDev& S, const float* xv, const float* lo, const int* part_tank, int n, int buf,
                            cudaStream_t st)
{
    if (n > 0)
        bin_flat_kernel<<<(n + 255) / 256, 256, 0, st>>>(S, (const float4*)xv, (const float4*)lo, part_tank, n, buf);
    return cudaGetLastError();
}

cudaError_t launch_set_body(const SimDev& S, const double* body, int buf, cudaStream_t st)
{
    set_body_kernel<<<(S.B + 127) / 128, 128, 0, st>>>(S, body, buf);
    return cudaGetLastError();
}

cudaError_t launch_get_state(const SimDev& S, float* xv, float* lo, double* body, int n_cells_total, int buf,
                             cudaStream_t st)
{
    if ((xv || lo) && n_cells_total > 0)
        gather_state_kernel<<<(n_cells_total + 7) / 8, 256, 0, st>>>(S, (float4*)xv, (float4*)lo, n_cells_total, buf);
    if (body) get_body_kernel<<<(S.B + 127) / 128, 128, 0, st>>>(S, body);
    return cudaGetLastError();
}

cudaError_t launch_set_run(RunDev* run, const RunDev& desc, cudaStream_t st)
{
    set_run_kernel<<<1, 1, 0, st>>>(run, desc);
    return cudaGetLastError();
}

cudaError_t launch_tangent_state(const SimDev& S, const float* txv_in, float* txv_out, const double* tb_in,
                                 double* tb_out, int n_cells_total, int buf, cudaStream_t st)
{
    const int grid = (n_cells_total + 7) / 8;
    if (txv_out) {
        if (n_cells_total > 0) gather_tangent_kernel<<<grid, 256, 0, st>>>(S, (float4*)txv_out, n_cells_total, buf);
        if (tb_out) body_tangent_kernel<<<(S.B + 127) / 128, 128, 0, st>>>(S, nullptr, tb_out);
    } else {
        if (n_cells_total > 0) scatter_tangent_kernel<<<grid, 256, 0, st>>>(S, (const float4*)txv_in, n_cells_total, buf);
        body_tangent_kernel<<<(S.B + 127) / 128, 128, 0, st>>>(S, tb_in, nullptr);
    }
    return cudaGetLastError();
}

}  // namespace sph
