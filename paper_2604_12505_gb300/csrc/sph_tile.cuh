// sph_tile.cuh -- tile staging shared by the step kernels and the adjoint
// kernels: a tile of TX x TY grid cells plus a one-cell halo is gathered into
// shared memory, each cell ordered by x (then particle index), and every own
// particle visits its 3x3 cells there and the ghost cells around it.
#pragma once

#include <climits>

#include "sph_common.cuh"

namespace sph {

template <int TX, int TY>
struct Shape {
    static constexpr int SX = TX + 2;
    static constexpr int SY = TY + 2;
    static constexpr int NC = SX * SY;       // staged cells (tile + halo)
    static constexpr int MAXS = NC * 12;     // staged particles (1.8x the lattice mean)
    static constexpr int MAXOWN = TX * TY * 12;  // own particles with a recorded neighbour list
    static constexpr int THREADS = (TX * TY >= 32) ? 256 : (TX * TY >= 16 ? 128 : (TX * TY >= 8 ? 64 : 32));
    // resident CTAs per SM asked of the compiler: the particle loops fit in 72
    // (force; 64 for 256-thread tiles) and 64 (density) registers, and the
    // rarely run staging and reduction code must not raise that (a 4x4 tile
    // keeps 7 and 8 CTAs per SM, an 8x4 tile 4 and 4)
    static constexpr int FORCE_MIN_CTAS = THREADS >= 256 ? 4 : 65536 / (THREADS * 72);
    static constexpr int DENSITY_MIN_CTAS = 65536 / (THREADS * 64);
};

__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Release/acquire fence at GPU scope: orders this thread's earlier memory
// accesses before its later ones as seen by other CTAs (lighter than the
// sequentially consistent __threadfence).  With a relaxed atomic counter it
// publishes data (store; fence; atomic) and consumes it (atomic; fence; load).
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Shared-memory staging of a tile and its halo
// ---------------------------------------------------------------------------
template <int TX, int TY, bool RHO, bool TAN = false>
struct Stage {
    using Sh = Shape<TX, TY>;
    int start[Sh::NC + 1];
    int own_row[TY + 1];
    float4 pv[Sh::MAXS];
    float2 plo[Sh::MAXS];         // low parts (x_lo, y_lo) of the staged positions
    int pid[Sh::MAXS];
    int pid_in[Sh::MAXS];         // particle index in global slot order (before ordering)
    unsigned int key_in[Sh::MAXS];  // ordering key of x in global slot order
    int slot[Sh::MAXS];
    unsigned char cell[Sh::MAXS];
    float2 rho[RHO ? Sh::MAXS : 1];
    float2 vlo[RHO ? Sh::MAXS : 1];           // low parts (vx_lo, vy_lo) of the velocities (force pass)
    float4 tpv[TAN ? Sh::MAXS : 1];           // tangent (dx, dy, dvx, dvy)
    float2 trho[(TAN && RHO) ? Sh::MAXS : 1];  // tangent (d rho, d(P / rho^2))
};

// Key with the IEEE-754 total order of x (NaNs included, -0 below +0): with
// the particle index as a tie-break the ranks inside a cell always form a
// permutation, whatever the values.
__device__ __forceinline__ unsigned int order_key(float x)
{
    const unsigned int u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Loads the counts, scans them, and gathers the particles of the (TX+2) x
// (TY+2) staged cells, each cell ordered by x with the particle index
// breaking ties (a deterministic order, whatever order the slots were
// claimed in).  Returns false (uniformly over the block) if the staged set
// does not fit.  The counts and the state are read through L2 (ld.global.cg):
// the density pass may stage before its grid dependency, from data that an
// earlier, completed grid wrote.
template <int TX, int TY, bool RHO, bool TAN>
__device__ bool stage_tile(const SimDev& S, const TankDev& T, int buf, int cx0, int cy0, Stage<TX, TY, RHO, TAN>& sm)
{
    using Sh = Shape<TX, TY>;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int* __restrict__ count = S.count[buf];
    for (int c = tid; c < Sh::NC; c += blockDim.x) {
        int ix = cx0 - 1 + c % Sh::SX, iy = cy0 - 1 + c / Sh::SX;
        int n = 0;
        if (ix >= 0 && ix < T.G && iy >= 0 && iy < T.G) n = min(max(__ldcg(count + T.cell_base + iy * T.G + ix), 0), kCap);
        sm.start[c] = n;
    }
    __syncthreads();
    if (warp == 0) {
        int carry = 0;
        for (int base = 0; base < Sh::NC; base += 32) {
            int c = base + lane;
            int v = c < Sh::NC ? sm.start[c] : 0;
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (c < Sh::NC) sm.start[c] = carry + incl - v;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) sm.start[Sh::NC] = carry;
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int r = 0; r < TY; ++r) {
            sm.own_row[r] = acc;
            int row = (r + 1) * Sh::SX;
            acc += sm.start[row + TX + 1] - sm.start[row + 1];
        }
        sm.own_row[TY] = acc;
    }
    const int total = sm.start[Sh::NC];
    int own = 0;  // own particles (every thread from the scanned starts; thread 0 also writes own_row)
    for (int r = 0; r < TY; ++r) own += sm.start[(r + 1) * Sh::SX + TX + 1] - sm.start[(r + 1) * Sh::SX + 1];
    if (own == 0) {
        // nothing to stage (the halo serves only the tile's own particles):
        // the stage is left empty, every cell start 0, so that no caller
        // reads staged particles that were not gathered
        __syncthreads();  // every thread has read the starts
        for (int c = tid; c <= Sh::NC; c += blockDim.x) sm.start[c] = 0;
        __syncthreads();
        return true;
    }
    if (total > Sh::MAXS) {
        if (tid == 0) atomicOr(&S.body[S.tiles[blockIdx.x].x].flags, SPH_FLAG_STAGE_FULL);
        __syncthreads();
        return false;
    }
    // pass 1: every staged slot at once -- its cell (binary search) and particle index
    for (int e = tid; e < total; e += blockDim.x) {
        int lo = 0, hi = Sh::NC;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (sm.start[mid] <= e) lo = mid; else hi = mid;
        }
        const int ix = cx0 - 1 + lo % Sh::SX, iy = cy0 - 1 + lo / Sh::SX;
        sm.cell[e] = (unsigned char)lo;
        const int gs = (T.cell_base + iy * T.G + ix) * kCap + (e - sm.start[lo]);
        sm.pid_in[e] = __ldcg(S.pid[buf] + gs);
        sm.key_in[e] = order_key(__ldcg(&S.pv[buf][gs].x));
    }
    __syncthreads();
    // pass 2: rank by (x, particle index) inside the cell and gather into
    // that order (reads only cell[], pid_in[], x_in[] and start[], which pass 2
    // never writes)
#pragma unroll 2
    for (int e = tid; e < total; e += blockDim.x) {
        const int c = sm.cell[e];
        const int a = sm.start[c];
        const int id = sm.pid_in[e];
        const unsigned int ke = sm.key_in[e];
        int rank = 0;
        for (int j = a; j < sm.start[c + 1]; ++j) {
            const unsigned int kj = sm.key_in[j];
            rank += (kj < ke) || (kj == ke && sm.pid_in[j] < id);
        }
        const int d = a + rank;
        const int ix = cx0 - 1 + c % Sh::SX, iy = cy0 - 1 + c / Sh::SX;
        const int gs = (T.cell_base + iy * T.G + ix) * kCap + (e - a);
        sm.pv[d] = __ldcg(S.pv[buf] + gs);
        const float4 lo = __ldcg(S.lo[buf] + gs);
        sm.plo[d] = make_float2(lo.x, lo.y);
        if (RHO) {
            sm.rho[d] = S.rhoP[gs];
            sm.vlo[d] = make_float2(lo.z, lo.w);
        }
        if constexpr (TAN) {
            sm.tpv[d] = S.tpv[buf][gs];
            if (RHO) sm.trho[d] = S.trho[gs];
        }
        sm.pid[d] = id;
        sm.slot[d] = gs;
    }
    __syncthreads();
    return true;
}

// The staged order of a tile as the density pass leaves it, so that the
// force pass stages the same particles in the same order (which the
// neighbour lists index) without counting, scanning and ranking again: per
// staged cell the first staged index (start[NC] = total; -1: the tile did
// not fit), per staged particle its global slot and staged cell (written only
// when the tile has own particles).
template <int TX, int TY>
struct StageRec {
    int start[Shape<TX, TY>::NC + 1];
    int slot[Shape<TX, TY>::MAXS];
    unsigned char cell[Shape<TX, TY>::MAXS];
};

template <int TX, int TY>
__device__ __forceinline__ StageRec<TX, TY>* stage_record(const SimDev& S, int tile)
{
    return reinterpret_cast<StageRec<TX, TY>*>(S.srec) + tile;
}

// Writes the record of the tile just staged (all threads).
template <int TX, int TY, bool RHO, bool TAN>
__device__ __forceinline__ void save_stage(const Stage<TX, TY, RHO, TAN>& sm, bool staged, StageRec<TX, TY>* rec)
{
    using Sh = Shape<TX, TY>;
    if (!staged) {
        if (threadIdx.x == 0) rec->start[Sh::NC] = -1;
        return;
    }
    for (int c = threadIdx.x; c <= Sh::NC; c += blockDim.x) rec->start[c] = sm.start[c];
    if (sm.own_row[TY] == 0) return;
    const int total = sm.start[Sh::NC];
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        rec->slot[i] = sm.slot[i];
        rec->cell[i] = sm.cell[i];
    }
}

// Stages a tile from its record: one round of loads for the cell starts and
// (speculatively, the whole list) the slots, one for the particle state.
// Returns false (uniformly) if the density pass could not stage the tile.
template <int TX, int TY, bool TAN>
__device__ __forceinline__ bool stage_from_record(const SimDev& S, int tank, int buf, const StageRec<TX, TY>* rec,
                                                  Stage<TX, TY, true, TAN>& sm)
{
    using Sh = Shape<TX, TY>;
    constexpr int KPT = (Sh::MAXS + Sh::THREADS - 1) / Sh::THREADS;
    const int tid = threadIdx.x;
    int r_slot[KPT], r_cell[KPT];
    for (int c = tid; c <= Sh::NC; c += Sh::THREADS) sm.start[c] = __ldcg(rec->start + c);
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
        const int i = tid + q * Sh::THREADS;
        r_slot[q] = i < Sh::MAXS ? __ldcg(rec->slot + i) : 0;
        r_cell[q] = i < Sh::MAXS ? (int)__ldcg(rec->cell + i) : 0;
    }
    __syncthreads();
    const int total = sm.start[Sh::NC];
    if (total < 0) {
        if (tid == 0) atomicOr(&S.body[tank].flags, SPH_FLAG_STAGE_FULL);
        __syncthreads();
        return false;
    }
    if (tid == 0) {
        int acc = 0;
        for (int r = 0; r < TY; ++r) {
            sm.own_row[r] = acc;
            const int row = (r + 1) * Sh::SX;
            acc += sm.start[row + TX + 1] - sm.start[row + 1];
        }
        sm.own_row[TY] = acc;
    }
    __syncthreads();
    if (sm.own_row[TY] == 0) return true;  // no own particle: the slot list was not written
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
        const int i = tid + q * Sh::THREADS;
        if (i < total) {
            const int gs = r_slot[q];
            sm.pv[i] = S.pv[buf][gs];
            const float4 lo = S.lo[buf][gs];
            sm.plo[i] = make_float2(lo.x, lo.y);
            sm.vlo[i] = make_float2(lo.z, lo.w);
            sm.rho[i] = S.rhoP[gs];
            if constexpr (TAN) {
                sm.tpv[i] = S.tpv[buf][gs];
                sm.trho[i] = S.trho[gs];
            }
            sm.pid[i] = S.pid[buf][gs];
            sm.slot[i] = gs;
            sm.cell[i] = (unsigned char)r_cell[q];
        }
    }
    __syncthreads();
    return true;
}

// First staged index in [lo, hi) whose x is not below v (a cell is sorted by
// x; with a NaN present the answer is only some index in [lo, hi]).
template <class Stg>
__device__ __forceinline__ int lower_x(const Stg& sm, int lo, int hi, float v)
{
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sm.pv[mid].x < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Smem index of the t-th own particle (own cells are TY contiguous row runs).
// The fluid neighbours that the density pass recorded for own particle t of
// a tile: for each of the three stencil rows, in row order, the staged
// indices zl - k for the set bits k of the row's mask (zl the row's last
// candidate), highest bit first -- the order in which that pass met them.  Returns false when nothing was recorded
// (t beyond the record, or a row of more than kNbrRowBits candidates); the
// caller then scans the stencil.
template <int MAXOWN, class F>
__device__ __forceinline__ bool for_recorded_neighbours(const SimDev& S, int tile, int t, F&& pair)
{
    if (t >= MAXOWN || S.nbn[(size_t)tile * MAXOWN + t] == kNbrNone) return false;
    const size_t o = (size_t)tile * (3 * MAXOWN) + t;
    unsigned int m[3];
    int a[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        m[r] = S.nbm[o + r * MAXOWN];
        a[r] = S.nba[o + r * MAXOWN];
    }
    // one loop over all recorded neighbours (lanes diverge only by their
    // totals), moving to the next non-empty row when a row's bits run out
    const int n = __popc(m[0]) + __popc(m[1]) + __popc(m[2]);
    unsigned int b = m[0], b1 = m[1], b2 = m[2];
    int ar = a[0], a1 = a[1], a2 = a[2];
    for (int k = 0; k < n; ++k) {
        if (b == 0) {
            b = b1; ar = a1; b1 = b2; a1 = a2; b2 = 0u;
            if (b == 0) { b = b1; ar = a1; b1 = 0u; }
        }
        const int lz = __clz(b);  // the highest set bit: the earliest candidate left
        const int j = ar - 31 + lz;
        b &= 0x7fffffffu >> lz;
        pair(j);
    }
    return true;
}

template <int TX, int TY, bool RHO, bool TAN>
__device__ __forceinline__ int own_index(int t, const Stage<TX, TY, RHO, TAN>& sm)
{
    using Sh = Shape<TX, TY>;
    int r = 0;
#pragma unroll
    for (int q = 1; q < TY; ++q) r += (t >= sm.own_row[q]);
    return sm.start[(r + 1) * Sh::SX + 1] + (t - sm.own_row[r]);
}

// The body-frame ghost cell of a fluid particle, or false when no ghost lies
// within its reach (inside the ghost-free disc, or off the grid); (ex, ey) is
// the body-frame position.  The body-frame position only selects cells, so
// FP32 suffices; the operations are explicitly rounded, so that every call
// site selects the same cell.
__device__ __forceinline__ bool ghost_cell(const TankDev& T, float xi, float yi, float bc, float bs, float brx,
                                           float bry, int& gx, int& gy, float& ex, float& ey)
{
    const float px = __fsub_rn(xi, brx), py = __fsub_rn(yi, bry);
    ex = __fadd_rn(__fmul_rn(bc, px), __fmul_rn(bs, py));
    ey = __fsub_rn(__fmul_rn(bc, py), __fmul_rn(bs, px));
    if (__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)) < T.ghost_rin2) return false;
    const float fx = floorf(__fmul_rn(__fsub_rn(ex, T.g_orig), T.g_inv_cell));
    const float fy = floorf(__fmul_rn(__fsub_rn(ey, T.g_orig), T.g_inv_cell));
    if (!(fx >= -1.0f && fx <= (float)T.G && fy >= -1.0f && fy <= (float)T.G)) return false;  // off the grid or NaN
    gx = (int)fx;
    gy = (int)fy;
    return true;
}

// Visits the ghosts of the 3x3 body-frame ghost cells around a fluid
// particle, reading the ghost-cell starts from global memory.
template <class F>
__device__ __forceinline__ void for_ghosts(const SimDev& S, const TankDev& T, float xi, float yi, float bc, float bs,
                                           float brx, float bry, F&& f)
{
    int gx, gy;
    float ex, ey;
    if (!ghost_cell(T, xi, yi, bc, bs, brx, bry, gx, gy, ex, ey)) return;
    const int x0 = max(gx - 1, 0), x1 = min(gx + 1, T.G - 1);
    if (x0 > x1) return;
    for (int yy = max(gy - 1, 0); yy <= min(gy + 1, T.G - 1); ++yy) {
        const int row = T.gcell_base + yy * T.G;
        const int a = __ldg(S.gstart + row + x0), b = __ldg(S.gstart + row + x1 + 1);
        for (int j = a; j < b; ++j) f(j);
    }
}

// The body state Eq. 21 needs, in the FP32 and two-float forms the body
// update writes.
struct GhostFrame {
    float2 dc, ds, drx, dry;
    float fvx, fvy, fw;
};

__device__ __forceinline__ GhostFrame ghost_frame(const BodyDev& b)
{
    return GhostFrame{b.dc, b.ds, b.drx, b.dry, b.fvx, b.fvy, b.fw};
}

// Eq. 21 for one ghost in two-float arithmetic: arm = R(theta) r_g^B,
// r_g = r + arm, v_g = rdot + thetadot z x arm.  gp = (x_hi, y_hi, x_lo, y_lo),
// gv = (v_x, v_y, arm_x, arm_y).
__device__ __forceinline__ void ghost_world(const GhostFrame& f, float4 gb, float4& gp, float4& gv)
{
    const float2 bx = make_float2(gb.x, gb.y), by = make_float2(gb.z, gb.w);
    const float2 sby = df_mul(f.ds, by);
    const float2 ax = df_add(df_mul(f.dc, bx), make_float2(-sby.x, -sby.y));
    const float2 ay = df_add(df_mul(f.ds, bx), df_mul(f.dc, by));
    const float2 gx = df_add(f.drx, ax), gy = df_add(f.dry, ay);
    const float armx = ax.x + ax.y, army = ay.x + ay.y;
    gp = make_float4(gx.x, gy.x, gx.y, gy.y);
    gv = make_float4(f.fvx - f.fw * army, f.fvy + f.fw * armx, armx, army);
}

// ---------------------------------------------------------------------------
// Ghost staging: the ghosts that a tile's wall particles reach, in shared
// memory, so that the per-particle ghost loops read neither the ghost-cell
// starts nor the ghosts from global memory (each a dependent L2 round trip)
// ---------------------------------------------------------------------------
constexpr int kGhostMax = 256;  // staged ghosts per tile
constexpr int kGhostDim = 16;   // staged ghost-cell rows and columns per tile

template <bool ON>
struct GhostStage {
    float4 gp[ON ? kGhostMax : 1];                    // world position (x_hi, y_hi, x_lo, y_lo)
    float4 gv[ON ? kGhostMax : 1];                    // (v_x, v_y, arm_x, arm_y)
    float bx[ON ? kGhostMax : 1];                     // body-frame x (a row of cells is sorted by it)
    int tab[ON ? kGhostDim : 1][kGhostDim + 1];      // ghost-cell starts of the staged cells (global index)
    int base[kGhostDim];                             // staged index of ghost g of row r: base[r] + g
    int pre[kGhostDim + 1];                          // first staged index of each row
    int box[4];                                      // first, last staged cell column; first, last row
};

enum { kGhostsNone = 0, kGhostsStaged = 1, kGhostsGlobal = 2 };

// Stages the ghosts around the wall particles among the tile's own particles
// (ghost-cell rows and columns of the bounding box of their 3x3 ghost cells).
// FILL: computes each ghost's world position and velocity (Eq. 21) and also
// stores them to S.gpos / S.gvel for the force pass and the adjoint;
// otherwise loads them from there.  Returns (uniformly) kGhostsNone when no
// own particle reaches a ghost, kGhostsGlobal when the box does not fit
// (the caller then visits the ghosts through global memory).
template <bool FILL, int TX, int TY, bool RHO, bool TAN>
__device__ __forceinline__ int stage_ghosts(const SimDev& S, const TankDev& T, const BodyDev& b, const Stage<TX, TY, RHO, TAN>& sm,
                            int n_own, GhostStage<true>& gs)
{
    if (threadIdx.x == 0) {
        gs.box[0] = INT_MAX;
        gs.box[1] = INT_MIN;
        gs.box[2] = INT_MAX;
        gs.box[3] = INT_MIN;
    }
    __syncthreads();
    const float bc = b.fc, bs = b.fs, brx = b.frx, bry = b.fry;
    int x0 = INT_MAX, x1 = INT_MIN, y0 = INT_MAX, y1 = INT_MIN;
    for (int t = threadIdx.x; t < n_own; t += blockDim.x) {
        const float4 pi = sm.pv[own_index(t, sm)];
        int gx, gy;
        float ex, ey;
        if (ghost_cell(T, pi.x, pi.y, bc, bs, brx, bry, gx, gy, ex, ey)) {
            x0 = min(x0, max(gx - 1, 0));
            x1 = max(x1, min(gx + 1, T.G - 1));
            y0 = min(y0, max(gy - 1, 0));
            y1 = max(y1, min(gy + 1, T.G - 1));
        }
    }
    x0 = __reduce_min_sync(0xffffffffu, x0);
    x1 = __reduce_max_sync(0xffffffffu, x1);
    y0 = __reduce_min_sync(0xffffffffu, y0);
    y1 = __reduce_max_sync(0xffffffffu, y1);
    if ((threadIdx.x & 31) == 0 && x0 <= x1) {
        atomicMin(&gs.box[0], x0);
        atomicMax(&gs.box[1], x1);
        atomicMin(&gs.box[2], y0);
        atomicMax(&gs.box[3], y1);
    }
    __syncthreads();
    const int X0 = gs.box[0], X1 = gs.box[1], Y0 = gs.box[2], Y1 = gs.box[3];
    if (X0 > X1) return kGhostsNone;
    const int nr = Y1 - Y0 + 1, nc = X1 - X0 + 1;
    if (nr > kGhostDim || nc > kGhostDim) return kGhostsGlobal;
    for (int i = threadIdx.x; i < nr * (nc + 1); i += blockDim.x) {
        const int r = i / (nc + 1), c = i - r * (nc + 1);
        gs.tab[r][c] = __ldg(S.gstart + T.gcell_base + (Y0 + r) * T.G + X0 + c);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int r = 0; r < nr; ++r) {
            gs.pre[r] = acc;
            gs.base[r] = acc - gs.tab[r][0];
            acc += gs.tab[r][nc] - gs.tab[r][0];
        }
        gs.pre[nr] = acc;
    }
    __syncthreads();
    const int total = gs.pre[nr];
    if (total > kGhostMax) return kGhostsGlobal;
    const GhostFrame fr = ghost_frame(b);
    for (int s = threadIdx.x; s < total; s += blockDim.x) {
        int r = 0;
        while (s >= gs.pre[r + 1]) ++r;
        const int g = s - gs.base[r];
        const float4 gb = __ldg(S.gB + g);
        gs.bx[s] = gb.x;
        if constexpr (FILL) {
            float4 gp, gv;
            ghost_world(fr, gb, gp, gv);
            gs.gp[s] = gp;
            gs.gv[s] = gv;
            S.gpos[g] = gp;
            S.gvel[g] = gv;
        } else {
            gs.gp[s] = __ldcg(S.gpos + g);
            gs.gv[s] = __ldcg(S.gvel + g);
        }
    }
    __syncthreads();
    return kGhostsStaged;
}

// First staged ghost in [lo, hi) whose body-frame x is not below v.
__device__ __forceinline__ int lower_bx(const GhostStage<true>& gs, int lo, int hi, float v)
{
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (gs.bx[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Visits the staged ghosts of the 3x3 ghost cells around a fluid particle
// that can lie within `clip` of it: f(global ghost index, staged index).  A
// row of cells whose body-frame y-range misses [y - clip, y + clip] is
// skipped, and a row is clipped to the x-range [x - clip, x + clip] by binary
// search (a row is sorted by body-frame x).  clip exceeds the support by a
// relative 1e-3, far above the FP32 error of the body-frame coordinates, so no
// ghost within the support is skipped.  The edge rows and columns of the
// grid, which may hold ghosts clamped into them, are not clipped.
template <class F>
__device__ __forceinline__ void for_staged_ghosts(const TankDev& T, const GhostStage<true>& gs, float xi, float yi,
                                                  float bc, float bs, float brx, float bry, float clip, F&& f)
{
    int gx, gy;
    float ex, ey;
    if (!ghost_cell(T, xi, yi, bc, bs, brx, bry, gx, gy, ex, ey)) return;
    const int x0 = max(gx - 1, 0), x1 = min(gx + 1, T.G - 1);
    if (x0 > x1) return;
    const int X0 = gs.box[0], X1 = gs.box[1], Y0 = gs.box[2], Y1 = gs.box[3];
    if (x0 < X0 || x1 > X1) return;  // never taken: the box holds every own particle's cells
    const bool clip_x = x0 > 0 && x1 < T.G - 1;
    for (int yy = max(gy - 1, 0); yy <= min(gy + 1, T.G - 1); ++yy) {
        if (yy < Y0 || yy > Y1) continue;  // likewise
        if (yy > 0 && yy < T.G - 1) {
            const float ylo = T.g_orig + (float)yy * T.g_cell;
            if (ylo > ey + clip || ylo + T.g_cell < ey - clip) continue;
        }
        const int r = yy - Y0, base = gs.base[r];
        int a = base + gs.tab[r][x0 - X0], b = base + gs.tab[r][x1 + 1 - X0];
        if (clip_x) {
            a = lower_bx(gs, a, b, ex - clip);
            b = lower_bx(gs, a, b, ex + clip);
        }
        for (int sg = a; sg < b; ++sg) f(sg - base, sg);
    }
}

}  // namespace sph
