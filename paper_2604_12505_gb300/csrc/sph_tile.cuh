// sph_tile.cuh -- tile staging shared by the step kernels and the adjoint
// kernels: a tile of TX x TY grid cells plus a one-cell halo is gathered into
// shared memory, each cell ordered by particle index, and every own particle
// visits its 3x3 cells there and the ghost cells around it.
#pragma once

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
};

__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Shared-memory staging of a tile and its halo
// ---------------------------------------------------------------------------
template <int TX, int TY, bool RHO, bool TAN = false>
struct Stage {
    using Sh = Shape<TX, TY>;
    int start[Sh::NC + 1];
    int own_row[TY + 1];
    float4 pv[Sh::MAXS];
    int pid[Sh::MAXS];
    int pid_in[Sh::MAXS];         // particle index in global slot order (before ordering)
    unsigned int key_in[Sh::MAXS];  // ordering key of x in global slot order
    int slot[Sh::MAXS];
    unsigned char cell[Sh::MAXS];
    float2 rho[RHO ? Sh::MAXS : 1];
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
// does not fit.
template <int TX, int TY, bool RHO, bool TAN>
__device__ bool stage_tile(const SimDev& S, const TankDev& T, int buf, int cx0, int cy0, Stage<TX, TY, RHO, TAN>& sm)
{
    using Sh = Shape<TX, TY>;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int* __restrict__ count = S.count[buf];
    for (int c = tid; c < Sh::NC; c += blockDim.x) {
        int ix = cx0 - 1 + c % Sh::SX, iy = cy0 - 1 + c / Sh::SX;
        int n = 0;
        if (ix >= 0 && ix < T.G && iy >= 0 && iy < T.G) n = min(count[T.cell_base + iy * T.G + ix], kCap);
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
        sm.pid_in[e] = S.pid[buf][gs];
        sm.key_in[e] = order_key(S.pv[buf][gs].x);
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
        sm.pv[d] = S.pv[buf][gs];
        if (RHO) sm.rho[d] = S.rhoP[gs];
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
template <int TX, int TY, bool RHO, bool TAN>
__device__ __forceinline__ int own_index(int t, const Stage<TX, TY, RHO, TAN>& sm)
{
    using Sh = Shape<TX, TY>;
    int r = 0;
#pragma unroll
    for (int q = 1; q < TY; ++q) r += (t >= sm.own_row[q]);
    return sm.start[(r + 1) * Sh::SX + 1] + (t - sm.own_row[r]);
}

// Visits the ghosts of the 3x3 body-frame ghost cells around a fluid
// particle; the body-frame position only selects cells, so FP32 suffices.
template <class F>
__device__ __forceinline__ void for_ghosts(const SimDev& S, const TankDev& T, float xi, float yi, float bc, float bs,
                                           float brx, float bry, F&& f)
{
    float px = xi - brx, py = yi - bry;
    float ex = bc * px + bs * py, ey = bc * py - bs * px;
    if (ex * ex + ey * ey < T.ghost_rin2) return;
    const float fx = floorf((ex - T.g_orig) * T.g_inv_cell), fy = floorf((ey - T.g_orig) * T.g_inv_cell);
    if (!(fx >= -1.0f && fx <= (float)T.G && fy >= -1.0f && fy <= (float)T.G)) return;  // off the grid or NaN
    const int gx = (int)fx, gy = (int)fy;
    int x0 = max(gx - 1, 0), x1 = min(gx + 1, T.G - 1);
    if (x0 > x1) return;
    for (int yy = max(gy - 1, 0); yy <= min(gy + 1, T.G - 1); ++yy) {
        int row = T.gcell_base + yy * T.G;
        int a = __ldg(S.gstart + row + x0), b = __ldg(S.gstart + row + x1 + 1);
        for (int j = a; j < b; ++j) f(j);
    }
}

}  // namespace sph
