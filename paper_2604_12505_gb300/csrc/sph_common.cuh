// sph_common.cuh -- device-side data layout and SPH arithmetic shared by the
// CUDA translation units of the simulator (not part of the C ABI).
//
// Layout in device memory (all tanks of a batch concatenated):
//   * neighbour grid, double-buffered by step parity: per cell a count and
//     SPH_CELL_CAPACITY slots; a slot holds float4 (x, y, vx, vy) and the
//     particle's global index.  The fluid state lives only in these slots:
//     the force kernel integrates a particle and writes it straight into its
//     cell of the other buffer (atomic slot claim), so no sort or scan pass
//     exists.  Within a cell the kernels order particles by x, then by
//     index, which makes every neighbour sum deterministic.
//   * per slot also the low parts (x_lo, y_lo, vx_lo, vy_lo) of the particle
//     state: the state is carried as two-float (hi + lo) FP32 pairs, so that
//     the kick and the drift of every step do not round the state to FP32
//     (at 0.5 m from the origin one FP32 position step is 6e-8 m, close to a
//     particle's motion in one step of the large tank); separations are
//     formed from hi and lo, the kernel arithmetic stays FP32.
//   * per-slot float2 (rho, P / rho^2) written by the density kernel.
//   * ghosts: body-frame positions (two-float) binned once into a body-frame
//     grid, and per step the world position as an FP32 (hi, lo) pair plus
//     FP32 velocity and lever arm (Eq. 21), written by the density pass for
//     every ghost it visits and read by the force pass.
//   * per tank: FP32/FP64 constants (TankDev), FP64 body state (BodyDev).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/sph.h"

namespace sph {

constexpr int kCap = SPH_CELL_CAPACITY;

struct TankDev {
    // FP32 constants of the kernels
    float h, inv_h, R2, h2;       // smoothing length, 1/h, fl32((2h)^2), fl32(h^2)
    float cW, cdW;                // sigma/h^2, sigma/h^3 (Eq. 22)
    float cS, cdS;                // 10/(pi h^5), -30/(pi h^5) (Eq. 23)
    float m, inv_m, k, rho0;      // particle mass, EOS (Eq. 11)
    float gamma1, visc_a, beta2, epsh2;  // gamma1, 2 alpha h, 2 beta, eps h^2
    float dt, gp_sign, grav_x, grav_y;
    float inv_cell;               // fl32(1/s)
    float g_orig, g_inv_cell;     // body-frame ghost grid origin (-W) and 1/s, FP32
    float ghost_rin2;             // particles with |xi|^2 below this see no ghost
    float clip;                   // 2h (1 + 1e-3): a candidate whose x-separation exceeds it lies outside the support
    float hclip;                  // h (1 + 1e-3): likewise for the ghost terms of the force pass (support h)
    float g_cell;                 // fl32(ghost-grid cell side)
    int gp_clamp;                 // Eq. 16 with max(P_i, 0)
    float Wf;                     // fl32(grid half-width W)
    float cover2;                 // fl32(cover radius^2): beyond it no tile is launched
    int G;                        // cells per side (fluid and ghost grid)
    int n_f, n_g;
    int cell_base;                // first cell of this tank in the global grid arrays
    int ghost_base;               // first ghost of this tank
    int gcell_base;               // first entry of this tank's ghost-cell table
    int pid_base;                 // first global particle index of this tank
    int outer_every;
    double W, cell;               // grid half-width and cell side (FP64)
    double m_body, J_body, dt_d;
    double inv_m_body, inv_J_body;
    double grav_xd, grav_yd;
};

struct BodyDev {
    // the first eight doubles are read as an array by the body update
    double r[2], th, v[2], w;     // r, theta, rdot, thetadot at the current step
    double c, s;                  // cos(theta), sin(theta)
    double anchor[2][2];          // FP64 anchor of grid buffer 0 / 1
    double tau_c;                 // controller torque held by the zero-order hold
    unsigned long long pairs;     // cumulative pair interactions
    // FP32 forms written once per step by the body update, so that no CTA
    // converts FP64 (the FP64 pipe of this GPU is narrow):
    float fc, fs, frx, fry;       // cos, sin, r rounded -- only used to select ghost cells
    float fo_next[2];             // fl32(r - W): origin of the grid the force pass bins into
    float2 dc, ds, drx, dry;      // cos, sin, r as two-float (hi, lo) splits of the FP64 values
    float fvx, fvy, fw;           // rdot, thetadot rounded to FP32
    // tangent (forward-mode derivative) of the body state, FP64, and its FP32 copy
    double tr[2], tth, tv[2], tw;
    float ftr[2], ftth, ftv[2], ftw;
    // fluid force, torque and particle-position sums of the current force
    // pass as 64-bit fixed point (units of 2^-32, two's complement): the
    // tiles add them with integer atomics, whose sum does not depend on the
    // order of the additions, and the tank's last tile reads and clears them
    unsigned long long acc[5];    // F_x, F_y, T, sum x, sum y
    unsigned int done;            // tiles (reduction groups in the tangent variant) finished in the current force pass
    int flags;                    // SPH_FLAG_* bits
};
// the body update stores these fields by lane (consecutive fields of one type)
static_assert(offsetof(BodyDev, th) == 2 * sizeof(double) && offsetof(BodyDev, s) == 7 * sizeof(double),
              "r, theta, rdot, thetadot, cos, sin lead BodyDev");
static_assert(offsetof(BodyDev, fo_next) == offsetof(BodyDev, fc) + 4 * sizeof(float), "fc .. fo_next contiguous");
static_assert(offsetof(BodyDev, dry) == offsetof(BodyDev, dc) + 3 * sizeof(float2), "dc .. dry contiguous");
static_assert(offsetof(BodyDev, fw) == offsetof(BodyDev, fvx) + 2 * sizeof(float), "fvx .. fw contiguous");

// Fixed point of the body accumulators: a value v is held as round(v 2^32).
// A two-float (hi, lo) sum converts term by term; scaling by a power of two
// is exact, and each conversion rounds once to the nearest unit (2.3e-10).
constexpr float kFixScale = 4294967296.0f;   // 2^32
constexpr double kFixUnit = 1.0 / 4294967296.0;

// Two-float (hi + lo) arithmetic on the FP32 pipe (error-free transformations,
// about 48 significant bits): used for ghost world positions (Eq. 21).
__host__ __device__ __forceinline__ float2 df_split(double v)
{
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

__device__ __forceinline__ float2 df_norm(float s, float e)
{
    const float hi = s + e;
    return make_float2(hi, e - (hi - s));
}

__device__ __forceinline__ float2 df_add(float2 a, float2 b)
{
    const float s = a.x + b.x;
    const float bb = s - a.x;
    const float e = (a.x - (s - bb)) + (b.x - bb) + a.y + b.y;
    return df_norm(s, e);
}

__device__ __forceinline__ float2 df_mul(float2 a, float2 b)
{
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    return df_norm(p, e);
}

// TwoSum: s + e = a + b exactly (s = fl(a + b)).
__device__ __forceinline__ float2 two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}

// Separation (x_i - x_j, y_i - y_j) of two particles held as hi + lo: the hi
// difference (exact for neighbours: Sterbenz) plus the lo difference, rounded
// once.  With lo = 0 it is exactly the FP32 difference of the hi parts.
__device__ __forceinline__ float2 sep_ff(float4 pi, float2 li, float4 pj, float2 lj)
{
    return make_float2(__fadd_rn(__fsub_rn(pi.x, pj.x), __fsub_rn(li.x, lj.x)),
                       __fadd_rn(__fsub_rn(pi.y, pj.y), __fsub_rn(li.y, lj.y)));
}

// Separation of a particle (hi + lo) from a ghost at gp = (x_hi, y_hi, x_lo, y_lo).
__device__ __forceinline__ float2 sep_fg(float4 pi, float2 li, float4 gp)
{
    return make_float2(__fadd_rn(__fsub_rn(pi.x, gp.x), __fsub_rn(li.x, gp.z)),
                       __fadd_rn(__fsub_rn(pi.y, gp.y), __fsub_rn(li.y, gp.w)));
}

struct RunDev {
    long long step;               // global inner-step counter
    long long step0;              // step counter at the start of the current call
    const double* u;              // [B, n_rows, 3] inputs (NULL: zero)
    long long u_tank_stride;      // doubles between tanks in u
    double* y;                    // [B, n_samples, SPH_NY] samples (NULL: none)
    long long y_tank_stride;
    const double* theta_ref;      // [B, n_samples] (NULL: 0)
    long long ref_stride;
    double ctrl_J, ctrl_w, ctrl_xi;
    int ctrl_on;
    float damping;                // relaxation: v <- (1 - damping) v after the kick (0: physical model)
    int body_fixed;               // relaxation: the tank is held at its pose
    const double* du;             // tangent of the input, [B, n_rows, 3] (NULL: 0)
    double* dy;                   // tangent samples [B, n_samples, SPH_NY] (NULL: none)
    unsigned int tanks_done;      // tanks finished in the current force pass
    int next_buf;                 // buffer of the next step's state, written by the force pass (step & 1)
};

// A two-float (hi + lo) compensated sum: error-free transformations keep
// about 48 significant bits, the accuracy of an FP64 sum, on the FP32 pipe.
struct F2 {
    float hi, lo;
};

__device__ __forceinline__ F2 f2_add(F2 a, F2 b)
{
    const float s = a.hi + b.hi;                           // TwoSum(a.hi, b.hi)
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    const float lo = e + a.lo + b.lo;
    const float hi = s + lo;                               // FastTwoSum renormalisation
    return F2{hi, lo - (hi - s)};
}

// Partial sums of one tile (or of a group of kTileGroup tiles), read back
// with three 16-byte loads:
//   a = (F_x hi, F_x lo, F_y hi, F_y lo)   fluid force on the body
//   b = (T hi, T lo, sum x hi, sum x lo)    torque; particle-position sum (sample steps)
//   c = (sum y hi, sum y lo, pairs, wall)   as int bits; pair interactions; any ghost pair
struct __align__(16) TilePartial {
    float4 a, b;
    int4 c;
};

constexpr int kTileGroup = 64;    // tiles per first-level reduction group
constexpr int kOneLevelLoads = 8; // one-level reduction up to this many partials per thread of a tile
constexpr int kNbrRowBits = 32;   // candidates of one stencil row the density pass can record as a bit mask
constexpr unsigned char kNbrNone = 255;  // neighbour count marking a particle whose rows were not recorded

// Optional per-particle outputs of an evaluation pass (indexed by particle).
struct EvalOut {
    float* rho;
    float* drho;
    float* acc;       // [N, 2]
    int* nbr;         // [N, 3]
    int* keys;        // [N]
    double* body;     // [B, 6]
    float* dacc;      // tangent variant: [N, 2] tangent of the fluid acceleration
    double* dbody;    // tangent variant: [B, 6] tangent of body_out
};

// Pointers of one simulator instance, passed by value to every kernel.
struct SimDev {
    const TankDev* tank;
    BodyDev* body;
    RunDev* run;
    float4* pv[2];
    float4* lo[2];                // low parts (x_lo, y_lo, vx_lo, vy_lo) of the state in each slot
    int* pid[2];
    int* count[2];
    float2* rhoP;                 // indexed by slot of the current buffer
    const int4* tiles;            // (tank, first cell x, first cell y, tile index within tank)
    const int* tile_tank_first;   // per tank: first tile (size B + 1)
    const int* group_first;       // per tank: first reduction group (size B + 1)
    TilePartial* partials;        // per tile
    TilePartial* gpartials;       // per group of kTileGroup tiles
    unsigned int* gdone;          // per group: tiles finished in the current force pass
    const float4* gB;             // body-frame ghost positions as two-float (x_hi, x_lo, y_hi, y_lo), sorted by ghost cell
    const int* gstart;            // per tank (G*G + 1) ghost-cell starts (global ghost index)
    float4* gpos;                 // per step: (hi_x, hi_y, lo_x, lo_y) world position, written by the density pass
    float4* gvel;                 // per step: (v_x, v_y, arm_x, arm_y)
    unsigned int* nbm;            // per tile [3 stencil rows][max own]: bit k set if staged particle zl - k is a fluid neighbour
    unsigned short* nba;          // per tile [3][max own]: zl, the row's last candidate (staged index)
    unsigned char* nbn;           // per tile [max own]: fluid neighbour count (kNbrNone: rows not recorded)
    unsigned char* srec;          // per tile: the staged order the density pass leaves for the force pass (StageRec)
    // forward-mode tangent (JVP) state, allocated on first use
    float4* tpv[2];               // per slot (dx, dy, dvx, dvy), binned with the primal
    float2* trho;                 // per slot (d rho, d(P / rho^2))
    float4* tgh;                  // per ghost (d r_g, d v_g)
    TilePartial* tpartials;       // tangent partials per tile / group
    TilePartial* tgpartials;
    int B;
    int n_tiles;
};

// ---------------------------------------------------------------------------
// Kernel arithmetic in FP32
// ---------------------------------------------------------------------------

// Cubic spline (Eq. 22): W(r) for r < 2h.
__device__ __forceinline__ float w_cubic(const TankDev& T, float r)
{
    float q = r * T.inv_h;
    float a = 2.0f - q, b = 1.0f - q;
    float f = a * a * a;
    if (q < 1.0f) f -= 4.0f * b * b * b;
    return T.cW * f;
}

// (dW/dr) / r for the cubic spline, 0 < r < 2h.
__device__ __forceinline__ float dw_cubic_over_r(const TankDev& T, float r, float inv_r)
{
    float q = r * T.inv_h;
    float a = 2.0f - q, b = 1.0f - q;
    float fp = -3.0f * a * a;
    if (q < 1.0f) fp += 12.0f * b * b;
    return T.cdW * fp * inv_r;
}

// d/dr of (dW/dr)/r for the cubic spline, given G = (dW/dr)/r: (W'' - G) / r.
__device__ __forceinline__ float dG_cubic_dr(const TankDev& T, float r, float inv_r, float G)
{
    float q = r * T.inv_h;
    float fpp = 6.0f * (2.0f - q);
    if (q < 1.0f) fpp -= 24.0f * (1.0f - q);
    return (T.cdW * T.inv_h * fpp - G) * inv_r;
}

// Squared distance with the exact operation sequence of the integer decisions:
// fma(dx, dx, dy*dy) with every operation rounded to nearest.
__device__ __forceinline__ float dist2(float dx, float dy)
{
    return __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
}

// Grid column of x: floor(fl32(fl32(x - o) * inv)) clamped to [0, G-1]; a
// clamped (or non-finite) position sets *out.
__device__ __forceinline__ int cell_coord(float x, float o, float inv, int G, bool* out)
{
    const float f = floorf(__fmul_rn(__fsub_rn(x, o), inv));
    if (f >= 0.0f && f <= (float)(G - 1)) return (int)f;
    *out = true;
    return (f > 0.0f) ? G - 1 : 0;  // NaN lands in column 0
}

}  // namespace sph
