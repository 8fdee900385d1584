// sph_noalloc.cu -- density evaluation that allocates no memory.
//
// Some callers cannot call cudaMalloc: code that runs under a fixed device
// memory budget decided up front (flight or real-time software that forbids
// allocation after start-up), or a plugin living inside a host application
// that owns every device allocation.  sph_density_noalloc serves them: it
// computes the ghost-corrected density of Eq. 14 for a fluid state the
// caller passes in, and keeps its working memory (a cell grid and the ghost
// world positions) in one file-scope device array instead of allocating it.
//
// That array is created when the library is loaded and stays on every GPU
// that loaded the library until the process exits.  All calls share it and
// it keeps the previous call's contents, so each call clears what must start
// at zero; two calls that overlap on the GPU (different streams, or the same
// call from two threads) race on it and must not be issued.
//
// A symbol's device address belongs to a CUDA context, not to a device
// number: a caller may make its own driver-API context current on a device,
// or reset the primary context.  So every call looks the address up again in
// the context that is current (cudaGetSymbolAddress allocates nothing) and
// never reuses an address from an earlier call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "../../include/sph.h"

namespace sph {
int set_last_error(int code, const char* msg);
}

namespace sph_noalloc {

constexpr int kMaxCells = 65536;     // grid of at most 256 x 256 cells
constexpr int kSlots = 32;           // particles per cell
constexpr int kMaxGhosts = 16384;

struct Scratch {
    int counts[kMaxCells];
    int slots[kMaxCells * kSlots];   // fluid index i, or n_fluid + ghost index
    float4 ghost[kMaxGhosts];        // (hi_x, hi_y, lo_x, lo_y) world position
    int overflow;
};

static __device__ __align__(256) Scratch g_scratch;   // about 8.6 MB per device

__global__ void clear_kernel(Scratch* s, int n_cells)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_cells) s->counts[i] = 0;
    if (i == 0) s->overflow = 0;
}

struct Geo {
    float ox, oy, inv_cell;   // FP32 grid origin and 1/s
    int G;
    float R2, cW, inv_h, m, gamma1;
    double rx, ry, c, s;      // body position and rotation
};

__device__ __forceinline__ int coord(float x, float o, float inv, int G)
{
    const float f = floorf(__fmul_rn(__fsub_rn(x, o), inv));
    if (f >= 0.0f && f <= (float)(G - 1)) return (int)f;
    return (f > 0.0f) ? G - 1 : 0;
}

// Bins the fluid particles and the ghosts (world positions from Eq. 21).
__global__ void bin_kernel(Scratch* s, Geo g, const float4* __restrict__ xv, int n, const double* __restrict__ gB,
                           int ng)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float px, py;
    int id;
    if (i < n) {
        const float4 p = xv[i];
        px = p.x;
        py = p.y;
        id = i;
    } else if (i < n + ng) {
        const int k = i - n;
        const double bx = gB[2 * k], by = gB[2 * k + 1];
        const double wx = g.rx + (g.c * bx - g.s * by), wy = g.ry + (g.s * bx + g.c * by);
        const float hx = (float)wx, hy = (float)wy;
        s->ghost[k] = make_float4(hx, hy, (float)(wx - (double)hx), (float)(wy - (double)hy));
        px = hx;
        py = hy;
        id = i;
    } else {
        return;
    }
    const int cell = coord(py, g.oy, g.inv_cell, g.G) * g.G + coord(px, g.ox, g.inv_cell, g.G);
    const int slot = atomicAdd(&s->counts[cell], 1);
    if (slot < kSlots)
        s->slots[cell * kSlots + slot] = id;
    else
        s->overflow = 1;
}

// rho_i = m (sum_fluid W + gamma1 sum_ghost W) over r < 2h, self included (Eq. 14).
__global__ void density_kernel(const Scratch* __restrict__ s, Geo g, const float4* __restrict__ xv, int n,
                               float* __restrict__ rho)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = xv[i];
    const int cx = coord(p.x, g.ox, g.inv_cell, g.G), cy = coord(p.y, g.oy, g.inv_cell, g.G);
    float sf = 0.f, sg = 0.f;
    for (int yy = max(cy - 1, 0); yy <= min(cy + 1, g.G - 1); ++yy)
        for (int xx = max(cx - 1, 0); xx <= min(cx + 1, g.G - 1); ++xx) {
            const int cell = yy * g.G + xx;
            const int cnt = min(s->counts[cell], kSlots);
            for (int k = 0; k < cnt; ++k) {
                const int id = s->slots[cell * kSlots + k];
                float dx, dy;
                if (id < n) {
                    const float4 q = xv[id];
                    dx = __fsub_rn(p.x, q.x);
                    dy = __fsub_rn(p.y, q.y);
                } else {
                    const float4 q = s->ghost[id - n];
                    dx = __fsub_rn(__fsub_rn(p.x, q.x), q.z);
                    dy = __fsub_rn(__fsub_rn(p.y, q.y), q.w);
                }
                const float r2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
                if (r2 < g.R2) {
                    const float q = sqrtf(r2) * g.inv_h;
                    const float a = 2.0f - q, b = 1.0f - q;
                    float w = a * a * a;
                    if (q < 1.0f) w -= 4.0f * b * b * b;
                    if (id < n)
                        sf += w;
                    else
                        sg += w;
                }
            }
        }
    rho[i] = g.m * g.cW * (sf + g.gamma1 * sg);
}

}  // namespace sph_noalloc

using namespace sph_noalloc;

extern "C" int sph_density_noalloc(const sph_params* p, const float* xv, int32_t n_fluid, const double* gB,
                                   int32_t n_ghost, const double* body, float* rho, void* stream)
{
    using sph::set_last_error;
    if (!p || !body || n_fluid < 0 || n_ghost < 0 || (n_fluid > 0 && (!xv || !rho)) || (n_ghost > 0 && !gB))
        return set_last_error(SPH_E_INVAL, "sph_density_noalloc: NULL pointer or negative count");
    if (!(p->dx > 0) || !(p->h_over_dx > 0) || !(p->R > 0) || p->n_rings < 0)
        return set_last_error(SPH_E_INVAL, "sph_density_noalloc: invalid sph_params");
    if (n_ghost > kMaxGhosts)
        return set_last_error(SPH_E_UNSUPPORTED, "sph_density_noalloc: more than 16384 ghost particles");
    if ((long long)n_fluid + n_ghost > (1ll << 30))
        return set_last_error(SPH_E_UNSUPPORTED, "sph_density_noalloc: more than 2^30 particles");
    const double h = p->h_over_dx * p->dx;
    const double cell = 2.0 * h * (1.0 + 1.0 / 1024.0);
    const double sg = (p->ghost_spacing > 0.0 ? p->ghost_spacing : 1.0) * p->dx;
    const double W = p->R + ((double)p->n_rings + 1.0) * std::max(p->dx, sg) + 2.0 * cell;
    const int G = (int)std::ceil(2.0 * W / cell);
    if ((long long)G * G > kMaxCells)
        return set_last_error(SPH_E_UNSUPPORTED, "sph_density_noalloc: neighbour grid wider than 256 x 256 cells "
                                                 "(tank radius over dx too large)");

    // the array's device address in the context current on this call (its
    // host-side name is only a stand-in and must never reach a kernel)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return set_last_error(SPH_E_CUDA, "sph_density_noalloc: no current CUDA device");
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr)
        return set_last_error(SPH_E_CUDA, "sph_density_noalloc: cudaGetSymbolAddress failed");
    Scratch* s = (Scratch*)ptr;
    if (n_fluid == 0) return SPH_OK;

    const double sigma = p->sigma_cubic > 0 ? p->sigma_cubic : 5.0 / (14.0 * 3.14159265358979323846);
    Geo g;
    g.ox = (float)(body[0] - W);
    g.oy = (float)(body[1] - W);
    g.inv_cell = (float)(1.0 / cell);
    g.G = G;
    g.R2 = (float)((2.0 * h) * (2.0 * h));
    g.cW = (float)(sigma / (h * h));
    g.inv_h = (float)(1.0 / h);
    g.m = (float)(p->rho0 * p->dx * p->dx);
    g.gamma1 = (float)p->gamma1;
    g.rx = body[0];
    g.ry = body[1];
    g.c = std::cos(body[2]);
    g.s = std::sin(body[2]);

    cudaStream_t st = (cudaStream_t)stream;
    const int n_cells = G * G;
    clear_kernel<<<(n_cells + 255) / 256, 256, 0, st>>>(s, n_cells);
    bin_kernel<<<(n_fluid + n_ghost + 255) / 256, 256, 0, st>>>(s, g, (const float4*)xv, n_fluid, gB, n_ghost);
    density_kernel<<<(n_fluid + 127) / 128, 128, 0, st>>>(s, g, (const float4*)xv, n_fluid, rho);
    if (cudaGetLastError() != cudaSuccess) return set_last_error(SPH_E_CUDA, "sph_density_noalloc: launch failed");
    // a cell that overflowed drops particles: report it (this waits for the stream)
    int overflow = 0;
    if (cudaMemcpyAsync(&overflow, &s->overflow, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return set_last_error(SPH_E_CUDA, "sph_density_noalloc: stream failed");
    if (overflow) return set_last_error(SPH_E_DIVERGED, "sph_density_noalloc: a grid cell held more than 32 particles");
    return SPH_OK;
}
