// sph_api.cu -- host implementation of the C ABI declared in include/sph.h.
//
// Tank construction (Section 3.2 geometry, done once per handle on the host),
// device allocation, graph-captured step chains and state transfer.  Every
// per-step computation runs in the kernels of sph_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sph.h"
#include "sph_common.cuh"
#include "sph_launch.h"

using namespace sph;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(SPH_E_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

constexpr double kPi = 3.14159265358979323846;
constexpr int kGraphSteps = 32;

struct TankHost {
    sph_params p;
    std::vector<double> xf;   // [n_f, 2] builder order
    std::vector<double> gB;   // [n_g, 2] builder order
    int n_f = 0, n_g = 0, G = 0;
    double h = 0, cell = 0, W = 0;
};

// Area of the part of the disk |p| <= R below the chord y = c.
double segment_area(double R, double c)
{
    if (c <= -R) return 0.0;
    if (c >= R) return kPi * R * R;
    return R * R * (kPi - std::acos(c / R)) + c * std::sqrt(R * R - c * c);
}

double chord_for_fill(double R, double fill)
{
    double lo = -R, hi = R, want = fill * kPi * R * R;
    for (int i = 0; i < 200; ++i) {
        double mid = 0.5 * (lo + hi);
        (segment_area(R, mid) < want ? lo : hi) = mid;
    }
    return 0.5 * (lo + hi);
}

int validate(const sph_params& p)
{
    if (!(p.R > 0) || !(p.dx > 0) || !(p.dx < p.R) || !(p.fill >= 0 && p.fill <= 1) || !(p.h_over_dx > 0) ||
        p.n_rings < 1 || p.outer_every < 1 || !(p.rho0 > 0) || !(p.m_body > 0) || !(p.J_body > 0) || !(p.dt > 0))
        return fail(SPH_E_INVAL, "invalid sph_params");
    return SPH_OK;
}

// Spacing of the ghosts along a ring and between rings.
double ghost_ds(const sph_params& p) { return (p.ghost_spacing > 0.0 ? p.ghost_spacing : 1.0) * p.dx; }

// Fluid lattice and ghost rings of one tank (geometry stated on sph_params).
void build_tank(TankHost& t)
{
    const sph_params& p = t.p;
    const double c = chord_for_fill(p.R, p.fill), rin = p.R - 0.5 * p.dx;
    const int L = (int)std::ceil(p.R / p.dx) + 2;
    for (int j = -L; j <= L; ++j)
        for (int i = -L; i <= L; ++i) {
            double x = ((double)i + 0.5) * p.dx, y = ((double)j + 0.5) * p.dx;
            if (x * x + y * y <= rin * rin && y <= c) {
                t.xf.push_back(x);
                t.xf.push_back(y);
            }
        }
    const double sg = ghost_ds(p);
    for (int k = 0; k < p.n_rings; ++k) {
        const double rk = p.R + ((double)k + 0.5) * sg;
        const int nk = (int)std::round(2.0 * kPi * rk / sg);
        for (int j = 0; j < nk; ++j) {
            const double phi = 2.0 * kPi * (double)j / (double)nk;
            t.gB.push_back(rk * std::cos(phi));
            t.gB.push_back(rk * std::sin(phi));
        }
    }
    t.n_f = (int)t.xf.size() / 2;
    t.n_g = (int)t.gB.size() / 2;
    t.h = p.h_over_dx * p.dx;
    t.cell = 2.0 * t.h * (1.0 + 1.0 / 1024.0);
    t.W = p.R + ((double)p.n_rings + 1.0) * std::max(p.dx, sg) + 2.0 * t.cell;
    t.G = (int)std::ceil(2.0 * t.W / t.cell);
}

// Radius around the tank centre that the launched tiles cover: the outer
// ghost ring plus a ring spacing and a grid cell.
double cover_radius(const TankHost& t)
{
    return t.p.R + ((double)t.p.n_rings + 1.0) * ghost_ds(t.p) + t.cell;
}

template <class T>
int dalloc(T** p, size_t n)
{
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) return fail(SPH_E_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return SPH_OK;
}

// Device buffers of one call, freed on every return path.
struct DevScratch {
    std::vector<void*> ptrs;
    template <class T>
    int get(T** p, size_t n)
    {
        const int rc = dalloc(p, n);
        if (rc == SPH_OK) ptrs.push_back((void*)*p);
        return rc;
    }
    ~DevScratch()
    {
        for (void* q : ptrs) cudaFree(q);
    }
};

// Rows [k0, k0 + n) of u [B, K, 3] into dst [B, n, 3].
cudaError_t slice_u(double* dst, const double* u, int B, int K, int k0, int n, cudaStream_t st)
{
    return cudaMemcpy2DAsync(dst, 3 * sizeof(double) * n, u + 3ll * k0, 3 * sizeof(double) * K,
                             3 * sizeof(double) * n, B, cudaMemcpyDeviceToDevice, st);
}

}  // namespace

namespace sph {
// Lets other translation units of the library set the last-error text.
int set_last_error(int code, const char* msg) { return fail(code, msg); }
}  // namespace sph

struct sph_sim {
    int B = 0;
    std::vector<TankHost> tanks;
    int n_f_total = 0, n_g_total = 0, n_cells_total = 0;
    int tile_code = 3;
    int n_tiles[SPH_TILE_COUNT + 1] = {0};
    SimDev S{};
    // owned device buffers
    TankDev* d_tank = nullptr;
    BodyDev* d_body = nullptr;
    RunDev* d_run = nullptr;
    int4* d_tiles[SPH_TILE_COUNT + 1] = {nullptr};
    int* d_tile_first[SPH_TILE_COUNT + 1] = {nullptr};
    int* d_group_first[SPH_TILE_COUNT + 1] = {nullptr};
    int* d_part_tank = nullptr;
    double* d_scratch_body = nullptr;
    float* d_scratch_xv = nullptr;
    float* d_scratch_lo = nullptr;
    long long host_step = 0;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_tile = 0;
    bool use_pdl = true;
    int max_tiles = 0, max_groups = 0;

    SimDev dev(int code = 0) const
    {
        if (code == 0) code = tile_code;
        SimDev s = S;
        s.tiles = d_tiles[code];
        s.tile_tank_first = d_tile_first[code];
        s.group_first = d_group_first[code];
        s.n_tiles = n_tiles[code];
        return s;
    }

    // chained: the previous launch on st was a step of the same sequence
    int step_launch(const EvalOut& E, int eval, cudaStream_t st, bool chained = false)
    {
        cudaError_t e = launch_step(dev(), E, eval, tile_code, n_tiles[tile_code], st, use_pdl && !eval, false,
                                    chained && !eval);
        if (e != cudaSuccess) return fail(SPH_E_CUDA, std::string("step launch: ") + cudaGetErrorString(e));
        return SPH_OK;
    }
};

namespace {

void free_sim(sph_sim* s)
{
    if (!s) return;
    if (s->graph) cudaGraphExecDestroy(s->graph);
    if (s->cap) cudaStreamDestroy(s->cap);
    cudaFree(s->d_tank);
    cudaFree(s->d_body);
    cudaFree(s->d_run);
    for (int c = 0; c <= SPH_TILE_COUNT; ++c) {
        cudaFree(s->d_tiles[c]);
        cudaFree(s->d_tile_first[c]);
        cudaFree(s->d_group_first[c]);
    }
    cudaFree(s->d_part_tank);
    cudaFree(s->d_scratch_body);
    cudaFree(s->d_scratch_xv);
    cudaFree(s->d_scratch_lo);
    for (int b = 0; b < 2; ++b) {
        cudaFree(s->S.pv[b]);
        cudaFree(s->S.lo[b]);
        cudaFree(s->S.pid[b]);
        cudaFree(s->S.count[b]);
    }
    cudaFree(s->S.rhoP);
    cudaFree(s->S.partials);
    cudaFree(s->S.gpartials);
    cudaFree(s->S.nbm);
    cudaFree(s->S.nba);
    cudaFree(s->S.nbn);
    cudaFree(s->S.srec);
    for (int b = 0; b < 2; ++b) cudaFree(s->S.tpv[b]);
    cudaFree(s->S.trho);
    cudaFree(s->S.tgh);
    cudaFree(s->S.tpartials);
    cudaFree(s->S.tgpartials);
    cudaFree(s->S.gdone);
    cudaFree((void*)s->S.gB);
    cudaFree((void*)s->S.gstart);
    cudaFree(s->S.gpos);
    cudaFree(s->S.gvel);
    delete s;
}

TankDev make_tank_dev(const TankHost& t)
{
    const sph_params& p = t.p;
    TankDev d{};
    const double h = t.h;
    const double sigma = p.sigma_cubic > 0 ? p.sigma_cubic : 5.0 / (14.0 * kPi);
    d.h = (float)h;
    d.inv_h = (float)(1.0 / h);
    d.R2 = (float)((2.0 * h) * (2.0 * h));
    d.h2 = (float)(h * h);
    d.cW = (float)(sigma / (h * h));
    d.cdW = (float)(sigma / (h * h * h));
    d.cS = (float)(10.0 / (kPi * std::pow(h, 5)));
    d.cdS = (float)(-30.0 / (kPi * std::pow(h, 5)));
    const double m = p.rho0 * p.dx * p.dx;
    d.m = (float)m;
    d.inv_m = (float)(1.0 / m);
    d.k = (float)p.k;
    d.rho0 = (float)p.rho0;
    d.gamma1 = (float)p.gamma1;
    d.visc_a = (float)(2.0 * p.alpha * h);
    d.beta2 = (float)(2.0 * p.beta);
    d.epsh2 = (float)(p.eps * h * h);
    d.dt = (float)p.dt;
    d.gp_sign = (float)p.ghost_pressure_sign;
    d.gp_clamp = p.ghost_pressure_clamp ? 1 : 0;
    d.grav_x = (float)p.grav_x;
    d.grav_y = (float)p.grav_y;
    d.inv_cell = (float)(1.0 / t.cell);
    d.g_orig = (float)(-t.W);
    d.g_inv_cell = (float)(1.0 / t.cell);
    double rmin = 1e300;
    for (int g = 0; g < t.n_g; ++g) rmin = std::min(rmin, std::hypot(t.gB[2 * g], t.gB[2 * g + 1]));
    const double rin = rmin - t.cell * 1.01;
    d.ghost_rin2 = rin > 0 ? (float)(rin * rin) : -1.0f;
    d.Wf = (float)t.W;
    d.cover2 = (float)(cover_radius(t) * cover_radius(t));
    d.clip = (float)(2.0 * t.h * (1.0 + 1e-3));
    d.hclip = (float)(t.h * (1.0 + 1e-3));
    d.g_cell = (float)t.cell;
    d.G = t.G;
    d.n_f = t.n_f;
    d.n_g = t.n_g;
    d.outer_every = p.outer_every;
    d.W = t.W;
    d.cell = t.cell;
    d.m_body = p.m_body;
    d.J_body = p.J_body;
    d.inv_m_body = 1.0 / p.m_body;
    d.inv_J_body = 1.0 / p.J_body;
    d.dt_d = p.dt;
    d.grav_xd = p.grav_x;
    d.grav_yd = p.grav_y;
    return d;
}

int create_impl(const sph_params* p, int B, cudaStream_t st, sph_sim** out)
{
    if (!p || !out || B < 1) return fail(SPH_E_INVAL, "sph_create: NULL argument or B < 1");
    *out = nullptr;
    for (int b = 0; b < B; ++b)
        if (validate(p[b])) return SPH_E_INVAL;
    sph_sim* s = new sph_sim();
    s->B = B;
    s->tanks.resize(B);
    std::vector<TankDev> td(B);
    std::vector<float> xv;
    std::vector<int> part_tank;
    std::vector<float4> gB_sorted;
    std::vector<int> gstart;
    int cell_base = 0, ghost_base = 0, gcell_base = 0, pid_base = 0;
    for (int b = 0; b < B; ++b) {
        TankHost& t = s->tanks[b];
        t.p = p[b];
        build_tank(t);
        if (t.G > 4096) {
            free_sim(s);
            return fail(SPH_E_UNSUPPORTED, "sph_create: grid wider than 4096 cells (dx too small for R)");
        }
        td[b] = make_tank_dev(t);
        td[b].cell_base = cell_base;
        td[b].ghost_base = ghost_base;
        td[b].gcell_base = gcell_base;
        td[b].pid_base = pid_base;
        // ghosts sorted by body-frame cell (stable), cell table with global indices
        const int G = t.G;
        // within a cell by body-frame x (then index), so that a row of cells is
        // sorted by x and the kernels can clip it to the support's x-range
        std::vector<int> key(t.n_g), order(t.n_g);
        for (int g = 0; g < t.n_g; ++g) {
            int cx = (int)std::floor((t.gB[2 * g] + t.W) / t.cell), cy = (int)std::floor((t.gB[2 * g + 1] + t.W) / t.cell);
            cx = std::min(std::max(cx, 0), G - 1);
            cy = std::min(std::max(cy, 0), G - 1);
            key[g] = cy * G + cx;
            order[g] = g;
        }
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
            if (key[a] != key[c]) return key[a] < key[c];
            return t.gB[2 * a] < t.gB[2 * c];
        });
        std::vector<int> cnt((size_t)G * G + 1, 0);
        for (int g = 0; g < t.n_g; ++g) cnt[key[g] + 1]++;
        for (size_t c = 0; c < (size_t)G * G; ++c) cnt[c + 1] += cnt[c];
        for (size_t c = 0; c <= (size_t)G * G; ++c) gstart.push_back(ghost_base + cnt[c]);
        for (int q = 0; q < t.n_g; ++q) {
            int g = order[q];
            const float2 bx = df_split(t.gB[2 * g]), by = df_split(t.gB[2 * g + 1]);
            gB_sorted.push_back(make_float4(bx.x, bx.y, by.x, by.y));
        }
        for (int i = 0; i < t.n_f; ++i) {
            xv.push_back((float)t.xf[2 * i]);
            xv.push_back((float)t.xf[2 * i + 1]);
            xv.push_back(0.f);
            xv.push_back(0.f);
            part_tank.push_back(b);
        }
        cell_base += G * G;
        ghost_base += t.n_g;
        gcell_base += G * G + 1;
        pid_base += t.n_f;
    }
    s->n_f_total = pid_base;
    s->n_g_total = ghost_base;
    s->n_cells_total = cell_base;
    if ((long long)cell_base * kCap > (1ll << 31) - 1) {
        free_sim(s);
        return fail(SPH_E_UNSUPPORTED, "sph_create: more than 2^31 grid slots");
    }
    // tile tables for every shape
    int max_tiles = 0, max_groups = 0;
    std::vector<std::vector<int4>> tiles(SPH_TILE_COUNT + 1);
    std::vector<std::vector<int>> first(SPH_TILE_COUNT + 1), gfirst(SPH_TILE_COUNT + 1);
    for (int code = 1; code <= SPH_TILE_COUNT; ++code) {
        int TX, TY;
        tile_dims(code, &TX, &TY);
        for (int b = 0; b < B; ++b) {
            first[code].push_back((int)tiles[code].size());
            const TankHost& th = s->tanks[b];
            const int G = th.G;
            // Launch order: tiles that meet the wall band first (their ghost
            // terms make them the longest, so they should take the first
            // SM slots), then the interior; row-major within each.  Tiles
            // wholly beyond the cover radius (the ghost rings plus a cell)
            // are not launched: a particle there has escaped the tank and is
            // flagged (SPH_FLAG_ESCAPED).  Every particle within the cover
            // radius lies in a launched tile.
            const double inner = th.p.R - 3.0 * th.cell;
            const double outer = cover_radius(th);
            int local = 0;
            for (int cls = 0; cls < 2; ++cls)
                for (int ty = 0; ty < G; ty += TY)
                    for (int tx = 0; tx < G; tx += TX) {
                        // nearest and farthest distance of the tile from the tank centre
                        const double x0 = tx * th.cell - th.W, x1 = (tx + TX) * th.cell - th.W;
                        const double y0 = ty * th.cell - th.W, y1 = (ty + TY) * th.cell - th.W;
                        const double nx = std::max(std::max(x0, -x1), 0.0), ny = std::max(std::max(y0, -y1), 0.0);
                        const double fx = std::max(std::fabs(x0), std::fabs(x1)), fy = std::max(std::fabs(y0), std::fabs(y1));
                        const double dmin = std::hypot(nx, ny), dmax = std::hypot(fx, fy);
                        const int c = dmin > outer ? 2 : (dmax < inner ? 1 : 0);
                        if (c == cls) tiles[code].push_back(make_int4(b, tx, ty, local++));
                    }
        }
        first[code].push_back((int)tiles[code].size());
        s->n_tiles[code] = (int)tiles[code].size();
        max_tiles = std::max(max_tiles, s->n_tiles[code]);
        int ng = 0;
        for (int b = 0; b < B; ++b) {
            gfirst[code].push_back(ng);
            ng += (first[code][b + 1] - first[code][b] + kTileGroup - 1) / kTileGroup;
        }
        gfirst[code].push_back(ng);
        max_groups = std::max(max_groups, ng);
    }
    s->tile_code = 3;

    int rc = SPH_OK;
    const size_t nslot = (size_t)s->n_cells_total * kCap;
    rc |= dalloc(&s->d_tank, B);
    rc |= dalloc(&s->d_body, B);
    rc |= dalloc(&s->d_run, 1);
    for (int code = 1; code <= SPH_TILE_COUNT; ++code) {
        rc |= dalloc(&s->d_tiles[code], tiles[code].size());
        rc |= dalloc(&s->d_tile_first[code], first[code].size());
        rc |= dalloc(&s->d_group_first[code], gfirst[code].size());
    }
    rc |= dalloc(&s->d_part_tank, s->n_f_total);
    rc |= dalloc(&s->d_scratch_body, 6 * (size_t)B);
    rc |= dalloc(&s->d_scratch_xv, 4 * (size_t)s->n_f_total);
    rc |= dalloc(&s->d_scratch_lo, 4 * (size_t)s->n_f_total);
    for (int b = 0; b < 2; ++b) {
        rc |= dalloc(&s->S.pv[b], nslot);
        rc |= dalloc(&s->S.lo[b], nslot);
        rc |= dalloc(&s->S.pid[b], nslot);
        rc |= dalloc(&s->S.count[b], s->n_cells_total);
    }
    rc |= dalloc(&s->S.rhoP, nslot);
    s->max_tiles = max_tiles;
    s->max_groups = max_groups;
    rc |= dalloc(&s->S.partials, max_tiles);
    rc |= dalloc(&s->S.gpartials, max_groups);
    {   // neighbour records: per tile 3 rows x (TX*TY*12) own particles, sized for the largest shape
        size_t nn = 0;
        for (int code = 1; code <= SPH_TILE_COUNT; ++code) {
            int TX, TY;
            tile_dims(code, &TX, &TY);
            nn = std::max(nn, (size_t)s->n_tiles[code] * TX * TY * 12);
        }
        rc |= dalloc(&s->S.nbm, 3 * nn);
        rc |= dalloc(&s->S.nba, 3 * nn);
        rc |= dalloc(&s->S.nbn, nn);
    }
    rc |= dalloc(&s->S.gdone, max_groups);
    rc |= dalloc(&s->S.srec, stage_record_bytes(s->n_tiles));
    float4* gB_d;
    int* gstart_d;
    rc |= dalloc(&gB_d, gB_sorted.size());
    rc |= dalloc(&gstart_d, gstart.size());
    s->S.gB = gB_d;
    s->S.gstart = gstart_d;
    rc |= dalloc(&s->S.gpos, s->n_g_total);
    rc |= dalloc(&s->S.gvel, s->n_g_total);
    if (rc) {
        std::string msg = g_err;
        free_sim(s);
        return fail(SPH_E_NOMEM, msg);
    }
    s->S.tank = s->d_tank;
    s->S.body = s->d_body;
    s->S.run = s->d_run;
    s->S.B = B;

#define CKF(call)                                                                                 \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            free_sim(s);                                                                          \
            return fail(SPH_E_CUDA, std::string(#call ": ") + cudaGetErrorString(e_));            \
        }                                                                                         \
    } while (0)
    CKF(cudaMemcpy(s->d_tank, td.data(), B * sizeof(TankDev), cudaMemcpyHostToDevice));
    CKF(cudaMemset(s->d_body, 0, B * sizeof(BodyDev)));
    CKF(cudaMemset(s->d_run, 0, sizeof(RunDev)));
    CKF(cudaMemset(s->S.gdone, 0, max_groups * sizeof(unsigned int)));
    for (int code = 1; code <= SPH_TILE_COUNT; ++code) {
        CKF(cudaMemcpy(s->d_tiles[code], tiles[code].data(), tiles[code].size() * sizeof(int4), cudaMemcpyHostToDevice));
        CKF(cudaMemcpy(s->d_tile_first[code], first[code].data(), first[code].size() * sizeof(int), cudaMemcpyHostToDevice));
        CKF(cudaMemcpy(s->d_group_first[code], gfirst[code].data(), gfirst[code].size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    CKF(cudaMemcpy(s->d_part_tank, part_tank.data(), part_tank.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (!gB_sorted.empty()) {
        CKF(cudaMemcpy(gB_d, gB_sorted.data(), gB_sorted.size() * sizeof(float4), cudaMemcpyHostToDevice));
    }
    CKF(cudaMemcpy(gstart_d, gstart.data(), gstart.size() * sizeof(int), cudaMemcpyHostToDevice));
    CKF(cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking));
    // initial state: fluid at rest on the lattice, body at the origin at rest
    std::vector<double> body0(6 * (size_t)B, 0.0);
    CKF(cudaMemcpy(s->d_scratch_xv, xv.data(), xv.size() * sizeof(float), cudaMemcpyHostToDevice));
    CKF(cudaMemcpy(s->d_scratch_body, body0.data(), body0.size() * sizeof(double), cudaMemcpyHostToDevice));
#undef CKF
    *out = s;
    int r2 = sph_set_state(s, s->d_scratch_xv, s->d_scratch_body, st);
    if (r2 == SPH_OK && cudaStreamSynchronize(st) != cudaSuccess) r2 = fail(SPH_E_CUDA, "sph_create: initial binning failed");
    if (r2 != SPH_OK) {
        free_sim(s);
        *out = nullptr;
    }
    return r2;
}

int ensure_graph(sph_sim* s)
{
    if (s->graph && s->graph_tile == s->tile_code) return SPH_OK;
    if (s->graph) {
        cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
    }
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
    EvalOut E{};
    for (int i = 0; i < kGraphSteps; ++i) {
        int rc = s->step_launch(E, 0, s->cap, i > 0);
        if (rc) {
            cudaStreamEndCapture(s->cap, &g);
            if (g) cudaGraphDestroy(g);
            return rc;
        }
    }
    CK(cudaStreamEndCapture(s->cap, &g));
    cudaError_t e = cudaGraphInstantiate(&s->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(SPH_E_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    s->graph_tile = s->tile_code;
    return SPH_OK;
}

long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

// The particle state as hi parts xv [N, 4] and low parts lo [N, 4] (NULL: not
// read back / zero), with the body [B, 6].  The public state calls exchange
// the hi parts only; the checkpoints of the adjoint and the autotuner's
// snapshot carry both, so that their restored state is the state they saved.
int get_state_full(sph_sim* sim, float* xv, float* lo, double* body, cudaStream_t st)
{
    const int buf = (int)(sim->host_step & 1);
    CK(launch_get_state(sim->S, xv, lo, body, sim->n_cells_total, buf, st));
    return SPH_OK;
}

int set_state_full(sph_sim* sim, const float* xv, const float* lo, const double* body, cudaStream_t st)
{
    const int buf = (int)(sim->host_step & 1);
    // both buffers: the cells beyond the cover radius belong to no launched
    // tile, so no density pass clears them, and a tile next to them stages
    // them as halo
    CK(cudaMemsetAsync(sim->S.count[buf], 0, sim->n_cells_total * sizeof(int), st));
    CK(cudaMemsetAsync(sim->S.count[buf ^ 1], 0, sim->n_cells_total * sizeof(int), st));
    CK(launch_set_body(sim->S, body, buf, st));
    CK(launch_bin_flat(sim->S, xv, lo, sim->d_part_tank, sim->n_f_total, buf, st));
    return SPH_OK;
}

}  // namespace

extern "C" {

const char* sph_last_error(void) { return g_err.c_str(); }

int sph_create(const sph_params* p, void* stream, sph_sim** out) { return create_impl(p, 1, (cudaStream_t)stream, out); }

int sph_create_batch(const sph_params* p, int32_t B, void* stream, sph_sim** out)
{
    return create_impl(p, B, (cudaStream_t)stream, out);
}

int sph_destroy(sph_sim* sim)
{
    if (!sim) return SPH_OK;
    cudaDeviceSynchronize();
    free_sim(sim);
    return SPH_OK;
}

int sph_counts(const sph_sim* sim, int32_t* B, int32_t* n_fluid, int32_t* n_ghost)
{
    if (!sim) return fail(SPH_E_INVAL, "sph_counts: NULL handle");
    if (B) *B = sim->B;
    for (int b = 0; b < sim->B; ++b) {
        if (n_fluid) n_fluid[b] = sim->tanks[b].n_f;
        if (n_ghost) n_ghost[b] = sim->tanks[b].n_g;
    }
    return SPH_OK;
}

int sph_ghosts_body(const sph_sim* sim, int32_t b, double* gB_host)
{
    if (!sim || !gB_host || b < 0 || b >= sim->B) return fail(SPH_E_INVAL, "sph_ghosts_body: bad argument");
    std::memcpy(gB_host, sim->tanks[b].gB.data(), sim->tanks[b].gB.size() * sizeof(double));
    return SPH_OK;
}

int sph_get_state(sph_sim* sim, float* xv, double* body, void* stream)
{
    if (!sim) return fail(SPH_E_INVAL, "sph_get_state: NULL handle");
    return get_state_full(sim, xv, nullptr, body, (cudaStream_t)stream);
}

int sph_set_state(sph_sim* sim, const float* xv, const double* body, void* stream)
{
    if (!sim || !body || (!xv && sim->n_f_total > 0)) return fail(SPH_E_INVAL, "sph_set_state: NULL argument");
    return set_state_full(sim, xv, nullptr, body, (cudaStream_t)stream);
}

int sph_samples_for(const sph_sim* sim, int32_t n_steps, int32_t* n_samples)
{
    if (!sim || !n_samples || n_steps < 0) return fail(SPH_E_INVAL, "sph_samples_for: bad argument");
    // all tanks of a batch share outer_every only if equal; samples are counted per tank 0
    const long long oe = sim->tanks[0].p.outer_every;
    const long long s0 = sim->host_step, s1 = sim->host_step + n_steps;
    *n_samples = (int32_t)(ceil_div(s1, oe) - ceil_div(s0, oe));
    return SPH_OK;
}

int sph_step(sph_sim* sim, const double* u, int32_t n_steps, const sph_ctrl* pd, double* y_out, void* stream)
{
    if (!sim || n_steps < 0) return fail(SPH_E_INVAL, "sph_step: bad argument");
    if (n_steps == 0) return SPH_OK;
    for (int b = 1; b < sim->B; ++b)
        if (sim->tanks[b].p.outer_every != sim->tanks[0].p.outer_every)
            return fail(SPH_E_UNSUPPORTED, "sph_step: tanks of a batch must share outer_every");
    cudaStream_t st = (cudaStream_t)stream;
    int32_t ns = 0;
    sph_samples_for(sim, n_steps, &ns);
    RunDev d{};
    d.u = u;
    d.u_tank_stride = 3ll * n_steps;
    d.y = y_out;
    d.y_tank_stride = (long long)ns * SPH_NY;
    if (pd && pd->enabled) {
        d.ctrl_on = 1;
        d.ctrl_J = pd->J;
        d.ctrl_w = pd->omega;
        d.ctrl_xi = pd->xi;
        d.theta_ref = pd->theta_ref;
        d.ref_stride = pd->ref_stride;
    }
    CK(launch_set_run(sim->d_run, d, st));
    int rc = ensure_graph(sim);
    if (rc) return rc;
    int left = n_steps;
    EvalOut E{};
    while (left >= kGraphSteps) {
        CK(cudaGraphLaunch(sim->graph, st));
        left -= kGraphSteps;
    }
    for (int i = 0; left > 0; --left, ++i) {
        rc = sim->step_launch(E, 0, st, i > 0);
        if (rc) return rc;
    }
    sim->host_step += n_steps;
    return SPH_OK;
}

int sph_relax(sph_sim* sim, int32_t n_steps, double damping, void* stream)
{
    if (!sim || n_steps < 0 || !(damping >= 0.0 && damping < 1.0)) return fail(SPH_E_INVAL, "sph_relax: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    RunDev d{};
    d.damping = (float)damping;
    d.body_fixed = 1;
    CK(launch_set_run(sim->d_run, d, st));
    EvalOut E{};
    for (int i = 0; i < n_steps; ++i) {
        int rc = sim->step_launch(E, 0, st, i > 0);
        if (rc) return rc;
    }
    sim->host_step += n_steps;
    return SPH_OK;
}

namespace {
// Tangent buffers of the forward-mode kernels, allocated on first use.
int ensure_tangent(sph_sim* sim)
{
    if (sim->S.trho) return SPH_OK;
    const size_t nslot = (size_t)sim->n_cells_total * kCap;
    int rc = SPH_OK;
    for (int b = 0; b < 2; ++b) rc |= dalloc(&sim->S.tpv[b], nslot);
    rc |= dalloc(&sim->S.trho, nslot);
    rc |= dalloc(&sim->S.tgh, sim->n_g_total);
    rc |= dalloc(&sim->S.tpartials, sim->max_tiles);
    rc |= dalloc(&sim->S.tgpartials, sim->max_groups);
    return rc ? SPH_E_NOMEM : SPH_OK;
}
}  // namespace

int sph_eval_jvp(sph_sim* sim, const double* u, const double* du, const float* dxv, const double* dbody,
                 float* dacc, double* dbody_acc, void* stream)
{
    if (!sim) return fail(SPH_E_INVAL, "sph_eval_jvp: NULL handle");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_tangent(sim);
    if (rc) return rc;
    const int code = sim->tile_code > 4 ? 4 : sim->tile_code;  // tangent kernels exist for tiles up to 8x4
    const SimDev S = sim->dev(code);
    const int buf = (int)(sim->host_step & 1);
    CK(launch_tangent_state(S, dxv, nullptr, dbody, nullptr, sim->n_cells_total, buf, st));
    RunDev d{};
    d.u = u;
    d.du = du;
    d.u_tank_stride = 3;
    CK(launch_set_run(sim->d_run, d, st));
    EvalOut E{};
    E.dacc = dacc;
    E.dbody = dbody_acc;
    cudaError_t e = launch_step(S, E, 1, code, sim->n_tiles[code], st, false, true);
    if (e != cudaSuccess) return fail(SPH_E_CUDA, std::string("sph_eval_jvp launch: ") + cudaGetErrorString(e));
    return SPH_OK;
}

int sph_jvp(sph_sim* sim, const double* u, const double* du, const float* dxv0, const double* dbody0, int32_t K,
            double* y_out, double* dy_out, float* dxv_out, double* dbody_out, void* stream)
{
    if (!sim || K < 0) return fail(SPH_E_INVAL, "sph_jvp: bad argument");
    for (int b = 1; b < sim->B; ++b)
        if (sim->tanks[b].p.outer_every != sim->tanks[0].p.outer_every)
            return fail(SPH_E_UNSUPPORTED, "sph_jvp: tanks of a batch must share outer_every");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_tangent(sim);
    if (rc) return rc;
    const int code = sim->tile_code > 4 ? 4 : sim->tile_code;  // tangent kernels exist for tiles up to 8x4
    const SimDev S = sim->dev(code);
    const int buf = (int)(sim->host_step & 1);
    CK(launch_tangent_state(S, dxv0, nullptr, dbody0, nullptr, sim->n_cells_total, buf, st));
    int32_t ns = 0;
    sph_samples_for(sim, K, &ns);
    RunDev d{};
    d.u = u;
    d.du = du;
    d.u_tank_stride = 3ll * K;
    d.y = y_out;
    d.dy = dy_out;
    d.y_tank_stride = (long long)ns * SPH_NY;
    CK(launch_set_run(sim->d_run, d, st));
    EvalOut E{};
    for (int i = 0; i < K; ++i) {
        cudaError_t e = launch_step(S, E, 0, code, sim->n_tiles[code], st, sim->use_pdl, true);
        if (e != cudaSuccess) return fail(SPH_E_CUDA, std::string("sph_jvp launch: ") + cudaGetErrorString(e));
    }
    sim->host_step += K;
    if (dxv_out || dbody_out) {
        float* tx = dxv_out ? dxv_out : sim->d_scratch_xv;
        CK(launch_tangent_state(S, nullptr, tx, nullptr, dbody_out, sim->n_cells_total, (int)(sim->host_step & 1), st));
    }
    return SPH_OK;
}

int sph_vjp(sph_sim* sim, const double* u, int32_t K, const double* ybar, const float* xvbar_K,
            const double* bodybar_K, float* xvbar0, double* bodybar0, double* ubar, int32_t checkpoint_every,
            void* stream)
{
    if (!sim || K < 0 || checkpoint_every < 1) return fail(SPH_E_INVAL, "sph_vjp: bad argument");
    for (int b = 1; b < sim->B; ++b)
        if (sim->tanks[b].p.outer_every != sim->tanks[0].p.outer_every)
            return fail(SPH_E_UNSUPPORTED, "sph_vjp: tanks of a batch must share outer_every");
    cudaStream_t st = (cudaStream_t)stream;
    const int B = sim->B, N = sim->n_f_total, C = checkpoint_every;
    const long long step0 = sim->host_step;
    const int oe = sim->tanks[0].p.outer_every > 0 ? sim->tanks[0].p.outer_every : 1;
    const int n_seg = (K + C - 1) / C;
    const size_t nxv = 4 * (size_t)N;
    DevScratch mem;
    float4 *adj0 = nullptr, *adj1 = nullptr;
    float *rhob = nullptr, *fbar = nullptr, *part = nullptr, *ck_xv = nullptr, *seg_xv = nullptr, *fin_xv = nullptr;
    float *ck_lo = nullptr, *seg_lo = nullptr, *fin_lo = nullptr;
    double *bbar = nullptr, *bpart = nullptr, *ck_b = nullptr, *seg_b = nullptr, *fin_b = nullptr, *us = nullptr;
    const int code = adjoint_tile_code();
    int rc = mem.get(&adj0, N) | mem.get(&adj1, N) | mem.get(&rhob, N) | mem.get(&fbar, 8 * (size_t)B) |
             mem.get(&part, 2 * (size_t)sim->max_tiles * 12) | mem.get(&bbar, 6 * (size_t)B) |
             mem.get(&bpart, 6 * (size_t)B) | mem.get(&ck_xv, nxv * (n_seg ? n_seg : 1)) |
             mem.get(&ck_b, 6 * (size_t)B * (n_seg ? n_seg : 1)) | mem.get(&seg_xv, nxv * C) |
             mem.get(&seg_b, 6 * (size_t)B * C) | mem.get(&fin_xv, nxv) | mem.get(&fin_b, 6 * (size_t)B) |
             mem.get(&us, 3 * (size_t)B * C) | mem.get(&ck_lo, nxv * (n_seg ? n_seg : 1)) |
             mem.get(&seg_lo, nxv * C) | mem.get(&fin_lo, nxv);
    if (rc) return SPH_E_NOMEM;
    // adjoint of the final state
    if (xvbar_K) CK(cudaMemcpyAsync(adj0, xvbar_K, nxv * sizeof(float), cudaMemcpyDeviceToDevice, st));
    else CK(cudaMemsetAsync(adj0, 0, nxv * sizeof(float), st));
    if (bodybar_K) CK(cudaMemcpyAsync(bbar, bodybar_K, 6 * B * sizeof(double), cudaMemcpyDeviceToDevice, st));
    else CK(cudaMemsetAsync(bbar, 0, 6 * B * sizeof(double), st));
    // forward: a checkpoint every C steps, then the final state
    for (int sgi = 0; sgi < n_seg; ++sgi) {
        const int k0 = sgi * C, n = std::min(C, K - k0);
        if ((rc = get_state_full(sim, ck_xv + nxv * sgi, ck_lo + nxv * sgi, ck_b + 6ll * B * sgi, st))) return rc;
        if (u) CK(slice_u(us, u, B, K, k0, n, st));
        if ((rc = sph_step(sim, u ? us : nullptr, n, nullptr, nullptr, stream))) return rc;
    }
    if ((rc = get_state_full(sim, fin_xv, fin_lo, fin_b, st))) return rc;
    AdjDev A{};
    A.rhobar = rhob;
    A.bbar = bbar;
    A.bbar_part = bpart;
    A.fbar = fbar;
    A.part = part;
    A.max_tiles = sim->max_tiles;
    A.ybar = ybar;
    int32_t ns = 0;
    {   // samples of the forward call
        long long first = (step0 + oe - 1) / oe, last = (step0 + K + oe - 1) / oe;
        ns = (int32_t)(last - first);
    }
    A.ybar_stride = (long long)ns * SPH_NY;
    A.ubar = ubar;
    A.ubar_stride = 3ll * K;
    const SimDev S = sim->dev(code);
    float4* cur = adj0;
    float4* nxt = adj1;
    for (int sgi = n_seg - 1; sgi >= 0; --sgi) {
        const int k0 = sgi * C, n1 = std::min(K, k0 + C);
        // recompute the states of the segment from its checkpoint
        sim->host_step = step0 + k0;
        CK(launch_set_step(sim->d_run, sim->host_step, st));
        if ((rc = set_state_full(sim, ck_xv + nxv * sgi, ck_lo + nxv * sgi, ck_b + 6ll * B * sgi, st))) return rc;
        for (int k = k0; k < n1; ++k) {
            if ((rc = get_state_full(sim, seg_xv + nxv * (k - k0), seg_lo + nxv * (k - k0), seg_b + 6ll * B * (k - k0),
                                     st)))
                return rc;
            if (k + 1 < n1) {
                if (u) CK(slice_u(us, u, B, K, k, 1, st));
                if ((rc = sph_step(sim, u ? us : nullptr, 1, nullptr, nullptr, stream))) return rc;
            }
        }
        for (int k = n1 - 1; k >= k0; --k) {
            sim->host_step = step0 + k;
            CK(launch_set_step(sim->d_run, sim->host_step, st));
            if ((rc = set_state_full(sim, seg_xv + nxv * (k - k0), seg_lo + nxv * (k - k0), seg_b + 6ll * B * (k - k0),
                                     st)))
                return rc;
            const long long g = step0 + k;
            A.k = k;
            A.row = (g % oe == 0) ? (int)(g / oe - (step0 + oe - 1) / oe) : -1;
            A.in = cur;
            A.out = nxt;
            CK(launch_adjoint_step(S, A, sim->n_tiles[code], st));
            std::swap(cur, nxt);
        }
    }
    if (xvbar0) CK(cudaMemcpyAsync(xvbar0, cur, nxv * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (bodybar0) CK(cudaMemcpyAsync(bodybar0, bbar, 6 * B * sizeof(double), cudaMemcpyDeviceToDevice, st));
    // leave the simulator at the final state, as sph_jvp does
    sim->host_step = step0 + K;
    CK(launch_set_step(sim->d_run, sim->host_step, st));
    if ((rc = set_state_full(sim, fin_xv, fin_lo, fin_b, st))) return rc;
    CK(cudaStreamSynchronize(st));  // the scratch buffers are freed on return
    return SPH_OK;
}

int sph_eval(sph_sim* sim, const double* u, float* rho, float* drho, float* acc, int32_t* nbr, int32_t* keys,
             double* body_out, void* stream)
{
    if (!sim) return fail(SPH_E_INVAL, "sph_eval: NULL handle");
    cudaStream_t st = (cudaStream_t)stream;
    RunDev d{};
    d.u = u;
    d.u_tank_stride = 3;
    CK(launch_set_run(sim->d_run, d, st));
    EvalOut E{rho, drho, acc, nbr, keys, body_out};
    return sim->step_launch(E, 1, st);
}

int sph_grid_info(sph_sim* sim, int32_t b, double* cell, double* half_width, int32_t* G, double* anchor_xy)
{
    if (!sim || b < 0 || b >= sim->B) return fail(SPH_E_INVAL, "sph_grid_info: bad argument");
    CK(cudaDeviceSynchronize());
    const TankHost& t = sim->tanks[b];
    if (cell) *cell = t.cell;
    if (half_width) *half_width = t.W;
    if (G) *G = t.G;
    if (anchor_xy) {
        BodyDev bd;
        CK(cudaMemcpy(&bd, sim->d_body + b, sizeof(BodyDev), cudaMemcpyDeviceToHost));
        const int buf = (int)(sim->host_step & 1);
        anchor_xy[0] = bd.anchor[buf][0];
        anchor_xy[1] = bd.anchor[buf][1];
    }
    return SPH_OK;
}

int sph_check(sph_sim* sim, int32_t* flags, int32_t reset, void* stream)
{
    if (!sim) return fail(SPH_E_INVAL, "sph_check: NULL handle");
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    std::vector<BodyDev> bd(sim->B);
    CK(cudaMemcpy(bd.data(), sim->d_body, sim->B * sizeof(BodyDev), cudaMemcpyDeviceToHost));
    int f = 0;
    for (auto& b : bd) f |= b.flags;
    if (flags) *flags = f;
    if (reset && f) {
        for (int b = 0; b < sim->B; ++b)
            CK(cudaMemset((char*)(sim->d_body + b) + offsetof(BodyDev, flags), 0, sizeof(int)));
        CK(cudaDeviceSynchronize());
    }
    if (f & ~SPH_FLAG_TIMEOUT) return fail(SPH_E_DIVERGED, "health check tripped: flags " + std::to_string(f));
    if (f) return fail(SPH_E_TIMEOUT, "a bounded device-side wait gave up");
    return SPH_OK;
}

int sph_pair_count(sph_sim* sim, int64_t* pairs, void* stream)
{
    if (!sim || !pairs) return fail(SPH_E_INVAL, "sph_pair_count: bad argument");
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    std::vector<BodyDev> bd(sim->B);
    CK(cudaMemcpy(bd.data(), sim->d_body, sim->B * sizeof(BodyDev), cudaMemcpyDeviceToHost));
    unsigned long long t = 0;
    for (auto& b : bd) t += b.pairs;
    *pairs = (int64_t)t;
    return SPH_OK;
}

int sph_set_tile(sph_sim* sim, int32_t tile)
{
    if (!sim || tile < 0 || tile > SPH_TILE_COUNT) return fail(SPH_E_INVAL, "sph_set_tile: bad tile code");
    sim->tile_code = tile == 0 ? 3 : tile;
    return SPH_OK;
}

int sph_autotune(sph_sim* sim, int32_t steps, int32_t* chosen, double* us_per_step, void* stream)
{
    if (!sim || steps < 1) return fail(SPH_E_INVAL, "sph_autotune: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    // snapshot: particles in index order, raw body records and run record
    std::vector<BodyDev> body(sim->B);
    RunDev run;
    CK(cudaStreamSynchronize(st));
    CK(cudaMemcpy(body.data(), sim->d_body, sim->B * sizeof(BodyDev), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&run, sim->d_run, sizeof(RunDev), cudaMemcpyDeviceToHost));
    int rc = get_state_full(sim, sim->d_scratch_xv, sim->d_scratch_lo, nullptr, st);
    if (rc) return rc;
    const long long step0 = sim->host_step;
    const int old_tile = sim->tile_code;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int best = old_tile;
    float best_ms = 1e30f;
    for (int code = 1; code <= SPH_TILE_COUNT; ++code) {
        sim->tile_code = code;
        rc = sph_step(sim, nullptr, 2, nullptr, nullptr, stream);
        if (rc) break;
        CK(cudaEventRecord(e0, st));
        rc = sph_step(sim, nullptr, steps, nullptr, nullptr, stream);
        if (rc) break;
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (us_per_step) us_per_step[code - 1] = 1000.0 * ms / steps;
        if (ms < best_ms) {
            best_ms = ms;
            best = code;
        }
        // restore the snapshot exactly (same anchors, same grid membership)
        sim->host_step = step0;
        CK(cudaMemcpy(sim->d_body, body.data(), sim->B * sizeof(BodyDev), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(sim->d_run, &run, sizeof(RunDev), cudaMemcpyHostToDevice));
        const int buf = (int)(step0 & 1);
        CK(cudaMemset(sim->S.count[buf], 0, sim->n_cells_total * sizeof(int)));
        CK(cudaMemset(sim->S.count[buf ^ 1], 0, sim->n_cells_total * sizeof(int)));
        CK(launch_bin_flat(sim->S, sim->d_scratch_xv, sim->d_scratch_lo, sim->d_part_tank, sim->n_f_total, buf, st));
        CK(cudaStreamSynchronize(st));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        sim->tile_code = old_tile;
        return rc;
    }
    sim->tile_code = best;
    if (chosen) *chosen = best;
    return SPH_OK;
}

int sph_time_kernels(sph_sim* sim, int32_t n_steps, double* us, void* stream)
{
    if (!sim || n_steps < 1 || !us) return fail(SPH_E_INVAL, "sph_time_kernels: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    RunDev d{};
    CK(launch_set_run(sim->d_run, d, st));
    cudaEvent_t ev[4];
    for (auto& e : ev) CK(cudaEventCreate(&e));
    double acc[3] = {0.0, 0.0, 0.0};
    const SimDev S = sim->dev();
    EvalOut E{};
    for (int i = 0; i < n_steps; ++i) {
        for (int ph = 0; ph < 3; ++ph) {
            CK(cudaEventRecord(ev[ph], st));
            CK(launch_phase(S, E, 0, sim->tile_code, sim->n_tiles[sim->tile_code], ph, st, false));
        }
        CK(cudaEventRecord(ev[3], st));
        CK(cudaEventSynchronize(ev[3]));
        for (int ph = 0; ph < 3; ++ph) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ev[ph], ev[ph + 1]));
            acc[ph] += ms;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    for (int ph = 0; ph < 3; ++ph) us[ph] = 1000.0 * acc[ph] / n_steps;
    sim->host_step += n_steps;
    return SPH_OK;
}

int sph_run_batch(const sph_params* p, int32_t B, const double* u_profiles, int32_t T, const sph_ctrl* pd,
                  double* y_out, int32_t* n_particles_out, void* stream)
{
    if (!p || B < 1 || T < 0) return fail(SPH_E_INVAL, "sph_run_batch: bad argument");
    sph_sim* s = nullptr;
    int rc = sph_create_batch(p, B, stream, &s);
    if (rc) return rc;
    if (n_particles_out) sph_counts(s, nullptr, n_particles_out, nullptr);
    rc = sph_step(s, u_profiles, T, pd, y_out, stream);
    if (rc == SPH_OK) rc = sph_check(s, nullptr, 0, stream);
    sph_destroy(s);
    return rc;
}

// Eq. 15 for the reference wall of the boundary sketch.  The lattice sums are
// taken point by point; the ghost sum, averaged over the offset of the ghost
// rows against the lattice, is the line integral (1 / s_g) \int W dx of each
// row (Simpson's rule on each polynomial piece of W along the row).
int sph_gamma1_estimate(const sph_params* p, double* gamma1)
{
    if (!p || !gamma1) return fail(SPH_E_INVAL, "sph_gamma1_estimate: NULL pointer");
    if (!(p->dx > 0) || !(p->h_over_dx > 0) || p->n_rings < 1)
        return fail(SPH_E_INVAL, "sph_gamma1_estimate: invalid sph_params");
    const double dx = p->dx, h = p->h_over_dx * p->dx, sg = ghost_ds(*p);
    const double sigma = p->sigma_cubic > 0.0 ? p->sigma_cubic : 5.0 / (14.0 * kPi);
    auto W = [&](double r) {  // Eq. 22 with the normalised constant
        const double q = r / h;
        if (q >= 2.0) return 0.0;
        double f = (2.0 - q) * (2.0 - q) * (2.0 - q);
        if (q < 1.0) f -= 4.0 * (1.0 - q) * (1.0 - q) * (1.0 - q);
        return sigma / (h * h) * f;
    };
    const int n = (int)std::ceil(2.0 * h / dx) + 1;
    double lattice = 0.0, fluid = 0.0;
    for (int b = -n; b <= n; ++b)
        for (int a = -n; a <= n; ++a) {
            const double w = W(dx * std::sqrt((double)(a * a + b * b)));
            lattice += w;
            if (b >= 0) fluid += w;
        }
    auto simpson = [&](double d, double x0, double x1) {  // \int_{x0}^{x1} W(sqrt(x^2 + d^2)) dx
        const int m = 4096;
        const double hx = (x1 - x0) / m;
        double acc = W(std::hypot(x0, d)) + W(std::hypot(x1, d));
        for (int i = 1; i < m; ++i) acc += (i & 1 ? 4.0 : 2.0) * W(std::hypot(x0 + i * hx, d));
        return acc * hx / 3.0;
    };
    double ghost = 0.0;
    for (int k = 0; k < p->n_rings; ++k) {
        const double d = 0.5 * dx + ((double)k + 0.5) * sg;  // depth of ghost row k below particle i
        if (d >= 2.0 * h) continue;
        const double x2 = std::sqrt(4.0 * h * h - d * d);
        double row;
        if (d < h) {
            const double x1 = std::sqrt(h * h - d * d);
            row = simpson(d, 0.0, x1) + simpson(d, x1, x2);
        } else {
            row = simpson(d, 0.0, x2);
        }
        ghost += 2.0 * row / sg;
    }
    if (!(ghost > 0.0)) return fail(SPH_E_INVAL, "sph_gamma1_estimate: no ghost row within the support");
    *gamma1 = (lattice - fluid) / ghost;
    return SPH_OK;
}

}  // extern "C"
