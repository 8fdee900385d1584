/*
 * sph_oracle.c -- plain, slow, FP64 CPU oracle of the two-dimensional SPH
 * fuel-sloshing model of "Data-driven Learning of LPV Surrogate Models of
 * Fuel Sloshing" (Section 3, Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
 * leg of bench.py load this library.  It shares no code, header, table or
 * constant with the CUDA library; the two meet only through arrays that the
 * tests pass to both.
 *
 * Everything is FP64 and follows the paper's formulas term by term:
 *   cubic-spline kernel ............ Eq. 22 (normalisation: see READINGS)
 *   spiky kernel ................... Eq. 23
 *   ghost kinematics ............... Eq. 21
 *   ghost-corrected density ........ Eq. 14
 *   equation of state .............. Eq. 11
 *   symmetric pressure force ....... Eq. 10 (enters with a minus, Eq. 9)
 *   artificial viscosity ........... Eq. 12
 *   ghost pressure / viscosity ..... Eqs. 16-19
 *   rigid body (Newton-Euler) ...... Eq. 20
 *   state transition ............... Algorithm 1
 *   first-order symplectic Euler ... Section 3.4
 *   PD attitude control, ZOH ....... Eq. 28 (Section 5.1.1)
 *
 * READINGS (where the paper is silent, garbled or inconsistent):
 *  R1 Eq. 22 prints 15/(14 pi h^2); that kernel integrates to 3 in 2-D, which
 *     contradicts the statement after Eq. 23 that it is normalised.  The
 *     normalised constant 5/(14 pi h^2) is the default (sigma_cubic <= 0);
 *     a caller may pass any other constant.
 *  R2 The density sum of Eq. 14 includes the particle itself (j = i).
 *  R3 Fluid and ghost particles share the mass m = rho0 * dx^2.
 *  R4 Eq. 11 is used unclamped: negative pressure is allowed.
 *  R5 Ghost particles enter only through Eqs. 14 and 16-19, never through the
 *     fluid-fluid sums of Eqs. 10 and 12 (no double counting).
 *  R6 The ghost pressure term acts like the fluid pressure term: with
 *     ghost_pressure_sign = -1 (default) it repels fluid for P > 0.  Algorithm 1
 *     adds Eq. 16 with a plus; ghost_pressure_sign = +1 runs that literal form.
 *  R7 The fluid-fluid artificial viscosity of Eq. 12 acts on every pair in
 *     the support (no clipping to approaching pairs); only Eq. 18 clips.
 *  R8 "First-order symplectic Euler" is kick-then-drift for fluid and body:
 *     v_{n+1} = v_n + dt a(x_n, v_n), x_{n+1} = x_n + dt v_{n+1}.
 *  R9 Tank construction: fluid on the lattice ((i+1/2)dx, (j+1/2)dx) inside
 *     the disk of radius R - dx/2 and below the chord whose circular segment
 *     has area fill * pi R^2; ghosts on n_rings rings of radius
 *     R + (k+1/2) s_g with round(2 pi r_k / s_g) equispaced particles each,
 *     s_g = ghost_spacing * dx (Table 2's single layer: 0.9 dx).
 *  R10 The "continuity sum" is the time derivative of Eq. 14 along the
 *     kinematic motion: m sum_f v_if . grad W + gamma1 m sum_g v_ig . grad W.
 *  R34 Eq. 16 takes P_i as printed by default; ghost_pressure_clamp = 1 takes
 *     max(P_i, 0), so that a particle under tension is not pulled into the
 *     wall (the paper is silent on the sign of P_i there).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Physical and numerical parameters (one tank).  Mirrored field by field by
 * the ctypes wrapper in oracle/sph.py. */
typedef struct {
    double R;            /* tank inner-wall radius [m] (Table 1)            */
    double fill;         /* filled fraction of the tank disk area           */
    double dx;           /* fluid lattice spacing [m]                       */
    double h_over_dx;    /* smoothing length h = h_over_dx * dx             */
    double rho0;         /* rest density [kg/m^2], Eq. 11                   */
    double k;            /* EOS stiffness, Eq. 11                           */
    double alpha;        /* viscous factor, Eq. 12                          */
    double beta;         /* fluid-boundary viscous factor, Eq. 18           */
    double gamma1;       /* boundary correcting factor, Eq. 14              */
    double eps;          /* singularity guard, Eqs. 12 and 18               */
    double m_body;       /* rigid-body mass, Eq. 20                         */
    double J_body;       /* rigid-body inertia, Eq. 20                      */
    double dt;           /* inner integration step                          */
    double grav_x;       /* fluid body acceleration (0: zero gravity)       */
    double grav_y;
    double sigma_cubic;  /* cubic-spline constant; <= 0 selects 5/(14 pi)   */
    double ghost_pressure_sign; /* -1 (reading R6) or +1 (literal)          */
    double ctrl_J;       /* controller inertia J of Eq. 28 (<= 0: J_body)   */
    double ctrl_omega;   /* controller bandwidth omega of Eq. 28            */
    double ctrl_xi;      /* controller damping xi of Eq. 28                 */
    int32_t n_rings;     /* number of ghost rings                           */
    int32_t outer_every; /* inner steps per sampling period T_s             */
    double ghost_spacing; /* ghost spacing over dx (Table 2: 0.9); <= 0: 1  */
    int32_t ghost_pressure_clamp; /* 1: Eq. 16 with max(P_i, 0) (reading R34) */
} orc_params;

#define ORC_NY 11 /* r_x r_y theta v_x v_y omega F_x F_y T c_x c_y */

static double orc_h(const orc_params* p) { return p->h_over_dx * p->dx; }
/* Ghost spacing s_g along a ring and between rings (R9). */
static double orc_ghost_ds(const orc_params* p)
{
    return (p->ghost_spacing > 0.0 ? p->ghost_spacing : 1.0) * p->dx;
}
static double orc_mass(const orc_params* p) { return p->rho0 * p->dx * p->dx; }
static double orc_sigma(const orc_params* p)
{
    return p->sigma_cubic > 0.0 ? p->sigma_cubic : 5.0 / (14.0 * M_PI);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Kernels, Eqs. 22 and 23                                            */
/* ------------------------------------------------------------------ */

/* Cubic spline W_cb(r; h) = sigma/h^2 * f(q), q = r/h (Eq. 22). */
double orc_w_cubic(double r, double h, double sigma)
{
    double q = r / h;
    double a = 2.0 - q, b = 1.0 - q, f;
    if (q < 1.0)
        f = a * a * a - 4.0 * b * b * b;
    else if (q < 2.0)
        f = a * a * a;
    else
        f = 0.0;
    return sigma / (h * h) * f;
}

/* dW_cb/dr, the radial derivative of Eq. 22. */
double orc_dw_cubic(double r, double h, double sigma)
{
    double q = r / h;
    double a = 2.0 - q, b = 1.0 - q, fp;
    if (q < 1.0)
        fp = -3.0 * a * a + 12.0 * b * b;
    else if (q < 2.0)
        fp = -3.0 * a * a;
    else
        fp = 0.0;
    return sigma / (h * h * h) * fp;
}

/* Spiky kernel W_s3(r; h) = 10/(pi h^5) (h - r)^3 for r <= h (Eq. 23). */
double orc_w_spiky(double r, double h)
{
    if (r > h) return 0.0;
    double d = h - r;
    return 10.0 / (M_PI * pow(h, 5)) * d * d * d;
}

/* dW_s3/dr. */
double orc_dw_spiky(double r, double h)
{
    if (r > h) return 0.0;
    double d = h - r;
    return -30.0 / (M_PI * pow(h, 5)) * d * d;
}

/* ------------------------------------------------------------------ */
/* Tank construction (reading R9)                                     */
/* ------------------------------------------------------------------ */

/* Area of {|p| <= R, p_y <= c}: the lower circular segment below the chord. */
static double segment_area(double R, double c)
{
    if (c <= -R) return 0.0;
    if (c >= R) return M_PI * R * R;
    return R * R * (M_PI - acos(c / R)) + c * sqrt(R * R - c * c);
}

/* Chord height c with segment_area(R, c) = fill * pi R^2, by bisection. */
double orc_fill_chord(double R, double fill)
{
    double target = fill * M_PI * R * R, lo = -R, hi = R;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (segment_area(R, mid) < target)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

static int lattice_extent(const orc_params* p) { return (int)ceil(p->R / p->dx) + 2; }

static int fluid_keep(const orc_params* p, double c, int i, int j, double* px, double* py)
{
    double x = ((double)i + 0.5) * p->dx;
    double y = ((double)j + 0.5) * p->dx;
    double rin = p->R - 0.5 * p->dx;
    double r2 = x * x + y * y;
    *px = x;
    *py = y;
    return (r2 <= rin * rin) && (y <= c);
}

static double ring_radius(const orc_params* p, int k) { return p->R + ((double)k + 0.5) * orc_ghost_ds(p); }

static int ring_count(const orc_params* p, int k)
{
    return (int)round(2.0 * M_PI * ring_radius(p, k) / orc_ghost_ds(p));
}

/* Particle counts of the tank of reading R9. */
int orc_tank_counts(const orc_params* p, int32_t* n_fluid, int32_t* n_ghost)
{
    if (!p || p->R <= 0 || p->dx <= 0 || p->fill < 0 || p->fill > 1 || p->n_rings < 0) return -1;
    double c = orc_fill_chord(p->R, p->fill), x, y;
    int L = lattice_extent(p), nf = 0, ng = 0;
    for (int j = -L; j <= L; ++j)
        for (int i = -L; i <= L; ++i) nf += fluid_keep(p, c, i, j, &x, &y);
    for (int k = 0; k < p->n_rings; ++k) ng += ring_count(p, k);
    *n_fluid = nf;
    *n_ghost = ng;
    return 0;
}

/* Fluid positions (row by row, y then x ascending) and body-frame ghost
 * positions (ring by ring, angle ascending). */
int orc_tank_build(const orc_params* p, double* xf, double* gB)
{
    double c = orc_fill_chord(p->R, p->fill), x, y;
    int L = lattice_extent(p), n = 0;
    for (int j = -L; j <= L; ++j)
        for (int i = -L; i <= L; ++i)
            if (fluid_keep(p, c, i, j, &x, &y)) {
                xf[2 * n] = x;
                xf[2 * n + 1] = y;
                ++n;
            }
    n = 0;
    for (int k = 0; k < p->n_rings; ++k) {
        double rk = ring_radius(p, k);
        int Nk = ring_count(p, k);
        for (int j = 0; j < Nk; ++j) {
            double phi = 2.0 * M_PI * (double)j / (double)Nk;
            gB[2 * n] = rk * cos(phi);
            gB[2 * n + 1] = rk * sin(phi);
            ++n;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Ghost kinematics, Eq. 21                                           */
/* ------------------------------------------------------------------ */

/* body = [r_x, r_y, theta, rdot_x, rdot_y, thetadot].  For each ghost:
 * arm = R(theta) r_g^B, r_g = arm + r, v_g = rdot + thetadot z x arm. */
void orc_ghost_world(int ng, const double* gB, const double* body, double* gw, double* gv, double* arm)
{
    double c = cos(body[2]), s = sin(body[2]);
    for (int g = 0; g < ng; ++g) {
        double bx = gB[2 * g], by = gB[2 * g + 1];
        double t1 = c * bx, t2 = s * by, t3 = s * bx, t4 = c * by;
        double ax = t1 - t2, ay = t3 + t4;
        if (arm) {
            arm[2 * g] = ax;
            arm[2 * g + 1] = ay;
        }
        gw[2 * g] = body[0] + ax;
        gw[2 * g + 1] = body[1] + ay;
        if (gv) {
            gv[2 * g] = body[3] - body[5] * ay;
            gv[2 * g + 1] = body[4] + body[5] * ax;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Neighbour search: a plain uniform bucket grid, or brute force        */
/* ------------------------------------------------------------------ */

typedef struct {
    int nx, ny, n;
    double x0, y0, cell;
    int* start; /* nx*ny + 1 */
    int* idx;   /* n */
} bucket_t;

static int bucket_build(bucket_t* b, int n, const double* xy, double cell)
{
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int i = 0; i < n; ++i) {
        xmin = fmin(xmin, xy[2 * i]);
        xmax = fmax(xmax, xy[2 * i]);
        ymin = fmin(ymin, xy[2 * i + 1]);
        ymax = fmax(ymax, xy[2 * i + 1]);
    }
    if (n == 0) xmin = xmax = ymin = ymax = 0.0;
    b->cell = cell;
    b->x0 = xmin - cell;
    b->y0 = ymin - cell;
    b->nx = (int)floor((xmax - b->x0) / cell) + 2;
    b->ny = (int)floor((ymax - b->y0) / cell) + 2;
    b->n = n;
    long nc = (long)b->nx * b->ny;
    b->start = (int*)calloc(nc + 1, sizeof(int));
    b->idx = (int*)malloc((n > 0 ? n : 1) * sizeof(int));
    int* key = (int*)malloc((n > 0 ? n : 1) * sizeof(int));
    if (!b->start || !b->idx || !key) {
        free(key);
        return -1;
    }
    for (int i = 0; i < n; ++i) {
        int cx = (int)floor((xy[2 * i] - b->x0) / cell);
        int cy = (int)floor((xy[2 * i + 1] - b->y0) / cell);
        key[i] = cy * b->nx + cx;
        b->start[key[i] + 1]++;
    }
    for (long c = 0; c < nc; ++c) b->start[c + 1] += b->start[c];
    int* fillp = (int*)malloc((nc > 0 ? nc : 1) * sizeof(int));
    if (!fillp) {
        free(key);
        return -1;
    }
    memcpy(fillp, b->start, nc * sizeof(int));
    for (int i = 0; i < n; ++i) b->idx[fillp[key[i]]++] = i; /* stable: ascending i per cell */
    free(fillp);
    free(key);
    return 0;
}

static void bucket_free(bucket_t* b)
{
    free(b->start);
    free(b->idx);
}

/* Collect the indices of points of `b` within distance < radius of (x, y),
 * in ascending index order per visited cell.  Returns the count. */
static int bucket_query(const bucket_t* b, const double* xy, double x, double y, double radius, int* out)
{
    int cnt = 0;
    double r2 = radius * radius;
    int cx = (int)floor((x - b->x0) / b->cell), cy = (int)floor((y - b->y0) / b->cell);
    for (int yy = cy - 1; yy <= cy + 1; ++yy) {
        if (yy < 0 || yy >= b->ny) continue;
        for (int xx = cx - 1; xx <= cx + 1; ++xx) {
            if (xx < 0 || xx >= b->nx) continue;
            int c = yy * b->nx + xx;
            for (int t = b->start[c]; t < b->start[c + 1]; ++t) {
                int j = b->idx[t];
                double ddx = x - xy[2 * j], ddy = y - xy[2 * j + 1];
                if (ddx * ddx + ddy * ddy < r2) out[cnt++] = j;
            }
        }
    }
    return cnt;
}

static int brute_query(int n, const double* xy, double x, double y, double radius, int* out)
{
    int cnt = 0;
    double r2 = radius * radius;
    for (int j = 0; j < n; ++j) {
        double ddx = x - xy[2 * j], ddy = y - xy[2 * j + 1];
        if (ddx * ddx + ddy * ddy < r2) out[cnt++] = j;
    }
    return cnt;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1: state -> accelerations                                */
/* ------------------------------------------------------------------ */

/*
 * Evaluates Algorithm 1 for one state.
 *   x, v      fluid positions / velocities, [nf, 2] world frame
 *   gB        ghost positions in the body frame, [ng, 2]
 *   body      [r_x, r_y, theta, rdot_x, rdot_y, thetadot]
 *   u         external input [F_x, F_y, tau] at the CoM (Section 2.1)
 *   brute     1: O(N^2) neighbour sums; 0: bucket grid (same sums)
 * Outputs (NULL allowed for the optional ones):
 *   rho, P    density (Eq. 14) and pressure (Eq. 11), [nf]
 *   acc       fluid accelerations, [nf, 2]
 *   drho      continuity sum (reading R10), [nf], optional
 *   fb        [F_x, F_y, T]: fluid force and torque on the body, Eq. 20
 *   body_acc  [rddot_x, rddot_y, thetaddot], Eq. 20 with u added
 *   fb_abs    [6], optional: scales of the terms that make up fb, summed over
 *             the fluid-ghost pairs (Eqs. 16-20) as magnitudes:
 *             [0..2] sum |f_x|, sum |f_y|, sum |arm x f| of the pair forces;
 *             [3..5] the same for rho_i df/drho_i (the change of each pair
 *             force under a relative change of its particle's density, which
 *             Eq. 11 amplifies by rho / (rho - rho0)).
 * Returns 0, or -1 on allocation failure.
 */
int orc_eval(const orc_params* p, int nf, const double* x, const double* v, int ng, const double* gB,
             const double* body, const double* u, int brute, double* rho, double* P, double* acc,
             double* drho, double* fb, double* body_acc, double* fb_abs)
{
    const double h = orc_h(p), m = orc_mass(p), sig = orc_sigma(p);
    const double H2 = 2.0 * h; /* cubic support */
    double* gw = (double*)malloc(sizeof(double) * 2 * (ng > 0 ? ng : 1));
    double* gv = (double*)malloc(sizeof(double) * 2 * (ng > 0 ? ng : 1));
    double* arm = (double*)malloc(sizeof(double) * 2 * (ng > 0 ? ng : 1));
    double* fbi = (double*)calloc(3 * (size_t)(nf > 0 ? nf : 1), sizeof(double));
    double* fba = (double*)calloc(6 * (size_t)(nf > 0 ? nf : 1), sizeof(double));
    if (!gw || !gv || !arm || !fbi || !fba) {
        free(gw), free(gv), free(arm), free(fbi), free(fba);
        return -1;
    }
    orc_ghost_world(ng, gB, body, gw, gv, arm); /* Algorithm 1, ghost loop */

    bucket_t bf, bg;
    if (!brute) {
        if (bucket_build(&bf, nf, x, H2) || bucket_build(&bg, ng, gw, H2)) return -1;
    }
    int cap = nf + ng + 1;
    int fail = 0;

    /* density (Eq. 14, reading R2) and continuity sum (reading R10) */
#pragma omp parallel
    {
        int* nb = (int*)malloc(sizeof(int) * cap);
        if (!nb) fail = 1;
#pragma omp for schedule(static)
        for (int i = 0; i < nf; ++i) {
            if (!nb) continue;
            double xi = x[2 * i], yi = x[2 * i + 1];
            int c = brute ? brute_query(nf, x, xi, yi, H2, nb) : bucket_query(&bf, x, xi, yi, H2, nb);
            double Sf = 0.0, Df = 0.0;
            for (int t = 0; t < c; ++t) {
                int j = nb[t];
                double rx = xi - x[2 * j], ry = yi - x[2 * j + 1];
                double r = sqrt(rx * rx + ry * ry);
                Sf += orc_w_cubic(r, h, sig);
                if (j != i && r > 0.0) {
                    double gw_r = orc_dw_cubic(r, h, sig) / r;
                    Df += ((v[2 * i] - v[2 * j]) * rx + (v[2 * i + 1] - v[2 * j + 1]) * ry) * gw_r;
                }
            }
            c = brute ? brute_query(ng, gw, xi, yi, H2, nb) : bucket_query(&bg, gw, xi, yi, H2, nb);
            double Sg = 0.0, Dg = 0.0;
            for (int t = 0; t < c; ++t) {
                int g = nb[t];
                double rx = xi - gw[2 * g], ry = yi - gw[2 * g + 1];
                double r = sqrt(rx * rx + ry * ry);
                Sg += orc_w_cubic(r, h, sig);
                if (r > 0.0) {
                    double gw_r = orc_dw_cubic(r, h, sig) / r;
                    Dg += ((v[2 * i] - gv[2 * g]) * rx + (v[2 * i + 1] - gv[2 * g + 1]) * ry) * gw_r;
                }
            }
            rho[i] = m * (Sf + p->gamma1 * Sg);  /* Eq. 14 */
            P[i] = p->k * (rho[i] - p->rho0);     /* Eq. 11 (reading R4) */
            if (drho) drho[i] = m * (Df + p->gamma1 * Dg);
        }
        free(nb);
    }

    /* forces: Eqs. 10 and 12 between fluid particles, Eqs. 16-19 with ghosts */
#pragma omp parallel
    {
        int* nb = (int*)malloc(sizeof(int) * cap);
        if (!nb) fail = 1;
#pragma omp for schedule(static)
        for (int i = 0; i < nf; ++i) {
            if (!nb) continue;
            double xi = x[2 * i], yi = x[2 * i + 1];
            double vxi = v[2 * i], vyi = v[2 * i + 1];
            double Pi_r2 = P[i] / (rho[i] * rho[i]);
            double ax = 0.0, ay = 0.0;
            int c = brute ? brute_query(nf, x, xi, yi, H2, nb) : bucket_query(&bf, x, xi, yi, H2, nb);
            for (int t = 0; t < c; ++t) {
                int j = nb[t];
                if (j == i) continue;
                double rx = xi - x[2 * j], ry = yi - x[2 * j + 1];
                double r2 = rx * rx + ry * ry, r = sqrt(r2);
                if (r <= 0.0) continue;
                double gradW = orc_dw_cubic(r, h, sig) / r; /* grad_i W = dW/dr r_ij / |r_ij| */
                double press = -(Pi_r2 + P[j] / (rho[j] * rho[j]));            /* -F^pressure, Eq. 10 */
                double vdotr = (vxi - v[2 * j]) * rx + (vyi - v[2 * j + 1]) * ry;
                double visc = 2.0 * p->alpha * h / (rho[i] + rho[j]) * vdotr / (r2 + p->eps * h * h); /* Eq. 12 */
                double s = m * (press + visc) * gradW;
                ax += s * rx;
                ay += s * ry;
            }
            c = brute ? brute_query(ng, gw, xi, yi, h, nb) : bucket_query(&bg, gw, xi, yi, h, nb);
            double fx_b = 0.0, fy_b = 0.0, t_b = 0.0;
            double sa[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            for (int t = 0; t < c; ++t) {
                int g = nb[t];
                double rx = xi - gw[2 * g], ry = yi - gw[2 * g + 1];
                double r2 = rx * rx + ry * ry, r = sqrt(r2);
                if (r <= 0.0) continue;
                double gradWs = orc_dw_spiky(r, h) / r;
                /* Eq. 16 with the sign of reading R6 (g2f pressure); reading
                 * R34 optionally clamps P_i at zero (the wall only pushes) */
                double qg = p->ghost_pressure_clamp ? fmax(Pi_r2, 0.0) : Pi_r2;
                double fp = p->ghost_pressure_sign * 2.0 * m * m * qg * gradWs;
                /* Eq. 18 with rho_g = rho_i (g2f viscosity) */
                double vdotr = (vxi - gv[2 * g]) * rx + (vyi - gv[2 * g + 1]) * ry;
                double fv = m * m * 2.0 * p->beta / (rho[i] + rho[i]) * fmin(vdotr, 0.0) / (r2 + p->eps * h * h) * gradWs;
                double fx = (fp + fv) * rx, fy = (fp + fv) * ry;
                ax += fx / m;
                ay += fy / m;
                /* Eqs. 17 and 19: f2g = -g2f; Eq. 20 force and torque about r */
                fx_b -= fx;
                fy_b -= fy;
                t_b -= arm[2 * g] * fy - arm[2 * g + 1] * fx;
                /* magnitudes: the pair force, and rho_i d/drho_i of it (Eq. 11:
                 * rho d(P/rho^2)/drho = k/rho - 2P/rho^2; Eq. 18: -f_v) */
                double dp = (qg == Pi_r2) ? p->ghost_pressure_sign * 2.0 * m * m * (p->k / rho[i] - 2.0 * Pi_r2) * gradWs : 0.0;
                double dx_ = (dp - fv) * rx, dy_ = (dp - fv) * ry;
                sa[0] += fabs(fx);
                sa[1] += fabs(fy);
                sa[2] += fabs(arm[2 * g] * fy - arm[2 * g + 1] * fx);
                sa[3] += fabs(dx_);
                sa[4] += fabs(dy_);
                sa[5] += fabs(arm[2 * g] * dy_ - arm[2 * g + 1] * dx_);
            }
            for (int q = 0; q < 6; ++q) fba[6 * i + q] = sa[q];
            acc[2 * i] = ax + p->grav_x; /* F^external = m g */
            acc[2 * i + 1] = ay + p->grav_y;
            fbi[3 * i] = fx_b;
            fbi[3 * i + 1] = fy_b;
            fbi[3 * i + 2] = t_b;
        }
        free(nb);
    }
    double Fx = 0.0, Fy = 0.0, T = 0.0;
    for (int i = 0; i < nf; ++i) {
        Fx += fbi[3 * i];
        Fy += fbi[3 * i + 1];
        T += fbi[3 * i + 2];
    }
    if (fb) {
        fb[0] = Fx;
        fb[1] = Fy;
        fb[2] = T;
    }
    if (fb_abs) {
        for (int q = 0; q < 6; ++q) fb_abs[q] = 0.0;
        for (int i = 0; i < nf; ++i)
            for (int q = 0; q < 6; ++q) fb_abs[q] += fba[6 * i + q];
    }
    if (body_acc) { /* Eq. 20 */
        body_acc[0] = (Fx + u[0]) / p->m_body;
        body_acc[1] = (Fy + u[1]) / p->m_body;
        body_acc[2] = (T + u[2]) / p->J_body;
    }
    if (!brute) {
        bucket_free(&bf);
        bucket_free(&bg);
    }
    free(gw), free(gv), free(arm), free(fbi), free(fba);
    return fail ? -1 : 0;
}

/* Shepard sum S_i = sum_j (m/rho_j) W_ij over fluid j (Eq. 7 with A = 1). */
int orc_shepard(const orc_params* p, int nf, const double* x, const double* rho, double* S)
{
    const double h = orc_h(p), m = orc_mass(p), sig = orc_sigma(p);
    for (int i = 0; i < nf; ++i) {
        double s = 0.0;
        for (int j = 0; j < nf; ++j) {
            double rx = x[2 * i] - x[2 * j], ry = x[2 * i + 1] - x[2 * j + 1];
            double r = sqrt(rx * rx + ry * ry);
            if (r < 2.0 * h) s += m / rho[j] * orc_w_cubic(r, h, sig);
        }
        S[i] = s;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Time integration (Section 3.4, reading R8) and the multi-rate loop  */
/* ------------------------------------------------------------------ */

/*
 * Runs n_steps inner steps in place.
 *   u          [n_steps, 3] external input per inner step (may be NULL = 0)
 *   theta_ref  reference angle per sampling period (may be NULL); used when
 *              use_ctrl != 0 by the PD law of Eq. 28 under zero-order hold:
 *              tau_k = J w^2 (ref_k - theta_k) - 2 xi J w thetadot_k.
 *   damping    velocity damping factor per step (0 for the physical model).
 *              damping > 0 is the relaxation of a spawned fluid to rest
 *              (Section 5.1): the tank is then held at its pose.
 *   y          [ceil(n_steps/outer_every), 11] outputs sampled before the
 *              step whose index is a multiple of outer_every (may be NULL):
 *              body state, fluid force/torque on the body, fluid CoM.
 *   fb_hist    [n_steps, 3] fluid force/torque on the body at every step
 *              (may be NULL).
 */
int orc_run(const orc_params* p, int nf, double* x, double* v, int ng, const double* gB, double* body,
            const double* u, const double* theta_ref, int use_ctrl, int n_steps, double damping, int brute,
            double* y, double* fb_hist)
{
    double* rho = (double*)malloc(sizeof(double) * (nf > 0 ? nf : 1));
    double* P = (double*)malloc(sizeof(double) * (nf > 0 ? nf : 1));
    double* acc = (double*)malloc(sizeof(double) * 2 * (nf > 0 ? nf : 1));
    if (!rho || !P || !acc) {
        free(rho), free(P), free(acc);
        return -1;
    }
    const int outer = p->outer_every > 0 ? p->outer_every : 1;
    const double dt = p->dt;
    const double Jc = p->ctrl_J > 0.0 ? p->ctrl_J : p->J_body;
    double tau_c = 0.0;
    int rc = 0;
    for (int n = 0; n < n_steps; ++n) {
        int k = n / outer;
        if (n % outer == 0 && use_ctrl) { /* Eq. 28, sampled, held by ZOH */
            double ref = theta_ref ? theta_ref[k] : 0.0;
            tau_c = Jc * p->ctrl_omega * p->ctrl_omega * (ref - body[2]) - 2.0 * p->ctrl_xi * Jc * p->ctrl_omega * body[5];
        }
        double uu[3] = {u ? u[3 * n] : 0.0, u ? u[3 * n + 1] : 0.0, (u ? u[3 * n + 2] : 0.0) + tau_c};
        double fb[3], ba[3];
        if (orc_eval(p, nf, x, v, ng, gB, body, uu, brute, rho, P, acc, NULL, fb, ba, NULL)) {
            rc = -1;
            break;
        }
        if (fb_hist) {
            fb_hist[3 * n] = fb[0];
            fb_hist[3 * n + 1] = fb[1];
            fb_hist[3 * n + 2] = fb[2];
        }
        if (y && n % outer == 0) {
            double cx = 0.0, cy = 0.0;
            for (int i = 0; i < nf; ++i) {
                cx += x[2 * i];
                cy += x[2 * i + 1];
            }
            double* yk = y + (size_t)ORC_NY * k;
            for (int q = 0; q < 6; ++q) yk[q] = body[q];
            yk[6] = fb[0];
            yk[7] = fb[1];
            yk[8] = fb[2];
            yk[9] = nf ? cx / nf : 0.0;
            yk[10] = nf ? cy / nf : 0.0;
        }
        /* kick then drift (reading R8) */
        for (int i = 0; i < nf; ++i) {
            v[2 * i] = (v[2 * i] + dt * acc[2 * i]) * (1.0 - damping);
            v[2 * i + 1] = (v[2 * i + 1] + dt * acc[2 * i + 1]) * (1.0 - damping);
            x[2 * i] += dt * v[2 * i];
            x[2 * i + 1] += dt * v[2 * i + 1];
        }
        if (damping > 0.0) continue; /* relaxation: the tank is held fixed */
        body[3] += dt * ba[0];
        body[4] += dt * ba[1];
        body[5] += dt * ba[2];
        body[0] += dt * body[3];
        body[1] += dt * body[4];
        body[2] += dt * body[5];
    }
    free(rho), free(P), free(acc);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Integer decisions in FP32 (the precision the GPU kernels take them in) */
/* ------------------------------------------------------------------ */

/*
 * Neighbour-grid convention: square cells of side s = 2h (1 + 1/1024),
 * half-width W = R + (n_rings + 1) max(dx, s_g) + 2 s around an FP64 anchor
 * point (s_g the ghost spacing),
 * G = ceil(2W / s) cells per side.  A position x (FP32) falls in column
 *   c = floor( fl32( fl32(x - o) * fl32(1/s) ) ),  o = fl32(anchor - W),
 * clamped to [0, G-1]; the key is row * G + column.
 */
int orc_grid_dims(const orc_params* p, double* cell, double* half_width, int32_t* G)
{
    double s = 2.0 * orc_h(p) * (1.0 + 1.0 / 1024.0);
    double W = p->R + ((double)p->n_rings + 1.0) * fmax(p->dx, orc_ghost_ds(p)) + 2.0 * s;
    *cell = s;
    *half_width = W;
    *G = (int32_t)ceil(2.0 * W / s);
    return 0;
}

int orc_cell_keys_f32(const orc_params* p, int n, const float* xy, int stride, double anchor_x, double anchor_y,
                      int32_t* keys)
{
    double s, W;
    int32_t G;
    orc_grid_dims(p, &s, &W, &G);
    float ox = (float)(anchor_x - W), oy = (float)(anchor_y - W);
    float inv = (float)(1.0 / s);
    for (int i = 0; i < n; ++i) {
        float tx = xy[(size_t)stride * i] - ox;
        float ty = xy[(size_t)stride * i + 1] - oy;
        tx = tx * inv;
        ty = ty * inv;
        int cx = (int)floorf(tx), cy = (int)floorf(ty);
        if (cx < 0) cx = 0;
        if (cx > G - 1) cx = G - 1;
        if (cy < 0) cy = 0;
        if (cy > G - 1) cy = G - 1;
        keys[i] = cy * G + cx;
    }
    return 0;
}

/*
 * Neighbour counts with FP32 predicates (brute force), for the particles
 * listed in qidx[nq] (all particles if qidx is NULL):
 *   n_ff[i]   #{ j != i : fma(dx, dx, dy*dy) < fl32((2h)^2) },  dx = x_i - x_j
 *   n_fg2[i]  #{ g : same with (2h)^2 }  (ghosts entering Eq. 14)
 *   n_fg1[i]  #{ g : same with h^2 }     (ghosts entering Eqs. 16 and 18)
 * For ghosts dx = (x_i - hi) - lo, hi = fl32(r_g), lo = fl32(r_g - hi),
 * r_g from Eq. 21 in FP64.
 */
int orc_neighbor_counts_f32(const orc_params* p, int nf, const float* xy, int stride, int ng, const double* gB,
                            const double* body, int nq, const int32_t* qidx, int32_t* n_ff, int32_t* n_fg2,
                            int32_t* n_fg1)
{
    double h = orc_h(p);
    float R2 = (float)((2.0 * h) * (2.0 * h));
    float h2 = (float)(h * h);
    double* gw = (double*)malloc(sizeof(double) * 2 * (ng > 0 ? ng : 1));
    if (!gw) return -1;
    orc_ghost_world(ng, gB, body, gw, NULL, NULL);
    if (!qidx) nq = nf;
    for (int q = 0; q < nq; ++q) {
        int i = qidx ? qidx[q] : q;
        float xi = xy[(size_t)stride * i], yi = xy[(size_t)stride * i + 1];
        int c = 0;
        for (int j = 0; j < nf; ++j) {
            if (j == i) continue;
            float ddx = xi - xy[(size_t)stride * j];
            float ddy = yi - xy[(size_t)stride * j + 1];
            float r2 = fmaf(ddx, ddx, ddy * ddy);
            c += r2 < R2;
        }
        n_ff[q] = c;
        int c2 = 0, c1 = 0;
        for (int g = 0; g < ng; ++g) {
            float hx = (float)gw[2 * g], hy = (float)gw[2 * g + 1];
            float lx = (float)(gw[2 * g] - (double)hx), ly = (float)(gw[2 * g + 1] - (double)hy);
            float ddx = (xi - hx) - lx;
            float ddy = (yi - hy) - ly;
            float r2 = fmaf(ddx, ddx, ddy * ddy);
            c2 += r2 < R2;
            c1 += r2 < h2;
        }
        n_fg2[q] = c2;
        n_fg1[q] = c1;
    }
    free(gw);
    return 0;
}

/*
 * Neighbour counts with the FP64 predicate r^2 < (2h)^2 (and r^2 < h^2) on
 * the FP32 inputs: the particle positions are the FP32 numbers given, taken
 * exactly into FP64; the ghosts are their FP64 world positions (Eq. 21).  The
 * differences of FP32 numbers are exact in FP64, so only the final sum of
 * squares rounds.  For each count the band count is the number of pairs with
 * |r^2 - s^2| <= band * s^2 (s the support): pairs so close to the support
 * boundary that a predicate evaluated in a lower precision may decide them
 * either way, where W and grad W vanish continuously.
 *   out[q][0..5] = n_ff, band_ff, n_fg2, band_fg2, n_fg1, band_fg1
 * for the particles listed in qidx[nq] (all particles if qidx is NULL).
 */
int orc_neighbor_counts_f64(const orc_params* p, int nf, const float* xy, int stride, int ng, const double* gB,
                            const double* body, int nq, const int32_t* qidx, double band, int32_t* out)
{
    const double h = orc_h(p);
    const double S2 = (2.0 * h) * (2.0 * h), H2 = h * h;
    double* gw = (double*)malloc(sizeof(double) * 2 * (ng > 0 ? ng : 1));
    if (!gw) return -1;
    orc_ghost_world(ng, gB, body, gw, NULL, NULL);
    if (!qidx) nq = nf;
#pragma omp parallel for schedule(static)
    for (int q = 0; q < nq; ++q) {
        int i = qidx ? qidx[q] : q;
        double xi = (double)xy[(size_t)stride * i], yi = (double)xy[(size_t)stride * i + 1];
        int n = 0, nb = 0;
        for (int j = 0; j < nf; ++j) {
            if (j == i) continue;
            double ddx = xi - (double)xy[(size_t)stride * j], ddy = yi - (double)xy[(size_t)stride * j + 1];
            double r2 = ddx * ddx + ddy * ddy;
            n += r2 < S2;
            nb += fabs(r2 - S2) <= band * S2;
        }
        int n2 = 0, b2 = 0, n1 = 0, b1 = 0;
        for (int g = 0; g < ng; ++g) {
            double ddx = xi - gw[2 * g], ddy = yi - gw[2 * g + 1];
            double r2 = ddx * ddx + ddy * ddy;
            n2 += r2 < S2;
            b2 += fabs(r2 - S2) <= band * S2;
            n1 += r2 < H2;
            b1 += fabs(r2 - H2) <= band * H2;
        }
        int32_t* o = out + 6 * (size_t)q;
        o[0] = n, o[1] = nb, o[2] = n2, o[3] = b2, o[4] = n1, o[5] = b1;
    }
    free(gw);
    return 0;
}

/*
 * The discrete switches of Algorithm 1 for one state (FP64): per fluid
 * particle i,
 *   out[i][0]  #{ j != i : r_ij < 2h }            (Eqs. 10, 12, 14)
 *   out[i][1]  #{ g : r_ig < 2h }                 (Eq. 14)
 *   out[i][2]  #{ g : r_ig < h }                  (Eqs. 16, 18)
 *   out[i][3]  #{ g : r_ig < h, v_ig . r_ig < 0 } (the min(., 0) of Eq. 18)
 * Two states whose counts agree for every particle take every switch the
 * same way, so the step map is smooth between them; where they differ, a
 * pair crossed a support or the viscosity clip between them.
 */
int orc_switch_counts(const orc_params* p, int nf, const double* x, const double* v, int ng, const double* gB,
                      const double* body, int32_t* out)
{
    const double h = orc_h(p);
    double* gw = (double*)malloc(sizeof(double) * 2 * (ng > 0 ? ng : 1));
    double* gv = (double*)malloc(sizeof(double) * 2 * (ng > 0 ? ng : 1));
    if (!gw || !gv) {
        free(gw), free(gv);
        return -1;
    }
    orc_ghost_world(ng, gB, body, gw, gv, NULL);
    bucket_t bf, bg;
    if (bucket_build(&bf, nf, x, 2.0 * h) || bucket_build(&bg, ng, gw, 2.0 * h)) return -1;
    int fail = 0;
#pragma omp parallel
    {
        int* nb = (int*)malloc(sizeof(int) * (nf + ng + 1));
        if (!nb) fail = 1;
#pragma omp for schedule(static)
        for (int i = 0; i < nf; ++i) {
            if (!nb) continue;
            const double xi = x[2 * i], yi = x[2 * i + 1];
            int32_t* o = out + 4 * (size_t)i;
            o[0] = bucket_query(&bf, x, xi, yi, 2.0 * h, nb) - 1; /* the particle itself is in its own list */
            o[1] = bucket_query(&bg, gw, xi, yi, 2.0 * h, nb);
            int c = bucket_query(&bg, gw, xi, yi, h, nb), app = 0;
            for (int t = 0; t < c; ++t) {
                int g = nb[t];
                double vr = (v[2 * i] - gv[2 * g]) * (xi - gw[2 * g]) + (v[2 * i + 1] - gv[2 * g + 1]) * (yi - gw[2 * g + 1]);
                app += vr < 0.0;
            }
            o[2] = c;
            o[3] = app;
        }
        free(nb);
    }
    bucket_free(&bf);
    bucket_free(&bg);
    free(gw), free(gv);
    return fail ? -1 : 0;
}

/*
 * Pair interactions of one evaluation of Algorithm 1 (FP64 predicates):
 * ordered fluid pairs j != i with r < 2h (Eqs. 10, 12) plus fluid-ghost pairs
 * with r < h (Eqs. 16, 18).
 */
long long orc_pair_count(const orc_params* p, int nf, const double* x, int ng, const double* gB, const double* body)
{
    const double h = orc_h(p);
    double* gw = (double*)malloc(sizeof(double) * 2 * (ng > 0 ? ng : 1));
    int* nb = (int*)malloc(sizeof(int) * (nf + ng + 1));
    if (!gw || !nb) {
        free(gw), free(nb);
        return -1;
    }
    orc_ghost_world(ng, gB, body, gw, NULL, NULL);
    bucket_t bf, bg;
    if (bucket_build(&bf, nf, x, 2.0 * h) || bucket_build(&bg, ng, gw, 2.0 * h)) return -1;
    long long total = 0;
    for (int i = 0; i < nf; ++i) {
        int c = bucket_query(&bf, x, x[2 * i], x[2 * i + 1], 2.0 * h, nb);
        total += c - 1; /* the particle itself is in its own list */
        total += bucket_query(&bg, gw, x[2 * i], x[2 * i + 1], h, nb);
    }
    bucket_free(&bf);
    bucket_free(&bg);
    free(gw), free(nb);
    return total;
}
