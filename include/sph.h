/*
 * sph.h -- C ABI of the GB300 SPH fuel-sloshing simulator.
 *
 * The simulator integrates the coupled fluid / rigid-body model of Section 3
 * of "Data-driven Learning of LPV Surrogate Models of Fuel Sloshing":
 * the state x = [r, theta, r_f, rdot, thetadot, rdot_f] evolves by the state
 * transition of Algorithm 1 under a first-order symplectic Euler step
 * (Section 3.4), with input u = [F_x, F_y, tau] applied at the centre of mass
 * (Section 2.1) and the measured output y of Eq. 1.
 *
 * Conventions for every call:
 *  - The return value is SPH_OK (0) or a negative SPH_E_* status; the text of
 *    the last error of the calling thread is available from sph_last_error().
 *  - The library owns the opaque sph_sim handle and every buffer inside it.
 *    The caller owns every array passed in or out.
 *  - Array pointers are DEVICE pointers unless the comment says "host".
 *    Arrays are dense, row-major, of the stated dtype and shape.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  Work is enqueued on it and the call returns without
 *    waiting, except where the comment says "blocks".
 *  - One sph_sim must not be used from two streams at the same time.
 *
 * Physical readings the simulator takes where the paper is silent or garbled
 * are stated on sph_params.
 */
#ifndef GB300_SPH_H
#define GB300_SPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    SPH_OK = 0,
    SPH_E_INVAL = -1,       /* bad argument (NULL, negative size, bad parameter) */
    SPH_E_NOMEM = -2,       /* device or host allocation failed                 */
    SPH_E_CUDA = -3,        /* a CUDA runtime call failed                       */
    SPH_E_DIVERGED = -4,    /* health check tripped (see SPH_FLAG_*)            */
    SPH_E_TIMEOUT = -5,     /* a bounded device-side wait gave up               */
    SPH_E_UNSUPPORTED = -6  /* valid request outside the implemented envelope   */
};

/* Health flags raised on the device and reported by sph_check(). */
enum {
    SPH_FLAG_NAN = 1,          /* a particle position or velocity became non-finite  */
    SPH_FLAG_ESCAPED = 2,      /* a particle left the tank: beyond the ghost rings by  */
                               /* more than a ring spacing and a grid cell            */
    SPH_FLAG_CELL_FULL = 4,    /* a grid cell exceeded SPH_CELL_CAPACITY particles    */
    SPH_FLAG_STAGE_FULL = 8,   /* a tile's staged neighbourhood exceeded shared memory */
    SPH_FLAG_TIMEOUT = 16      /* a bounded wait inside a persistent kernel gave up  */
};

#define SPH_CELL_CAPACITY 32   /* particles per neighbour-grid cell               */
#define SPH_NY 11              /* per-sample output record, see sph_step()         */

/*
 * Parameters of one tank.  Geometry, lattice and defaults:
 *  - fluid particles sit on the lattice ((i+1/2)dx, (j+1/2)dx) inside the
 *    disk of radius R - dx/2 and below the chord whose circular segment has
 *    area fill * pi * R^2; ghost particles sit on n_rings rings of radius
 *    R + (k+1/2) s_g, round(2 pi r_k / s_g) per ring, fixed in the body
 *    frame (Section 3.2, Eq. 21), with s_g = ghost_spacing * dx (Table 2's
 *    single layer of ghosts is 0.9 times as long as a fluid particle);
 *  - fluid and ghosts share the mass m = rho0 * dx^2, h = h_over_dx * dx;
 *  - sigma_cubic <= 0 selects the normalised cubic-spline constant
 *    5/(14 pi) (Eq. 22 prints 15/(14 pi), whose 2-D integral is 3);
 *  - ghost_pressure_sign = -1 makes the ghost pressure of Eq. 16 repel fluid
 *    at positive pressure; +1 is the literal sign of Algorithm 1;
 *  - ghost_pressure_clamp = 1 takes Eq. 16 with max(P_i, 0): the wall only
 *    pushes, and a particle under tension (P_i < 0, which the unclamped
 *    Eq. 11 gives near a free surface) is not pulled into the ghosts; 0 uses
 *    P_i as printed;
 *  - the density sum of Eq. 14 includes the particle itself, Eq. 11 is not
 *    clamped, and ghosts enter only Eqs. 14 and 16-19.
 */
typedef struct sph_params {
    double R;                   /* tank inner-wall radius [m]                 */
    double fill;                /* filled area fraction in [0, 1]             */
    double dx;                  /* fluid lattice spacing [m]                  */
    double h_over_dx;           /* smoothing length over spacing              */
    double rho0;                /* rest density [kg/m^2], Eq. 11              */
    double k;                   /* EOS stiffness, Eq. 11                      */
    double alpha;               /* viscous factor, Eq. 12                     */
    double beta;                /* boundary viscous factor, Eq. 18            */
    double gamma1;              /* boundary correcting factor, Eq. 14         */
    double eps;                 /* singularity guard, Eqs. 12 and 18          */
    double m_body;              /* rigid-body mass, Eq. 20                    */
    double J_body;              /* rigid-body inertia, Eq. 20                 */
    double dt;                  /* inner step [s]                             */
    double grav_x, grav_y;      /* fluid body acceleration (0 = zero gravity) */
    double sigma_cubic;         /* <= 0: 5/(14 pi)                            */
    double ghost_pressure_sign; /* -1 (default reading) or +1 (literal)       */
    int32_t n_rings;            /* ghost rings (>= 1)                         */
    int32_t outer_every;        /* inner steps per sampling period T_s (>= 1) */
    double ghost_spacing;       /* ghost spacing s_g over dx; <= 0 selects 1  */
    int32_t ghost_pressure_clamp; /* 1: Eq. 16 with max(P_i, 0); 0: as printed */
} sph_params;

/*
 * PD attitude controller of Eq. 28 (Section 5.1.1): at every sampling
 * instant tau_k = J w^2 (theta_ref_k - theta_k) - 2 xi J w thetadot_k is
 * computed from the body state and held (zero-order hold) for outer_every
 * inner steps, added to the input torque.
 */
typedef struct sph_ctrl {
    double J;                   /* <= 0: the body inertia J_body               */
    double omega;               /* bandwidth w [rad/s]                         */
    double xi;                  /* damping ratio                               */
    const double* theta_ref;    /* device [B, n_samples] reference, or NULL (0) */
    int32_t ref_stride;         /* elements between tanks in theta_ref          */
    int32_t enabled;            /* 0: no controller                            */
} sph_ctrl;

typedef struct sph_sim sph_sim;

/* Text of the calling thread's last error ("" if none). */
const char* sph_last_error(void);

/*
 * Builds B = 1 tank from *p (host struct), allocates its device state and
 * bins the initial fluid (at rest, body at the origin at rest).  Blocks.
 */
int sph_create(const sph_params* p, void* stream, sph_sim** out);

/*
 * Builds B independent tanks (host array p[B], uneven particle counts) that
 * step together: every call below then acts on all tanks at once and its
 * per-tank arrays gain a leading dimension B.  Blocks.
 */
int sph_create_batch(const sph_params* p, int32_t B, void* stream, sph_sim** out);

/* Frees everything owned by the handle.  Blocks on the device. NULL is a no-op. */
int sph_destroy(sph_sim* sim);

/* host: number of tanks, and per-tank fluid / ghost counts (arrays of B, or NULL). */
int sph_counts(const sph_sim* sim, int32_t* B, int32_t* n_fluid, int32_t* n_ghost);

/* host [n_ghost, 2]: body-frame ghost positions r_g^B of tank b (Eq. 21), in
 * the order the tank builder produced them (ring by ring, angle ascending). */
int sph_ghosts_body(const sph_sim* sim, int32_t b, double* gB_host);

/*
 * State transfer.  xv: float32 [N_total, 4] rows (x, y, vx, vy) in the world
 * frame, tanks concatenated, particles of a tank in builder order.  body:
 * float64 [B, 6] rows (r_x, r_y, theta, rdot_x, rdot_y, thetadot).
 * sph_set_state re-bins the fluid; it also clears the held controller torque.
 * xv may be NULL when the handle holds no fluid particles (every tank empty).
 */
int sph_get_state(sph_sim* sim, float* xv, double* body, void* stream);
int sph_set_state(sph_sim* sim, const float* xv, const double* body, void* stream);

/*
 * Advances every tank by n_steps inner steps (Algorithm 1 + symplectic Euler).
 *  u      float64 [B, n_steps, 3] input (F_x, F_y, tau) per inner step, or
 *         NULL for zero input.
 *  pd     host struct, or NULL (no controller).
 *  y_out  float64 [B, n_samples, SPH_NY] or NULL.  A sample is taken before
 *         every inner step whose global index is a multiple of outer_every;
 *         n_samples is the number of such steps in this call.  Record:
 *         r_x r_y theta rdot_x rdot_y thetadot | F_x F_y T (fluid force and
 *         torque on the body, Eq. 20) | c_x c_y (fluid centre of mass).
 * Health checks run on the device; call sph_check() to read them.
 */
int sph_step(sph_sim* sim, const double* u, int32_t n_steps, const sph_ctrl* pd, double* y_out, void* stream);

/*
 * Relaxation of a spawned fluid to rest (Section 5.1): n_steps inner steps
 * with zero input, the tank held at its current pose, and every fluid
 * velocity multiplied by (1 - damping) after its kick (0 <= damping < 1).
 * No samples are recorded.  Call sph_step afterwards for the physical model.
 */
int sph_relax(sph_sim* sim, int32_t n_steps, double damping, void* stream);

/* host: number of samples sph_step(n_steps) would record from the current step. */
int sph_samples_for(const sph_sim* sim, int32_t n_steps, int32_t* n_samples);

/*
 * One evaluation of Algorithm 1 on the current state, without stepping.
 * Every output is optional (NULL to skip); per-particle outputs are in the
 * order of sph_get_state.
 *  u        float64 [B, 3] input, or NULL (zero)
 *  rho      float32 [N] density (Eq. 14)
 *  drho     float32 [N] continuity sum: time derivative of Eq. 14 along the
 *           kinematic motion of fluid and ghosts
 *  acc      float32 [N, 2] fluid acceleration (Algorithm 1)
 *  nbr      int32 [N, 3] neighbour counts: fluid pairs r < 2h (j != i),
 *           ghosts r < 2h (Eq. 14), ghosts r < h (Eqs. 16, 18); the
 *           predicate is fma(dx,dx,dy*dy) < fl32(support^2) in FP32
 *  keys     int32 [N] cell key of the particle in the current neighbour grid
 *  body_out float64 [B, 6]: F_x F_y T (Eq. 20 fluid terms) and
 *           rddot_x rddot_y thetaddot (Eq. 20 with u)
 */
int sph_eval(sph_sim* sim, const double* u, float* rho, float* drho, float* acc, int32_t* nbr, int32_t* keys,
             double* body_out, void* stream);

/*
 * Neighbour-grid geometry of tank b (host outputs): cell side s =
 * 2h (1 + 1/1024), G cells per side, half-width W, and the FP64 anchor the
 * current grid is centred on.  A position x falls in column
 * floor(fl32(fl32(x - fl32(anchor - W)) * fl32(1/s))) clamped to [0, G-1].
 * Blocks.
 */
int sph_grid_info(sph_sim* sim, int32_t b, double* cell, double* half_width, int32_t* G, double* anchor_xy);

/*
 * Blocks until the stream is idle, then reports the OR of the health flags
 * of all tanks in *flags (may be NULL).  Returns SPH_E_DIVERGED if any flag
 * is set, SPH_E_TIMEOUT if only SPH_FLAG_TIMEOUT is set, else SPH_OK.
 * reset != 0 clears the flags afterwards.
 */
int sph_check(sph_sim* sim, int32_t* flags, int32_t reset, void* stream);

/* Blocks; total fluid-fluid (r < 2h, ordered) plus fluid-ghost (r < h) pair
 * interactions evaluated by all sph_step calls so far, summed over tanks. */
int sph_pair_count(sph_sim* sim, int64_t* pairs, void* stream);

/*
 * Forward-mode derivative (JVP) of K inner steps: the linearization of the
 * state transition of Algorithm 1 plus symplectic Euler along the
 * trajectory it computes (Section 3.5: Jacobians of the simulator).  The
 * primal state advances by K steps exactly as sph_step would with input u
 * (no controller), and a tangent is carried alongside it; the neighbour set
 * of each step is the one the primal uses.
 *  u        float64 [B, K, 3] input (NULL: zero)
 *  du       float64 [B, K, 3] tangent of the input (NULL: zero)
 *  dxv0     float32 [N, 4] tangent of the fluid state (x, y, vx, vy) (NULL: zero)
 *  dbody0   float64 [B, 6] tangent of the body state (NULL: zero)
 *  y_out    float64 [B, n_samples, SPH_NY] primal samples, as sph_step (NULL: none)
 *  dy_out   float64 [B, n_samples, SPH_NY] tangent of the samples (NULL: none)
 *  dxv_out  float32 [N, 4] tangent of the final fluid state (NULL: none)
 *  dbody_out float64 [B, 6] tangent of the final body state (NULL: none)
 * Tangent kernels exist for tile shapes up to 8x4; a larger chosen shape is
 * replaced by 8x4 for this call.  Allocates the tangent buffers on first use.
 */
int sph_jvp(sph_sim* sim, const double* u, const double* du, const float* dxv0, const double* dbody0, int32_t K,
            double* y_out, double* dy_out, float* dxv_out, double* dbody_out, void* stream);

/*
 * Jacobian-vector product of the continuous dynamics xdot = f(x, u)
 * (Section 5.2, the linearisation of Algorithm 1) at the current state, with
 * the neighbour set of the current step and no controller; the state is not
 * advanced.  Given the tangent of the state and of the input:
 *  u          float64 [B, 3] input (NULL: zero), device
 *  du         float64 [B, 3] input tangent (NULL: zero), device
 *  dxv        float32 [N, 4] fluid state tangent (dx, dy, dvx, dvy) in the
 *             order of sph_get_state (NULL: zero), device
 *  dbody      float64 [B, 6] body state tangent (r, theta, rdot, thetadot
 *             components as in sph_get_state; NULL: zero), device
 * returns the tangent of the fluid accelerations
 *  dacc       float32 [N, 2] out (NULL: skip), device
 * and of the body's F_x, F_y, T_b (Eq. 20 fluid terms) and rddot_x,
 * rddot_y, thetaddot (Eq. 20 with u)
 *  dbody_acc  float64 [B, 6] out (NULL: skip), device.
 * The position rows of f are the velocities themselves, so (dxv, dbody) and
 * these outputs give A v = (df/dx) v whole.  Tangent kernels exist for tile
 * shapes up to 8x4 (a larger shape is replaced by 8x4 for this call).
 * Allocates the tangent buffers on first use.
 */
int sph_eval_jvp(sph_sim* sim, const double* u, const double* du, const float* dxv, const double* dbody,
                 float* dacc, double* dbody_acc, void* stream);

/*
 * Reverse-mode (adjoint) derivative of K steps: the transpose of the map
 * sph_jvp linearises (Section 3.5, Jacobians of the simulator), no
 * controller, the neighbour set of each step frozen.  From the current state
 * and the input u, given the adjoints of that K-step call's samples and of
 * the final state, computes the adjoints of the initial state and of u:
 *  u          float64 [B, K, 3] input (NULL: zero), device
 *  ybar       float64 [B, n_samples, SPH_NY] adjoint of the samples sph_step(K)
 *             would record from the current step (NULL: zero)
 *  xvbar_K    float32 [N, 4] adjoint of the final fluid state (NULL: zero)
 *  bodybar_K  float64 [B, 6] adjoint of the final body state (NULL: zero)
 *  xvbar0     float32 [N, 4] out: adjoint of the initial fluid state (NULL: skip)
 *  bodybar0   float64 [B, 6] out: adjoint of the initial body state (NULL: skip)
 *  ubar       float64 [B, K, 3] out: adjoint of u (NULL: skip)
 * The forward pass keeps a checkpoint every checkpoint_every steps; the
 * reverse sweep recomputes each segment from its checkpoint and runs the
 * adjoint kernels on 4x4 tiles (device memory of about K / checkpoint_every +
 * checkpoint_every states, allocated for the call).  The simulator is left at
 * state K, as after sph_jvp.  Blocks until done.
 */
int sph_vjp(sph_sim* sim, const double* u, int32_t K, const double* ybar, const float* xvbar_K,
            const double* bodybar_K, float* xvbar0, double* bodybar0, double* ubar, int32_t checkpoint_every,
            void* stream);

/*
 * Kernel-shape control.  tile = 0 lets the library pick; otherwise one of
 * the codes 1..SPH_TILE_COUNT (cell blocks 2x2, 4x2, 4x4, 8x4, 8x8).
 * sph_autotune times every shape on the current state for `steps` steps,
 * restores the state and keeps the fastest; host out: chosen code and the
 * measured microseconds per step of each shape (array of SPH_TILE_COUNT, or
 * NULL).  Blocks.
 */
#define SPH_TILE_COUNT 5
int sph_set_tile(sph_sim* sim, int32_t tile);
int sph_autotune(sph_sim* sim, int32_t steps, int32_t* chosen, double* us_per_step, void* stream);

/*
 * Advances n_steps with zero input, launching the three kernels of a step
 * (density pass, force pass, body update) one by one with CUDA events
 * between them on `stream`; host us[3] receives their mean durations in
 * microseconds.  Blocks.
 */
int sph_time_kernels(sph_sim* sim, int32_t n_steps, double* us, void* stream);

/*
 * One-shot batched data generation (Eq. 2): builds B tanks from p[B], runs
 * T inner steps with inputs u_profiles [B, T, 3] (device) and controller pd
 * (host, may be NULL), writes the samples y_out [B, ceil(T/outer_every),
 * SPH_NY] (device) and the fluid counts n_particles_out[B] (host, may be
 * NULL), frees everything.  Blocks.
 */
int sph_run_batch(const sph_params* p, int32_t B, const double* u_profiles, int32_t T, const sph_ctrl* pd,
                  double* y_out, int32_t* n_particles_out, void* stream);

/*
 * Boundary correcting factor gamma1 of Eq. 14, estimated by Eq. 15 for a
 * representative wall configuration (Section 3.5; the boundary sketch of
 * Section 3.2): a straight wall, the fluid lattice of spacing dx on one side
 * (rows at (b + 1/2) dx, b >= 0), the n_rings ghost rows of spacing s_g =
 * ghost_spacing * dx on the other (rows at -(k + 1/2) s_g), and the particle
 * in the first fluid row.  rho_i / m_i is the kernel sum of an interior
 * particle of the same lattice, and the ghost sum is averaged over the
 * offset of the ghost rows along the wall:
 *   gamma1 = (sum_lattice W - sum_fluid W) / mean sum_ghost W   (Eq. 22 W).
 * Uses h_over_dx, dx, ghost_spacing, n_rings and sigma_cubic of *p (host);
 * writes *gamma1 (host).  Host computation only, no device work.
 * SPH_E_INVAL: NULL pointer, dx or h_over_dx not positive, n_rings < 1, or
 * no ghost row within the support.
 */
int sph_gamma1_estimate(const sph_params* p, double* gamma1);

/*
 * Density without any memory allocation.  The paper has no counterpart: this
 * call exists for callers that cannot call cudaMalloc, such as software that
 * must fix its device memory before it starts running (flight or real-time
 * loops) or a plugin inside an application that owns all device memory.
 *
 * Computes the ghost-corrected density of Eq. 14 (self term included, the
 * neighbour search of sph_eval) for a state the caller passes in:
 *  p       host tank parameters (geometry, h, rho0, gamma1, sigma_cubic)
 *  xv      device float32 [n_fluid, 4] fluid rows (x, y, vx, vy), world frame
 *  gB      device float64 [n_ghost, 2] ghost positions in the body frame
 *  body    HOST float64 [6] body state (r_x, r_y, theta, ...)
 *  rho     device float32 [n_fluid] output
 * Its working memory is one fixed device array inside the library (about
 * 8.6 MB, created when the library loads, kept by every GPU that loads the
 * library until the process exits): at most 256 x 256 neighbour-grid cells
 * (set by R / dx), 16384 ghosts and 32 particles per cell.  Larger requests
 * return SPH_E_UNSUPPORTED with a message, and a crowded cell returns
 * SPH_E_DIVERGED.  Each call looks up the array's device address in the
 * CUDA context current on the calling thread (this allocates nothing), so a
 * caller may switch contexts or reset the device between calls.  Every call
 * reuses the same array, so calls must not overlap on the GPU: two calls
 * issued on different streams or from different threads at the same time
 * race.  The call waits for the stream to finish (it reads an overflow flag
 * back), so it cannot be issued on a stream that is being captured into a
 * CUDA graph.
 */
int sph_density_noalloc(const sph_params* p, const float* xv, int32_t n_fluid, const double* gB, int32_t n_ghost,
                        const double* body, float* rho, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GB300_SPH_H */
