/*
 * lpv.h -- C ABI of the GB300 LPV surrogate of fuel sloshing (Section 4 of
 * "Data-driven Learning of LPV Surrogate Models of Fuel Sloshing").
 *
 * Model (Eqs. 24 and 25, feedthrough D = 0 as in Section 5.3.2):
 *     x_{k+1} = A(p_k) x_k + B(p_k) u_k,     y_k = C(p_k) x_k,
 *     [[A, B], [C, D]] = M_0 + sum_{i=1..n_p} p_{k,i} M_i,
 * with an external scheduling signal p (here fill fraction and body angular
 * rate) instead of a learned scheduling network.  Data and outputs are in
 * physical units; the model keeps per-channel scales and works internally on
 * u / s_u, y / s_y and (p - m_p) / s_p.  The state starts at zero (the fluid
 * starts at rest, Section 2.2), so y holds deviations from the at-rest loads.
 *
 * Conventions (as in sph.h): SPH-style int status codes (0 = OK, negative =
 * error, text from sph_last_error()), library-owned opaque handle, device
 * pointers unless marked "host", row-major dense arrays, `stream` is a
 * cudaStream_t passed as void*.
 */
#ifndef GB300_LPV_H
#define GB300_LPV_H

#include <stdint.h>

#include "sph.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lpv_config {
    int32_t n_x, n_u, n_y, n_p;  /* n_x + n_u <= 15, n_x + n_y <= 16, n_p <= 2 */
    int32_t na;                  /* ARX order of the least-squares start; n_x = na * n_y */
    int32_t adam_iters;          /* Adam iterations per restart (Section 5.3.2: 2000)    */
    int32_t restarts;            /* random restarts, best training loss kept (paper: 8)  */
    int32_t lbfgs_iters;         /* L-BFGS iterations after Adam, per restart (0: none)  */
    double lr, beta1, beta2, adam_eps;  /* Adam step size and moments                 */
    double sigma2;               /* l2 weight of the parameters, Eq. 27 (paper: 1e-4)   */
    double init_scale;           /* std of the normal draw of M_1..M_np per restart      */
    uint64_t seed;               /* seed of that draw                                    */
    double rho_max;              /* spectral radius bound of the least-squares start     */
} lpv_config;

/* Rigid body and attitude controller of the closed loop (Eq. 20 without fluid
 * particles, Eq. 28 under zero-order hold). */
typedef struct lpv_body {
    double m, J;                 /* body mass and inertia                              */
    double Ts;                   /* sampling period of the surrogate                   */
    int32_t n_sub;               /* kick-then-drift substeps of the body per period    */
    int32_t reserved;
    double ctrl_J, ctrl_omega, ctrl_xi;  /* PD gains J w^2, 2 xi J w; ctrl_J <= 0: J   */
} lpv_body;

typedef struct lpv_model lpv_model;

int lpv_create(const lpv_config* cfg, lpv_model** out);
int lpv_destroy(lpv_model* m);

/*
 * Parameters in host memory.  W: float32 [1 + n_p][n_x + n_y][n_x + n_u], the
 * blocks M_0..M_np (entries of the D blocks are ignored and kept zero).
 * scales: float32 [n_u + n_y + 4 n_p] = s_u, s_y, m_p, s_p, p_lo, p_hi: input
 * and output scales, scheduling mean and standard deviation, and the range of
 * the scheduling the model was identified on (+-inf: unbounded).
 */
int lpv_set_params(lpv_model* m, const float* W, const float* scales);
int lpv_get_params(const lpv_model* m, float* W, float* scales);

/*
 * Data sets D_N (Eq. 2): u float32 [n_traj, T, n_u], y float32 [n_traj, T,
 * n_y], p float32 [n_traj, T, n_p], device.
 *
 * lpv_normalize: sets s_u, s_y to the root mean square, m_p, s_p to the
 * mean and standard deviation and p_lo, p_hi to the minimum and maximum of
 * each channel over the data (FP64 sums).
 *
 * lpv_init_ls: FP64 least-squares fit of the MIMO ARX model
 *   y_k = sum_{i=1..na} A_i y_{k-i} + sum_{i=1..na} B_i u_{k-i}
 * on the normalised data (normal equations accumulated and solved in FP64 on
 * the device), written as M_0 in observer-canonical form; M_i (i >= 1) = 0.
 * The start is a stable model: when the spectral radius rho of the state
 * matrix exceeds cfg.rho_max (> 0), every characteristic root is scaled by
 * lam = rho_max / rho (A_i <- lam^i A_i, B_i <- lam^i B_i, so the impulse
 * response h_k becomes lam^k h_k); rho is estimated on the device from
 * ||A^(2^s)||^(1/2^s) by 40 normalised FP64 squarings.  With 0 < rho_max < 1
 * that stable model is then handed over as its balanced realisation (equal,
 * diagonal controllability and observability Gramians, states by decreasing
 * Hankel singular value, each column of C signed so that its largest entry is
 * positive): the same input-output map, but without the near-defective
 * companion structure whose poles move by O(delta^(1/n)) under rounding of
 * the weights.
 * theta_out (host, may be NULL) receives the regression coefficients
 * [na*n_y + na*n_u][n_y] (rows: y_{k-1}..y_{k-na}, u_{k-1}..u_{k-na}).  Blocks.
 */
int lpv_normalize(lpv_model* m, const float* u, const float* y, const float* p, int32_t n_traj, int32_t T,
                  void* stream);
int lpv_init_ls(lpv_model* m, const float* u, const float* y, int32_t n_traj, int32_t T, double* theta_out,
                void* stream);

/*
 * Loss of Eqs. 4 and 27 on normalised data, free-run simulation from x_0 = 0:
 *   J = mean_{traj, k} ||y_k - y_hat_k||^2 + sigma2 / 2 ||W||^2,
 * and its gradient by backpropagation through time on tensor cores
 * (mma.sync BF16 with FP32 accumulation, operands split in two BF16 halves).
 * loss (host) and grad (host, layout of W) may be NULL.  Blocks.
 */
int lpv_loss_grad(lpv_model* m, const float* u, const float* y, const float* p, int32_t n_traj, int32_t T,
                  double* loss, float* grad, void* stream);

/*
 * iters Adam steps on the data (Section 4: Adam before L-BFGS; L-BFGS is not
 * implemented).  A step whose loss comes out non-finite or more than ten
 * times the loss of the last accepted iterate is rejected: the weights return
 * to that iterate and the same Adam direction is retried with half the step
 * (the halving persists until the optimiser is reset by lpv_set_params or
 * lpv_init_ls).  loss_history (host [iters], may be NULL) records the loss of
 * every iterate tried.  Blocks.
 */
int lpv_train(lpv_model* m, const float* u, const float* y, const float* p, int32_t n_traj, int32_t T,
              int32_t iters, double* loss_history, void* stream);

/*
 * The identification of Section 5.3.2: lpv_normalize, lpv_init_ls, then for
 * each restart the B and C blocks of M_1..M_np drawn from N(0,
 * init_scale^2) (their A blocks start at 0, so the start keeps the stable
 * spectrum of M_0 for every p), adam_iters Adam steps and lbfgs_iters
 * L-BFGS iterations; keeps the restart with the lowest training loss.  best_loss (host)
 * may be NULL.  Returns SPH_E_DIVERGED (and no model) when no restart ends
 * with a finite loss.  Blocks.
 */
/*
 * iters L-BFGS iterations (Section 5.3.2: after Adam): two-loop recursion over
 * the last 10 curvature pairs in FP64 on the device, unit quasi-Newton step
 * with Armijo backtracking (sufficient decrease 1e-4, halving); a pair is
 * kept only when s.y > 0.  Stops early at a point where no decrease is found.
 * loss_history (host [iters], may be NULL) records the accepted losses (the
 * last one repeated after an early stop).  Resets the Adam state.  Blocks.
 */
int lpv_lbfgs(lpv_model* m, const float* u, const float* y, const float* p, int32_t n_traj, int32_t T, int32_t iters,
              double* loss_history, void* stream);

int lpv_fit(const float* u, const float* y, const float* p, int32_t n_traj, int32_t T, const lpv_config* cfg,
            lpv_model** out, double* best_loss, void* stream);

/* Free-run prediction y_out float32 [n_traj, T, n_y] in physical units. */
int lpv_predict(const lpv_model* m, const float* u, const float* p, int32_t n_traj, int32_t T, float* y_out,
                void* stream);

/*
 * Closed-loop batched simulation (Sections 5.1.1 and 5.4) of B independent
 * runs of T sampling periods: per period the PD torque of Eq. 28 is computed
 * from the sampled attitude and held, u = [F_x, F_y, tau + tau_c], p = [fill,
 * thetadot] clamped to [p_lo, p_hi] (the model holds only on the scheduling
 * range it was identified on), the surrogate gives the sloshing loads (its first three outputs:
 * F_x, F_y, T on the body), and the rigid body (Eq. 20) takes n_sub
 * kick-then-drift substeps under them.  Inputs (device, float64): F [B, T, 2],
 * tau [B, T], theta_ref [B, T], fill [B].  Output out float64 [B, T, 6]:
 * r_x r_y theta rdot_x rdot_y thetadot sampled before each period.
 */
int lpv_simulate(const lpv_model* m, int32_t B, const double* F, const double* tau, const double* theta_ref,
                 const double* fill, int32_t T, const lpv_body* body, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GB300_LPV_H */
