/*
 * slpv.h -- C ABI of the self-scheduled LPV surrogate of the paper's
 * identification study (Section 4, Eqs. 24-27; Section 5.3.2), with its
 * integrator augmentation and its use in closed loop (Section 5.1.1).
 *
 * Model (n_u = n_y = 3, n_p = 1, feedthrough D = 0, x_0 = 0):
 *   z_k = [x_k; u_k / s_u],   p_k = eta(z_k),
 *   eta(z) = w3 . tanh(W2 tanh(W1 z + b1) + b2) + b3   (two hidden tanh layers of 4),
 *   [x_{k+1}; y_k] = (M_0 + p_k M_1) z_k,   M_i = [[A_i, B_i], [C_i, D_i = 0]],
 *   velocities = y_k * s_y  (the model maps u = [F_x, F_y, tau] to
 *   [rdot_x, rdot_y, thetadot] at the sampling period T_s),
 *   positions  e_{k+1} = e_k + T_s * velocities_k, e_0 = 0 (augmentation).
 * Parameters theta (float32, n_theta = 2 (nx+3)^2 + 4 (nx+3) + 29 values) in
 * the order M_0, M_1 (row-major (nx+3) x (nx+3), the D blocks stored and held
 * at zero), W1 (4 x (nx+3)), b1 (4), W2 (4 x 4), b2 (4), w3 (4), b3 (1).
 * scales: float32 [6] = s_u (3), s_y (3): the data are divided by them.
 *
 * Conventions: every function returns 0 (SPH_OK) or a negative SPH_E_* code
 * (sph.h); sph_last_error() gives the text.  Array arguments are DEVICE
 * pointers unless marked host, row-major and contiguous, owned by the
 * caller; calls are asynchronous on `stream` unless stated.
 */
#ifndef SLPV_H
#define SLPV_H

#include <stdint.h>

#include "sph.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slpv_config {
    int32_t nx;                 /* state dimension: 2, 4 (the paper's), 6 or 8  */
    float sigma2;               /* l2 weight of Eq. 27 on all of theta          */
} slpv_config;

typedef struct slpv_model slpv_model;

/* Number of values in theta for state dimension nx (host). */
int slpv_n_params(int32_t nx, int32_t* n_theta);

/* Creates a model with theta = 0 and unit scales.  Blocks. */
int slpv_create(const slpv_config* cfg, slpv_model** out);
int slpv_destroy(slpv_model* m);

/* host float32 theta [n_theta] and scales [6]; set zeroes the D blocks. */
int slpv_set_params(slpv_model* m, const float* theta, const float* scales);
int slpv_get_params(const slpv_model* m, float* theta, float* scales);

/*
 * Data scales: s_u, s_y = root mean square of each input and output channel
 * over u, y [n_traj, T, 3] (float32); stored in the model.  Blocks.
 * SPH_E_INVAL: a channel that is identically zero.
 */
int slpv_normalize(slpv_model* m, const float* u, const float* y, int32_t n_traj, int32_t T, void* stream);

/*
 * Least-squares LTI start of M_0, in place of the ssest fit of Section
 * 5.3.2: the first-order ARX model y_{k+1} = A1 y_k + B1 u_k fitted in FP64
 * by the normal equations (ridge 1e-12 tr(G)/6) over all samples of u, y
 * [n_traj, T, 3] divided by the stored scales, realised with the velocities
 * as the first three states: A_0 = [[A1, 0], [0, 0]], B_0 = [[B1], [0]],
 * C_0 = [I, 0]; M_1 and the network set to zero.  Needs nx >= 3.  Blocks.
 * SPH_E_DIVERGED: singular normal equations.
 */
int slpv_init_ls(slpv_model* m, const float* u, const float* y, int32_t n_traj, int32_t T, void* stream);

/*
 * Free-run loss of Eq. 27 (x_0 = 0, so the sigma_x term vanishes):
 *   J = mean over the n_traj * T samples of ||y_k / s_y - y_hat_k||^2 + sigma2/2 ||theta||^2
 * and its gradient by backpropagation through time, through the state
 * recursion and the scheduling map.  loss_out: device double [1]; grad_out:
 * device float [n_theta] or NULL (loss only).  stage selects the entries
 * that train (the others get a zero gradient): 0 all, 1 M_0 only (the LTI
 * stage), 2 M_1 and the network only (M_0 held).  SPH_E_INVAL for another
 * value.  Sums are taken in a fixed order: results are deterministic.
 */
int slpv_loss_grad(slpv_model* m, const float* u, const float* y, int32_t n_traj, int32_t T, int32_t stage,
                   double* loss_out, float* grad_out, void* stream);

/*
 * iters Adam steps (Kingma and Ba; b1 0.9, b2 0.999, eps 1e-8, step lr) on
 * theta from its current value; loss_hist: device double [iters] or NULL,
 * the loss at each iterate.  A step whose loss is not finite or exceeds ten
 * times the last accepted loss is undone and retried at half the step.
 * stage as in slpv_loss_grad.
 */
int slpv_train(slpv_model* m, const float* u, const float* y, int32_t n_traj, int32_t T, int32_t iters, float lr,
               int32_t stage, double* loss_hist, void* stream);

/*
 * L-BFGS refinement after Adam (Section 5.3.2): up to iters iterations from
 * the current theta; the two-loop recursion over the last 10 curvature pairs
 * runs in FP64 on the device, the step is 1 (0.01 / |g| after a reset)
 * halved until Armijo's condition (1e-4) holds.  Stops early at a point
 * without descent; stage as in slpv_loss_grad.  loss_hist: HOST double
 * [iters] or NULL (the accepted loss per iteration, the last one repeated
 * after a stop).  Blocks.
 * SPH_E_DIVERGED: the loss at the start is not finite.
 */
int slpv_lbfgs(slpv_model* m, const float* u, const float* y, int32_t n_traj, int32_t T, int32_t iters,
               int32_t stage, double* loss_hist, void* stream);

/*
 * Free run of the augmented surrogate from rest over u [n_traj, T, 3]
 * (physical units): vel_out [n_traj, T, 3] = velocities (physical), pos_out
 * [n_traj, T, 3] = positions e_k (before step k), either may be NULL.
 */
int slpv_predict(const slpv_model* m, const float* u, int32_t n_traj, int32_t T, double Ts, float* vel_out,
                 float* pos_out, void* stream);

/*
 * B closed-loop runs of the augmented surrogate under the PD law of Eq. 28
 * (zero-order hold over T_s): at sample k the controller reads theta_k
 * (augmented state) and thetadot_k = C(p) x_k with p = eta(x_k, u_{k-1}),
 * the input held when the sample is taken (u_{-1} = 0); u_k = [F_k, tau_k +
 * tau_c,k] is applied and the model steps with p_k = eta(x_k, u_k).
 * F [B, T, 2], tau [B, T], theta_ref [B, T] (float64); out [B, T, 6] float32
 * rows (r_x, r_y, theta, rdot_x, rdot_y, thetadot), positions before step k
 * and the velocities of step k.  J, omega, xi as in sph_ctrl (J > 0).
 */
int slpv_simulate(const slpv_model* m, int32_t B, int32_t T, const double* F, const double* tau,
                  const double* theta_ref, double Ts, double J, double omega, double xi, float* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SLPV_H */
