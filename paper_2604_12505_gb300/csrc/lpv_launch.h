// lpv_launch.h -- host-side launchers of the LPV kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include "lpv_common.cuh"

namespace lpv {

struct BodyParHost {
    float inv_m, inv_J, dt, n, n_half, kp, kd;
};

// Warps of 16 trajectories needed for n trajectories.
inline int warps_for(int n) { return (n + 15) / 16; }

// mode 0: prediction into y_out; mode 1: loss partials per warp and BPTT history.
cudaError_t launch_forward(int mode, const float* Wp, const Dims& d, const float* u, const float* p, const float* y,
                           int n_traj, int T, float* y_out, float* hist, double* loss_part, float grad_scale,
                           cudaStream_t st);
cudaError_t launch_backward(const float* Wp, const Dims& d, const float* u, const float* p, int n_traj, int T,
                            const float* hist, float* gpart, cudaStream_t st);
cudaError_t launch_closed_loop(const float* Wp, const Dims& d, int B, int T, const double* F, const double* tau,
                               const double* ref, const double* fill, const BodyParHost& bp, double* out,
                               cudaStream_t st);
// grad = sum of the warp partials (FP64, fixed order) + sigma2 W, masked to the
// trainable entries; *loss = sum loss_part / n_samples + sigma2 / 2 ||W||^2;
// if loss_hist is not NULL the loss is also stored at loss_hist[it].
cudaError_t launch_reduce(const float* gpart, int n_warps, const double* loss_part, const float* Wp, const Dims& d,
                          double sigma2, double n_samples, float* grad, double* loss, double* loss_hist, int it,
                          cudaStream_t st);
cudaError_t launch_adam(float* Wp, float* m, float* v, float* Wb, float* mb, float* vb, float* lr_scale,
                        double* acc_loss, const float* grad, const double* loss, const Dims& d, float lr, float b1,
                        float b2, float eps, float c1, float c2, cudaStream_t st);
// Per channel over n rows: sum u^2 (n_u), sum y^2 (n_y), sum p and sum p^2 (n_p),
// written to stats[n_u + n_y + 2 n_p] (FP64).  part: scratch of 256 x 32 doubles.
cudaError_t launch_stats(const float* u, const float* y, const float* p, long long n, int nu, int ny, int np,
                         double* part, double* stats, cudaStream_t st);
// FP64 Gram matrix of the extended ARX rows [phi_k, y_k] (normalised data):
// part[n_blocks][n_ext * n_ext]; then the solve writes the coefficients
// theta[n_reg][n_y], the observer-canonical M_0 into Wp and zero M_i (i >= 1).
// status[0] = 0 on success, 1 if the normal matrix is not positive definite.
int gram_blocks();
cudaError_t launch_gram(const float* u, const float* y, int n_traj, int T, const Dims& d, int na, double* part,
                        cudaStream_t st);
// rho_max > 0: the roots of the start are scaled into |z| <= rho_max; rho_out
// (device, may be NULL) receives the spectral radius before scaling.
cudaError_t launch_ls_solve(const double* part, const Dims& d, int na, double rho_max, double* theta, float* Wp,
                            int* status, double* rho_out, cudaStream_t st);

// L-BFGS state (device): FP64 master weights, gradient, search direction,
// kLbfgsM curvature pairs (S, Y, rho), count[0] = stored pairs, count[1] =
// next slot, gd[0] = g.d, gd[1] = g.g.
constexpr int kLbfgsM = 10;
struct LbfgsDev {
    double *W, *g, *d, *S, *Y, *rho, *gd;
    int* count;
};
cudaError_t launch_lbfgs_init(const float* Wp, const float* grad, const Dims& d, const LbfgsDev& L, cudaStream_t st);
cudaError_t launch_lbfgs_dir(const LbfgsDev& L, cudaStream_t st);
cudaError_t launch_lbfgs_try(float* Wp, const Dims& d, const LbfgsDev& L, double step, cudaStream_t st);
cudaError_t launch_lbfgs_accept(const float* grad, const Dims& d, const LbfgsDev& L, double step, cudaStream_t st);

}  // namespace lpv
