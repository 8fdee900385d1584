// lpv_api.cu -- host implementation of the C ABI declared in include/lpv.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lpv.h"
#include "lpv_common.cuh"
#include "lpv_launch.h"

namespace sph {
int set_last_error(int code, const char* msg);
}

using namespace lpv;

struct lpv_model {
    lpv_config cfg{};
    Dims d{};
    float *Wp = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    float* hist = nullptr;
    size_t hist_cap = 0;
    float* gpart = nullptr;
    double* loss_part = nullptr;
    size_t warp_cap = 0;
    double *d_loss = nullptr, *d_hist = nullptr;
    int hist_len = 0;
    double *stats_part = nullptr, *stats = nullptr, *gram_part = nullptr, *theta = nullptr, *rho = nullptr;
    int* status = nullptr;
    float *Wb = nullptr, *mb = nullptr, *vb = nullptr, *lr_scale = nullptr;  // last accepted Adam iterate
    double* acc_loss = nullptr;                                              // and its loss
    double* lb = nullptr;  // L-BFGS state (allocated on first use)
    int* lb_count = nullptr;
    int adam_t = 0;
};

namespace {

int err(int code, const std::string& msg) { return sph::set_last_error(code, msg.c_str()); }

#define LCK(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return err(SPH_E_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

// Adam restarts from the current weights: zero moments, the current weights as
// the last accepted iterate, full step size.
int reset_optimizer(lpv_model* M)
{
    for (float* p : {M->m, M->v, M->mb, M->vb}) LCK(cudaMemset(p, 0, kWN * sizeof(float)));
    LCK(cudaMemcpy(M->Wb, M->Wp, kWN * sizeof(float), cudaMemcpyDeviceToDevice));
    const float one = 1.f;
    const double inf = INFINITY;
    LCK(cudaMemcpy(M->lr_scale, &one, sizeof(float), cudaMemcpyHostToDevice));
    LCK(cudaMemcpy(M->acc_loss, &inf, sizeof(double), cudaMemcpyHostToDevice));
    M->adam_t = 0;
    return SPH_OK;
}

template <class T>
int grow(T** p, size_t* cap, size_t n)
{
    if (*cap >= n && *p) return SPH_OK;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc((void**)p, (n ? n : 1) * sizeof(T)) != cudaSuccess) return err(SPH_E_NOMEM, "lpv: cudaMalloc failed");
    *cap = n;
    return SPH_OK;
}

// Warps launched for n trajectories (whole blocks of 4 warps).
size_t launched_warps(int n_traj) { return (size_t)((warps_for(n_traj) + 3) / 4) * 4; }

int workspace(lpv_model* M, int n_traj, int T)
{
    const size_t warps = launched_warps(n_traj);
    if (M->warp_cap < warps) {
        cudaFree(M->gpart);
        cudaFree(M->loss_part);
        M->gpart = nullptr;
        M->loss_part = nullptr;
        M->warp_cap = 0;
        if (cudaMalloc(&M->gpart, warps * kWN * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&M->loss_part, warps * sizeof(double)) != cudaSuccess)
            return err(SPH_E_NOMEM, "lpv: cudaMalloc failed");
        M->warp_cap = warps;
    }
    return grow(&M->hist, &M->hist_cap, (size_t)n_traj * T * 16);
}

int check_data(const lpv_model* M, const float* u, const float* y, const float* p, int n_traj, int T)
{
    if (!M || !u || !y || n_traj < 1 || T < 1 || (M->d.np > 0 && !p)) return err(SPH_E_INVAL, "lpv: bad data arguments");
    return SPH_OK;
}

}  // namespace

extern "C" {

int lpv_create(const lpv_config* cfg, lpv_model** out)
{
    if (!cfg || !out) return err(SPH_E_INVAL, "lpv_create: NULL argument");
    const lpv_config& c = *cfg;
    if (c.n_x < 1 || c.n_u < 1 || c.n_y < 3 || c.n_p < 0 || c.n_p > 2 || c.n_x + c.n_u > 15 || c.n_x + c.n_y > 16 ||
        c.na < 1 || c.n_x != c.na * c.n_y || c.na * (c.n_y + c.n_u) + c.n_y > 32)
        return err(SPH_E_UNSUPPORTED,
                   "lpv_create: dimensions outside n_x + n_u <= 15, n_x + n_y <= 16, n_y >= 3, n_p <= 2, "
                   "n_x = na * n_y, na (n_y + n_u) + n_y <= 32");
    lpv_model* M = new lpv_model();
    M->cfg = c;
    Dims& d = M->d;
    d.nx = c.n_x;
    d.nu = c.n_u;
    d.ny = c.n_y;
    d.np = c.n_p;
    d.nkt = 1 + c.n_p;
    for (int i = 0; i < 16; ++i) d.inv_su[i] = d.sy[i] = d.inv_sy[i] = 1.f;
    for (int i = 0; i < 2; ++i) {
        d.pm[i] = 0.f;
        d.inv_ps[i] = 1.f;
        d.plo[i] = -INFINITY;
        d.phi[i] = INFINITY;
    }
    bool ok = cudaMalloc(&M->Wp, kWN * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&M->m, kWN * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&M->v, kWN * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&M->grad, kWN * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&M->d_loss, sizeof(double)) == cudaSuccess &&
              cudaMalloc(&M->stats_part, 256 * 64 * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&M->stats, 64 * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&M->gram_part, (size_t)gram_blocks() * 1024 * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&M->theta, 32 * 16 * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&M->rho, sizeof(double)) == cudaSuccess &&
              cudaMalloc(&M->status, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&M->Wb, kWN * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&M->mb, kWN * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&M->vb, kWN * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&M->lr_scale, sizeof(float)) == cudaSuccess &&
              cudaMalloc(&M->acc_loss, sizeof(double)) == cudaSuccess;
    if (ok) ok = cudaMemset(M->Wp, 0, kWN * sizeof(float)) == cudaSuccess && reset_optimizer(M) == SPH_OK;
    if (!ok) {
        lpv_destroy(M);
        return err(SPH_E_NOMEM, "lpv_create: allocation failed");
    }
    *out = M;
    return SPH_OK;
}

int lpv_destroy(lpv_model* M)
{
    if (!M) return SPH_OK;
    cudaDeviceSynchronize();
    for (void* p : {(void*)M->Wp, (void*)M->m, (void*)M->v, (void*)M->grad, (void*)M->hist, (void*)M->gpart,
                    (void*)M->loss_part, (void*)M->d_loss, (void*)M->d_hist, (void*)M->stats_part, (void*)M->stats,
                    (void*)M->gram_part, (void*)M->theta, (void*)M->rho, (void*)M->status, (void*)M->Wb,
                    (void*)M->mb, (void*)M->vb, (void*)M->lr_scale, (void*)M->acc_loss, (void*)M->lb,
                    (void*)M->lb_count})
        cudaFree(p);
    delete M;
    return SPH_OK;
}

int lpv_set_params(lpv_model* M, const float* W, const float* scales)
{
    if (!M) return err(SPH_E_INVAL, "lpv_set_params: NULL model");
    const Dims& d = M->d;
    if (W) {
        std::vector<float> Wp(kWN, 0.f);
        const int nr = d.nx + d.ny, nc = d.nx + d.nu;
        for (int kt = 0; kt < d.nkt; ++kt)
            for (int o = 0; o < nr; ++o)
                for (int f = 0; f < nc; ++f)
                    if (trainable(d, o, kt * kFB + f)) Wp[o * kFB * kMaxKT + kt * kFB + f] = W[(kt * nr + o) * nc + f];
        LCK(cudaMemcpy(M->Wp, Wp.data(), kWN * sizeof(float), cudaMemcpyHostToDevice));
        if (int rc = reset_optimizer(M)) return rc;
    }
    if (scales) {
        Dims& dm = M->d;
        const float* s = scales;
        for (int i = 0; i < dm.nu; ++i) dm.inv_su[i] = 1.f / s[i];
        for (int i = 0; i < dm.ny; ++i) {
            dm.sy[i] = s[dm.nu + i];
            dm.inv_sy[i] = 1.f / s[dm.nu + i];
        }
        for (int i = 0; i < dm.np; ++i) {
            dm.pm[i] = s[dm.nu + dm.ny + i];
            dm.inv_ps[i] = 1.f / s[dm.nu + dm.ny + dm.np + i];
            dm.plo[i] = s[dm.nu + dm.ny + 2 * dm.np + i];
            dm.phi[i] = s[dm.nu + dm.ny + 3 * dm.np + i];
        }
    }
    return SPH_OK;
}

int lpv_get_params(const lpv_model* M, float* W, float* scales)
{
    if (!M) return err(SPH_E_INVAL, "lpv_get_params: NULL model");
    const Dims& d = M->d;
    if (W) {
        std::vector<float> Wp(kWN);
        LCK(cudaMemcpy(Wp.data(), M->Wp, kWN * sizeof(float), cudaMemcpyDeviceToHost));
        const int nr = d.nx + d.ny, nc = d.nx + d.nu;
        for (int kt = 0; kt < d.nkt; ++kt)
            for (int o = 0; o < nr; ++o)
                for (int f = 0; f < nc; ++f) W[(kt * nr + o) * nc + f] = Wp[o * kFB * kMaxKT + kt * kFB + f];
    }
    if (scales) {
        for (int i = 0; i < d.nu; ++i) scales[i] = 1.f / d.inv_su[i];
        for (int i = 0; i < d.ny; ++i) scales[d.nu + i] = d.sy[i];
        for (int i = 0; i < d.np; ++i) {
            scales[d.nu + d.ny + i] = d.pm[i];
            scales[d.nu + d.ny + d.np + i] = 1.f / d.inv_ps[i];
            scales[d.nu + d.ny + 2 * d.np + i] = d.plo[i];
            scales[d.nu + d.ny + 3 * d.np + i] = d.phi[i];
        }
    }
    return SPH_OK;
}

int lpv_normalize(lpv_model* M, const float* u, const float* y, const float* p, int32_t n_traj, int32_t T,
                  void* stream)
{
    int rc = check_data(M, u, y, p, n_traj, T);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Dims& d = M->d;
    const long long n = (long long)n_traj * T;
    LCK(launch_stats(u, y, p, n, d.nu, d.ny, d.np, M->stats_part, M->stats, st));
    double s[64];
    LCK(cudaMemcpyAsync(s, M->stats, 64 * sizeof(double), cudaMemcpyDeviceToHost, st));
    LCK(cudaStreamSynchronize(st));
    auto safe = [](double v) { return (v > 1e-30 && std::isfinite(v)) ? v : 1.0; };
    for (int i = 0; i < d.nu; ++i) d.inv_su[i] = (float)(1.0 / safe(std::sqrt(s[i] / n)));
    for (int i = 0; i < d.ny; ++i) {
        const double sy = safe(std::sqrt(s[d.nu + i] / n));
        d.sy[i] = (float)sy;
        d.inv_sy[i] = (float)(1.0 / sy);
    }
    for (int i = 0; i < d.np; ++i) {
        const double mean = s[d.nu + d.ny + i] / n;
        const double var = s[d.nu + d.ny + d.np + i] / n - mean * mean;
        d.pm[i] = (float)mean;
        d.inv_ps[i] = (float)(1.0 / safe(std::sqrt(std::max(var, 0.0))));
        d.plo[i] = (float)s[32 + i];
        d.phi[i] = (float)s[32 + d.np + i];
    }
    return SPH_OK;
}

int lpv_init_ls(lpv_model* M, const float* u, const float* y, int32_t n_traj, int32_t T, double* theta_out,
                void* stream)
{
    if (!M || !u || !y || n_traj < 1 || T <= M->cfg.na) return err(SPH_E_INVAL, "lpv_init_ls: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int na = M->cfg.na;
    LCK(launch_gram(u, y, n_traj, T, M->d, na, M->gram_part, st));
    LCK(launch_ls_solve(M->gram_part, M->d, na, M->cfg.rho_max, M->theta, M->Wp, M->status, M->rho, st));
    int status = 0;
    LCK(cudaMemcpyAsync(&status, M->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    LCK(cudaStreamSynchronize(st));
    if (status) return err(SPH_E_DIVERGED, "lpv_init_ls: the normal equations are not positive definite");
    const int nreg = na * (M->d.ny + M->d.nu);
    if (theta_out) LCK(cudaMemcpy(theta_out, M->theta, (size_t)nreg * M->d.ny * sizeof(double), cudaMemcpyDeviceToHost));
    return reset_optimizer(M);
    return SPH_OK;
}

namespace {
// forward (loss + history), backward, reduction: grad and loss on the device
int loss_grad_device(lpv_model* M, const float* u, const float* y, const float* p, int n_traj, int T,
                     double* loss_hist, int it, cudaStream_t st)
{
    int rc = workspace(M, n_traj, T);
    if (rc) return rc;
    const double n = (double)n_traj * T;
    LCK(launch_forward(1, M->Wp, M->d, u, p, y, n_traj, T, nullptr, M->hist, M->loss_part, (float)(2.0 / n), st));
    LCK(launch_backward(M->Wp, M->d, u, p, n_traj, T, M->hist, M->gpart, st));
    LCK(launch_reduce(M->gpart, (int)launched_warps(n_traj), M->loss_part, M->Wp, M->d, M->cfg.sigma2, n, M->grad,
                      M->d_loss, loss_hist, it, st));
    return SPH_OK;
}
}  // namespace

int lpv_loss_grad(lpv_model* M, const float* u, const float* y, const float* p, int32_t n_traj, int32_t T,
                  double* loss, float* grad, void* stream)
{
    int rc = check_data(M, u, y, p, n_traj, T);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    rc = loss_grad_device(M, u, y, p, n_traj, T, nullptr, 0, st);
    if (rc) return rc;
    LCK(cudaStreamSynchronize(st));
    if (loss) LCK(cudaMemcpy(loss, M->d_loss, sizeof(double), cudaMemcpyDeviceToHost));
    if (grad) {
        std::vector<float> g(kWN);
        LCK(cudaMemcpy(g.data(), M->grad, kWN * sizeof(float), cudaMemcpyDeviceToHost));
        const Dims& d = M->d;
        const int nr = d.nx + d.ny, nc = d.nx + d.nu;
        for (int kt = 0; kt < d.nkt; ++kt)
            for (int o = 0; o < nr; ++o)
                for (int f = 0; f < nc; ++f) grad[(kt * nr + o) * nc + f] = g[o * kFB * kMaxKT + kt * kFB + f];
    }
    return SPH_OK;
}

int lpv_train(lpv_model* M, const float* u, const float* y, const float* p, int32_t n_traj, int32_t T, int32_t iters,
              double* loss_history, void* stream)
{
    int rc = check_data(M, u, y, p, n_traj, T);
    if (rc) return rc;
    if (iters < 0) return err(SPH_E_INVAL, "lpv_train: negative iteration count");
    cudaStream_t st = (cudaStream_t)stream;
    if (M->hist_len < iters) {
        cudaFree(M->d_hist);
        M->d_hist = nullptr;
        M->hist_len = 0;
        if (cudaMalloc(&M->d_hist, (size_t)(iters ? iters : 1) * sizeof(double)) != cudaSuccess)
            return err(SPH_E_NOMEM, "lpv_train: cudaMalloc failed");
        M->hist_len = iters;
    }
    const lpv_config& c = M->cfg;
    for (int it = 0; it < iters; ++it) {
        rc = loss_grad_device(M, u, y, p, n_traj, T, M->d_hist, it, st);
        if (rc) return rc;
        const int t = ++M->adam_t;
        const float c1 = (float)(1.0 / (1.0 - std::pow(c.beta1, t))), c2 = (float)(1.0 / (1.0 - std::pow(c.beta2, t)));
        LCK(launch_adam(M->Wp, M->m, M->v, M->Wb, M->mb, M->vb, M->lr_scale, M->acc_loss, M->grad, M->d_loss, M->d, (float)c.lr, (float)c.beta1, (float)c.beta2,
                        (float)c.adam_eps, c1, c2, st));
    }
    LCK(cudaStreamSynchronize(st));
    if (loss_history && iters)
        LCK(cudaMemcpy(loss_history, M->d_hist, (size_t)iters * sizeof(double), cudaMemcpyDeviceToHost));
    return SPH_OK;
}

int lpv_lbfgs(lpv_model* M, const float* u, const float* y, const float* p, int32_t n_traj, int32_t T, int32_t iters,
              double* loss_history, void* stream)
{
    int rc = check_data(M, u, y, p, n_traj, T);
    if (rc) return rc;
    if (iters < 0) return err(SPH_E_INVAL, "lpv_lbfgs: negative iteration count");
    cudaStream_t st = (cudaStream_t)stream;
    if (!M->lb) {
        const size_t n = (size_t)kWN * (3 + 2 * kLbfgsM) + kLbfgsM + 2;
        if (cudaMalloc(&M->lb, n * sizeof(double)) != cudaSuccess || cudaMalloc(&M->lb_count, 2 * sizeof(int)) != cudaSuccess)
            return err(SPH_E_NOMEM, "lpv_lbfgs: cudaMalloc failed");
    }
    LbfgsDev L;
    L.W = M->lb;
    L.g = L.W + kWN;
    L.d = L.g + kWN;
    L.S = L.d + kWN;
    L.Y = L.S + (size_t)kLbfgsM * kWN;
    L.rho = L.Y + (size_t)kLbfgsM * kWN;
    L.gd = L.rho + kLbfgsM;
    L.count = M->lb_count;
    auto loss_now = [&](double* out) -> int {
        int r = loss_grad_device(M, u, y, p, n_traj, T, nullptr, 0, st);
        if (r) return r;
        LCK(cudaMemcpyAsync(out, M->d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        LCK(cudaStreamSynchronize(st));
        return SPH_OK;
    };
    double f = 0.0;
    if ((rc = loss_now(&f))) return rc;
    if (!std::isfinite(f)) return err(SPH_E_DIVERGED, "lpv_lbfgs: the loss at the start is not finite");
    LCK(launch_lbfgs_init(M->Wp, M->grad, M->d, L, st));
    constexpr double kArmijo = 1e-4;
    int it = 0;
    for (; it < iters; ++it) {
        LCK(launch_lbfgs_dir(L, st));
        double gd[2];
        int cnt[2];
        LCK(cudaMemcpyAsync(gd, L.gd, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        LCK(cudaMemcpyAsync(cnt, L.count, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        LCK(cudaStreamSynchronize(st));
        if (!(gd[0] < 0.0)) break;  // stationary point
        // unit quasi-Newton step; after a reset, a step of 0.01 in the weights
        double step = cnt[0] > 0 ? 1.0 : std::min(1.0, 0.01 / std::sqrt(gd[1]));
        bool ok = false;
        double fn = 0.0;
        for (int tries = 0; tries < 40; ++tries) {
            LCK(launch_lbfgs_try(M->Wp, M->d, L, step, st));
            if ((rc = loss_now(&fn))) return rc;
            if (std::isfinite(fn) && fn <= f + kArmijo * step * gd[0]) {
                ok = true;
                break;
            }
            step *= 0.5;
        }
        if (!ok) {  // no decrease along d: keep the last accepted point
            LCK(launch_lbfgs_try(M->Wp, M->d, L, 0.0, st));
            break;
        }
        LCK(launch_lbfgs_accept(M->grad, M->d, L, step, st));
        f = fn;
        if (loss_history) loss_history[it] = f;
    }
    if (loss_history)
        for (int k = it; k < iters; ++k) loss_history[k] = f;
    LCK(cudaStreamSynchronize(st));
    return reset_optimizer(M);
}

int lpv_fit(const float* u, const float* y, const float* p, int32_t n_traj, int32_t T, const lpv_config* cfg,
            lpv_model** out, double* best_loss, void* stream)
{
    if (!out) return err(SPH_E_INVAL, "lpv_fit: NULL output");
    lpv_model* M = nullptr;
    int rc = lpv_create(cfg, &M);
    if (rc) return rc;
    const int restarts = cfg->restarts > 0 ? cfg->restarts : 1;
    std::vector<lpv_model*> R(restarts, nullptr);
    std::vector<cudaStream_t> S(restarts, nullptr);
    auto bail = [&](int code) {
        std::string msg = sph_last_error();
        for (int r = 0; r < restarts; ++r) {
            if (S[r]) cudaStreamDestroy(S[r]);
            lpv_destroy(R[r]);
        }
        lpv_destroy(M);
        return err(code, msg);
    };
    if ((rc = lpv_normalize(M, u, y, p, n_traj, T, stream))) return bail(rc);
    if ((rc = lpv_init_ls(M, u, y, n_traj, T, nullptr, stream))) return bail(rc);
    const Dims& d = M->d;
    const int nr = d.nx + d.ny, nc = d.nx + d.nu, nw = d.nkt * nr * nc;
    std::vector<float> W0(nw);
    if ((rc = lpv_get_params(M, W0.data(), nullptr))) return bail(rc);
    // The restarts are independent: each gets a model of its own, a stream of
    // its own and a host thread that drives its Adam and L-BFGS loops, so
    // that their launches (a few dozen warps each) fill the GPU together and
    // the line searches' host round trips overlap.  Every restart computes
    // exactly what it would alone, so the best one is the same as in a
    // sequential loop.
    std::vector<std::vector<float>> Wr(restarts, W0);
    for (int r = 0; r < restarts; ++r) {
        // M_0 from the least-squares fit; the B and C blocks of M_i ~ N(0,
        // init_scale^2) (Section 5.3.2), their A blocks 0 so that A(p) = A_0
        // keeps the stable spectrum of the start for every p
        std::mt19937_64 gen(cfg->seed + 1000003ull * (uint64_t)r);
        std::normal_distribution<double> nd(0.0, cfg->init_scale);
        for (int i = nr * nc; i < nw; ++i) {
            const int o = (i / nc) % nr, f = i % nc;
            const double draw = nd(gen);
            Wr[r][i] = (o < d.nx && f < d.nx) ? 0.f : (float)draw;
        }
        if ((rc = lpv_create(cfg, &R[r]))) return bail(rc);
        R[r]->d = M->d;  // the normalisation of the data, exactly
        if ((rc = lpv_set_params(R[r], Wr[r].data(), nullptr))) return bail(rc);
        if (cudaStreamCreateWithFlags(&S[r], cudaStreamNonBlocking) != cudaSuccess) {
            S[r] = nullptr;
            return bail(err(SPH_E_CUDA, "lpv_fit: cudaStreamCreate failed"));
        }
    }
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)  // the data are complete before other streams read them
        return bail(err(SPH_E_CUDA, "lpv_fit: cudaStreamSynchronize failed"));
    std::vector<int> codes(restarts, SPH_OK);
    std::vector<double> loss(restarts, INFINITY);
    std::vector<std::string> msgs(restarts);
    {
        std::vector<std::thread> th;
        th.reserve(restarts);
        for (int r = 0; r < restarts; ++r)
            th.emplace_back([&, r] {
                lpv_model* m = R[r];
                void* st = (void*)S[r];
                int c = lpv_train(m, u, y, p, n_traj, T, cfg->adam_iters, nullptr, st);
                if (!c && cfg->lbfgs_iters > 0) c = lpv_lbfgs(m, u, y, p, n_traj, T, cfg->lbfgs_iters, nullptr, st);
                double L = INFINITY;
                if (!c) c = lpv_loss_grad(m, u, y, p, n_traj, T, &L, nullptr, st);
                codes[r] = c;
                loss[r] = c ? INFINITY : L;
                if (c) msgs[r] = sph_last_error();
            });
        for (auto& t : th) t.join();
    }
    int best_r = -1;
    for (int r = 0; r < restarts; ++r) {
        if (codes[r] == SPH_E_DIVERGED) continue;  // this restart ended with a non-finite loss
        if (codes[r]) {
            err(codes[r], msgs[r]);
            return bail(codes[r]);
        }
        if (!std::isfinite(loss[r])) continue;
        if (best_r < 0 || loss[r] < loss[best_r]) best_r = r;  // first of equal losses, as in order
    }
    if (best_r < 0) {
        err(SPH_E_DIVERGED, "lpv_fit: no restart ended with a finite training loss");
        return bail(SPH_E_DIVERGED);
    }
    std::vector<float> Wbest(nw);
    if ((rc = lpv_get_params(R[best_r], Wbest.data(), nullptr))) return bail(rc);
    for (int r = 0; r < restarts; ++r) {
        cudaStreamDestroy(S[r]);
        lpv_destroy(R[r]);
    }
    if ((rc = lpv_set_params(M, Wbest.data(), nullptr))) {
        std::string msg = sph_last_error();
        lpv_destroy(M);
        return err(rc, msg);
    }
    if (best_loss) *best_loss = loss[best_r];
    *out = M;
    return SPH_OK;
}

int lpv_predict(const lpv_model* M, const float* u, const float* p, int32_t n_traj, int32_t T, float* y_out,
                void* stream)
{
    if (!M || !u || !y_out || n_traj < 1 || T < 1 || (M->d.np > 0 && !p)) return err(SPH_E_INVAL, "lpv_predict: bad arguments");
    LCK(launch_forward(0, M->Wp, M->d, u, p, nullptr, n_traj, T, y_out, nullptr, nullptr, 0.f, (cudaStream_t)stream));
    return SPH_OK;
}

int lpv_simulate(const lpv_model* M, int32_t B, const double* F, const double* tau, const double* theta_ref,
                 const double* fill, int32_t T, const lpv_body* body, double* out, void* stream)
{
    if (!M || !F || !tau || !theta_ref || !fill || !body || !out || B < 1 || T < 1 || body->n_sub < 1 ||
        !(body->m > 0) || !(body->J > 0) || !(body->Ts > 0))
        return err(SPH_E_INVAL, "lpv_simulate: bad arguments");
    if (M->d.ny < 3) return err(SPH_E_UNSUPPORTED, "lpv_simulate: the surrogate needs outputs F_x, F_y, T");
    const double Jc = body->ctrl_J > 0 ? body->ctrl_J : body->J;
    BodyParHost h;
    h.inv_m = (float)(1.0 / body->m);
    h.inv_J = (float)(1.0 / body->J);
    h.dt = (float)(body->Ts / body->n_sub);
    h.n = (float)body->n_sub;
    h.n_half = (float)(0.5 * body->n_sub * (body->n_sub + 1));
    h.kp = (float)(Jc * body->ctrl_omega * body->ctrl_omega);
    h.kd = (float)(2.0 * body->ctrl_xi * Jc * body->ctrl_omega);
    LCK(launch_closed_loop(M->Wp, M->d, B, T, F, tau, theta_ref, fill, h, out, (cudaStream_t)stream));
    return SPH_OK;
}

}  // extern "C"
