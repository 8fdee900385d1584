// sph_launch.h -- host-side launchers of the simulator kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include "sph_common.cuh"

namespace sph {

void tile_dims(int code, int* tx, int* ty);
// Bytes of the per-tile staging records for the tile counts of every shape
// (n_tiles indexed by tile code 1..SPH_TILE_COUNT).
size_t stage_record_bytes(const int* n_tiles);
// pdl: launch with programmatic stream serialization (the kernels wait on
// their predecessor with griddepcontrol before reading its results).
// tan: the forward-mode tangent variants (tile codes 1..4 only).
// Phases: 0 density pass, 1 force pass, 2 body update (the tangent variant's
// force pass updates the body itself, its phase 2 launches nothing).
// chained: this step directly follows a step of the same launch sequence
// (its density pass is the programmatic dependent of the previous step's
// body update), so that pass may stage the tile and sum the fluid part of
// Eq. 14 before its grid dependency: everything it reads there was written
// by the previous force pass, which completed before the body update passed
// its own dependency.
cudaError_t launch_phase(const SimDev& S, const EvalOut& E, int eval, int tile_code, int n_tiles, int phase,
                         cudaStream_t st, bool pdl, bool tan = false, bool chained = false);
cudaError_t launch_step(const SimDev& S, const EvalOut& E, int eval, int tile_code, int n_tiles, cudaStream_t st,
                        bool pdl, bool tan = false, bool chained = false);
// State transfer: xv [N, 4] the hi parts of the particle state, lo [N, 4] its
// low parts (NULL: zero on binning, not read back on gathering).
cudaError_t launch_bin_flat(const SimDev& S, const float* xv, const float* lo, const int* part_tank, int n, int buf,
                            cudaStream_t st);
cudaError_t launch_set_body(const SimDev& S, const double* body, int buf, cudaStream_t st);
cudaError_t launch_get_state(const SimDev& S, float* xv, float* lo, double* body, int n_cells_total, int buf,
                             cudaStream_t st);
// Tangent state: with txv_out == NULL sets the tangent from txv_in / tb_in
// (NULL: zero); otherwise reads it into txv_out / tb_out.
cudaError_t launch_tangent_state(const SimDev& S, const float* txv_in, float* txv_out, const double* tb_in,
                                 double* tb_out, int n_cells_total, int buf, cudaStream_t st);
cudaError_t launch_set_run(RunDev* run, const RunDev& desc, cudaStream_t st);

// Reverse-mode step (sph_adjoint.cu).  Adjoint arrays are indexed by particle
// index (the order of sph_get_state); body adjoints are (r_x, r_y, theta,
// rdot_x, rdot_y, thetadot).
struct AdjDev {
    const float4* in;        // [N] adjoint of (x, v) after the step
    float4* out;             // [N] adjoint of (x, v) before the step
    float* rhobar;           // [N] density adjoint (work)
    double* bbar;            // [B * 6] body adjoint: after the step on entry, before it on exit
    double* bbar_part;       // [B * 6] work: the integration part
    float* fbar;             // [B * 8] work: F_b, T_b and centre-of-mass adjoints of the step
    float* part;             // [2][max_tiles][12] work: per-tile body partials
    int max_tiles;
    const double* ybar;      // [B, n_samples, SPH_NY] sample adjoints (NULL: 0)
    long long ybar_stride;   // doubles between tanks
    double* ubar;            // [B, K, 3] input adjoints (NULL: not written)
    long long ubar_stride;
    int k;                   // step index within the call
    int row;                 // sample row of this step, -1: not sampled
};
int adjoint_tile_code();
cudaError_t launch_adjoint_step(const SimDev& S, const AdjDev& A, int n_tiles, cudaStream_t st);
cudaError_t launch_set_step(RunDev* run, long long step, cudaStream_t st);

}  // namespace sph
