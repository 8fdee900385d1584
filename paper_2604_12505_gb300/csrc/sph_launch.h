// sph_launch.h -- host-side launchers of the simulator kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include "sph_common.cuh"

namespace sph {

void tile_dims(int code, int* tx, int* ty);
// pdl: launch with programmatic stream serialization (the kernels wait on
// their predecessor with griddepcontrol before reading its results).
// tan: the forward-mode tangent variants (tile codes 1..4 only).
cudaError_t launch_phase(const SimDev& S, const EvalOut& E, int eval, int tile_code, int n_tiles, int phase,
                         cudaStream_t st, bool pdl, bool tan = false);
cudaError_t launch_step(const SimDev& S, const EvalOut& E, int eval, int tile_code, int n_tiles, cudaStream_t st,
                        bool pdl, bool tan = false);
cudaError_t launch_bin_flat(const SimDev& S, const float* xv, const int* part_tank, int n, int buf, cudaStream_t st);
cudaError_t launch_set_body(const SimDev& S, const double* body, int buf, cudaStream_t st);
cudaError_t launch_get_state(const SimDev& S, float* xv, double* body, int n_cells_total, int buf, cudaStream_t st);
// Tangent state: with txv_out == NULL sets the tangent from txv_in / tb_in
// (NULL: zero); otherwise reads it into txv_out / tb_out.
cudaError_t launch_tangent_state(const SimDev& S, const float* txv_in, float* txv_out, const double* tb_in,
                                 double* tb_out, int n_cells_total, int buf, cudaStream_t st);
cudaError_t launch_set_run(RunDev* run, const RunDev& desc, cudaStream_t st);

}  // namespace sph
