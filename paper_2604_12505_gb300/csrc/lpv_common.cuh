// lpv_common.cuh -- device-side layout of the LPV surrogate (internal).
//
// Weights live in one padded FP32 matrix Wp[16][48]: row o is an output
// (o < n_x: next state, n_x <= o < n_x + n_y: y), column kt*16 + f is the
// feature f of scheduling block kt (f < n_x: state, n_x <= f < n_x + n_u:
// input, rest zero; block 0 is M_0, block i is M_i multiplied by p_i).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace lpv {

constexpr int kO = 16;      // padded outputs
constexpr int kFB = 16;     // padded features per scheduling block
constexpr int kMaxKT = 3;   // 1 + max n_p
constexpr int kWN = kO * kFB * kMaxKT;  // 768 padded weights

struct Dims {
    int nx, nu, ny, np, nkt;  // nkt = 1 + np
    float inv_su[16];          // 1 / s_u
    float sy[16], inv_sy[16];  // s_y and 1 / s_y
    float pm[2], inv_ps[2];    // scheduling mean, 1 / std
    float plo[2], phi[2];      // scheduling range of the data (closed-loop clamp)
};

// 1 where a padded weight is trainable (not padding, not a D block).
__host__ __device__ __forceinline__ bool trainable(const Dims& d, int o, int col)
{
    const int kt = col / kFB, f = col % kFB;
    if (kt >= d.nkt || o >= d.nx + d.ny || f >= d.nx + d.nu) return false;
    if (o >= d.nx && f >= d.nx) return false;  // feedthrough D = 0
    return true;
}

}  // namespace lpv
