// fold.h -- host launcher of the register-resident heat Diamond kernel (fold.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "schemes.cuh"

namespace sw {

// True when k_heat_fold has an instantiation for this precision and base width
// (W = 32 K, K in {4, 8, 16, 32}).
bool fold_supported(int precision, int W);

// One complete Diamond phase (parity p: 1 seam centred, 2 tile centred) of a
// periodic heat problem with M tiles; flanks in the k_swept_phase layout with
// S structures per buffer. `warps` warps share the M diamonds in contiguous chains.
cudaError_t launch_fold(int precision, int W, int p, int64_t M, int64_t S, const void *flank_in,
                        void *flank_out, const HeatParams &prm, int64_t warps, cudaStream_t st);

// Warps per SM the launcher aims for at this precision / width (register bound).
int fold_warps_per_sm(int precision, int W);

}  // namespace sw
