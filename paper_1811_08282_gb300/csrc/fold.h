// fold.h -- host launchers of the register-resident phase kernels: heat (fold.cu)
// and Euler (fold_euler.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "euler.cuh"
#include "heat.cuh"

namespace sw {

// True when k_heat_fold has an instantiation for this precision and base width
// (W = 32 K, K in {2, 4, 8, 16, 32}).
bool fold_supported(int precision, int W);

// One phase of a periodic heat problem with M tiles (p: 0 Up Triangle, 1 seam
// centred, 2 tile centred), `lower` / `upper` levels in its two halves, storing
// the Down Triangle's row when write_lower is set (write_upper must be 0).
// Flanks in the k_swept_phase layout with S structures per buffer; `warps` warps
// share the M structures in contiguous chains.
struct FoldPhase {
    int p;
    int64_t n, M, S;
    int64_t nstruct;  // structures 0 .. nstruct-1 of the phase run here (M, or fewer in a hybrid run)
    int lower, upper, write_lower, write_upper;
    const void *flank_in;
    void *flank_out;
    void *state;
};
cudaError_t launch_fold(int precision, int W, const FoldPhase &ph, const HeatParams &prm, int64_t warps,
                        cudaStream_t st);

// Warps per SM the launcher aims for at this precision / width (register bound).
int fold_warps_per_sm(int precision, int W);

// Euler: true when k_euler_fold has an instantiation (FP64: W = 128; FP32 and
// FP32 hi/lo: W = 128, 256).
bool euler_fold_supported(int precision, int W);

// One phase of an Euler problem, periodic or transmissive, whose upper half is
// complete (or absent): nstruct structures (transmissive seam-centred phases have
// M + 1, the two at the domain ends half outside it). Flanks in the k_swept_phase
// layout with the fields of the Euler policies.
struct EulerFoldPhase {
    int p, periodic;
    int64_t n, M, nstruct, S;
    int lower, upper, write_lower;
    const void *flank_in;
    void *flank_out;
    void *state;
};
cudaError_t launch_euler_fold(int precision, int W, const EulerFoldPhase &ph, const EulerParams &prm, int64_t warps,
                              cudaStream_t st);
int euler_fold_warps_per_sm(int precision, int W);

}  // namespace sw
