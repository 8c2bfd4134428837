// fold.cu -- instantiations and launcher of the register-resident heat Diamond kernel.
#include "fold.h"
#include "fold_heat.cuh"

#include "../../include/swept.h"

namespace sw {

bool fold_supported(int precision, int W) {
    if (precision < SW_FP64 || precision > SW_FP32_COMP) return false;
    return W == 64 || W == 128 || W == 256 || W == 512 || W == 1024;
}

// Measured on GB300 at N = 2^24 (diamond phases, 4-warp CTAs; multiples of 4 keep
// the SMs evenly loaded): FP32 peaks at 24 warps/SM up to W = 512, 12 at W = 1024;
// FP32 hi/lo at 24 (W = 128), 16 (256), 12 (512). FP64 with half the cells on the
// integer pipes wants more warps in flight: 32 at W = 128, 16 at W = 256; the
// FP64-only widths (512, 1024) peak at 8.
int fold_warps_per_sm(int precision, int W) {
    if (precision == SW_FP32) return W >= 1024 ? 12 : 24;
    if (precision == SW_FP32_COMP) return W <= 128 ? 24 : (W == 256 ? 16 : (W == 512 ? 12 : 8));
    return W <= 128 ? 32 : (W == 256 ? 16 : 8);
}

template <int K, class C>
static cudaError_t go(const FoldPhase &ph, const HeatParams &prm, int64_t warps, cudaStream_t st) {
    using T = typename C::T;
    FoldArgs<T> a{};
    a.p = ph.p;
    a.n = ph.n;
    a.tiles = ph.M;
    a.nstruct = ph.nstruct;
    a.nstruct_max = ph.S;
    a.lower = ph.lower;
    a.upper = ph.upper;
    a.write_lower = ph.write_lower;
    a.write_upper = ph.write_upper;
    a.flank_in = reinterpret_cast<const T *>(ph.flank_in);
    a.flank_out = reinterpret_cast<T *>(ph.flank_out);
    a.state = reinterpret_cast<T *>(ph.state);
    if (warps > ph.nstruct) warps = ph.nstruct;
    if (warps < 1) warps = 1;
    const int64_t blocks = (warps + 3) / 4;  // 4 warps per CTA
    k_heat_fold<K, C><<<(unsigned)blocks, 128, 0, st>>>(a, prm);
    return cudaGetLastError();
}

template <class C>
static cudaError_t by_width(int W, const FoldPhase &ph, const HeatParams &prm, int64_t warps, cudaStream_t st) {
    switch (W) {
    case 64: return go<2, C>(ph, prm, warps, st);
    case 128: return go<4, C>(ph, prm, warps, st);
    case 256: return go<8, C>(ph, prm, warps, st);
    case 512: return go<16, C>(ph, prm, warps, st);
    case 1024: return go<32, C>(ph, prm, warps, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fold(int precision, int W, const FoldPhase &ph, const HeatParams &prm, int64_t warps,
                        cudaStream_t st) {
    switch (precision) {
    case SW_FP64: return by_width<FoldF64>(W, ph, prm, warps, st);
    case SW_FP32: return by_width<FoldF32>(W, ph, prm, warps, st);
    default: return by_width<FoldComp>(W, ph, prm, warps, st);
    }
}

}  // namespace sw
