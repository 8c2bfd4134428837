// fold_euler.cu -- instantiations and launcher of the register-resident Euler phase kernel.
#include "fold.h"
#include "fold_euler.cuh"

#include "../../include/swept.h"

namespace sw {

bool euler_fold_supported(int precision, int W) {
    if (precision == SW_FP64) return W == 128;
    if (precision == SW_FP32 || precision == SW_FP32_COMP) return W == 128 || W == 256;
    return false;
}

// Measured on GB300 (one Diamond phase, N = 2^22): FP32 is fastest at 20 warps per SM
// (its launch bound keeps 5 CTAs resident), FP32 hi/lo at 16, FP64 at 8 (register bound).
int euler_fold_warps_per_sm(int precision, int W) {
    if (precision == SW_FP64) return 8;
    if (precision == SW_FP32) return 20;
    return 16;
}

template <int K, class C>
static cudaError_t go(const EulerFoldPhase &ph, const EulerParams &prm, int64_t warps, cudaStream_t st) {
    using T = typename C::T;
    EFoldArgs<T> a{};
    a.p = ph.p;
    a.periodic = ph.periodic;
    a.n = ph.n;
    a.tiles = ph.M;
    a.nstruct = ph.nstruct;
    a.nstruct_max = ph.S;
    a.lower = ph.lower;
    a.upper = ph.upper;
    a.write_lower = ph.write_lower;
    a.flank_in = reinterpret_cast<const T *>(ph.flank_in);
    a.flank_out = reinterpret_cast<T *>(ph.flank_out);
    a.state = reinterpret_cast<T *>(ph.state);
    if (warps > ph.nstruct) warps = ph.nstruct;
    if (warps < 1) warps = 1;
    const int64_t blocks = (warps + 3) / 4;  // 4 warps per CTA
    k_euler_fold<K, C><<<(unsigned)blocks, 128, 0, st>>>(a, prm);
    return cudaGetLastError();
}

cudaError_t launch_euler_fold(int precision, int W, const EulerFoldPhase &ph, const EulerParams &prm, int64_t warps,
                              cudaStream_t st) {
    if (!euler_fold_supported(precision, W)) return cudaErrorInvalidValue;
    switch (precision) {
    case SW_FP64: return go<4, EFoldPlain<OpsD>>(ph, prm, warps, st);
    case SW_FP32: return W == 128 ? go<4, EFoldPlain<OpsF>>(ph, prm, warps, st) : go<8, EFoldPlain<OpsF>>(ph, prm, warps, st);
    default: return W == 128 ? go<4, EFoldComp>(ph, prm, warps, st) : go<8, EFoldComp>(ph, prm, warps, st);
    }
}

}  // namespace sw
