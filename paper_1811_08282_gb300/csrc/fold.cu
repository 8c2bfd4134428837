// fold.cu -- instantiations and launcher of the register-resident heat Diamond kernel.
#include "fold.h"
#include "fold_heat.cuh"

#include "../../include/swept.h"

namespace sw {

bool fold_supported(int precision, int W) {
    if (precision < SW_FP64 || precision > SW_FP32_COMP) return false;
    return W == 128 || W == 256 || W == 512 || W == 1024;
}

int fold_warps_per_sm(int precision, int W) {
    if (precision == SW_FP32) return W >= 1024 ? 8 : 16;
    return W >= 512 ? 8 : 16;
}

template <int K, class C>
static cudaError_t go(int p, int64_t M, int64_t S, const void *fin, void *fout, const HeatParams &prm,
                      int64_t warps, cudaStream_t st) {
    using T = typename C::T;
    FoldArgs<T> a{};
    a.p = p;
    a.tiles = M;
    a.nstruct_max = S;
    a.flank_in = reinterpret_cast<const T *>(fin);
    a.flank_out = reinterpret_cast<T *>(fout);
    if (warps > M) warps = M;
    if (warps < 1) warps = 1;
    const int64_t blocks = (warps + 3) / 4;  // 4 warps per CTA
    k_heat_fold<K, C><<<(unsigned)blocks, 128, 0, st>>>(a, prm);
    return cudaGetLastError();
}

template <class C>
static cudaError_t by_width(int W, int p, int64_t M, int64_t S, const void *fin, void *fout,
                            const HeatParams &prm, int64_t warps, cudaStream_t st) {
    switch (W) {
    case 128: return go<4, C>(p, M, S, fin, fout, prm, warps, st);
    case 256: return go<8, C>(p, M, S, fin, fout, prm, warps, st);
    case 512: return go<16, C>(p, M, S, fin, fout, prm, warps, st);
    case 1024: return go<32, C>(p, M, S, fin, fout, prm, warps, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fold(int precision, int W, int p, int64_t M, int64_t S, const void *flank_in,
                        void *flank_out, const HeatParams &prm, int64_t warps, cudaStream_t st) {
    switch (precision) {
    case SW_FP64: return by_width<FoldF64>(W, p, M, S, flank_in, flank_out, prm, warps, st);
    case SW_FP32: return by_width<FoldF32>(W, p, M, S, flank_in, flank_out, prm, warps, st);
    default: return by_width<FoldComp>(W, p, M, S, flank_in, flank_out, prm, warps, st);
    }
}

}  // namespace sw
