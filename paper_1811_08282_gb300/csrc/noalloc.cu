// noalloc.cu -- sw_run_noalloc: the swept run without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside a framework whose
// memory pool owns the device (a direct cudaMalloc there either fails or
// escapes the pool's accounting), and latency-critical loops that forbid any
// allocation after start-up (cudaMalloc/cudaFree can synchronise the device).
// For them this entry point runs the same swept phases as sw_run, but keeps the
// flank buffers (the only scratch the phases need) in one static device array
// compiled into the library. Every GPU that loads libswept.so holds this array
// (SW_NOALLOC_SCRATCH_BYTES) until the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents. Nothing in it has to start at zero: each phase writes the flanks
// it hands on before the next phase reads them. Calls that overlap on the GPU
// (different streams, or different host threads) race on the array and give
// wrong results; serialise them. The problem is validated by the same rules as
// sw_create and runs in the same data-structure form as sw_run would choose.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "../../include/swept.h"
#include "problem.h"
#include "euler.cuh"
#include "heat.cuh"
#include "heat_policy.cuh"
#include "swept_phase.cuh"

using namespace sw;

namespace {

static __device__ __align__(256) unsigned char sw_noalloc_scratch[SW_NOALLOC_SCRATCH_BYTES];

// Host code may not use &sw_noalloc_scratch as a device address (it names a
// host-side stand-in). The real address is looked up with the caller's device
// current on every call: a host-side lookup that allocates nothing, so a device
// reset or a new primary context, after which the module is loaded again and
// the array may sit elsewhere, never leaves a stale address behind. The first
// lookup on a device also loads the library's device code there.
int scratch_address(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, sw_noalloc_scratch);
    if (e != cudaSuccess || !p) return SW_ERR_CUDA;
    *out = p;
    return SW_OK;
}

// Bytes of one flank buffer, rounded up to 256, or 0 when two of them would not
// fit in the static array. The structure count is compared against the bound
// before any product is formed, so no size can wrap.
template <class P> size_t flank_buffer_bytes(int64_t S, int W) {
    const size_t per_struct = size_t(P::NSNAP) * 2 * size_t(W) * sizeof(typename P::T);
    if (S <= 0 || size_t(S) > SW_NOALLOC_SCRATCH_BYTES / (2 * per_struct)) return 0;
    const size_t bytes = (size_t(S) * per_struct + 255) / 256 * 256;
    return 2 * bytes <= SW_NOALLOC_SCRATCH_BYTES ? bytes : 0;
}

template <class P>
int run_phases(const sw_problem &prob, int W, void *scratch, void *state, int64_t L, cudaStream_t st) {
    using T = typename P::T;
    constexpr int R = P::R;
    const int H = W / 2, HL = H / R;  // levels per phase half (radius-2 windows: W/4)
    const int64_t M = prob.n / W, S = M + 1;
    const size_t buf_bytes = flank_buffer_bytes<P>(S, W);
    if (buf_bytes == 0) return SW_ERR_TOO_LARGE;
    T *flank[2] = {reinterpret_cast<T *>(scratch),
                   reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(scratch) + buf_bytes)};
    const size_t smem = swept_smem_elems<P>(W) * sizeof(T);
    if (smem > 227 * 1024) return SW_ERR_UNSUPPORTED;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_swept_phase<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return SW_ERR_CUDA;
    const int threads = std::min(512, std::max(32, (W / 2 + 31) / 32 * 32));
    typename P::Params prm{};
    if constexpr (std::is_same<typename P::Params, HeatParams>::value) {
        prm.r = prob.r;
        prm.rf = (float)prob.r;
        prm.rf_lo = (float)(prob.r - (double)prm.rf);
    } else {
        prm.gamma = prob.gamma;
        prm.gm1 = prob.gamma - 1.0;
        prm.lam = prob.dt_dx;
        prm.hlam = 0.5 * prob.dt_dx;
        prm.gammaf = (float)prob.gamma;
        prm.gm1f = (float)(prob.gamma - 1.0);
        prm.lamf = (float)prob.dt_dx;
        prm.hlamf = (float)(0.5 * prob.dt_dx);
    }
    const bool periodic = prob.boundary == SW_PERIODIC;
    const int64_t P_last = (L + HL - 1) / HL;
    for (int64_t p = 0; p <= P_last; ++p) {
        PhaseArgs<T> a{};
        a.n = prob.n;
        a.W = W;
        a.H = H;
        a.periodic = periodic ? 1 : 0;
        a.p = (p == 0) ? 0 : (int)(2 - (p & 1));
        a.F = p * HL;
        a.lower = (p == 0) ? 0 : (int)std::min<int64_t>(HL, L - (p - 1) * HL);
        a.upper = (p == P_last) ? 0 : (int)std::min<int64_t>(HL - 1, L - p * HL);
        a.write_lower = (p == P_last) ? 1 : 0;
        a.write_upper = (a.upper > 0 && p * HL + a.upper == L) ? 1 : 0;
        a.tiles = M;
        a.nstruct = (p & 1) ? (periodic ? M : M + 1) : M;
        a.nstruct_max = S;
        a.flank_in = (p == 0) ? nullptr : flank[(p - 1) & 1];
        a.flank_out = flank[p & 1];
        a.state = reinterpret_cast<T *>(state);
        k_swept_phase<P><<<(unsigned)a.nstruct, threads, smem, st>>>(a, prm);
        // stop at the first launch that fails (nothing else is pending: checked on entry)
        if (cudaGetLastError() != cudaSuccess) return SW_ERR_CUDA;
    }
    return SW_OK;
}

}  // namespace

extern "C" int sw_run_noalloc(const sw_problem *p, void *state, int64_t nsteps, void *stream) {
    if (!p || !state || nsteps < 0) return SW_ERR_BAD_ARG;
    if (validate_problem(p) != SW_OK) return SW_ERR_BAD_ARG;
    // the generic phase kernel and the two data-structure forms only
    if (p->method != SW_SWEPT || (p->flags & ~(SW_FLAG_GENERIC | SW_FLAG_LENGTHENED | SW_FLAG_FLATTENED)))
        return SW_ERR_BAD_ARG;
    const int W = p->tile_width ? p->tile_width : default_tile_width(*p);
    if (W == 0) return SW_ERR_BAD_ARG;
    const bool flat = euler_flattened(*p, W);
    const int warn = (p->scheme == SW_HEAT && p->r > 0.5) ? SW_WARN_UNSTABLE : SW_OK;
    if (nsteps == 0) return warn;
    // a CUDA error already pending on this thread belongs to earlier work: report it
    // without launching (and without clearing it) rather than mistake it for ours
    if (cudaPeekAtLastError() != cudaSuccess) return SW_ERR_CUDA;
    void *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != SW_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t L = nsteps * (p->scheme == SW_HEAT ? 1 : (flat ? 2 : 4));
    if (p->scheme == SW_HEAT) {
        switch (p->precision) {
        case SW_FP64: rc = run_phases<HeatPolicy<0>>(*p, W, scratch, state, L, st); break;
        case SW_FP32: rc = run_phases<HeatPolicy<1>>(*p, W, scratch, state, L, st); break;
        default: rc = run_phases<HeatPolicy<2>>(*p, W, scratch, state, L, st); break;
        }
    } else if (flat) {
        switch (p->precision) {
        case SW_FP64: rc = run_phases<EulerFlatPolicy<0>>(*p, W, scratch, state, L, st); break;
        case SW_FP32: rc = run_phases<EulerFlatPolicy<1>>(*p, W, scratch, state, L, st); break;
        default: rc = run_phases<EulerFlatPolicyComp>(*p, W, scratch, state, L, st); break;
        }
    } else {
        switch (p->precision) {
        case SW_FP64: rc = run_phases<EulerPolicy<0>>(*p, W, scratch, state, L, st); break;
        case SW_FP32: rc = run_phases<EulerPolicy<1>>(*p, W, scratch, state, L, st); break;
        default: rc = run_phases<EulerPolicyComp>(*p, W, scratch, state, L, st); break;
        }
    }
    return rc != SW_OK ? rc : warn;
}
