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
// wrong results; serialise them.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "../../include/swept.h"
#include "schemes.cuh"
#include "swept_phase.cuh"

using namespace sw;

namespace {

static __device__ __align__(256) unsigned char sw_noalloc_scratch[SW_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Host code may not use &sw_noalloc_scratch as a device address (it names a
// host-side stand-in). Look the real address up once per device, with that
// device current, and cache it.
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SW_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SW_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, sw_noalloc_scratch);
        if (e != cudaSuccess || !p) return SW_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SW_OK;
}

template <class P>
int run_phases(const sw_problem &prob, int W, void *scratch, void *state, int64_t L, cudaStream_t st) {
    using T = typename P::T;
    const int H = W / 2;
    const int64_t M = prob.n / W, S = M + 1;
    const size_t buf_elems = size_t(P::NSNAP) * size_t(S) * 2 * W;
    const size_t buf_bytes = (buf_elems * sizeof(T) + 255) / 256 * 256;
    if (2 * buf_bytes > SW_NOALLOC_SCRATCH_BYTES) return SW_ERR_TOO_LARGE;
    T *flank[2] = {reinterpret_cast<T *>(scratch),
                   reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(scratch) + buf_bytes)};
    const size_t smem = swept_smem_elems<P>(W) * sizeof(T);
    if (smem > 227 * 1024) return SW_ERR_UNSUPPORTED;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_swept_phase<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return SW_ERR_CUDA;
    int threads = std::min(512, std::max(32, (W / 2 + 31) / 32 * 32));
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
    const int64_t P_last = (L + H - 1) / H;
    for (int64_t p = 0; p <= P_last; ++p) {
        PhaseArgs<T> a{};
        a.n = prob.n;
        a.W = W;
        a.H = H;
        a.periodic = periodic ? 1 : 0;
        a.p = (p == 0) ? 0 : (int)(2 - (p & 1));
        a.F = p * H;
        a.lower = (p == 0) ? 0 : (int)std::min<int64_t>(H, L - (p - 1) * H);
        a.upper = (p == P_last) ? 0 : (int)std::min<int64_t>(H - 1, L - p * H);
        a.write_lower = (p == P_last) ? 1 : 0;
        a.write_upper = (a.upper > 0 && p * H + a.upper == L) ? 1 : 0;
        a.tiles = M;
        a.nstruct = (p & 1) ? (periodic ? M : M + 1) : M;
        a.nstruct_max = S;
        a.flank_in = (p == 0) ? nullptr : flank[(p - 1) & 1];
        a.flank_out = flank[p & 1];
        a.state = reinterpret_cast<T *>(state);
        k_swept_phase<P><<<(unsigned)a.nstruct, threads, smem, st>>>(a, prm);
    }
    return cudaGetLastError() == cudaSuccess ? SW_OK : SW_ERR_CUDA;
}

}  // namespace

extern "C" int sw_run_noalloc(const sw_problem *p, void *state, int64_t nsteps, void *stream) {
    if (!p || !state || nsteps < 0) return SW_ERR_BAD_ARG;
    if (p->method != SW_SWEPT || p->flags != 0) return SW_ERR_BAD_ARG;
    if (p->scheme != SW_HEAT && p->scheme != SW_EULER) return SW_ERR_BAD_ARG;
    if (p->precision < SW_FP64 || p->precision > SW_FP32_COMP) return SW_ERR_BAD_ARG;
    if (p->boundary != SW_PERIODIC && p->boundary != SW_TRANSMISSIVE) return SW_ERR_BAD_ARG;
    if (p->scheme == SW_HEAT ? !(p->r > 0.0 && p->r < 1e6)
                             : !(p->dt_dx > 0.0 && p->gamma > 1.0 && p->gamma < 1e6))
        return SW_ERR_BAD_ARG;
    int W = p->tile_width;
    if (W == 0) {
        for (W = SW_MAX_TILE; W >= SW_MIN_TILE; W >>= 1)
            if (p->n % W == 0 && p->n >= 2 * (int64_t)W) break;
        if (W < SW_MIN_TILE) return SW_ERR_BAD_ARG;
    }
    if (W < SW_MIN_TILE || W > SW_MAX_TILE || (W & 1) || p->n < 2 * (int64_t)W || p->n % W != 0)
        return SW_ERR_BAD_ARG;
    if (nsteps == 0) return SW_OK;
    void *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != SW_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t L = nsteps * (p->scheme == SW_HEAT ? 1 : 4);
    if (p->scheme == SW_HEAT) {
        switch (p->precision) {
        case SW_FP64: return run_phases<HeatPolicy<0>>(*p, W, scratch, state, L, st);
        case SW_FP32: return run_phases<HeatPolicy<1>>(*p, W, scratch, state, L, st);
        default: return run_phases<HeatPolicy<2>>(*p, W, scratch, state, L, st);
        }
    }
    switch (p->precision) {
    case SW_FP64: return run_phases<EulerPolicy<0>>(*p, W, scratch, state, L, st);
    case SW_FP32: return run_phases<EulerPolicy<1>>(*p, W, scratch, state, L, st);
    default: return run_phases<EulerPolicyComp>(*p, W, scratch, state, L, st);
    }
}
