// api.cu -- C ABI of libswept.so (declared in include/swept.h): problem
// validation, scratch ownership (with guard words), the host-side phase planner
// of the swept rule (Section 4.1: generic, register-resident and flattened phase
// kernels), the per-step loop (Section 4.3, both Euler forms), CUDA-graph replay
// of a run, the hybrid CPU/GPU split of Section 4.2 (the host share runs
// cpu_phase.h on a thread pool), plus conversion, conservation and positivity
// utilities. GPU compute runs in the kernels of swept_phase.cuh, fold_*.cuh and
// perstep.cuh; this file plans, launches and moves the hybrid run's flank slots.
#include <cuda_runtime.h>

#include <algorithm>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/swept.h"
#include "cpu_phase.h"
#include "problem.h"
#include "fold.h"
#include "perstep.cuh"
#include "euler.cuh"
#include "heat.cuh"
#include "heat_policy.cuh"
#include "swept_phase.cuh"

using namespace sw;

namespace {

// Persistent host threads for the host share of a hybrid run: run(f) calls f(t) for
// t = 0 .. size-1, t = 0 on the calling thread, and returns when all calls have.
class HostPool {
   public:
    explicit HostPool(int n) : n_(n) {
        for (int t = 1; t < n; ++t) th_.emplace_back([this, t] { loop(t); });
    }
    ~HostPool() {
        {
            std::lock_guard<std::mutex> g(m_);
            stop_ = true;
            ++gen_;
        }
        cv_.notify_all();
        for (auto &t : th_) t.join();
    }
    int size() const { return n_; }
    void run(const std::function<void(int)> &f) {
        {
            std::lock_guard<std::mutex> g(m_);
            job_ = &f;
            pending_ = n_ - 1;
            ++gen_;
        }
        cv_.notify_all();
        f(0);
        std::unique_lock<std::mutex> lk(m_);
        done_.wait(lk, [&] { return pending_ == 0; });
        job_ = nullptr;
    }

   private:
    void loop(int t) {
        int64_t seen = 0;
        for (;;) {
            const std::function<void(int)> *job;
            {
                std::unique_lock<std::mutex> lk(m_);
                cv_.wait(lk, [&] { return gen_ != seen; });
                seen = gen_;
                if (stop_) return;
                job = job_;
            }
            (*job)(t);
            std::lock_guard<std::mutex> g(m_);
            if (--pending_ == 0) done_.notify_one();
        }
    }
    int n_;
    std::vector<std::thread> th_;
    std::mutex m_;
    std::condition_variable cv_, done_;
    const std::function<void(int)> *job_ = nullptr;
    int64_t gen_ = 0;
    int pending_ = 0;
    bool stop_ = false;
};

}  // namespace

struct sw_handle {
    sw_problem prob;
    int W = 0, H = 0, threads = 0;
    int64_t M = 0, S = 0;       // tiles, structures per flank buffer
    size_t esize = 0;           // element size of the working precision
    int nsnap = 0, nio = 0;     // snapshot fields, state planes
    size_t smem = 0;            // dynamic shared memory per swept CTA
    void *flank[2] = {nullptr, nullptr};
    size_t flank_bytes = 0;
    void *scratch = nullptr;    // per-step ping-pong planes / Q* planes
    size_t scratch_bytes = 0;
    void *dev_state = nullptr;  // device copy used by sw_run_host
    int *d_status = nullptr;    // [0] latched status, [1..2] first bad cell (int64)
    double *d_partial = nullptr;
    double *d_sums = nullptr;
    HeatParams hp{};
    EulerParams ep{};
    int64_t last_launches = 0;
    int device = 0;
    // tracing: event pairs around the first `ev_cap` launches of a run
    std::vector<cudaEvent_t> events;
    std::vector<int32_t> kinds;
    int64_t ev_cap = 0, ev_used = 0;
    int sms = 152;  // streaming multiprocessors of the device
    // hybrid runs: pinned host mirrors of the flank buffers and the state, host threads
    void *h_flank[2] = {nullptr, nullptr};
    void *h_state = nullptr;
    HostPool *pool = nullptr;
    cudaEvent_t hy_ev[2] = {nullptr, nullptr};
    // SW_FLAG_GRAPH: the captured run for the last (state, nsteps) pair
    cudaStream_t gstream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    void *g_state = nullptr;
    int64_t g_steps = -1, g_launches = 0;
};

namespace {

constexpr int kRedBlocks = 1024;
constexpr size_t kGuardBytes = 256;     // guard after each scratch buffer
constexpr unsigned char kGuardByte = 0xA5;
constexpr int kRedThreads = 256;

int scheme_nv(const sw_problem &p) { return p.scheme == SW_HEAT ? 1 : 3; }

int planes_of(const sw_problem &p) {
    const int nv = scheme_nv(p);
    return p.precision == SW_FP32_COMP ? 2 * nv : nv;
}

size_t elem_size(const sw_problem &p) { return p.precision == SW_FP64 ? sizeof(double) : sizeof(float); }

// the form a handle runs in (Section 4.3): fixed at sw_create from the problem and its W
bool flattened(const sw_problem &p) { return euler_flattened(p, p.tile_width); }

int swept_threads(int W) {
    int t = W / 2;
    t = (t + 31) / 32 * 32;
    return std::min(512, std::max(32, t));
}

template <class P> size_t swept_smem(int W) { return swept_smem_elems<P>(W) * sizeof(typename P::T); }

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SW_OK;
    if (e == cudaErrorMemoryAllocation) return SW_ERR_OOM;
    return SW_ERR_CUDA;
}

template <class P> int prepare_swept_kernel(size_t smem) {
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_swept_phase<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return SW_OK;
}

// Record the start / end event of launch `i` of the current run (tracing only).
inline void trace_begin(sw_handle *h, int64_t i, int32_t kind, cudaStream_t st) {
    if (i < h->ev_cap) {
        cudaEventRecord(h->events[2 * i], st);
        h->kinds[i] = kind;
    }
}
inline void trace_end(sw_handle *h, int64_t i, cudaStream_t st) {
    if (i < h->ev_cap) {
        cudaEventRecord(h->events[2 * i + 1], st);
        h->ev_used = i + 1;
    }
}

// Host scheme matching each GPU storage policy (same fields, same per-cell arithmetic);
// void for policies the host share does not run (the flattened form).
template <class P> struct HostOf {
    using type = void;
};
template <> struct HostOf<HeatPolicy<0>> {
    using type = HostHeatPlain<HostOpsD>;
    static type make(const sw_handle *h) { return type{h->hp.r}; }
};
template <> struct HostOf<HeatPolicy<1>> {
    using type = HostHeatPlain<HostOpsF>;
    static type make(const sw_handle *h) { return type{h->hp.rf}; }
};
template <> struct HostOf<HeatPolicy<2>> {
    using type = HostHeatComp;
    static type make(const sw_handle *h) { return type{h->hp.rf, h->hp.rf_lo}; }
};
template <> struct HostOf<EulerPolicy<0>> {
    using type = HostEuler<HostOpsD, false>;
    static type make(const sw_handle *h) { return type{eu_k<HostOpsD>(h->ep), {}}; }
};
template <> struct HostOf<EulerPolicy<1>> {
    using type = HostEuler<HostOpsF, false>;
    static type make(const sw_handle *h) { return type{eu_k<HostOpsF>(h->ep), {}}; }
};
template <> struct HostOf<EulerPolicyComp> {
    using type = HostEuler<HostOpsF, true>;
    static type make(const sw_handle *h) { return type{eu_k<HostOpsF>(h->ep), {}}; }
};

// A hybrid run (Section 4.2's affinity split): the GPU runs structures 0 .. Mg-1 of every
// phase, the host threads the rest.
struct Hybrid {
    int64_t Mg;
    int64_t first = INT64_MAX, last = -1;  // state cells the host wrote
};

// Copy the flank slot of structure b (all fields, both sides) between the device and its
// pinned host mirror.
cudaError_t copy_slot(sw_handle *h, int buf, int64_t b, bool to_device, cudaStream_t st) {
    const size_t es = h->esize;
    const size_t pitch = size_t(h->S) * 2 * h->W * es, width = size_t(2) * h->W * es;
    const size_t off = size_t(b) * 2 * h->W * es;
    char *dv = static_cast<char *>(h->flank[buf]) + off;
    char *hv = static_cast<char *>(h->h_flank[buf]) + off;
    return to_device ? cudaMemcpy2DAsync(dv, pitch, hv, pitch, width, h->nsnap, cudaMemcpyHostToDevice, st)
                     : cudaMemcpy2DAsync(hv, pitch, dv, pitch, width, h->nsnap, cudaMemcpyDeviceToHost, st);
}

// Copy state cells [j0, j1] of every plane between the device state and the host mirror.
cudaError_t copy_cells(sw_handle *h, void *state, int64_t j0, int64_t j1, bool to_device, cudaStream_t st) {
    if (j1 < j0) return cudaSuccess;
    const size_t es = h->esize, pitch = size_t(h->prob.n) * es, width = size_t(j1 - j0 + 1) * es;
    char *dv = static_cast<char *>(state) + size_t(j0) * es;
    char *hv = static_cast<char *>(h->h_state) + size_t(j0) * es;
    return to_device ? cudaMemcpy2DAsync(dv, pitch, hv, pitch, width, h->nio, cudaMemcpyHostToDevice, st)
                     : cudaMemcpy2DAsync(hv, pitch, dv, pitch, width, h->nio, cudaMemcpyDeviceToHost, st);
}

template <class P>
int launch_swept(sw_handle *h, void *state, int64_t L, cudaStream_t st, Hybrid *hy = nullptr) {
    using T = typename P::T;
    const int H = h->H, W = h->W;
    const int HL = H / P::R;  // levels per phase half
    const int64_t P_last = (L + HL - 1) / HL;
    const bool periodic = h->prob.boundary == SW_PERIODIC;
    // periodic heat at W = 32K: every phase except a truncated upper half (which stores its
    // row mid-way) runs on the register-resident kernel
    const bool fold = std::is_same<typename P::Params, HeatParams>::value && periodic &&
                      !(h->prob.flags & SW_FLAG_GENERIC) && fold_supported(h->prob.precision, W);
    const int64_t fold_warps = int64_t(h->sms) * fold_warps_per_sm(h->prob.precision, W);
    // Euler at W = 128 (and 256 in FP32), on request only (it is the slower kernel on GB300)
    const bool efold = std::is_same<typename P::Params, EulerParams>::value && P::R == 1 &&
                       (h->prob.flags & SW_FLAG_EULER_FOLD) && !(h->prob.flags & SW_FLAG_GENERIC) &&
                       euler_fold_supported(h->prob.precision, W);
    const int64_t efold_warps = int64_t(h->sms) * euler_fold_warps_per_sm(h->prob.precision, W);
    int64_t launches = 0;
    using Sch = typename HostOf<P>::type;
    constexpr bool kHost = !std::is_void<Sch>::value;
    using SchV = typename std::conditional<kHost, Sch, int>::type;
    std::vector<SchV> sch;
    std::vector<std::vector<T>> work;
    std::vector<WrittenRange> written;
    if (hy && !kHost) return SW_ERR_BAD_ARG;
    if constexpr (kHost) if (hy) {
        const int nt = h->pool->size();
        for (int t = 0; t < nt; ++t) sch.push_back(HostOf<P>::make(h));
        work.assign(nt, std::vector<T>(size_t(2) * Sch::NF * (W + 2)));
        written.assign(nt, WrittenRange{});
        // the host's tiles of the initial state
        cudaError_t e = copy_cells(h, state, hy->Mg * W, h->prob.n - 1, false, st);
        if (e == cudaSuccess) e = cudaEventRecord(h->hy_ev[1], st);
        if (e != cudaSuccess) return cuda_status(e);
    }
    for (int64_t p = 0; p <= P_last; ++p) {
        PhaseArgs<T> a{};
        a.n = h->prob.n;
        a.W = W;
        a.H = H;
        a.periodic = periodic ? 1 : 0;
        // the kernel needs only "Up or not" and the parity of p
        a.p = (p == 0) ? 0 : (int)(2 - (p & 1));
        a.F = p * HL;
        a.lower = (p == 0) ? 0 : (int)std::min<int64_t>(HL, L - (p - 1) * HL);
        a.upper = (p == P_last) ? 0 : (int)std::min<int64_t>(HL - 1, L - p * HL);
        a.write_lower = (p == P_last) ? 1 : 0;
        a.write_upper = (a.upper > 0 && p * HL + a.upper == L) ? 1 : 0;
        a.tiles = h->M;
        a.nstruct = (p & 1) ? (periodic ? h->M : h->M + 1) : h->M;
        a.nstruct_max = h->S;
        a.flank_in = (p == 0) ? nullptr : reinterpret_cast<const T *>(h->flank[(p - 1) & 1]);
        a.flank_out = reinterpret_cast<T *>(h->flank[p & 1]);
        a.state = reinterpret_cast<T *>(state);
        typename P::Params prm;
        if constexpr (std::is_same<typename P::Params, HeatParams>::value) prm = h->hp;
        else prm = h->ep;
        const int64_t nstruct = a.nstruct;
        if (hy) {
            // the host's flank slot of phase p-1 that a GPU structure of phase p reads: the
            // seam structure Mg (p even), or the last tile M-1 across the periodic wrap (p odd)
            const int64_t slot = (p == 0) ? -1 : ((p & 1) == 0 ? hy->Mg : (periodic ? h->M - 1 : -1));
            if (slot >= 0) {
                cudaError_t e = copy_slot(h, (int)((p - 1) & 1), slot, true, st);
                if (e != cudaSuccess) return cuda_status(e);
            }
            a.nstruct = hy->Mg;
        }
        trace_begin(h, launches, p == 0 ? 0 : (p == P_last ? 2 : 1), st);
        if (fold && !a.write_upper) {
            FoldPhase ph{a.p, a.n, h->M, h->S, a.nstruct, a.lower, a.upper, a.write_lower, a.write_upper,
                         a.flank_in, a.flank_out, state};
            cudaError_t e = launch_fold(h->prob.precision, W, ph, h->hp, fold_warps, st);
            if (e != cudaSuccess) return cuda_status(e);
        } else if (efold && !a.write_upper) {
            EulerFoldPhase ph{a.p, a.periodic, a.n, h->M, a.nstruct, h->S, a.lower, a.upper, a.write_lower,
                              a.flank_in, a.flank_out, state};
            cudaError_t e = launch_euler_fold(h->prob.precision, W, ph, h->ep, efold_warps, st);
            if (e != cudaSuccess) return cuda_status(e);
        } else {
            k_swept_phase<P><<<(unsigned)a.nstruct, h->threads, h->smem, st>>>(a, prm);
        }
        trace_end(h, launches, st);
        ++launches;
        if constexpr (kHost) if (hy) {
            // the GPU's flank slot of phase p that a host structure of phase p+1 reads: the
            // last GPU tile Mg-1 (p even), or the seam structure 0 across the periodic wrap (p odd)
            const int64_t slot = (p == P_last) ? -1 : ((p & 1) == 0 ? hy->Mg - 1 : (periodic ? 0 : -1));
            cudaError_t e = cudaSuccess;
            if (slot >= 0) e = copy_slot(h, (int)(p & 1), slot, false, st);
            if (e == cudaSuccess) e = cudaEventRecord(h->hy_ev[p & 1], st);
            // the host's structures of phase p, once the GPU's slots of phase p-1 have arrived
            if (e == cudaSuccess) e = cudaEventSynchronize(h->hy_ev[(p + 1) & 1]);
            if (e != cudaSuccess) return cuda_status(e);
            HostPhase<T> hp{a.n, W, H, a.periodic, a.p, a.F, a.lower, a.upper, a.write_lower, a.write_upper,
                            h->M, h->S,
                            p == 0 ? nullptr : static_cast<const T *>(h->h_flank[(p - 1) & 1]),
                            static_cast<T *>(h->h_flank[p & 1]), static_cast<T *>(h->h_state)};
            const int64_t b0 = hy->Mg, cnt = nstruct - hy->Mg;
            const int nt = h->pool->size();
            h->pool->run([&](int t) {
                const int64_t lo = b0 + cnt * t / nt, hi = b0 + cnt * (t + 1) / nt;
                for (int64_t b = lo; b < hi; ++b) cpu_structure(sch[t], hp, b, work[t].data(), written[t]);
            });
        }
    }
    h->last_launches = launches;
    if constexpr (kHost) if (hy) {
        for (const WrittenRange &w : written) {
            hy->first = std::min(hy->first, w.first);
            hy->last = std::max(hy->last, w.last);
        }
        cudaError_t e = copy_cells(h, state, hy->first, hy->last, true, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return cuda_status(cudaGetLastError());
}

unsigned grid_for(int64_t work, int threads, int cap) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

int launch_perstep_heat(sw_handle *h, void *state, int64_t nsteps, cudaStream_t st) {
    const int64_t n = h->prob.n;
    const int periodic = h->prob.boundary == SW_PERIODIC;
    const size_t bytes = size_t(planes_of(h->prob)) * n * h->esize;
    void *bufs[2] = {state, h->scratch};
    int64_t launches = 0;
    const int cap = 152 * 16;
    constexpr int64_t kMixedMinCells = int64_t(1) << 21;  // ~7 waves of 152 x 2048 threads at 1 cell each
    // vector width: the caller's state may start anywhere; the scratch planes are 256-byte
    // aligned, so the state's own alignment (and n, for the second plane) decides
    const uintptr_t align = reinterpret_cast<uintptr_t>(state);
    const bool a16 = align % 16 == 0, a32 = align % 32 == 0;
    for (int64_t s = 0; s < nsteps; ++s) {
        void *in = bufs[s & 1], *out = bufs[(s + 1) & 1];
        trace_begin(h, launches, 3, st);
        switch (h->prob.precision) {
        case SW_FP64:
            // large grids: four (or two) cells per thread, half of them on the integer
            // pipes; a smaller grid is latency-bound, and one cell per thread on the FP64
            // pipe keeps the dependent chains short
            if (n >= kMixedMinCells && n % 4 == 0 && a32)
                k_heat_step<OpsD, 4><<<grid_for(n / 4, 256, cap), 256, 0, st>>>(
                    (const double *)in, (double *)out, n, h->hp.r, periodic);
            else if (n >= kMixedMinCells && n % 2 == 0 && a16)
                k_heat_step<OpsD, 2><<<grid_for(n / 2, 256, cap), 256, 0, st>>>(
                    (const double *)in, (double *)out, n, h->hp.r, periodic);
            else
                k_heat_step<OpsD, 1><<<grid_for(n, 256, cap), 256, 0, st>>>((const double *)in, (double *)out,
                                                                             n, h->hp.r, periodic);
            break;
        case SW_FP32:
            // 32 bytes per thread and iteration keeps enough loads in flight for HBM
            if (n % 8 == 0 && a32)
                k_heat_step<OpsF, 8><<<grid_for(n / 8, 256, cap), 256, 0, st>>>((const float *)in, (float *)out,
                                                                                 n, h->hp.rf, periodic);
            else if (n % 4 == 0 && a16)
                k_heat_step<OpsF, 4><<<grid_for(n / 4, 256, cap), 256, 0, st>>>((const float *)in, (float *)out,
                                                                                 n, h->hp.rf, periodic);
            else
                k_heat_step<OpsF, 1><<<grid_for(n, 256, cap), 256, 0, st>>>((const float *)in, (float *)out, n,
                                                                             h->hp.rf, periodic);
            break;
        default:
            if (n % 8 == 0 && a32)
                k_heat_step_comp<8><<<grid_for(n / 8, 256, cap), 256, 0, st>>>(
                    (const float *)in, (float *)out, n, h->hp.rf, h->hp.rf_lo, periodic);
            else if (n % 4 == 0 && a16)
                k_heat_step_comp<4><<<grid_for(n / 4, 256, cap), 256, 0, st>>>(
                    (const float *)in, (float *)out, n, h->hp.rf, h->hp.rf_lo, periodic);
            else
                k_heat_step_comp<1><<<grid_for(n, 256, cap), 256, 0, st>>>((const float *)in, (float *)out, n,
                                                                            h->hp.rf, h->hp.rf_lo, periodic);
            break;
        }
        trace_end(h, launches, st);
        ++launches;
    }
    if (nsteps & 1) {
        cudaError_t e = cudaMemcpyAsync(state, h->scratch, bytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_status(e);
    }
    h->last_launches = launches;
    return cuda_status(cudaGetLastError());
}

template <class O, bool COMP>
int launch_perstep_euler_t(sw_handle *h, void *state, int64_t nsteps, cudaStream_t st) {
    using T = typename O::T;
    const int64_t n = h->prob.n;
    const int periodic = h->prob.boundary == SW_PERIODIC;
    const int B = 256;
    const size_t smem = (size_t(3) * (B + 4) + (B + 4) + (B + 2) + size_t(3) * (B + 1)) * sizeof(T);
    const unsigned grid = (unsigned)((n + B - 1) / B);
    T *q = reinterpret_cast<T *>(state);
    T *s = reinterpret_cast<T *>(h->scratch);
    if (!flattened(h->prob)) {
        // lengthened form: four 3-point sub-step launches per step
        const size_t smem4 = (size_t(4) * (B + 2) + size_t(3) * (B + 1)) * sizeof(T);
        for (int64_t k = 0; k < nsteps; ++k) {
            trace_begin(h, 4 * k, 3, st);
            k_euler_sub<O, 0, COMP><<<grid, B, smem4, st>>>(q, s, n, h->ep, periodic);
            trace_end(h, 4 * k, st);
            trace_begin(h, 4 * k + 1, 3, st);
            k_euler_sub<O, 1, COMP><<<grid, B, smem4, st>>>(q, s, n, h->ep, periodic);
            trace_end(h, 4 * k + 1, st);
            trace_begin(h, 4 * k + 2, 3, st);
            k_euler_sub<O, 2, COMP><<<grid, B, smem4, st>>>(q, s, n, h->ep, periodic);
            trace_end(h, 4 * k + 2, st);
            trace_begin(h, 4 * k + 3, 3, st);
            k_euler_sub<O, 3, COMP><<<grid, B, smem4, st>>>(q, s, n, h->ep, periodic);
            trace_end(h, 4 * k + 3, st);
        }
        h->last_launches = 4 * nsteps;
        return cuda_status(cudaGetLastError());
    }
    for (int64_t k = 0; k < nsteps; ++k) {
        trace_begin(h, 2 * k, 3, st);
        k_euler_stage<O, false, COMP><<<grid, B, smem, st>>>(q, s, n, h->ep, periodic);
        trace_end(h, 2 * k, st);
        trace_begin(h, 2 * k + 1, 3, st);
        k_euler_stage<O, true, COMP><<<grid, B, smem, st>>>(q, s, n, h->ep, periodic);
        trace_end(h, 2 * k + 1, st);
    }
    h->last_launches = 2 * nsteps;
    return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------- utilities
__global__ void k_pack(const double *__restrict__ src, void *__restrict__ dst, int64_t count, int prec) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = src[i];
        if (prec == SW_FP64) {
            reinterpret_cast<double *>(dst)[i] = x;
        } else if (prec == SW_FP32) {
            reinterpret_cast<float *>(dst)[i] = __double2float_rn(x);
        } else {
            const float hi = __double2float_rn(x);
            const float lo = __double2float_rn(x - (double)hi);
            // layout: all hi planes, then all lo planes
            reinterpret_cast<float *>(dst)[i] = hi;
            reinterpret_cast<float *>(dst)[count + i] = lo;
        }
    }
}

__global__ void k_unpack(const void *__restrict__ src, double *__restrict__ dst, int64_t count, int prec) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (prec == SW_FP64) dst[i] = reinterpret_cast<const double *>(src)[i];
        else if (prec == SW_FP32) dst[i] = (double)reinterpret_cast<const float *>(src)[i];
        else
            dst[i] = (double)reinterpret_cast<const float *>(src)[i] +
                     (double)reinterpret_cast<const float *>(src)[count + i];
    }
}

// Deterministic FP64 sum of plane v: block b sums a fixed contiguous chunk with a
// fixed tree; the partials are summed in a fixed order by one block.
__device__ __forceinline__ double state_value(const void *st, int64_t n, int v, int64_t i, int prec, int nv) {
    if (prec == SW_FP64) return reinterpret_cast<const double *>(st)[v * n + i];
    const float *f = reinterpret_cast<const float *>(st);
    if (prec == SW_FP32) return (double)f[v * n + i];
    return (double)f[v * n + i] + (double)f[(nv + v) * n + i];
}

__global__ void __launch_bounds__(kRedThreads) k_sum_partial(const void *st, int64_t n, int nv, int prec,
                                                             double *partial) {
    __shared__ double red[kRedThreads];
    const int v = blockIdx.y;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * chunk;
    const int64_t hi = lo + chunk < n ? lo + chunk : n;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += state_value(st, n, v, i, prec, nv);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[v * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_sum_final(const double *partial, int nblocks, int nv, double *out) {
    __shared__ double red[kRedThreads];
    for (int v = 0; v < nv; ++v) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < nblocks; i += blockDim.x) acc += partial[v * nblocks + i];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[v] = red[0];
        __syncthreads();
    }
}

// Positivity / NaN scan of an Euler state; records the smallest bad index.
__global__ void k_check_physical(const void *st, int64_t n, int prec, double gamma,
                                 unsigned long long *first_bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double rho = state_value(st, n, 0, i, prec, 3);
        const double m = state_value(st, n, 1, i, prec, 3);
        const double E = state_value(st, n, 2, i, prec, 3);
        const double p = (gamma - 1.0) * (E - 0.5 * m * (m / rho));
        const bool ok = rho > 0.0 && p > 0.0 && isfinite(rho) && isfinite(m) && isfinite(E);
        if (!ok) atomicMin(first_bad, (unsigned long long)i);
    }
}

}  // namespace

namespace sw {

int validate_problem(const sw_problem *p) {
    if (!p) return SW_ERR_BAD_ARG;
    if (p->scheme != SW_HEAT && p->scheme != SW_EULER) return SW_ERR_BAD_ARG;
    if (p->precision < SW_FP64 || p->precision > SW_FP32_COMP) return SW_ERR_BAD_ARG;
    if (p->boundary != SW_PERIODIC && p->boundary != SW_TRANSMISSIVE) return SW_ERR_BAD_ARG;
    if (p->method != SW_SWEPT && p->method != SW_PERSTEP) return SW_ERR_BAD_ARG;
    if (p->flags & ~(SW_FLAG_GENERIC | SW_FLAG_EULER_FOLD | SW_FLAG_LENGTHENED | SW_FLAG_FLATTENED | SW_FLAG_GRAPH))
        return SW_ERR_BAD_ARG;
    if ((p->flags & SW_FLAG_LENGTHENED) && (p->flags & SW_FLAG_FLATTENED)) return SW_ERR_BAD_ARG;
    if (p->n < 4 || p->n > (int64_t(1) << 40)) return SW_ERR_BAD_ARG;
    if (p->scheme == SW_HEAT) {
        if (!(p->r > 0.0) || !(p->r < 1e6)) return SW_ERR_BAD_ARG;
    } else {
        if (!(p->dt_dx > 0.0) || !(p->gamma > 1.0) || !(p->gamma < 1e6)) return SW_ERR_BAD_ARG;
    }
    if (p->method == SW_SWEPT) {
        const int W = p->tile_width;
        if (W != 0) {
            if (W < SW_MIN_TILE || W > SW_MAX_TILE || (W & 1)) return SW_ERR_BAD_ARG;
            if (p->n % W != 0 || p->n < 2 * (int64_t)W) return SW_ERR_BAD_ARG;
            // an explicitly flattened Euler problem: radius-2 windows, W/4 levels per phase half
            if (p->scheme == SW_EULER && (p->flags & SW_FLAG_FLATTENED) && (W % 4 != 0 || W < 8))
                return SW_ERR_BAD_ARG;
        }
    } else if (p->tile_width < 0) {
        return SW_ERR_BAD_ARG;
    }
    return SW_OK;
}

}  // namespace sw

// ===================================================================== C ABI
extern "C" {

int sw_abi_version(void) { return SW_ABI_VERSION; }

const char *sw_status_string(int s) {
    switch (s) {
    case SW_OK: return "ok";
    case SW_WARN_UNSTABLE: return "warning: heat r > 1/2, FTCS is unstable";
    case SW_ERR_BAD_ARG: return "bad argument";
    case SW_ERR_CUDA: return "CUDA error";
    case SW_ERR_OOM: return "out of device memory";
    case SW_ERR_TIMEOUT: return "device-side wait timed out";
    case SW_ERR_NONPHYSICAL: return "non-physical state (rho <= 0, p <= 0 or NaN)";
    case SW_ERR_UNSUPPORTED: return "unsupported configuration";
    case SW_ERR_CORRUPT: return "a guard word after a scratch buffer was overwritten (out-of-bounds write)";
    case SW_ERR_TOO_LARGE:
        return "problem needs more flank scratch than the static no-allocation buffer holds "
               "(SW_NOALLOC_SCRATCH_BYTES)";
    default: return "unknown status";
    }
}

int sw_state_planes(const sw_problem *p) {
    if (validate_problem(p) != SW_OK) return SW_ERR_BAD_ARG;
    return planes_of(*p);
}

int64_t sw_state_bytes(const sw_problem *p) {
    if (validate_problem(p) != SW_OK) return SW_ERR_BAD_ARG;
    return int64_t(planes_of(*p)) * p->n * int64_t(elem_size(*p));
}

int sw_create(const sw_problem *p, sw_handle **out) {
    if (!out) return SW_ERR_BAD_ARG;
    int rc = validate_problem(p);
    if (rc != SW_OK) return rc;
    sw_handle *h = new (std::nothrow) sw_handle();
    if (!h) return SW_ERR_OOM;
    h->prob = *p;
    cudaGetDevice(&h->device);
    if (cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || h->sms <= 0)
        h->sms = 152;
    h->esize = elem_size(*p);
    h->nio = planes_of(*p);
    // scheme constants, rounded once on the host
    h->hp.r = p->r;
    h->hp.rf = (float)p->r;
    h->hp.rf_lo = (float)(p->r - (double)h->hp.rf);
    h->ep.gamma = p->gamma;
    h->ep.gm1 = p->gamma - 1.0;
    h->ep.lam = p->dt_dx;
    h->ep.hlam = 0.5 * p->dt_dx;
    h->ep.gammaf = (float)p->gamma;
    h->ep.gm1f = (float)(p->gamma - 1.0);
    h->ep.lamf = (float)p->dt_dx;
    h->ep.hlamf = (float)(0.5 * p->dt_dx);

    auto fail = [&](int code) {
        sw_destroy(h);
        return code;
    };
    cudaError_t e;
    if (p->method == SW_SWEPT) {
        h->W = p->tile_width ? p->tile_width : default_tile_width(*p);
        if (h->W == 0) return fail(SW_ERR_BAD_ARG);
        h->prob.tile_width = h->W;  // the form (Section 4.3) follows the width in use
        h->H = h->W / 2;
        h->M = p->n / h->W;
        h->S = h->M + 1;
        h->threads = swept_threads(h->W);
        int prc = SW_OK;
        if (p->scheme == SW_HEAT) {
            switch (p->precision) {
            case SW_FP64: h->nsnap = HeatPolicy<0>::NSNAP; h->smem = swept_smem<HeatPolicy<0>>(h->W);
                prc = prepare_swept_kernel<HeatPolicy<0>>(h->smem); break;
            case SW_FP32: h->nsnap = HeatPolicy<1>::NSNAP; h->smem = swept_smem<HeatPolicy<1>>(h->W);
                prc = prepare_swept_kernel<HeatPolicy<1>>(h->smem); break;
            default: h->nsnap = HeatPolicy<2>::NSNAP; h->smem = swept_smem<HeatPolicy<2>>(h->W);
                prc = prepare_swept_kernel<HeatPolicy<2>>(h->smem); break;
            }
        } else if (flattened(h->prob)) {
            switch (p->precision) {
            case SW_FP64: h->nsnap = EulerFlatPolicy<0>::NSNAP; h->smem = swept_smem<EulerFlatPolicy<0>>(h->W);
                prc = prepare_swept_kernel<EulerFlatPolicy<0>>(h->smem); break;
            case SW_FP32: h->nsnap = EulerFlatPolicy<1>::NSNAP; h->smem = swept_smem<EulerFlatPolicy<1>>(h->W);
                prc = prepare_swept_kernel<EulerFlatPolicy<1>>(h->smem); break;
            default: h->nsnap = EulerFlatPolicyComp::NSNAP; h->smem = swept_smem<EulerFlatPolicyComp>(h->W);
                prc = prepare_swept_kernel<EulerFlatPolicyComp>(h->smem); break;
            }
        } else {
            switch (p->precision) {
            case SW_FP64: h->nsnap = EulerPolicy<0>::NSNAP; h->smem = swept_smem<EulerPolicy<0>>(h->W);
                prc = prepare_swept_kernel<EulerPolicy<0>>(h->smem); break;
            case SW_FP32: h->nsnap = EulerPolicy<1>::NSNAP; h->smem = swept_smem<EulerPolicy<1>>(h->W);
                prc = prepare_swept_kernel<EulerPolicy<1>>(h->smem); break;
            default: h->nsnap = EulerPolicyComp::NSNAP; h->smem = swept_smem<EulerPolicyComp>(h->W);
                prc = prepare_swept_kernel<EulerPolicyComp>(h->smem); break;
            }
        }
        if (prc != SW_OK) return fail(prc);
        if (h->smem > 227 * 1024) return fail(SW_ERR_UNSUPPORTED);
        h->flank_bytes = size_t(h->nsnap) * size_t(h->S) * 2 * h->W * h->esize;
        for (int i = 0; i < 2; ++i) {
            e = cudaMalloc(&h->flank[i], h->flank_bytes + kGuardBytes);
            if (e == cudaSuccess)
                e = cudaMemset(static_cast<char *>(h->flank[i]) + h->flank_bytes, kGuardByte, kGuardBytes);
            if (e != cudaSuccess) return fail(cuda_status(e));
        }
    } else {
        if (p->scheme == SW_HEAT) h->scratch_bytes = size_t(h->nio) * p->n * h->esize;
        else h->scratch_bytes = size_t(4) * p->n * h->esize;  // Q* planes, ratio plane (lengthened form)
        e = cudaMalloc(&h->scratch, h->scratch_bytes + kGuardBytes);
        if (e == cudaSuccess)
            e = cudaMemset(static_cast<char *>(h->scratch) + h->scratch_bytes, kGuardByte, kGuardBytes);
        if (e != cudaSuccess) return fail(cuda_status(e));
    }
    e = cudaMalloc(&h->d_status, 4 * sizeof(int));
    if (e != cudaSuccess) return fail(cuda_status(e));
    e = cudaMemset(h->d_status, 0, 4 * sizeof(int));
    if (e != cudaSuccess) return fail(cuda_status(e));
    e = cudaMalloc(&h->d_partial, size_t(kRedBlocks) * 3 * sizeof(double));
    if (e != cudaSuccess) return fail(cuda_status(e));
    e = cudaMalloc(&h->d_sums, 4 * sizeof(double));
    if (e != cudaSuccess) return fail(cuda_status(e));
    *out = h;
    if (p->scheme == SW_HEAT && p->r > 0.5) return SW_WARN_UNSTABLE;
    return SW_OK;
}

void sw_destroy(sw_handle *h) {
    if (!h) return;
    cudaDeviceSynchronize();
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    cudaFree(h->flank[0]);
    cudaFree(h->flank[1]);
    cudaFree(h->scratch);
    cudaFree(h->dev_state);
    cudaFree(h->d_status);
    cudaFree(h->d_partial);
    cudaFree(h->d_sums);
    cudaFreeHost(h->h_flank[0]);
    cudaFreeHost(h->h_flank[1]);
    cudaFreeHost(h->h_state);
    for (cudaEvent_t e : h->hy_ev)
        if (e) cudaEventDestroy(e);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->gstream) cudaStreamDestroy(h->gstream);
    delete h->pool;
    delete h;
}

int32_t sw_tile_width(const sw_handle *h) { return h ? h->W : 0; }

int64_t sw_last_launch_count(const sw_handle *h) { return h ? h->last_launches : 0; }

int sw_set_timing(sw_handle *h, int64_t capacity) {
    if (!h || capacity < 0 || capacity > (int64_t(1) << 24)) return SW_ERR_BAD_ARG;
    while ((int64_t)h->events.size() < 2 * capacity) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return cuda_status(err);
        h->events.push_back(e);
    }
    h->kinds.assign((size_t)capacity, 0);
    h->ev_cap = capacity;
    h->ev_used = 0;
    return SW_OK;
}

int64_t sw_launch_times(sw_handle *h, float *ms, int32_t *kind, int64_t cap) {
    if (!h || cap < 0 || (cap > 0 && (!ms || !kind))) return SW_ERR_BAD_ARG;
    const int64_t cnt = std::min(cap, h->ev_used);
    for (int64_t i = 0; i < cnt; ++i) {
        cudaError_t e = cudaEventSynchronize(h->events[2 * i + 1]);
        if (e != cudaSuccess) return cuda_status(e);
        e = cudaEventElapsedTime(&ms[i], h->events[2 * i], h->events[2 * i + 1]);
        if (e != cudaSuccess) return cuda_status(e);
        kind[i] = h->kinds[i];
    }
    return cnt;
}

namespace {

// The launches of one run (swept phases or per-step launches), enqueued on `st`.
int run_direct(sw_handle *h, void *state, int64_t nsteps, cudaStream_t st) {
    const sw_problem &p = h->prob;
    if (p.method == SW_SWEPT) {
        const int64_t L = nsteps * (p.scheme == SW_HEAT ? 1 : 4);
        if (p.scheme == SW_HEAT) {
            switch (p.precision) {
            case SW_FP64: return launch_swept<HeatPolicy<0>>(h, state, L, st);
            case SW_FP32: return launch_swept<HeatPolicy<1>>(h, state, L, st);
            default: return launch_swept<HeatPolicy<2>>(h, state, L, st);
            }
        }
        if (flattened(p)) {
            const int64_t L2 = 2 * nsteps;  // two stages per step
            switch (p.precision) {
            case SW_FP64: return launch_swept<EulerFlatPolicy<0>>(h, state, L2, st);
            case SW_FP32: return launch_swept<EulerFlatPolicy<1>>(h, state, L2, st);
            default: return launch_swept<EulerFlatPolicyComp>(h, state, L2, st);
            }
        }
        switch (p.precision) {
        case SW_FP64: return launch_swept<EulerPolicy<0>>(h, state, L, st);
        case SW_FP32: return launch_swept<EulerPolicy<1>>(h, state, L, st);
        default: return launch_swept<EulerPolicyComp>(h, state, L, st);
        }
    }
    if (p.scheme == SW_HEAT) return launch_perstep_heat(h, state, nsteps, st);
    switch (p.precision) {
    case SW_FP64: return launch_perstep_euler_t<OpsD, false>(h, state, nsteps, st);
    case SW_FP32: return launch_perstep_euler_t<OpsF, false>(h, state, nsteps, st);
    default: return launch_perstep_euler_t<OpsF, true>(h, state, nsteps, st);
    }
}

// SW_FLAG_GRAPH: capture the run once on a private stream (tracing off), keep the
// instantiated graph for this (state, nsteps) pair, replay it on the caller's stream.
int run_graph(sw_handle *h, void *state, int64_t nsteps, cudaStream_t st) {
    if (!(h->gexec && h->g_state == state && h->g_steps == nsteps)) {
        cudaError_t e = cudaSuccess;
        if (!h->gstream) e = cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_status(e);
        if (h->gexec) {
            cudaGraphExecDestroy(h->gexec);
            h->gexec = nullptr;
        }
        const int64_t cap = h->ev_cap;
        h->ev_cap = 0;
        e = cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            h->ev_cap = cap;
            return cuda_status(e);
        }
        const int rc = run_direct(h, state, nsteps, h->gstream);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(h->gstream, &g);
        h->ev_cap = cap;
        if (rc != SW_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return rc != SW_OK ? rc : cuda_status(e);
        }
        e = cudaGraphInstantiate(&h->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            h->gexec = nullptr;
            return cuda_status(e);
        }
        h->g_state = state;
        h->g_steps = nsteps;
        h->g_launches = h->last_launches;
    }
    h->last_launches = h->g_launches;
    h->ev_used = 0;
    return cuda_status(cudaGraphLaunch(h->gexec, st));
}

}  // namespace

int sw_run(sw_handle *h, void *state, int64_t nsteps, void *stream) {
    if (!h || !state || nsteps < 0) return SW_ERR_BAD_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    h->last_launches = 0;
    h->ev_used = 0;
    if (nsteps == 0) return SW_OK;
    if (h->prob.flags & SW_FLAG_GRAPH) return run_graph(h, state, nsteps, st);
    return run_direct(h, state, nsteps, st);
}

int sw_hybrid_split(int64_t tiles, int32_t work_factor, int32_t cpu_threads, int64_t *gpu_tiles,
                    int64_t *tiles_per_thread) {
    if (tiles < 2 || work_factor < 1 || cpu_threads < 1 || cpu_threads > 4096) return SW_ERR_BAD_ARG;
    // Eq. 1: the GPU takes work_factor times the tiles of one host thread
    const int64_t per = tiles / (int64_t(work_factor) + cpu_threads);
    if (per < 1) return SW_ERR_BAD_ARG;
    const int64_t g = tiles - per * cpu_threads;
    if (gpu_tiles) *gpu_tiles = g;
    if (tiles_per_thread) *tiles_per_thread = per;
    return SW_OK;
}

int sw_run_hybrid(sw_handle *h, void *state, int64_t nsteps, int32_t work_factor, int32_t cpu_threads,
                  void *stream) {
    if (!h || !state || nsteps < 0) return SW_ERR_BAD_ARG;
    if (h->prob.method != SW_SWEPT || flattened(h->prob)) return SW_ERR_BAD_ARG;
    int64_t Mg = 0;
    int rc = sw_hybrid_split(h->M, work_factor, cpu_threads, &Mg, nullptr);
    if (rc != SW_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    h->last_launches = 0;
    h->ev_used = 0;
    if (nsteps == 0) return SW_OK;
    if (!h->h_state) {
        cudaError_t e = cudaHostAlloc(&h->h_flank[0], h->flank_bytes, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaHostAlloc(&h->h_flank[1], h->flank_bytes, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaHostAlloc(&h->h_state, size_t(h->nio) * h->prob.n * h->esize, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->hy_ev[0], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->hy_ev[1], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (!h->pool || h->pool->size() != cpu_threads) {
        delete h->pool;
        h->pool = new (std::nothrow) HostPool(cpu_threads);
        if (!h->pool) return SW_ERR_OOM;
    }
    Hybrid hy{Mg};
    const sw_problem &p = h->prob;
    const int64_t L = nsteps * (p.scheme == SW_HEAT ? 1 : 4);
    if (p.scheme == SW_HEAT) {
        switch (p.precision) {
        case SW_FP64: return launch_swept<HeatPolicy<0>>(h, state, L, st, &hy);
        case SW_FP32: return launch_swept<HeatPolicy<1>>(h, state, L, st, &hy);
        default: return launch_swept<HeatPolicy<2>>(h, state, L, st, &hy);
        }
    }
    switch (p.precision) {
    case SW_FP64: return launch_swept<EulerPolicy<0>>(h, state, L, st, &hy);
    case SW_FP32: return launch_swept<EulerPolicy<1>>(h, state, L, st, &hy);
    default: return launch_swept<EulerPolicyComp>(h, state, L, st, &hy);
    }
}

int sw_run_host(sw_handle *h, const void *state_in, void *state_out, int64_t nsteps, void *stream) {
    if (!h || !state_in || !state_out || nsteps < 0) return SW_ERR_BAD_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t bytes = size_t(h->nio) * h->prob.n * h->esize;
    if (!h->dev_state) {
        cudaError_t e = cudaMalloc(&h->dev_state, bytes);
        if (e != cudaSuccess) return cuda_status(e);
    }
    cudaError_t e = cudaMemcpyAsync(h->dev_state, state_in, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_status(e);
    int rc = sw_run(h, h->dev_state, nsteps, stream);
    if (rc != SW_OK) return rc;
    e = cudaMemcpyAsync(state_out, h->dev_state, bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_status(e);
    return cuda_status(cudaStreamSynchronize(st));
}

int sw_pack_fp64(const sw_problem *p, const double *src, void *dst, void *stream) {
    if (validate_problem(p) != SW_OK || !src || !dst) return SW_ERR_BAD_ARG;
    const int64_t count = int64_t(scheme_nv(*p)) * p->n;
    k_pack<<<grid_for(count, 256, 152 * 8), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(src, dst, count,
                                                                                               p->precision);
    return cuda_status(cudaGetLastError());
}

int sw_unpack_fp64(const sw_problem *p, const void *src, double *dst, void *stream) {
    if (validate_problem(p) != SW_OK || !src || !dst) return SW_ERR_BAD_ARG;
    const int64_t count = int64_t(scheme_nv(*p)) * p->n;
    k_unpack<<<grid_for(count, 256, 152 * 8), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(src, dst, count,
                                                                                                 p->precision);
    return cuda_status(cudaGetLastError());
}

int sw_conservation(sw_handle *h, const void *state, double *sums_host, void *stream) {
    if (!h || !state || !sums_host) return SW_ERR_BAD_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int nv = scheme_nv(h->prob);
    dim3 grid(kRedBlocks, nv);
    k_sum_partial<<<grid, kRedThreads, 0, st>>>(state, h->prob.n, nv, h->prob.precision, h->d_partial);
    k_sum_final<<<1, kRedThreads, 0, st>>>(h->d_partial, kRedBlocks, nv, h->d_sums);
    cudaError_t e = cudaMemcpyAsync(sums_host, h->d_sums, nv * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_status(e);
    return cuda_status(cudaStreamSynchronize(st));
}

int sw_check_physical(sw_handle *h, const void *state, int64_t *cell, void *stream) {
    if (!h || !state) return SW_ERR_BAD_ARG;
    if (h->prob.scheme != SW_EULER) return SW_ERR_BAD_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long *bad = reinterpret_cast<unsigned long long *>(h->d_partial);
    cudaError_t e = cudaMemsetAsync(bad, 0xff, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_status(e);
    k_check_physical<<<grid_for(h->prob.n, 256, 152 * 8), 256, 0, st>>>(state, h->prob.n, h->prob.precision,
                                                                          h->prob.gamma, bad);
    unsigned long long host = 0;
    e = cudaMemcpyAsync(&host, bad, sizeof(host), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    const bool ok = host == ~0ull;
    if (cell) *cell = ok ? -1 : (int64_t)host;
    if (!ok) {
        const int code = SW_ERR_NONPHYSICAL;
        cudaMemcpy(h->d_status, &code, sizeof(int), cudaMemcpyHostToDevice);
        return SW_ERR_NONPHYSICAL;
    }
    return SW_OK;
}

int sw_sync_status(sw_handle *h, void *stream) {
    if (!h) return SW_ERR_BAD_ARG;
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_status(e);
    int code = 0;
    e = cudaMemcpy(&code, h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    if (code != 0) cudaMemset(h->d_status, 0, sizeof(int));
    // guards after the scratch buffers
    void *bufs[3] = {h->flank[0], h->flank[1], h->scratch};
    const size_t ends[3] = {h->flank_bytes, h->flank_bytes, h->scratch_bytes};
    unsigned char g[kGuardBytes];
    for (int i = 0; i < 3; ++i) {
        if (!bufs[i]) continue;
        char *at = static_cast<char *>(bufs[i]) + ends[i];
        e = cudaMemcpy(g, at, kGuardBytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_status(e);
        for (size_t k = 0; k < kGuardBytes; ++k) {
            if (g[k] != kGuardByte) {
                cudaMemset(at, kGuardByte, kGuardBytes);
                if (code == 0) code = SW_ERR_CORRUPT;
                break;
            }
        }
    }
    return code;
}

int sw_debug_corrupt_guard(sw_handle *h, int32_t which) {
    if (!h || which < 0 || which > 2) return SW_ERR_BAD_ARG;
    void *buf = which < 2 ? h->flank[which] : h->scratch;
    if (!buf) return SW_ERR_BAD_ARG;
    const size_t end = which < 2 ? h->flank_bytes : h->scratch_bytes;
    return cuda_status(cudaMemset(static_cast<char *>(buf) + end + 17, 0x00, 1));
}

}  // extern "C"
