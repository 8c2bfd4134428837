// batch.cu -- many independent 1D problems in one persistent launch (sw_batch_*),
// and the tile-width autotuner (sw_autotune).
//
// Work items are (phase, problem, chunk of structures) in phase-major order; CTAs
// take them from a device-side counter. An item of phase p waits (bounded spin)
// until the structures of phase p-1 it depends on -- its left and right
// neighbours, the same two as in Section 4.1's Communication step -- have
// published their phase, runs each structure with the same device code as the
// per-phase kernel (so results equal sw_run's bitwise), and publishes. Items only
// wait on items taken earlier, and a CTA only takes an item when it is running,
// so every wait ends. The launch (plus the reset of the counter and the flags)
// is captured once in a CUDA graph and replayed by every sw_batch_run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/swept.h"
#include "problem.h"
#include "euler.cuh"
#include "heat.cuh"
#include "heat_policy.cuh"
#include "swept_phase.cuh"

using namespace sw;

namespace {

constexpr int kBatchThreads = 128;  // default threads per CTA (sw_batch_set_threads: 64, 128 or 256)
constexpr int kChunk = 8;  // structures per work item

struct BatchDesc {
    int32_t scheme, periodic, W, flat;  // flat: Euler in the flattened form (Section 4.3)
    int64_t n, M, S, L, P_last;
    int64_t chunks_even, chunks_odd;  // work items per even / odd phase
    int64_t ep_tile, ep_seam;         // offsets of this problem's flags in the flag array
    HeatParams hp;
    EulerParams ep;
    void *state;
    void *flank[2];
};

struct BatchTables {
    const BatchDesc *desc;
    const int32_t *perm;       // problems sorted by number of phases, descending
    const int64_t *cum_even;   // prefix sums of chunks (sorted order), even phases
    const int64_t *cum_odd;    // same, odd phases
    const int32_t *active;     // problems that have phase p (a prefix of the sorted order)
    const int64_t *off;        // first item of phase p
    int64_t pmax;
    int64_t total;
    int *flags;                // per structure: phases completed
    unsigned long long *queue;
    int *status;               // [0] status, [1] abort
    long long budget;          // spin budget in clock cycles
    int drop_publish;          // failure-injection hook for tests: see sw_batch_debug
};

template <int PREC> struct EulerPolicyOf { using type = EulerPolicy<PREC>; };
template <> struct EulerPolicyOf<2> { using type = EulerPolicyComp; };
template <int PREC> struct EulerFlatOf { using type = EulerFlatPolicy<PREC>; };
template <> struct EulerFlatOf<2> { using type = EulerFlatPolicyComp; };

template <class T>
__device__ __forceinline__ PhaseArgs<T> batch_args(const BatchDesc &d, int64_t p) {
    PhaseArgs<T> a{};
    const int H = d.W / 2;
    const int HL = d.flat ? H / 2 : H;  // levels per phase half (radius-2 windows when flattened)
    a.n = d.n;
    a.W = d.W;
    a.H = H;
    a.periodic = d.periodic;
    a.p = (p == 0) ? 0 : (int)(2 - (p & 1));
    a.F = p * HL;
    a.lower = (p == 0) ? 0 : (int)min((int64_t)HL, d.L - (p - 1) * HL);
    a.upper = (p == d.P_last) ? 0 : (int)min((int64_t)(HL - 1), d.L - p * HL);
    a.write_lower = (p == d.P_last) ? 1 : 0;
    a.write_upper = (a.upper > 0 && p * HL + a.upper == d.L) ? 1 : 0;
    a.tiles = d.M;
    a.nstruct = (p & 1) ? (d.periodic ? d.M : d.M + 1) : d.M;
    a.nstruct_max = d.S;
    a.flank_in = (p == 0) ? nullptr : reinterpret_cast<const T *>(d.flank[(p - 1) & 1]);
    a.flank_out = reinterpret_cast<T *>(d.flank[p & 1]);
    a.state = reinterpret_cast<T *>(d.state);
    return a;
}

__device__ __forceinline__ int64_t upper_index(const int64_t *v, int64_t lo, int64_t hi, int64_t x) {
    // largest i in [lo, hi) with v[i] <= x (v non-decreasing, v[lo] <= x)
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (v[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// NT threads per CTA; the launch bound keeps the register budget per thread of the
// 128-thread form (64 registers in FP32, 128 in FP64) whatever NT is
template <int PREC, int NT>
__global__ void __launch_bounds__(NT, (PREC == 0 ? 4 : 8) * 128 / NT) k_batch(BatchTables t) {
    using HP = HeatPolicy<PREC>;
    using EP = typename EulerPolicyOf<PREC>::type;
    using EF = typename EulerFlatOf<PREC>::type;
    using T = typename HP::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);
    __shared__ long long s_item;
    __shared__ int s_go, s_q;
    __shared__ long long s_p, s_b0, s_b1;
    volatile int *abortp = t.status + 1;

    for (;;) {
        __syncthreads();  // the previous item is done with shared memory
        if (threadIdx.x == 0) {
            long long item = (long long)t.total;
            if (!*abortp) item = (long long)atomicAdd(t.queue, 1ull);
            s_item = item;
            if (item < t.total) {
                const int64_t p = upper_index(t.off, 0, t.pmax + 1, item);
                const int64_t k = item - t.off[p];
                const int64_t *cum = (p & 1) ? t.cum_odd : t.cum_even;
                const int64_t r = upper_index(cum, 0, t.active[p], k);
                const int q = t.perm[r];
                const BatchDesc &d = t.desc[q];
                const int64_t cnt = (p & 1) ? (d.periodic ? d.M : d.M + 1) : d.M;
                const int64_t b0 = (k - cum[r]) * kChunk;
                s_q = q;
                s_p = p;
                s_b0 = b0;
                s_b1 = min(b0 + kChunk, cnt);
            }
        }
        __syncthreads();
        if (s_item >= t.total) return;
        const int q = s_q;
        const int64_t p = s_p, b0 = s_b0, b1 = s_b1;
        const BatchDesc &d = t.desc[q];

        // wait for the phase p-1 structures this chunk reads (one thread per flag)
        if (threadIdx.x == 0) s_go = 1;
        __syncthreads();
        if (p >= 1) {
            int64_t lo, hi;  // neighbour structures of phase p-1, inclusive range
            int *fl;
            int64_t cnt_prev;
            if (p & 1) {  // seams b read tiles b-1 and b
                lo = b0 - 1;
                hi = b1 - 1;
                fl = t.flags + d.ep_tile;
                cnt_prev = d.M;
            } else {      // tiles b read seams b and b+1
                lo = b0;
                hi = b1;
                fl = t.flags + d.ep_seam;
                cnt_prev = d.periodic ? d.M : d.M + 1;
            }
            const int64_t j = lo + threadIdx.x;
            if (j <= hi) {
                int64_t s = j;
                bool exists = true;
                if (d.periodic) s = (s % cnt_prev + cnt_prev) % cnt_prev;
                else exists = s >= 0 && s < cnt_prev;
                if (exists) {
                    volatile int *f = fl + s;
                    const long long start = clock64();
                    while (*f < p) {
                        if (*abortp || clock64() - start > t.budget) {
                            if (!*abortp) {
                                atomicCAS(t.status, 0, SW_ERR_TIMEOUT);
                                atomicExch(t.status + 1, 1);
                            }
                            s_go = 0;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
            }
        }
        __syncthreads();
        if (!s_go) return;
        __threadfence();  // order the flank reads after the flags seen

        for (int64_t b = b0; b < b1; ++b) {
            if (d.scheme == SW_HEAT) {
                const PhaseArgs<T> a = batch_args<T>(d, p);
                swept_structure<HP, true>(a, d.hp, b, smem);
            } else if (d.flat) {
                const PhaseArgs<T> a = batch_args<T>(d, p);
                swept_structure<EF, true>(a, d.ep, b, smem);
            } else {
                const PhaseArgs<T> a = batch_args<T>(d, p);
                swept_structure<EP, true>(a, d.ep, b, smem);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();  // flanks and state visible before the flag
                int *fl = t.flags + ((p & 1) ? d.ep_seam : d.ep_tile);
                const bool drop = t.drop_publish && q == 0 && p == 0 && b == 0;
                if (!drop) atomicExch(fl + b, (int)(p + 1));
            }
        }
    }
}

int cuda_status_b(cudaError_t e) {
    if (e == cudaSuccess) return SW_OK;
    if (e == cudaErrorMemoryAllocation) return SW_ERR_OOM;
    return SW_ERR_CUDA;
}

size_t smem_for(int scheme, int prec, int W, bool flat) {
    if (flat) {
        if (prec == SW_FP64) return swept_smem_elems<EulerFlatPolicy<0>>(W) * 8;
        if (prec == SW_FP32) return swept_smem_elems<EulerFlatPolicy<1>>(W) * 4;
        return swept_smem_elems<EulerFlatPolicyComp>(W) * 4;
    }
    if (scheme == SW_HEAT) {
        if (prec == SW_FP64) return swept_smem_elems<HeatPolicy<0>>(W) * 8;
        if (prec == SW_FP32) return swept_smem_elems<HeatPolicy<1>>(W) * 4;
        return swept_smem_elems<HeatPolicy<2>>(W) * 4;
    }
    if (prec == SW_FP64) return swept_smem_elems<EulerPolicy<0>>(W) * 8;
    if (prec == SW_FP32) return swept_smem_elems<EulerPolicy<1>>(W) * 4;
    return swept_smem_elems<EulerPolicyComp>(W) * 4;
}

int nsnap_for(int scheme, int prec, bool flat) {
    if (flat) return prec == SW_FP32_COMP ? EulerFlatPolicyComp::NSNAP : EulerFlatPolicy<1>::NSNAP;
    if (scheme == SW_HEAT) return prec == SW_FP32_COMP ? 2 : 1;
    return prec == SW_FP32_COMP ? EulerPolicyComp::NSNAP : 7;
}

}  // namespace

struct sw_batch {
    int precision = 0;
    int threads = kBatchThreads;  // per CTA of the persistent kernel
    int32_t count = 0;
    int64_t nsteps = 0;
    std::vector<BatchDesc> desc;
    void *d_desc = nullptr, *d_tables = nullptr, *d_flags = nullptr, *d_queue = nullptr, *d_status = nullptr;
    std::vector<void *> flanks;
    BatchTables tab{};
    size_t flags_bytes = 0;
    size_t smem = 0;
    int grid = 0;
    cudaStream_t capture_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long budget = 2000000000LL;  // ~1 s at 2 GHz
    int drop_publish = 0;
};

namespace {

template <int PREC> const void *kernel_for_nt(int nt) {
    switch (nt) {
    case 64: return (const void *)k_batch<PREC, 64>;
    case 256: return (const void *)k_batch<PREC, 256>;
    default: return (const void *)k_batch<PREC, 128>;
    }
}

const void *batch_kernel(int prec, int nt) {
    return prec == SW_FP64 ? kernel_for_nt<0>(nt) : prec == SW_FP32 ? kernel_for_nt<1>(nt) : kernel_for_nt<2>(nt);
}

// The persistent grid for b->threads: every CTA the device can hold at once (items never
// wait on items taken later, so a smaller resident set is also safe), at most one per item.
cudaError_t configure_grid(sw_batch *b) {
    const void *fn = batch_kernel(b->precision, b->threads);
    cudaError_t e = cudaSuccess;
    if (b->smem > 48 * 1024) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, b->threads, b->smem);
    if (e != cudaSuccess) return e;
    b->grid = std::max(1, per_sm) * std::max(1, sms);
    if ((int64_t)b->grid > b->tab.total) b->grid = (int)std::max<int64_t>(b->tab.total, 1);
    return cudaSuccess;
}

template <int PREC> void launch_batch(const sw_batch *b, const BatchTables &t, cudaStream_t st) {
    switch (b->threads) {
    case 64: k_batch<PREC, 64><<<b->grid, 64, b->smem, st>>>(t); break;
    case 256: k_batch<PREC, 256><<<b->grid, 256, b->smem, st>>>(t); break;
    default: k_batch<PREC, 128><<<b->grid, 128, b->smem, st>>>(t); break;
    }
}

}  // namespace

extern "C" {

void sw_batch_destroy(sw_batch *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    for (void *f : b->flanks) cudaFree(f);
    cudaFree(b->d_desc);
    cudaFree(b->d_tables);
    cudaFree(b->d_flags);
    cudaFree(b->d_queue);
    cudaFree(b->d_status);
    delete b;
}

int sw_batch_create(const sw_problem *probs, void *const *states, int32_t count, int64_t nsteps,
                    sw_batch **out) {
    if (!probs || !states || !out || count <= 0 || nsteps < 0) return SW_ERR_BAD_ARG;
    const int prec = probs[0].precision;
    for (int32_t i = 0; i < count; ++i) {
        const sw_problem &p = probs[i];
        if (!states[i] || p.precision != prec || p.method != SW_SWEPT) return SW_ERR_BAD_ARG;
        // the rules of sw_create, an explicit width, and flags 0 or an Euler form (Section 4.3)
        if (validate_problem(&p) != SW_OK || p.tile_width == 0) return SW_ERR_BAD_ARG;
        if (p.flags & ~(SW_FLAG_LENGTHENED | SW_FLAG_FLATTENED)) return SW_ERR_BAD_ARG;
        if (p.scheme != SW_EULER && p.flags != 0) return SW_ERR_BAD_ARG;
    }
    sw_batch *b = new (std::nothrow) sw_batch();
    if (!b) return SW_ERR_OOM;
    b->precision = prec;
    b->count = count;
    b->nsteps = nsteps;
    auto fail = [&](int code) {
        sw_batch_destroy(b);
        return code;
    };
    cudaError_t e;
    const size_t es = prec == SW_FP64 ? 8 : 4;
    b->desc.resize(count);
    int64_t flag_total = 0, pmax = 0;
    for (int32_t i = 0; i < count; ++i) {
        const sw_problem &p = probs[i];
        BatchDesc &d = b->desc[i];
        std::memset(&d, 0, sizeof(d));
        d.scheme = p.scheme;
        d.periodic = p.boundary == SW_PERIODIC;
        d.W = p.tile_width;
        d.flat = euler_flattened(p, p.tile_width) ? 1 : 0;  // the form sw_run would take
        d.n = p.n;
        d.M = p.n / p.tile_width;
        d.S = d.M + 1;
        d.L = nsteps * (p.scheme == SW_HEAT ? 1 : (d.flat ? 2 : 4));
        const int64_t HL = d.flat ? d.W / 4 : d.W / 2;  // levels per phase half
        d.P_last = (d.L + HL - 1) / HL;
        d.chunks_even = (d.M + kChunk - 1) / kChunk;
        d.chunks_odd = ((d.periodic ? d.M : d.M + 1) + kChunk - 1) / kChunk;
        d.ep_tile = flag_total;
        d.ep_seam = flag_total + d.M;
        flag_total += 2 * d.M + 1;
        d.hp.r = p.r;
        d.hp.rf = (float)p.r;
        d.hp.rf_lo = (float)(p.r - (double)d.hp.rf);
        d.ep.gamma = p.gamma;
        d.ep.gm1 = p.gamma - 1.0;
        d.ep.lam = p.dt_dx;
        d.ep.hlam = 0.5 * p.dt_dx;
        d.ep.gammaf = (float)p.gamma;
        d.ep.gm1f = (float)(p.gamma - 1.0);
        d.ep.lamf = (float)p.dt_dx;
        d.ep.hlamf = (float)(0.5 * p.dt_dx);
        d.state = states[i];
        if (d.L > 0) {
            const size_t fb = size_t(nsnap_for(p.scheme, prec, d.flat)) * d.S * 2 * d.W * es;
            for (int k = 0; k < 2; ++k) {
                void *f = nullptr;
                e = cudaMalloc(&f, fb);
                if (e != cudaSuccess) return fail(cuda_status_b(e));
                b->flanks.push_back(f);
                d.flank[k] = f;
            }
        }
        pmax = std::max(pmax, d.L > 0 ? d.P_last : (int64_t)-1);
        b->smem = std::max(b->smem, smem_for(p.scheme, prec, d.W, d.flat));
    }
    if (b->smem > 227 * 1024) return fail(SW_ERR_UNSUPPORTED);
    // decode tables: problems sorted by phase count (descending); phase p holds a prefix
    std::vector<int32_t> perm(count);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int32_t x, int32_t y) {
        const int64_t px = b->desc[x].L > 0 ? b->desc[x].P_last : -1;
        const int64_t py = b->desc[y].L > 0 ? b->desc[y].P_last : -1;
        return px > py;
    });
    std::vector<int64_t> cum_even(count + 1, 0), cum_odd(count + 1, 0);
    for (int32_t r = 0; r < count; ++r) {
        cum_even[r + 1] = cum_even[r] + b->desc[perm[r]].chunks_even;
        cum_odd[r + 1] = cum_odd[r] + b->desc[perm[r]].chunks_odd;
    }
    const int64_t nphase = pmax + 1;  // 0 when nothing runs
    std::vector<int32_t> active(std::max<int64_t>(nphase, 1), 0);
    std::vector<int64_t> off(nphase + 1, 0);
    for (int64_t p = 0; p < nphase; ++p) {
        int32_t a = 0;
        while (a < count && b->desc[perm[a]].L > 0 && b->desc[perm[a]].P_last >= p) ++a;
        active[p] = a;
        off[p + 1] = off[p] + ((p & 1) ? cum_odd[a] : cum_even[a]);
    }
    const int64_t total = off[nphase];
    // one device block: desc | perm | cum_even | cum_odd | active | off
    const size_t sz_desc = sizeof(BatchDesc) * count;
    const size_t o_perm = (sz_desc + 255) / 256 * 256;
    const size_t o_ce = o_perm + (sizeof(int32_t) * count + 255) / 256 * 256;
    const size_t o_co = o_ce + (sizeof(int64_t) * (count + 1) + 255) / 256 * 256;
    const size_t o_act = o_co + (sizeof(int64_t) * (count + 1) + 255) / 256 * 256;
    const size_t o_off = o_act + (sizeof(int32_t) * active.size() + 255) / 256 * 256;
    const size_t tbytes = o_off + sizeof(int64_t) * off.size();
    std::vector<unsigned char> host(tbytes, 0);
    std::memcpy(host.data(), b->desc.data(), sz_desc);
    std::memcpy(host.data() + o_perm, perm.data(), sizeof(int32_t) * count);
    std::memcpy(host.data() + o_ce, cum_even.data(), sizeof(int64_t) * (count + 1));
    std::memcpy(host.data() + o_co, cum_odd.data(), sizeof(int64_t) * (count + 1));
    std::memcpy(host.data() + o_act, active.data(), sizeof(int32_t) * active.size());
    std::memcpy(host.data() + o_off, off.data(), sizeof(int64_t) * off.size());
    e = cudaMalloc(&b->d_tables, tbytes);
    if (e != cudaSuccess) return fail(cuda_status_b(e));
    e = cudaMemcpy(b->d_tables, host.data(), tbytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(cuda_status_b(e));
    b->flags_bytes = sizeof(int) * std::max<int64_t>(flag_total, 1);
    e = cudaMalloc(&b->d_flags, b->flags_bytes);
    if (e != cudaSuccess) return fail(cuda_status_b(e));
    e = cudaMalloc(&b->d_queue, sizeof(unsigned long long));
    if (e != cudaSuccess) return fail(cuda_status_b(e));
    e = cudaMalloc(&b->d_status, 2 * sizeof(int));
    if (e != cudaSuccess) return fail(cuda_status_b(e));
    e = cudaMemset(b->d_status, 0, 2 * sizeof(int));
    if (e != cudaSuccess) return fail(cuda_status_b(e));
    unsigned char *tb = reinterpret_cast<unsigned char *>(b->d_tables);
    b->tab.desc = reinterpret_cast<const BatchDesc *>(tb);
    b->tab.perm = reinterpret_cast<const int32_t *>(tb + o_perm);
    b->tab.cum_even = reinterpret_cast<const int64_t *>(tb + o_ce);
    b->tab.cum_odd = reinterpret_cast<const int64_t *>(tb + o_co);
    b->tab.active = reinterpret_cast<const int32_t *>(tb + o_act);
    b->tab.off = reinterpret_cast<const int64_t *>(tb + o_off);
    b->tab.pmax = std::max<int64_t>(nphase - 1, 0);
    b->tab.total = total;
    b->tab.flags = reinterpret_cast<int *>(b->d_flags);
    b->tab.queue = reinterpret_cast<unsigned long long *>(b->d_queue);
    b->tab.status = reinterpret_cast<int *>(b->d_status);
    e = configure_grid(b);
    if (e != cudaSuccess) return fail(cuda_status_b(e));
    e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(cuda_status_b(e));
    *out = b;
    return SW_OK;
}

int sw_batch_debug(sw_batch *b, int64_t wait_budget_cycles, int32_t drop_publish) {
    if (!b || wait_budget_cycles <= 0) return SW_ERR_BAD_ARG;
    b->budget = wait_budget_cycles;
    b->drop_publish = drop_publish ? 1 : 0;
    if (b->exec) {  // parameters are baked into the graph: rebuild it on the next run
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
    }
    return SW_OK;
}

static cudaError_t batch_enqueue(sw_batch *b, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(b->d_flags, 0, b->flags_bytes, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b->d_status, 0, 2 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (b->tab.total == 0) return cudaSuccess;
    BatchTables t = b->tab;
    t.budget = b->budget;
    t.drop_publish = b->drop_publish;
    if (b->precision == SW_FP64) launch_batch<0>(b, t, st);
    else if (b->precision == SW_FP32) launch_batch<1>(b, t, st);
    else launch_batch<2>(b, t, st);
    return cudaGetLastError();
}

int sw_batch_run(sw_batch *b, void *stream) {
    if (!b) return SW_ERR_BAD_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (!b->exec) {
        e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_status_b(e);
        cudaError_t ee = batch_enqueue(b, b->capture_stream);
        e = cudaStreamEndCapture(b->capture_stream, &b->graph);
        if (ee != cudaSuccess) return cuda_status_b(ee);
        if (e != cudaSuccess) return cuda_status_b(e);
        e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) return cuda_status_b(e);
    }
    return cuda_status_b(cudaGraphLaunch(b->exec, st));
}

int sw_batch_status(sw_batch *b, void *stream) {
    if (!b) return SW_ERR_BAD_ARG;
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_status_b(e);
    int st[2] = {0, 0};
    e = cudaMemcpy(st, b->d_status, sizeof(st), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status_b(e);
    return st[0];
}

int64_t sw_batch_items(const sw_batch *b) { return b ? b->tab.total : 0; }

int sw_batch_set_threads(sw_batch *b, int32_t threads) {
    if (!b || (threads != 64 && threads != 128 && threads != 256)) return SW_ERR_BAD_ARG;
    cudaError_t e = cudaDeviceSynchronize();  // no launch of the old configuration in flight
    if (e != cudaSuccess) return cuda_status_b(e);
    b->threads = threads;
    e = configure_grid(b);
    if (e != cudaSuccess) return cuda_status_b(e);
    if (b->exec) {  // the launch configuration is baked into the graph: capture it again
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
    }
    return SW_OK;
}

int sw_autotune(sw_problem *inout, int64_t probe_steps, void *stream) {
    if (!inout || probe_steps <= 0) return SW_ERR_BAD_ARG;
    sw_problem p = *inout;
    p.method = SW_SWEPT;
    p.tile_width = 0;
    if (sw_state_planes(&p) < 0) return SW_ERR_BAD_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t bytes = sw_state_bytes(&p);
    void *state = nullptr;
    cudaError_t e = cudaMalloc(&state, (size_t)bytes);
    if (e != cudaSuccess) return cuda_status_b(e);
    // the probe state (the kernels' cost depends on the data): heat 1.5 + sin of 8 waves, smooth
    // and of one sign, so that the FP64 integer-pipe path takes the cells it takes on smooth
    // fields (a zero state would send every one of them to the FP64 pipe); Euler a uniform state
    // at rest, (rho, m, E) = (1, 0, 2.5), stable at any dt/dx a caller may give
    {
        const int64_t nv = p.scheme == SW_HEAT ? 1 : 3;
        std::vector<double> h((size_t)(nv * p.n), 0.0);
        const double k = 2.0 * 3.14159265358979323846 * 8.0 / (double)p.n;
        for (int64_t i = 0; i < p.n; ++i) {
            if (p.scheme == SW_HEAT) {
                h[(size_t)i] = 1.5 + std::sin(k * (double)i);
            } else {
                h[(size_t)i] = 1.0;
                h[(size_t)(2 * p.n + i)] = 2.5;
            }
        }
        double *d64 = nullptr;
        e = cudaMalloc(&d64, sizeof(double) * h.size());
        if (e != cudaSuccess) {
            cudaFree(state);
            return cuda_status_b(e);
        }
        cudaMemcpy(d64, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice);
        sw_pack_fp64(&p, d64, state, stream);
        cudaStreamSynchronize(st);
        cudaFree(d64);
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best_w = 0, best_form = 0;
    float best_t = 0.f;
    // Euler without an explicit form: both data-structure forms of Section 4.3 are timed
    const bool both_forms = p.scheme == SW_EULER && !(p.flags & (SW_FLAG_LENGTHENED | SW_FLAG_FLATTENED));
    for (int W = SW_MIN_TILE; W <= SW_MAX_TILE; W *= 2) {
        if (W < 32 || p.n % W || p.n < 2 * (int64_t)W) continue;
        for (int k = 0; k < (both_forms ? 2 : 1); ++k) {
            sw_problem q = p;
            q.tile_width = W;
            if (both_forms) q.flags |= (k == 0 ? SW_FLAG_LENGTHENED : SW_FLAG_FLATTENED);
            sw_handle *h = nullptr;
            if (sw_create(&q, &h) < 0) continue;
            sw_run(h, state, probe_steps, stream);  // warm-up
            cudaEventRecord(e0, st);
            sw_run(h, state, probe_steps, stream);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            sw_destroy(h);
            if (best_w == 0 || ms < best_t) {
                best_w = W;
                best_t = ms;
                best_form = both_forms ? (k == 0 ? SW_FLAG_LENGTHENED : SW_FLAG_FLATTENED) : 0;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(state);
    if (best_w == 0) return SW_ERR_UNSUPPORTED;
    inout->tile_width = best_w;
    inout->flags |= best_form;
    return SW_OK;
}

}  // extern "C"
