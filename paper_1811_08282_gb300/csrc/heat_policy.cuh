// heat_policy.cuh -- how the generic swept-phase driver stores a heat cell
// (FP64, FP32, FP32 hi/lo): row fields, snapshot fields, state planes, update.
#pragma once
#include "heat.cuh"

namespace sw {

// Storage policy for the swept driver. Row fields per position: two slots
// (levels alternate between them, the "two values per point" of Section 4.1);
// a snapshot (flank entry) is the value at one level.
template <int PREC> struct HeatPolicy;

template <> struct HeatPolicy<0> {  // FP64
    using T = double;
    using O = OpsD;
    static constexpr int NROW = 2, NSNAP = 1, NIO = 1;
    static constexpr bool INJECT_AHEAD = true;
    static constexpr int R = 1;  // stencil radius: windows change by R cells per level
    static constexpr bool TWO_PASS = false;
    static constexpr int NSCR = 0;
    static constexpr int MIN_BLOCKS = 4;  // launch bound: resident 512-thread blocks per SM
    using Params = HeatParams;
    static __device__ __forceinline__ void load_state(T *row, int rs, int s, const T *st, int64_t n, int64_t j) {
        row[s] = st[j];
    }
    static __device__ __forceinline__ void store_state(const T *row, int rs, int s, int64_t level, T *st,
                                                       int64_t n, int64_t j) {
        st[j] = row[(level & 1) * rs + s];
    }
    // snapshot field f (only 0) of cell s at `level`: the level's slot
    static __device__ __forceinline__ T get_field(const T *row, int rs, int s, int64_t level, int f) {
        return row[(level & 1) * rs + s];
    }
    static __device__ __forceinline__ void set_field(T *row, int rs, int s, int64_t level, int f, T v) {
        row[(level & 1) * rs + s] = v;
    }
    static __device__ __forceinline__ void step(const Params &p, T *row, int rs, int s, int64_t level, bool gl,
                                                bool gr) {
        const T *cur = row + (level & 1) * rs;
        T u = cur[s];
        T a = gl ? u : cur[s - 1];
        T b = gr ? u : cur[s + 1];
        row[((level + 1) & 1) * rs + s] = heat_update<O>(p.r, a, u, b);
    }
};

template <> struct HeatPolicy<1> {  // FP32
    using T = float;
    using O = OpsF;
    static constexpr int NROW = 2, NSNAP = 1, NIO = 1;
    static constexpr bool INJECT_AHEAD = true;
    static constexpr int R = 1;  // stencil radius: windows change by R cells per level
    static constexpr bool TWO_PASS = false;
    static constexpr int NSCR = 0;
    static constexpr int MIN_BLOCKS = 4;  // launch bound: resident 512-thread blocks per SM
    using Params = HeatParams;
    static __device__ __forceinline__ void load_state(T *row, int rs, int s, const T *st, int64_t n, int64_t j) {
        row[s] = st[j];
    }
    static __device__ __forceinline__ void store_state(const T *row, int rs, int s, int64_t level, T *st,
                                                       int64_t n, int64_t j) {
        st[j] = row[(level & 1) * rs + s];
    }
    // snapshot field f (only 0) of cell s at `level`: the level's slot
    static __device__ __forceinline__ T get_field(const T *row, int rs, int s, int64_t level, int f) {
        return row[(level & 1) * rs + s];
    }
    static __device__ __forceinline__ void set_field(T *row, int rs, int s, int64_t level, int f, T v) {
        row[(level & 1) * rs + s] = v;
    }
    static __device__ __forceinline__ void step(const Params &p, T *row, int rs, int s, int64_t level, bool gl,
                                                bool gr) {
        const T *cur = row + (level & 1) * rs;
        T u = cur[s];
        T a = gl ? u : cur[s - 1];
        T b = gr ? u : cur[s + 1];
        row[((level + 1) & 1) * rs + s] = heat_update<O>(p.rf, a, u, b);
    }
};

template <> struct HeatPolicy<2> {  // FP32 hi/lo compensated
    using T = float;
    static constexpr int NROW = 4, NSNAP = 2, NIO = 2;  // row: h0 l0 h1 l1; planes: hi, lo
    static constexpr bool INJECT_AHEAD = true;
    static constexpr int R = 1;  // stencil radius: windows change by R cells per level
    static constexpr bool TWO_PASS = false;
    static constexpr int NSCR = 0;
    static constexpr int MIN_BLOCKS = 3;  // launch bound: resident 512-thread blocks per SM
    using Params = HeatParams;
    static __device__ __forceinline__ void load_state(T *row, int rs, int s, const T *st, int64_t n, int64_t j) {
        row[s] = st[j];
        row[rs + s] = st[n + j];
    }
    static __device__ __forceinline__ void store_state(const T *row, int rs, int s, int64_t level, T *st,
                                                       int64_t n, int64_t j) {
        const int k = (int)(level & 1) * 2;
        st[j] = row[k * rs + s];
        st[n + j] = row[(k + 1) * rs + s];
    }
    // snapshot field f of cell s at `level`: 0 high part, 1 low part of the level's slot
    static __device__ __forceinline__ T get_field(const T *row, int rs, int s, int64_t level, int f) {
        return row[((int)(level & 1) * 2 + f) * rs + s];
    }
    static __device__ __forceinline__ void set_field(T *row, int rs, int s, int64_t level, int f, T v) {
        row[((int)(level & 1) * 2 + f) * rs + s] = v;
    }
    static __device__ __forceinline__ void step(const Params &p, T *row, int rs, int s, int64_t level, bool gl,
                                                bool gr) {
        const int k = (int)(level & 1) * 2;
        const T *h = row + k * rs;
        const T *l = row + (k + 1) * rs;
        HL u{h[s], l[s]};
        HL a = gl ? u : HL{h[s - 1], l[s - 1]};
        HL b = gr ? u : HL{h[s + 1], l[s + 1]};
        HL o = heat_update_comp(p.rf, p.rf_lo, a, u, b);
        const int kn = 2 - k;
        row[kn * rs + s] = o.h;
        row[(kn + 1) * rs + s] = o.l;
    }
};

}  // namespace sw
