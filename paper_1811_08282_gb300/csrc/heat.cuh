// heat.cuh -- FTCS heat equation (Section 4.2): the per-cell update in FP64,
// FP32 and FP32 hi/lo, and the storage policies the swept-phase driver uses.
//
// u' = u + r((u_{j-1} + u_{j+1}) - 2u), evaluated as fma(r, fma(-2, u, a + b), u)
// (FP64, FP32) and as a hi/lo pair with an error-free state update (FP32_COMP).
#pragma once
#include "common.cuh"

namespace sw {

// ============================================================================
// Heat
// ============================================================================
template <class O>
__device__ __forceinline__ typename O::T heat_update(typename O::T r, typename O::T a,
                                                     typename O::T u, typename O::T b) {
    using T = typename O::T;
    return O::fma_(r, O::fma_(T(-2), u, O::add(a, b)), u);
}

struct HL {
    float h, l;
};

// Compensated FTCS update of u = u.h + u.l (FP32 pair): the second difference is
// formed from exactly-split differences of the high parts plus the low parts,
// scaled by r = rh + rl, and added to the state with TwoSum so that increments
// far below half an ulp of u are kept in the low part instead of rounding away.
__device__ __forceinline__ HL heat_update_comp(float rh, float rl, HL a, HL u, HL b) {
    float d1, e1, d2, e2;
    two_sum(a.h, -u.h, d1, e1);
    two_sum(b.h, -u.h, d2, e2);
    float low = __fadd_rn(__fadd_rn(e1, e2), __fmaf_rn(-2.0f, u.l, __fadd_rn(a.l, b.l)));
    float d = __fadd_rn(__fadd_rn(d1, d2), low);
    float delta = __fmaf_rn(rh, d, __fmul_rn(rl, d));
    float s, e;
    two_sum(u.h, delta, s, e);
    HL out;
    fast_two_sum(s, __fadd_rn(u.l, e), out.h, out.l);
    return out;
}

struct HeatParams {
    double r;       // FP64 r
    float rf;       // r rounded to float
    float rf_lo;    // r - rf, rounded to float
};

// Storage policy for the swept driver. Row fields per position: two slots
// (levels alternate between them, the "two values per point" of Section 4.1);
// a snapshot (flank entry) is the value at one level.
template <int PREC> struct HeatPolicy;

template <> struct HeatPolicy<0> {  // FP64
    using T = double;
    using O = OpsD;
    static constexpr int NROW = 2, NSNAP = 1, NIO = 1;
    static constexpr bool INJECT_AHEAD = true;
    static constexpr bool TWO_PASS = false;
    static constexpr int NSCR = 0;
    using Params = HeatParams;
    static __device__ __forceinline__ void load_state(T *row, int rs, int s, const T *st, int64_t n, int64_t j) {
        row[s] = st[j];
    }
    static __device__ __forceinline__ void store_state(const T *row, int rs, int s, int64_t level, T *st,
                                                       int64_t n, int64_t j) {
        st[j] = row[(level & 1) * rs + s];
    }
    static __device__ __forceinline__ void snap_out(const T *row, int rs, int s, int64_t level, T *stg, int ss,
                                                    int e) {
        stg[e] = row[(level & 1) * rs + s];
    }
    static __device__ __forceinline__ void snap_in(T *row, int rs, int s, int64_t level, const T *stg, int ss,
                                                   int e) {
        row[(level & 1) * rs + s] = stg[e];
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
    static constexpr bool TWO_PASS = false;
    static constexpr int NSCR = 0;
    using Params = HeatParams;
    static __device__ __forceinline__ void load_state(T *row, int rs, int s, const T *st, int64_t n, int64_t j) {
        row[s] = st[j];
    }
    static __device__ __forceinline__ void store_state(const T *row, int rs, int s, int64_t level, T *st,
                                                       int64_t n, int64_t j) {
        st[j] = row[(level & 1) * rs + s];
    }
    static __device__ __forceinline__ void snap_out(const T *row, int rs, int s, int64_t level, T *stg, int ss,
                                                    int e) {
        stg[e] = row[(level & 1) * rs + s];
    }
    static __device__ __forceinline__ void snap_in(T *row, int rs, int s, int64_t level, const T *stg, int ss,
                                                   int e) {
        row[(level & 1) * rs + s] = stg[e];
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
    static constexpr bool TWO_PASS = false;
    static constexpr int NSCR = 0;
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
    static __device__ __forceinline__ void snap_out(const T *row, int rs, int s, int64_t level, T *stg, int ss,
                                                    int e) {
        const int k = (int)(level & 1) * 2;
        stg[e] = row[k * rs + s];
        stg[ss + e] = row[(k + 1) * rs + s];
    }
    static __device__ __forceinline__ void snap_in(T *row, int rs, int s, int64_t level, const T *stg, int ss,
                                                   int e) {
        const int k = (int)(level & 1) * 2;
        row[k * rs + s] = stg[e];
        row[(k + 1) * rs + s] = stg[ss + e];
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
