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

}  // namespace sw
