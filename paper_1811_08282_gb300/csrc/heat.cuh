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
#pragma nv_exec_check_disable
template <class O>
SW_HD typename O::T heat_update(typename O::T r, typename O::T a, typename O::T u, typename O::T b) {
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
// O: OpsF on the device, HostOpsF on the host.
#pragma nv_exec_check_disable
template <class O>
SW_HD HL heat_update_comp_t(float rh, float rl, HL a, HL u, HL b) {
    float d1, e1, d2, e2;
    two_sum_t<O>(a.h, -u.h, d1, e1);
    two_sum_t<O>(b.h, -u.h, d2, e2);
    const float low = O::add(O::add(e1, e2), O::fma_(-2.0f, u.l, O::add(a.l, b.l)));
    const float d = O::add(O::add(d1, d2), low);
    const float delta = O::fma_(rh, d, O::mul(rl, d));
    float s, e;
    two_sum_t<O>(u.h, delta, s, e);
    HL out;
    fast_two_sum_t<O>(s, O::add(u.l, e), out.h, out.l);
    return out;
}

__device__ __forceinline__ HL heat_update_comp(float rh, float rl, HL a, HL u, HL b) {
    return heat_update_comp_t<OpsF>(rh, rl, a, u, b);
}

struct HeatParams {
    double r;       // FP64 r
    float rf;       // r rounded to float
    float rf_lo;    // r - rf, rounded to float
};

}  // namespace sw
