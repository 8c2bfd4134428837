// common.cuh -- rounding-controlled arithmetic and small helpers shared by the
// swept-phase and per-step kernels of libswept.so.
//
// Every floating-point operation of the schemes goes through these wrappers so
// that the compiler cannot contract a multiply and an add differently in two
// kernels: the swept and the per-step kernels then evaluate the same rounded
// sequence per cell and agree bitwise (Section 4.1: the swept rule uses the same
// numerical method as the classic decomposition).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sw {

struct OpsD {
    using T = double;
    static __device__ __forceinline__ T add(T a, T b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ T sub(T a, T b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ T mul(T a, T b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ T div(T a, T b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ T sqrt_(T a) { return __dsqrt_rn(a); }
    static __device__ __forceinline__ T fma_(T a, T b, T c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ T abs_(T a) { return fabs(a); }
};

struct OpsF {
    using T = float;
    static __device__ __forceinline__ T add(T a, T b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ T sub(T a, T b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ T mul(T a, T b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ T div(T a, T b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ T sqrt_(T a) { return __fsqrt_rn(a); }
    static __device__ __forceinline__ T fma_(T a, T b, T c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ T abs_(T a) { return fabsf(a); }
};

// Error-free transformations (Knuth's TwoSum; Dekker's Fast2Sum, valid when
// |a| >= |b| or a == 0). Written with the non-contracting intrinsics above.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float aa = __fsub_rn(s, bb);
    e = __fadd_rn(__fsub_rn(a, aa), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// Global index wrap for periodic domains (|j| < 2n).
__device__ __forceinline__ int64_t wrap_index(int64_t j, int64_t n) {
    if (j < 0) return j + n;
    if (j >= n) return j - n;
    return j;
}

// Bounded spin budget for device-side waits (persistent kernels): ~1 s at 2 GHz.
constexpr long long kSpinBudgetCycles = 2000000000LL;

}  // namespace sw
