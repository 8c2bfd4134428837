// common.cuh -- rounding-controlled arithmetic and small helpers shared by the
// swept-phase and per-step kernels of libswept.so.
//
// Every floating-point operation of the schemes goes through these wrappers so
// that the compiler cannot contract a multiply and an add differently in two
// kernels: the swept and the per-step kernels then evaluate the same rounded
// sequence per cell and agree bitwise (Section 4.1: the swept rule uses the same
// numerical method as the classic decomposition).
#pragma once
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

// Functions that the GPU kernels and the host share of a hybrid run both evaluate.
#if defined(__CUDACC__)
#define SW_HD __host__ __device__ __forceinline__
#else
#define SW_HD inline
#endif

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

// Host counterparts of OpsD / OpsF, for the host cores' share of a hybrid run:
// the host's IEEE operations, with fma() where the device uses a fused
// multiply-add. The translation units that instantiate them are compiled without
// floating-point contraction, so each operation rounds exactly as its device
// counterpart and a host evaluation of the same template gives the same bits.
struct HostOpsD {
    using T = double;
    static inline T add(T a, T b) { return a + b; }
    static inline T sub(T a, T b) { return a - b; }
    static inline T mul(T a, T b) { return a * b; }
    static inline T div(T a, T b) { return a / b; }
    static inline T sqrt_(T a) { return std::sqrt(a); }
    static inline T fma_(T a, T b, T c) { return std::fma(a, b, c); }
    static inline T abs_(T a) { return std::fabs(a); }
};

struct HostOpsF {
    using T = float;
    static inline T add(T a, T b) { return a + b; }
    static inline T sub(T a, T b) { return a - b; }
    static inline T mul(T a, T b) { return a * b; }
    static inline T div(T a, T b) { return a / b; }
    static inline T sqrt_(T a) { return std::sqrt(a); }
    static inline T fma_(T a, T b, T c) { return std::fma(a, b, c); }
    static inline T abs_(T a) { return std::fabs(a); }
};

// Error-free transformations (Knuth's TwoSum; Dekker's Fast2Sum, valid when
// |a| >= |b| or a == 0), over an operation set O.
#pragma nv_exec_check_disable
template <class O>
SW_HD void two_sum_t(typename O::T a, typename O::T b, typename O::T &s, typename O::T &e) {
    s = O::add(a, b);
    const typename O::T bb = O::sub(s, a);
    const typename O::T aa = O::sub(s, bb);
    e = O::add(O::sub(a, aa), O::sub(b, bb));
}

#pragma nv_exec_check_disable
template <class O>
SW_HD void fast_two_sum_t(typename O::T a, typename O::T b, typename O::T &s, typename O::T &e) {
    s = O::add(a, b);
    e = O::sub(b, O::sub(s, a));
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) { two_sum_t<OpsF>(a, b, s, e); }
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    fast_two_sum_t<OpsF>(a, b, s, e);
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
