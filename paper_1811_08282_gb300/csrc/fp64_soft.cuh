// fp64_soft.cuh -- the FP64 FTCS update u' = fma(r, fma(-2, u, a + b), u)
// (Section 4.2) evaluated with 64-bit integer arithmetic, bit for bit as the
// three IEEE 754 operations round it (round to nearest even, each operation
// rounded once: IEEE 754-2008, 4.3.1 and 5.4.1).
//
// GB300 issues FP64 operations at about two per SM per clock, 1/32 of its
// integer rate, so an FP64 stencil leaves most issue slots idle. Cells updated
// through this routine run on the integer pipes beside cells on the FP64 pipe.
//
// The three neighbours of a smooth field are close in magnitude and of one sign,
// so the update works on magnitudes in one fixed-point frame tied to u's
// exponent eu: a value is an integer F times 2^(eu - 1079), in which u's
// significand is shifted left by 4 bits.
//   1. a + b is an exact integer sum; rounding it to 53 significant bits gives
//      RN(a + b) (the frame holds every bit of a and b whose exponents lie in
//      [eu - 4, eu + 4]).
//   2. s - 2u is again exact, and so is RN(s - 2u) = d while |d| < 2^53 frame
//      units, i.e. |d| < |u| / 8: a second difference that large leaves the path.
//   3. r*d is a small correction to u: in units of ulp(u) it is
//      k = r*d / ulp(u), an integer plus a fraction taken from the 128-bit
//      product of r's and d's significands. RN(u + r*d) is u's bit pattern plus
//      or minus round(k) as long as the result stays in u's binade (or lands
//      exactly on the next power of two), where the spacing is ulp(u); an exact
//      tie goes to the neighbour whose last bit is even.
// Anything else -- mixed signs, operands outside the exponent window, |d| >= |u|/8,
// a zero or subnormal u, a result leaving u's binade, r outside [2^-29, 2^3) -- clears
// `ok`, and the caller evaluates the update with the FP64 instructions
// (heat_update_fp64) instead.
#pragma once
#include <cstdint>
#include <cstring>

#include "common.cuh"
#include "heat.cuh"

namespace sw {
namespace soft64 {

constexpr uint64_t kSign = 0x8000000000000000ull;
constexpr uint64_t kFrac = 0x000FFFFFFFFFFFFFull;
constexpr uint64_t kHidden = 0x0010000000000000ull;

SW_HD uint64_t bits(double x) {
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    std::memcpy(&b, &x, 8);
    return b;
#endif
}

SW_HD double value(uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double x;
    std::memcpy(&x, &b, 8);
    return x;
#endif
}

// Leading zeros of a 32-bit word (32 for zero).
SW_HD int clz32(uint32_t x) {
#if defined(__CUDA_ARCH__)
    return __clz((int)x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}

// High 64 bits of the 128-bit product a*b.
SW_HD uint64_t mulhi(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// 64-bit shifts by a count below 32, as two 32-bit funnel shifts.
SW_HD uint64_t shl_small(uint64_t m, unsigned s) {
#if defined(__CUDA_ARCH__)
    const uint32_t lo = (uint32_t)m, hi = (uint32_t)(m >> 32);
    return ((uint64_t)__funnelshift_l(lo, hi, s) << 32) | (uint32_t)(lo << s);
#else
    return m << s;
#endif
}

SW_HD uint64_t shr_small(uint64_t m, unsigned s) {
#if defined(__CUDA_ARCH__)
    const uint32_t lo = (uint32_t)m, hi = (uint32_t)(m >> 32);
    return ((uint64_t)(hi >> s) << 32) | __funnelshift_r(lo, hi, s);
#else
    return m >> s;
#endif
}

// m in [2^53, 2^63 - 2^10) rounded to 53 significant bits, to nearest even. It
// has 1 to 10 bits below the 53rd significant one, all in the low word, so the
// leading-zero count of the high word gives the shift.
SW_HD uint64_t round53(uint64_t m) {
    const unsigned sh = (unsigned)(11 - clz32((uint32_t)(m >> 32)));
    const uint32_t lo = (uint32_t)m;
    const uint32_t bias = (1u << (sh - 1)) - 1u + ((lo >> sh) & 1u);  // ties to even
    return (m + bias) & ~(uint64_t)((1u << sh) - 1u);
}

// r unpacked once per launch.
struct HeatR {
    uint64_t m11;     // r's significand << 11
    uint64_t hm1;     // 2^(c0 - 1) - 1
    uint64_t lomask;  // m11 * x has a bit set below 2^64 iff x & lomask != 0
    unsigned c0;      // 1026 - (r's biased exponent): r*d / ulp(u) = m11 |F_d| / 2^(64 + c0)
    uint32_t neg;     // 1 if r < 0
    bool usable;      // r normal and c0 in [1, 31]: r in [2^-29, 2^3)
};

SW_HD HeatR make_heat_r(double r) {
    const uint64_t b = bits(r);
    const int er = (int)((b >> 52) & 0x7FF);
    HeatR h;
    h.m11 = ((b & kFrac) | kHidden) << 11;
    const int c0 = 1026 - er;
    h.usable = er != 0 && c0 >= 1 && c0 <= 31;
    h.c0 = h.usable ? (unsigned)c0 : 1u;
    h.hm1 = (1ull << (h.c0 - 1)) - 1u;
    // the product's low 64 bits vanish iff v2(m11) + v2(x) >= 64
    int v2 = 0;
    while (((h.m11 >> v2) & 1u) == 0) ++v2;
    h.lomask = (1ull << (64 - v2)) - 1u;
    h.neg = (uint32_t)(b >> 63);
    return h;
}

// Bits of fma(r, fma(-2, u, a + b), u) (each operation rounded to nearest even),
// from the bit patterns of a, u, b. Fast path: a, u, b of one sign, so the
// frame holds magnitudes and s - 2u carries d's sign relative to u's.
// `ok` false: the result is meaningless and the update must be evaluated with
// the FP64 instructions.
SW_HD uint64_t heat_update(const HeatR &r, uint64_t A, uint64_t U, uint64_t B, bool &ok) {
    const uint32_t ah = (uint32_t)(A >> 32), uh = (uint32_t)(U >> 32), bh = (uint32_t)(B >> 32);
    const int eu = (int)((uh >> 20) & 0x7FF);
    const int da = (int)((ah >> 20) & 0x7FF) - eu + 4;
    const int db = (int)((bh >> 20) & 0x7FF) - eu + 4;
    // one sign; u normal, far from overflow and underflow; a and b in
    // [2^(eu-1027), 2^(eu-1018)): every intermediate is a normal double, frame < 2^62
    ok = (((ah ^ uh) | (bh ^ uh)) >> 31) == 0 && (unsigned)(eu - 64) <= 1976u && (unsigned)da <= 8u &&
         (unsigned)db <= 8u;
    const uint64_t fa = shl_small((A & kFrac) | kHidden, (unsigned)da & 15u);
    const uint64_t fb = shl_small((B & kFrac) | kHidden, (unsigned)db & 15u);
    const uint64_t s = round53(fa + fb);                           // |RN(a + b)|, >= 2^53
    const int64_t dd = (int64_t)(s - (((U & kFrac) | kHidden) << 5));  // exact (s - 2u) / sign(u)
    const uint64_t dsg = (uint64_t)(dd >> 63);
    const uint64_t dm = ((uint64_t)dd ^ dsg) - dsg;                // |d|: exact below 2^53
    ok = ok && (dm >> 53) == 0;
    // k = r |d| / ulp(u) = (ph + pl 2^-64) / 2^c0
    const uint64_t ph = mulhi(r.m11, dm);
    const bool plo = (dm & r.lomask) != 0;
    // round to nearest; an exact tie (nothing below ph) goes to the k whose parity
    // is U's, so that U +- k is even
    const uint32_t kbit = (uint32_t)shr_small(ph, r.c0) & 1u;
    const uint64_t inc = plo ? 1u : ((kbit ^ (uint32_t)U) & 1u);
    const uint64_t k = shr_small(ph + r.hm1 + inc, r.c0);
    const uint64_t mu = U & kFrac;
    // |u + r d| >= |u| iff r d has u's sign: sign(r) xor sign(d / sign(u)) is 0
    const bool grow = ((uint32_t)dsg & 1u) == r.neg;
    ok = ok && (grow ? mu + k <= kHidden : k < mu);
    return grow ? U + k : U - k;
}

#if defined(__CUDACC__)
// The FP64-pipe evaluation of a cell that left the integer path's range. Kept
// out of line: the rare branch to it can then never become FP64 instructions
// issued (predicated off) on every cell.
static __device__ __noinline__ double heat_update_fp64(double r, double a, double u, double b) {
    return sw::heat_update<OpsD>(r, a, u, b);
}
#endif

}  // namespace soft64
}  // namespace sw
