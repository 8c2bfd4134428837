// fp64_soft2d.cuh -- the 2D five-point FTCS update
//   u' = fma(rx, fma(-2, u, a + b), fma(ry, fma(-2, u, d + e), u))
// (the 2D heat kernels' per-cell function) evaluated with 64-bit integer arithmetic, bit
// for bit as the six IEEE 754 operations round it (round to nearest even, each operation
// rounded once), on the frame and rounding pieces of fp64_soft.cuh's 1D update.
#pragma once
#include "fp64_soft.cuh"

namespace sw {
namespace soft64 {

// The 2D five-point update fma(rx, fma(-2, u, a + b), fma(ry, fma(-2, u, d + e), u)) on the
// integer pipes: two second differences formed in u's frame as heat_update forms d, then two
// rounded corrections in that frame. The inner one, RN(u + ry yd), must land strictly inside
// u's binade (so that the outer one keeps u's ulp); the outer one, RN(inner + rx xd), rounds
// an exact tie to the neighbour whose last bit is even relative to the inner result, and may
// land on the next power of two as heat_update's result may.

// (RN(p + q) - 2u) / sign(u) in u's frame, exact, for neighbours P, Q of U (bit patterns; uh and
// eu: U's high word and biased exponent). Clears `ok` for a neighbour of another sign or outside
// [2^(eu-1027), 2^(eu-1018)).
SW_HD int64_t frame_second_diff(uint64_t P, uint64_t Q, uint64_t U, uint32_t uh, int eu, bool &ok) {
    const uint32_t ph = (uint32_t)(P >> 32), qh = (uint32_t)(Q >> 32);
    const int dp = (int)((ph >> 20) & 0x7FF) - eu + 4;
    const int dq = (int)((qh >> 20) & 0x7FF) - eu + 4;
    ok = ok && (((ph ^ uh) | (qh ^ uh)) >> 31) == 0 && (unsigned)dp <= 8u && (unsigned)dq <= 8u;
    const uint64_t fp = shl_small((P & kFrac) | kHidden, (unsigned)dp & 15u);
    const uint64_t fq = shl_small((Q & kFrac) | kHidden, (unsigned)dq & 15u);
    return (int64_t)(round53(fp + fq) - (((U & kFrac) | kHidden) << 5));
}

// round(r |d| / ulp(u)) for |d| = dm frame units (dm < 2^53), to nearest; an exact tie goes to
// the k with the parity of `base`, so that base +- k is even
SW_HD uint64_t round_correction(const HeatR &r, uint64_t dm, uint64_t base) {
    const uint64_t ph = mulhi(r.m11, dm);
    const bool plo = (dm & r.lomask) != 0;
    const uint32_t kbit = (uint32_t)shr_small(ph, r.c0) & 1u;
    const uint64_t inc = plo ? 1u : ((kbit ^ (uint32_t)base) & 1u);
    return shr_small(ph + r.hm1 + inc, r.c0);
}

// Bits of the 2D update from the bit patterns of the x-neighbours A, B, the cell U and the
// y-neighbours D, E. `ok` false: the result is meaningless; evaluate with the FP64 instructions.
SW_HD uint64_t heat2d_update(const HeatR &rx, const HeatR &ry, uint64_t A, uint64_t B, uint64_t U, uint64_t D,
                             uint64_t E, bool &ok) {
    const uint32_t uh = (uint32_t)(U >> 32);
    const int eu = (int)((uh >> 20) & 0x7FF);
    ok = (unsigned)(eu - 64) <= 1976u && rx.usable && ry.usable;
    const int64_t ddy = frame_second_diff(D, E, U, uh, eu, ok);
    const int64_t ddx = frame_second_diff(A, B, U, uh, eu, ok);
    const uint64_t sy = (uint64_t)(ddy >> 63), sx = (uint64_t)(ddx >> 63);
    const uint64_t dmy = ((uint64_t)ddy ^ sy) - sy, dmx = ((uint64_t)ddx ^ sx) - sx;
    ok = ok && ((dmy | dmx) >> 53) == 0;
    // inner = RN(u + ry yd), strictly inside u's binade
    const uint64_t ky = round_correction(ry, dmy, U);
    const uint64_t mu = U & kFrac;
    const bool gy = ((uint32_t)sy & 1u) == ry.neg;
    ok = ok && (gy ? mu + ky < kHidden : ky < mu);
    const uint64_t I = gy ? U + ky : U - ky;
    // RN(inner + rx xd) in the same frame
    const uint64_t kx = round_correction(rx, dmx, I);
    const uint64_t mi = I & kFrac;
    const bool gx = ((uint32_t)sx & 1u) == rx.neg;
    ok = ok && (gx ? mi + kx <= kHidden : kx < mi);
    return gx ? I + kx : I - kx;
}

}  // namespace soft64
}  // namespace sw
