// problem.h -- internal (not part of the C ABI): the one validation of an
// sw_problem and the rules that turn its fields into a run plan, shared by
// every entry point that takes a problem (sw_create, sw_run_noalloc, batches).
#pragma once
#include <cstdint>

#include "../../include/swept.h"

namespace sw {

// SW_OK or SW_ERR_BAD_ARG: the field rules of include/swept.h (scheme, precision,
// boundary, method, flags, 4 <= n <= 2^40, r / dt_dx / gamma ranges, and for a
// swept problem an explicit W: even, SW_MIN_TILE..SW_MAX_TILE, divides n with
// at least two tiles, W % 4 == 0 and W >= 8 when the flattened form is asked for).
int validate_problem(const sw_problem *p);

// The Euler data-structure form of Section 4.3 that a problem runs in, at base
// width W (ignored for per-step runs): flattened (two 5-point stages per step)
// or lengthened (four 3-point sub-steps). An explicit SW_FLAG_FLATTENED or
// SW_FLAG_LENGTHENED decides; otherwise per-step runs are flattened, a swept run
// with SW_FLAG_EULER_FOLD is lengthened (the register-resident kernel is built
// on it), and other swept runs are flattened whenever W allows radius-2 windows
// (W % 4 == 0, W >= 8), else lengthened. Every form gives the same bits; the
// default follows the measured speed (flattened is the faster swept form on
// GB300 in every precision). Heat: always false.
inline bool euler_flattened(const sw_problem &p, int W) {
    if (p.scheme != SW_EULER) return false;
    if (p.flags & SW_FLAG_FLATTENED) return true;
    if (p.flags & SW_FLAG_LENGTHENED) return false;
    if (p.method == SW_PERSTEP) return true;
    if (p.flags & SW_FLAG_EULER_FOLD) return false;
    return W % 4 == 0 && W >= 8;
}

// Default swept base width: the largest of 1024, 512, ..., 4 that divides n with
// at least two tiles (Section 6 recommends large blocks); an explicitly
// flattened Euler problem needs W >= 8. 0 when none fits.
inline int default_tile_width(const sw_problem &p) {
    const int floor = (p.scheme == SW_EULER && (p.flags & SW_FLAG_FLATTENED)) ? 8 : SW_MIN_TILE;
    for (int W = SW_MAX_TILE; W >= floor; W >>= 1)
        if (p.n % W == 0 && p.n >= 2 * (int64_t)W) return W;
    return 0;
}

}  // namespace sw
