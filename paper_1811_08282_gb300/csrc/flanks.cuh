// flanks.cuh -- layout of the flank buffers that carry the Communication step of
// the swept rule (Section 4.1, Fig. 1b/1d) between phases: for every structure
// of a phase, the two outermost cells on each side at each of its upper levels.
#pragma once
#include <cstdint>

#include "common.cuh"

namespace sw {

// Flank buffer element ((f * S + b) * 2 + side) * W + (2*j + k):
// field f, structure b, side 0 = left / 1 = right, level offset j, cell k of the pair.
template <class T>
SW_HD int64_t flank_off(int64_t S, int W, int f, int64_t b, int side) {
    return ((f * S + b) * 2 + side) * (int64_t)W;
}

}  // namespace sw
