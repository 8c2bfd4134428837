// fold_heat.cuh -- register-resident Diamond phase for the heat equation
// (Section 4.1, Fig. 1c), periodic grids, complete diamonds only.
//
// One warp owns a chain of consecutive diamonds of one phase. A diamond's
// lower half widens (2, 4, ..., W cells per level) and its upper half narrows
// (W-2, ..., 2): on its own it keeps half the lanes idle. Here the warp runs
// the upper half of diamond k and the lower half of diamond k+1 on the same
// levels: with diamond k+1's window shifted by W/2 around the warp, the two
// active regions are exact complements, so every lane updates a live cell on
// every level. The W cells of the folded window live in registers, K = W/32
// per lane; neighbours cross lanes by shuffle (cyclically), and the only cells
// that differ from a plain cyclic FTCS update are the four next to the seam
// between the two diamonds, whose outer inputs come from the previous phase's
// flanks: those inputs are swapped in by a select on the owner lane before the
// one update every cell gets. The level loop is unrolled by K so that every
// such cell is a compile-time register slot; its owner lane is computed at
// run time.
//
// Flanks are read and written in the same global layout as k_swept_phase, so
// the two kernels mix freely within one run (the generic kernel does the Up
// and Down triangles and any truncated phase), and the per-cell update is the
// same function, so results are bitwise identical.
//
// FP64: every other register slot evaluates the update with integer arithmetic
// (fp64_soft.cuh, the same bits), so that the FP64 pipe -- two operations per SM
// per clock on GB300 -- and the integer pipes each carry half the cells.
#pragma once
#include "flanks.cuh"
#include "fp64_soft.cuh"
#include "heat.cuh"

namespace sw {

// Cell policies: value type, update and warp shuffle.
// SOFT_EVERY = s > 0: register slot j with j % s == s - 1 is updated on the integer
// pipes (soft64::heat_update) instead of the FP64 pipe, with the same bits.
struct FoldF32 {
    using T = float;
    using V = float;
    static constexpr int NSNAP = 1;
    static constexpr int SOFT_EVERY = 0;
    static __device__ __forceinline__ V upd(const HeatParams &p, V a, V u, V b) {
        return heat_update<OpsF>(p.rf, a, u, b);
    }
    static __device__ __forceinline__ V shfl(V x, int src) { return __shfl_sync(0xffffffffu, x, src); }
    static __device__ __forceinline__ V zero() { return 0.f; }
    static __device__ __forceinline__ V idle() { return 0.f; }
    static __device__ __forceinline__ V load(const T *p, int64_t plane, int64_t i) { return p[i]; }
    static __device__ __forceinline__ void store(T *p, int64_t plane, int64_t i, V x) { p[i] = x; }
    // entries i, i + 1 (i even) in one 8-byte store
    static __device__ __forceinline__ void store2(T *p, int64_t plane, int64_t i, V x, V y) {
        *reinterpret_cast<float2 *>(p + i) = make_float2(x, y);
    }
};

struct FoldF64 {
    using T = double;
    using V = double;
    static constexpr int NSNAP = 1;
    static constexpr int SOFT_EVERY = 2;  // half the cells on the integer pipes
    static __device__ __forceinline__ V upd(const HeatParams &p, V a, V u, V b) {
        return heat_update<OpsD>(p.r, a, u, b);
    }
    static __device__ __forceinline__ V upd_soft(const soft64::HeatR &h, V a, V u, V b, bool &ok) {
        return soft64::value(soft64::heat_update(h, soft64::bits(a), soft64::bits(u), soft64::bits(b), ok));
    }
    static __device__ __forceinline__ V shfl(V x, int src) { return __shfl_sync(0xffffffffu, x, src); }
    static __device__ __forceinline__ V zero() { return 0.0; }
    // register cells outside the live region are updated and never read; 1.0 keeps
    // them on the integer path (a zero would send the warp to the FP64 fallback)
    static __device__ __forceinline__ V idle() { return 1.0; }
    static __device__ __forceinline__ V load(const T *p, int64_t plane, int64_t i) { return p[i]; }
    static __device__ __forceinline__ void store(T *p, int64_t plane, int64_t i, V x) { p[i] = x; }
    // entries i, i + 1 (i even) in one 16-byte store
    static __device__ __forceinline__ void store2(T *p, int64_t plane, int64_t i, V x, V y) {
        *reinterpret_cast<double2 *>(p + i) = make_double2(x, y);
    }
};

struct FoldComp {
    using T = float;
    using V = HL;
    static constexpr int NSNAP = 2;  // flank planes: high parts, low parts
    static constexpr int SOFT_EVERY = 0;
    static __device__ __forceinline__ V upd(const HeatParams &p, V a, V u, V b) {
        return heat_update_comp(p.rf, p.rf_lo, a, u, b);
    }
    static __device__ __forceinline__ V shfl(V x, int src) {
        return HL{__shfl_sync(0xffffffffu, x.h, src), __shfl_sync(0xffffffffu, x.l, src)};
    }
    static __device__ __forceinline__ V zero() { return HL{0.f, 0.f}; }
    static __device__ __forceinline__ V idle() { return HL{0.f, 0.f}; }
    static __device__ __forceinline__ V load(const T *p, int64_t plane, int64_t i) {
        return HL{p[i], p[plane + i]};
    }
    static __device__ __forceinline__ void store(T *p, int64_t plane, int64_t i, V x) {
        p[i] = x.h;
        p[plane + i] = x.l;
    }
    // entries i, i + 1 (i even) of both planes, one 8-byte store each
    static __device__ __forceinline__ void store2(T *p, int64_t plane, int64_t i, V x, V y) {
        *reinterpret_cast<float2 *>(p + i) = make_float2(x.h, y.h);
        *reinterpret_cast<float2 *>(p + plane + i) = make_float2(x.l, y.l);
    }
};

template <class T> struct FoldArgs {
    int p;                // 0: Up Triangle; 1: seam-centred phase (odd); 2: tile-centred (even)
    int64_t n;            // cells
    int64_t tiles;        // M (periodic: structures per phase)
    int64_t nstruct;      // structures run by this launch: 0 .. nstruct-1 (M, or fewer in a hybrid run)
    int64_t nstruct_max;  // structures per flank buffer (flank layout of k_swept_phase)
    int lower, upper;     // levels of the lower / upper halves in this phase
    int write_lower;      // Down Triangle: the lower half ends at the run's last level; store its row
    int write_upper;      // must be 0 (a truncated upper half runs on the generic phase kernel)
    const T *flank_in;
    T *flank_out;
    T *state;             // state planes (FoldComp: high plane, then low plane)
};

// Store the cells of one structure that the folded window holds at z in [zlo, zhi]
// (zlo may be negative: the range wraps), z = window position in the frame of the
// structure, y = (z + yoff) mod W its cell relative to the window start `start`.
template <int K, class C>
__device__ __forceinline__ void fold_store_row(const typename C::V (&v)[K], int lane, int shift, int zlo, int zhi,
                                               int yoff, int64_t start, int64_t n, typename C::T *state) {
    constexpr int W = 32 * K;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int x = lane * K + j;
        int z = x - shift * K;
        if (z < 0) z += W;
        const bool in = (zlo >= 0) ? (z >= zlo && z <= zhi) : (z >= zlo + W || z <= zhi);
        if (in) {
            int y = z + yoff;
            if (y >= W) y -= W;
            int64_t cell = start + y;
            cell %= n;
            if (cell < 0) cell += n;
            C::store(state, n, cell, v[j]);
        }
    }
}

template <int K, class C>
__global__ void __launch_bounds__(128) k_heat_fold(FoldArgs<typename C::T> a, HeatParams prm) {
    using T = typename C::T;
    using V = typename C::V;
    constexpr int W = 32 * K, H = W / 2;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t M = a.tiles, NS = a.nstruct;
    const int64_t b0 = gw * NS / nw, b1 = (gw + 1) * NS / nw;
    if (b0 >= b1) return;  // whole warp
    const int64_t S = a.nstruct_max;
    const int64_t plane = S * 2 * (int64_t)W;  // flank field stride (FoldComp: low parts)
    const bool up = a.p == 0;
    const int imax = up ? a.upper : (a.lower > a.upper ? a.lower : a.upper);

    // integer-pipe slots for K = 4 .. 8 (beyond, the extra registers spill; at K = 2, W = 64,
    // the grids that choose it are small and latency-bound, where the integer path's long
    // dependent chain costs more than the FP64 pipe it frees: 1.17 against 0.80 ms for
    // N = 16384 x 1000 steps): r unpacked once (an r outside its range fails every soft
    // update, which then runs on the FP64 pipe)
    constexpr int SOFT = (K >= 4 && K <= 8) ? C::SOFT_EVERY : 0;
    soft64::HeatR hr{};
    if constexpr (SOFT > 0) hr = soft64::make_heat_r(prm.r);
    V v[K];
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = C::idle();
    int shift = 0;  // lanes by which the finishing diamond's frame is rotated (0 or 16)

    // Up Triangle: no pairing (two full rows cannot share the window); the iteration
    // t finishes structure t-1's upper half after loading its row. Diamonds and the
    // Down Triangle: iteration t runs structure t-1's upper half with structure t's
    // lower half.
    for (int64_t t = 0; t <= b1 - b0; ++t) {
        const bool hasL = !up && t < b1 - b0 && a.lower > 0;
        const bool hasU = (up ? t < b1 - b0 : t > 0) && a.upper > 0;
        const int64_t bL = b0 + t, bU = up ? bL : bL - 1;
        if (up && !(t < b1 - b0)) break;
        int64_t lb, rb;
        if (a.p & 1) {
            lb = (bL - 1 + M) % M;
            rb = bL % M;
        } else {
            lb = bL % M;
            rb = (bL + 1) % M;
        }
        const T *srcL = a.flank_in + flank_off<T>(S, W, 0, hasL ? lb : 0, 1);  // left neighbour's right flank
        const T *srcR = a.flank_in + flank_off<T>(S, W, 0, hasL ? rb : 0, 0);  // right neighbour's left flank
        T *dU0 = a.flank_out + flank_off<T>(S, W, 0, bU < 0 ? 0 : bU, 0);
        T *dU1 = a.flank_out + flank_off<T>(S, W, 0, bU < 0 ? 0 : bU, 1);
        T *dL0 = a.flank_out + flank_off<T>(S, W, 0, bL % S, 0);
        T *dL1 = a.flank_out + flank_off<T>(S, W, 0, bL % S, 1);
        // window start (cell of relative position 0) of the starting structure
        const int64_t startL = (a.p & 1) ? bL * W - H : bL * W;

        if (up) {
            // the initial row of tile bU, relative cell y at window position z = y (shift 0)
            const int64_t base = bU * W + (int64_t)lane * K;
#pragma unroll
            for (int j = 0; j < K; ++j) v[j] = C::load(a.state, a.n, base + j);
            if (lane == 0) {
                C::store(dU0, plane, 0, v[0]);
                C::store(dU0, plane, 1, v[1]);
            }
            if (lane == 31) {
                C::store(dU1, plane, 0, v[K - 2]);
                C::store(dU1, plane, 1, v[K - 1]);
            }
        }

        // flank entries 2(i-1)+k arrive in chunks of 32 (16 levels), one per lane, double-buffered
        V cL = C::zero(), cR = C::zero(), nL = C::zero(), nR = C::zero();
        if (hasL) {
            cL = C::load(srcL, plane, lane);
            cR = C::load(srcR, plane, lane);
            if (W > 32) {
                nL = C::load(srcL, plane, 32 + lane);
                nR = C::load(srcR, plane, 32 + lane);
            }
        }

        for (int g = 0; g * K < imax; ++g) {
#pragma unroll
            for (int u = 0; u < K; ++u) {
                const int i = g * K + u + 1;  // level within the phase half, 1..H
                if (i > imax) break;
                const bool Lact = hasL && i <= a.lower;
                const bool Uact = hasU && i <= a.upper;
                const int e = i - 1;
                if (Lact && (e & 15) == 0 && e > 0) {
                    cL = nL;
                    cR = nR;
                    const int c = (e >> 4) + 1;
                    if (32 * c < W) {
                        nL = C::load(srcL, plane, 32 * c + lane);
                        nR = C::load(srcR, plane, 32 * c + lane);
                    }
                }
                const int eo = 2 * (e & 15);
                const V fl0 = C::shfl(cL, eo), fl1 = C::shfl(cL, eo + 1);
                const V fr0 = C::shfl(cR, eo), fr1 = C::shfl(cR, eo + 1);
                const V left_in = C::shfl(v[K - 1], (lane + 31) & 31);
                const V right_in = C::shfl(v[0], (lane + 1) & 31);

                // The four cells next to the seam between the two diamonds take some inputs
                // from the flanks instead of the registers (slots static, owner lanes not):
                //   z = W-i  (slot K-1-u): left <- fl0, self <- fl1, right <- fr0 on the first level
                //   z = W-i+1 (slot K-u):  left <- fl1
                //   z = i-1  (slot u):     self <- fr0, right <- fr1, left <- fl1 on the first level
                //   z = i-2  (slot u-1):   right <- fr0
                const bool first = (u == 0) && (g == 0);  // i == 1
                const int sA = K - 1 - u, sB = (K - u) % K, sC = u, sD = (u + K - 1) % K;
                const bool pA = Lact && lane == ((31 - g + shift) & 31);
                const bool pB = Lact && !first && lane == ((((u == 0) ? 32 : 31) - g + shift) & 31);
                const bool pC = Lact && lane == ((g + shift) & 31);
                const bool pD = Lact && !first && lane == ((((u == 0) ? g - 1 : g) + shift + 32) & 31);
                V nv[K];
                V xs[K], cs[K], ys[K];  // inputs of the integer-pipe slots, for a fallback
                bool oks[K];
                bool okall = true;
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    V x = (j == 0) ? left_in : v[j - 1];
                    V c = v[j];
                    V y = (j == K - 1) ? right_in : v[j + 1];
                    if (j == sA) {
                        x = pA ? fl0 : x;
                        c = pA ? fl1 : c;
                        if (first) y = pA ? fr0 : y;
                    }
                    if (j == sB) x = pB ? fl1 : x;
                    if (j == sC) {
                        c = pC ? fr0 : c;
                        y = pC ? fr1 : y;
                        if (first) x = pC ? fl1 : x;
                    }
                    if (j == sD) y = pD ? fr0 : y;
                    if constexpr (SOFT > 0) {
                        if (j % SOFT == SOFT - 1) {
                            nv[j] = C::upd_soft(hr, x, c, y, oks[j]);
                            okall = okall && oks[j] && hr.usable;
                            xs[j] = x;
                            cs[j] = c;
                            ys[j] = y;
                            continue;
                        }
                    }
                    nv[j] = C::upd(prm, x, c, y);
                }
                if constexpr (SOFT > 0) {
                    // rare (a neighbour far from u in magnitude, a zero): the whole warp
                    // branches, and the flagged cells are updated on the FP64 pipe
                    if (__any_sync(0xffffffffu, !okall)) {
#pragma unroll
                        for (int j = SOFT - 1; j < K; j += SOFT)
                            if (!(oks[j] && hr.usable)) nv[j] = soft64::heat_update_fp64(prm.r, xs[j], cs[j], ys[j]);
                    }
                }
#pragma unroll
                for (int j = 0; j < K; ++j) v[j] = nv[j];

                // flank entries of the finishing diamond at level F + i (j = i): the pairs
                // [2i], [2i + 1] are the cells z = i, i + 1 (left) and z = W - 2 - i, W - 1 - i
                // (right), adjacent register slots of one lane at every unrolled level but
                // u = K - 2, where each pair straddles two lanes: one vector store per pair
                if (Uact && i <= H - 1) {
                    if (u != K - 2) {
                        {   // left: slots (u + 1) % K, (u + 2) % K of lane g + (u + 1) / K
                            const int s = (u + 1) % K, lz = g + (u + 1) / K;
                            if (lane == ((lz + shift) & 31)) C::store2(dU0, plane, 2 * i, v[s], v[s + 1]);
                        }
                        {   // right: slots q, q + 1 (q = K - 3 - u mod K) of lane 31 - g (- 1 if q < 0)
                            const int q = K - 3 - u;
                            const int s = (q % K + K) % K, lz = 31 - g + (q < 0 ? -1 : 0);
                            if (lane == ((lz + shift + 32) & 31)) C::store2(dU1, plane, 2 * i, v[s], v[s + 1]);
                        }
                    } else {
                        {   // z = i  -> left flank [2i]
                            const int s = (u + 1) % K, lz = g + (u + 1) / K;
                            if (lane == ((lz + shift) & 31)) C::store(dU0, plane, 2 * i, v[s]);
                        }
                        {   // z = i + 1 -> left flank [2i + 1]
                            const int s = (u + 2) % K, lz = g + (u + 2) / K;
                            if (lane == ((lz + shift) & 31)) C::store(dU0, plane, 2 * i + 1, v[s]);
                        }
                        {   // z = W - 2 - i -> right flank [2i]
                            const int q = K - 3 - u;
                            const int s = (q % K + K) % K, lz = 31 - g + (q < 0 ? -1 : 0);
                            if (lane == ((lz + shift + 32) & 31)) C::store(dU1, plane, 2 * i, v[s]);
                        }
                        {   // z = W - 1 - i -> right flank [2i + 1]
                            const int q = K - 2 - u;
                            const int s = (q % K + K) % K, lz = 31 - g + (q < 0 ? -1 : 0);
                            if (lane == ((lz + shift + 32) & 31)) C::store(dU1, plane, 2 * i + 1, v[s]);
                        }
                    }
                }
                // the starting diamond's full row (level F): its flank entries j = 0
                if (Lact && i == H && a.upper > 0) {
                    if (lane == ((16 + shift) & 31)) {
                        C::store(dL0, plane, 0, v[0]);
                        C::store(dL0, plane, 1, v[1 % K]);
                    }
                    if (lane == ((15 + shift) & 31)) {
                        C::store(dL1, plane, 0, v[K - 2]);
                        C::store(dL1, plane, 1, v[K - 1]);
                    }
                }
            }
        }
        // Down Triangle: the lower half ends at the run's last level (the loop's last level)
        if (a.write_lower && hasL) fold_store_row<K, C>(v, lane, shift, -a.lower, a.lower - 1, H, startL, a.n, a.state);
        if (!up) shift ^= 16;
    }
}

}  // namespace sw
