// swept_phase.cuh -- one launch = one swept phase (Section 4.1, Fig. 1) over all
// structures (triangles / diamonds) of that phase, one CTA per structure.
//
// Geometry for a 3-point stencil (radius 1; the policy's radius R scales it: a
// half spans H/R levels and windows change by R cells per level, see
// swept_structure) with H = W/2, tiles [tW, tW+W), level = sub-step index:
//   phase p has full level F = p*H and centres c = t*W + H (p even, tile centred)
//   or c = t*W (p odd, centred on the seam between tiles t-1 and t).
//   lower half (p >= 1): levels F-H+i, i = 1..H, cells [c-i, c+i-1]   (widening)
//   upper half:          levels F+i,   i = 1..H-1, cells [c-H+i, c+H-1-i] (narrowing)
//   Phase 0 = Up Triangle (upper half only, from the initial row); the phases
//   with both halves are Diamonds; the last phase is the Down Triangle (lower
//   half only). Lower(p) and upper(p-1) tile every level, so each (cell, level)
//   is computed exactly once: the swept rule does no redundant work.
// Communication (Fig. 1b, 1d): after its upper half a structure has exported,
// for every level F+j (j = 0..H-1), the two outermost cells on each side (its
// "flanks"); the lower half of the next phase at centre c' takes the right
// flank of the structure at c'-H and the left flank of the one at c'+H. Flanks
// travel through HBM between launches (global buffers, double-buffered by phase).
// A run that stops at a level L between full levels truncates the last upper
// half and the Down Triangle at L, so any number of sub-steps needs no extra
// per-step launches.
#pragma once
#include "common.cuh"
#include "flanks.cuh"

namespace sw {

template <class T> struct PhaseArgs {
    int64_t n;           // cells
    int W, H;
    int periodic;        // 1 periodic, 0 transmissive
    int p;               // phase index
    int64_t F;           // full level of this phase (p*H)
    int lower;           // lower-half levels computed (0 for p == 0)
    int upper;           // upper-half levels computed
    int write_lower;     // lower half ends at the final level: store its top row
    int write_upper;     // upper half ends at the final level: store its top row
    int64_t nstruct;     // structures in this phase
    int64_t nstruct_max; // structures per flank buffer
    int64_t tiles;       // M = n / W
    const T *flank_in;   // previous phase's flanks
    T *flank_out;        // this phase's flanks
    T *state;            // state planes (layout of the policy)
};

// Flank loads: plain within a launch sequence (the L1 is not reused across
// launches); L2-only (ld.global.cg) inside a persistent kernel, where another CTA
// may have rewritten a flank that this SM's L1 still holds from an earlier item.
// Input entries are staged in chunks of levels (kFlankChunk).
template <bool CG, class T> __device__ __forceinline__ T flank_ld(const T *p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// Levels of neighbour flank entries staged per cooperative load.
constexpr int kFlankChunk = 32;

// Shared memory of one structure, in elements of P::T: the row (NROW fields of
// W+2R positions), per-position scratch (NSCR fields), and a chunk of staged input
// flank entries (2R per level and side). Output flank entries go from the row to
// global memory directly.
template <class P> __host__ __device__ constexpr size_t swept_smem_elems(int W) {
    return size_t(P::NROW + P::NSCR) * (W + 2 * P::R) + size_t(P::NSNAP) * 2 * 2 * P::R * (kFlankChunk + 1);
}

// One sub-step over row positions [lo, hi]. Radius 1: two-pass policies first
// compute per-position intermediates on [lo-1, hi+1] into scratch, then update
// cells. Radius 2 (flattened Euler stage): pressures, ratios, faces, update.
// `mid` runs (all threads) before the last pass, which reads the row on [lo, hi]
// only: the row positions outside it that the earlier passes read are free again,
// so the next level's flank inputs can be injected there without a barrier.
template <class P, class GL, class GR, class AFTER, class MID>
__device__ __forceinline__ void swept_level(const typename P::Params &prm, typename P::T *row, int rs,
                                            typename P::T *scr, int64_t lev, int lo, int hi, int slo, int shi,
                                            GL ghost_l, GR ghost_r, AFTER after, MID mid) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if constexpr (P::R == 2) {
        for (int s = lo - 2 + tid; s <= hi + 2; s += nt) P::pass_p(prm, row, rs, scr, s, lev);
        __syncthreads();
        for (int s = lo - 1 + tid; s <= hi + 1; s += nt) P::pass_th(scr, rs, s);
        __syncthreads();
        for (int s = lo + tid; s <= hi + 1; s += nt) P::pass_f(prm, row, rs, scr, s, lev);
        __syncthreads();
        mid();
        for (int s = lo + tid; s <= hi; s += nt) {
            P::pass_u(prm, row, rs, scr, s, lev);
            after(s);
        }
    } else if constexpr (P::TWO_PASS) {
        for (int s = lo - 1 + tid; s <= hi + 1; s += nt)
            P::pre(prm, row, rs, scr, s, lev, lo, hi, slo, shi, ghost_l(s), ghost_r(s - 1));
        __syncthreads();
        mid();
        for (int s = lo + tid; s <= hi; s += nt) {
            P::step(prm, row, rs, scr, s, lev, ghost_l(s), ghost_r(s));
            after(s);
        }
    } else {
        for (int s = lo + tid; s <= hi; s += nt) {
            P::step(prm, row, rs, s, lev, ghost_l(s), ghost_r(s));
            after(s);
        }
    }
}

// The work of one structure (triangle or diamond) `b` of one phase, done by one
// CTA (all its threads must call it). smem: swept_smem_elems<P>(W) elements.
// Stencil radius R = P::R: a phase half spans HL = H / R levels, the lower half's
// window [c - R i, c + R i) widens and the upper half's [c - H + R i, c + H - R i)
// narrows by R cells per side and level, and a flank entry per level and side is
// the 2R outermost cells (2R HL = W entries per side, the layout of R = 1).
template <class P, bool CG>
__device__ __forceinline__ void swept_structure(const PhaseArgs<typename P::T> &a,
                                                const typename P::Params &prm, int64_t b,
                                                typename P::T *smem) {
    using T = typename P::T;
    constexpr int R = P::R, R2 = 2 * P::R;
    T *row = smem;
    const int W = a.W, H = a.H, HL = a.H / R;
    const int rs = W + 2 * R;             // row stride (positions 0..W+2R-1)
    T *scr = row + P::NROW * rs;          // [NSCR][rs]
    T *chunk = scr + P::NSCR * rs;        // [NSNAP][2 sides][2R (kFlankChunk + 1)] staged flank entries
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t n = a.n;
    const int64_t S = a.nstruct_max;
    const int64_t c = (a.p & 1) ? b * W : b * W + H;
    const int64_t base = c - H - R;       // cell of row position 0

    // valid row positions (transmissive domains clip to [0, n))
    int slo = 0, shi = rs - 1;
    if (!a.periodic) {
        if (base < 0) slo = (int)(-base);
        if (base + rs - 1 > n - 1) shi = (int)(n - 1 - base);
    }
    auto cell = [&](int s) -> int64_t { return a.periodic ? wrap_index(base + s, n) : base + s; };
    auto ghost_l = [&](int s) -> bool { return !a.periodic && base + s == 0; };
    auto ghost_r = [&](int s) -> bool { return !a.periodic && base + s == n - 1; };
    // radius 2: the cells beyond a transmissive end are copies of the end cell (the
    // clamped halo of the per-step flattened kernel); refreshed before every level
    auto ghost_fill = [&](int64_t lev) {
        if constexpr (R == 2) {
            if (slo == 0 && shi == rs - 1) return;
            for (int t = tid; t < 2 * R * P::NROW; t += nt) {
                const int side = t / (R * P::NROW), rem = t % (R * P::NROW), d = rem / P::NROW + 1,
                          f = rem % P::NROW;
                const int s = side == 0 ? slo - d : shi + d, src = side == 0 ? slo : shi;
                if ((side == 0 ? slo > 0 : shi < rs - 1) && s >= 0 && s < rs)
                    P::set_field(row, rs, s, lev, f, P::get_field(row, rs, src, lev, f));
            }
            __syncthreads();
        }
    };
    // this structure's flank entry e of `side` (0 left, 1 right) at level `lev`: every field
    auto publish = [&](int s, int64_t lev, int side, int e) {
        if (!a.flank_out || a.upper <= 0) return;
#pragma unroll
        for (int f = 0; f < P::NSNAP; ++f)
            a.flank_out[flank_off<T>(S, W, f, b, side) + e] = P::get_field(row, rs, s, lev, f);
    };
    // the full row (level F): flank entries j = 0, the 2R outermost cells of each side
    auto publish_full = [&](int s, int64_t lev) {
        if (s >= R && s < R + R2) publish(s, lev, 0, s - R);
        if (s >= W - R && s < W + R) publish(s, lev, 1, s - (W - R));
    };

    if (a.p == 0) {
        // Up Triangle: the initial row [c-H, c+H) at level 0 (always inside the domain)
        for (int s = R + tid; s < W + R; s += nt) {
            P::load_state(row, rs, s, a.state, n, base + s);
            publish_full(s, 0);
        }
        __syncthreads();
    } else {
        // neighbours in phase p-1: left has centre c-H, right has centre c+H
        int64_t lb, rb;
        if (a.p & 1) { lb = b - 1; rb = b; }   // seam centred: tiles b-1 and b
        else { lb = b; rb = b + 1; }           // tile centred: seams b and b+1
        bool has_l = true, has_r = true;
        if (a.periodic) {
            const int64_t M = a.tiles;
            lb = (lb + M) % M;
            rb = rb % M;
        } else {
            if (a.p & 1) { has_l = b > 0; has_r = b < a.tiles; }
        }
        // Communication: the neighbours' flank entries are staged in chunks of CH levels
        // (all fields, both sides, one overlapping entry group so that an injection one
        // level ahead stays inside the chunk), loaded cooperatively from global memory;
        // step i injects the flank group of level F-HL+i-1 from the chunk into the row.
        const int cs = R2 * (kFlankChunk + 1);  // entries per (field, side) in the chunk
        int i0 = 1;                             // first step the chunk serves
        auto load_chunk = [&](int first) {
            i0 = first;
            for (int t = tid; t < P::NSNAP * 2 * cs; t += nt) {
                const int f = t / (2 * cs), rem = t % (2 * cs), side = rem / cs, e = rem % cs;
                const int64_t idx = (int64_t)R2 * (first - 1) + e;
                if (idx < W && (side == 0 ? has_l : has_r))
                    chunk[t] = flank_ld<CG>(a.flank_in +
                                            flank_off<T>(S, W, f, side == 0 ? lb : rb, side == 0 ? 1 : 0) + idx);
            }
        };
        auto inject = [&](int i) {
            for (int t = tid; t < 2 * R2 * P::NSNAP; t += nt) {
                const int side = t / (R2 * P::NSNAP), rem = t % (R2 * P::NSNAP);
                const int k = rem / P::NSNAP, f = rem % P::NSNAP;
                const int s = side == 0 ? H - R * i + k : H + R * i + k;
                if ((side == 0 ? has_l : has_r) && s >= slo && s <= shi)
                    P::set_field(row, rs, s, a.F - HL + i - 1, f, chunk[(f * 2 + side) * cs + R2 * (i - i0) + k]);
            }
        };
        if (a.lower > 0) {
            load_chunk(1);
            __syncthreads();
        }
        // level 1's inputs up front; later levels' inputs are injected one level ahead: after
        // the level's update (slot policies) or before its last pass (in-place policies)
        if (a.lower > 0) {
            inject(1);
            __syncthreads();
        }
        constexpr bool kMidInject = !P::INJECT_AHEAD && (P::TWO_PASS || P::R == 2);
        for (int i = 1; i <= a.lower; ++i) {
            const int64_t lev = a.F - HL + i - 1;  // level read; level lev+1 written
            if (i > 1 && (i - 1) % kFlankChunk == 0) {  // the previous level ended with a barrier
                load_chunk(i);
                __syncthreads();
            }
            if (!P::INJECT_AHEAD && !kMidInject && i > 1) {
                inject(i);
                __syncthreads();
            }
            ghost_fill(lev);
            int lo = H + R - R * i, hi = H + R + R * i - 1;
            if (lo < slo) lo = slo;
            if (hi > shi) hi = shi;
            const bool last = (i == a.lower);
            swept_level<P>(
                prm, row, rs, scr, lev, lo, hi, slo, shi, ghost_l, ghost_r,
                [&](int s) {
                    if (i == HL) publish_full(s, lev + 1);  // full level F reached
                    if (last && a.write_lower) P::store_state(row, rs, s, lev + 1, a.state, n, cell(s));
                },
                [&] {
                    if (kMidInject && i < a.lower) inject(i + 1);
                });
            if (P::INJECT_AHEAD && i < a.lower) inject(i + 1);
            __syncthreads();
        }
    }

    // upper half: levels F+1 .. F+upper on the narrowing window; flank entries j = i
    for (int i = 1; i <= a.upper; ++i) {
        const int64_t lev = a.F + i - 1;
        ghost_fill(lev);
        int lo = R + R * i, hi = W + R - 1 - R * i;
        const int el = lo, er = hi + 1 - R2;  // first position of the left / right entry group
        if (lo < slo) lo = slo;
        if (hi > shi) hi = shi;
        const bool last = (i == a.upper);
        swept_level<P>(
            prm, row, rs, scr, lev, lo, hi, slo, shi, ghost_l, ghost_r,
            [&](int s) {
                if (s >= el && s < el + R2) publish(s, lev + 1, 0, R2 * i + (s - el));
                if (s >= er && s < er + R2) publish(s, lev + 1, 1, R2 * i + (s - er));
                if (last && a.write_upper) P::store_state(row, rs, s, lev + 1, a.state, n, cell(s));
            },
            [] {});
        __syncthreads();
    }
}

template <class P>
__global__ void __launch_bounds__(512, P::MIN_BLOCKS) k_swept_phase(PhaseArgs<typename P::T> a,
                                                                    typename P::Params prm) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    swept_structure<P, false>(a, prm, (int64_t)blockIdx.x, reinterpret_cast<typename P::T *>(smem_raw));
}

}  // namespace sw
