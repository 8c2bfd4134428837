// cpu_phase.h -- the host cores' share of a hybrid CPU/GPU swept run (Section 4.2:
// the GPU work factor, Eq. 1, splits the tiles between the GPU and the host
// processes). One host thread runs whole structures (Up Triangle, Diamond, Down
// Triangle; Section 4.1, Fig. 1) of one phase, with the geometry and the flank
// layout of the GPU phase kernels, so that the two sides exchange flank slots
// verbatim, and with the same per-cell functions instantiated on the host's IEEE
// operations (common.cuh), so that every cell agrees bitwise with the GPU.
//
// A structure keeps its row (positions 0..W+1, cell = base + position) as two
// full-state rows, the level being computed from the previous one; the lower
// half's four outer inputs per level come from the neighbours' flanks, the
// upper half's flank entries are exported after each level.
#pragma once
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "euler.cuh"
#include "flanks.cuh"
#include "heat.cuh"

namespace sw {

// One phase as the host sees it: host copies of the flank buffers (same layout
// as the device ones) and of the state planes.
template <class T> struct HostPhase {
    int64_t n;
    int W, H;
    int periodic;
    int p;             // 0 Up Triangle, 1 seam-centred, 2 tile-centred
    int64_t F;         // full level of the phase
    int lower, upper;  // levels of the two halves
    int write_lower, write_upper;
    int64_t tiles, nstruct_max;
    const T *flank_in;
    T *flank_out;
    T *state;          // NIO planes of n
};

// Host cell schemes: NF fields per cell (= the flank fields of the GPU policy),
// NIO state planes, and one level over a window of positions.
template <class O> struct HostHeatPlain {
    using T = typename O::T;
    static constexpr int NF = 1, NIO = 1;
    T r;
    // positions lo..hi of `nx` from `pv` (field planes of stride rs); g0 / g1: position of
    // the domain's first / last cell when a transmissive end is in the window, else -1
    void level(const T *pv, T *nx, int rs, int lo, int hi, int64_t, int g0, int g1) const {
        const T *__restrict a = pv;
        T *__restrict o = nx;
        for (int s = lo; s <= hi; ++s) o[s] = heat_update<O>(r, a[s - 1], a[s], a[s + 1]);
        if (g0 >= lo && g0 <= hi) o[g0] = heat_update<O>(r, a[g0], a[g0], g0 == g1 ? a[g0] : a[g0 + 1]);
        if (g1 >= lo && g1 <= hi && g1 != g0) o[g1] = heat_update<O>(r, a[g1 - 1], a[g1], a[g1]);
        (void)rs;
    }
};

struct HostHeatComp {
    using T = float;
    static constexpr int NF = 2, NIO = 2;  // high part, low part
    float rh, rl;
    void level(const T *pv, T *nx, int rs, int lo, int hi, int64_t, int g0, int g1) const {
        const T *h = pv, *l = pv + rs;
        T *oh = nx, *ol = nx + rs;
        auto one = [&](int s, int sa, int sb) {
            const HL out = heat_update_comp_t<HostOpsF>(rh, rl, HL{h[sa], l[sa]}, HL{h[s], l[s]}, HL{h[sb], l[sb]});
            oh[s] = out.h;
            ol[s] = out.l;
        };
        for (int s = lo; s <= hi; ++s) one(s, s - 1, s + 1);
        if (g0 >= lo && g0 <= hi) one(g0, g0, g0 == g1 ? g0 : g0 + 1);
        if (g1 >= lo && g1 <= hi && g1 != g0) one(g1, g1 - 1, g1);
    }
};

// Euler, lengthened cycle (level % 4: ratio of Q, predictor, ratio of Q*, final).
// COMP: fields Q^n high (0..2), low (3..5), Q* (6..8), ratio (9); plain: Q^n (0..2),
// Q* (3..5), ratio (6). Pressures and face fluxes once per position, as on the GPU.
template <class O, bool COMP> struct HostEuler {
    using T = typename O::T;
    static constexpr int NF = COMP ? 10 : 7, NIO = COMP ? 6 : 3;
    static constexpr int QS = COMP ? 6 : 3, TH = COMP ? 9 : 6;
    EulerK<O> k;
    mutable std::vector<T> scr;  // pressures or face fluxes per position
    void level(const T *pv, T *nx, int rs, int lo, int hi, int64_t lev, int g0, int g1) const {
        if ((int)scr.size() < 3 * rs) scr.assign(3 * rs, T(0));
        const int kind = (int)(lev & 3);
        for (int f = 0; f < NF; ++f) std::memcpy(nx + f * rs + lo, pv + f * rs + lo, sizeof(T) * (hi - lo + 1));
        if (kind == 0 || kind == 2) {
            const T *q = pv + (kind == 0 ? 0 : QS) * rs;
            const int a = (g0 >= lo && g0 <= hi) ? lo : lo - 1, b = (g1 >= lo && g1 <= hi) ? hi : hi + 1;
            for (int s = a; s <= b; ++s) scr[s] = eu_pressure<O>(k, q[s], q[rs + s], q[2 * rs + s]);
            for (int s = lo; s <= hi; ++s) {
                const T pm = (s == g0) ? scr[s] : scr[s - 1], pp = (s == g1) ? scr[s] : scr[s + 1];
                nx[TH * rs + s] = eu_ratio<O>(pm, scr[s], pp);
            }
        } else {
            const T *q = pv + (kind == 1 ? 0 : QS) * rs;
            const T *th = pv + TH * rs;
            // face between positions s-1 and s, s in lo..hi+1
            for (int s = lo; s <= hi + 1; ++s) {
                int a = s - 1, b = s;
                T tha, thb;
                if (s == g0) { a = s; tha = T(0); thb = th[s]; }
                else if (s - 1 == g1) { b = s - 1; tha = th[s - 1]; thb = T(0); }
                else { tha = th[s - 1]; thb = th[s]; }
                T f0, f1, f2;
                eu_face_flux<O>(k, q[a], q[rs + a], q[2 * rs + a], tha, q[b], q[rs + b], q[2 * rs + b], thb, f0, f1, f2);
                scr[s] = f0;
                scr[rs + s] = f1;
                scr[2 * rs + s] = f2;
            }
            for (int s = lo; s <= hi; ++s) {
                for (int v = 0; v < 3; ++v) {
                    const T d = O::sub(scr[v * rs + s + 1], scr[v * rs + s]);
                    if constexpr (!COMP) {
                        if (kind == 1) nx[(QS + v) * rs + s] = eu_update<O>(pv[v * rs + s], k.hlam, d);
                        else nx[v * rs + s] = eu_update<O>(pv[v * rs + s], k.lam, d);
                    } else {
                        if (kind == 1) {
                            nx[(QS + v) * rs + s] = eu_comp_predict<O>(pv[v * rs + s], pv[(3 + v) * rs + s], k.hlam, d);
                        } else {
                            float nh, nl;
                            eu_comp_final<O>(pv[v * rs + s], pv[(3 + v) * rs + s], k.lam, d, nh, nl);
                            nx[v * rs + s] = nh;
                            nx[(3 + v) * rs + s] = nl;
                        }
                    }
                }
            }
        }
    }
};

// Cells [first, last] of the state written by this host thread (for the copy-back).
struct WrittenRange {
    int64_t first = INT64_MAX, last = -1;
    void add(int64_t a, int64_t b) {
        first = std::min(first, a);
        last = std::max(last, b);
    }
};

// Structure b of one phase. `work`: 2 * NF * (W + 2) elements of scratch.
template <class Sch>
void cpu_structure(const Sch &sch, const HostPhase<typename Sch::T> &a, int64_t b, typename Sch::T *work,
                   WrittenRange &wr) {
    using T = typename Sch::T;
    constexpr int NF = Sch::NF;
    const int W = a.W, H = a.H, rs = W + 2;
    const int64_t n = a.n, M = a.tiles, S = a.nstruct_max;
    const int64_t c = (a.p & 1) ? b * W : b * W + H;
    const int64_t base = c - H - 1;  // cell of position 0
    int slo = 0, shi = W + 1;
    if (!a.periodic) {
        if (base < 0) slo = (int)(-base);
        if (base + W + 1 > n - 1) shi = (int)(n - 1 - base);
    }
    auto cell = [&](int s) -> int64_t {
        int64_t j = base + s;
        if (a.periodic) {
            if (j < 0) j += n;
            if (j >= n) j -= n;
        }
        return j;
    };
    // positions of the domain's end cells (transmissive), else -1
    const int g0 = (!a.periodic && base < 0 && -base <= W + 1) ? (int)(-base) : -1;
    const int g1 = (!a.periodic && n - 1 - base >= 0 && n - 1 - base <= W + 1) ? (int)(n - 1 - base) : -1;
    T *pv = work, *nx = work + NF * rs;
    const int64_t fs = S * 2 * (int64_t)W;  // flank field stride
    auto snap_out = [&](const T *row, int s, int side, int e) {
        T *d = a.flank_out + flank_off<T>(S, W, 0, b, side) + e;
        for (int f = 0; f < NF; ++f) d[f * fs] = row[f * rs + s];
    };
    auto store_row = [&](const T *row, int lo, int hi) {
        for (int s = lo; s <= hi; ++s) {
            const int64_t j = cell(s);
            for (int f = 0; f < Sch::NIO; ++f) a.state[f * n + j] = row[f * rs + s];
        }
        if (lo <= hi) {
            const int64_t j0 = cell(lo), j1 = cell(hi);
            if (j0 <= j1) wr.add(j0, j1);
            else {  // wraps (periodic)
                wr.add(j0, n - 1);
                wr.add(0, j1);
            }
        }
    };

    if (a.p == 0) {
        for (int s = 1; s <= W; ++s) {
            const int64_t j = cell(s);
            for (int f = 0; f < NF; ++f) pv[f * rs + s] = f < Sch::NIO ? a.state[f * n + j] : T(0);
        }
        snap_out(pv, 1, 0, 0);
        snap_out(pv, 2, 0, 1);
        snap_out(pv, W - 1, 1, 0);
        snap_out(pv, W, 1, 1);
    } else {
        int64_t lb, rb;
        bool has_l = true, has_r = true;
        if (a.p & 1) {
            lb = b - 1;
            rb = b;
        } else {
            lb = b;
            rb = b + 1;
        }
        if (a.periodic) {
            lb = (lb + M) % M;
            rb = rb % M;
        } else if (a.p & 1) {
            has_l = b > 0;
            has_r = b < M;
        }
        const T *inL = a.flank_in + flank_off<T>(S, W, 0, has_l ? lb : 0, 1);
        const T *inR = a.flank_in + flank_off<T>(S, W, 0, has_r ? rb : 0, 0);
        for (int i = 1; i <= a.lower; ++i) {
            const int64_t lev = a.F - H + i - 1;
            // the four outer inputs of this level, at level lev
            for (int t = 0; t < 4; ++t) {
                const int side = t >> 1, kk = t & 1;
                const int s = side == 0 ? H - i + kk : H + i + kk;
                if ((side == 0 ? has_l : has_r) && s >= slo && s <= shi) {
                    const T *src = (side == 0 ? inL : inR) + 2 * (i - 1) + kk;
                    for (int f = 0; f < NF; ++f) pv[f * rs + s] = src[f * fs];
                }
            }
            const int lo = std::max(H + 1 - i, slo), hi = std::min(H + i, shi);
            sch.level(pv, nx, rs, lo, hi, lev, g0, g1);
            std::swap(pv, nx);
            if (i == H && a.upper > 0) {
                if (1 >= slo && 1 <= shi) snap_out(pv, 1, 0, 0);
                if (2 >= slo && 2 <= shi) snap_out(pv, 2, 0, 1);
                if (W - 1 >= slo && W - 1 <= shi) snap_out(pv, W - 1, 1, 0);
                if (W >= slo && W <= shi) snap_out(pv, W, 1, 1);
            }
            if (i == a.lower && a.write_lower) store_row(pv, lo, hi);
        }
    }
    for (int i = 1; i <= a.upper; ++i) {
        const int64_t lev = a.F + i - 1;
        const int lo = std::max(1 + i, slo), hi = std::min(W - i, shi);
        sch.level(pv, nx, rs, lo, hi, lev, g0, g1);
        std::swap(pv, nx);
        if (1 + i >= lo && 1 + i <= hi) snap_out(pv, 1 + i, 0, 2 * i);
        if (2 + i >= lo && 2 + i <= hi) snap_out(pv, 2 + i, 0, 2 * i + 1);
        if (W - 1 - i >= lo && W - 1 - i <= hi) snap_out(pv, W - 1 - i, 1, 2 * i);
        if (W - i >= lo && W - i <= hi) snap_out(pv, W - i, 1, 2 * i + 1);
        if (i == a.upper && a.write_upper) store_row(pv, lo, hi);
    }
}

}  // namespace sw
