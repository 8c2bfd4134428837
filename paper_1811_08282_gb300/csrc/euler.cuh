// euler.cuh -- the second-order finite-volume Euler scheme (Section 4.2; state
// and sub-step structure of Section 4.3 / Fig. 2): per-cell arithmetic in the
// operation order of the scheme definition (no fused multiply-add, IEEE division
// and square root, so FP64 results are reproducible bit for bit), and the
// storage policies of the swept-phase driver. Lengthened sub-step cycle, by
// sub-step index k = level % 4:
//   k = 0: pressure ratio of Q^n            (stored in th)
//   k = 1: predictor  Q* = Q^n - (lambda/2) (F_{i+1/2} - F_{i-1/2})(Q^n, th)
//   k = 2: pressure ratio of Q*
//   k = 3: final      Q^{n+1} = Q^n - lambda (F_{i+1/2} - F_{i-1/2})(Q*, th*)
#pragma once
#include <type_traits>

#include "common.cuh"

namespace sw {

// ============================================================================
// Euler
// ============================================================================
struct EulerParams {
    double gamma, gm1, lam, hlam;  // gm1 = gamma - 1, hlam = lambda / 2 (rounded as FP64)
    float gammaf, gm1f, lamf, hlamf;
};

template <class O> struct EulerK {
    using T = typename O::T;
    T gamma, gm1, lam, hlam;
};

#pragma nv_exec_check_disable
template <class O>
SW_HD typename O::T eu_pressure(const EulerK<O> &k, typename O::T rho, typename O::T m,
                                                     typename O::T E) {
    using T = typename O::T;
    T u = O::div(m, rho);
    return O::mul(k.gm1, O::sub(E, O::mul(O::mul(T(0.5), m), u)));
}

#pragma nv_exec_check_disable
template <class O>
SW_HD typename O::T eu_ratio(typename O::T pm, typename O::T p0, typename O::T pp) {
    using T = typename O::T;
    T dm = O::sub(p0, pm);
    T dp = O::sub(pp, p0);
    if ((dm > T(0) && dp > T(0)) || (dm < T(0) && dp < T(0))) return O::div(dm, dp);
    return T(0);
}

#pragma nv_exec_check_disable
template <class O>
SW_HD void eu_phys_flux(const EulerK<O> &k, typename O::T rho, typename O::T m,
                                             typename O::T E, typename O::T &f0, typename O::T &f1,
                                             typename O::T &f2, typename O::T &speed) {
    using T = typename O::T;
    T u = O::div(m, rho);
    T p = O::mul(k.gm1, O::sub(E, O::mul(O::mul(T(0.5), m), u)));
    T c = O::sqrt_(O::div(O::mul(k.gamma, p), rho));
    f0 = m;
    f1 = O::add(O::mul(m, u), p);
    f2 = O::mul(O::add(E, p), u);
    speed = O::add(O::abs_(u), c);
}

// Numerical flux at the face between cell a (left) and cell b (right).
#pragma nv_exec_check_disable
template <class O>
SW_HD void eu_face_flux(const EulerK<O> &k, typename O::T a0, typename O::T a1,
                                             typename O::T a2, typename O::T tha, typename O::T b0,
                                             typename O::T b1, typename O::T b2, typename O::T thb,
                                             typename O::T &o0, typename O::T &o1, typename O::T &o2) {
    using T = typename O::T;
    T phl = tha < T(1) ? tha : T(1);
    T phr = thb > T(1) ? O::div(T(1), thb) : (thb > T(0) ? T(1) : T(0));
    T hl = O::mul(T(0.5), phl), hr = O::mul(T(0.5), phr);
    T d0 = O::sub(b0, a0), d1 = O::sub(b1, a1), d2 = O::sub(b2, a2);
    T l0 = O::add(a0, O::mul(hl, d0)), l1 = O::add(a1, O::mul(hl, d1)), l2 = O::add(a2, O::mul(hl, d2));
    T r0 = O::sub(b0, O::mul(hr, d0)), r1 = O::sub(b1, O::mul(hr, d1)), r2 = O::sub(b2, O::mul(hr, d2));
    T fl0, fl1, fl2, sl, fr0, fr1, fr2, sr;
    eu_phys_flux<O>(k, l0, l1, l2, fl0, fl1, fl2, sl);
    eu_phys_flux<O>(k, r0, r1, r2, fr0, fr1, fr2, sr);
    T s = sl > sr ? sl : sr;
    T hs = O::mul(T(0.5), s);
    o0 = O::sub(O::mul(T(0.5), O::add(fl0, fr0)), O::mul(hs, O::sub(r0, l0)));
    o1 = O::sub(O::mul(T(0.5), O::add(fl1, fr1)), O::mul(hs, O::sub(r1, l1)));
    o2 = O::sub(O::mul(T(0.5), O::add(fl2, fr2)), O::mul(hs, O::sub(r2, l2)));
}

#pragma nv_exec_check_disable
template <class O>
SW_HD EulerK<O> eu_k(const EulerParams &p) {
    if constexpr (std::is_same<typename O::T, double>::value) return EulerK<O>{p.gamma, p.gm1, p.lam, p.hlam};
    else return EulerK<O>{p.gammaf, p.gm1f, p.lamf, p.hlamf};
}

// State updates of the two flux sub-steps, shared by every kernel and the host:
// plain forms Q - c dF; hi/lo form: predictor Q* = h + (l - (lambda/2) dF) in FP32,
// final (h, l) + (-lambda dF) with TwoSum / Fast2Sum.
#pragma nv_exec_check_disable
template <class O>
SW_HD typename O::T eu_update(typename O::T q, typename O::T c, typename O::T d) {
    return O::sub(q, O::mul(c, d));
}

#pragma nv_exec_check_disable
template <class O>
SW_HD float eu_comp_predict(float h, float l, float hlam, float d) {
    return O::add(h, O::sub(l, O::mul(hlam, d)));
}

#pragma nv_exec_check_disable
template <class O>
SW_HD void eu_comp_final(float h, float l, float lam, float d, float &nh, float &nl) {
    const float delta = -O::mul(lam, d);
    float sm, e;
    two_sum_t<O>(h, delta, sm, e);
    fast_two_sum_t<O>(sm, O::add(l, e), nh, nl);
}

// Row fields (FP64 / FP32): 0..2 Q^n, 3..5 Q*, 6 pressure ratio -- the seven values
// per point of the lengthened state (Section 4.3). Updates are in place: a
// sub-step reads one group of fields of its neighbours and writes another group
// of its own, so no second buffer is needed (the alternation of Section 4.1).
template <int PREC> struct EulerPolicy {
    static_assert(PREC == 0 || PREC == 1, "plain Euler policy is FP64 or FP32");
    using O = typename std::conditional<PREC == 0, OpsD, OpsF>::type;
    using T = typename O::T;
    static constexpr int NROW = 7, NSNAP = 7, NIO = 3;
    static constexpr bool INJECT_AHEAD = false;
    static constexpr int R = 1;  // stencil radius: windows change by R cells per level
    static constexpr bool TWO_PASS = true;
    static constexpr int NSCR = 3;  // face flux components (or the pressure) per position
    // launch bound (resident 512-thread CTAs per SM): FP32 trades a few spilled values for
    // three CTAs (40 registers; 10-13 % faster than two on GB300), FP64 keeps up to 128 registers
    static constexpr int MIN_BLOCKS = PREC == 0 ? 1 : 3;
    using Params = EulerParams;
    static __device__ __forceinline__ void load_state(T *row, int rs, int s, const T *st, int64_t n, int64_t j) {
        row[s] = st[j];
        row[rs + s] = st[n + j];
        row[2 * rs + s] = st[2 * n + j];
    }
    static __device__ __forceinline__ void store_state(const T *row, int rs, int s, int64_t level, T *st,
                                                       int64_t n, int64_t j) {
        st[j] = row[s];
        st[n + j] = row[rs + s];
        st[2 * n + j] = row[2 * rs + s];
    }
    // snapshot field f of cell s (every row field is part of the snapshot)
    static __device__ __forceinline__ T get_field(const T *row, int rs, int s, int64_t level, int f) {
        return row[f * rs + s];
    }
    static __device__ __forceinline__ void set_field(T *row, int rs, int s, int64_t level, int f, T v) {
        row[f * rs + s] = v;
    }
    // Two passes per sub-step (the per-cell results are those of evaluating both
    // faces and all three pressures per cell; each is computed once here):
    // pre():  ratio sub-steps -> p at each position in [lo-1, hi+1];
    //         flux sub-steps  -> the face flux between positions s-1 and s, s in [lo, hi+1].
    // step(): the cell update from the scratch values.
    // gl: cell s is the domain's first cell; gr_prev: cell s-1 is its last (transmissive).
    static __device__ __forceinline__ void pre(const Params &prm, const T *row, int rs, T *scr, int s,
                                               int64_t level, int lo, int hi, int slo, int shi, bool gl,
                                               bool gr_prev) {
        const EulerK<O> k = eu_k<O>(prm);
        const int kind = (int)(level & 3);
        if (kind == 0 || kind == 2) {
            if (s < slo || s > shi) return;
            const T *q = row + (kind == 0 ? 0 : 3) * rs;
            scr[s] = eu_pressure<O>(k, q[s], q[rs + s], q[2 * rs + s]);
        } else {
            if (s < lo) return;
            const T *q = row + (kind == 1 ? 0 : 3) * rs;
            const T *th = row + 6 * rs;
            int a = s - 1, b = s;
            T tha, thb;
            if (gl) { a = s; tha = T(0); thb = th[s]; }
            else if (gr_prev) { b = s - 1; tha = th[s - 1]; thb = T(0); }
            else { tha = th[s - 1]; thb = th[s]; }
            T f0, f1, f2;
            eu_face_flux<O>(k, q[a], q[rs + a], q[2 * rs + a], tha, q[b], q[rs + b], q[2 * rs + b], thb, f0, f1,
                            f2);
            scr[s] = f0;
            scr[rs + s] = f1;
            scr[2 * rs + s] = f2;
        }
    }
    static __device__ __forceinline__ void step(const Params &prm, T *row, int rs, const T *scr, int s,
                                                int64_t level, bool gl, bool gr) {
        const EulerK<O> k = eu_k<O>(prm);
        const int kind = (int)(level & 3);
        if (kind == 0 || kind == 2) {
            const T pm = gl ? scr[s] : scr[s - 1], pp = gr ? scr[s] : scr[s + 1];
            row[6 * rs + s] = eu_ratio<O>(pm, scr[s], pp);
        } else {
            const T c = (kind == 1) ? k.hlam : k.lam;
            T *out = row + (kind == 1 ? 3 : 0) * rs;
            const T q0 = row[s], q1 = row[rs + s], q2 = row[2 * rs + s];
            out[s] = eu_update<O>(q0, c, O::sub(scr[s + 1], scr[s]));
            out[rs + s] = eu_update<O>(q1, c, O::sub(scr[rs + s + 1], scr[rs + s]));
            out[2 * rs + s] = eu_update<O>(q2, c, O::sub(scr[2 * rs + s + 1], scr[2 * rs + s]));
        }
    }
};

// FP32 hi/lo compensated Euler. Row fields: 0..2 Q^n high, 3..5 Q^n low, 6..8 Q*
// (plain FP32), 9 pressure ratio. Fluxes and ratios are evaluated in FP32 from
// the high parts; the state update Q^n - c dF is applied with TwoSum.
struct EulerPolicyComp {
    using O = OpsF;
    using T = float;
    static constexpr int NROW = 10, NSNAP = 10, NIO = 6;
    static constexpr bool INJECT_AHEAD = false;
    static constexpr int R = 1;  // stencil radius: windows change by R cells per level
    static constexpr bool TWO_PASS = true;
    static constexpr int NSCR = 3;
    static constexpr int MIN_BLOCKS = 3;  // as EulerPolicy<FP32>
    using Params = EulerParams;
    static __device__ __forceinline__ void load_state(T *row, int rs, int s, const T *st, int64_t n, int64_t j) {
#pragma unroll
        for (int f = 0; f < 6; ++f) row[f * rs + s] = st[f * n + j];
    }
    static __device__ __forceinline__ void store_state(const T *row, int rs, int s, int64_t level, T *st,
                                                       int64_t n, int64_t j) {
#pragma unroll
        for (int f = 0; f < 6; ++f) st[f * n + j] = row[f * rs + s];
    }
    // snapshot field f of cell s (every row field is part of the snapshot)
    static __device__ __forceinline__ T get_field(const T *row, int rs, int s, int64_t level, int f) {
        return row[f * rs + s];
    }
    static __device__ __forceinline__ void set_field(T *row, int rs, int s, int64_t level, int f, T v) {
        row[f * rs + s] = v;
    }
    // Two passes per sub-step, as in EulerPolicy; fluxes and pressures from the
    // high parts (Q^n) or the plain FP32 Q*.
    static __device__ __forceinline__ void pre(const Params &prm, const T *row, int rs, T *scr, int s,
                                               int64_t level, int lo, int hi, int slo, int shi, bool gl,
                                               bool gr_prev) {
        const EulerK<O> k = eu_k<O>(prm);
        const int kind = (int)(level & 3);
        if (kind == 0 || kind == 2) {
            if (s < slo || s > shi) return;
            const T *q = row + (kind == 0 ? 0 : 6) * rs;
            scr[s] = eu_pressure<O>(k, q[s], q[rs + s], q[2 * rs + s]);
        } else {
            if (s < lo) return;
            const T *q = row + (kind == 1 ? 0 : 6) * rs;
            const T *th = row + 9 * rs;
            int a = s - 1, b = s;
            T tha, thb;
            if (gl) { a = s; tha = T(0); thb = th[s]; }
            else if (gr_prev) { b = s - 1; tha = th[s - 1]; thb = T(0); }
            else { tha = th[s - 1]; thb = th[s]; }
            T f0, f1, f2;
            eu_face_flux<O>(k, q[a], q[rs + a], q[2 * rs + a], tha, q[b], q[rs + b], q[2 * rs + b], thb, f0, f1,
                            f2);
            scr[s] = f0;
            scr[rs + s] = f1;
            scr[2 * rs + s] = f2;
        }
    }
    static __device__ __forceinline__ void step(const Params &prm, T *row, int rs, const T *scr, int s,
                                                int64_t level, bool gl, bool gr) {
        const EulerK<O> k = eu_k<O>(prm);
        const int kind = (int)(level & 3);
        if (kind == 0 || kind == 2) {
            const T pm = gl ? scr[s] : scr[s - 1], pp = gr ? scr[s] : scr[s + 1];
            row[9 * rs + s] = eu_ratio<O>(pm, scr[s], pp);
        } else {
            const T df[3] = {__fsub_rn(scr[s + 1], scr[s]), __fsub_rn(scr[rs + s + 1], scr[rs + s]),
                             __fsub_rn(scr[2 * rs + s + 1], scr[2 * rs + s])};
            if (kind == 1) {
#pragma unroll
                for (int v = 0; v < 3; ++v)
                    row[(6 + v) * rs + s] = eu_comp_predict<O>(row[v * rs + s], row[(3 + v) * rs + s], k.hlam, df[v]);
            } else {
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    T nh, nl;
                    eu_comp_final<O>(row[v * rs + s], row[(3 + v) * rs + s], k.lam, df[v], nh, nl);
                    row[v * rs + s] = nh;
                    row[(3 + v) * rs + s] = nl;
                }
            }
        }
    }
};

// Flattened form (Section 4.3, Fig. 2): two 5-point stages per step, one level
// each (level % 2: 0 predictor from Q, 1 final from Q*); the pressure ratio is
// recomputed inside the stage instead of being stored. Stencil radius 2: a swept
// window changes by two cells per level and a flank entry pair becomes a quad.
// Row fields: Q^n (0..2), Q* (3..5); hi/lo: Q^n high (0..2), low (3..5), Q* (6..8).
// Four passes per level over the window [lo, hi]: pressures on [lo-2, hi+2],
// ratios on [lo-1, hi+1], face fluxes between s-1 and s for s in [lo, hi+1], the
// update on [lo, hi]. Every value is the one the lengthened form computes.
// Scratch fields: pressure (0), ratio (1), face flux (2..4).
template <class O_, bool COMP> struct EulerFlatBase {
    using O = O_;
    using T = typename O::T;
    static constexpr int NROW = COMP ? 9 : 6, NSNAP = NROW, NIO = COMP ? 6 : 3;
    static constexpr int QS = COMP ? 6 : 3;
    static constexpr int R = 2;
    static constexpr int NSCR = 5;
    static constexpr bool INJECT_AHEAD = false;
    static constexpr bool TWO_PASS = false;
    static constexpr int MIN_BLOCKS = std::is_same<T, float>::value ? 3 : 1;  // as EulerPolicy
    using Params = EulerParams;
    static __device__ __forceinline__ void load_state(T *row, int rs, int s, const T *st, int64_t n, int64_t j) {
#pragma unroll
        for (int f = 0; f < NIO; ++f) row[f * rs + s] = st[f * n + j];
    }
    static __device__ __forceinline__ void store_state(const T *row, int rs, int s, int64_t level, T *st,
                                                       int64_t n, int64_t j) {
#pragma unroll
        for (int f = 0; f < NIO; ++f) st[f * n + j] = row[f * rs + s];
    }
    static __device__ __forceinline__ T get_field(const T *row, int rs, int s, int64_t level, int f) {
        return row[f * rs + s];
    }
    static __device__ __forceinline__ void set_field(T *row, int rs, int s, int64_t level, int f, T v) {
        row[f * rs + s] = v;
    }
    static __device__ __forceinline__ const T *group(const T *row, int rs, int64_t level) {
        return row + ((level & 1) == 0 ? 0 : QS) * rs;
    }
    static __device__ __forceinline__ void pass_p(const Params &prm, const T *row, int rs, T *scr, int s,
                                                  int64_t level) {
        const EulerK<O> k = eu_k<O>(prm);
        const T *q = group(row, rs, level);
        scr[s] = eu_pressure<O>(k, q[s], q[rs + s], q[2 * rs + s]);
    }
    static __device__ __forceinline__ void pass_th(T *scr, int rs, int s) {
        scr[rs + s] = eu_ratio<O>(scr[s - 1], scr[s], scr[s + 1]);
    }
    static __device__ __forceinline__ void pass_f(const Params &prm, const T *row, int rs, T *scr, int s,
                                                  int64_t level) {
        const EulerK<O> k = eu_k<O>(prm);
        const T *q = group(row, rs, level);
        const T *th = scr + rs;
        T f0, f1, f2;
        eu_face_flux<O>(k, q[s - 1], q[rs + s - 1], q[2 * rs + s - 1], th[s - 1], q[s], q[rs + s], q[2 * rs + s],
                        th[s], f0, f1, f2);
        scr[2 * rs + s] = f0;
        scr[3 * rs + s] = f1;
        scr[4 * rs + s] = f2;
    }
    static __device__ __forceinline__ void pass_u(const Params &prm, T *row, int rs, const T *scr, int s,
                                                  int64_t level) {
        const EulerK<O> k = eu_k<O>(prm);
        const bool pred = (level & 1) == 0;
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const T d = O::sub(scr[(2 + v) * rs + s + 1], scr[(2 + v) * rs + s]);
            if constexpr (!COMP) {
                if (pred) row[(QS + v) * rs + s] = eu_update<O>(row[v * rs + s], k.hlam, d);
                else row[v * rs + s] = eu_update<O>(row[v * rs + s], k.lam, d);
            } else {
                if (pred) {
                    row[(QS + v) * rs + s] = eu_comp_predict<O>(row[v * rs + s], row[(3 + v) * rs + s], k.hlam, d);
                } else {
                    float nh, nl;
                    eu_comp_final<O>(row[v * rs + s], row[(3 + v) * rs + s], k.lam, d, nh, nl);
                    row[v * rs + s] = nh;
                    row[(3 + v) * rs + s] = nl;
                }
            }
        }
    }
};

template <int PREC> using EulerFlatPolicy = EulerFlatBase<typename std::conditional<PREC == 0, OpsD, OpsF>::type, false>;
using EulerFlatPolicyComp = EulerFlatBase<OpsF, true>;

}  // namespace sw

