// fold_euler.cuh -- register-resident Up / Diamond / Down phases for the Euler
// equations (Section 4.1, Fig. 1; lengthened sub-step cycle of Section 4.3),
// periodic or transmissive grids, complete upper halves only.
//
// The folding is that of the heat kernel (fold_heat.cuh): one warp owns a chain
// of consecutive structures of one phase and runs the upper half of structure
// k together with the lower half of structure k+1, whose window is rotated by
// W/2 so that the two active regions are complements; each lane holds K = W/32
// consecutive cells, a cell being the 7 values of the lengthened state (Q^n,
// Q*, pressure ratio; hi/lo form: 10). Both regions are on the same level, so
// the sub-step kind (level % 4) is the same for the whole warp, and unrolling
// the level loop by K (a multiple of 4) makes it a compile-time constant.
//
// Ratio levels (kinds 0, 2): each lane evaluates the pressure of its K cells,
// takes its neighbours' by shuffle, and updates the ratio. Flux levels (kinds
// 1, 3): each lane evaluates the K faces to the left of its cells, the face to
// the right of its last cell comes from the next lane by shuffle, so every face
// flux is evaluated once, as in the per-step kernel. Near the seams between the
// two regions four cells take inputs from the previous phase's flanks (as in
// the heat kernel); in face terms two faces get a flank value as one input and
// each seam needs one extra face with both inputs from the flanks, which each
// lane evaluates in one spare face slot (only the two lanes at the seams use
// it). On transmissive grids the structures at the domain ends are taken as
// whole diamonds whose cells outside [0, n) are never read by a real cell: the
// faces at the two domain ends take the ghost rule of the scheme (the outer
// input is the end cell itself, with ratio 0), and the row store skips them.
//
// Flanks are read and written in the layout of k_swept_phase with the fields of
// the Euler policies, so the kernels mix within one run, and every value goes
// through the same per-cell functions: results are bitwise identical to the
// generic and per-step kernels.
#pragma once
#include <type_traits>

#include "euler.cuh"
#include "flanks.cuh"

namespace sw {

// Cell policies: field layout of the lengthened state and the two state updates.
template <class O_> struct EFoldPlain {
    using O = O_;
    using T = typename O::T;
    static constexpr int NF = 7;   // Q^n (0..2), Q* (3..5), ratio (6)
    static constexpr int NIO = 3;  // state planes
    static constexpr int QS = 3, TH = 6;
    // launch bound (resident 128-thread CTAs per SM): FP32 trades a few spilled values for
    // 20 warps per SM, the best of a sweep; FP64 keeps all its registers
    static constexpr int MIN_BLOCKS = std::is_same<T, float>::value ? 5 : 1;
    // predictor: Q* = Q^n - (lambda/2) dF
    static __device__ __forceinline__ void predict(T (&c)[NF], const EulerK<O> &k, const T (&d)[3]) {
#pragma unroll
        for (int v = 0; v < 3; ++v) c[QS + v] = eu_update<O>(c[v], k.hlam, d[v]);
    }
    // final: Q^{n+1} = Q^n - lambda dF
    static __device__ __forceinline__ void final_(T (&c)[NF], const EulerK<O> &k, const T (&d)[3]) {
#pragma unroll
        for (int v = 0; v < 3; ++v) c[v] = eu_update<O>(c[v], k.lam, d[v]);
    }
};

struct EFoldComp {
    using O = OpsF;
    using T = float;
    static constexpr int NF = 10;  // Q^n high (0..2), Q^n low (3..5), Q* (6..8), ratio (9)
    static constexpr int NIO = 6;
    static constexpr int QS = 6, TH = 9;
    static constexpr int MIN_BLOCKS = 4;  // 16 warps per SM, the best of a sweep
    static __device__ __forceinline__ void predict(T (&c)[NF], const EulerK<O> &k, const T (&d)[3]) {
#pragma unroll
        for (int v = 0; v < 3; ++v) c[QS + v] = eu_comp_predict<O>(c[v], c[3 + v], k.hlam, d[v]);
    }
    static __device__ __forceinline__ void final_(T (&c)[NF], const EulerK<O> &k, const T (&d)[3]) {
#pragma unroll
        for (int v = 0; v < 3; ++v) eu_comp_final<O>(c[v], c[3 + v], k.lam, d[v], c[v], c[3 + v]);
    }
};

template <class T> struct EFoldArgs {
    int p;                // 0: Up Triangle; 1: seam-centred phase (odd); 2: tile-centred (even)
    int periodic;         // 1 periodic, 0 transmissive
    int64_t n;            // cells
    int64_t tiles;        // M = n / W
    int64_t nstruct;      // structures in this phase (transmissive odd phases: M + 1)
    int64_t nstruct_max;  // structures per flank buffer
    int lower, upper;     // levels of the lower / upper halves
    int write_lower;      // Down Triangle: store the lower half's last row
    const T *flank_in;
    T *flank_out;
    T *state;             // NIO planes of n
};

// Face inputs: the flux group (3 values) and the ratio of one cell.
template <class T> struct EFace {
    T q0, q1, q2, th;
};

template <class T> __device__ __forceinline__ T ef_shfl(T x, int src) { return __shfl_sync(0xffffffffu, x, src); }

template <class C>
__device__ __forceinline__ void ef_shfl_cell(typename C::T (&o)[C::NF], const typename C::T (&c)[C::NF], int src) {
#pragma unroll
    for (int f = 0; f < C::NF; ++f) o[f] = ef_shfl(c[f], src);
}

template <class O>
__device__ __forceinline__ void ef_face(const EulerK<O> &k, const EFace<typename O::T> &a, const EFace<typename O::T> &b,
                                        typename O::T (&f)[3]) {
    eu_face_flux<O>(k, a.q0, a.q1, a.q2, a.th, b.q0, b.q1, b.q2, b.th, f[0], f[1], f[2]);
}

template <int K, class C>
__global__ void __launch_bounds__(128, C::MIN_BLOCKS) k_euler_fold(EFoldArgs<typename C::T> a, EulerParams prm) {
    using T = typename C::T;
    using O = typename C::O;
    constexpr int W = 32 * K, H = W / 2, NF = C::NF;
    static_assert(K % 4 == 0, "levels are unrolled by K, which must cover whole sub-step cycles");
    const EulerK<O> k = eu_k<O>(prm);
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t M = a.tiles, NS = a.nstruct, n = a.n;
    const int64_t b0 = gw * NS / nw, b1 = (gw + 1) * NS / nw;
    if (b0 >= b1) return;  // whole warp
    const int64_t S = a.nstruct_max;
    const int64_t plane = S * 2 * (int64_t)W;  // flank field stride
    const bool up = a.p == 0;
    const int imax = up ? a.upper : (a.lower > a.upper ? a.lower : a.upper);
    // only chains holding a structure at a domain end apply the ghost rule (warp-uniform)
    const bool edge = !a.periodic && (b0 == 0 || b1 == NS);

    T v[K][NF];
#pragma unroll
    for (int j = 0; j < K; ++j)
#pragma unroll
        for (int f = 0; f < NF; ++f) v[j][f] = T(0);
    int shift = 0;  // lanes by which the finishing structure's frame is rotated (0 or 16)

    for (int64_t t = 0; t <= b1 - b0; ++t) {
        if (up && t == b1 - b0) break;
        const bool hasL = !up && t < b1 - b0 && a.lower > 0;
        const bool hasU = (up ? t < b1 - b0 : t > 0) && a.upper > 0;
        if (!hasL && !hasU) break;  // Down Triangle: no upper half to finish
        const int64_t bL = b0 + t, bU = up ? bL : bL - 1;
        int64_t lb, rb;
        bool okL, okR;
        if (a.p & 1) {
            lb = bL - 1;
            rb = bL;
        } else {
            lb = bL;
            rb = bL + 1;
        }
        if (a.periodic) {
            lb = (lb + M) % M;
            rb = rb % M;
            okL = okR = true;
        } else {
            okL = lb >= 0;
            okR = rb <= ((a.p & 1) ? M - 1 : M);
        }
        // a missing neighbour (transmissive domain end) feeds only cells outside [0, n):
        // read any valid entry instead
        const T *srcL = a.flank_in + flank_off<T>(S, W, 0, (hasL && okL) ? lb : 0, 1);
        const T *srcR = a.flank_in + flank_off<T>(S, W, 0, (hasL && okR) ? rb : 0, 0);
        T *dU0 = a.flank_out + flank_off<T>(S, W, 0, bU < 0 ? 0 : bU, 0);
        T *dU1 = a.flank_out + flank_off<T>(S, W, 0, bU < 0 ? 0 : bU, 1);
        T *dL0 = a.flank_out + flank_off<T>(S, W, 0, bL % S, 0);
        T *dL1 = a.flank_out + flank_off<T>(S, W, 0, bL % S, 1);
        const int64_t startL = (a.p & 1) ? bL * W - H : bL * W;  // first cell of the starting structure's window
        const int64_t startU = up ? bU * W : startL - W;          // ... of the finishing structure's

        if (up) {
            const int64_t base = bU * W + (int64_t)lane * K;
#pragma unroll
            for (int j = 0; j < K; ++j) {
#pragma unroll
                for (int f = 0; f < NF; ++f) v[j][f] = f < C::NIO ? a.state[f * n + base + j] : T(0);
            }
            if (lane == 0) {
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    dU0[f * plane + 0] = v[0][f];
                    dU0[f * plane + 1] = v[1][f];
                }
            }
            if (lane == 31) {
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    dU1[f * plane + 0] = v[K - 2][f];
                    dU1[f * plane + 1] = v[K - 1][f];
                }
            }
        }

        // global cell of window position z (current frame) at level i, or -2^62 when no region holds it
        auto gcell = [&](int z, int i) -> int64_t {
            z &= W - 1;
            if (hasU && i <= a.upper && z >= i && z <= W - 1 - i) return startU + z;
            if (!up && hasL && i <= a.lower && (z >= W - i || z <= i - 1)) return startL + H + (z < H ? z : z - W);
            return INT64_MIN / 2;
        };

        // flank entries 2(i-1)+k arrive in chunks of 32 (16 levels), one per lane and side; each lane
        // also evaluates the pressure of its entries in the field group its level's ratio sub-step reads
        T cL[NF], cR[NF], pcL = T(0), pcR = T(0);
#pragma unroll
        for (int f = 0; f < NF; ++f) cL[f] = cR[f] = T(0);
        const int pg = ((lane >> 1) & 2) ? C::QS : 0;  // entry level e = 16c + lane/2: kind e % 4

        for (int g = 0; g * K < imax; ++g) {
#pragma unroll
            for (int u = 0; u < K; ++u) {
                const int i = g * K + u + 1;  // level within the phase half, 1..H
                if (i > imax) break;
                const bool Lact = hasL && i <= a.lower;
                const bool Uact = hasU && i <= a.upper;
                const int e = i - 1;
                if (hasL && (e & 15) == 0) {
                    const int c = e >> 4;
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        cL[f] = srcL[f * plane + 32 * c + lane];
                        cR[f] = srcR[f * plane + 32 * c + lane];
                    }
                    const T l0 = pg ? cL[C::QS] : cL[0], l1 = pg ? cL[C::QS + 1] : cL[1], l2 = pg ? cL[C::QS + 2] : cL[2];
                    const T r0 = pg ? cR[C::QS] : cR[0], r1 = pg ? cR[C::QS + 1] : cR[1], r2 = pg ? cR[C::QS + 2] : cR[2];
                    pcL = eu_pressure<O>(k, l0, l1, l2);
                    pcR = eu_pressure<O>(k, r0, r1, r2);
                }
                const int eo = 2 * (e & 15);
                const bool first = (u == 0) && (g == 0);  // i == 1
                const int sA = K - 1 - u, sB = (K - u) % K, sC = u, sD = (u + K - 1) % K;
                const int lA = (31 - g + shift) & 31;
                const int lB = (((u == 0) ? 32 : 31) - g + shift) & 31;
                const int lC = (g + shift) & 31;
                const int lD = (((u == 0) ? g - 1 : g) + shift + 32) & 31;
                const bool pA = Lact && lane == lA;
                const bool pC = Lact && lane == lC;
                // the seam cells' own state at the previous level comes from the flanks
                T fl1[NF], fr0[NF];
                ef_shfl_cell<C>(fl1, cL, eo + 1);
                ef_shfl_cell<C>(fr0, cR, eo);
                const int zl = lane * K - shift * K;  // window position of slot 0 (mod W)

                if ((u & 3) == 0 || (u & 3) == 2) {
                    // ------------------------------------------------ pressure ratio
                    const int G = ((u & 3) == 0) ? 0 : C::QS;
                    T P[K];
#pragma unroll
                    for (int j = 0; j < K; ++j) P[j] = eu_pressure<O>(k, v[j][G], v[j][G + 1], v[j][G + 2]);
                    const T Pl = ef_shfl(P[K - 1], (lane + 31) & 31);
                    const T Pr = ef_shfl(P[0], (lane + 1) & 31);
                    const T pfl0 = ef_shfl(pcL, eo), pfl1 = ef_shfl(pcL, eo + 1);
                    const T pfr0 = ef_shfl(pcR, eo), pfr1 = ef_shfl(pcR, eo + 1);
                    const bool pB = Lact && !first && lane == lB;
                    const bool pD = Lact && !first && lane == lD;
#pragma unroll
                    for (int j = 0; j < K; ++j) {
                        T x = (j == 0) ? Pl : P[j - 1];
                        T c = P[j];
                        T y = (j == K - 1) ? Pr : P[j + 1];
                        if (j == sA) {
                            x = pA ? pfl0 : x;
                            c = pA ? pfl1 : c;
                            if (first) y = pA ? pfr0 : y;
                        }
                        if (j == sB) x = pB ? pfl1 : x;
                        if (j == sC) {
                            c = pC ? pfr0 : c;
                            y = pC ? pfr1 : y;
                            if (first) x = pC ? pfl1 : x;
                        }
                        if (j == sD) y = pD ? pfr0 : y;
                        if (edge) {
                            const int64_t gc = gcell(zl + j, i);
                            if (gc == 0) x = c;
                            if (gc == n - 1) y = c;
                        }
                        const T th = eu_ratio<O>(x, c, y);
                        if (j == sA) {
#pragma unroll
                            for (int f = 0; f < NF; ++f) v[j][f] = pA ? fl1[f] : v[j][f];
                        }
                        if (j == sC) {
#pragma unroll
                            for (int f = 0; f < NF; ++f) v[j][f] = pC ? fr0[f] : v[j][f];
                        }
                        v[j][C::TH] = th;
                    }
                } else {
                    // ------------------------------------------------ flux sub-step
                    const int G = ((u & 3) == 1) ? 0 : C::QS;
                    const bool pB = Lact && lane == lB;  // on the first level this is the lane of C
                    EFace<T> fl0{ef_shfl(cL[G], eo), ef_shfl(cL[G + 1], eo), ef_shfl(cL[G + 2], eo), ef_shfl(cL[C::TH], eo)};
                    EFace<T> fr1{ef_shfl(cR[G], eo + 1), ef_shfl(cR[G + 1], eo + 1), ef_shfl(cR[G + 2], eo + 1),
                                 ef_shfl(cR[C::TH], eo + 1)};
                    const EFace<T> f1{fl1[G], fl1[G + 1], fl1[G + 2], fl1[C::TH]};
                    const EFace<T> r0{fr0[G], fr0[G + 1], fr0[G + 2], fr0[C::TH]};
                    const int ln = (lane + 31) & 31;
                    const EFace<T> lin{ef_shfl(v[K - 1][G], ln), ef_shfl(v[K - 1][G + 1], ln), ef_shfl(v[K - 1][G + 2], ln),
                                       ef_shfl(v[K - 1][C::TH], ln)};
                    T Fx[K + 1][3];
#pragma unroll
                    for (int j = 0; j < K; ++j) {
                        EFace<T> lf = (j == 0) ? lin : EFace<T>{v[j - 1][G], v[j - 1][G + 1], v[j - 1][G + 2], v[j - 1][C::TH]};
                        EFace<T> rf{v[j][G], v[j][G + 1], v[j][G + 2], v[j][C::TH]};
                        if (j == sB && pB) lf = f1;
                        if (j == sC && pC) rf = r0;
                        if (edge) {
                            const int z = (zl + j) & (W - 1);
                            const bool isA = Lact && z == ((W - i) & (W - 1));
                            const bool zmC = Lact && ((z - 1) & (W - 1)) == ((i - 1) & (W - 1));
                            if (gcell(z, i) == 0 && !isA) lf = EFace<T>{rf.q0, rf.q1, rf.q2, T(0)};
                            if (gcell(z - 1, i) == n - 1 && !zmC) rf = EFace<T>{lf.q0, lf.q1, lf.q2, T(0)};
                        }
                        ef_face<O>(k, lf, rf, Fx[j]);
                    }
                    // spare face slot: lane of A -> (fl0, fl1), lane of C -> (fr0, fr1)
                    EFace<T> ea = pC ? r0 : fl0, eb = pC ? fr1 : f1;
                    if (edge) {
                        if (pA && gcell(zl + sA, i) == 0) ea = EFace<T>{eb.q0, eb.q1, eb.q2, T(0)};
                        if (pC && gcell(zl + sC, i) == n - 1) eb = EFace<T>{ea.q0, ea.q1, ea.q2, T(0)};
                    }
                    T E[3];
                    ef_face<O>(k, ea, eb, E);
                    const int rn = (lane + 1) & 31;
                    Fx[K][0] = ef_shfl(Fx[0][0], rn);
                    Fx[K][1] = ef_shfl(Fx[0][1], rn);
                    Fx[K][2] = ef_shfl(Fx[0][2], rn);
#pragma unroll
                    for (int j = 0; j < K; ++j) {
                        T d[3];
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            const T Lq = (j == sA && pA) ? E[q] : Fx[j][q];
                            const T Rq = (j == sC && pC) ? E[q] : Fx[j + 1][q];
                            d[q] = O::sub(Rq, Lq);
                        }
                        if (j == sA) {
#pragma unroll
                            for (int f = 0; f < NF; ++f) v[j][f] = pA ? fl1[f] : v[j][f];
                        }
                        if (j == sC) {
#pragma unroll
                            for (int f = 0; f < NF; ++f) v[j][f] = pC ? fr0[f] : v[j][f];
                        }
                        if ((u & 3) == 1) C::predict(v[j], k, d);
                        else C::final_(v[j], k, d);
                    }
                }

                // flank entries of the finishing structure at level F + i (j = i)
                if (Uact && i <= H - 1) {
                    {   // z = i  -> left flank [2i]
                        const int s = (u + 1) % K, lz = g + (u + 1) / K;
                        if (lane == ((lz + shift) & 31)) {
#pragma unroll
                            for (int f = 0; f < NF; ++f) dU0[f * plane + 2 * i] = v[s][f];
                        }
                    }
                    {   // z = i + 1 -> left flank [2i + 1]
                        const int s = (u + 2) % K, lz = g + (u + 2) / K;
                        if (lane == ((lz + shift) & 31)) {
#pragma unroll
                            for (int f = 0; f < NF; ++f) dU0[f * plane + 2 * i + 1] = v[s][f];
                        }
                    }
                    {   // z = W - 2 - i -> right flank [2i]
                        const int q = K - 3 - u;
                        const int s = (q % K + K) % K, lz = 31 - g + (q < 0 ? -1 : 0);
                        if (lane == ((lz + shift + 32) & 31)) {
#pragma unroll
                            for (int f = 0; f < NF; ++f) dU1[f * plane + 2 * i] = v[s][f];
                        }
                    }
                    {   // z = W - 1 - i -> right flank [2i + 1]
                        const int q = K - 2 - u;
                        const int s = (q % K + K) % K, lz = 31 - g + (q < 0 ? -1 : 0);
                        if (lane == ((lz + shift + 32) & 31)) {
#pragma unroll
                            for (int f = 0; f < NF; ++f) dU1[f * plane + 2 * i + 1] = v[s][f];
                        }
                    }
                }
                // the starting structure's full row (level F): its flank entries j = 0
                if (Lact && i == H && a.upper > 0) {
                    if (lane == ((16 + shift) & 31)) {
#pragma unroll
                        for (int f = 0; f < NF; ++f) {
                            dL0[f * plane + 0] = v[0][f];
                            dL0[f * plane + 1] = v[1 % K][f];
                        }
                    }
                    if (lane == ((15 + shift) & 31)) {
#pragma unroll
                        for (int f = 0; f < NF; ++f) {
                            dL1[f * plane + 0] = v[K - 2][f];
                            dL1[f * plane + 1] = v[K - 1][f];
                        }
                    }
                }
            }
        }
        // Down Triangle: the lower half ends at the run's last level; store its row
        if (a.write_lower && hasL) {
            const int lw = a.lower;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                int z = lane * K + j - shift * K;
                if (z < 0) z += W;
                if (z >= W - lw || z <= lw - 1) {
                    int64_t cell = startL + H + (z < H ? z : z - W);
                    if (a.periodic) {
                        cell %= n;
                        if (cell < 0) cell += n;
                    }
                    if (cell >= 0 && cell < n) {
#pragma unroll
                        for (int f = 0; f < C::NIO; ++f) a.state[f * n + cell] = v[j][f];
                    }
                }
            }
        }
        if (!up) shift ^= 16;
    }
}

}  // namespace sw
