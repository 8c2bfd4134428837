// heat2d.cu -- the swept rule in two dimensions for the FTCS heat equation
// (5-point stencil): Section 6 names the extension to two dimensions as future
// work. Entry points sw2d_* (include/swept.h), the per-step kernel, and the
// three swept kernels with their host planner.
//
// The decomposition is the product of two 1D swept decompositions (Section 4.1).
// Per dimension, phase p has structures centred at c_p(b) = b*W + (p even ? W/2 : 0);
// between the full levels F_{p-1} and F_p = p*H (H = W/2), at local step i, the
// line is cut into lower windows of phase p, [c - i, c + i - 1] (widening), and
// upper windows of phase p - 1, [c' - H + i, c' + H - 1 - i] (narrowing). The
// plane is cut into the four products:
//   pyramid     upper x upper   needs nothing from outside (phase p - 1's octahedra
//                               compute them, as their upper part)
//   x-bridge    lower x upper   imports the two outermost columns of the pyramids
//                               left and right of it, level by level
//   y-bridge    upper x lower   imports the two outermost rows of the pyramids
//                               below and above it
//   octahedron  lower x lower   imports the bridges' outermost columns / rows and
//                               three corner cells of the four diagonal pyramids;
//                               at i = H it is the full tile at F_p, and it then
//                               narrows again as the pyramid of phase p.
// A phase is a bridges launch and an octahedra launch; the first launch builds
// the pyramids of phase 0 from the state ("Up"), the last octahedra stop at the
// full level and store the tiles ("Down"). Every (cell, level) is computed once.
// Strips: per region, side and step, 2 x W values (the 2-cell-deep edge of its
// window at that step, 256-byte granularity per buffer), written by one launch and
// read by the next, double-buffered by phase for the pyramids.
//
// Shared memory: one frame of (W+2) x (W+3) positions around a region's centre
// (W+3: an odd row stride, so column reads of the strips spread over the banks),
// two level slots; a level is computed into slot (level & 1) from the other.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/swept.h"
#include "common.cuh"
#include "fp64_soft2d.cuh"

using namespace sw;

namespace {

// The per-cell update (the same function in every kernel, so swept and per-step
// runs agree bit for bit): fma(rx, fma(-2, u, a + b), fma(ry, fma(-2, u, d + e), u)).
template <class O>
__device__ __forceinline__ typename O::T heat2d_update(typename O::T rx, typename O::T ry, typename O::T a,
                                                       typename O::T b, typename O::T u, typename O::T d,
                                                       typename O::T e) {
    using T = typename O::T;
    const T yd = O::fma_(T(-2), u, O::add(d, e));
    const T xd = O::fma_(T(-2), u, O::add(a, b));
    return O::fma_(rx, xd, O::fma_(ry, yd, u));
}

template <class T> struct Ops2D;
template <> struct Ops2D<double> { using O = OpsD; };
template <> struct Ops2D<float> { using O = OpsF; };

// FP64: half the cells go through the integer pipes (soft64::heat2d_update, the same bits as
// the FP64 instructions give; FP64 issues at 1/32 of the integer rate on GB300, so a 2D update
// of 6 FP64 instructions leaves the integer pipes idle). A cell outside the integer path's
// range (mixed signs, a neighbour far from u in magnitude, a result leaving u's binade) is
// evaluated here instead, out of line, so that its FP64 instructions issue only when a lane
// of the warp needs them.
__device__ __noinline__ double heat2d_update_fp64(double rx, double ry, double a, double b, double u, double d,
                                                 double e) {
    return heat2d_update<OpsD>(rx, ry, a, b, u, d, e);
}
__device__ __forceinline__ double heat2d_update_int(const soft64::HeatR &hx, const soft64::HeatR &hy, double rx,
                                                    double ry, double a, double b, double u, double d, double e) {
    bool ok;
    const uint64_t v = soft64::heat2d_update(hx, hy, soft64::bits(a), soft64::bits(b), soft64::bits(u),
                                             soft64::bits(d), soft64::bits(e), ok);
    return ok ? soft64::value(v) : heat2d_update_fp64(rx, ry, a, b, u, d, e);
}

constexpr int kThreads2D = 256;       // per-step kernel; FP64 swept kernels; FP32 bridges at W >= 128
constexpr int kThreads2DWide = 1024;  // FP32 Up / octahedra at W >= 128: one CTA per SM fits the frame

// Threads of a swept CTA. The kernels are instantiated for 128, 256 and 1024 threads
// (sw2d_set_threads), each with a launch bound that keeps the resident-CTA count the frame's
// shared memory allows at W = 64 (FP32: 6 per SM, FP64: 3; one at 1024). Defaults, measured
// on 8192^2 x 2048 steps: FP32 below W = 128, 128 threads (six CTAs per SM at W = 64: fewer
// threads give each more cells per level against the per-level costs; 843 against 730
// Gcell-updates/s with 256); FP32 from W = 128 (one CTA per SM), 1024 for the Up and
// octahedra launches and 256 for the bridges; FP64, 256 (bound by its pipe; 90.4 against
// 89.4 with 128).
__host__ __device__ constexpr int swept_threads2d(size_t es, int W, bool bridges) {
    return es == 8 ? kThreads2D : (W < 128 ? 128 : (bridges ? kThreads2D : kThreads2DWide));
}
template <class T, int NT> constexpr int min_ctas2d() { return NT >= kThreads2DWide ? 1 : (sizeof(T) == 4 ? 6 : 3); }

// Swept kernels compiled for one tile width WC (0: W read from the arguments). With W a
// constant, the frame's row stride, the slot size and the strip offsets are immediates, which
// takes the shared-memory address arithmetic out of the FP32 walker's inner loop (FP32 is
// bound by instruction issue; FP64 by its pipe, so it keeps the generic form). Instantiated
// for FP32 at W = 32 and 64 with 128 or 256 threads, and W = 128 with 256 or 1024.
template <class T, int NT, int WC> constexpr bool specialised2d() {
    return sizeof(T) == 4 && (((WC == 32 || WC == 64) && (NT == 128 || NT == kThreads2D)) ||
                              (WC == 128 && (NT == kThreads2D || NT == kThreads2DWide)));
}

// ceil(2^32 / w) for w = 2 .. kMagicMax: umulhi(t, magic[w]) = t / w while t * w < 2^32 (the
// band and column of a window's walker, the line of a strip element); filled from the host at
// sw2d_create, identical on every device
constexpr int kMagicMax = 1026;
__constant__ unsigned c_magic[kMagicMax + 1];


// ------------------------------------------------------------------ per-step
// V consecutive cells of a row as 16-byte vector accesses (VEC) or scalars.
template <class T, int V, bool VEC> struct RowIO {
    static __device__ __forceinline__ void load(const T *p, T (&x)[V]) {
#pragma unroll
        for (int k = 0; k < V; ++k) x[k] = p[k];
    }
    static __device__ __forceinline__ void store(T *p, const T (&x)[V]) {
#pragma unroll
        for (int k = 0; k < V; ++k) p[k] = x[k];
    }
};
template <> struct RowIO<float, 4, true> {
    static __device__ __forceinline__ void load(const float *p, float (&x)[4]) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
    static __device__ __forceinline__ void store(float *p, const float (&x)[4]) {
        *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
    }
};
template <> struct RowIO<double, 4, true> {
    static __device__ __forceinline__ void load(const double *p, double (&x)[4]) {
        const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
        x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
    }
    static __device__ __forceinline__ void store(double *p, const double (&x)[4]) {
        reinterpret_cast<double2 *>(p)[0] = make_double2(x[0], x[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(x[2], x[3]);
    }
};

// One step over the whole grid: each thread takes V consecutive cells of a row (item
// = row * (nx / V) + chunk, grid-stride); x-neighbours at the chunk's ends and the
// rows above and below come through the caches. VEC: the row pieces move as 16-byte
// vectors (the launcher checks the alignment of the state and of nx). FP64 with V = 4:
// cells 1 and 3 of every thread on the integer pipes, 0 and 2 on the FP64 pipe.
template <class T, int V, bool VEC>
__global__ void __launch_bounds__(kThreads2D) k2d_step(const T *__restrict__ in, T *__restrict__ out, int64_t nx,
                                                       int64_t ny, T rx, T ry, int periodic, soft64::HeatR hx,
                                                       soft64::HeatR hy) {
    using O = typename Ops2D<T>::O;
    using IO = RowIO<T, V, VEC>;
    const int64_t chunks = nx / V, items = chunks * ny;
    for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < items;
         it += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = it / chunks, i0 = (it - j * chunks) * V;
        const int64_t jd = j > 0 ? j - 1 : (periodic ? ny - 1 : 0);
        const int64_t ju = j < ny - 1 ? j + 1 : (periodic ? 0 : ny - 1);
        const T *row = in + j * nx, *rd = in + jd * nx, *ru = in + ju * nx;
        T c[V], d[V], e[V];
        IO::load(row + i0, c);
        IO::load(rd + i0, d);
        IO::load(ru + i0, e);
        const T left = i0 > 0 ? row[i0 - 1] : (periodic ? row[nx - 1] : c[0]);
        const T right = i0 + V < nx ? row[i0 + V] : (periodic ? row[0] : c[V - 1]);
        T o[V];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const T a = k > 0 ? c[k - 1] : left;
            const T b = k < V - 1 ? c[k + 1] : right;
            if constexpr (sizeof(T) == 8 && V == 4) {
                if (k & 1) {
                    o[k] = heat2d_update_int(hx, hy, rx, ry, a, b, c[k], d[k], e[k]);
                    continue;
                }
            }
            o[k] = heat2d_update<O>(rx, ry, a, b, c[k], d[k], e[k]);
        }
        IO::store(out + j * nx + i0, o);
    }
}

// ------------------------------------------------------------------ swept
template <class T> struct Swept2DArgs {
    int64_t nx, ny;
    int Mx, My, W, H;
    int p;              // phase index
    int64_t F;          // full level of phase p (p * H)
    int last;           // octahedra: the last phase (store the tiles, no pyramid after)
    T *state;
    const T *pin_x, *pin_y;  // pyramid strips of phase p - 1
    T *pout_x, *pout_y;      // pyramid strips of phase p
    T *brx, *bry;            // bridge strips of phase p
    T rx, ry;
    soft64::HeatR hrx, hry;  // rx, ry unpacked for the integer path (FP64)
};

__device__ __forceinline__ int centre2d(int p, int b, int W) { return b * W + ((p & 1) ? 0 : W / 2); }

// phase p - 1 neighbours (centred at c - H and c + H) of structure b of phase p
__device__ __forceinline__ void nbrs(int p, int b, int M, int &lo, int &hi) {
    if (p & 1) {
        lo = (b - 1 + M) % M;
        hi = b % M;
    } else {
        lo = b % M;
        hi = (b + 1) % M;
    }
}

// Strips: one buffer holds, per tile, 2 sides x H steps x 2 lines x W values; element
// (tile, side, step i, line k, r) sits at ((tile * 2 + side) * H + i) * 2W + k * W + r. A
// kernel forms the 64-bit base of each strip block it touches once and indexes the rest
// (below 4 * H * W) in 32 bits.
template <class T> __device__ __forceinline__ T *strip_block(T *buf, int tile, int side, int H, int W) {
    return buf + ((int64_t)tile * 2 + side) * H * 2 * W;
}
__device__ __forceinline__ int strip_at(int i, int k, int W) { return (i * 2 + k) * W; }

// The shared frame of a region centred at (cx, cy), in local coordinates: the absolute
// (unwrapped) position (x, y) is (X, Y) = (x - cx + H + 1, y - cy + H + 1), 0 <= X, Y <= W + 1.
// Window bounds at step i in local coordinates: upper (narrowing) [i + 1, W - i], lower
// (widening) [H + 1 - i, H + i].
template <class T> struct Frame {
    T *s;
    int RS, slot;
    __device__ __forceinline__ int idx(int64_t lev, int X, int Y) const { return ((int)lev & 1) * slot + Y * RS + X; }
    __device__ __forceinline__ T &at(int64_t lev, int X, int Y) const { return s[idx(lev, X, Y)]; }
};

// `LINES` strip lines of `len` elements each over a block of NT threads, packed: element t
// of the block's LINES * len is (line t / len, entry t % len), so consecutive threads take
// consecutive entries across line ends and short lines leave no lane idle (measured ahead of
// one line per warp in FP32, where issue slots bind). t * len < 2^32: t < 8 * (W + 2).
template <int NT, int LINES, class Fn> __device__ __forceinline__ void over_lines(int len, Fn &&fn) {
    const unsigned m = c_magic[len];  // len >= 2 whenever the loop runs
    for (int t = (int)threadIdx.x; t < LINES * len; t += NT) {
        const int q = (int)__umulhi((unsigned)t, m), r = t - q * len;
        fn(q, r);
    }
}

// A strip injection in two halves, so that the loads of a level's inputs overlap the compute
// of the level before: fetch() reads this thread's first E entries of the LINES x len strip
// entries (packed as in over_lines) into registers together with their frame indices, put()
// writes them into the frame after the compute and takes any entries beyond E x NT directly.
// get(q, r): the entry's value; where(q, r): its index in the frame's storage.
template <class T, int NT, int LINES, int E> struct Staged {
    T v[E];
    int pos[E];
    template <class Get, class Where> __device__ __forceinline__ void fetch(int len, Get &&get, Where &&where) {
        const unsigned m = c_magic[len];
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const int t = (int)threadIdx.x + j * NT;
            v[j] = T(0);
            pos[j] = -1;
            if (t < LINES * len) {
                const int q = (int)__umulhi((unsigned)t, m), r = t - q * len;
                v[j] = get(q, r);
                pos[j] = where(q, r);
            }
        }
    }
    template <class Get, class Where>
    __device__ __forceinline__ void put(T *s, int len, Get &&get, Where &&where) const {
#pragma unroll
        for (int j = 0; j < E; ++j)
            if (pos[j] >= 0) s[pos[j]] = v[j];
        if (LINES * len > E * NT) {
            const unsigned m = c_magic[len];
            for (int t = (int)threadIdx.x + E * NT; t < LINES * len; t += NT) {
                const int q = (int)__umulhi((unsigned)t, m), r = t - q * len;
                s[where(q, r)] = get(q, r);
            }
        }
    }
};

__device__ __forceinline__ int64_t wrap(int64_t x, int64_t n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// compute the window [X0, X1] x [Y0, Y1] (local) at level lev from lev - 1 with a block of
// NT threads. The quotients come from the constant table (t * w < 2^32 throughout: t < (W +
// 2)^2 <= 120^2 for FP64, t < NT for FP32).
//  FP64 (bound by the FP64 pipe, which is paid per warp instruction): the threads run over
//    the window's cells in row-major order, consecutive threads on consecutive cells, so
//    every warp instruction but the last of a level has all 32 lanes busy.
//  FP32 (bound by instruction issue): each thread walks down one column over a band of
//    consecutive rows: nb = min(h, floor(NT / w)) bands of ceil(h / nb) rows per column,
//    consecutive threads on consecutive columns (a warp's shared-memory accesses are
//    consecutive). The walker carries the cell above and the cell itself in registers, so
//    a cell costs three shared loads (left, right, below) and one store, and the row
//    mapping is paid once per band instead of once per cell; four rows are loaded before
//    any of them is stored.
template <int NT, class T>
__device__ __forceinline__ void compute_window(const Frame<T> &f, int64_t lev, int X0, int X1, int Y0, int Y1, T rx,
                                               T ry, const soft64::HeatR &hx, const soft64::HeatR &hy) {
    using O = typename Ops2D<T>::O;
    const int RS = f.RS;
    const T *src = f.s + (((int)lev - 1) & 1) * f.slot;
    T *dst = f.s + ((int)lev & 1) * f.slot;
    const unsigned w = (unsigned)(X1 - X0 + 1), h = (unsigned)(Y1 - Y0 + 1);  // both >= 2
    if constexpr (sizeof(T) == 8) {
        const unsigned cnt = w * h, m = c_magic[w];
        const int org = Y0 * RS + X0;
        // Cells in pairs t, t + nt: the first on the integer pipes, the second on the FP64 pipe
        // (uniform over the warp; a window smaller than two rounds of the block thus leans to the
        // integer pipes, which the FP64-bound kernel has to spare). The stride is read from
        // blockDim, not the compile-time NT: with a constant stride the unrolled loop ran 7 %
        // slower (FP64 pipe only, W = 64, 8192^2).
        const unsigned nt = blockDim.x;
#pragma unroll 2
        for (unsigned t = threadIdx.x; t < cnt; t += 2 * nt) {
            {
                const unsigned yy = __umulhi(t, m), xx = t - yy * w;
                const int q = org + (int)yy * RS + (int)xx;
                dst[q] = heat2d_update_int(hx, hy, rx, ry, src[q - 1], src[q + 1], src[q], src[q - RS], src[q + RS]);
            }
            const unsigned t2 = t + nt;
            if (t2 < cnt) {
                const unsigned yy = __umulhi(t2, m), xx = t2 - yy * w;
                const int q = org + (int)yy * RS + (int)xx;
                dst[q] = heat2d_update<O>(rx, ry, src[q - 1], src[q + 1], src[q], src[q - RS], src[q + RS]);
            }
        }
    } else {
        const unsigned nb = min(max(__umulhi(NT, c_magic[w]), 1u), h);
        const unsigned L = nb == 1 ? h : __umulhi(h + nb - 1, c_magic[nb]);
        const unsigned t = threadIdx.x;
        if (t >= w * nb) return;
        const unsigned band = __umulhi(t, c_magic[w]), col = t - band * w;
        const unsigned ya = band * L;
        if (ya >= h) return;
        const int rows = (int)(min(h, ya + L) - ya);
        int q = (Y0 + (int)ya) * RS + X0 + (int)col;
        T up = src[q - RS], c = src[q];
        int y = 0;
        for (; y + 4 <= rows; y += 4) {
            T l[4], r[4], d[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                l[k] = src[q + k * RS - 1];
                r[k] = src[q + k * RS + 1];
                d[k] = src[q + (k + 1) * RS];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                dst[q + k * RS] = heat2d_update<O>(rx, ry, l[k], r[k], c, up, d[k]);
                up = c;
                c = d[k];
            }
            q += 4 * RS;
        }
        for (; y < rows; ++y) {
            const T dn = src[q + RS];
            dst[q] = heat2d_update<O>(rx, ry, src[q - 1], src[q + 1], c, up, dn);
            up = c;
            c = dn;
            q += RS;
        }
    }
}

// export the 2-deep edges of the pyramid window at step i, [i + 1, W - i]^2 (local): line q
// < 4 is an x-strip (columns i+1+k / W-i-1+k over the window's rows), q >= 4 a y-strip (rows
// over its columns); side = (q >> 1) & 1, k = q & 1. sxb / syb: this tile's strip blocks.
template <int NT, class T>
__device__ __forceinline__ void export_pyramid(const Frame<T> &f, int64_t lev, int i, int H, int W, T *sxb,
                                               T *syb) {
    over_lines<NT, 8>(W - 2 * i, [&](int q, int r) {
        const int side = (q >> 1) & 1, k = q & 1;
        const int edge = side == 0 ? i + 1 + k : W - i - 1 + k;
        const int off = strip_at(side * H + i, k, W) + r;
        if (q < 4) sxb[off] = f.at(lev, edge, i + 1 + r);
        else syb[off] = f.at(lev, i + 1 + r, edge);
    });
}

// The upper part of a structure (the pyramid): steps 0..H-1 from the full tile at level F
// (already in the frame), exporting both kinds of strips per step.
template <int NT, class T>
__device__ void pyramid_part(const Frame<T> &f, const Swept2DArgs<T> &a, int W, int H, int64_t F, int tile, T *sx,
                             T *sy) {
    T *sxb = strip_block(sx, tile, 0, H, W), *syb = strip_block(sy, tile, 0, H, W);
    export_pyramid<NT>(f, F, 0, H, W, sxb, syb);
    for (int i = 1; i < H; ++i) {
        compute_window<NT>(f, F + i, i + 1, W - i, i + 1, W - i, a.rx, a.ry, a.hrx, a.hry);
        __syncthreads();
        export_pyramid<NT>(f, F + i, i, H, W, sxb, syb);
    }
}

// Up: the pyramids of phase 0 from the state (level 0); a warp per row of the tile
template <class T, int NT, int WC>
__global__ void __launch_bounds__(NT, (min_ctas2d<T, NT>())) k2d_up(Swept2DArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int bx = blockIdx.x % a.Mx, by = blockIdx.x / a.Mx;
    const int W = WC ? WC : a.W, H = W / 2;
    const Frame<T> f{reinterpret_cast<T *>(smem_raw), W + 3, (W + 2) * (W + 3)};
    const int64_t gx0 = (int64_t)centre2d(0, bx, W) - H, gy0 = (int64_t)centre2d(0, by, W) - H;
    for (int Y = 1 + (int)(threadIdx.x >> 5); Y <= W; Y += NT / 32) {
        const T *row = a.state + wrap(gy0 + Y - 1, a.ny) * a.nx;
        for (int X = 1 + (int)(threadIdx.x & 31); X <= W; X += 32) f.at(0, X, Y) = row[wrap(gx0 + X - 1, a.nx)];
    }
    __syncthreads();
    pyramid_part<NT>(f, a, W, H, 0, blockIdx.x, a.pout_x, a.pout_y);
}

// Bridges of phase p: blockIdx.y = 0 x-bridges (lower in x, upper in y), 1 y-bridges.
template <class T, int NT, int WC>
__global__ void __launch_bounds__(NT, (min_ctas2d<T, NT>())) k2d_bridges(Swept2DArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b0 = blockIdx.x % a.Mx, b1 = blockIdx.x / a.Mx;  // (x index, y index)
    const int W = WC ? WC : a.W, H = W / 2;
    const bool xb = blockIdx.y == 0;
    const Frame<T> f{reinterpret_cast<T *>(smem_raw), W + 3, (W + 2) * (W + 3)};
    int lo, hi;  // the two pyramids it imports from (phase p - 1 indices along its lower direction)
    nbrs(a.p, xb ? b0 : b1, xb ? a.Mx : a.My, lo, hi);
    const int tlo = xb ? b1 * a.Mx + lo : lo * a.Mx + b0;
    const int thi = xb ? b1 * a.Mx + hi : hi * a.Mx + b0;
    // the low-side pyramid exports its high side (1), the high-side pyramid its low side (0)
    const T *src = xb ? a.pin_x : a.pin_y;
    const T *plo = strip_block(src, tlo, 1, H, W), *phi = strip_block(src, thi, 0, H, W);
    T *dst = strip_block(xb ? a.brx : a.bry, blockIdx.x, 0, H, W);
    const int64_t base = a.F - H;  // level of step 0
    // step i's inputs at level base + i - 1: the pyramids' strips at step i - 1, all of
    // their W - 2(i-1) entries (rows i + r for an x-bridge, columns for a y-bridge); line q:
    // k = q & 1, high-side neighbour q >> 1
    // (staged: step i + 1's strip loads are issued before step i's compute and written after it,
    // to positions of the slot being written that lie outside step i's window)
    int si = 1;  // the step whose inputs get() / where() address
    auto get = [&](int q, int r) { return ((q >> 1) ? phi : plo)[strip_at(si - 1, q & 1, W) + r]; };
    auto where = [&](int q, int r) {
        const int across = (q >> 1) ? H + si + (q & 1) : H - si + (q & 1);
        return xb ? f.idx(base + si - 1, across, si + r) : f.idx(base + si - 1, si + r, across);
    };
    Staged<T, NT, 4, 2> stage;
    stage.fetch(W, get, where);
    stage.put(f.s, W, get, where);
    __syncthreads();
    for (int i = 1; i < H; ++i) {
        si = i + 1;
        if (si < H) stage.fetch(W - 2 * i, get, where);
        // the widening direction's window [H + 1 - i, H + i], the narrowing one's [i + 1, W - i]
        if (xb) compute_window<NT>(f, base + i, H + 1 - i, H + i, i + 1, W - i, a.rx, a.ry, a.hrx, a.hry);
        else compute_window<NT>(f, base + i, i + 1, W - i, H + 1 - i, H + i, a.rx, a.ry, a.hrx, a.hry);
        if (si < H) stage.put(f.s, W - 2 * i, get, where);
        __syncthreads();
        // export the edges along the widening direction's normal: an x-bridge its bottom and
        // top two rows (2i columns), a y-bridge its left and right two columns (2i rows);
        // line q: k = q & 1, side q >> 1
        over_lines<NT, 4>(2 * i, [&](int q, int r) {
            const int k = q & 1, side = q >> 1;
            const int edge = side == 0 ? i + 1 + k : W - i - 1 + k;
            const T v = xb ? f.at(base + i, H + 1 - i + r, edge) : f.at(base + i, edge, H + 1 - i + r);
            dst[strip_at(side * H + i, k, W) + r] = v;
        });
    }
}

// Octahedra of phase p: the lower part (lower x lower) up to the full tile at F, then the
// pyramid of phase p (or, in the last phase, the tile stored to the state).
template <class T, int NT, int WC>
__global__ void __launch_bounds__(NT, (min_ctas2d<T, NT>())) k2d_octa(Swept2DArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int bx = blockIdx.x % a.Mx, by = blockIdx.x / a.Mx;
    const int W = WC ? WC : a.W, H = W / 2;
    const Frame<T> f{reinterpret_cast<T *>(smem_raw), W + 3, (W + 2) * (W + 3)};
    int lx, rx, lb, rt;
    nbrs(a.p, bx, a.Mx, lx, rx);
    nbrs(a.p, by, a.My, lb, rt);
    // the bridges' strips it imports: the y-bridges left (their right side) and right (their
    // left side), the x-bridges below (their top side) and above (their bottom side)
    const T *pl = strip_block(a.bry, by * a.Mx + lx, 1, H, W), *pr = strip_block(a.bry, by * a.Mx + rx, 0, H, W);
    const T *pb = strip_block(a.brx, lb * a.Mx + bx, 1, H, W), *pt = strip_block(a.brx, rt * a.Mx + bx, 0, H, W);
    const int64_t base = a.F - H;
    // step i's inputs at level base + i - 1, staged as in the bridges: line q of 2(i - 1)
    // entries, k = q & 1, which = q >> 1 (0 left, 1 right, 2 below, 3 above)
    int si = 1;
    auto get = [&](int q, int r) {
        const int which = q >> 1;
        const T *sb = which == 0 ? pl : which == 1 ? pr : which == 2 ? pb : pt;
        return sb[strip_at(si - 1, q & 1, W) + r];
    };
    auto where = [&](int q, int r) {
        const int across = (q & 2) ? H + si + (q & 1) : H - si + (q & 1);
        return (q >> 1) < 2 ? f.idx(base + si - 1, across, H + 2 - si + r) : f.idx(base + si - 1, H + 2 - si + r, across);
    };
    // corners: from the x-strips of the four diagonal pyramids of phase p - 1 at step i - 1
    // (entry = row - the pyramid's first row at that step: H + i above, i - H below); threads
    // 0..11, three cells per corner
    T cv = T(0);
    int cpos = -1;
    auto corner = [&](int i) {
        if (threadIdx.x < 12) {
            const int c = threadIdx.x / 3, e = threadIdx.x % 3;
            const bool right = c & 1, top = c >> 1;
            const int tp = (top ? rt : lb) * a.Mx + (right ? rx : lx);
            int X, Y, k;
            if (e < 2) {  // both new columns at the corner row
                k = e;
                X = right ? H + i + k : H - i + k;
                Y = top ? H + i : H + 1 - i;
            } else {  // the inner new column, one row further out
                k = right ? 0 : 1;
                X = right ? H + i : H + 1 - i;
                Y = top ? H + i + 1 : H - i;
            }
            const int entry = top ? Y - (H + i) : Y + H - i;
            cv = strip_block(a.pin_x, tp, right ? 0 : 1, H, W)[strip_at(i - 1, k, W) + entry];
            cpos = f.idx(base + i - 1, X, Y);
        }
    };
    Staged<T, NT, 8, 2> stage;
    corner(1);  // step 1: no bridge entries yet (length 0)
    if (cpos >= 0) f.s[cpos] = cv;
    __syncthreads();
    for (int i = 1; i <= H; ++i) {
        si = i + 1;
        if (si <= H) {
            stage.fetch(2 * i, get, where);
            corner(si);
        }
        compute_window<NT>(f, base + i, H + 1 - i, H + i, H + 1 - i, H + i, a.rx, a.ry, a.hrx, a.hry);
        if (si <= H) {
            stage.put(f.s, 2 * i, get, where);
            if (cpos >= 0) f.s[cpos] = cv;
        }
        __syncthreads();
    }
    if (a.last) {  // the full tile at F, a warp per row
        const int64_t gx0 = (int64_t)centre2d(a.p, bx, W) - H, gy0 = (int64_t)centre2d(a.p, by, W) - H;
        for (int Y = 1 + (int)(threadIdx.x >> 5); Y <= W; Y += NT / 32) {
            T *row = a.state + wrap(gy0 + Y - 1, a.ny) * a.nx;
            for (int X = 1 + (int)(threadIdx.x & 31); X <= W; X += 32) row[wrap(gx0 + X - 1, a.nx)] = f.at(a.F, X, Y);
        }
        return;
    }
    pyramid_part<NT>(f, a, W, H, a.F, blockIdx.x, a.pout_x, a.pout_y);
}

int cuda_status2d(cudaError_t e) {
    if (e == cudaSuccess) return SW_OK;
    if (e == cudaErrorMemoryAllocation) return SW_ERR_OOM;
    return SW_ERR_CUDA;
}

size_t smem2d(int W, size_t es) { return size_t(2) * (W + 2) * (W + 3) * es; }

int max_width2d(size_t es) {
    int best = 0;
    for (int W = 8; W <= 1024; W += 2)
        if (smem2d(W, es) <= size_t(227) * 1024) best = W;
    return best;
}

}  // namespace

struct sw_handle2d {
    sw_heat2d prob{};
    int W = 0, H = 0, Mx = 0, My = 0;
    int nt = 0, nt_br = 0;  // threads per swept CTA: Up and octahedra, bridges
    size_t es = 0, smem = 0;
    void *pyrx[2] = {nullptr, nullptr}, *pyry[2] = {nullptr, nullptr};
    void *brx = nullptr, *bry = nullptr;
    void *plane = nullptr;  // per-step ping-pong plane
    int64_t last_launches = 0;
    std::vector<cudaEvent_t> events;
    std::vector<int32_t> kinds;
    int64_t ev_cap = 0, ev_used = 0;
};

namespace {

int validate2d(const sw_heat2d *p) {
    if (!p) return SW_ERR_BAD_ARG;
    if (p->precision != SW_FP64 && p->precision != SW_FP32) return SW_ERR_BAD_ARG;
    if (p->boundary != SW_PERIODIC && p->boundary != SW_TRANSMISSIVE) return SW_ERR_BAD_ARG;
    if (p->method != SW_SWEPT && p->method != SW_PERSTEP) return SW_ERR_BAD_ARG;
    if (p->nx < 4 || p->ny < 4 || p->nx > (int64_t(1) << 36) || p->ny > (int64_t(1) << 36) ||
        p->nx * p->ny > (int64_t(1) << 36))
        return SW_ERR_BAD_ARG;
    if (!(p->rx > 0.0) || !(p->ry > 0.0) || !(p->rx < 1e6) || !(p->ry < 1e6)) return SW_ERR_BAD_ARG;
    if (p->method == SW_SWEPT) {
        if (p->boundary != SW_PERIODIC) return SW_ERR_BAD_ARG;
        const int W = p->tile_width ? p->tile_width : 64;
        if (W < 8 || W > SW_MAX_TILE || (W & 1)) return SW_ERR_BAD_ARG;
        if (p->nx % W || p->ny % W || p->nx < 2 * (int64_t)W || p->ny < 2 * (int64_t)W) return SW_ERR_BAD_ARG;
        if (p->nx / W > (1 << 30) || p->ny / W > (1 << 30) || (p->nx / W) * (p->ny / W) > (int64_t(1) << 31))
            return SW_ERR_BAD_ARG;
    } else if (p->tile_width < 0) {
        return SW_ERR_BAD_ARG;
    }
    return SW_OK;
}

void trace2d_begin(sw_handle2d *h, int64_t i, int32_t kind, cudaStream_t st) {
    if (i < h->ev_cap) {
        cudaEventRecord(h->events[2 * i], st);
        h->kinds[i] = kind;
    }
}
void trace2d_end(sw_handle2d *h, int64_t i, cudaStream_t st) {
    if (i < h->ev_cap) {
        cudaEventRecord(h->events[2 * i + 1], st);
        h->ev_used = i + 1;
    }
}

unsigned grid2d(int64_t work, int cap) {
    int64_t g = (work + kThreads2D - 1) / kThreads2D;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

// the swept kernels of one element type, thread count and compiled width: kind 0 Up, 1
// bridges, 2 octahedra
template <class T, int NT, int WC> void launch2d_k(int kind, unsigned tiles, size_t smem, cudaStream_t st,
                                                   const Swept2DArgs<T> &a) {
    if (kind == 0) k2d_up<T, NT, WC><<<tiles, NT, smem, st>>>(a);
    else if (kind == 1) k2d_bridges<T, NT, WC><<<dim3(tiles, 2), NT, smem, st>>>(a);
    else k2d_octa<T, NT, WC><<<tiles, NT, smem, st>>>(a);
}
template <class T, int NT> void launch2d_nt(int kind, unsigned tiles, size_t smem, cudaStream_t st,
                                            const Swept2DArgs<T> &a) {
    if constexpr (specialised2d<T, NT, 32>()) {
        if (a.W == 32) return launch2d_k<T, NT, 32>(kind, tiles, smem, st, a);
    }
    if constexpr (specialised2d<T, NT, 64>()) {
        if (a.W == 64) return launch2d_k<T, NT, 64>(kind, tiles, smem, st, a);
    }
    if constexpr (specialised2d<T, NT, 128>()) {
        if (a.W == 128) return launch2d_k<T, NT, 128>(kind, tiles, smem, st, a);
    }
    launch2d_k<T, NT, 0>(kind, tiles, smem, st, a);
}
template <class T> void launch2d(int kind, int nt, unsigned tiles, size_t smem, cudaStream_t st,
                                 const Swept2DArgs<T> &a) {
    if (nt == 128) launch2d_nt<T, 128>(kind, tiles, smem, st, a);
    else if (nt == kThreads2D) launch2d_nt<T, kThreads2D>(kind, tiles, smem, st, a);
    else launch2d_nt<T, kThreads2DWide>(kind, tiles, smem, st, a);
}
// the dynamic shared-memory limit of the swept kernels of <T, NT, WC>
template <class T, int NT, int WC> cudaError_t allow_smem2d_k(size_t smem) {
    const void *fns[3] = {(const void *)k2d_up<T, NT, WC>, (const void *)k2d_bridges<T, NT, WC>,
                          (const void *)k2d_octa<T, NT, WC>};
    for (const void *fn : fns) {
        const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
// ... for the kernels a handle of width W may launch at this thread count
template <class T, int NT> cudaError_t allow_smem2d(int W, size_t smem) {
    if constexpr (specialised2d<T, NT, 32>()) {
        if (W == 32) return allow_smem2d_k<T, NT, 32>(smem);
    }
    if constexpr (specialised2d<T, NT, 64>()) {
        if (W == 64) return allow_smem2d_k<T, NT, 64>(smem);
    }
    if constexpr (specialised2d<T, NT, 128>()) {
        if (W == 128) return allow_smem2d_k<T, NT, 128>(smem);
    }
    return allow_smem2d_k<T, NT, 0>(smem);
}
template <class T> cudaError_t allow_smem2d_all(int W, size_t smem) {
    cudaError_t e = allow_smem2d<T, 128>(W, smem);
    if (e == cudaSuccess) e = allow_smem2d<T, kThreads2D>(W, smem);
    if (e == cudaSuccess) e = allow_smem2d<T, kThreads2DWide>(W, smem);
    return e;
}

// `steps` per-step launches, ping-pong between the state and the handle's plane; the
// result ends in the state
template <class T>
int run_perstep2d(sw_handle2d *h, T *state, int64_t steps, cudaStream_t st, int64_t &launches) {
    const int64_t nx = h->prob.nx, ny = h->prob.ny;
    const int periodic = h->prob.boundary == SW_PERIODIC;
    const T rx = (T)h->prob.rx, ry = (T)h->prob.ry;
    const soft64::HeatR hx = soft64::make_heat_r(h->prob.rx), hy = soft64::make_heat_r(h->prob.ry);
    T *bufs[2] = {state, reinterpret_cast<T *>(h->plane)};
    const int cap = 152 * 16;
    // 16-byte row pieces need the state (the scratch plane is 256-byte aligned) and every
    // row start on 16 bytes: nx a multiple of 4 cells
    const bool vec = nx % 4 == 0 && reinterpret_cast<uintptr_t>(state) % 16 == 0;
    for (int64_t s = 0; s < steps; ++s) {
        const T *in = bufs[s & 1];
        T *out = bufs[(s + 1) & 1];
        trace2d_begin(h, launches, 3, st);
        if (vec)
            k2d_step<T, 4, true><<<grid2d(nx / 4 * ny, cap), kThreads2D, 0, st>>>(in, out, nx, ny, rx, ry, periodic, hx,
                                                                                  hy);
        else if (nx % 4 == 0)
            k2d_step<T, 4, false><<<grid2d(nx / 4 * ny, cap), kThreads2D, 0, st>>>(in, out, nx, ny, rx, ry,
                                                                                   periodic, hx, hy);
        else
            k2d_step<T, 1, false><<<grid2d(nx * ny, cap), kThreads2D, 0, st>>>(in, out, nx, ny, rx, ry, periodic, hx,
                                                                               hy);
        trace2d_end(h, launches, st);
        ++launches;
    }
    if (steps & 1) {
        cudaError_t e = cudaMemcpyAsync(state, h->plane, size_t(nx * ny) * sizeof(T), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_status2d(e);
    }
    return SW_OK;
}

template <class T> int run2d(sw_handle2d *h, void *state_v, int64_t nsteps, cudaStream_t st) {
    T *state = reinterpret_cast<T *>(state_v);
    int64_t launches = 0;
    int rc = SW_OK;
    if (h->prob.method == SW_SWEPT) {
        const int H = h->H;
        const int64_t P = nsteps / H, R = nsteps % H;
        if (P >= 1) {
            Swept2DArgs<T> a{};
            a.nx = h->prob.nx;
            a.ny = h->prob.ny;
            a.Mx = h->Mx;
            a.My = h->My;
            a.W = h->W;
            a.H = H;
            a.state = state;
            a.rx = (T)h->prob.rx;
            a.ry = (T)h->prob.ry;
            a.hrx = soft64::make_heat_r(h->prob.rx);
            a.hry = soft64::make_heat_r(h->prob.ry);
            a.brx = reinterpret_cast<T *>(h->brx);
            a.bry = reinterpret_cast<T *>(h->bry);
            const unsigned tiles = (unsigned)(h->Mx * h->My);
            const int nt = h->nt;
            for (int64_t p = 0; p <= P; ++p) {
                a.p = (int)(p & 1) ? 1 : 2;  // only the parity of p matters to the kernels
                if (p == 0) a.p = 0;
                a.F = p * H;
                a.last = p == P ? 1 : 0;
                a.pin_x = p == 0 ? nullptr : reinterpret_cast<const T *>(h->pyrx[(p - 1) & 1]);
                a.pin_y = p == 0 ? nullptr : reinterpret_cast<const T *>(h->pyry[(p - 1) & 1]);
                a.pout_x = reinterpret_cast<T *>(h->pyrx[p & 1]);
                a.pout_y = reinterpret_cast<T *>(h->pyry[p & 1]);
                if (p == 0) {
                    trace2d_begin(h, launches, 0, st);
                    launch2d<T>(0, nt, tiles, h->smem, st, a);
                    trace2d_end(h, launches++, st);
                    continue;
                }
                trace2d_begin(h, launches, 1, st);
                launch2d<T>(1, h->nt_br, tiles, h->smem, st, a);
                trace2d_end(h, launches++, st);
                trace2d_begin(h, launches, p == P ? 4 : 2, st);
                launch2d<T>(2, nt, tiles, h->smem, st, a);
                trace2d_end(h, launches++, st);
            }
        }
        if (cudaGetLastError() != cudaSuccess) return SW_ERR_CUDA;
        // the remaining steps (fewer than W/2) with the per-step kernel: the same bits
        rc = run_perstep2d<T>(h, state, P >= 1 ? R : nsteps, st, launches);
    } else {
        rc = run_perstep2d<T>(h, state, nsteps, st, launches);
    }
    h->last_launches = launches;
    if (rc != SW_OK) return rc;
    return cuda_status2d(cudaGetLastError());
}

}  // namespace

extern "C" {

int sw2d_create(const sw_heat2d *p, sw_handle2d **out) {
    if (!out) return SW_ERR_BAD_ARG;
    const int v = validate2d(p);
    if (v != SW_OK) return v;
    sw_handle2d *h = new (std::nothrow) sw_handle2d();
    if (!h) return SW_ERR_OOM;
    h->prob = *p;
    h->es = p->precision == SW_FP64 ? sizeof(double) : sizeof(float);
    auto fail = [&](int code) {
        sw2d_destroy(h);
        return code;
    };
    cudaError_t e = cudaMalloc(&h->plane, size_t(p->nx * p->ny) * h->es);
    if (e != cudaSuccess) return fail(cuda_status2d(e));
    {   // the row-mapping multipliers (the same values on every device; written once per create)
        unsigned magic[kMagicMax + 1];
        magic[0] = 0;
        magic[1] = 0;  // never used: windows and strips are at least 2 wide, one band needs no division
        for (int w = 2; w <= kMagicMax; ++w) magic[w] = 0xFFFFFFFFu / (unsigned)w + 1u;
        e = cudaMemcpyToSymbol(c_magic, magic, sizeof(magic));
        if (e != cudaSuccess) return fail(cuda_status2d(e));
    }
    if (p->method == SW_SWEPT) {
        h->W = p->tile_width ? p->tile_width : 64;
        h->H = h->W / 2;
        h->Mx = (int)(p->nx / h->W);
        h->My = (int)(p->ny / h->W);
        if (h->W > max_width2d(h->es)) return fail(SW_ERR_UNSUPPORTED);
        h->smem = smem2d(h->W, h->es);
        h->nt = swept_threads2d(h->es, h->W, false);
        h->nt_br = swept_threads2d(h->es, h->W, true);
        e = p->precision == SW_FP64 ? allow_smem2d_all<double>(h->W, h->smem)
                                    : allow_smem2d_all<float>(h->W, h->smem);
        if (e != cudaSuccess) return fail(cuda_status2d(e));
        // per buffer: tiles x 2 sides x H steps x 2 x W values
        const size_t bytes = size_t(h->Mx) * h->My * 2 * h->H * 2 * h->W * h->es;
        void **bufs[6] = {&h->pyrx[0], &h->pyrx[1], &h->pyry[0], &h->pyry[1], &h->brx, &h->bry};
        for (void **b : bufs) {
            e = cudaMalloc(b, bytes);
            if (e != cudaSuccess) return fail(cuda_status2d(e));
        }
    }
    *out = h;
    return (p->rx + p->ry > 0.5) ? SW_WARN_UNSTABLE : SW_OK;
}

void sw2d_destroy(sw_handle2d *h) {
    if (!h) return;
    cudaDeviceSynchronize();
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    cudaFree(h->plane);
    cudaFree(h->pyrx[0]);
    cudaFree(h->pyrx[1]);
    cudaFree(h->pyry[0]);
    cudaFree(h->pyry[1]);
    cudaFree(h->brx);
    cudaFree(h->bry);
    delete h;
}

int sw2d_run(sw_handle2d *h, void *state, int64_t nsteps, void *stream) {
    if (!h || !state || nsteps < 0) return SW_ERR_BAD_ARG;
    h->last_launches = 0;
    h->ev_used = 0;
    if (nsteps == 0) return SW_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    return h->prob.precision == SW_FP64 ? run2d<double>(h, state, nsteps, st) : run2d<float>(h, state, nsteps, st);
}

int64_t sw2d_last_launch_count(const sw_handle2d *h) { return h ? h->last_launches : 0; }

int32_t sw2d_tile_width(const sw_handle2d *h) { return h ? h->W : 0; }

int sw2d_set_threads(sw_handle2d *h, int32_t threads, int32_t bridge_threads) {
    if (!h || h->prob.method != SW_SWEPT) return SW_ERR_BAD_ARG;
    if (threads == 0) threads = swept_threads2d(h->es, h->W, false);
    if (bridge_threads == 0) bridge_threads = swept_threads2d(h->es, h->W, true);
    auto ok = [](int32_t t) { return t == 128 || t == kThreads2D || t == kThreads2DWide; };
    if (!ok(threads) || !ok(bridge_threads)) return SW_ERR_BAD_ARG;
    h->nt = threads;
    h->nt_br = bridge_threads;
    return SW_OK;
}

int32_t sw2d_threads(const sw_handle2d *h, int32_t bridges) { return h ? (bridges ? h->nt_br : h->nt) : 0; }

int sw2d_set_timing(sw_handle2d *h, int64_t capacity) {
    if (!h || capacity < 0 || capacity > (int64_t(1) << 24)) return SW_ERR_BAD_ARG;
    while ((int64_t)h->events.size() < 2 * capacity) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return cuda_status2d(err);
        h->events.push_back(e);
    }
    h->kinds.assign((size_t)capacity, 0);
    h->ev_cap = capacity;
    h->ev_used = 0;
    return SW_OK;
}

int64_t sw2d_launch_times(sw_handle2d *h, float *ms, int32_t *kind, int64_t cap) {
    if (!h || cap < 0 || (cap > 0 && (!ms || !kind))) return SW_ERR_BAD_ARG;
    const int64_t cnt = std::min(cap, h->ev_used);
    for (int64_t i = 0; i < cnt; ++i) {
        cudaError_t e = cudaEventSynchronize(h->events[2 * i + 1]);
        if (e != cudaSuccess) return cuda_status2d(e);
        e = cudaEventElapsedTime(&ms[i], h->events[2 * i], h->events[2 * i + 1]);
        if (e != cudaSuccess) return cuda_status2d(e);
        kind[i] = h->kinds[i];
    }
    return cnt;
}

}  // extern "C"
