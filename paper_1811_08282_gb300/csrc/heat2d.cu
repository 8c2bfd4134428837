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

constexpr int kThreads2D = 256;       // per-step kernel; swept kernels at W < 128
constexpr int kThreads2DWide = 1024;  // swept kernels at W >= 128: one CTA per SM fits the frame

// Threads of a swept CTA: the frame of W >= 128 leaves room for one CTA per SM, which then
// takes all the warps it can. The kernels are instantiated for both counts, each with a
// launch bound that keeps the narrow form at its resident-CTA count (FP32: 6 per SM,
// FP64: 3, what the frame's shared memory allows at W = 64).
__host__ __device__ constexpr int swept_threads2d(int W) { return W >= 128 ? kThreads2DWide : kThreads2D; }

// ceil(2^32 / w) for every window width w = 1 .. kMagicMax (the row of cell t of a window w
// wide is umulhi(t, magic[w])); filled from the host at sw2d_create, identical on every device
constexpr int kMagicMax = 1026;
__constant__ unsigned c_magic[kMagicMax + 1];

// The quotient and remainder of t by len for the strip loops (t < 8 * len, 2 <= len <=
// kMagicMax: exact, since t * len < 2^32)
__device__ __forceinline__ void div_len(int t, int len, int &q, int &r) {
    q = (int)__umulhi((unsigned)t, c_magic[len]);
    r = t - q * len;
}

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
// vectors (the launcher checks the alignment of the state and of nx).
template <class T, int V, bool VEC>
__global__ void __launch_bounds__(kThreads2D) k2d_step(const T *__restrict__ in, T *__restrict__ out, int64_t nx,
                                                       int64_t ny, T rx, T ry, int periodic) {
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

// strip element (tile, side, step, k, r): one buffer holds 2 sides x H steps x 2 x W per tile
__device__ __forceinline__ int64_t strip_off(int tile, int side, int i, int k, int H, int W) {
    return ((((int64_t)tile * 2 + side) * H + i) * 2 + k) * W;
}

// The shared frame of a region centred at (cx, cy): position (x, y) absolute (unwrapped)
// -> (x - cx + H + 1, y - cy + H + 1).
template <class T> struct Frame {
    T *s;
    int RS, slot, cx, cy, H;
    __device__ __forceinline__ T &at(int64_t lev, int x, int y) const {
        return s[(int)(lev & 1) * slot + (y - cy + H + 1) * RS + (x - cx + H + 1)];
    }
};

// compute the window [x0, x1] x [y0, y1] at level lev from lev - 1: the block's threads
// run over the window's cells in row-major order (consecutive threads on consecutive
// cells of a row), so narrow windows keep every lane busy; the row of cell t is
// umulhi(t, ceil(2^32 / w)), exact while t * w < 2^32 (t < w * h <= 2^16 here).
template <class T>
__device__ __forceinline__ void compute_window(const Frame<T> &f, int64_t lev, int x0, int x1, int y0, int y1, T rx,
                                               T ry) {
    using O = typename Ops2D<T>::O;
    const unsigned w = (unsigned)(x1 - x0 + 1), cnt = w * (unsigned)(y1 - y0 + 1);
    const unsigned m = c_magic[w];  // ceil(2^32 / w), w >= 2
    const T *src = f.s + (int)((lev - 1) & 1) * f.slot;
    T *dst = f.s + (int)(lev & 1) * f.slot;
    const int org = (y0 - f.cy + f.H + 1) * f.RS + (x0 - f.cx + f.H + 1);
    // a thread's cells are independent: unrolled, their shared-memory loads overlap
#pragma unroll 4
    for (unsigned t = threadIdx.x; t < cnt; t += blockDim.x) {
        const unsigned yy = __umulhi(t, m), xx = t - yy * w;
        const int q = org + (int)yy * f.RS + (int)xx;
        dst[q] = heat2d_update<O>(rx, ry, src[q - 1], src[q + 1], src[q], src[q - f.RS], src[q + f.RS]);
    }
}

// export the 2-deep edges of a pyramid window (x-strips: columns x0, x0+1 / x1-1, x1 over
// rows y0..y1; y-strips: rows over columns) at step i
template <class T>
__device__ __forceinline__ void export_pyramid(const Frame<T> &f, int64_t lev, int x0, int x1, int y0, int y1,
                                               T *sx, T *sy, int tile, int i, int H, int W) {
    const int len = x1 - x0 + 1;  // square window
    for (int t = threadIdx.x; t < 8 * len; t += blockDim.x) {
        int q, r;  // q: which of the 8 edge lines
        div_len(t, len, q, r);
        const int side = (q >> 1) & 1, k = q & 1;
        if (q < 4) {  // x-strips
            const int x = side == 0 ? x0 + k : x1 - 1 + k;
            sx[strip_off(tile, side, i, k, H, W) + r] = f.at(lev, x, y0 + r);
        } else {
            const int y = side == 0 ? y0 + k : y1 - 1 + k;
            sy[strip_off(tile, side, i, k, H, W) + r] = f.at(lev, x0 + r, y);
        }
    }
}

// The upper part of a structure of phase q (the pyramid): steps 0..H-1 from the full
// tile at level F (already in the frame), exporting both kinds of strips per step.
template <class T>
__device__ void pyramid_part(const Frame<T> &f, const Swept2DArgs<T> &a, int64_t F, int tile, T *sx, T *sy) {
    const int H = a.H, cx = f.cx, cy = f.cy;
    export_pyramid(f, F, cx - H, cx + H - 1, cy - H, cy + H - 1, sx, sy, tile, 0, H, a.W);
    for (int i = 1; i < H; ++i) {
        compute_window(f, F + i, cx - H + i, cx + H - 1 - i, cy - H + i, cy + H - 1 - i, a.rx, a.ry);
        __syncthreads();
        export_pyramid(f, F + i, cx - H + i, cx + H - 1 - i, cy - H + i, cy + H - 1 - i, sx, sy, tile, i, H, a.W);
    }
}

// Up: the pyramids of phase 0 from the state (level 0)
template <class T, int NT>
__global__ void __launch_bounds__(NT, NT == kThreads2D ? (sizeof(T) == 4 ? 6 : 3) : 1) k2d_up(Swept2DArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int bx = blockIdx.x % a.Mx, by = blockIdx.x / a.Mx;
    const int RS = a.W + 3, H = a.H;
    Frame<T> f{reinterpret_cast<T *>(smem_raw), RS, (a.W + 2) * RS, centre2d(0, bx, a.W), centre2d(0, by, a.W), H};
    for (int t = threadIdx.x; t < a.W * a.W; t += blockDim.x) {
        const int y = f.cy - H + t / a.W, x = f.cx - H + t % a.W;
        f.at(0, x, y) = a.state[(int64_t)((y + a.ny) % a.ny) * a.nx + (x + a.nx) % a.nx];
    }
    __syncthreads();
    pyramid_part(f, a, 0, blockIdx.x, a.pout_x, a.pout_y);
}

// Bridges of phase p: blockIdx.y = 0 x-bridges (lower in x, upper in y), 1 y-bridges.
template <class T, int NT>
__global__ void __launch_bounds__(NT, NT == kThreads2D ? (sizeof(T) == 4 ? 6 : 3) : 1) k2d_bridges(Swept2DArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b0 = blockIdx.x % a.Mx, b1 = blockIdx.x / a.Mx;  // (x index, y index)
    const int W = a.W, H = a.H, RS = W + 3;
    const bool xb = blockIdx.y == 0;
    // x-bridge: centre (c_p(b0), c_{p-1}(b1)); y-bridge: (c_{p-1}(b0), c_p(b1))
    const int cx = centre2d(xb ? a.p : a.p - 1, b0, W), cy = centre2d(xb ? a.p - 1 : a.p, b1, W);
    Frame<T> f{reinterpret_cast<T *>(smem_raw), RS, (W + 2) * RS, cx, cy, H};
    int lo, hi;  // the two pyramids it imports from (phase p - 1 indices along its lower direction)
    nbrs(a.p, xb ? b0 : b1, xb ? a.Mx : a.My, lo, hi);
    const int tlo = xb ? b1 * a.Mx + lo : lo * a.Mx + b0;
    const int thi = xb ? b1 * a.Mx + hi : hi * a.Mx + b0;
    const int tile = blockIdx.x;
    const int64_t base = a.F - H;  // level of step 0
    // step i's inputs at level base + i - 1: the pyramids' strips at step i - 1, all of
    // their W - 2(i-1) entries (rows for an x-bridge, columns for a y-bridge)
    auto inject = [&](int i) {
        const int len = W - 2 * (i - 1);
        const T *src = xb ? a.pin_x : a.pin_y;
        for (int t = threadIdx.x; t < 4 * len; t += blockDim.x) {
            int q, r;  // q: (neighbour, k)
            div_len(t, len, q, r);
            const int k = q & 1, hiside = q >> 1;
            // the low-side pyramid exports its high side (1), the high-side pyramid its low side (0)
            const T v = src[strip_off(hiside ? thi : tlo, hiside ? 0 : 1, i - 1, k, H, W) + r];
            if (xb) {
                const int x = hiside ? cx + i - 1 + k : cx - i - 1 + k;
                f.at(base + i - 1, x, cy - H + i - 1 + r) = v;
            } else {
                const int y = hiside ? cy + i - 1 + k : cy - i - 1 + k;
                f.at(base + i - 1, cx - H + i - 1 + r, y) = v;
            }
        }
    };
    inject(1);
    __syncthreads();
    for (int i = 1; i < H; ++i) {
        int x0, x1, y0, y1;
        if (xb) {
            x0 = cx - i; x1 = cx + i - 1; y0 = cy - H + i; y1 = cy + H - 1 - i;
        } else {
            x0 = cx - H + i; x1 = cx + H - 1 - i; y0 = cy - i; y1 = cy + i - 1;
        }
        compute_window(f, base + i, x0, x1, y0, y1, a.rx, a.ry);
        if (i + 1 < H) inject(i + 1);  // other positions of the slot being written
        __syncthreads();
        // export the edges along the widening direction's normal: an x-bridge its bottom and
        // top two rows (2i columns), a y-bridge its left and right two columns (2i rows)
        const int len = 2 * i;
        T *dst = xb ? a.brx : a.bry;
        for (int t = threadIdx.x; t < 4 * len; t += blockDim.x) {
            int q, r;
            div_len(t, len, q, r);
            const int k = q & 1, side = q >> 1;
            T v;
            if (xb) v = f.at(base + i, x0 + r, side == 0 ? y0 + k : y1 - 1 + k);
            else v = f.at(base + i, side == 0 ? x0 + k : x1 - 1 + k, y0 + r);
            dst[strip_off(tile, side, i, k, H, W) + r] = v;
        }
    }
}

// Octahedra of phase p: the lower part (lower x lower) up to the full tile at F, then the
// pyramid of phase p (or, in the last phase, the tile stored to the state).
template <class T, int NT>
__global__ void __launch_bounds__(NT, NT == kThreads2D ? (sizeof(T) == 4 ? 6 : 3) : 1) k2d_octa(Swept2DArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int bx = blockIdx.x % a.Mx, by = blockIdx.x / a.Mx;
    const int W = a.W, H = a.H, RS = W + 3;
    const int cx = centre2d(a.p, bx, W), cy = centre2d(a.p, by, W);
    Frame<T> f{reinterpret_cast<T *>(smem_raw), RS, (W + 2) * RS, cx, cy, H};
    int lx, rx, lb, rt;
    nbrs(a.p, bx, a.Mx, lx, rx);
    nbrs(a.p, by, a.My, lb, rt);
    const int64_t base = a.F - H;
    auto inject = [&](int i) {
        const int64_t lev = base + i - 1;
        const int x0 = cx - i, x1 = cx + i - 1, y0 = cy - i, y1 = cy + i - 1;
        const int len = 2 * (i - 1);  // the bridges' strips at step i - 1
        if (len > 0) {
            for (int t = threadIdx.x; t < 8 * len; t += blockDim.x) {
                int q, r;
                div_len(t, len, q, r);
                const int k = q & 1, which = q >> 1;
                // 0: y-bridge on the left (its right columns), 1: on the right (its left columns),
                // 2: x-bridge below (its top rows), 3: above (its bottom rows)
                if (which < 2) {
                    const int tb = by * a.Mx + (which == 0 ? lx : rx);
                    const T v = a.bry[strip_off(tb, which == 0 ? 1 : 0, i - 1, k, H, W) + r];
                    const int x = which == 0 ? x0 - 1 + k : x1 + k;
                    f.at(lev, x, cy - i + 1 + r) = v;
                } else {
                    const int tb = (which == 2 ? lb : rt) * a.Mx + bx;
                    const T v = a.brx[strip_off(tb, which == 2 ? 1 : 0, i - 1, k, H, W) + r];
                    const int y = which == 2 ? y0 - 1 + k : y1 + k;
                    f.at(lev, cx - i + 1 + r, y) = v;
                }
            }
        }
        // corners: from the x-strips of the four diagonal pyramids of phase p - 1 at step i - 1
        if (threadIdx.x < 12) {
            const int c = threadIdx.x / 3, e = threadIdx.x % 3;
            const bool right = c & 1, top = c >> 1;
            const int tp = (top ? rt : lb) * a.Mx + (right ? rx : lx);
            const int side = right ? 0 : 1;
            const int ystart = top ? cy + i - 1 : cy - W + i - 1;  // the pyramid's window start
            const int ycorner = top ? y1 : y0, yout = top ? y1 + 1 : y0 - 1;
            int x, y, k;
            if (e < 2) {  // both new columns at the corner row
                k = e;
                x = right ? x1 + k : x0 - 1 + k;
                y = ycorner;
            } else {  // the inner new column, one row further out
                k = right ? 0 : 1;
                x = right ? x1 : x0;
                y = yout;
            }
            f.at(lev, x, y) = a.pin_x[strip_off(tp, side, i - 1, k, H, W) + (y - ystart)];
        }
    };
    inject(1);
    __syncthreads();
    for (int i = 1; i <= H; ++i) {
        compute_window(f, base + i, cx - i, cx + i - 1, cy - i, cy + i - 1, a.rx, a.ry);
        if (i < H) inject(i + 1);
        __syncthreads();
    }
    if (a.last) {
        for (int t = threadIdx.x; t < W * W; t += blockDim.x) {
            const int y = cy - H + t / W, x = cx - H + t % W;
            a.state[(int64_t)((y + a.ny) % a.ny) * a.nx + (x + a.nx) % a.nx] = f.at(a.F, x, y);
        }
        return;
    }
    pyramid_part(f, a, a.F, blockIdx.x, a.pout_x, a.pout_y);
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

// `steps` per-step launches, ping-pong between the state and the handle's plane; the
// result ends in the state
template <class T>
int run_perstep2d(sw_handle2d *h, T *state, int64_t steps, cudaStream_t st, int64_t &launches) {
    const int64_t nx = h->prob.nx, ny = h->prob.ny;
    const int periodic = h->prob.boundary == SW_PERIODIC;
    const T rx = (T)h->prob.rx, ry = (T)h->prob.ry;
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
            k2d_step<T, 4, true><<<grid2d(nx / 4 * ny, cap), kThreads2D, 0, st>>>(in, out, nx, ny, rx, ry, periodic);
        else if (nx % 4 == 0)
            k2d_step<T, 4, false><<<grid2d(nx / 4 * ny, cap), kThreads2D, 0, st>>>(in, out, nx, ny, rx, ry,
                                                                                   periodic);
        else
            k2d_step<T, 1, false><<<grid2d(nx * ny, cap), kThreads2D, 0, st>>>(in, out, nx, ny, rx, ry, periodic);
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
            a.brx = reinterpret_cast<T *>(h->brx);
            a.bry = reinterpret_cast<T *>(h->bry);
            const unsigned tiles = (unsigned)(h->Mx * h->My);
            const int nt = swept_threads2d(h->W);
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
                    if (nt == kThreads2D) k2d_up<T, kThreads2D><<<tiles, nt, h->smem, st>>>(a);
                    else k2d_up<T, kThreads2DWide><<<tiles, nt, h->smem, st>>>(a);
                    trace2d_end(h, launches++, st);
                    continue;
                }
                trace2d_begin(h, launches, 1, st);
                if (nt == kThreads2D) k2d_bridges<T, kThreads2D><<<dim3(tiles, 2), nt, h->smem, st>>>(a);
                else k2d_bridges<T, kThreads2DWide><<<dim3(tiles, 2), nt, h->smem, st>>>(a);
                trace2d_end(h, launches++, st);
                trace2d_begin(h, launches, p == P ? 4 : 2, st);
                if (nt == kThreads2D) k2d_octa<T, kThreads2D><<<tiles, nt, h->smem, st>>>(a);
                else k2d_octa<T, kThreads2DWide><<<tiles, nt, h->smem, st>>>(a);
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
        magic[1] = 0;  // never used: windows are at least 2 wide
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
        const void *fns[6];
        if (p->precision == SW_FP64) {
            fns[0] = (const void *)k2d_up<double, kThreads2D>;
            fns[1] = (const void *)k2d_bridges<double, kThreads2D>;
            fns[2] = (const void *)k2d_octa<double, kThreads2D>;
            fns[3] = (const void *)k2d_up<double, kThreads2DWide>;
            fns[4] = (const void *)k2d_bridges<double, kThreads2DWide>;
            fns[5] = (const void *)k2d_octa<double, kThreads2DWide>;
        } else {
            fns[0] = (const void *)k2d_up<float, kThreads2D>;
            fns[1] = (const void *)k2d_bridges<float, kThreads2D>;
            fns[2] = (const void *)k2d_octa<float, kThreads2D>;
            fns[3] = (const void *)k2d_up<float, kThreads2DWide>;
            fns[4] = (const void *)k2d_bridges<float, kThreads2DWide>;
            fns[5] = (const void *)k2d_octa<float, kThreads2DWide>;
        }
        for (const void *fn : fns) {
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->smem);
            if (e != cudaSuccess) return fail(cuda_status2d(e));
        }
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
