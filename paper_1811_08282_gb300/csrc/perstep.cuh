// perstep.cuh -- the per-time-step ("Classic") kernels of Section 4.3 / Fig. 2a:
// every launch reads the whole state from HBM and writes it back once.
//
// Heat: one launch per step, V consecutive cells per thread (vector loads),
// neighbours from adjacent lanes by warp shuffle, warp-edge neighbours by a
// cached scalar load. Euler: the flattened form, two launches per step
// (predictor, final), a CTA stages its cells plus a 2-cell halo in shared
// memory and evaluates each face flux once. Both call the same per-cell
// functions as the swept phases, so the two decompositions agree bitwise.
#pragma once
#include <type_traits>

#include "fp64_soft.cuh"
#include "euler.cuh"
#include "heat.cuh"
#include "heat_policy.cuh"

namespace sw {

// Vector types of V consecutive elements; V > 1 needs V * sizeof(T)-byte aligned
// addresses (the launcher checks the state pointer before choosing V).
struct alignas(32) Float8 {
    float4 a, b;
};
struct alignas(32) Double4 {
    double2 a, b;
};
template <class T, int V> struct VecT;
template <> struct VecT<double, 1> { using type = double; };
template <> struct VecT<double, 2> { using type = double2; };
template <> struct VecT<double, 4> { using type = Double4; };
template <> struct VecT<float, 1> { using type = float; };
template <> struct VecT<float, 4> { using type = float4; };
template <> struct VecT<float, 8> { using type = Float8; };

template <class T, int V>
__device__ __forceinline__ void vload(const T *p, T (&v)[V]) {
    using VT = typename VecT<T, V>::type;
    VT x = *reinterpret_cast<const VT *>(p);
    const T *e = reinterpret_cast<const T *>(&x);
#pragma unroll
    for (int k = 0; k < V; ++k) v[k] = e[k];
}

template <class T, int V>
__device__ __forceinline__ void vstore(T *p, const T (&v)[V]) {
    using VT = typename VecT<T, V>::type;
    VT x;
    T *e = reinterpret_cast<T *>(&x);
#pragma unroll
    for (int k = 0; k < V; ++k) e[k] = v[k];
    *reinterpret_cast<VT *>(p) = x;
}

__device__ __forceinline__ int64_t nb_index(int64_t j, int64_t n, int periodic) {
    if (j < 0) return periodic ? j + n : 0;
    if (j >= n) return periodic ? j - n : n - 1;
    return j;
}

// One FTCS step, FP64 or FP32, `in` -> `out` (distinct buffers).
template <class O, int V>
__global__ void __launch_bounds__(256) k_heat_step(const typename O::T *__restrict__ in,
                                                   typename O::T *__restrict__ out, int64_t n,
                                                   typename O::T r, int periodic) {
    using T = typename O::T;
    // FP64 with two or more cells per thread: the odd cells are updated on the
    // integer pipes (soft64::heat_update, the same bits) beside the FP64 pipe
    constexpr bool SOFT = std::is_same<T, double>::value && V >= 2;
    soft64::HeatR hr{};
    if constexpr (SOFT) hr = soft64::make_heat_r((double)r);
    const int64_t nch = n / V;
    const int64_t nch_r = (nch + 31) & ~int64_t(31);
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < nch_r; ch += stride) {
        const bool act = ch < nch;
        const int64_t j0 = ch * V;
        T v[V];
        if (act) vload<T, V>(in + j0, v);
        else {
#pragma unroll
            for (int k = 0; k < V; ++k) v[k] = T(0);
        }
        T left = __shfl_up_sync(0xffffffffu, v[V - 1], 1);
        T right = __shfl_down_sync(0xffffffffu, v[0], 1);
        if (act) {
            if (lane == 0) left = in[nb_index(j0 - 1, n, periodic)];
            if (lane == 31 || ch + 1 >= nch) right = in[nb_index(j0 + V, n, periodic)];
            T o[V];
            bool okall = true;
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const T a = (k == 0) ? left : v[k - 1];
                const T b = (k == V - 1) ? right : v[k + 1];
                if constexpr (SOFT) {
                    if (k & 1) {
                        bool ok;
                        o[k] = soft64::value(soft64::heat_update(hr, soft64::bits(a), soft64::bits(v[k]),
                                                                 soft64::bits(b), ok));
                        okall = okall && ok && hr.usable;
                        continue;
                    }
                }
                o[k] = heat_update<O>(r, a, v[k], b);
            }
            if constexpr (SOFT) {
                if (__any_sync(__activemask(), !okall)) {
                    // some cell left the integer path's range: odd slots on the FP64 pipe
#pragma unroll
                    for (int k = 1; k < V; k += 2)
                        o[k] = soft64::heat_update_fp64((double)r, v[k - 1], v[k], (k == V - 1) ? right : v[k + 1]);
                }
            }
            vstore<T, V>(out + j0, o);
        }
    }
}

// One compensated FTCS step on (hi, lo) planes: in = [hi | lo], out = [hi | lo].
template <int V>
__global__ void __launch_bounds__(256) k_heat_step_comp(const float *__restrict__ in, float *__restrict__ out,
                                                        int64_t n, float rh, float rl, int periodic) {
    const int64_t nch = n / V;
    const int64_t nch_r = (nch + 31) & ~int64_t(31);
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float *inl = in + n;
    float *outl = out + n;
    for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < nch_r; ch += stride) {
        const bool act = ch < nch;
        const int64_t j0 = ch * V;
        float h[V], l[V];
        if (act) {
            vload<float, V>(in + j0, h);
            vload<float, V>(inl + j0, l);
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k) h[k] = l[k] = 0.f;
        }
        HL left{__shfl_up_sync(0xffffffffu, h[V - 1], 1), __shfl_up_sync(0xffffffffu, l[V - 1], 1)};
        HL right{__shfl_down_sync(0xffffffffu, h[0], 1), __shfl_down_sync(0xffffffffu, l[0], 1)};
        if (act) {
            if (lane == 0) {
                const int64_t j = nb_index(j0 - 1, n, periodic);
                left = HL{in[j], inl[j]};
            }
            if (lane == 31 || ch + 1 >= nch) {
                const int64_t j = nb_index(j0 + V, n, periodic);
                right = HL{in[j], inl[j]};
            }
            float oh[V], ol[V];
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const HL a = (k == 0) ? left : HL{h[k - 1], l[k - 1]};
                const HL b = (k == V - 1) ? right : HL{h[k + 1], l[k + 1]};
                HL o = heat_update_comp(rh, rl, a, HL{h[k], l[k]}, b);
                oh[k] = o.h;
                ol[k] = o.l;
            }
            vstore<float, V>(out + j0, oh);
            vstore<float, V>(outl + j0, ol);
        }
    }
}

// One stage of the flattened Euler step. FINAL = false (predictor): reads Q
// (planes q), writes Q* (planes s). FINAL = true: reads Q* (fluxes) and Q
// (own cell), writes Q in place. Block of B = blockDim.x cells plus a 2-cell halo.
// COMP: q holds [hi(3) | lo(3)] planes, s holds 3 FP32 planes.
template <class O, bool FINAL, bool COMP>
__global__ void __launch_bounds__(256) k_euler_stage(typename O::T *__restrict__ q, typename O::T *__restrict__ s,
                                                     int64_t n, EulerParams prm, int periodic) {
    using T = typename O::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int B = blockDim.x;
    const int NL = B + 4;  // staged cells x0-2 .. x0+B+1
    T *src = reinterpret_cast<T *>(smem_raw);  // [3][NL]
    T *pr = src + 3 * NL;                      // [NL]
    T *th = pr + NL;                           // [B+2]: cells x0-1 .. x0+B
    T *fx = th + (B + 2);                      // [3][B+1]: faces x0-1/2 .. x0+B-1/2
    const EulerK<O> k = eu_k<O>(prm);
    const int tid = threadIdx.x;
    const int64_t x0 = (int64_t)blockIdx.x * B;
    const T *in = FINAL ? s : q;
    for (int l = tid; l < NL; l += B) {
        const int64_t j = nb_index(x0 - 2 + l, n, periodic);
        const T r0 = in[j], r1 = in[n + j], r2 = in[2 * n + j];
        src[l] = r0;
        src[NL + l] = r1;
        src[2 * NL + l] = r2;
        pr[l] = eu_pressure<O>(k, r0, r1, r2);
    }
    __syncthreads();
    for (int t = tid; t < B + 2; t += B) th[t] = eu_ratio<O>(pr[t], pr[t + 1], pr[t + 2]);
    __syncthreads();
    for (int m = tid; m <= B; m += B) {
        // face between cells x0-1+m (staged index m+1, ratio index m) and x0+m (m+2, m+1)
        T f0, f1, f2;
        eu_face_flux<O>(k, src[m + 1], src[NL + m + 1], src[2 * NL + m + 1], th[m], src[m + 2],
                        src[NL + m + 2], src[2 * NL + m + 2], th[m + 1], f0, f1, f2);
        fx[m] = f0;
        fx[(B + 1) + m] = f1;
        fx[2 * (B + 1) + m] = f2;
    }
    __syncthreads();
    const int64_t i = x0 + tid;
    if (i < n) {
        const T d0 = O::sub(fx[tid + 1], fx[tid]);
        const T d1 = O::sub(fx[(B + 1) + tid + 1], fx[(B + 1) + tid]);
        const T d2 = O::sub(fx[2 * (B + 1) + tid + 1], fx[2 * (B + 1) + tid]);
        if constexpr (!COMP) {
            const T c = FINAL ? k.lam : k.hlam;
            T *dst = FINAL ? q : s;
            dst[i] = eu_update<O>(q[i], c, d0);
            dst[n + i] = eu_update<O>(q[n + i], c, d1);
            dst[2 * n + i] = eu_update<O>(q[2 * n + i], c, d2);
        } else {
            const T dv[3] = {d0, d1, d2};
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                const float h = q[v * n + i], lo = q[(3 + v) * n + i];
                if (!FINAL) {
                    s[v * n + i] = eu_comp_predict<O>(h, lo, k.hlam, dv[v]);
                } else {
                    float nh, nl;
                    eu_comp_final<O>(h, lo, k.lam, dv[v], nh, nl);
                    q[v * n + i] = nh;
                    q[(3 + v) * n + i] = nl;
                }
            }
        }
    }
}

// One sub-step of the lengthened Euler step (Section 4.3, Fig. 2: four 3-point
// sub-steps per step, the pressure ratio stored between them), one launch each:
// KIND 0 ratio of Q, 1 predictor Q*, 2 ratio of Q*, 3 final. q: the state planes
// (COMP: high 3, low 3); s: scratch planes Q* (0..2) and ratio (3). A block of B
// cells stages its cells plus one halo cell per side; transmissive ends clamp the
// halo to the end cell, whose ratio is 0 (its one-sided difference vanishes), so the
// halo is the scheme's ghost cell. Same per-cell functions as every other form.
template <class O, int KIND, bool COMP>
__global__ void __launch_bounds__(256) k_euler_sub(typename O::T *__restrict__ q, typename O::T *__restrict__ s,
                                                   int64_t n, EulerParams prm, int periodic) {
    using T = typename O::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int B = blockDim.x, NL = B + 2;
    T *g = reinterpret_cast<T *>(smem_raw);  // [3][NL] flux / pressure group, cells x0-1 .. x0+B
    T *aux = g + 3 * NL;                      // [NL] pressure (ratio kinds) or ratio (flux kinds)
    T *fx = aux + NL;                         // [3][B+1] face fluxes x0-1/2 .. x0+B-1/2
    const EulerK<O> k = eu_k<O>(prm);
    const int tid = threadIdx.x;
    const int64_t x0 = (int64_t)blockIdx.x * B;
    const T *src = (KIND <= 1) ? q : s;  // Q (high parts) or Q*
    for (int l = tid; l < NL; l += B) {
        const int64_t j = nb_index(x0 - 1 + l, n, periodic);
        const T r0 = src[j], r1 = src[n + j], r2 = src[2 * n + j];
        g[l] = r0;
        g[NL + l] = r1;
        g[2 * NL + l] = r2;
        if constexpr (KIND == 0 || KIND == 2) aux[l] = eu_pressure<O>(k, r0, r1, r2);
        else aux[l] = s[3 * n + j];
    }
    __syncthreads();
    const int64_t i = x0 + tid;
    if constexpr (KIND == 0 || KIND == 2) {
        if (i < n) s[3 * n + i] = eu_ratio<O>(aux[tid], aux[tid + 1], aux[tid + 2]);
    } else {
        for (int m = tid; m <= B; m += B) {
            T f0, f1, f2;
            eu_face_flux<O>(k, g[m], g[NL + m], g[2 * NL + m], aux[m], g[m + 1], g[NL + m + 1], g[2 * NL + m + 1],
                            aux[m + 1], f0, f1, f2);
            fx[m] = f0;
            fx[(B + 1) + m] = f1;
            fx[2 * (B + 1) + m] = f2;
        }
        __syncthreads();
        if (i < n) {
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                const T d = O::sub(fx[v * (B + 1) + tid + 1], fx[v * (B + 1) + tid]);
                if constexpr (!COMP) {
                    if constexpr (KIND == 1) s[v * n + i] = eu_update<O>(q[v * n + i], k.hlam, d);
                    else q[v * n + i] = eu_update<O>(q[v * n + i], k.lam, d);
                } else {
                    if constexpr (KIND == 1) {
                        s[v * n + i] = eu_comp_predict<O>(q[v * n + i], q[(3 + v) * n + i], k.hlam, d);
                    } else {
                        float nh, nl;
                        eu_comp_final<O>(q[v * n + i], q[(3 + v) * n + i], k.lam, d, nh, nl);
                        q[v * n + i] = nh;
                        q[(3 + v) * n + i] = nl;
                    }
                }
            }
        }
    }
}

}  // namespace sw
