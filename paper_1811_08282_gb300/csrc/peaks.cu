// peaks.cu -- libpeaks.so: measured issue rates of the pipes the stencil kernels
// are bound by on this GPU (the FP64 pipe, the FP32 FMA pipe and the integer ALU
// pipe), for the roofline denominators: the driver's peak file has an HBM copy and
// a bf16 GEMM figure but nothing for FP64 or the integer pipes.
//
// Each thread runs eight independent dependency chains (enough to cover the pipe
// latency at full occupancy) of one operation for `iters` iterations; the grid is
// 8 CTAs of 256 threads per SM. The result of every chain reaches one store, so
// nothing is removed as dead code. Timed with CUDA events around one launch after a
// warm-up launch.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma_chains(T *out, T a, T b, int iters) {
    T x0 = T(threadIdx.x) * T(1e-3), x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
    T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    const T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == T(-1234.5)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// integer ALU: one three-input logical operation (LOP3) per chain step; each chain also
// reads its neighbour's previous value, so no step can be folded away. (Integer adds
// may issue on other pipes, so they are left out: this measures the ALU pipe alone.)
__global__ void __launch_bounds__(256) k_alu_chains(uint32_t *out, uint32_t a, uint32_t b, int iters) {
    uint32_t x0 = threadIdx.x, x1 = x0 * 3u + 1u, x2 = x0 * 5u + 2u, x3 = x0 * 7u + 3u;
    uint32_t x4 = x0 * 11u + 4u, x5 = x0 * 13u + 5u, x6 = x0 * 17u + 6u, x7 = x0 * 19u + 7u;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
        const uint32_t y0 = x0;
        x0 = (x0 ^ x1) & a; x1 = (x1 ^ x2) | b; x2 = (x2 ^ x3) & a; x3 = (x3 ^ x4) | b;
        x4 = (x4 ^ x5) & a; x5 = (x5 ^ x6) | b; x6 = (x6 ^ x7) & a; x7 = (x7 ^ y0) | b;
    }
    const uint32_t s = ((x0 ^ x1) + (x2 ^ x3)) ^ ((x4 ^ x5) + (x6 ^ x7));
    if (s == 0x9E3779B9u) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class K>
double time_ms(K launch) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
    if (cudaEventCreate(&e1) != cudaSuccess) return -1.0;
    launch();  // warm-up
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    float ms = -1.f;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess)
        cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

}  // namespace

extern "C" {

// Thread-level operations per second of one kind: 0 FP64 FMA, 1 FP32 FMA, 2 integer
// ALU (LOP3). `iters` chain steps per thread; returns < 0 on
// a CUDA error. Uses a small scratch buffer of its own (allocated and freed here).
double pk_rate(int kind, int iters) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1.0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1.0;
    const int blocks = sms * 8, threads = 256;
    void *buf = nullptr;
    if (cudaMalloc(&buf, size_t(blocks) * threads * 8) != cudaSuccess) return -1.0;
    double ms = -1.0, per_step = 8.0;
    if (kind == 0) {
        ms = time_ms([&] { k_fma_chains<double><<<blocks, threads>>>((double *)buf, 0.9999999, 1e-7, iters); });
    } else if (kind == 1) {
        ms = time_ms([&] { k_fma_chains<float><<<blocks, threads>>>((float *)buf, 0.99999f, 1e-5f, iters); });
    } else {
        ms = time_ms([&] { k_alu_chains<<<blocks, threads>>>((uint32_t *)buf, 0x7F4A7C15u, 0x85EBCA6Bu, iters); });
    }
    cudaFree(buf);
    if (ms <= 0.0) return -1.0;
    return double(blocks) * threads * iters * per_step / (ms * 1e-3);
}

}  // extern "C"
