// microbench.cu -- pipe-throughput micro-benchmarks used to put the sweep kernel on an
// ALU roofline: the sweep moves almost no bytes per sample, so its ceiling is the issue
// rate of the FP32 (FMA), integer and MUFU (transcendental) pipes.  Each kernel runs
// ILP independent dependency chains per thread of one instruction class.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/hjg.h"
#include "sampler.cuh"

namespace {

constexpr int kIlp = 8;
constexpr int kThreads = 256;

// Independent 32x32 -> 64-bit unsigned multiplies (IMAD.WIDE.U32), the Philox round's
// product: 8 chains per thread, each multiply feeding the next through its high word.
__global__ void __launch_bounds__(kThreads) imad_wide_pipe(int64_t iters, float* sink) {
    uint32_t x[kIlp];
#pragma unroll
    for (int j = 0; j < kIlp; ++j) x[j] = threadIdx.x * 7919u + j;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kIlp; ++j) {
            const uint64_t p = (uint64_t)0xD2511F53u * x[j];
            x[j] = (uint32_t)(p >> 32) + (uint32_t)p;
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < kIlp; ++j) acc ^= x[j];
    if (acc == 0x9E3779B9u) sink[threadIdx.x] = (float)acc;
}

// The low or the high 32 bits of a 32x32 product alone (mul.lo.u32 / mul.hi.u32).
template <bool HI>
__global__ void __launch_bounds__(kThreads) imul_half_pipe(int64_t iters, float* sink) {
    uint32_t x[kIlp];
#pragma unroll
    for (int j = 0; j < kIlp; ++j) x[j] = threadIdx.x * 7919u + j + 1u;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kIlp; ++j) {
            uint32_t y;
            if (HI) asm("mul.hi.u32 %0, %1, %2;" : "=r"(y) : "r"(x[j]), "r"(0xD2511F53u));
            else asm("mul.lo.u32 %0, %1, %2;" : "=r"(y) : "r"(x[j]), "r"(0xD2511F53u));
            x[j] = y ^ (uint32_t)j;
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < kIlp; ++j) acc ^= x[j];
    if (acc == 0x9E3779B9u) sink[threadIdx.x] = (float)acc;
}

// Philox4x32-10 with each round's products formed by separate high and low multiplies.
__device__ __forceinline__ uint4 philox_split(uint4 ctr, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t h0, l0, h1, l1;
        asm("mul.hi.u32 %0, %1, %2;" : "=r"(h0) : "r"(ctr.x), "r"(hjg::kPhiloxM0));
        asm("mul.lo.u32 %0, %1, %2;" : "=r"(l0) : "r"(ctr.x), "r"(hjg::kPhiloxM0));
        asm("mul.hi.u32 %0, %1, %2;" : "=r"(h1) : "r"(ctr.z), "r"(hjg::kPhiloxM1));
        asm("mul.lo.u32 %0, %1, %2;" : "=r"(l1) : "r"(ctr.z), "r"(hjg::kPhiloxM1));
        ctr = make_uint4(h1 ^ ctr.y ^ k0, l1, h0 ^ ctr.w ^ k1, l0);
        k0 += hjg::kPhiloxW0;
        k1 += hjg::kPhiloxW1;
    }
    return ctr;
}

// Philox4x32-10 with one product of each round widening and the other split.
__device__ __forceinline__ uint4 philox_mixed(uint4 ctr, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)hjg::kPhiloxM0 * ctr.x;
        uint32_t h1, l1;
        asm("mul.hi.u32 %0, %1, %2;" : "=r"(h1) : "r"(ctr.z), "r"(hjg::kPhiloxM1));
        asm("mul.lo.u32 %0, %1, %2;" : "=r"(l1) : "r"(ctr.z), "r"(hjg::kPhiloxM1));
        ctr = make_uint4(h1 ^ ctr.y ^ k0, l1, (uint32_t)(p0 >> 32) ^ ctr.w ^ k1, (uint32_t)p0);
        k0 += hjg::kPhiloxW0;
        k1 += hjg::kPhiloxW1;
    }
    return ctr;
}

__global__ void __launch_bounds__(kThreads) philox_mixed_pipe(int64_t iters, float* sink) {
    uint32_t acc = 0;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = 0; i < iters; ++i) {
        const uint4 r = philox_mixed(make_uint4(blockIdx.x, (uint32_t)i * 65536u + t, 9u, 0u), 0x1234u, 0x5678u);
        acc ^= r.x ^ r.y ^ r.z ^ r.w;
    }
    if (acc == 0x9E3779B9u) sink[threadIdx.x] = (float)acc;
}

__global__ void __launch_bounds__(kThreads) philox_split_pipe(int64_t iters, float* sink) {
    uint32_t acc = 0;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = 0; i < iters; ++i) {
        const uint4 r = philox_split(make_uint4(blockIdx.x, (uint32_t)i * 65536u + t, 9u, 0u), 0x1234u, 0x5678u);
        acc ^= r.x ^ r.y ^ r.z ^ r.w;
    }
    if (acc == 0x9E3779B9u) sink[threadIdx.x] = (float)acc;
}

template <int OP>
__device__ __forceinline__ float step(float x) {
    if (OP == HJG_MB_FFMA) return fmaf(x, 0.9999f, 0.0001f);
    if (OP == HJG_MB_EX2) return hjg::ex2_approx(-x);
    if (OP == HJG_MB_LG2) return hjg::lg2_approx(fabsf(x) + 1.0f);
    if (OP == HJG_MB_SIN) return hjg::sin_approx(x);
    if (OP == HJG_MB_COS) return hjg::cos_approx(x);
    if (OP == HJG_MB_SQRT) return hjg::sqrt_approx(x);
    return x;
}

template <int OP>
__global__ void __launch_bounds__(kThreads) float_pipe(int64_t iters, float* sink) {
    float x[kIlp];
#pragma unroll
    for (int j = 0; j < kIlp; ++j) x[j] = 0.25f + 0.01f * (threadIdx.x + j);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kIlp; ++j) x[j] = step<OP>(x[j]);
    }
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < kIlp; ++j) acc += x[j];
    if (acc == 1234.5f) sink[threadIdx.x] = acc;   // keeps the chains live
}

// Philox4x32-10 blocks with the sweep's counter layout (state and sweep words fixed per
// CTA, block index varying): the sampler's integer work, IMAD.WIDE and LOP3.
__global__ void __launch_bounds__(kThreads) philox_pipe(int64_t iters, float* sink) {
    uint32_t acc = 0;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = 0; i < iters; ++i) {
        const uint4 r = hjg::philox4x32_10(make_uint4(blockIdx.x, (uint32_t)i * 65536u + t, 9u, 0u),
                                           0x1234u, 0x5678u);
        acc ^= r.x ^ r.y ^ r.z ^ r.w;
    }
    if (acc == 0x9E3779B9u) sink[threadIdx.x] = (float)acc;
}

// Full Box-Muller normals from Philox blocks, as the sweep draws them (8 per block).
__global__ void __launch_bounds__(kThreads) normals_pipe(int64_t iters, float* sink) {
    hjg::bm_table_fill();
    __syncthreads();
    float acc = 0.0f;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = 0; i < iters; ++i) {
        float z[hjg::kNormalsPerBlock];
        hjg::block_normals<hjg::kNormalsPerBlock>((uint32_t)i * 65536u + t, blockIdx.x, 3u, 0x1234u, 0x5678u, z);
#pragma unroll
        for (int q = 0; q < hjg::kNormalsPerBlock; ++q) acc += z[q];
    }
    if (acc == 1234.5f) sink[threadIdx.x] = acc;
}

}  // namespace

extern "C" hjg_status hjg_microbench(int op, int64_t iters, double* ops_per_s, double* ms) {
    if (!ops_per_s || iters < 1) return HJG_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HJG_ECUDA;
    float* sink = nullptr;
    if (cudaMalloc(&sink, kThreads * sizeof(float)) != cudaSuccess) return HJG_ENOMEM;
    const int grid = sms * 8;
    double per_thread_iter = kIlp;
    auto launch = [&]() {
        switch (op) {
        case HJG_MB_FFMA: float_pipe<HJG_MB_FFMA><<<grid, kThreads>>>(iters, sink); break;
        case HJG_MB_EX2: float_pipe<HJG_MB_EX2><<<grid, kThreads>>>(iters, sink); break;
        case HJG_MB_LG2: float_pipe<HJG_MB_LG2><<<grid, kThreads>>>(iters, sink); break;
        case HJG_MB_SIN: float_pipe<HJG_MB_SIN><<<grid, kThreads>>>(iters, sink); break;
        case HJG_MB_COS: float_pipe<HJG_MB_COS><<<grid, kThreads>>>(iters, sink); break;
        case HJG_MB_SQRT: float_pipe<HJG_MB_SQRT><<<grid, kThreads>>>(iters, sink); break;
        case HJG_MB_PHILOX: philox_pipe<<<grid, kThreads>>>(iters, sink); break;
        case HJG_MB_NORMALS: normals_pipe<<<grid, kThreads>>>(iters, sink); break;
        case HJG_MB_IMAD_WIDE: imad_wide_pipe<<<grid, kThreads>>>(iters, sink); break;
        case HJG_MB_IMUL_LO: imul_half_pipe<false><<<grid, kThreads>>>(iters, sink); break;
        case HJG_MB_IMUL_HI: imul_half_pipe<true><<<grid, kThreads>>>(iters, sink); break;
        case HJG_MB_PHILOX_SPLIT: philox_split_pipe<<<grid, kThreads>>>(iters, sink); break;
        case HJG_MB_PHILOX_MIXED: philox_mixed_pipe<<<grid, kThreads>>>(iters, sink); break;
        }
    };
    if (op == HJG_MB_PHILOX || op == HJG_MB_PHILOX_SPLIT || op == HJG_MB_PHILOX_MIXED)
        per_thread_iter = 1.0;   // Philox blocks
    if (op == HJG_MB_NORMALS) per_thread_iter = hjg::kNormalsPerBlock;  // normals
    if (op < HJG_MB_FFMA || op > HJG_MB_PHILOX_MIXED) { cudaFree(sink); return HJG_EINVAL; }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch();   // warm-up
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float t = 0;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess || cudaGetLastError() != cudaSuccess) return HJG_ECUDA;
    *ops_per_s = (double)grid * kThreads * (double)iters * per_thread_iter / (t * 1e-3);
    if (ms) *ms = t;
    return HJG_OK;
}
