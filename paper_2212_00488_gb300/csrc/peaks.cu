// Throughput microbenchmarks for the fused kernel's roofline denominators:
// dependency-free chains of 32-bit integer add, xor and min (the operations
// the algorithmic count of Eqs. 3-9 consists of), population count, and
// 16-byte shared-memory loads. Each kernel runs many independent chains per
// thread with every SM full of warps, so the measured rate is the hardware's
// issue or pipe limit for that operation, not a latency.
#include "internal.cuh"

#include "stereo.h"

namespace stereo {
namespace {

constexpr int kChains = 8;
constexpr int kPeakNT = 256;

__device__ __forceinline__ uint32_t op_add(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm volatile("add.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t op_xor(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm volatile("xor.b32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t op_min(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm volatile("min.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t op_popc(uint32_t a)
{
    uint32_t r;
    asm volatile("popc.b32 %0, %1;" : "=r"(r) : "r"(a));
    return r;
}

// 3 operations per chain and iteration (add, xor, min).
__global__ void __launch_bounds__(kPeakNT) int_alu_kernel(uint32_t *out, int iters, uint32_t seed)
{
    uint32_t v[kChains];
    const uint32_t k = seed ^ threadIdx.x;
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = k + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = op_add(v[c], k);
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = op_xor(v[c], seed);
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = op_min(v[c], k | 0x80000000u);
    }
    uint32_t r = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) r ^= v[c];
    if (r == seed) out[blockIdx.x] = r;             // never true in practice; keeps the work alive
}

// 1 population count per chain and iteration.
__global__ void __launch_bounds__(kPeakNT) popc_kernel(uint32_t *out, int iters, uint32_t seed)
{
    uint32_t v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = seed ^ (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = op_popc(v[c]);
    }
    uint32_t r = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) r ^= v[c];
    if (r == seed) out[blockIdx.x] = r;
}

// 16-byte shared-memory loads, consecutive threads on consecutive 16-byte
// words (no bank conflicts); kChains independent loads per iteration.
__global__ void __launch_bounds__(kPeakNT) lds_kernel(uint32_t *out, int iters, uint32_t seed)
{
    __shared__ uint4 buf[kChains][kPeakNT];
#pragma unroll
    for (int c = 0; c < kChains; ++c) buf[c][threadIdx.x] = make_uint4(seed + c, threadIdx.x, c, seed);
    __syncthreads();
    uint32_t acc = 0;
    const int t = threadIdx.x;
    for (int i = 0; i < iters; ++i) {
        uint4 r[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            const uint4 *p = &buf[c][(t + i) & (kPeakNT - 1)];
            asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(r[c].x), "=r"(r[c].y), "=r"(r[c].z), "=r"(r[c].w)
                         : "r"((uint32_t)__cvta_generic_to_shared(p)));
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc += r[c].x ^ r[c].w;
    }
    if (acc == 0xFFFFFFFFu) out[blockIdx.x] = acc;
}

template <class K>
double time_kernel(K kernel, int grid, uint32_t *out, int iters, cudaStream_t s, float &ms)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    kernel<<<grid, kPeakNT, 0, s>>>(out, iters / 8, 1u);   // warm-up
    cudaEventRecord(e0, s);
    kernel<<<grid, kPeakNT, 0, s>>>(out, iters, 12345u);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

}  // namespace
}  // namespace stereo

extern "C" int stereo_measure_peaks(int device, double *int_ops_per_s, double *popc_per_s, double *lds_bytes_per_s)
{
    using namespace stereo;
    if (!int_ops_per_s || !popc_per_s || !lds_bytes_per_s) return STEREO_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return STEREO_ECUDA;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return STEREO_ECUDA;
    uint32_t *out = nullptr;
    if (cudaMalloc(&out, sizeof(uint32_t) * nsm * 8) != cudaSuccess) return STEREO_ENOMEM;
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(out);
        return STEREO_ECUDA;
    }
    const int grid = nsm * 8;                       // 8 CTAs of 256 threads: 64 warps per SM
    const double threads = (double)grid * kPeakNT;
    float ms = 0.f;
    const int it_alu = 4096, it_popc = 4096, it_lds = 2048;
    time_kernel(int_alu_kernel, grid, out, it_alu, s, ms);
    *int_ops_per_s = threads * it_alu * kChains * 3 / (ms * 1e-3);
    time_kernel(popc_kernel, grid, out, it_popc, s, ms);
    *popc_per_s = threads * it_popc * kChains / (ms * 1e-3);
    time_kernel(lds_kernel, grid, out, it_lds, s, ms);
    *lds_bytes_per_s = threads * it_lds * kChains * 16.0 / (ms * 1e-3);
    const cudaError_t e = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    cudaFree(out);
    return e == cudaSuccess ? STEREO_OK : STEREO_ECUDA;
}
