// snn_microbench.cu -- the atomic and gather rates that bound the event-driven
// delivery (S1) and potentiation (S4) on this GPU, measured with the access
// patterns those kernels use.
//
// Delivery adds every synaptic weight into its target's Q16 input (the
// paper's Sec. 2 steps 2.4-2.5, current injection) and reads the target's
// last spike time for depression (2.6); potentiation gathers every source's
// spike history.  Targets are scattered over an array the size of the net's
// input array, so the bound is the rate of int32 reductions and 4-byte
// gathers at scattered addresses in L2 (or in shared memory, when a column's
// inputs are staged there), not the HBM copy bandwidth.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "snn.h"

namespace {

constexpr int kBlock = 256;
constexpr int kUnrollMb = 8;
constexpr uint32_t kWindow = 1250;     // words of one column's inputs

__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    // integer finaliser (xor-shift-multiply), a cheap stateless hash
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__device__ __forceinline__ uint32_t below(uint32_t r, uint32_t n) { return __umulhi(r, n); }

// mode 0: red.global.add.s32 at uniformly random words of the array
// mode 1: the same inside one 1250-word window per warp (a column's inputs),
//         the window moving every 64 reductions
// mode 2: 32 consecutive words per warp instruction (a coalesced flush)
// mode 3: 4-byte loads at uniformly random words (a gather)
// mode 4: atomicAdd on shared memory at random words of a 1250-word window
__global__ void __launch_bounds__(kBlock) k_mb(int32_t *a, uint32_t n, uint32_t ops, int mode, int32_t *sink)
{
    __shared__ int32_t s_win[kWindow];
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t warp = gtid >> 5, lane = threadIdx.x & 31;
    int32_t acc = 0;
    if (mode == 4) {
        for (uint32_t i = threadIdx.x; i < kWindow; i += blockDim.x) s_win[i] = 0;
        __syncthreads();
    }
    for (uint32_t k0 = 0; k0 < ops; k0 += kUnrollMb) {
        uint32_t idx[kUnrollMb];
#pragma unroll
        for (int u = 0; u < kUnrollMb; ++u) {
            const uint32_t k = k0 + u;
            const uint32_t r = mix32(gtid * 0x9E3779B9u + k * 0x85ebca6bu + 0x1234567u);
            if (mode == 0 || mode == 3) {
                idx[u] = below(r, n);
            } else if (mode == 1) {
                const uint32_t win = below(mix32(warp * 977u + (k >> 6)), n - kWindow);
                idx[u] = win + below(r, kWindow);
            } else if (mode == 2) {
                idx[u] = (below(mix32(warp * 131u + k), n / 32u) * 32u) + lane;
            } else {
                idx[u] = below(r, kWindow);
            }
        }
        if (mode == 3) {
#pragma unroll
            for (int u = 0; u < kUnrollMb; ++u) acc ^= __ldcg(a + idx[u]);
        } else if (mode == 4) {
#pragma unroll
            for (int u = 0; u < kUnrollMb; ++u) atomicAdd(&s_win[idx[u]], 1);
        } else {
#pragma unroll
            for (int u = 0; u < kUnrollMb; ++u)
                asm volatile("red.global.add.s32 [%0], %1;" ::"l"(a + idx[u]), "r"(1) : "memory");
        }
    }
    if (mode == 4) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < kWindow; i += blockDim.x) acc += s_win[i];
    }
    if (acc == 0x7fffffff) sink[0] = acc;     // keeps the loads and the shared sums live
}

}  // namespace

extern "C" int snn_microbench_atomics(size_t array_bytes, uint32_t ops_per_thread, void *cuda_stream,
                                      snn_atomic_rates *out)
{
    if (!out || array_bytes < (size_t)kWindow * 8 || array_bytes > ((size_t)1 << 34) || ops_per_thread == 0)
        return SNN_EINVAL;
    const uint32_t n = (uint32_t)std::min<size_t>(array_bytes / 4, 0xffffffffu);
    const uint32_t ops = (ops_per_thread + kUnrollMb - 1) / kUnrollMb * kUnrollMb;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mb, kBlock, 0) != cudaSuccess)
        return SNN_ECUDA;
    const int grid = sms * std::max(1, per_sm);
    int32_t *a = nullptr, *sink = nullptr;
    if (cudaMalloc(&a, (size_t)n * 4) != cudaSuccess) {
        cudaGetLastError();
        return SNN_ENOMEM;
    }
    if (cudaMalloc(&sink, 16) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(a);
        return SNN_ENOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double rate[5] = {0, 0, 0, 0, 0};
    int rc = SNN_OK;
    cudaMemsetAsync(a, 0, (size_t)n * 4, s);
    for (int mode = 0; mode < 5 && rc == SNN_OK; ++mode) {
        k_mb<<<grid, kBlock, 0, s>>>(a, n, ops, mode, sink);    // warm-up
        cudaEventRecord(e0, s);
        k_mb<<<grid, kBlock, 0, s>>>(a, n, ops, mode, sink);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = SNN_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        rate[mode] = (double)grid * kBlock * ops / (ms * 1e-3) / 1e9;
    }
    if (cudaGetLastError() != cudaSuccess) rc = SNN_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(a);
    out->red_global_random_gops = rate[0];
    out->red_global_window_gops = rate[1];
    out->red_global_coalesced_gops = rate[2];
    out->ld_global_random_gops = rate[3];
    out->atom_shared_window_gops = rate[4];
    out->array_bytes = (double)n * 4;
    out->threads = (double)grid * kBlock;
    return rc;
}
