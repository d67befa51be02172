// Block-wide exclusive scan of one int per thread (blocks of up to 256 threads,
// a multiple of 32).
#pragma once

namespace esim {

// Returns this thread's exclusive prefix; `total` receives the block sum.
// s_warp must hold blockDim.x / 32 ints of shared memory; every thread of the
// block calls it.
__device__ __forceinline__ int block_exclusive_scan(int v, int* s_warp, int& total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    int base = 0;
    total = 0;
    const int nw = (int)(blockDim.x >> 5);
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        if (w >= nw) break;
        const int c = s_warp[w];
        base += (w < wid) ? c : 0;
        total += c;
    }
    __syncthreads();
    return base + x - v;
}

// The same for 64-bit values; s_warp must hold blockDim.x / 32 values.
__device__ __forceinline__ unsigned long long block_exclusive_scan64(unsigned long long v, unsigned long long* s_warp,
                                                                     unsigned long long& total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    unsigned long long base = 0;
    total = 0;
    const int nw = (int)(blockDim.x >> 5);
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        if (w >= nw) break;
        const unsigned long long c = s_warp[w];
        base += (w < wid) ? c : 0ull;
        total += c;
    }
    __syncthreads();
    return base + x - v;
}

}  // namespace esim
