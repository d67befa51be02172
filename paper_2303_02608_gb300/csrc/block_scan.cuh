// Block-wide exclusive scan of one int per thread (blocks of 256 threads).
#pragma once

namespace esim {

// Returns this thread's exclusive prefix; `total` receives the block sum.
// s_warp must hold 8 ints of shared memory; every thread of the block calls it.
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
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const int c = s_warp[w];
        base += (w < wid) ? c : 0;
        total += c;
    }
    __syncthreads();
    return base + x - v;
}

}  // namespace esim
