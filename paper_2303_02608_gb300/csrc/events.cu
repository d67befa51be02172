// Ordered event writer (Eq. 1 records at fixed frame times).
//
// The solve kernel leaves a signed per-pixel event count p*n in a map and,
// in the simulator's own path, already sums |p*n| per 2048-pixel chunk and
// sets one bit per emitting pixel in a mask, so only the write launch runs and
// it reads counts only under set bits (the frame's other counts are stale:
// the ingest clears the mask, not the map); the stand-alone writer runs both
// launches below on a dense map.
// Either way the records come out in canonical order (row, column, repeat)
// without sorting and without atomics on the output position, so the output
// is deterministic:
//   1. count: each 2048-pixel chunk sums |p*n| (counts beyond
//      kMaxCountPerPixel in magnitude set a status bit instead).
//   2. write: each chunk's CTA adds up the counts of all earlier chunks for
//      its offset, rescans its pixels and writes its records there.  The
//      buffer is a ring: position pos sits at pos mod capacity.  A record
//      that would leave more than capacity records undrained (from the
//      positions drained when the frame was pushed on) is dropped and the
//      sticky overflow bit is set; the total still counts it.
#include "internal.h"
#include "block_scan.cuh"

namespace esim {

namespace {

constexpr int kThreads = 256;
constexpr int kPer = kChunk / kThreads;  // 8 pixels per thread

__global__ void __launch_bounds__(kThreads) event_count_kernel(EventParams p)
{
    __shared__ int s_warp[kThreads / 32];
    const long long p0 = (long long)blockIdx.x * kChunk + (long long)threadIdx.x * kPer;
    int c = 0;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        if (p0 + k >= p.n_pix) continue;
        const int v = p.nev[p0 + k];
        if (v > kMaxCountPerPixel || v < -kMaxCountPerPixel) bad = true;
        else c += v < 0 ? -v : v;
    }
    if (bad) atomicOr(&p.ctrl->status, kStatusCountRange);
    int total;
    block_exclusive_scan(c, s_warp, total);
    if (threadIdx.x == 0) p.chunk_cnt[blockIdx.x] = (uint32_t)total;
}

// Sum of chunk_cnt[0, n) by the whole block (every thread gets the sum).
__device__ __forceinline__ unsigned long long block_prefix_count(const uint32_t* cnt, int n, unsigned long long* s_red)
{
    unsigned long long v = 0;
    for (int j = (int)threadIdx.x; j < n; j += kThreads) v += cnt[j];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long t = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) t += s_red[w];
    return t;
}

// Each chunk finds its output offset itself: the event total before this
// frame (ev_base) plus the counts of all earlier chunks, summed by the block
// (no CTA waits on another and no serial scan); the last chunk's CTA records
// the new total.
__global__ void __launch_bounds__(kThreads) event_write_kernel(EventParams p)
{
    __shared__ int s_warp[kThreads / 32];
    __shared__ unsigned long long s_red[kThreads / 32];
    const bool last = blockIdx.x == gridDim.x - 1;
    const uint32_t cnt = p.chunk_cnt[blockIdx.x];
    if (cnt == 0u && !last) return;   // no events in this chunk
    const long long p0 = (long long)blockIdx.x * kChunk + (long long)threadIdx.x * kPer;
    int v[kPer];
    if (p.ev_mask) {
        // the thread's 8 pixels are one byte of the chunk's 64 mask words
        const uint32_t word = p.ev_mask[(size_t)blockIdx.x * (kChunk / 32) + (threadIdx.x >> 2)];
        const uint32_t m = (word >> ((threadIdx.x & 3u) * 8u)) & 0xffu;
#pragma unroll
        for (int k = 0; k < kPer; ++k) v[k] = ((m >> k) & 1u) ? p.nev[p0 + k] : 0;
    } else if (p0 + kPer <= p.n_pix && ((reinterpret_cast<uintptr_t>(p.nev + p0) & 15u) == 0)) {
        const int4 a = *reinterpret_cast<const int4*>(p.nev + p0);
        const int4 b = *reinterpret_cast<const int4*>(p.nev + p0 + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int k = 0; k < kPer; ++k) v[k] = (p0 + k < p.n_pix) ? p.nev[p0 + k] : 0;
    }
    const unsigned long long drained = p.drained;
    const unsigned long long before = p.ctrl->ev_base + block_prefix_count(p.chunk_cnt, blockIdx.x, s_red);
    const bool range_ok = (p.ctrl->status & kStatusCountRange) == 0u;
    if (last && threadIdx.x == 0) {
        if (!range_ok) {
            p.ctrl->ev_total = ~0ull;   // the map was out of range: nothing is written
        } else {
            p.ctrl->ev_total = before + cnt;
            p.ctrl->ev_cum += before + cnt - p.ctrl->ev_base;
            p.ctrl->frame_end[p.frame % kFrameEnds] = before + cnt;
        }
    }
    if (cnt == 0u || !range_ok) return;
    // the ring index of the chunk's first record: one division per CTA,
    // published by the scan's barriers
    __shared__ unsigned long long s_base_idx;
    if (threadIdx.x == 0) s_base_idx = p.capacity ? before % p.capacity : 0ull;
    int c = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) c += abs(v[k]);
    int total;
    const int off = block_exclusive_scan(c, s_warp, total);
    if (total == 0) return;
    // positions run on from the earlier frames' records; position pos is kept
    // at pos mod capacity while it leaves the undrained records (from
    // `drained` on) no more than capacity long, else it is dropped
    unsigned long long pos = before + (unsigned long long)off;
    unsigned long long idx = s_base_idx + (unsigned long long)off;
    if (idx >= p.capacity) idx = p.capacity ? idx % p.capacity : 0ull;   // rare: a wrap inside the chunk
    bool overflow = false;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int n = abs(v[k]);
        if (n == 0) continue;
        const long long pix = p0 + k;
        const uint32_t x = (uint32_t)(pix % p.W), y = (uint32_t)(pix / p.W);
        const uint32_t w1 = x | (y << 16);
        const uint32_t w2 = (uint32_t)(uint8_t)(int8_t)(v[k] > 0 ? 1 : -1);
        for (int e = 0; e < n; ++e) {
            if (pos - drained >= p.capacity) {
                overflow = true;
            } else {
                uint32_t* rec = reinterpret_cast<uint32_t*>(p.events + idx);
                rec[0] = p.frame;
                rec[1] = w1;
                rec[2] = w2;
            }
            ++pos;
            if (++idx == p.capacity) idx = 0;
        }
    }
    if (overflow) atomicOr(&p.ctrl->status, kStatusOverflow);
}

}  // namespace

cudaError_t launch_event_write(const EventParams& p, cudaStream_t s)
{
    event_write_kernel<<<p.n_chunks, kThreads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_events(const EventParams& p, cudaStream_t s)
{
    event_count_kernel<<<p.n_chunks, kThreads, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    event_write_kernel<<<p.n_chunks, kThreads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace esim
