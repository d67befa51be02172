// Ordered event writer (Eq. 1 records at fixed frame times).
//
// The regression kernel leaves a signed per-pixel event count p*n in a map
// and, in the simulator's own path, already sums |p*n| per 2048-pixel chunk
// and scans the chunk counts (its last CTA), so only the write launch runs.
// The stand-alone writer runs both launches below.  Either way the records
// come out in canonical order (row, column, repeat) without sorting and
// without atomics on the output position, so the output is deterministic:
//   1. count: each 2048-pixel chunk sums |p*n|; the last CTA to finish (ticket
//      from an atomic counter, after a release fence) scans the chunk counts
//      into global offsets and advances the event total.  No CTA waits on
//      another.
//   2. write: each chunk rescans its pixels and writes its records at its
//      offset.  Records past the buffer capacity are dropped and the sticky
//      overflow bit is set; the total still counts them.
#include "internal.h"
#include "block_scan.cuh"

namespace esim {

namespace {

constexpr int kThreads = 256;
constexpr int kPer = kChunk / kThreads;  // 8 pixels per thread

__global__ void __launch_bounds__(kThreads) event_count_kernel(EventParams p)
{
    __shared__ int s_warp[kThreads / 32];
    __shared__ bool s_last;
    const long long p0 = (long long)blockIdx.x * kChunk + (long long)threadIdx.x * kPer;
    int c = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k)
        if (p0 + k < p.n_pix) c += abs(p.nev[p0 + k]);
    int total;
    block_exclusive_scan(c, s_warp, total);
    if (threadIdx.x == 0) {
        p.chunk_cnt[blockIdx.x] = (uint32_t)total;
        __threadfence();
        const uint32_t ticket = atomicAdd(&p.ctrl->chunk_done, 1u);
        s_last = (ticket == (uint32_t)p.n_chunks - 1u);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // last CTA: exclusive scan of the chunk counts, in chunk order
    unsigned long long running = *(volatile unsigned long long*)&p.ctrl->ev_total;
    for (int base = 0; base < p.n_chunks; base += kThreads) {
        const int j = base + threadIdx.x;
        const int v = (j < p.n_chunks) ? (int)*(volatile uint32_t*)&p.chunk_cnt[j] : 0;
        int seg;
        const int off = block_exclusive_scan(v, s_warp, seg);
        if (j < p.n_chunks) p.chunk_off[j] = running + (unsigned long long)off;
        running += (unsigned long long)seg;
    }
    if (threadIdx.x == 0) {
        const unsigned long long added = running - p.ctrl->ev_total;
        p.ctrl->ev_total = running;
        p.ctrl->ev_cum += added;
    }
}

__global__ void __launch_bounds__(kThreads) event_write_kernel(EventParams p)
{
    __shared__ int s_warp[kThreads / 32];
    if (p.chunk_cnt[blockIdx.x] == 0u) return;   // no events in this chunk
    const long long p0 = (long long)blockIdx.x * kChunk + (long long)threadIdx.x * kPer;
    int v[kPer];
    int c = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        v[k] = (p0 + k < p.n_pix) ? p.nev[p0 + k] : 0;
        c += abs(v[k]);
    }
    int total;
    const int off = block_exclusive_scan(c, s_warp, total);
    if (total == 0) return;
    unsigned long long pos = p.chunk_off[blockIdx.x] + (unsigned long long)off;
    bool overflow = false;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int n = abs(v[k]);
        if (n == 0) continue;
        const long long pix = p0 + k;
        const uint32_t x = (uint32_t)(pix % p.W), y = (uint32_t)(pix / p.W);
        const uint32_t w1 = x | (y << 16);
        const uint32_t w2 = (uint32_t)(uint8_t)(int8_t)(v[k] > 0 ? 1 : -1);
        for (int e = 0; e < n; ++e, ++pos) {
            if (pos >= p.capacity) {
                overflow = true;
                continue;
            }
            uint32_t* rec = reinterpret_cast<uint32_t*>(p.events + pos);
            rec[0] = p.frame;
            rec[1] = w1;
            rec[2] = w2;
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
