// Ingest + Proposition-1 test + stream compaction (one kernel, one pass over
// the frame).
//
// Per pixel: luminance -> log brightness y = ln(Y + eps) (Section 1.1,
// Section 2.1: y := L = log E; or y as given in FP16 by the renderer), write
// (y, features) into the ring slot of this frame (FP32, or FP16 + BF16 in the
// mixed form), then, in adaptive mode, evaluate the test of Proposition 1
// (Eqs. 6-9) with the model kept since the pixel's last event:
//     Delta R = (beta^T (x^c - xhat^c))^2 >= C^2   ->   flag the pixel.
// The image-coordinate part of x^c - xhat^c is zero (same pixel), so only the
// seven feature slopes enter.  Flagged pixels of the CTA's 32x8 tile are
// compacted in raster order with warp ballots and a block prefix; the tile is
// appended to the active-tile queue, and its pixels to a frame-wide flagged
// list (the tile's run padded to a multiple of four entries, so that groups of
// four aligned entries never straddle two tiles), with one atomic each per tile.
//
// Memory traffic per pixel (fp32 RGB input): 40 B in (radiance 12, normal 12,
// albedo 12, depth 4; variance is not read), 32 B ring write, 32 B model read
// (beta and sigma = beta . x^c; adaptive, t >= 1), 1 B flag; the event-pixel
// mask (1 bit per pixel) is cleared instead of the 4-byte per-pixel counts.
#include "ingest_pixel.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace esim {

__global__ void __launch_bounds__(kTilePix, 8) ingest_test_kernel(IngestParams p)
{
    const int tile = blockIdx.x;
    const int lx = threadIdx.x & 31;
    const int ly = threadIdx.x >> 5;
    const int x = (tile % p.tiles_x) * kTileX + lx;
    const int y = (tile / p.tiles_x) * kTileY + ly;
    const int flag = ingest_pixel(p, x, y);
    {
        // n_tiles * kTilePix covers both the chunk counts and the mask words
        const int g = blockIdx.x * kTilePix + threadIdx.x;
        if (g < p.n_chunks) p.chunk_cnt[g] = 0u;
        if (g < p.n_mask_words) p.ev_mask[g] = 0u;
    }
    if (!p.test) return;  // the regression walks every tile densely

    // Compact flagged pixels of the tile in raster order.
    __shared__ int warp_cnt[kTilePix / 32];
    const unsigned ballot = __ballot_sync(0xffffffffu, flag);
    if (lx == 0) warp_cnt[ly] = __popc(ballot);
    __syncthreads();
    int base = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kTilePix / 32; ++w) {
        const int c = warp_cnt[w];
        base += (w < ly) ? c : 0;
        total += c;
    }
    __shared__ uint32_t s_list_base;
    if (threadIdx.x == 0) {
        p.tile_nflag[tile] = total;
        if (total > 0) {
            const uint32_t slot = atomicAdd(&p.ctrl->tile_count, 1u);
            p.tile_queue[slot] = (uint32_t)tile;
            atomicAdd(&p.ctrl->flag_total, (uint32_t)total);
            s_list_base = atomicAdd(&p.ctrl->list_len, (uint32_t)((total + 3) & ~3));
            p.tile_base[tile] = s_list_base;
        }
    }
    __syncthreads();
    if (total > 0 && (int)threadIdx.x < ((-total) & 3))
        p.flag_list[s_list_base + total + threadIdx.x] = 0xffffffffu;
    if (flag) {
        const int pos = base + __popc(ballot & ((1u << lx) - 1u));
        p.tile_pix[(size_t)tile * kTilePix + pos] = (uint8_t)threadIdx.x;
        p.flag_list[s_list_base + pos] = (uint32_t)((size_t)y * p.W + x);
    }
}

// Staged form, for FP16 log brightness + BF16 feature frames in the precision
// form.  Persistent CTAs walk tiles blockIdx.x, blockIdx.x + gridDim.x, ...;
// thread 0 keeps the inputs and model planes of the next kIngestStages tiles
// landing by TMA, one mbarrier per stage, so each CTA has a tile of loads in
// flight while it converts, tests and compacts the current one (the one-tile
// kernel above waits for its loads with nothing else in flight).  Each thread
// takes a horizontal pair of pixels (2t, 2t + 1 in the tile's raster order:
// row t / 16, columns 2 (t % 16) and one more), reading both FP16/BF16 values
// of every plane with one 32-bit shared load.  One block barrier per tile: it
// releases the stage and publishes the warp counts.  The atomics that place a
// tile in the queue and the list are issued by thread 0 and their results used
// one tile later (thread 0 publishes the list position before the next
// barrier; every thread then writes the previous tile's list entries), so no
// thread waits for an atomic's round trip.  Same per-pixel arithmetic and the
// same raster-order compaction as ingest_test_kernel.
// Stage layout (bytes): model planes 0-1 as [2][8][128] f32 at 0, log
// brightness [8][32] u16 at 8192, features [7][8][32] u16 at 8704.
constexpr int kStageModel = 0, kStageY = 8192, kStageF = 8704;
constexpr int kPairThreads = kTilePix / 2;
static_assert(kStageF + 7 * kTilePix * 2 == kIngestStageBytes, "staged ingest layout");

__global__ void __launch_bounds__(kPairThreads) ingest_staged_kernel(const __grid_constant__ CUtensorMap map_y,
                                                                     const __grid_constant__ CUtensorMap map_f,
                                                                     const __grid_constant__ CUtensorMap map_s,
                                                                     const IngestParams p)
{
    extern __shared__ __align__(128) unsigned char sm_raw[];
    unsigned char* sm = sm_raw + ((128u - (smem_addr(sm_raw) & 127u)) & 127u);
    __shared__ uint64_t full[kIngestStages];
    __shared__ __align__(16) int warp_cnt[2][kPairThreads / 32];   // by tile parity
    __shared__ uint32_t s_base[2];                                 // list position of the tile's run, by parity
    const int t = (int)threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    const int row = t >> 4, col = 2 * (t & 15);
    // the model planes are needed only by the test
    const uint32_t tx_bytes = (uint32_t)(p.test ? kIngestStageBytes : kIngestStageBytes - kStageY);
    auto tile_of = [&](int j) { return (int)blockIdx.x + j * (int)gridDim.x; };
    auto issue = [&](int j) {
        const int tile = tile_of(j);
        if (tile >= p.n_tiles) return;
        const int st = j % kIngestStages;
        unsigned char* buf = sm + st * kIngestStageBytes;
        const int x0 = (tile % p.tiles_x) * kTileX, y0 = (tile / p.tiles_x) * kTileY;
        mbar_arrive_expect_tx(&full[st], tx_bytes);
        tma_load_2d(buf + kStageY, &map_y, &full[st], x0, y0);
        tma_load_3d(buf + kStageF, &map_f, &full[st], x0, y0, 0);
        if (p.test) tma_load_3d(buf + kStageModel, &map_s, &full[st], 4 * x0, y0, 0);
    };
    if (t == 0) {
        for (int st = 0; st < kIngestStages; ++st) mbar_init(&full[st], 1);
        mbar_fence_init();
        for (int j = 0; j < kIngestStages; ++j) issue(j);
    }
    __syncthreads();
    // tile coordinates advance by gridDim.x tiles per step
    const int step_x = (int)(gridDim.x % (unsigned)p.tiles_x), step_y = (int)(gridDim.x / (unsigned)p.tiles_x);
    int tx = (int)(blockIdx.x % (unsigned)p.tiles_x), ty = (int)(blockIdx.x / (unsigned)p.tiles_x);
    // thread 0: the previous tile's queue slot and list position, still in flight
    bool pend = false;
    int pend_tile = 0;
    uint32_t pend_slot = 0, pend_lb = 0;
    auto publish = [&](int jp) {
        if (!pend) return;
        p.tile_queue[pend_slot] = (uint32_t)pend_tile;
        p.tile_base[pend_tile] = pend_lb;
        s_base[jp & 1] = pend_lb;
        pend = false;
    };
    // this thread's list entries of the previous tile, written one tile later
    int d_f0 = 0, d_f1 = 0, d_pos = 0, d_tile = 0, d_total = 0;
    uint32_t d_pix = 0;
    auto write_deferred = [&](uint32_t base) {
        if (d_total > 0 && t < ((-d_total) & 3)) p.flag_list[base + d_total + t] = 0xffffffffu;
        if (d_f0) {
            p.tile_pix[(size_t)d_tile * kTilePix + d_pos] = (uint8_t)(2 * t);
            p.flag_list[base + d_pos] = d_pix;
        }
        if (d_f1) {
            p.tile_pix[(size_t)d_tile * kTilePix + d_pos + d_f0] = (uint8_t)(2 * t + 1);
            p.flag_list[base + d_pos + d_f0] = d_pix + 1u;
        }
    };
    int j = 0;
    bool timed_out = false;
    for (;; ++j) {
        const int tile = tile_of(j);
        if (tile >= p.n_tiles) break;
        const int st = j % kIngestStages;
        const unsigned char* buf = sm + st * kIngestStageBytes;
        const int x = tx * kTileX + col;
        const int y = ty * kTileY + row;
        tx += step_x;
        ty += step_y;
        if (tx >= p.tiles_x) {
            tx -= p.tiles_x;
            ++ty;
        }
        const bool ok = mbar_wait_bounded(&full[st], (uint32_t)(j / kIngestStages) & 1u, p.poll_limit);
        int f0 = 0, f1 = 0;
        if (ok && y < p.H && x < p.W) {
            const uint32_t yy = reinterpret_cast<const uint32_t*>(buf + kStageY)[t];
            uint32_t fq[7];
#pragma unroll
            for (int k = 0; k < 7; ++k) fq[k] = reinterpret_cast<const uint32_t*>(buf + kStageF)[k * kPairThreads + t];
            const float4* ss = reinterpret_cast<const float4*>(buf + kStageModel);
            const size_t i = (size_t)y * p.W + x;
            const size_t ii = (size_t)y * p.pitch + x;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                if (e == 1 && x + 1 >= p.W) break;
                float f[7];
                unsigned short q[7];
#pragma unroll
                for (int k = 0; k < 7; ++k) {
                    q[k] = (unsigned short)(e ? fq[k] >> 16 : fq[k] & 0xffffu);
                    f[k] = __uint_as_float((uint32_t)q[k] << 16) * p.fscale[k];
                }
                const unsigned short yh = (unsigned short)(e ? yy >> 16 : yy & 0xffffu);
                const int fl = ingest_store_test<true>(p, i + e, ii + e, __half2float(__ushort_as_half(yh)), -1.0f,
                                                       f, q, (int)yh, [&](float4& b0, float4& b1) {
                                                           b0 = ss[2 * t + e];
                                                           b1 = ss[kTilePix + 2 * t + e];
                                                       });
                if (e == 0) f0 = fl;
                else f1 = fl;
            }
        }
        {
            const int g = tile * kTilePix + 2 * t;
            if (g < p.n_chunks) p.chunk_cnt[g] = 0u;
            if (g + 1 < p.n_chunks) p.chunk_cnt[g + 1] = 0u;
            if (g < p.n_mask_words) p.ev_mask[g] = 0u;
            if (g + 1 < p.n_mask_words) p.ev_mask[g + 1] = 0u;
        }
        const unsigned b0 = __ballot_sync(0xffffffffu, f0), b1 = __ballot_sync(0xffffffffu, f1);
        if (lane == 0) warp_cnt[j & 1][warp] = __popc(b0) + __popc(b1);
        if (t == 0) publish(j - 1);
        // every thread is past its reads of stage st, warp_cnt[j & 1] is
        // complete, and s_base[(j - 1) & 1] is published
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        if (t == 0) issue(j + kIngestStages);
        if (!p.test) continue;   // the regression walks every tile densely
        if (j > 0) write_deferred(s_base[(j - 1) & 1]);

        const int4 c = *reinterpret_cast<const int4*>(warp_cnt[j & 1]);
        const int total = c.x + c.y + c.z + c.w;
        const int base = (warp > 0 ? c.x : 0) + (warp > 1 ? c.y : 0) + (warp > 2 ? c.z : 0);
        if (t == 0) {
            p.tile_nflag[tile] = total;
            if (total > 0) {   // results used one tile later (publish)
                pend_slot = atomicAdd(&p.ctrl->tile_count, 1u);
                atomicAdd(&p.ctrl->flag_total, (uint32_t)total);
                pend_lb = atomicAdd(&p.ctrl->list_len, (uint32_t)((total + 3) & ~3));
                pend_tile = tile;
                pend = true;
            }
        }
        const unsigned lt = (1u << lane) - 1u;
        d_f0 = f0;
        d_f1 = f1;
        d_pos = base + __popc(b0 & lt) + __popc(b1 & lt);
        d_pix = (uint32_t)((size_t)y * p.W + x);
        d_tile = tile;
        d_total = total;
    }
    if (!timed_out && p.test && j > 0) {
        if (t == 0) publish(j - 1);
        __syncthreads();   // the last tile's list position
        write_deferred(s_base[(j - 1) & 1]);
    }
    if (timed_out && t == 0) {
        // record the timeout; give the copies still in flight (tiles j .. j +
        // kIngestStages - 1) a bounded wait to land before the CTA exits
        atomicOr(&p.ctrl->status, kStatusTimeout);
        for (int k = j; k < j + kIngestStages; ++k)
            if (tile_of(k) < p.n_tiles)
                mbar_wait_bounded(&full[k % kIngestStages], (uint32_t)(k / kIngestStages) & 1u, p.poll_limit);
    }
}

cudaError_t launch_ingest(const IngestParams& p, int n_tiles, cudaStream_t s)
{
    ingest_test_kernel<<<n_tiles, kTilePix, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_ingest_staged(const CUtensorMap& map_y, const CUtensorMap& map_f, const CUtensorMap& map_s,
                                 const IngestParams& p, int grid, cudaStream_t s)
{
    ingest_staged_kernel<<<grid, kPairThreads, kIngestStages * kIngestStageBytes + 128, s>>>(map_y, map_f, map_s, p);
    return cudaGetLastError();
}

int ingest_staged_grid(int sms)
{
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ingest_staged_kernel, kPairThreads,
                                                      kIngestStages * kIngestStageBytes + 128) != cudaSuccess ||
        per < 1)
        per = 1;
    return per * sms;
}

}  // namespace esim
