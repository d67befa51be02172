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
// (beta and sigma = beta . x^c; adaptive, t >= 1), 1 B flag + 4 B event-count
// clear.
#include "ingest_pixel.cuh"
#include "internal.h"

namespace esim {

__global__ void __launch_bounds__(kTilePix) ingest_test_kernel(IngestParams p)
{
    const int tile = blockIdx.x;
    const int lx = threadIdx.x & 31;
    const int ly = threadIdx.x >> 5;
    const int x = (tile % p.tiles_x) * kTileX + lx;
    const int y = (tile / p.tiles_x) * kTileY + ly;
    const int flag = ingest_pixel(p, x, y);
    {
        const int g = blockIdx.x * kTilePix + threadIdx.x;
        if (g < p.n_chunks) p.chunk_cnt[g] = 0u;
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

cudaError_t launch_ingest(const IngestParams& p, int n_tiles, cudaStream_t s)
{
    ingest_test_kernel<<<n_tiles, kTilePix, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace esim
