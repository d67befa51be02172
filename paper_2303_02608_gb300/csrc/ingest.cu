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
// list, with one atomic each per tile.
//
// Memory traffic per pixel (fp32 RGB input): 40 B in (radiance 12, normal 12,
// albedo 12, depth 4; variance is not read), 32 B ring write, 32 B model read
// (beta and sigma = beta . x^c; adaptive, t >= 1), 1 B flag + 4 B event-count
// clear.
#include "internal.h"

namespace esim {

__global__ void __launch_bounds__(kTilePix) ingest_test_kernel(IngestParams p)
{
    const int tile = blockIdx.x;
    const int lx = threadIdx.x & 31;
    const int ly = threadIdx.x >> 5;
    const int x = (tile % p.tiles_x) * kTileX + lx;
    const int y = (tile / p.tiles_x) * kTileY + ly;
    const bool inside = x < p.W && y < p.H;
    const size_t N = (size_t)p.W * p.H;
    int flag = 0;
    if (inside) {
        const size_t i = (size_t)y * p.W + x;
        float yv;
        if (p.rad_fmt == ESIM_AD_LOGLUMA_F16) {
            yv = __half2float(reinterpret_cast<const __half*>(p.rad)[i]);
        } else {
            const float* rad = reinterpret_cast<const float*>(p.rad);
            float Y;
            if (p.rad_fmt == ESIM_AD_RGB_F32) {
                // Rec.709 luminance of the RGB radiance
                Y = 0.2126f * __ldg(rad + i) + 0.7152f * __ldg(rad + N + i) + 0.0722f * __ldg(rad + 2 * N + i);
            } else {
                Y = __ldg(rad + i);
            }
            yv = logf(Y + p.log_eps);
        }
        float f[7];   // normal xyz, depth, albedo rgb
        if (p.feat_fmt == ESIM_AD_FEAT_BF16) {
#pragma unroll
            for (int j = 0; j < 7; ++j)
                f[j] = __uint_as_float((uint32_t)__ldg(p.feat_bf16 + j * N + i) << 16) * p.fscale[j];
        } else {
            f[0] = __ldg(p.normal + i);
            f[1] = __ldg(p.normal + N + i);
            f[2] = __ldg(p.normal + 2 * N + i);
            f[3] = __ldg(p.depth + i);
            f[4] = __ldg(p.albedo + i);
            f[5] = __ldg(p.albedo + N + i);
            f[6] = __ldg(p.albedo + 2 * N + i);
        }
        if (p.mixed) {
            // FP16 log brightness and BF16 features; the test below sees the
            // stored (dequantised) values, as the regression will
            unsigned short q[7];
#pragma unroll
            for (int j = 0; j < 7; ++j) {
                q[j] = __bfloat16_as_ushort(__float2bfloat16_rn(f[j] * p.inv_fscale[j]));
                f[j] = __uint_as_float((uint32_t)q[j] << 16) * p.fscale[j];
            }
            reinterpret_cast<uint4*>(p.ring)[(size_t)p.slot * N + i] =
                pack_mixed(__half_as_ushort(__float2half_rn(yv)), q);
        } else {
            float4* ring = reinterpret_cast<float4*>(p.ring);
            ring[(size_t)(2 * p.slot) * N + i] = make_float4(yv, f[0], f[1], f[2]);
            ring[(size_t)(2 * p.slot + 1) * N + i] = make_float4(f[3], f[4], f[5], f[6]);
        }
        const float n0 = f[0], n1 = f[1], n2 = f[2], d = f[3], a0 = f[4], a1 = f[5], a2 = f[6];
        if (p.test) {
            // beta^T (x^c - xhat) = sigma - beta . xhat, sigma = beta . x^c kept in the model
            const float4 b0 = p.state[i];
            const float4 b1 = p.state[N + i];
            const float s = b1.w - dot7(b0, b1, n0, n1, n2, d, a0, a1, a2);
            flag = (s * s >= p.C * p.C) ? 1 : 0;
        } else {
            flag = 1;
        }
        p.flag[i] = (uint8_t)flag;
        p.nev[i] = 0;
    }
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
            s_list_base = atomicAdd(&p.ctrl->flag_total, (uint32_t)total);
        }
    }
    __syncthreads();
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
