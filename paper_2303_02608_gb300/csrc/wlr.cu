// Weighted local regression (Eqs. 3-5) with fused event emission (Eq. 1).
//
// Work unit: a 32x8 pixel tile.  For each frame tau of the temporal window
// t-T+1..t the tile plus an r-pixel halo of that frame's ring slot
// ((32+2r) x (8+2r) pixels x 2 float4 half-planes) is staged in shared memory
// by one 4-D TMA load.  CTAs are persistent: they pull work items (tiles, or
// chunks of a tile's flagged pixels) from a counter and keep up to three staged
// frames in flight, so the copy of the next frame or item overlaps the
// arithmetic on the current one.  Pixels outside the image arrive zero-filled and are never
// read: each centre's offset range is clipped to the image instead.
//
// Each regressed pixel is owned by g lanes (g = 1 when its tile is densely
// flagged, up to 32 when it holds few flagged pixels); the lanes split the
// window's offsets, accumulate the weighted Gram matrix of z = (1, u) and the
// right-hand side in registers, and are reduced with warp shuffles.  Regressors
// are the feature differences scaled by k / (h b_j), k = sqrt(log2(e) / 2), so
// the product Gaussian of Eq. 5 is one exp2:  w = 2^(-|u|^2).  The slopes are
// mapped back to natural units afterwards; the ridge lambda * W * |beta|^2 is
// added on the scaled diagonal as lambda * W * s_j^2.  The 10x10 system is
// Jacobi-equilibrated and solved by Cholesky in fp32.
//
// Epilogue (Eq. 1, fixed frame times): Delta L = alpha - L_last,
// n = floor(|Delta L| / C); if n >= 1 the pixel emits n events of polarity
// sign(Delta L) (recorded in the per-pixel count map for the ordered event
// writer), L_last moves by p n C and the model (beta, x^c) is replaced by the
// new fit (Fig. 1: the model is kept until a new event).  Frame 0 only
// initialises L_last = alpha and the model.
#include "block_scan.cuh"
#include "internal.h"
#include "ptx.cuh"
#include "wlr_math.cuh"
#include "sparse_stage.cuh"

namespace esim {

namespace {

}  // namespace

// Per-stage metadata published by the producer thread with each staged frame.
struct StageInfo {
    int tile;   // tile index, or -1: no more work (end of the CTA's stream)
    int k;      // position in the temporal window: tau = t - k
    int first;  // first entry of the tile's pixel list in this work item
    int count;  // pixels in this work item
};

// Per-CTA shared-memory layout (after 128-byte alignment):
//   nbuf stage buffers, each 2 half-planes of (32+2r) x (8+2r) float4
//   full[nbuf] mbarriers, released[nbuf] counters, info[nbuf], window table [(2r+1)^2] float4
struct SmemLayout {
    int buf_bytes, nbuf, table_off, bar_off, info_off, total;
};

__host__ __device__ inline SmemLayout smem_layout(int r, int nbuf, bool mixed)
{
    SmemLayout L;
    const int stage = (mixed ? 1 : 2) * (kTileX + 2 * r) * (kTileY + 2 * r) * 16;
    L.buf_bytes = (stage + 127) & ~127;
    L.nbuf = nbuf;
    L.bar_off = nbuf * L.buf_bytes;
    L.info_off = L.bar_off + 2 * nbuf * 8;
    L.table_off = (L.info_off + nbuf * (int)sizeof(StageInfo) + 15) & ~15;
    L.total = L.table_off + (2 * r + 1) * (2 * r + 1) * 16 + 128;  // + alignment slack
    return L;
}

// Persistent regression kernel.  Each CTA pulls work items from a counter
// (every tile in dense mode, chunks of the active-tile queue otherwise) and
// keeps up to nbuf staged frames in flight, each a (work item, tau) pair
// published in `info` and landed by TMA on full[b].  Every warp consumes every
// stage in order and then counts itself out of the buffer; the warp that
// releases a buffer last issues that buffer's next copy at once, so no warp
// waits for another and copies start as early as possible.
template <bool kDense, bool kMixed>
__global__ void __launch_bounds__(kTilePix, 2)
    wlr_kernel(const __grid_constant__ CUtensorMap tmap, const WlrParams p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations must be 128-byte aligned; the allocation has 128 bytes of slack
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    const SmemLayout L = smem_layout(p.r, p.nbuf, kMixed);
    const int plane = p.sw * p.sh;                      // 16-byte records per half-plane
    const uint32_t stage_bytes = (uint32_t)((kMixed ? 1 : 2) * plane * 16);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    int* released = reinterpret_cast<int*>(full + L.nbuf);
    StageInfo* info = reinterpret_cast<StageInfo*>(smem + L.info_off);
    float4* table = reinterpret_cast<float4*>(smem + L.table_off);
    const int lane = threadIdx.x & 31;
    if (!kDense && *(volatile uint32_t*)&p.ctrl->flag_total <= p.sparse_max && p.sparse_max > 0)
        return;  // the sparse kernel's frame
    const int n_work = kDense ? p.n_tiles : (int)*(volatile uint32_t*)&p.ctrl->tile_count;
    const int side = 2 * p.r + 1;
    const int nq = side * side;
    const float spx = p.s_coord_px;

    // window walk table for lanes that split one interior pixel's window:
    // (smem offset, u_dx, u_dy, -(u_dx^2 + u_dy^2)) per offset
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        const int ox = q % side - p.r, oy = q / side - p.r;
        const float u1 = (float)ox * spx, u2 = (float)oy * spx;
        table[q] = make_float4(__int_as_float(oy * p.sw + ox), u1, u2, -fmaf(u1, u1, u2 * u2));
    }
    if (threadIdx.x == 0) {
        for (int b = 0; b < L.nbuf; ++b) {
            mbar_init(&full[b], 1);
            released[b] = 0;
        }
        mbar_fence_init();
    }
    __syncthreads();

    // ---- work items.  Dense: one per tile.  Queue: each active tile's pixel
    // list is cut into chunks of `chunk` pixels (chosen from this frame's flagged
    // total so that every CTA gets several items), item w -> (queue slot w / per,
    // chunk w % per); chunks past a tile's count are empty and skipped.
    int chunk = kTilePix, per = 1, n_items = n_work;
    if (!kDense) {
        const uint32_t total = *(volatile uint32_t*)&p.ctrl->flag_total;
        const uint32_t target = total / (uint32_t)(gridDim.x * 8u);
        chunk = 16;
        while (chunk < kTilePix && (uint32_t)chunk < target) chunk <<= 1;
        per = kTilePix / chunk;
        n_items = n_work * per;
    }

    // ---- producer state, shared by whichever thread issues the next stage;
    // kept in shared memory so the consumers' accumulators keep the registers.
    // Stages are issued strictly in order: issuing stage S waits (bounded) until
    // stage S-1 has been issued.
    struct Producer {
        int tile, k, first, count, issued, done, ok;
    };
    __shared__ Producer pr_store;
    volatile Producer* pr = &pr_store;
    if (threadIdx.x == 0) {
        pr->tile = -1;
        pr->k = pr->first = pr->count = pr->issued = pr->done = 0;
        pr->ok = 1;
    }
    auto produce = [&](int S) {
        for (uint32_t spin = 0; pr->issued != S && !pr->done; ++spin) {
            if (spin > (1u << 26)) {
                pr->ok = 0;
                return;
            }
        }
        if (pr->done) return;
        const int b = S % L.nbuf;
        if (pr->tile < 0 || pr->k == p.n_tau) {
            int tile = -1, first = 0, count = 0;
            while (pr->ok) {
                const int w = (int)atomicAdd(&p.ctrl->work_next, 1u);
                if (w >= n_items) break;
                if (kDense) {
                    tile = w;
                    count = kTilePix;
                    break;
                }
                const int t = (int)p.tile_queue[w / per];
                const int np = p.tile_nflag[t];
                const int f = (w % per) * chunk;
                if (f >= np) continue;               // empty chunk
                tile = t;
                first = f;
                count = min(chunk, np - f);
                break;
            }
            if (tile < 0) {
                pr->done = 1;
                pr->tile = -1;
                info[b].tile = -1;
                __threadfence_block();
                mbar_arrive(&full[b]);               // end of stream, no copy
                pr->issued = S + 1;
                return;
            }
            pr->tile = tile;
            pr->first = first;
            pr->count = count;
            pr->k = 0;
        }
        const int tile = pr->tile, k = pr->k;
        info[b].tile = tile;
        info[b].k = k;
        info[b].first = pr->first;
        info[b].count = pr->count;
        const int tx0 = (tile % p.tiles_x) * kTileX, ty0 = (tile / p.tiles_x) * kTileY;
        const int slot = (p.t - k) % p.T;
        pr->k = k + 1;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&full[b], stage_bytes);
        tma_load_4d(smem + b * L.buf_bytes, &tmap, &full[b], 0, tx0 - p.r, ty0 - p.r,
                    kMixed ? slot : 2 * slot);
        __threadfence_block();
        pr->issued = S + 1;
    };
    // ---- consumer state
    Acc acc;
    const float* sf = kMixed ? p.q_scale : p.s_feat;   // regressor scale of a stored value
    float cf[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) cf[j] = 0.0f;
    int g = 1, lg = 0, sub = 0, npix = 0, cx = 0, cy = 0, sx = 0, sy = 0;
    int dxlo = 0, dxhi = 0, dylo = 0, dyhi = 0;
    bool active = false;
    bool timed_out = false;
    __shared__ unsigned long long s_pairs, s_pix, s_fp64;
    if (threadIdx.x == 0) {
        s_pairs = 0ull;
        s_pix = 0ull;
        s_fp64 = 0ull;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int i = 0; i < L.nbuf; ++i) produce(i);

    int s_fail = 0;
    for (int s = 0;; ++s) {
        const int b = s % L.nbuf;
        if (!mbar_wait_bounded(&full[b], (uint32_t)((s / L.nbuf) & 1))) {
            timed_out = true;
            s_fail = s;
            break;
        }
        const StageInfo in = info[b];
        if (in.tile < 0) break;
        const float4* P0 = reinterpret_cast<const float4*>(smem + b * L.buf_bytes);
        const float4* P1 = P0 + plane;
        const uint4* PM = reinterpret_cast<const uint4*>(smem + b * L.buf_bytes);
        // accumulate the neighbour at staged index si (either ring form)
        auto at = [&](int si, float u1, float u2, float en0) {
            if (kMixed)
                accumulate(acc, PM[si], u1, u2, en0, sf, cf);
            else
                accumulate(acc, P0[si], P1[si], u1, u2, en0, sf, cf);
        };
        if (in.k == 0) {
            // new tile: assign lanes to its regressed pixels
            const int tx0 = (in.tile % p.tiles_x) * kTileX, ty0 = (in.tile / p.tiles_x) * kTileY;
            npix = in.count;
            lg = 0;
            if (!kDense) lg = npix > 128 ? 0 : npix > 64 ? 1 : npix > 32 ? 2 : npix > 16 ? 3 : npix > 8 ? 4 : 5;
            g = 1 << lg;
            const int item = (int)threadIdx.x >> lg;
            sub = (int)threadIdx.x & (g - 1);
            active = item < npix;
            const int lidx = kDense ? (int)threadIdx.x
                                    : (active ? (int)p.tile_pix[(size_t)in.tile * kTilePix + in.first + item] : 0);
            const int lx = lidx & (kTileX - 1), ly = lidx / kTileX;
            cx = tx0 + lx;
            cy = ty0 + ly;
            if (cx >= p.W || cy >= p.H) active = false;
            dxlo = max(-p.r, -cx);
            dxhi = min(p.r, p.W - 1 - cx);
            dylo = max(-p.r, -cy);
            dyhi = min(p.r, p.H - 1 - cy);
            sx = lx + p.r;
            sy = ly + p.r;
#pragma unroll
            for (int i = 0; i < NG; ++i) acc.G[i] = 0.0f;
#pragma unroll
            for (int i = 0; i < NZ; ++i) acc.B[i] = 0.0f;
            if (active) {
                float c[7];
                if (kMixed) {
                    float yc;
                    unpack_mixed(PM[sy * p.sw + sx], yc, c);
                } else {
                    const float4 c0 = P0[sy * p.sw + sx];
                    const float4 c1 = P1[sy * p.sw + sx];
                    c[0] = c0.y; c[1] = c0.z; c[2] = c0.w; c[3] = c1.x; c[4] = c1.y; c[5] = c1.z; c[6] = c1.w;
                }
#pragma unroll
                for (int j = 0; j < 7; ++j) cf[j] = c[j] * sf[j];
            }
        }
        if (active) {
            const int nx = dxhi - dxlo + 1;
            if (g == 1) {
                for (int oy = dylo; oy <= dyhi; ++oy) {
                    const float u2 = (float)oy * spx;
                    const float en_row = -u2 * u2;
                    const int row = (sy + oy) * p.sw + sx;
                    float u1 = (float)dxlo * spx;
                    // the mixed form's larger loop body runs faster without unrolling
                    constexpr int kRowUnroll = kMixed ? 1 : 3;
#pragma unroll kRowUnroll
                    for (int ox = dxlo; ox <= dxhi; ++ox) {
                        at(row + ox, u1, u2, fmaf(-u1, u1, en_row));
                        u1 += spx;
                    }
                }
            } else if (nx == side && dyhi - dylo + 1 == side) {
                // interior pixel: walk the full window through the table
                const int cbase = sy * p.sw + sx;
                for (int q = sub; q < nq; q += g) {
                    const float4 e = table[q];
                    at(cbase + __float_as_int(e.x), e.y, e.z, e.w);
                }
            } else {
                // window clipped by the image border
                const int nvalid = nx * (dyhi - dylo + 1);
                int ox = dxlo + sub % nx;
                int oy = dylo + sub / nx;
                for (int q = sub; q < nvalid; q += g) {
                    const int si = (sy + oy) * p.sw + sx + ox;
                    const float u1 = (float)ox * spx;
                    const float u2 = (float)oy * spx;
                    at(si, u1, u2, -fmaf(u1, u1, u2 * u2));
                    ox += g;
                    while (ox > dxhi) {
                        ox -= nx;
                        ++oy;
                    }
                }
            }
        }
        // count this warp out of the buffer; the last warp refills it
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            if (atomicAdd(&released[b], 1) == kTilePix / 32 - 1) {
                released[b] = 0;
                __threadfence_block();
                produce(s + L.nbuf);
            }
        }

        if (in.k == p.n_tau - 1) {
            // last frame of the window for this tile: reduce, solve, emit
            if (!kDense && g > 1) {
                for (int off = g >> 1; off >= 1; off >>= 1) {
#pragma unroll
                    for (int i = 0; i < NG; ++i) acc.G[i] += __shfl_xor_sync(0xffffffffu, acc.G[i], off);
#pragma unroll
                    for (int i = 0; i < NZ; ++i) acc.B[i] += __shfl_xor_sync(0xffffffffu, acc.B[i], off);
                }
            }
            if (active && sub == 0) {
                atomicAdd(&s_pairs, (unsigned long long)((dxhi - dxlo + 1) * (dyhi - dylo + 1) * p.n_tau));
                atomicAdd(&s_pix, 1ull);
                solve_and_emit<kMixed>(p, acc, cx, cy, &s_fp64);
            }
        }
    }

    if (timed_out) {
        // give copies already issued into the other buffers (and a late one into
        // the buffer that timed out) a bounded chance to land before the CTA exits
        for (int k = 1; k <= L.nbuf; ++k) {
            const int st = s_fail + (k % L.nbuf);
            mbar_wait_bounded(&full[st % L.nbuf], (uint32_t)((st / L.nbuf) & 1), 1u << 20);
        }
    }
    __syncthreads();   // every thread's counter updates are in before thread 0 reads them
    finish(p, s_pairs, s_pix, s_fp64, timed_out || (threadIdx.x == 0 && !pr->ok));
}

// Sparse-frame regression.  When few pixels are flagged they lie on thin
// feature edges, a handful per tile, and staging a whole tile window per work
// item would move far more data than it feeds.  Here each warp takes four
// consecutive entries of the frame's flagged list (the test kernel pads every
// tile's run to a multiple of four, so the four pixels share a tile and are
// usually adjacent along an edge), 8 lanes per pixel (16 or 32 when the item
// holds only two or one pixel, the tail of a tile's run).  For each frame of the
// temporal window the warp copies the bounding box of its pixels' windows
// from the ring into its own shared-memory buffer with 16-byte asynchronous
// copies (and hints the next frame's box into L2), then the lanes split each
// window's offsets and accumulate from shared memory; boxes too large for the
// buffer are read through L1 instead.  Warps fetch work independently; there
// is no block barrier inside the loop.
template <bool kMixed>
__global__ void __launch_bounds__(kTilePix, 2) wlr_sparse_kernel(const WlrParams p)
{
    if (p.sparse_max == 0 || *(volatile uint32_t*)&p.ctrl->flag_total > p.sparse_max)
        return;  // the tile-staged kernel's frame
    using S = SparseStage<kMixed>;
    extern __shared__ __align__(16) unsigned char sm[];
    const SparseLayout L = sparse_layout(p.r, kMixed);
    float4* table = reinterpret_cast<float4*>(sm);
    const bool can_stage = L.buf_bytes > 0 && p.sparse_stage;
    __shared__ unsigned long long s_pairs, s_pix, s_fp64;
    const int side = 2 * p.r + 1, nq = side * side;
    const float spx = p.s_coord_px;
    const size_t N = (size_t)p.W * p.H;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        const int ox = q % side - p.r, oy = q / side - p.r;
        const float u1 = (float)ox * spx, u2 = (float)oy * spx;
        table[q] = make_float4(__int_as_float(oy * S::pitch + ox), u1, u2, -fmaf(u1, u1, u2 * u2));
    }
    if (threadIdx.x == 0) {
        s_pairs = 0ull;
        s_pix = 0ull;
        s_fp64 = 0ull;
    }
    __syncthreads();
    const uint32_t n_list = *(volatile uint32_t*)&p.ctrl->list_len;
    const uint32_t tail_len = 2u * gridDim.x * (kTilePix / 32);
    const uint32_t tail0 = n_list > tail_len ? (n_list - tail_len) & ~3u : 0u;   // multiple of 4
    const float* sf = kMixed ? p.q_scale : p.s_feat;
    const float4* ringf = reinterpret_cast<const float4*>(p.ring);
    const uint4* ringm = reinterpret_cast<const uint4*>(p.ring);
    const int lane = threadIdx.x & 31;
    const int slot_t = p.t % p.T;
    unsigned char* wbuf = sm + L.buf_off + (threadIdx.x >> 5) * L.buf_bytes;
    uint4* bufm = reinterpret_cast<uint4*>(wbuf);
    float4* buf0 = reinterpret_cast<float4*>(wbuf);
    float4* buf1 = buf0 + S::pitch * S::rows;
    Acc acc;
    float cf[7];
    for (;;) {
        // Four-entry items until the last stretch of the list; that stretch
        // (half an item per warp of the grid) goes out one pixel at a time, so
        // the warps run out of work together instead of one item apart.
        uint32_t base = 0, single = 0;
        if (lane == 0) {
            base = atomicAdd(&p.ctrl->work_next, (uint32_t)kSparsePerWarp);
            if (base >= tail0) {
                base = tail0 + atomicAdd(&p.ctrl->tail_next, 1u);
                single = 1;
            }
        }
        base = __shfl_sync(0xffffffffu, base, 0);
        single = __shfl_sync(0xffffffffu, single, 0);
        if (base >= n_list) break;
        const uint32_t e4 = (single && (lane & 3)) ? kListPad : p.flag_list[base + (single ? 0 : (lane & 3))];
        // an item's m real entries come first (padding closes a tile's run);
        // 8 lanes per pixel for m = 3, 4, 16 for m = 2, 32 for m = 1
        const int m = __popc(__ballot_sync(0xffffffffu, e4 != kListPad) & 0xfu);
        if (m == 0) continue;   // a padding entry of the tail
        const int lg = m >= 3 ? 3 : 6 - m;
        const int g = 1 << lg;
        const int grp = lane >> lg, sub = lane & (g - 1);
        const uint32_t entry = __shfl_sync(0xffffffffu, e4, grp);
        const bool active = grp < m;
        const uint32_t pix = active ? entry : 0u;
        const int cx = (int)(pix % (uint32_t)p.W), cy = (int)(pix / (uint32_t)p.W);
#pragma unroll
        for (int i = 0; i < NG; ++i) acc.G[i] = 0.0f;
#pragma unroll
        for (int i = 0; i < NZ; ++i) acc.B[i] = 0.0f;
        const int dxlo = max(-p.r, -cx), dxhi = min(p.r, p.W - 1 - cx);
        const int dylo = max(-p.r, -cy), dyhi = min(p.r, p.H - 1 - cy);
        const int nx = dxhi - dxlo + 1, ny = dyhi - dylo + 1;
        // bounding box of the warp's windows (clipped to the image)
        const int bx0 = __reduce_min_sync(0xffffffffu, active ? cx + dxlo : 0x7fffffff);
        const int by0 = __reduce_min_sync(0xffffffffu, active ? cy + dylo : 0x7fffffff);
        const int bx1 = __reduce_max_sync(0xffffffffu, active ? cx + dxhi : -1);
        const int by1 = __reduce_max_sync(0xffffffffu, active ? cy + dyhi : -1);
        const int bw = bx1 - bx0 + 1, bh = by1 - by0 + 1;
        const bool staged = can_stage && bw > 0 && bw <= S::pitch && bh <= S::rows;   // warp-uniform
        if (active) {
            float c[7];
            if (kMixed) {
                float yc;
                unpack_mixed(__ldg(ringm + (size_t)slot_t * N + pix), yc, c);
            } else {
                const float4 c0 = __ldg(ringf + (size_t)(2 * slot_t) * N + pix);
                const float4 c1 = __ldg(ringf + (size_t)(2 * slot_t + 1) * N + pix);
                c[0] = c0.y; c[1] = c0.z; c[2] = c0.w; c[3] = c1.x; c[4] = c1.y; c[5] = c1.z; c[6] = c1.w;
            }
#pragma unroll
            for (int j = 0; j < 7; ++j) cf[j] = c[j] * sf[j];
        }
        const bool interior = nx == side && ny == side;
        for (int k = 0; k < p.n_tau; ++k) {
            const int slot = (p.t - k) % p.T;
            if (staged) {
                // box of this frame -> the warp's buffer (bw <= 32: one record per lane per row)
                __syncwarp();   // every lane is done with the previous frame's box
                const size_t row0 = (size_t)by0 * p.W + bx0 + lane;
                if (lane < bw) {
                    for (int i = 0; i < bh; ++i) {
                        const size_t g = row0 + (size_t)i * p.W;
                        if (kMixed) {
                            cp_async16(bufm + i * S::pitch + lane, ringm + (size_t)slot * N + g);
                        } else {
                            cp_async16(buf0 + i * S::pitch + lane, ringf + (size_t)(2 * slot) * N + g);
                            cp_async16(buf1 + i * S::pitch + lane, ringf + (size_t)(2 * slot + 1) * N + g);
                        }
                    }
                }
                if (k + 1 < p.n_tau) {
                    // hint the next frame's box into L2 while this one lands and is summed
                    const int nslot = (p.t - k - 1) % p.T;
                    const int lines = (bw * S::rec + 127) >> 7;
                    for (int j = lane; j < bh * lines; j += 32) {
                        const int i = j / lines, l = j - i * lines;
                        const size_t g = (size_t)(by0 + i) * p.W + bx0;
                        const char* row = kMixed
                            ? reinterpret_cast<const char*>(ringm + (size_t)nslot * N + g)
                            : reinterpret_cast<const char*>(ringf + (size_t)(2 * nslot) * N + g);
                        prefetch_l2(row + l * 128);
                        if (!kMixed) prefetch_l2(row + (size_t)N * 16 + l * 128);
                    }
                }
                cp_async_wait_all();
                __syncwarp();   // the box is visible to every lane of the warp
                if (active) {
                    const int cb = (cy - by0) * S::pitch + (cx - bx0);
                    auto at = [&](int si, float u1, float u2, float en0) {
                        if (kMixed)
                            accumulate(acc, bufm[si], u1, u2, en0, sf, cf);
                        else
                            accumulate(acc, buf0[si], buf1[si], u1, u2, en0, sf, cf);
                    };
                    if (interior) {
#pragma unroll 1
                        for (int q = sub; q < nq; q += g) {
                            const float4 e = table[q];
                            at(cb + __float_as_int(e.x), e.y, e.z, e.w);
                        }
                    } else {
                        const int nvalid = nx * ny;
                        int ox = dxlo + sub % nx;
                        int oy = dylo + sub / nx;
#pragma unroll 1
                        for (int q = sub; q < nvalid; q += g) {
                            const float u1 = (float)ox * spx, u2 = (float)oy * spx;
                            at(cb + oy * S::pitch + ox, u1, u2, -fmaf(u1, u1, u2 * u2));
                            ox += g;
                            while (ox > dxhi) {
                                ox -= nx;
                                ++oy;
                            }
                        }
                    }
                }
            } else if (active) {
                // box too large for the buffer: read the windows through L1
                const float4* __restrict__ R0 = ringf + (size_t)(2 * slot) * N + pix;
                const float4* __restrict__ R1 = ringf + (size_t)(2 * slot + 1) * N + pix;
                const uint4* __restrict__ RM = ringm + (size_t)slot * N + pix;
                auto at = [&](int d, float u1, float u2, float en0) {
                    if (kMixed)
                        accumulate(acc, __ldg(RM + d), u1, u2, en0, sf, cf);
                    else
                        accumulate(acc, __ldg(R0 + d), __ldg(R1 + d), u1, u2, en0, sf, cf);
                };
                // (rare: the window walked offset by offset, clipped or not)
                const int nvalid = nx * ny;
                int ox = dxlo + sub % nx;
                int oy = dylo + sub / nx;
#pragma unroll 1
                for (int q = sub; q < nvalid; q += g) {
                    const float u1 = (float)ox * spx, u2 = (float)oy * spx;
                    at(oy * p.W + ox, u1, u2, -fmaf(u1, u1, u2 * u2));
                    ox += g;
                    while (ox > dxhi) {
                        ox -= nx;
                        ++oy;
                    }
                }
            }
        }
#pragma unroll
        for (int off = g >> 1; off >= 1; off >>= 1) {
#pragma unroll
            for (int i = 0; i < NG; ++i) acc.G[i] += __shfl_xor_sync(0xffffffffu, acc.G[i], off);
#pragma unroll
            for (int i = 0; i < NZ; ++i) acc.B[i] += __shfl_xor_sync(0xffffffffu, acc.B[i], off);
        }
        if (active && sub == 0) {
            atomicAdd(&s_pairs, (unsigned long long)(nx * ny * p.n_tau));
            atomicAdd(&s_pix, 1ull);
            solve_and_emit<kMixed, true>(p, acc, cx, cy, &s_fp64);
        }
    }
    __syncthreads();
    finish(p, s_pairs, s_pix, s_fp64, false);
}

int wlr_sparse_smem(int r, bool mixed) { return sparse_layout(r, mixed).total; }

cudaError_t wlr_sparse_prepare(int r, bool mixed)
{
    const int bytes = wlr_sparse_smem(r, mixed);
    return mixed ? cudaFuncSetAttribute(wlr_sparse_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
                 : cudaFuncSetAttribute(wlr_sparse_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

int wlr_sparse_grid(int num_sms, bool mixed, int r)
{
    int per_sm = 0;
    const int bytes = wlr_sparse_smem(r, mixed);
    const cudaError_t e = mixed
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wlr_sparse_kernel<true>, kTilePix, bytes)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wlr_sparse_kernel<false>, kTilePix, bytes);
    if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm * num_sms;
}

cudaError_t launch_wlr_sparse(const WlrParams& p, bool mixed, int grid, cudaStream_t s)
{
    const int bytes = wlr_sparse_smem(p.r, mixed);
    if (mixed)
        wlr_sparse_kernel<true><<<grid, kTilePix, bytes, s>>>(p);
    else
        wlr_sparse_kernel<false><<<grid, kTilePix, bytes, s>>>(p);
    return cudaGetLastError();
}

SmemLayout host_layout(int r, bool mixed, int max_smem_per_sm)
{
    // three stages in flight when two CTAs still fit on an SM, else two
    SmemLayout L3 = smem_layout(r, 3, mixed);
    if (2 * (L3.total + 1024) <= max_smem_per_sm) return L3;
    return smem_layout(r, 2, mixed);
}

size_t wlr_smem_bytes(int r, bool mixed, int max_smem_per_sm, int* nbuf)
{
    const SmemLayout L = host_layout(r, mixed, max_smem_per_sm);
    *nbuf = L.nbuf;
    return (size_t)L.total;
}

template <bool kMixed>
static cudaError_t prepare_one(int smem_bytes)
{
    cudaError_t e = cudaFuncSetAttribute(wlr_kernel<true, kMixed>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(wlr_kernel<false, kMixed>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem_bytes);
}

cudaError_t wlr_prepare(int smem_bytes, bool mixed)
{
    return mixed ? prepare_one<true>(smem_bytes) : prepare_one<false>(smem_bytes);
}

int wlr_grid(int smem_bytes, int num_sms, bool mixed)
{
    int per_sm = 0;
    const cudaError_t e = mixed
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wlr_kernel<false, true>, kTilePix, smem_bytes)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wlr_kernel<false, false>, kTilePix, smem_bytes);
    if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm * num_sms;
}

cudaError_t launch_wlr(const CUtensorMap& tmap, const WlrParams& p, bool mixed, int grid,
                       int smem_bytes, cudaStream_t s)
{
    if (mixed) {
        if (p.dense)
            wlr_kernel<true, true><<<grid, kTilePix, smem_bytes, s>>>(tmap, p);
        else
            wlr_kernel<false, true><<<grid, kTilePix, smem_bytes, s>>>(tmap, p);
    } else {
        if (p.dense)
            wlr_kernel<true, false><<<grid, kTilePix, smem_bytes, s>>>(tmap, p);
        else
            wlr_kernel<false, false><<<grid, kTilePix, smem_bytes, s>>>(tmap, p);
    }
    return cudaGetLastError();
}

}  // namespace esim
