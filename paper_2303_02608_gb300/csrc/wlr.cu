// Weighted local regression (Eqs. 3-5) with event emission (Eq. 1), in two
// passes per frame.
//
// Pass 1 accumulates.  For every regressed pixel the kernel-weighted sums of
// the normal equations over the spatio-temporal window (the Gram matrix of
// z = (1, u) and the right-hand side, 65 numbers) are summed in registers and
// stored as one 272-byte Gram record.  Two kernels share this pass and pick
// frames by flag density:
//   wlr_kernel         - tile-staged: a 32x8 pixel tile plus an r-pixel halo of
//                        one ring frame per stage, landed by one 4-D TMA load,
//                        up to three stages in flight per persistent CTA; every
//                        pixel of a tile (dense frames) or the tile's flagged
//                        pixels (adaptive frames with many flags);
//   wlr_sparse_kernel  - per-warp window boxes of four flagged pixels, landed by
//                        bulk asynchronous copies (adaptive frames with few flags).
// Each regressed pixel is owned by g lanes (g = 1 when a tile is densely
// flagged, up to 32); the lanes split the window's offsets, accumulate in
// packed FP32 pairs, and are reduced with warp shuffles.  Regressors are the
// feature differences scaled by k / (h b_j), k = sqrt(log2(e) / 2), so the
// product Gaussian of Eq. 5 is one exp2:  w = 2^(-|u|^2).
//
// Pass 2 (wlr_solve_kernel) solves each record: the ridge lambda * W * |beta|^2
// added on the scaled diagonal as lambda * W * s_j^2, Jacobi equilibration and
// an FP32 Cholesky (the mixed form adds one refinement step and sends systems
// with condition estimate above 1e6 to a compensated re-accumulation and an
// FP64 solve); the slopes are mapped back to natural units.  It then applies
// Eq. 1 at a fixed frame time: Delta L = alpha - L_last,
// n = floor(|Delta L| / C); if n >= 1 the pixel emits n events of polarity
// sign(Delta L) (recorded in the per-pixel count map for the ordered event
// writer), L_last moves by p n C and the model (beta, x^c) is replaced by the
// new fit (Fig. 1: the model is kept until a new event).  Frame 0 only
// initialises L_last = alpha and the model.  Its last CTA scans the per-chunk
// event counts for the writer.
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
    // (u_dx, u_dy, -(u_dx^2 + u_dy^2), smem offset) per offset
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        const int ox = q % side - p.r, oy = q / side - p.r;
        const float u1 = (float)ox * spx, u2 = (float)oy * spx;
        table[q] = make_float4(u1, u2, -fmaf(u1, u1, u2 * u2), __int_as_float(oy * p.sw + ox));
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
    AccP acc;
    const float* sf = kMixed ? p.q_scale : p.s_feat;   // regressor scale of a stored value
    PairConst kc;
    {
        float cf0[7];
#pragma unroll
        for (int j = 0; j < 7; ++j) cf0[j] = 0.0f;
        kc = pair_const(sf, cf0);
    }
    int g = 1, lg = 0, sub = 0, npix = 0, cx = 0, cy = 0, sx = 0, sy = 0;
    uint32_t entry = 0;
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
    // the first stages are issued before any warp waits on them: a warp whose
    // other lanes spun on stage 0 while its lane 0 was still issuing it could
    // starve that lane until the bounded wait gave up
    __syncthreads();

    int s_fail = 0;
    for (int s = 0;; ++s) {
        const int b = s % L.nbuf;
        __syncwarp();   // lane 0 may still be issuing a stage: no lane polls while it does
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
                accp(acc, PM[si], make_float2(u1, u2), en0, kc);
            else
                accp(acc, P0[si], P1[si], make_float2(u1, u2), en0, kc);
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
            if (!kDense && active) entry = p.tile_base[in.tile] + (uint32_t)(in.first + item);
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
            if (kDense) entry = (uint32_t)cy * (uint32_t)p.W + (uint32_t)cx;
            accp_zero(acc);
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
                float cf[7];
#pragma unroll
                for (int j = 0; j < 7; ++j) cf[j] = c[j] * sf[j];
                kc = pair_const(sf, cf);
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
                    constexpr int kRowUnroll = 1;
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
                    at(cbase + __float_as_int(e.w), e.x, e.y, e.z);
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
            // last frame of the window for this tile: reduce and store the sums
            if (!kDense && g > 1) accp_reduce(acc, g);
            if (active) {
                accp_store(acc, p.gram + (size_t)entry * kGramStride, sub, g);
                if (sub == 0) {
                    atomicAdd(&s_pairs, (unsigned long long)((dxhi - dxlo + 1) * (dyhi - dylo + 1) * p.n_tau));
                    atomicAdd(&s_pix, 1ull);
                }
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
    finish(p, s_pairs, s_pix, 0ull, timed_out || (threadIdx.x == 0 && !pr->ok), false);
}

// Sparse-frame regression (accumulation; wlr_solve_kernel solves and emits).
// When few pixels are flagged they lie on thin feature edges, a handful per
// tile, and staging a whole tile window per work item would move far more
// data than it feeds.  Here each warp takes four consecutive entries of the
// frame's flagged list (the test kernel pads every tile's run to a multiple
// of four, so the four pixels share a tile and are usually adjacent along an
// edge), 8 lanes per pixel (16 or 32 when the item holds only two or one
// pixel, the tail of a tile's run).  For each frame of the temporal window the
// bounding box of the four windows (clipped to the image) is copied from the
// ring into the warp's shared memory by bulk asynchronous copies (the TMA
// engine, one row per lane, completing on the warp's mbarrier).  Boxes of up
// to 20 x 20 records are double-buffered: frame k+1's copy is issued before
// frame k is summed.  Larger boxes take the whole buffer one frame at a time;
// boxes too large for it are read through L1.  The lanes split each window's
// offsets and accumulate the 65 sums in packed FP32 pairs; the g lanes of a
// pixel are then reduced by shuffles and store one Gram record at the pixel's
// position in the flagged list.  Warps fetch work independently; there is no
// block barrier inside the loop, and every mbarrier wait is bounded.
template <bool kMixed>
__global__ void __launch_bounds__(kTilePix, 2) wlr_sparse_kernel(const WlrParams p)
{
    if (p.sparse_max == 0 || *(volatile uint32_t*)&p.ctrl->flag_total > p.sparse_max)
        return;  // the tile-staged kernel's frame
    extern __shared__ __align__(128) unsigned char sm[];
    const BoxLayout L = box_layout(p.r);
    __shared__ unsigned long long s_pairs, s_pix;
    const int side = 2 * p.r + 1, nq = side * side;
    const float spx = p.s_coord_px;
    const size_t N = (size_t)p.W * p.H;
    // window tables (u_dx, u_dy, -(u_dx^2 + u_dy^2), box offset) for the two row pitches
    float4* tab_s = reinterpret_cast<float4*>(sm + L.tab_small);
    float4* tab_l = reinterpret_cast<float4*>(sm + L.tab_large);
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        const int ox = q % side - p.r, oy = q / side - p.r;
        const float u1 = (float)ox * spx, u2 = (float)oy * spx;
        const float en0 = -fmaf(u1, u1, u2 * u2);
        tab_s[q] = make_float4(u1, u2, en0, __int_as_float(oy * kPitchSmall + ox));
        tab_l[q] = make_float4(u1, u2, en0, __int_as_float(oy * kPitchLarge + ox));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L.bar_off) + 2 * warp;
    unsigned char* wbuf = sm + L.buf_off + warp * kBoxBytes;
    if (threadIdx.x == 0) {
        s_pairs = 0ull;
        s_pix = 0ull;
    }
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const uint32_t n_list = *(volatile uint32_t*)&p.ctrl->list_len;
    const uint32_t tail_len = 2u * gridDim.x * (kTilePix / 32);
    const uint32_t tail0 = n_list > tail_len ? (n_list - tail_len) & ~3u : 0u;   // multiple of 4
    const float* sf = kMixed ? p.q_scale : p.s_feat;
    const float4* ringf = reinterpret_cast<const float4*>(p.ring);
    const uint4* ringm = reinterpret_cast<const uint4*>(p.ring);
    const int slot_t = p.t % p.T;
    const uint32_t poll = p.poll_limit;
    uint32_t phase = 0u;        // bit b: parity of bar[b]'s next phase completion
    bool timed_out = false;
    bool first_item = true;
    AccP acc;
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
        // The m pixels go together when the bounding box of their windows fits
        // the buffer; otherwise (pixels spread across their tile) one at a
        // time with all 32 lanes, each pass staging its own window.
        auto box_mode = [&](int bw, int bh) {   // 2: double-buffered halves, 1: whole buffer, 0: none
            if (!p.sparse_stage) return 0;
            if (kMixed && bw <= kPitchSmall && bh <= kRowsSmall) return 2;
            if (kMixed && bw <= kPitchLarge && bh <= kRowsLarge) return 1;
            if (!kMixed && bw <= kPitchSmall && bh <= kRowsSmall) return 1;
            return 0;
        };
        int passes = 1;
        bool split = false;
        if (m > 1 && p.sparse_stage && side <= kPitchSmall) {
            const int lg0 = m >= 3 ? 3 : 6 - m;
            const int grp0 = lane >> lg0;
            const bool act0 = grp0 < m;
            const uint32_t px0 = __shfl_sync(0xffffffffu, e4, grp0);
            const int x0 = (int)(px0 % (uint32_t)p.W), y0 = (int)(px0 / (uint32_t)p.W);
            const int ux0 = __reduce_min_sync(0xffffffffu, act0 ? max(x0 - p.r, 0) : 0x7fffffff);
            const int uy0 = __reduce_min_sync(0xffffffffu, act0 ? max(y0 - p.r, 0) : 0x7fffffff);
            const int ux1 = __reduce_max_sync(0xffffffffu, act0 ? min(x0 + p.r, p.W - 1) : -1);
            const int uy1 = __reduce_max_sync(0xffffffffu, act0 ? min(y0 + p.r, p.H - 1) : -1);
            if (box_mode(ux1 - ux0 + 1, uy1 - uy0 + 1) == 0) {
                split = true;
                passes = m;
            }
        }
        for (int part = 0; part < passes; ++part) {
        const int lg = split ? 5 : (m >= 3 ? 3 : 6 - m);
        const int g = 1 << lg;
        const int grp = split ? 0 : lane >> lg, sub = lane & (g - 1);
        const uint32_t pix_e = __shfl_sync(0xffffffffu, e4, split ? part : grp);
        const bool active = grp < m;
        const uint32_t pix = active ? pix_e : 0u;
        const uint32_t entry = base + (uint32_t)(split ? part : grp);
        const int cx = (int)(pix % (uint32_t)p.W), cy = (int)(pix / (uint32_t)p.W);
        const int dxlo = max(-p.r, -cx), dxhi = min(p.r, p.W - 1 - cx);
        const int dylo = max(-p.r, -cy), dyhi = min(p.r, p.H - 1 - cy);
        const int nx = dxhi - dxlo + 1, ny = dyhi - dylo + 1;
        // bounding box of the pass's windows (clipped to the image)
        const int bx0 = __reduce_min_sync(0xffffffffu, active ? cx + dxlo : 0x7fffffff);
        const int by0 = __reduce_min_sync(0xffffffffu, active ? cy + dylo : 0x7fffffff);
        const int bx1 = __reduce_max_sync(0xffffffffu, active ? cx + dxhi : -1);
        const int by1 = __reduce_max_sync(0xffffffffu, active ? cy + dyhi : -1);
        const int bw = bx1 - bx0 + 1, bh = by1 - by0 + 1;
        const int mode = box_mode(bw, bh);   // warp-uniform; 0: windows read through L1
        const int P = (mode == 2 || !kMixed) ? kPitchSmall : kPitchLarge;
        const float4* tab = P == kPitchSmall ? tab_s : tab_l;
        PairConst kc;
        {
            float c[7] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            if (active) {
                if (kMixed) {
                    float yc;
                    unpack_mixed(__ldg(ringm + (size_t)slot_t * N + pix), yc, c);
                } else {
                    const float4 c0 = __ldg(ringf + (size_t)(2 * slot_t) * N + pix);
                    const float4 c1 = __ldg(ringf + (size_t)(2 * slot_t + 1) * N + pix);
                    c[0] = c0.y; c[1] = c0.z; c[2] = c0.w; c[3] = c1.x; c[4] = c1.y; c[5] = c1.z; c[6] = c1.w;
                }
            }
            float cf[7];
#pragma unroll
            for (int j = 0; j < 7; ++j) cf[j] = c[j] * sf[j];
            kc = pair_const(sf, cf);
        }
        accp_zero(acc);
        // Copy frame k of the box into half b (mode 2) or the whole buffer
        // (mode 1).  Every lane is past its reads of that region first.
        auto issue = [&](int b, int k) {
            __syncwarp();
            fence_proxy_async_smem();
            if (p.withhold_copy && first_item && k == 0) return;   // test: this phase never completes
            const int slot = (p.t - k) % p.T;
            const uint32_t rowb = (uint32_t)bw * 16u;
            if (lane == 0) mbar_arrive_expect_tx(&bar[b], (uint32_t)bh * rowb * (kMixed ? 1u : 2u));
            __syncwarp();
            if (lane < bh) {
                const size_t gi = (size_t)(by0 + lane) * p.W + bx0;
                unsigned char* dst = wbuf + (mode == 2 ? b * (kBoxBytes / 2) : 0) + lane * P * 16;
                if (kMixed) {
                    bulk_load(dst, ringm + (size_t)slot * N + gi, rowb, &bar[b]);
                } else {
                    bulk_load(dst, ringf + (size_t)(2 * slot) * N + gi, rowb, &bar[b]);
                    bulk_load(dst + kBoxBytes / 2, ringf + (size_t)(2 * slot + 1) * N + gi, rowb, &bar[b]);
                }
            }
        };
        const bool interior = nx == side && ny == side;
        if (mode) issue(0, 0);
        for (int k = 0; k < p.n_tau; ++k) {
            if (mode) {
                const int b = mode == 2 ? (k & 1) : 0;
                const bool ahead = mode == 2 && k + 1 < p.n_tau;
                if (ahead) issue(b ^ 1, k + 1);
                const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar[b], (phase >> b) & 1u, poll));
                phase ^= 1u << b;
                if (!ok) {
                    // give the copies still in flight a bounded chance to land, then stop
                    mbar_wait_bounded(&bar[b], ((phase >> b) & 1u) ^ 1u, poll);
                    if (ahead) mbar_wait_bounded(&bar[b ^ 1], (phase >> (b ^ 1)) & 1u, poll);
                    timed_out = true;
                    break;
                }
                const unsigned char* buf = wbuf + (mode == 2 ? b * (kBoxBytes / 2) : 0);
                auto at = [&](int si, float u1, float u2, float en0) {
                    if (kMixed)
                        accp(acc, reinterpret_cast<const uint4*>(buf)[si], make_float2(u1, u2), en0, kc);
                    else
                        accp(acc, reinterpret_cast<const float4*>(buf)[si],
                             reinterpret_cast<const float4*>(buf + kBoxBytes / 2)[si], make_float2(u1, u2), en0, kc);
                };
                if (active) {
                    const int cb = (cy - by0) * P + (cx - bx0);
                    if (interior) {
#pragma unroll 1
                        for (int q = sub; q < nq; q += g) {
                            const float4 e = tab[q];
                            at(cb + __float_as_int(e.w), e.x, e.y, e.z);
                        }
                    } else {
                        const int nvalid = nx * ny;
                        int ox = dxlo + sub % nx;
                        int oy = dylo + sub / nx;
#pragma unroll 1
                        for (int q = sub; q < nvalid; q += g) {
                            const float u1 = (float)ox * spx, u2 = (float)oy * spx;
                            at(cb + oy * P + ox, u1, u2, -fmaf(u1, u1, u2 * u2));
                            ox += g;
                            while (ox > dxhi) {
                                ox -= nx;
                                ++oy;
                            }
                        }
                    }
                }
                if (mode == 1 && k + 1 < p.n_tau) issue(0, k + 1);
            } else if (active) {
                // box too large for the buffer: read the windows through L1
                const int slot = (p.t - k) % p.T;
                const float4* __restrict__ R0 = ringf + (size_t)(2 * slot) * N + pix;
                const float4* __restrict__ R1 = ringf + (size_t)(2 * slot + 1) * N + pix;
                const uint4* __restrict__ RM = ringm + (size_t)slot * N + pix;
                const int nvalid = nx * ny;
                int ox = dxlo + sub % nx;
                int oy = dylo + sub / nx;
#pragma unroll 1
                for (int q = sub; q < nvalid; q += g) {
                    const float u1 = (float)ox * spx, u2 = (float)oy * spx;
                    const int d = oy * p.W + ox;
                    if (kMixed)
                        accp(acc, __ldg(RM + d), make_float2(u1, u2), -fmaf(u1, u1, u2 * u2), kc);
                    else
                        accp(acc, __ldg(R0 + d), __ldg(R1 + d), make_float2(u1, u2), -fmaf(u1, u1, u2 * u2), kc);
                    ox += g;
                    while (ox > dxhi) {
                        ox -= nx;
                        ++oy;
                    }
                }
            }
        }
        first_item = false;
        if (timed_out) break;
        accp_reduce(acc, g);
        if (active) {
            accp_store(acc, p.gram + (size_t)entry * kGramStride, sub, g);
            if (sub == 0) {
                atomicAdd(&s_pairs, (unsigned long long)(nx * ny * p.n_tau));
                atomicAdd(&s_pix, 1ull);
            }
        }
        }   // passes
        if (timed_out) break;
    }
    __syncthreads();
    finish(p, s_pairs, s_pix, 0ull, timed_out, false);
}

constexpr int kSolveThreads = 128;

// Error-free sum of two floats (Knuth's TwoSum): s + err == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err)
{
    s = __fadd_rn(a, b);
    const float bb = __fadd_rn(s, -a);
    err = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
}

// Ill-conditioned system of pixel pix, one warp: the 65 sums are accumulated
// again from the ring with compensated FP32 arithmetic (each product term
// rounded once, each running sum carried as an unevaluated pair hi + lo by
// TwoSum; feature differences taken before scaling, which is exact for the
// stored BF16 values), lane l owning sums l, l + 32 and l + 64 (sums 0-54 are
// the Gram triangle in tri() order, 55-64 the right-hand side).  Lane 0 then
// adds the ridge and solves the equilibrated system by Cholesky in FP64 and
// emits.  sys: 66 doubles of this warp's shared memory.
template <bool kMixed>
__device__ __noinline__ void refine_fp64(const WlrParams& p, uint32_t pix, const float (&s2)[NZ], double* sys)
{
    const int lane = threadIdx.x & 31;
    const size_t N = (size_t)p.W * p.H;
    const int cx = (int)(pix % (uint32_t)p.W), cy = (int)(pix / (uint32_t)p.W);
    const float* sf = kMixed ? p.q_scale : p.s_feat;
    const float4* ringf = reinterpret_cast<const float4*>(p.ring);
    const uint4* ringm = reinterpret_cast<const uint4*>(p.ring);
    auto load = [&](int slot, size_t i, float& y, float (&f)[7]) {
        if (kMixed) {
            unpack_mixed(__ldg(ringm + (size_t)slot * N + i), y, f);
        } else {
            const float4 a = __ldg(ringf + (size_t)(2 * slot) * N + i);
            const float4 b = __ldg(ringf + (size_t)(2 * slot + 1) * N + i);
            y = a.x; f[0] = a.y; f[1] = a.z; f[2] = a.w; f[3] = b.x; f[4] = b.y; f[5] = b.z; f[6] = b.w;
        }
    };
    float yc, c[7];
    load(p.t % p.T, pix, yc, c);
    // the (row, column) of each owned sum; column 10 is the log brightness
    int oi[3], oj[3];
    float hi[3] = {0.0f, 0.0f, 0.0f}, lo[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        const int idx = lane + 32 * o;
        int i = 0, j = 0;
        if (idx < NG) {
            while (tri(i + 1, 0) <= idx) ++i;
            j = idx - tri(i, 0);
        } else if (idx < NG + NZ) {
            i = 10;
            j = idx - NG;
        } else {
            i = -1;
        }
        oi[o] = i;
        oj[o] = j;
    }
    const int dxlo = max(-p.r, -cx), dxhi = min(p.r, p.W - 1 - cx);
    const int dylo = max(-p.r, -cy), dyhi = min(p.r, p.H - 1 - cy);
    for (int k = 0; k < p.n_tau; ++k) {
        const int slot = (p.t - k) % p.T;
        for (int oy = dylo; oy <= dyhi; ++oy) {
            for (int ox = dxlo; ox <= dxhi; ++ox) {
                float y, f[7];
                load(slot, (size_t)(cy + oy) * p.W + cx + ox, y, f);
                float z[NZ + 1];
                z[0] = 1.0f;
                z[1] = __fmul_rn((float)ox, p.s_coord_px);
                z[2] = __fmul_rn((float)oy, p.s_coord_px);
#pragma unroll
                for (int j = 0; j < 7; ++j) z[3 + j] = __fmul_rn(__fadd_rn(f[j], -c[j]), sf[j]);
                z[NZ] = y;
                float en = 0.0f;
#pragma unroll
                for (int j = 1; j < NZ; ++j) en = fmaf(-z[j], z[j], en);
                const float w = exp2f(en);
#pragma unroll
                for (int o = 0; o < 3; ++o) {
                    if (oi[o] < 0) continue;
                    const float t = __fmul_rn(__fmul_rn(w, z[oi[o]]), z[oj[o]]);
                    float sum, err;
                    two_sum(hi[o], t, sum, err);
                    hi[o] = sum;
                    lo[o] = __fadd_rn(lo[o], err);
                }
            }
        }
    }
#pragma unroll
    for (int o = 0; o < 3; ++o)
        if (oi[o] >= 0) sys[lane + 32 * o] = (double)hi[o] + (double)lo[o];
    __syncwarp();
    if (lane == 0) {
        double A[NG], b[NZ], dsc[NZ];
        for (int i = 0; i < NG; ++i) A[i] = sys[i];
        for (int i = 0; i < NZ; ++i) b[i] = sys[NG + i];
        const double Wsum = A[0];
        for (int j = 1; j < NZ; ++j) A[tri(j, j)] += (double)p.ridge * Wsum * (double)s2[j];
        for (int i = 0; i < NZ; ++i) dsc[i] = 1.0 / sqrt(A[tri(i, i)]);
        for (int i = 0; i < NZ; ++i) {
            for (int j = 0; j <= i; ++j) A[tri(i, j)] *= dsc[i] * dsc[j];
            b[i] *= dsc[i];
        }
        double dinv[NZ], zz[NZ], x[NZ];
        for (int j = 0; j < NZ; ++j) {
            double sj = A[tri(j, j)];
            for (int k = 0; k < j; ++k) sj -= A[tri(j, k)] * A[tri(j, k)];
            sj = sj > 1e-300 ? sj : 1e-300;
            const double l = sqrt(sj);
            A[tri(j, j)] = l;
            dinv[j] = 1.0 / l;
            for (int i = j + 1; i < NZ; ++i) {
                double v = A[tri(i, j)];
                for (int k = 0; k < j; ++k) v -= A[tri(i, k)] * A[tri(j, k)];
                A[tri(i, j)] = v * dinv[j];
            }
        }
        for (int i = 0; i < NZ; ++i) {
            double v = b[i];
            for (int k = 0; k < i; ++k) v -= A[tri(i, k)] * zz[k];
            zz[i] = v * dinv[i];
        }
        for (int i = NZ - 1; i >= 0; --i) {
            double v = zz[i];
            for (int k = i + 1; k < NZ; ++k) v -= A[tri(k, i)] * x[k];
            x[i] = v * dinv[i];
        }
        float theta[NZ];
        for (int i = 0; i < NZ; ++i) theta[i] = (float)(x[i] * dsc[i]);
        emit<kMixed>(p, cx, cy, theta);
    }
    __syncwarp();
}

// Solve and emit (Eqs. 4-5 and Eq. 1) for every Gram record of the frame:
// one thread per record (pixel index in dense frames, flagged-list position
// otherwise; list padding is skipped).  FP32 form: equilibrated FP32
// Cholesky.  Mixed form: FP32 Cholesky plus one refinement step; systems
// whose condition estimate exceeds 1e6 are set aside and, after each pass of
// the block, re-accumulated by one warp each with compensated FP32 sums and
// solved by FP64 Cholesky (refine_fp64).  The last CTA scans the per-chunk
// event counts for the ordered writer.
template <bool kMixed>
__global__ void __launch_bounds__(kSolveThreads, 3) wlr_solve_kernel(const WlrParams p)
{
    __shared__ uint32_t s_ill[kSolveThreads];
    __shared__ int s_nill;
    __shared__ unsigned long long s_fp64;
    __shared__ double s_sys[kSolveThreads / 32][66];
    if (threadIdx.x == 0) {
        s_nill = 0;
        s_fp64 = 0ull;
    }
    __syncthreads();
    const uint32_t n = p.dense ? (uint32_t)((size_t)p.W * p.H) : *(volatile uint32_t*)&p.ctrl->list_len;
    float s2[NZ];
    s2[0] = 0.0f;
    s2[1] = p.s_coord * p.s_coord;
    s2[2] = s2[1];
#pragma unroll
    for (int j = 0; j < 7; ++j) s2[3 + j] = p.s_feat[j] * p.s_feat[j];
    const uint32_t stride = gridDim.x * kSolveThreads;
    for (uint32_t b0 = blockIdx.x * kSolveThreads; b0 < n; b0 += stride) {   // same trip count in the block
        const uint32_t e = b0 + threadIdx.x;
        uint32_t pix = kListPad;
        if (e < n) pix = p.dense ? e : p.flag_list[e];
        bool ill = false;
        if (pix != kListPad) {
            const float* rec = p.gram + (size_t)e * kGramStride;
            float theta[NZ];
            if (kMixed) {
                ill = !solve_refined_rec(rec, s2, p.ridge, theta);
            } else {
                Acc acc;
                gram_load(rec, acc);
                solve(acc, s2, p.ridge, theta);
            }
            if (!ill) emit<kMixed>(p, (int)(pix % (uint32_t)p.W), (int)(pix / (uint32_t)p.W), theta);
            else s_ill[atomicAdd(&s_nill, 1)] = pix;
        }
        if (kMixed && __syncthreads_or(ill)) {
            const int nill = s_nill;
            for (int i = (int)(threadIdx.x >> 5); i < nill; i += kSolveThreads / 32)
                refine_fp64<kMixed>(p, s_ill[i], s2, s_sys[threadIdx.x >> 5]);
            __syncthreads();
            if (threadIdx.x == 0) {
                s_fp64 += (unsigned long long)nill;
                s_nill = 0;
            }
            __syncthreads();
        }
    }
    __syncthreads();
    finish(p, 0ull, 0ull, s_fp64, false, true);
}

int wlr_sparse_smem(int r, bool /*mixed*/) { return box_layout(r).total; }

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

int wlr_solve_grid(int num_sms) { return 3 * num_sms; }   // one wave at 3 CTAs per SM

cudaError_t launch_wlr_solve(const WlrParams& p, bool mixed, int grid, cudaStream_t s)
{
    if (mixed)
        wlr_solve_kernel<true><<<grid, kSolveThreads, 0, s>>>(p);
    else
        wlr_solve_kernel<false><<<grid, kSolveThreads, 0, s>>>(p);
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
