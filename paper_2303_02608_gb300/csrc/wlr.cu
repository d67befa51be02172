// Weighted local regression (Eqs. 3-5) with event emission (Eq. 1), in two
// passes per frame.
//
// Pass 1 accumulates.  For every regressed pixel the kernel-weighted sums of
// the normal equations over the spatio-temporal window (the Gram matrix of
// z = (1, u) and the right-hand side, 65 numbers) are summed in registers and
// stored as one 272-byte Gram record.  Two forms share this pass:
//   tile-staged   - a 32x8 pixel tile plus an r-pixel halo of one ring frame
//                   per stage, landed by one 4-D TMA load, up to three stages in
//                   flight per persistent CTA; every pixel of every tile (dense
//                   frames, wlr_dense_kernel) or the flagged pixels of the queued
//                   tiles (adaptive frames with many flags);
//   window boxes  - per-warp boxes covering the windows of four flagged pixels,
//                   landed by bulk asynchronous copies (adaptive frames with few
//                   flags).
// Adaptive frames launch wlr_adaptive_kernel, which picks the form on the
// device from the frame's flagged total.
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
#include "regress.cuh"

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
__device__ __forceinline__ void tile_body(const CUtensorMap& tmap, const WlrParams& p)
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


// Dense frames (frame 0, exhaustive mode): every tile, tile-staged.
template <bool kMixed>
__global__ void __launch_bounds__(kTilePix, 2)
    wlr_dense_kernel(const __grid_constant__ CUtensorMap tmap, const WlrParams p)
{
    tile_body<true, kMixed>(tmap, p);
}

// Adaptive frames: one launch that picks its form on the device from the
// frame's flagged total (known only after the test kernel ran): per-warp
// window boxes when at most sparse_max pixels are flagged, else the
// tile-staged kernel over the flagged-tile queue.
template <bool kMixed>
__global__ void __launch_bounds__(kTilePix, 2)
    wlr_adaptive_kernel(const __grid_constant__ CUtensorMap tmap, const WlrParams p)
{
    if (p.sparse_max > 0 && *(volatile uint32_t*)&p.ctrl->flag_total <= p.sparse_max)
        sparse_body<kSparsePerWarp, kMixed>(p, SingleSeq{&p});
    else
        tile_body<false, kMixed>(tmap, p);
}

// Solve and emit (Eqs. 4-5 and Eq. 1) for every Gram record of the frame:
// one thread per record (pixel index in dense frames, flagged-list position
// otherwise; list padding is skipped).  FP32 form: equilibrated FP32
// Cholesky.  Mixed form: FP32 Cholesky plus one refinement step; systems
// whose condition estimate exceeds 1e6 are set aside and, after each pass of
// the block, re-accumulated by one warp each with compensated FP32 sums and
// solved by FP64 Cholesky (refine_fp64).  Block 0 records the event total
// before this frame (ev_base) for the ordered writer.
template <bool kMixed>
__global__ void __launch_bounds__(kSolveThreads, 3) wlr_solve_kernel(const WlrParams p)
{
    if (threadIdx.x == 0 && blockIdx.x == 0)
        p.ctrl->ev_base = p.ctrl->ev_total;   // records not yet drained come first
    const uint32_t n = p.dense ? (uint32_t)((size_t)p.W * p.H) : *(volatile uint32_t*)&p.ctrl->list_len;
    const unsigned long long fp64 = solve_records<kMixed>(p, SingleSeq{&p}, n);
    finish(p, 0ull, 0ull, fp64, false, false);
}

int wlr_sparse_smem(int r, bool /*mixed*/) { return box_layout(r).total; }

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
static cudaError_t prepare_one(int smem_dense, int smem_adaptive)
{
    cudaError_t e = cudaFuncSetAttribute(wlr_dense_kernel<kMixed>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_dense);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(wlr_adaptive_kernel<kMixed>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem_adaptive);
}

cudaError_t wlr_prepare(int smem_dense, int smem_adaptive, bool mixed)
{
    return mixed ? prepare_one<true>(smem_dense, smem_adaptive) : prepare_one<false>(smem_dense, smem_adaptive);
}

int wlr_grid(int smem_bytes, int num_sms, bool mixed, bool adaptive)
{
    int per_sm = 0;
    cudaError_t e;
    if (adaptive)
        e = mixed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wlr_adaptive_kernel<true>, kTilePix, smem_bytes)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wlr_adaptive_kernel<false>, kTilePix, smem_bytes);
    else
        e = mixed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wlr_dense_kernel<true>, kTilePix, smem_bytes)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wlr_dense_kernel<false>, kTilePix, smem_bytes);
    if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm * num_sms;
}

cudaError_t launch_wlr(const CUtensorMap& tmap, const WlrParams& p, bool mixed, int grid, int smem_bytes,
                       cudaStream_t s)
{
    if (mixed) {
        if (p.dense)
            wlr_dense_kernel<true><<<grid, kTilePix, smem_bytes, s>>>(tmap, p);
        else
            wlr_adaptive_kernel<true><<<grid, kTilePix, smem_bytes, s>>>(tmap, p);
    } else {
        if (p.dense)
            wlr_dense_kernel<false><<<grid, kTilePix, smem_bytes, s>>>(tmap, p);
        else
            wlr_adaptive_kernel<false><<<grid, kTilePix, smem_bytes, s>>>(tmap, p);
    }
    return cudaGetLastError();
}

}  // namespace esim
