// Batching form: many independent sequences of uneven resolution advanced one
// frame each per step, as one CUDA graph per step:
//   1. copy of the step table (per-sequence frame pointers and frame index),
//   2. clear of the per-step counters and the per-chunk event counts,
//   3. one ingest/test launch over the tiles of every sequence (tile shape
//      16x16, 32x8 or 64x4 pixels); flagged pixels of all sequences are
//      compacted into one queue of (sequence, pixel) entries (sequence in the
//      top 8 bits), each tile's run padded to four entries,
//   4. one persistent accumulation launch over that queue (the single-sequence
//      window-box form: per-warp boxes of an item's windows landed by bulk
//      asynchronous copies, packed FP32 sums, one Gram record per entry; the
//      item size, hence lanes per pixel, is a template choice),
//   5. one solve launch over the records (solve, Eq. 1 emission into each
//      sequence's maps, scan of the per-chunk event counts),
//   6. one event-writer launch over the chunks of every sequence.
// The tile shape and the lanes per pixel are picked jointly by an autotuner
// that times the nine pairs on the first adaptive steps.  Each sequence keeps
// its own ring, model state and maps, exactly as a single-sequence context
// does; the per-pixel arithmetic is shared with it.
#include <errno.h>
#include <stdio.h>
#include <sys/stat.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "block_scan.cuh"
#include "ingest_pixel.cuh"
#include "sparse_stage.cuh"
#include "internal.h"
#include "wlr_math.cuh"
#include "regress.cuh"

namespace esim {
namespace {

constexpr int kMaxSeq = 255;
constexpr uint32_t kPixBits = 24;
constexpr uint32_t kPixMask = (1u << kPixBits) - 1u;

// Per-sequence, per-step description (device table, rewritten every step).
struct SeqStep {
    IngestParams ip;       // frame inputs, ring slot, test on/off
    WlrParams wp;          // frame index, window, maps; chunk_cnt points at the sequence's chunks
    int active;            // the sequence advances this step
    int tile_base;         // first global tile of the sequence
    int chunk_base;        // first global event chunk of the sequence
    uint32_t frame;        // frame index written into its events
};

struct BatchGlobal {
    const SeqStep* steps;
    const uint16_t* tile_seq;    // global tile -> sequence
    const uint16_t* chunk_seq;   // global chunk -> sequence
    uint32_t* flag_list;         // (seq << 24) | pixel
    uint32_t* chunk_cnt;         // [total chunks]
    unsigned long long* chunk_off;
    esim_ad_batch_event* events;
    unsigned long long capacity;
    int total_tiles, total_chunks, r;
    int tx;                      // tile width in pixels (tile height 256 / tx)
    float s_px;
    Ctrl* ctrl;
};

// Tile shapes the autotuner chooses from: width in pixels (height 256 / width).
constexpr int kTileShapes = 3;
constexpr int kTileWidths[kTileShapes] = {16, 32, 64};

// Sequences of a batch: list entries are (sequence << 24) | pixel.
struct BatchSeq {
    const SeqStep* steps;
    __device__ __forceinline__ SeqView view(uint32_t e) const
    {
        const WlrParams& sp = steps[e >> kPixBits].wp;
        return {sp.W, sp.H, sp.t, sp.T, sp.n_tau, sp.ring};
    }
    __device__ __forceinline__ uint32_t pixel(uint32_t e) const { return e & kPixMask; }
    __device__ __forceinline__ const WlrParams& params(uint32_t e) const { return steps[e >> kPixBits].wp; }
};

__global__ void __launch_bounds__(kTilePix) batch_ingest_kernel(BatchGlobal g)
{
    const int gt = blockIdx.x;
    const int seq = g.tile_seq[gt];
    const SeqStep& st = g.steps[seq];
    if (!st.active) return;
    const IngestParams& p = st.ip;
    const int tile = gt - st.tile_base;
    const int ty = kTilePix / g.tx;
    const int x = (tile % p.tiles_x) * g.tx + (int)threadIdx.x % g.tx;
    const int y = (tile / p.tiles_x) * ty + (int)threadIdx.x / g.tx;
    const int flag = ingest_pixel(p, x, y);
    // compact this tile's regressed pixels into the global queue, in raster
    // order within the tile (= thread order)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __shared__ int warp_cnt[kTilePix / 32];
    __shared__ uint32_t s_base;
    const unsigned ballot = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) warp_cnt[wid] = __popc(ballot);
    __syncthreads();
    int base = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kTilePix / 32; ++w) {
        const int c = warp_cnt[w];
        base += (w < wid) ? c : 0;
        total += c;
    }
    if (threadIdx.x == 0 && total > 0) {
        atomicAdd(&g.ctrl->flag_total, (uint32_t)total);
        // the tile's run is padded to a multiple of 4 entries (items never straddle tiles)
        s_base = atomicAdd(&g.ctrl->list_len, (uint32_t)((total + 3) & ~3));
    }
    __syncthreads();
    if (total > 0 && (int)threadIdx.x < ((-total) & 3)) g.flag_list[s_base + total + threadIdx.x] = kListPad;
    if (flag) {
        const int pos = base + __popc(ballot & ((1u << lane) - 1u));
        g.flag_list[s_base + pos] = ((uint32_t)seq << kPixBits) | (uint32_t)((size_t)y * p.W + x);
    }
}

// Pass 1: one persistent launch over the queue of every sequence, in the
// single-sequence window-box form (items of kItem entries; an item stays
// inside one tile of one sequence).
template <int kItem, bool kMixed>
__global__ void __launch_bounds__(kTilePix, 2) batch_wlr_kernel(BatchGlobal g, const WlrParams gp)
{
    sparse_body<kItem, kMixed>(gp, BatchSeq{g.steps});
}

// Pass 2: solve every record and emit into its sequence's maps; the last CTA
// scans the per-chunk event counts of all sequences for the writer.
template <bool kMixed>
__global__ void __launch_bounds__(kSolveThreads, 3) batch_solve_kernel(BatchGlobal g, const WlrParams gp)
{
    const uint32_t n = *(volatile uint32_t*)&g.ctrl->list_len;
    const unsigned long long fp64 = solve_records<kMixed>(gp, BatchSeq{g.steps}, n);
    finish(gp, 0ull, 0ull, fp64, false, true);
}

__global__ void __launch_bounds__(kTilePix) batch_event_write_kernel(BatchGlobal g)
{
    constexpr int kPer = kChunk / kTilePix;
    __shared__ int s_warp[kTilePix / 32];
    const int gc = blockIdx.x;
    if (g.chunk_cnt[gc] == 0u) return;
    const int seq = g.chunk_seq[gc];
    const SeqStep& st = g.steps[seq];
    const WlrParams& sp = st.wp;
    const long long n_pix = (long long)sp.W * sp.H;
    const long long p0 = (long long)(gc - st.chunk_base) * kChunk + (long long)threadIdx.x * kPer;
    int v[kPer];
    int c = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        v[k] = (p0 + k < n_pix) ? sp.nev[p0 + k] : 0;
        c += abs(v[k]);
    }
    int total;
    const int off = block_exclusive_scan(c, s_warp, total);
    unsigned long long pos = g.chunk_off[gc] + (unsigned long long)off;
    bool overflow = false;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int n = abs(v[k]);
        if (n == 0) continue;
        const long long pix = p0 + k;
        const uint32_t x = (uint32_t)(pix % sp.W), y = (uint32_t)(pix / sp.W);
        const uint32_t w1 = x | (y << 16);
        const uint32_t w2 = (uint32_t)(uint8_t)(int8_t)(v[k] > 0 ? 1 : -1) | ((uint32_t)seq << 16);
        for (int e = 0; e < n; ++e, ++pos) {
            if (pos >= g.capacity) {
                overflow = true;
                continue;
            }
            uint32_t* rec = reinterpret_cast<uint32_t*>(g.events + pos);
            rec[0] = st.frame;
            rec[1] = w1;
            rec[2] = w2;
        }
    }
    if (overflow) atomicOr(&g.ctrl->status, kStatusOverflow);
}

typedef void (*WlrKernel)(BatchGlobal, const WlrParams);

// lanes per pixel 8, 16, 32 <-> items of 4, 2, 1 queue entries
WlrKernel pick_kernel(int lanes, bool mixed)
{
    if (mixed) {
        if (lanes == 8) return batch_wlr_kernel<4, true>;
        if (lanes == 32) return batch_wlr_kernel<1, true>;
        return batch_wlr_kernel<2, true>;
    }
    if (lanes == 8) return batch_wlr_kernel<4, false>;
    if (lanes == 32) return batch_wlr_kernel<1, false>;
    return batch_wlr_kernel<2, false>;
}

const double kExp2Scale = 0.84932180028801904272;

}  // namespace
}  // namespace esim

using namespace esim;

struct esim_ad_batch {
    std::vector<esim_ad_config> cfg;
    int n = 0;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    bool mixed = false;
    // per sequence
    std::vector<size_t> N;
    std::vector<int> n_chunks, chunk_base;
    // per tile shape: tiles across, tile count and first global tile of each
    // sequence; global tile -> sequence table
    std::vector<int> tiles_x[kTileShapes], n_tiles[kTileShapes], tile_base[kTileShapes];
    int total_tiles_s[kTileShapes] = {0, 0, 0};
    uint16_t* tile_seq_s[kTileShapes] = {nullptr, nullptr, nullptr};
    float* gram = nullptr;   // Gram records, one per queue entry
    std::vector<void*> ring;
    std::vector<float4*> state;
    std::vector<float*> alpha;
    std::vector<uint8_t*> flag;
    std::vector<int32_t*> nev;
    std::vector<uint64_t> t;        // frames pushed per sequence
    // global
    int total_chunks = 0;
    size_t total_pix = 0;
    uint16_t* chunk_seq = nullptr;
    uint32_t* flag_list = nullptr;
    uint32_t* chunk_cnt = nullptr;
    unsigned long long* chunk_off = nullptr;
    esim_ad_batch_event* events = nullptr;
    Ctrl* ctrl = nullptr;
    SeqStep* d_steps = nullptr;
    SeqStep* h_steps[2] = {nullptr, nullptr};   // pinned, alternating
    cudaEvent_t h_free[2] = {nullptr, nullptr};
    int cur = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int grid = 0;
    int solve_grid = 0;
    int smem = 0;        // dynamic shared memory of the accumulation launch
    int lanes = 8;       // lanes per pixel (items of 32 / lanes entries)
    int shape = 1;       // tile shape index into kTileWidths
    bool tuned = false;
    int tune_stage = 0;                         // candidates measured so far
    float tune_ms[9] = {};
    unsigned long long tune_reg[9] = {};
    cudaEvent_t tune_ev[18] = {};
    unsigned long long reg_before = 0;
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_cls;
    size_t prof_used = 0;
    uint64_t prof_kernels = 0;
    esim_ad_status sticky = ESIM_AD_OK;
    uint64_t steps = 0;
};

namespace {

// Tuning candidates: (tile shape index, lanes per pixel), all nine pairs.
constexpr int kNumCandidates = 9;
const int kCandLanes[3] = {8, 16, 32};

std::string cache_key(const esim_ad_batch* b)
{
    char k[128];
    snprintf(k, sizeof(k), "batch r=%d T=%d precision=%d sms=%d", b->cfg[0].radius, b->cfg[0].frames,
             b->cfg[0].precision, b->num_sms);
    return k;
}

// Cached choice encoded as 100 * tile shape index + lanes per pixel.
bool cache_lookup(const esim_ad_batch* b, int* shape, int* lanes)
{
    const int v = tune_cache_lookup(cache_key(b).c_str());
    const int sh = v / 100, l = v % 100;
    if (sh < 0 || sh >= kTileShapes || (l != 8 && l != 16 && l != 32)) return false;
    *shape = sh;
    *lanes = l;
    return true;
}

void cache_store(const esim_ad_batch* b, int shape, int lanes)
{
    tune_cache_store(cache_key(b).c_str(), 100 * shape + lanes);
}

void batch_release(esim_ad_batch* b)
{
    for (int i = 0; i < b->n; ++i) {
        if (i < (int)b->ring.size() && b->ring[i]) cudaFree(b->ring[i]);
        if (i < (int)b->state.size() && b->state[i]) cudaFree(b->state[i]);
        if (i < (int)b->alpha.size() && b->alpha[i]) cudaFree(b->alpha[i]);
        if (i < (int)b->flag.size() && b->flag[i]) cudaFree(b->flag[i]);
        if (i < (int)b->nev.size() && b->nev[i]) cudaFree(b->nev[i]);
    }
    void* g[] = {b->tile_seq_s[0], b->tile_seq_s[1], b->tile_seq_s[2], b->chunk_seq, b->flag_list, b->gram,
                 b->chunk_cnt, b->chunk_off, b->events, b->ctrl, b->d_steps};
    for (void* p : g)
        if (p) cudaFree(p);
    for (int k = 0; k < 2; ++k) {
        if (b->h_steps[k]) cudaFreeHost(b->h_steps[k]);
        if (b->h_free[k]) cudaEventDestroy(b->h_free[k]);
        if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
    }
    for (cudaEvent_t e : b->tune_ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : b->prof_ev) cudaEventDestroy(e);
}

BatchGlobal globals(const esim_ad_batch* b, int shape)
{
    BatchGlobal g;
    g.steps = b->d_steps;
    g.tile_seq = b->tile_seq_s[shape];
    g.chunk_seq = b->chunk_seq;
    g.flag_list = b->flag_list;
    g.chunk_cnt = b->chunk_cnt;
    g.chunk_off = b->chunk_off;
    g.events = b->events;
    g.capacity = b->cfg[0].event_capacity;
    g.total_tiles = b->total_tiles_s[shape];
    g.total_chunks = b->total_chunks;
    g.tx = kTileWidths[shape];
    g.r = b->cfg[0].radius;
    g.s_px = (float)(kExp2Scale / ((double)b->cfg[0].h * b->cfg[0].radius));
    g.ctrl = b->ctrl;
    return g;
}

// Parameters shared by every sequence of the batch (window, bandwidths,
// ridge), the queue, the Gram records and the accounting of finish(); the
// per-sequence ones travel in the step table.
WlrParams global_wlr(const esim_ad_batch* b)
{
    const esim_ad_config& c0 = b->cfg[0];
    WlrParams p;
    memset(&p, 0, sizeof(p));
    p.r = c0.radius;
    p.T = c0.frames;
    p.mixed = b->mixed ? 1 : 0;
    p.s_coord = (float)(kExp2Scale / c0.h);
    p.s_coord_px = (float)(kExp2Scale / ((double)c0.h * c0.radius));
    for (int j = 0; j < 7; ++j) {
        p.s_feat[j] = (float)(kExp2Scale / ((double)c0.h * c0.bandwidth[j]));
        p.fscale[j] = b->mixed ? c0.feature_scale[j] : 1.0f;
        p.q_scale[j] = (float)((double)p.s_feat[j] * p.fscale[j]);
    }
    p.ridge = c0.ridge;
    p.sparse_stage = 1;
    p.poll_limit = kPollLimit;
    p.withhold_copy = 0;
    p.flag_list = b->flag_list;
    p.gram = b->gram;
    p.chunk_cnt = b->chunk_cnt;
    p.chunk_off = b->chunk_off;
    p.n_chunks = b->total_chunks;
    p.emit_events = 1;
    p.ctrl = b->ctrl;
    return p;
}

// Fill the host step table for the frames of this step.
void fill_steps(esim_ad_batch* b, SeqStep* h, const esim_ad_frame* frames, int shape)
{
    const esim_ad_config& c0 = b->cfg[0];
    for (int i = 0; i < b->n; ++i) {
        SeqStep& st = h[i];
        memset(&st, 0, sizeof(st));
        const esim_ad_config& c = b->cfg[i];
        const esim_ad_frame& f = frames[i];
        const bool act = f.radiance != nullptr;
        st.active = act ? 1 : 0;
        st.tile_base = b->tile_base[shape][i];
        st.chunk_base = b->chunk_base[i];
        const uint64_t t64 = b->t[i];
        const int t = (int)(t64 % 0x7fffffff);
        st.frame = (uint32_t)t64;
        IngestParams& ip = st.ip;
        ip.rad = f.radiance;
        ip.normal = f.normal;
        ip.albedo = f.albedo;
        ip.depth = f.depth;
        ip.feat_bf16 = reinterpret_cast<const unsigned short*>(f.features);
        ip.rad_fmt = c0.radiance_fmt;
        ip.feat_fmt = c0.feature_fmt;
        ip.mixed = b->mixed ? 1 : 0;
        for (int j = 0; j < 7; ++j) {
            const float fs = (c0.feature_fmt == ESIM_AD_FEAT_BF16 || b->mixed) ? c0.feature_scale[j] : 1.0f;
            ip.fscale[j] = fs;
            ip.inv_fscale[j] = 1.0f / fs;
        }
        ip.W = c.width;
        ip.H = c.height;
        ip.pitch = f.pitch_elems ? f.pitch_elems : c.width;
        ip.tiles_x = b->tiles_x[shape][i];
        ip.slot = t % c0.frames;
        ip.test = (c0.mode == ESIM_AD_ADAPTIVE && t64 > 0) ? 1 : 0;
        ip.log_eps = c0.log_eps;
        ip.C = c.contrast;
        ip.guard_kappa = c.guard_kappa > 0.0f ? c.guard_kappa : 0.0f;
        ip.variance = ip.guard_kappa > 0.0f ? f.variance : nullptr;
        ip.ring = b->ring[i];
        ip.state = b->state[i];
        ip.flag = b->flag[i];
        ip.nev = b->nev[i];
        WlrParams& wp = st.wp;
        wp.W = c.width;
        wp.H = c.height;
        wp.r = c0.radius;
        wp.T = c0.frames;
        wp.t = t;
        wp.n_tau = (int)((t64 + 1) < (uint64_t)c0.frames ? (t64 + 1) : (uint64_t)c0.frames);
        wp.tiles_x = b->tiles_x[shape][i];
        wp.n_tiles = b->n_tiles[shape][i];
        wp.mixed = b->mixed ? 1 : 0;
        wp.init = t64 == 0 ? 1 : 0;
        wp.C = c.contrast;
        wp.s_coord = (float)(kExp2Scale / c0.h);
        wp.s_coord_px = (float)(kExp2Scale / ((double)c0.h * c0.radius));
        for (int j = 0; j < 7; ++j) {
            wp.s_feat[j] = (float)(kExp2Scale / ((double)c0.h * c0.bandwidth[j]));
            wp.fscale[j] = b->mixed ? c0.feature_scale[j] : 1.0f;
            wp.q_scale[j] = (float)((double)wp.s_feat[j] * wp.fscale[j]);
        }
        wp.ridge = c0.ridge;
        wp.ring = b->ring[i];
        wp.state = b->state[i];
        wp.alpha = b->alpha[i];
        wp.nev = b->nev[i];
        wp.chunk_cnt = b->chunk_cnt + b->chunk_base[i];
        wp.chunk_off = b->chunk_off + b->chunk_base[i];
        wp.n_chunks = b->n_chunks[i];
        wp.emit_events = 1;
        wp.ctrl = b->ctrl;
    }
}

// Enqueue one step's work (after the step table has been copied) on stream s.
cudaError_t enqueue_step_body(esim_ad_batch* b, int shape, int lanes, cudaStream_t s, bool profile)
{
    const BatchGlobal g = globals(b, shape);
    const WlrParams gp = global_wlr(b);
    auto rec = [&](int cls, bool start) {
        if (!profile) return;
        if (start) {
            if (2 * b->prof_used + 2 > b->prof_ev.size())
                for (int k = 0; k < 2; ++k) {
                    cudaEvent_t e;
                    if (cudaEventCreate(&e) == cudaSuccess) b->prof_ev.push_back(e);
                }
            b->prof_cls.resize(b->prof_used + 1);
            b->prof_cls[b->prof_used] = cls;
            cudaEventRecord(b->prof_ev[2 * b->prof_used], s);
        } else {
            cudaEventRecord(b->prof_ev[2 * b->prof_used + 1], s);
            ++b->prof_used;
        }
    };
    cudaError_t e = cudaMemsetAsync(b->ctrl, 0, kCtrlPerFrameBytes, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b->chunk_cnt, 0, (size_t)b->total_chunks * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    rec(0, true);
    batch_ingest_kernel<<<b->total_tiles_s[shape], kTilePix, 0, s>>>(g);
    rec(0, false);
    rec(1, true);
    pick_kernel(lanes, b->mixed)<<<b->grid, kTilePix, b->smem, s>>>(g, gp);
    if (b->mixed)
        batch_solve_kernel<true><<<b->solve_grid, kSolveThreads, 0, s>>>(g, gp);
    else
        batch_solve_kernel<false><<<b->solve_grid, kSolveThreads, 0, s>>>(g, gp);
    rec(1, false);
    rec(2, true);
    batch_event_write_kernel<<<b->total_chunks, kTilePix, 0, s>>>(g);
    rec(2, false);
    b->prof_kernels += 4;
    return cudaGetLastError();
}

cudaError_t build_graphs(esim_ad_batch* b, int shape, int lanes)
{
    for (int k = 0; k < 2; ++k) {
        if (b->graph[k]) {
            cudaGraphExecDestroy(b->graph[k]);
            b->graph[k] = nullptr;
        }
        // captured on a private stream (the caller's may be the legacy default
        // stream, which cannot be captured); launched on the caller's stream
        cudaGraph_t gr;
        cudaStream_t cs;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cs);
            return e;
        }
        cudaMemcpyAsync(b->d_steps, b->h_steps[k], sizeof(SeqStep) * b->n, cudaMemcpyHostToDevice, cs);
        const uint64_t kern = b->prof_kernels;
        enqueue_step_body(b, shape, lanes, cs, false);
        b->prof_kernels = kern;
        e = cudaStreamEndCapture(cs, &gr);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return e;
        e = cudaGraphInstantiate(&b->graph[k], gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

esim_ad_status esim_ad_batch_init(const esim_ad_config* cfgs, int32_t n_seq, void* cuda_stream,
                                  esim_ad_batch** out)
{
    if (!cfgs || !out || n_seq < 1 || n_seq > kMaxSeq) return ESIM_AD_EINVAL;
    const esim_ad_config& c0 = cfgs[0];
    for (int i = 0; i < n_seq; ++i) {
        const esim_ad_config& c = cfgs[i];
        if (c.struct_size != sizeof(esim_ad_config) || c.width < 1 || c.height < 1 || c.width > 65535 ||
            c.height > 65535 || (long long)c.width * c.height > (1ll << kPixBits) || !(c.contrast > 0.0f))
            return ESIM_AD_EINVAL;
        if (c.radius != c0.radius || c.frames != c0.frames || c.mode != c0.mode ||
            c.radiance_fmt != c0.radiance_fmt || c.feature_fmt != c0.feature_fmt || c.precision != c0.precision ||
            c.h != c0.h || c.log_eps != c0.log_eps || c.ridge != c0.ridge ||
            memcmp(c.bandwidth, c0.bandwidth, sizeof(c.bandwidth)) != 0 ||
            memcmp(c.feature_scale, c0.feature_scale, sizeof(c.feature_scale)) != 0)
            return ESIM_AD_EINVAL;
    }
    // the shared fields go through the single-sequence checks
    {
        const esim_ad_config& probe = c0;
        if (probe.radius < 1 || probe.radius > kMaxRadius || probe.frames < 1 || probe.frames > kMaxFrames ||
            (probe.mode != ESIM_AD_ADAPTIVE && probe.mode != ESIM_AD_EXHAUSTIVE) || !(probe.h > 0.0f) ||
            !(probe.ridge > 0.0f) || probe.log_eps < 0.0f || probe.event_capacity < 1 ||
            (probe.precision != ESIM_AD_FP32 && probe.precision != ESIM_AD_MIXED) ||
            (probe.radiance_fmt != ESIM_AD_LUMA_F32 && probe.radiance_fmt != ESIM_AD_RGB_F32 &&
             probe.radiance_fmt != ESIM_AD_LOGLUMA_F16) ||
            (probe.feature_fmt != ESIM_AD_FEAT_F32 && probe.feature_fmt != ESIM_AD_FEAT_BF16))
            return ESIM_AD_EINVAL;
        for (int j = 0; j < 7; ++j)
            if (!(probe.bandwidth[j] > 0.0f)) return ESIM_AD_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return ESIM_AD_ECUDA;
    }
    esim_ad_batch* b = new (std::nothrow) esim_ad_batch();
    if (!b) return ESIM_AD_ENOMEM;
    b->cfg.assign(cfgs, cfgs + n_seq);
    b->n = n_seq;
    b->stream = (cudaStream_t)cuda_stream;
    b->device = dev;
    b->mixed = c0.precision == ESIM_AD_MIXED;
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    b->N.resize(n_seq);
    b->n_chunks.resize(n_seq);
    b->chunk_base.resize(n_seq);
    for (int sh = 0; sh < kTileShapes; ++sh) {
        b->tiles_x[sh].resize(n_seq);
        b->n_tiles[sh].resize(n_seq);
        b->tile_base[sh].resize(n_seq);
    }
    b->ring.assign(n_seq, nullptr);
    b->state.assign(n_seq, nullptr);
    b->alpha.assign(n_seq, nullptr);
    b->flag.assign(n_seq, nullptr);
    b->nev.assign(n_seq, nullptr);
    b->t.assign(n_seq, 0);
    std::vector<uint16_t> tseq[kTileShapes], cseq;
    int max_tiles = 0;
    for (int i = 0; i < n_seq; ++i) {
        const esim_ad_config& c = cfgs[i];
        b->N[i] = (size_t)c.width * c.height;
        b->n_chunks[i] = (int)((b->N[i] + kChunk - 1) / kChunk);
        b->chunk_base[i] = b->total_chunks;
        b->total_chunks += b->n_chunks[i];
        b->total_pix += b->N[i];
        cseq.insert(cseq.end(), b->n_chunks[i], (uint16_t)i);
        for (int sh = 0; sh < kTileShapes; ++sh) {
            const int tw = kTileWidths[sh], th = kTilePix / tw;
            b->tiles_x[sh][i] = (c.width + tw - 1) / tw;
            b->n_tiles[sh][i] = b->tiles_x[sh][i] * ((c.height + th - 1) / th);
            b->tile_base[sh][i] = b->total_tiles_s[sh];
            b->total_tiles_s[sh] += b->n_tiles[sh][i];
            tseq[sh].insert(tseq[sh].end(), b->n_tiles[sh][i], (uint16_t)i);
        }
    }
    for (int sh = 0; sh < kTileShapes; ++sh) max_tiles = std::max(max_tiles, b->total_tiles_s[sh]);
    const size_t list_cap = b->total_pix + 4 * (size_t)max_tiles;   // queue entries incl. tile padding
    auto fail = [&](esim_ad_status st) {
        cudaGetLastError();
        batch_release(b);
        delete b;
        return st;
    };
    const size_t ring_rec = b->mixed ? 1 : 2;
    for (int i = 0; i < n_seq; ++i) {
        const size_t N = b->N[i];
        if (cudaMalloc(&b->ring[i], ring_rec * c0.frames * N * 16) != cudaSuccess ||
            cudaMalloc((void**)&b->state[i], 4 * N * sizeof(float4)) != cudaSuccess ||
            cudaMalloc((void**)&b->alpha[i], N * sizeof(float)) != cudaSuccess ||
            cudaMalloc((void**)&b->flag[i], N) != cudaSuccess ||
            cudaMalloc((void**)&b->nev[i], N * sizeof(int32_t)) != cudaSuccess)
            return fail(ESIM_AD_ENOMEM);
        if (cudaMemset(b->state[i], 0, 4 * N * sizeof(float4)) != cudaSuccess ||
            cudaMemset(b->nev[i], 0, N * sizeof(int32_t)) != cudaSuccess)
            return fail(ESIM_AD_ECUDA);
    }
    for (int sh = 0; sh < kTileShapes; ++sh)
        if (cudaMalloc((void**)&b->tile_seq_s[sh], tseq[sh].size() * 2) != cudaSuccess) return fail(ESIM_AD_ENOMEM);
    if (cudaMalloc((void**)&b->chunk_seq, cseq.size() * 2) != cudaSuccess ||
        cudaMalloc((void**)&b->flag_list, list_cap * 4) != cudaSuccess ||
        cudaMalloc((void**)&b->gram, list_cap * kGramRecordBytes) != cudaSuccess ||
        cudaMalloc((void**)&b->chunk_cnt, (size_t)b->total_chunks * 4) != cudaSuccess ||
        cudaMalloc((void**)&b->chunk_off, (size_t)b->total_chunks * 8) != cudaSuccess ||
        cudaMalloc((void**)&b->events, (size_t)c0.event_capacity * sizeof(esim_ad_batch_event)) != cudaSuccess ||
        cudaMalloc((void**)&b->ctrl, sizeof(Ctrl)) != cudaSuccess ||
        cudaMalloc((void**)&b->d_steps, sizeof(SeqStep) * n_seq) != cudaSuccess)
        return fail(ESIM_AD_ENOMEM);
    for (int k = 0; k < 2; ++k) {
        if (cudaMallocHost((void**)&b->h_steps[k], sizeof(SeqStep) * n_seq) != cudaSuccess)
            return fail(ESIM_AD_ENOMEM);
        if (cudaEventCreateWithFlags(&b->h_free[k], cudaEventDisableTiming) != cudaSuccess)
            return fail(ESIM_AD_ECUDA);
        memset(b->h_steps[k], 0, sizeof(SeqStep) * n_seq);
    }
    for (cudaEvent_t& e : b->tune_ev)
        if (cudaEventCreate(&e) != cudaSuccess) return fail(ESIM_AD_ECUDA);
    for (int sh = 0; sh < kTileShapes; ++sh)
        if (cudaMemcpy(b->tile_seq_s[sh], tseq[sh].data(), tseq[sh].size() * 2, cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return fail(ESIM_AD_ECUDA);
    if (cudaMemcpy(b->chunk_seq, cseq.data(), cseq.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->ctrl, 0, sizeof(Ctrl)) != cudaSuccess)
        return fail(ESIM_AD_ECUDA);
    // the accumulation kernels' dynamic shared memory: window tables and per-warp boxes
    b->smem = box_layout(b->cfg[0].radius).total;
    for (int lanes : {8, 16, 32})
        if (cudaFuncSetAttribute(pick_kernel(lanes, b->mixed), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 b->smem) != cudaSuccess)
            return fail(ESIM_AD_ECUDA);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pick_kernel(16, b->mixed), kTilePix, b->smem) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    cudaGetLastError();
    b->grid = per_sm * b->num_sms;
    b->solve_grid = 3 * b->num_sms;
    // tile shape and lanes per pixel: forced (both variables set), cached, or
    // tuned on the first adaptive steps
    {
        const char* el = getenv("ESIM_AD_BATCH_LANES");
        const char* et = getenv("ESIM_AD_BATCH_TILE");
        const int l = el ? atoi(el) : 0, tw = et ? atoi(et) : 0;
        int sh = -1;
        for (int k = 0; k < kTileShapes; ++k)
            if (kTileWidths[k] == tw) sh = k;
        if ((l == 8 || l == 16 || l == 32) && sh >= 0) {
            b->lanes = l;
            b->shape = sh;
            b->tuned = true;
        }
    }
    if (!b->tuned && cache_lookup(b, &b->shape, &b->lanes)) b->tuned = true;
    if (build_graphs(b, b->shape, b->lanes) != cudaSuccess) return fail(ESIM_AD_ECUDA);
    *out = b;
    return ESIM_AD_OK;
}

esim_ad_status esim_ad_batch_step(esim_ad_batch* b, const esim_ad_frame* frames)
{
    if (!b || !frames) return ESIM_AD_EINVAL;
    if (b->sticky != ESIM_AD_OK) return ESIM_AD_ESTATE;
    for (int i = 0; i < b->n; ++i) {
        const esim_ad_frame& f = frames[i];
        if (!f.radiance) continue;
        if (f.on_host) return ESIM_AD_EINVAL;
        if (f.pitch_elems != 0 && f.pitch_elems < b->cfg[i].width) return ESIM_AD_EINVAL;
        if (b->cfg[0].feature_fmt == ESIM_AD_FEAT_BF16 ? !f.features : (!f.normal || !f.albedo || !f.depth))
            return ESIM_AD_EINVAL;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    const int k = b->cur;
    // the pinned table k was last read by the step launched two steps ago
    if (cudaEventSynchronize(b->h_free[k]) != cudaSuccess) return ESIM_AD_ECUDA;
    // the tuning steps run their own candidate's tile shape
    const bool tuning0 = !b->tuned && b->cfg[0].mode == ESIM_AD_ADAPTIVE;
    const int cand = b->tune_stage;
    const int step_shape = tuning0 ? cand / 3 : b->shape;
    fill_steps(b, b->h_steps[k], frames, step_shape);
    bool any_init = false, any_active = false;
    for (int i = 0; i < b->n; ++i)
        if (frames[i].radiance) {
            any_active = true;
            any_init |= b->t[i] == 0;
        }
    cudaError_t e = cudaSuccess;
    // autotuning: the first adaptive steps without sequence starts time one candidate each
    const bool tuning = !b->tuned && any_active && !any_init && b->cfg[0].mode == ESIM_AD_ADAPTIVE;
    if (tuning || b->prof_on) {
        // direct launches (timed) instead of the graph
        e = cudaMemcpyAsync(b->d_steps, b->h_steps[k], sizeof(SeqStep) * b->n, cudaMemcpyHostToDevice, b->stream);
        const int lanes = tuning ? kCandLanes[cand % 3] : b->lanes;
        if (tuning) cudaEventRecord(b->tune_ev[2 * cand], b->stream);
        if (e == cudaSuccess) e = enqueue_step_body(b, step_shape, lanes, b->stream, b->prof_on);
        if (tuning) cudaEventRecord(b->tune_ev[2 * cand + 1], b->stream);
    } else if (step_shape == b->shape) {
        e = cudaGraphLaunch(b->graph[k], b->stream);
        b->prof_kernels += 4;
    } else {
        // a start-up step while tuning is pending: the graph's tile shape may differ
        e = cudaMemcpyAsync(b->d_steps, b->h_steps[k], sizeof(SeqStep) * b->n, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = enqueue_step_body(b, step_shape, b->lanes, b->stream, false);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->h_free[k], b->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
        return ESIM_AD_ECUDA;
    }
    if (tuning) {
        // per-regression time of this candidate (the step's regressions from the counters)
        Ctrl h;
        cudaMemcpyAsync(&h, b->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream);
        cudaStreamSynchronize(b->stream);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, b->tune_ev[2 * cand], b->tune_ev[2 * cand + 1]);
        b->tune_ms[cand] = ms;
        b->tune_reg[cand] = h.regressions - b->reg_before;
        b->reg_before = h.regressions;
        if (++b->tune_stage == kNumCandidates) {
            // the pair with the least step time per regressed pixel
            int best = 4;   // 32x8 tiles, 8 lanes
            double best_cost = 1e300;
            for (int c = 0; c < kNumCandidates; ++c) {
                const double cost = b->tune_ms[c] / (double)(b->tune_reg[c] ? b->tune_reg[c] : 1);
                if (cost < best_cost) {
                    best_cost = cost;
                    best = c;
                }
            }
            b->shape = best / 3;
            b->lanes = kCandLanes[best % 3];
            b->tuned = true;
            cache_store(b, b->shape, b->lanes);
            if (build_graphs(b, b->shape, b->lanes) != cudaSuccess) return ESIM_AD_ECUDA;
        }
    } else if (!b->tuned) {
        // keep the regression count current for the tuning steps to come
        Ctrl h;
        cudaMemcpyAsync(&h, b->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream);
        cudaStreamSynchronize(b->stream);
        b->reg_before = h.regressions;
    }
    for (int i = 0; i < b->n; ++i)
        if (frames[i].radiance) b->t[i] += 1;
    b->cur ^= 1;
    b->steps += 1;
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    return ESIM_AD_OK;
}

esim_ad_status esim_ad_batch_events(esim_ad_batch* b, esim_ad_batch_event* dst, uint64_t cap, uint64_t* n_out,
                                    int dst_is_device)
{
    if (!b || !n_out || (cap > 0 && !dst)) return ESIM_AD_EINVAL;
    if (b->sticky != ESIM_AD_OK) return ESIM_AD_ESTATE;
    Ctrl h;
    if (cudaMemcpyAsync(&h, b->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return ESIM_AD_ECUDA;
    if (h.status & kStatusTimeout) b->sticky = ESIM_AD_ETIMEOUT;
    else if (h.status & kStatusOverflow) b->sticky = ESIM_AD_EOVERFLOW;
    *n_out = h.ev_total;
    if (b->sticky != ESIM_AD_OK) return b->sticky;
    if (cap < h.ev_total) return ESIM_AD_ENOSPACE;
    if (h.ev_total > 0) {
        if (cudaMemcpyAsync(dst, b->events, h.ev_total * sizeof(esim_ad_batch_event),
                            dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
            cudaMemsetAsync(&b->ctrl->ev_total, 0, sizeof(unsigned long long), b->stream) != cudaSuccess ||
            cudaStreamSynchronize(b->stream) != cudaSuccess)
            return ESIM_AD_ECUDA;
    }
    return ESIM_AD_OK;
}

esim_ad_status esim_ad_batch_reset_sequence(esim_ad_batch* b, int32_t seq)
{
    if (!b || seq < 0 || seq >= b->n) return ESIM_AD_EINVAL;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return ESIM_AD_ECUDA;
    b->t[seq] = 0;
    return ESIM_AD_OK;
}

esim_ad_status esim_ad_batch_denoised(esim_ad_batch* b, int32_t seq, float* alpha, uint8_t* flags,
                                      int dst_is_device)
{
    if (!b || seq < 0 || seq >= b->n) return ESIM_AD_EINVAL;
    const cudaMemcpyKind k = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t N = b->N[seq];
    if ((alpha && cudaMemcpyAsync(alpha, b->alpha[seq], N * sizeof(float), k, b->stream) != cudaSuccess) ||
        (flags && cudaMemcpyAsync(flags, b->flag[seq], N, k, b->stream) != cudaSuccess) ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return ESIM_AD_ECUDA;
    return ESIM_AD_OK;
}

esim_ad_status esim_ad_batch_get_state(esim_ad_batch* b, int32_t seq, float* l_last, float* beta, float* xc)
{
    if (!b || seq < 0 || seq >= b->n) return ESIM_AD_EINVAL;
    const size_t N = b->N[seq];
    std::vector<float4> h(4 * N);
    if (cudaMemcpyAsync(h.data(), b->state[seq], 4 * N * sizeof(float4), cudaMemcpyDeviceToHost, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return ESIM_AD_ECUDA;
    for (size_t i = 0; i < N; ++i) {
        const float4 b0 = h[i], b1 = h[N + i], x0 = h[2 * N + i], x1 = h[3 * N + i];
        if (l_last) l_last[i] = x1.w;
        if (beta) {
            float* q = beta + 7 * i;
            q[0] = b0.x; q[1] = b0.y; q[2] = b0.z; q[3] = b0.w; q[4] = b1.x; q[5] = b1.y; q[6] = b1.z;
        }
        if (xc) {
            float* q = xc + 7 * i;
            q[0] = x0.x; q[1] = x0.y; q[2] = x0.z; q[3] = x0.w; q[4] = x1.x; q[5] = x1.y; q[6] = x1.z;
        }
    }
    return ESIM_AD_OK;
}

esim_ad_status esim_ad_batch_stats(esim_ad_batch* b, esim_ad_stats* out, int32_t* lanes_out)
{
    if (!b || !out) return ESIM_AD_EINVAL;
    Ctrl h;
    if (cudaMemcpyAsync(&h, b->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return ESIM_AD_ECUDA;
    out->frames = b->steps;
    out->regressions = h.regressions;
    out->events = h.ev_cum;
    out->pixels = b->total_pix;
    out->fp64_solves = h.fp64_solves;
    out->staged_ingests = 0;   // the batched ingest has one form
    if (lanes_out) *lanes_out = b->lanes;
    return ESIM_AD_OK;
}

esim_ad_status esim_ad_batch_tiling(esim_ad_batch* b, int32_t* tile_w, int32_t* tile_h, int32_t* lanes)
{
    if (!b) return ESIM_AD_EINVAL;
    if (tile_w) *tile_w = kTileWidths[b->shape];
    if (tile_h) *tile_h = kTilePix / kTileWidths[b->shape];
    if (lanes) *lanes = b->lanes;
    return ESIM_AD_OK;
}

esim_ad_status esim_ad_batch_profile_enable(esim_ad_batch* b, int on)
{
    if (!b) return ESIM_AD_EINVAL;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return ESIM_AD_ECUDA;
    b->prof_on = on != 0;
    b->prof_used = 0;
    b->prof_kernels = 0;
    return ESIM_AD_OK;
}

esim_ad_status esim_ad_batch_profile_get(esim_ad_batch* b, esim_ad_profile* out)
{
    if (!b || !out) return ESIM_AD_EINVAL;
    Ctrl h;
    if (cudaMemcpyAsync(&h, b->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return ESIM_AD_ECUDA;
    memset(out, 0, sizeof(*out));
    for (size_t k = 0; k < b->prof_used; ++k) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, b->prof_ev[2 * k], b->prof_ev[2 * k + 1]) != cudaSuccess) return ESIM_AD_ECUDA;
        out->launches[b->prof_cls[k]] += 1;
        out->ms[b->prof_cls[k]] += ms;
    }
    out->kernels = b->prof_kernels;
    out->neighbours = h.neighbours;
    out->regressions = h.regressions;
    return ESIM_AD_OK;
}

void esim_ad_batch_destroy(esim_ad_batch* b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    batch_release(b);
    delete b;
}

}  // extern "C"
