// Host side of the C ABI declared in include/esim_ad.h: configuration checks,
// device memory, the TMA descriptor of the frame ring, and the per-frame
// launch sequence of the hot path.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "internal.h"

using namespace esim;

namespace {

// sqrt(log2(e) / 2): scaling a regressor by k/(h b) turns the product
// Gaussian exp(-sum (d/(h b))^2 / 2) of Eq. 5 into 2^(-sum u^2).
const double kExp2Scale = 0.84932180028801904272;

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Allocation-failure injection for tests: ESIM_AD_FAULT_ALLOC=<k> makes the
// k-th device allocation of the process (1-based) fail with ENOMEM.
int g_alloc_seq = 0;

bool fault_alloc_now()
{
    const char* s = getenv("ESIM_AD_FAULT_ALLOC");
    ++g_alloc_seq;
    if (!s || !*s) return false;
    return atoi(s) == g_alloc_seq;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

struct esim_ad_ctx {
    esim_ad_config cfg;
    cudaStream_t stream = nullptr;
    cudaStream_t copy_stream = nullptr;
    // The event writer of a frame runs on its own stream, beside the next
    // frame's ingest and pass 1; the context's stream waits for it (ev_written)
    // before the next solve and before anything that reads what it writes.
    cudaStream_t writer_stream = nullptr;
    cudaEvent_t ev_solved = nullptr;
    cudaEvent_t ev_wr[kFrameEnds] = {};   // after frame f's writer (frame 0: its solve), at f % kFrameEnds
    int last_wr = 0;                      // slot of the latest pushed frame
    bool writer_pending = false;
    // drains of single frames copy on their own stream, so that they wait for
    // that frame's writer only, not for the frames pushed after it
    cudaStream_t drain_stream = nullptr;
    uint64_t drained = 0;                 // event positions drained so far
    unsigned long long* hmark = nullptr;  // pinned: a frame's end mark and the status word
    int device = 0;
    int W = 0, H = 0;
    size_t N = 0;
    int tiles_x = 0, tiles_y = 0, n_tiles = 0, n_chunks = 0;
    int smem_bytes = 0;          // dense tile-staged regression
    int smem_adaptive = 0;       // adaptive regression: the larger of its two forms
    int nbuf = 2;
    int wlr_grid = 0;
    int adaptive_grid = 0;
    int solve_grid = 0;
    int sparse_stage = 1;        // sparse kernel stages window boxes (ESIM_AD_SPARSE_STAGE=0: L1 only)
    int test_withhold = 0;       // ESIM_AD_TEST_WITHHOLD_COPY=1: timeout injection for tests
    bool mixed = false;
    uint32_t sparse_max = 0;     // adaptive frames with at most this many flagged pixels use the sparse kernel
    float4* ring = nullptr;
    float4* state = nullptr;
    float* alpha = nullptr;
    uint8_t* flag = nullptr;
    int32_t* nev = nullptr;
    uint32_t* tile_queue = nullptr;
    int32_t* tile_nflag = nullptr;
    uint8_t* tile_pix = nullptr;
    uint32_t* flag_list = nullptr;
    uint32_t* tile_base = nullptr;
    float* gram = nullptr;       // Gram records of the frame's regressed pixels
    uint32_t* chunk_cnt = nullptr;
    unsigned long long* chunk_off = nullptr;
    uint32_t* ev_mask = nullptr;  // one bit per pixel that emits (64 words per chunk), two buffers by frame parity
    esim_ad_event* events = nullptr;
    Ctrl* ctrl = nullptr;
    float* staging[2] = {nullptr, nullptr};   // host-frame landing buffers [11][H][W]
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};
    cudaEvent_t ev_consumed[2] = {nullptr, nullptr};
    int staging_next = 0;
    CUtensorMap tmap;
    // staged ingest (precision form, FP16/BF16 frames): the model-state map is
    // fixed; the input maps are encoded per frame (its pointers and pitch)
    CUtensorMap ingest_map_s;
    bool ingest_staged = false;
    int ingest_grid = 0;
    uint64_t staged_ingests = 0;   // frames that took the staged ingest since init/reset
    // kernel timing (esim_ad_profile_enable)
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_events;      // pool, pairs (start, stop)
    std::vector<int> prof_class;               // class of each recorded pair
    size_t prof_used = 0;                      // pairs recorded
    uint64_t prof_kernels = 0;                 // kernel launches while profiling
    uint64_t t = 0;
    esim_ad_status sticky = ESIM_AD_OK;
};

namespace {

esim_ad_status dev_alloc(void** p, size_t bytes)
{
    if (fault_alloc_now()) return ESIM_AD_ENOMEM;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return ESIM_AD_ENOMEM;
    }
    return ESIM_AD_OK;
}

bool finite_pos(float v) { return isfinite(v) && v > 0.0f; }

esim_ad_status check_config(const esim_ad_config* c)
{
    if (!c || c->struct_size != sizeof(esim_ad_config)) return ESIM_AD_EINVAL;
    if (c->width < 1 || c->height < 1 || c->width > 65535 || c->height > 65535) return ESIM_AD_EINVAL;
    if (c->radius < 1 || c->radius > kMaxRadius) return ESIM_AD_EINVAL;
    if (c->frames < 1 || c->frames > kMaxFrames) return ESIM_AD_EINVAL;
    if (c->mode != ESIM_AD_ADAPTIVE && c->mode != ESIM_AD_EXHAUSTIVE) return ESIM_AD_EINVAL;
    if (c->radiance_fmt != ESIM_AD_LUMA_F32 && c->radiance_fmt != ESIM_AD_RGB_F32 &&
        c->radiance_fmt != ESIM_AD_LOGLUMA_F16)
        return ESIM_AD_EINVAL;
    if (c->feature_fmt != ESIM_AD_FEAT_F32 && c->feature_fmt != ESIM_AD_FEAT_BF16) return ESIM_AD_EINVAL;
    if (c->precision != ESIM_AD_FP32 && c->precision != ESIM_AD_MIXED) return ESIM_AD_EINVAL;
    if (c->feature_fmt == ESIM_AD_FEAT_BF16 || c->precision == ESIM_AD_MIXED)
        for (int j = 0; j < 7; ++j)
            if (!finite_pos(c->feature_scale[j])) return ESIM_AD_EINVAL;
    if (!finite_pos(c->contrast) || !finite_pos(c->h) || !finite_pos(c->ridge)) return ESIM_AD_EINVAL;
    for (int j = 0; j < 7; ++j)
        if (!finite_pos(c->bandwidth[j])) return ESIM_AD_EINVAL;
    if (!isfinite(c->log_eps) || c->log_eps < 0.0f) return ESIM_AD_EINVAL;
    if (!isfinite(c->guard_kappa)) return ESIM_AD_EINVAL;
    if (c->event_capacity < 1 || c->event_capacity > (1ull << 36)) return ESIM_AD_EINVAL;
    return ESIM_AD_OK;
}

void release(esim_ad_ctx* c)
{
    void* ptrs[] = {c->ring, c->state, c->alpha, c->flag, c->nev, c->tile_queue, c->tile_nflag,
                    c->tile_pix, c->flag_list, c->tile_base, c->gram, c->chunk_cnt, c->chunk_off, c->ev_mask, c->events,
                    c->ctrl, c->staging[0], c->staging[1]};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int i = 0; i < 2; ++i) {
        if (c->ev_copied[i]) cudaEventDestroy(c->ev_copied[i]);
        if (c->ev_consumed[i]) cudaEventDestroy(c->ev_consumed[i]);
    }
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->writer_stream) cudaStreamDestroy(c->writer_stream);
    if (c->drain_stream) cudaStreamDestroy(c->drain_stream);
    if (c->hmark) cudaFreeHost(c->hmark);
    if (c->ev_solved) cudaEventDestroy(c->ev_solved);
    for (cudaEvent_t e : c->ev_wr)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : c->prof_events) cudaEventDestroy(e);
    c->prof_events.clear();
}

// Bracket one launch with a pair of pooled events when profiling is on.
struct ProfScope {
    esim_ad_ctx* c;
    cudaStream_t s;
    size_t pair = (size_t)-1;
    ProfScope(esim_ad_ctx* ctx, int cls, cudaStream_t stream) : c(ctx), s(stream)
    {
        if (!c->prof_on) return;
        if (2 * c->prof_used + 2 > c->prof_events.size()) {
            for (int k = 0; k < 2; ++k) {
                cudaEvent_t e;
                if (cudaEventCreate(&e) != cudaSuccess) return;
                c->prof_events.push_back(e);
            }
        }
        pair = c->prof_used++;
        if (c->prof_class.size() < c->prof_used) c->prof_class.resize(c->prof_used);
        c->prof_class[pair] = cls;
        cudaEventRecord(c->prof_events[2 * pair], s);
    }
    ~ProfScope()
    {
        if (pair != (size_t)-1) cudaEventRecord(c->prof_events[2 * pair + 1], s);
    }
};

// Order the context's stream after the latest frame's event writer.
cudaError_t join_writer(esim_ad_ctx* c)
{
    return c->writer_pending ? cudaStreamWaitEvent(c->stream, c->ev_wr[c->last_wr], 0) : cudaSuccess;
}

// Synchronise the context's stream, the event writer included.
cudaError_t sync_stream(esim_ad_ctx* c)
{
    const cudaError_t e = join_writer(c);
    return e != cudaSuccess ? e : cudaStreamSynchronize(c->stream);
}

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    }
    return fn;
}

// Tiled map without swizzle or interleave; out-of-range elements read as zero.
bool encode_tiled(CUtensorMap* m, CUtensorMapDataType dt, cuuint32_t rank, const void* ptr, const cuuint64_t* dims,
                  const cuuint64_t* strides, const cuuint32_t* box)
{
    EncodeTiledFn fn = encode_fn();
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return fn && fn(m, dt, rank, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Input maps of one FP16/BF16 frame for the staged ingest: {W, H} log
// brightness and {W, H, 7} features, boxes of one 32 x 8 tile.  False when the
// frame does not meet TMA's rules (16-byte aligned planes, row pitch a
// multiple of 16 bytes) or the encode fails: the frame takes the one-tile
// kernel then.
bool encode_frame_maps(const esim_ad_ctx* c, const esim_ad_frame* f, CUtensorMap* my, CUtensorMap* mf)
{
    const size_t pitch = f->pitch_elems ? (size_t)f->pitch_elems : (size_t)c->W;
    if ((pitch * 2) % 16 != 0 || (reinterpret_cast<uintptr_t>(f->radiance) & 15u) ||
        (reinterpret_cast<uintptr_t>(f->features) & 15u))
        return false;
    const cuuint64_t dy[2] = {(cuuint64_t)c->W, (cuuint64_t)c->H};
    const cuuint64_t sy[1] = {(cuuint64_t)pitch * 2};
    const cuuint32_t by[2] = {(cuuint32_t)kTileX, (cuuint32_t)kTileY};
    const cuuint64_t df[3] = {(cuuint64_t)c->W, (cuuint64_t)c->H, 7};
    const cuuint64_t sf[2] = {(cuuint64_t)pitch * 2, (cuuint64_t)pitch * 2 * c->H};
    const cuuint32_t bf[3] = {(cuuint32_t)kTileX, (cuuint32_t)kTileY, 7};
    return encode_tiled(my, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, f->radiance, dy, sy, by) &&
           encode_tiled(mf, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, f->features, df, sf, bf);
}

esim_ad_status encode_ring_map(esim_ad_ctx* c)
{
    // ring viewed as a 4-D tensor of 16-byte records: FP32 form {4 floats, W, H,
    // 2T half-planes}, box of both half-planes; mixed form {8 halves, W, H, T}
    const bool mixed = c->cfg.precision == ESIM_AD_MIXED;
    const cuuint64_t dims[4] = {mixed ? 8u : 4u, (cuuint64_t)c->W, (cuuint64_t)c->H,
                                (cuuint64_t)((mixed ? 1 : 2) * c->cfg.frames)};
    const cuuint64_t strides[3] = {16, (cuuint64_t)16 * c->W, (cuuint64_t)16 * c->W * c->H};
    const cuuint32_t box[4] = {mixed ? 8u : 4u, (cuuint32_t)(kTileX + 2 * c->cfg.radius),
                               (cuuint32_t)(kTileY + 2 * c->cfg.radius), mixed ? 1u : 2u};
    return encode_tiled(&c->tmap, mixed ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                        c->ring, dims, strides, box)
               ? ESIM_AD_OK
               : ESIM_AD_ECUDA;
}

esim_ad_status sync_and_check(esim_ad_ctx* c, Ctrl* host_ctrl)
{
    Ctrl tmp;
    Ctrl* h = host_ctrl ? host_ctrl : &tmp;
    if (join_writer(c) != cudaSuccess ||
        cudaMemcpyAsync(h, c->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return ESIM_AD_ECUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return ESIM_AD_ECUDA;
    if (h->status & kStatusTimeout) c->sticky = ESIM_AD_ETIMEOUT;
    else if (h->status & kStatusOverflow) c->sticky = ESIM_AD_EOVERFLOW;
    return ESIM_AD_OK;
}

}  // namespace

extern "C" {

const char* esim_ad_status_string(esim_ad_status s)
{
    switch (s) {
    case ESIM_AD_OK: return "ok";
    case ESIM_AD_EINVAL: return "invalid argument";
    case ESIM_AD_ENOMEM: return "out of memory";
    case ESIM_AD_ECUDA: return "CUDA error";
    case ESIM_AD_EOVERFLOW: return "event buffer overflow";
    case ESIM_AD_ETIMEOUT: return "device wait timed out";
    case ESIM_AD_ESTATE: return "context unusable after an earlier error";
    case ESIM_AD_ENOSPACE: return "destination buffer too small";
    }
    return "unknown status";
}

esim_ad_status esim_ad_init(const esim_ad_config* cfg, void* cuda_stream, esim_ad_ctx** out)
{
    if (!out) return ESIM_AD_EINVAL;
    esim_ad_status st = check_config(cfg);
    if (st != ESIM_AD_OK) return st;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return ESIM_AD_ECUDA;
    }
    esim_ad_ctx* c = new (std::nothrow) esim_ad_ctx();
    if (!c) return ESIM_AD_ENOMEM;
    c->cfg = *cfg;
    c->stream = (cudaStream_t)cuda_stream;
    c->device = dev;
    c->W = cfg->width;
    c->H = cfg->height;
    c->N = (size_t)c->W * c->H;
    c->tiles_x = (c->W + kTileX - 1) / kTileX;
    c->tiles_y = (c->H + kTileY - 1) / kTileY;
    c->n_tiles = c->tiles_x * c->tiles_y;
    c->n_chunks = (int)((c->N + kChunk - 1) / kChunk);
    int max_smem_sm = 0, num_sms = 0;
    if (cudaDeviceGetAttribute(&max_smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return ESIM_AD_ECUDA;
    }
    c->mixed = cfg->precision == ESIM_AD_MIXED;
    c->smem_bytes = (int)wlr_smem_bytes(cfg->radius, c->mixed, max_smem_sm, &c->nbuf);
    const size_t N = c->N, T = (size_t)cfg->frames;
    struct {
        void** p;
        size_t bytes;
    } allocs[] = {
        {(void**)&c->ring, 2 * T * N * sizeof(float4)},
        {(void**)&c->state, 4 * N * sizeof(float4)},
        {(void**)&c->alpha, N * sizeof(float)},
        {(void**)&c->flag, N},
        {(void**)&c->nev, N * sizeof(int32_t)},
        {(void**)&c->tile_queue, (size_t)c->n_tiles * sizeof(uint32_t)},
        {(void**)&c->tile_nflag, (size_t)c->n_tiles * sizeof(int32_t)},
        {(void**)&c->tile_pix, (size_t)c->n_tiles * kTilePix},
        {(void**)&c->flag_list, (N + 4 * (size_t)c->n_tiles) * sizeof(uint32_t)},   // + tile padding
        {(void**)&c->tile_base, (size_t)c->n_tiles * sizeof(uint32_t)},
        {(void**)&c->gram, (N + 4 * (size_t)c->n_tiles) * kGramRecordBytes},       // one per list entry or pixel
        {(void**)&c->chunk_cnt, 2 * (size_t)c->n_chunks * sizeof(uint32_t)},
        {(void**)&c->chunk_off, (size_t)c->n_chunks * sizeof(unsigned long long)},
        {(void**)&c->ev_mask, 2 * (size_t)c->n_chunks * (kChunk / 32) * sizeof(uint32_t)},
        {(void**)&c->events, (size_t)cfg->event_capacity * sizeof(esim_ad_event)},
        {(void**)&c->ctrl, sizeof(Ctrl)},
    };
    for (auto& a : allocs) {
        st = dev_alloc(a.p, a.bytes);
        if (st != ESIM_AD_OK) {
            release(c);
            delete c;
            return st;
        }
    }
    if (cudaMemset(c->ctrl, 0, sizeof(Ctrl)) != cudaSuccess ||
        cudaMemset(c->alpha, 0, N * sizeof(float)) != cudaSuccess ||
        cudaMemset(c->flag, 0, N) != cudaSuccess || cudaMemset(c->nev, 0, N * sizeof(int32_t)) != cudaSuccess ||
        cudaMemset(c->ev_mask, 0, 2 * (size_t)c->n_chunks * (kChunk / 32) * sizeof(uint32_t)) != cudaSuccess ||
        [&] {
            // the writer stream at the highest priority: its CTAs take the SMs as
            // the frame's solve drains, ahead of the next frame's ingest, instead
            // of waiting behind that frame's register-filling kernels
            int lo = 0, hi = 0;
            if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) return false;
            return cudaStreamCreateWithPriority(&c->writer_stream, cudaStreamNonBlocking, hi) == cudaSuccess;
        }() == false ||
        cudaStreamCreateWithFlags(&c->drain_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaHostAlloc((void**)&c->hmark, 2 * sizeof(unsigned long long), cudaHostAllocDefault) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_solved, cudaEventDisableTiming) != cudaSuccess ||
        [&] {
            for (cudaEvent_t& e : c->ev_wr)
                if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return false;
            return true;
        }() == false ||
        cudaMemset(c->state, 0, 4 * N * sizeof(float4)) != cudaSuccess) {
        release(c);
        delete c;
        return ESIM_AD_ECUDA;
    }
    {
        const int sp = wlr_sparse_smem(cfg->radius, c->mixed);
        c->smem_adaptive = c->smem_bytes > sp ? c->smem_bytes : sp;
    }
    if (encode_ring_map(c) != ESIM_AD_OK ||
        wlr_prepare(c->smem_bytes, c->smem_adaptive, c->mixed) != cudaSuccess) {
        cudaGetLastError();
        release(c);
        delete c;
        return ESIM_AD_ECUDA;
    }
    c->wlr_grid = wlr_grid(c->smem_bytes, num_sms, c->mixed, false);
    c->adaptive_grid = wlr_grid(c->smem_adaptive, num_sms, c->mixed, true);
    c->solve_grid = wlr_solve_grid(num_sms);
    // staged ingest for FP16/BF16 frames in the precision form (frames of at
    // least one tile); ESIM_AD_INGEST_STAGED=0 keeps the one-tile kernel
    if (c->mixed && cfg->radiance_fmt == ESIM_AD_LOGLUMA_F16 && cfg->feature_fmt == ESIM_AD_FEAT_BF16 &&
        c->W >= kTileX && c->H >= kTileY) {
        const char* e = getenv("ESIM_AD_INGEST_STAGED");
        // the model state {float4 [4][H][W]} as {4W, H, 4} floats; box: planes 0-1 of one tile
        const cuuint64_t dims[3] = {(cuuint64_t)4 * c->W, (cuuint64_t)c->H, 4};
        const cuuint64_t strides[2] = {(cuuint64_t)16 * c->W, (cuuint64_t)16 * c->W * c->H};
        const cuuint32_t box[3] = {(cuuint32_t)(4 * kTileX), (cuuint32_t)kTileY, 2};
        if (!(e && *e == '0') &&
            encode_tiled(&c->ingest_map_s, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->state, dims, strides, box)) {
            c->ingest_staged = true;
            c->ingest_grid = ingest_staged_grid(num_sms);
        }
    }
    // default: frames with up to 1/8 of the pixels flagged take the sparse kernel
    // (measured faster than tile staging at the 1-2% densities of edge-like
    // flag patterns); ESIM_AD_SPARSE_MAX overrides it (0: always the tile-staged
    // kernel; large: always sparse)
    c->sparse_max = (uint32_t)(c->N / 8);
    if (const char* e = getenv("ESIM_AD_SPARSE_MAX")) {
        if (*e) c->sparse_max = (uint32_t)strtoul(e, nullptr, 10);
    }
    if (const char* e = getenv("ESIM_AD_SPARSE_STAGE")) {
        if (*e == '0') c->sparse_stage = 0;
    }
    // Timeout injection for tests: ESIM_AD_TEST_WITHHOLD_COPY=1 makes every
    // warp of the sparse regression kernel skip issuing its first window-box
    // copy (nothing is in flight for that barrier) and bounds each mbarrier
    // wait to 64 polls, so the wait gives up, the kernel records the timeout
    // and returns; the normal bound is unchanged otherwise.
    if (const char* e = getenv("ESIM_AD_TEST_WITHHOLD_COPY")) {
        if (*e == '1') c->test_withhold = 1;
    }
    *out = c;
    return ESIM_AD_OK;
}

// Copy a host frame into one of two device landing buffers on the copy
// stream, ordered after the kernels that last read that buffer; the compute
// stream then waits for the copy.  Returns the device-side plane pointers.
static esim_ad_status stage_host_frame(esim_ad_ctx* c, const esim_ad_frame* f, esim_ad_frame* dev,
                                       int* slot_out)
{
    const size_t N = c->N;
    const int s = c->staging_next;
    if (!c->copy_stream) {
        if (cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
            return ESIM_AD_ECUDA;
        for (int i = 0; i < 2; ++i) {
            if (cudaEventCreateWithFlags(&c->ev_copied[i], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&c->ev_consumed[i], cudaEventDisableTiming) != cudaSuccess)
                return ESIM_AD_ECUDA;
            if (cudaEventRecord(c->ev_consumed[i], c->stream) != cudaSuccess) return ESIM_AD_ECUDA;
        }
    }
    if (!c->staging[s]) {
        esim_ad_status st = dev_alloc((void**)&c->staging[s], 11 * N * sizeof(float));
        if (st != ESIM_AD_OK) return st;
    }
    unsigned char* base = reinterpret_cast<unsigned char*>(c->staging[s]);
    if (cudaStreamWaitEvent(c->copy_stream, c->ev_consumed[s], 0) != cudaSuccess) return ESIM_AD_ECUDA;
    // landing layout: radiance at 0 (up to 3N floats), features after it, the
    // guard's variance plane last
    // each input (planes of `elem` bytes, rows of `pitch` elements on the host)
    // lands densely packed; the staged frame has row pitch = width
    struct Copy {
        const void* src;
        size_t off, elem;
        int planes;
    };
    Copy cp[5];
    int n = 0;
    const int rad_planes = c->cfg.radiance_fmt == ESIM_AD_RGB_F32 ? 3 : 1;
    const size_t rad_elem = c->cfg.radiance_fmt == ESIM_AD_LOGLUMA_F16 ? 2 : 4;
    cp[n++] = {f->radiance, 0, rad_elem, rad_planes};
    *dev = *f;
    dev->on_host = 0;
    dev->pitch_elems = 0;
    dev->radiance = base;
    if (c->cfg.feature_fmt == ESIM_AD_FEAT_BF16) {
        cp[n++] = {f->features, 12 * N, 2, 7};
        dev->features = base + 12 * N;
    } else {
        cp[n++] = {f->normal, 12 * N, 4, 3};
        cp[n++] = {f->albedo, 24 * N, 4, 3};
        cp[n++] = {f->depth, 36 * N, 4, 1};
        dev->normal = reinterpret_cast<const float*>(base + 12 * N);
        dev->albedo = reinterpret_cast<const float*>(base + 24 * N);
        dev->depth = reinterpret_cast<const float*>(base + 36 * N);
    }
    if (c->cfg.guard_kappa > 0.0f && f->variance) {
        cp[n++] = {f->variance, 40 * N, 4, 1};
        dev->variance = reinterpret_cast<const float*>(base + 40 * N);
    } else {
        dev->variance = nullptr;
    }
    const size_t pitch = f->pitch_elems ? (size_t)f->pitch_elems : (size_t)c->W;
    for (int k = 0; k < n; ++k) {
        const size_t e = cp[k].elem;
        cudaError_t err;
        if (pitch == (size_t)c->W)
            err = cudaMemcpyAsync(base + cp[k].off, cp[k].src, cp[k].planes * N * e, cudaMemcpyHostToDevice,
                                  c->copy_stream);
        else   // all planes at once: rows of W elements out of rows of `pitch`
            err = cudaMemcpy2DAsync(base + cp[k].off, c->W * e, cp[k].src, pitch * e, c->W * e,
                                    (size_t)cp[k].planes * c->H, cudaMemcpyHostToDevice, c->copy_stream);
        if (err != cudaSuccess) return ESIM_AD_ECUDA;
    }
    if (cudaEventRecord(c->ev_copied[s], c->copy_stream) != cudaSuccess) return ESIM_AD_ECUDA;
    if (cudaStreamWaitEvent(c->stream, c->ev_copied[s], 0) != cudaSuccess) return ESIM_AD_ECUDA;
    *slot_out = s;
    c->staging_next ^= 1;
    return ESIM_AD_OK;
}

esim_ad_status esim_ad_push_frame(esim_ad_ctx* c, const esim_ad_frame* fin)
{
    if (!c || !fin || !fin->radiance) return ESIM_AD_EINVAL;
    if (fin->pitch_elems != 0 && fin->pitch_elems < c->W) return ESIM_AD_EINVAL;
    if (c->cfg.feature_fmt == ESIM_AD_FEAT_BF16 ? !fin->features
                                                : (!fin->normal || !fin->albedo || !fin->depth))
        return ESIM_AD_EINVAL;
    if (c->sticky != ESIM_AD_OK) return ESIM_AD_ESTATE;
    DeviceGuard guard(c->device);
    esim_ad_frame staged;
    const esim_ad_frame* f = fin;
    int slot = -1;
    if (fin->on_host) {
        esim_ad_status st = stage_host_frame(c, fin, &staged, &slot);
        if (st != ESIM_AD_OK) return st;
        f = &staged;
    }
    const int t = (int)(c->t % 0x7fffffff);
    const bool adaptive_test = c->cfg.mode == ESIM_AD_ADAPTIVE && c->t > 0;
    // chunk counts and the event-pixel mask alternate by frame parity, so the
    // previous frame's writer reads its own while this frame's ingest clears these
    const int par = (int)(c->t & 1);
    if (cudaMemsetAsync(c->ctrl, 0, kCtrlPerFrameBytes, c->stream) != cudaSuccess) return ESIM_AD_ECUDA;

    IngestParams ip;
    ip.rad = f->radiance;
    ip.normal = f->normal;
    ip.albedo = f->albedo;
    ip.depth = f->depth;
    ip.feat_bf16 = reinterpret_cast<const unsigned short*>(f->features);
    ip.rad_fmt = c->cfg.radiance_fmt;
    ip.feat_fmt = c->cfg.feature_fmt;
    ip.mixed = c->mixed ? 1 : 0;
    for (int j = 0; j < 7; ++j) {
        const float fs = (c->cfg.feature_fmt == ESIM_AD_FEAT_BF16 || c->mixed) ? c->cfg.feature_scale[j] : 1.0f;
        ip.fscale[j] = fs;
        ip.inv_fscale[j] = 1.0f / fs;
    }
    ip.W = c->W;
    ip.H = c->H;
    ip.pitch = f->pitch_elems ? f->pitch_elems : c->W;
    ip.tiles_x = c->tiles_x;
    ip.slot = t % c->cfg.frames;
    ip.test = adaptive_test ? 1 : 0;
    ip.log_eps = c->cfg.log_eps;
    ip.C = c->cfg.contrast;
    ip.guard_kappa = c->cfg.guard_kappa > 0.0f ? c->cfg.guard_kappa : 0.0f;
    ip.variance = ip.guard_kappa > 0.0f ? f->variance : nullptr;
    ip.ring = c->ring;
    ip.state = c->state;
    ip.flag = c->flag;
    ip.nev = c->nev;
    ip.tile_queue = c->tile_queue;
    ip.tile_nflag = c->tile_nflag;
    ip.tile_pix = c->tile_pix;
    ip.chunk_cnt = c->chunk_cnt + par * c->n_chunks;
    ip.n_chunks = c->n_chunks;
    ip.flag_list = c->flag_list;
    ip.tile_base = c->tile_base;
    ip.ev_mask = c->ev_mask + (size_t)par * c->n_chunks * (kChunk / 32);
    ip.n_mask_words = c->n_chunks * (kChunk / 32);
    ip.n_tiles = c->n_tiles;
    ip.poll_limit = kPollLimit;
    ip.ctrl = c->ctrl;
    {
        ProfScope ps(c, 0, c->stream);
        CUtensorMap my, mf;
        cudaError_t err;
        if (c->ingest_staged && encode_frame_maps(c, f, &my, &mf)) {
            err = launch_ingest_staged(my, mf, c->ingest_map_s, ip, c->ingest_grid, c->stream);
            ++c->staged_ingests;
        } else
            err = launch_ingest(ip, c->n_tiles, c->stream);
        if (err != cudaSuccess) return ESIM_AD_ECUDA;
        c->prof_kernels += 1;
    }
    if (slot >= 0 && cudaEventRecord(c->ev_consumed[slot], c->stream) != cudaSuccess)
        return ESIM_AD_ECUDA;

    WlrParams wp;
    wp.W = c->W;
    wp.H = c->H;
    wp.r = c->cfg.radius;
    wp.T = c->cfg.frames;
    wp.t = t;
    wp.n_tau = (int)((c->t + 1) < (uint64_t)c->cfg.frames ? (c->t + 1) : (uint64_t)c->cfg.frames);
    wp.tiles_x = c->tiles_x;
    wp.n_tiles = c->n_tiles;
    wp.nbuf = c->nbuf;
    wp.dense = adaptive_test ? 0 : 1;
    wp.init = c->t == 0 ? 1 : 0;
    wp.sw = kTileX + 2 * c->cfg.radius;
    wp.sh = kTileY + 2 * c->cfg.radius;
    wp.C = c->cfg.contrast;
    wp.s_coord = (float)(kExp2Scale / c->cfg.h);
    wp.s_coord_px = (float)(kExp2Scale / ((double)c->cfg.h * c->cfg.radius));
    wp.mixed = c->mixed ? 1 : 0;
    for (int j = 0; j < 7; ++j) {
        wp.s_feat[j] = (float)(kExp2Scale / ((double)c->cfg.h * c->cfg.bandwidth[j]));
        wp.fscale[j] = c->mixed ? c->cfg.feature_scale[j] : 1.0f;
        wp.q_scale[j] = (float)((double)wp.s_feat[j] * wp.fscale[j]);
    }
    wp.ridge = c->cfg.ridge;
    wp.ring = c->ring;
    wp.state = c->state;
    wp.alpha = c->alpha;
    wp.nev = c->nev;
    wp.tile_queue = c->tile_queue;
    wp.tile_nflag = c->tile_nflag;
    wp.tile_pix = c->tile_pix;
    wp.chunk_cnt = c->chunk_cnt + par * c->n_chunks;
    wp.chunk_off = c->chunk_off;
    wp.n_chunks = c->n_chunks;
    wp.emit_events = c->t > 0 ? 1 : 0;
    wp.sparse_max = c->sparse_max;
    wp.flag_list = c->flag_list;
    wp.sparse_stage = c->sparse_stage;
    wp.tile_base = c->tile_base;
    wp.gram = c->gram;
    wp.poll_limit = c->test_withhold ? 64u : kPollLimit;
    wp.withhold_copy = c->test_withhold;
    wp.ev_mask = c->ev_mask + (size_t)par * c->n_chunks * (kChunk / 32);
    wp.ctrl = c->ctrl;
    {
        ProfScope ps(c, 1, c->stream);
        // pass 1: dense frames tile-staged over every tile; adaptive frames in one
        // launch that picks window boxes or the tile queue from the flagged total
        const int grid = wp.dense ? (c->n_tiles < c->wlr_grid ? c->n_tiles : c->wlr_grid) : c->adaptive_grid;
        if (launch_wlr(c->tmap, wp, c->mixed, grid, wp.dense ? c->smem_bytes : c->smem_adaptive, c->stream) !=
            cudaSuccess)
            return ESIM_AD_ECUDA;
        // pass 2: solve every accumulated system and emit; it follows the
        // previous frame's event writer (it sets ev_base from that frame's total)
        if (join_writer(c) != cudaSuccess ||
            launch_wlr_solve(wp, c->mixed, c->solve_grid, c->stream) != cudaSuccess)
            return ESIM_AD_ECUDA;
        c->prof_kernels += 2;
    }

    if (c->t > 0) {
        EventParams ep;
        ep.nev = c->nev;
        ep.drained = c->drained;
        ep.n_pix = (long long)c->N;
        ep.W = c->W;
        ep.n_chunks = c->n_chunks;
        ep.frame = (uint32_t)c->t;
        ep.chunk_cnt = c->chunk_cnt + par * c->n_chunks;
        ep.ev_mask = c->ev_mask + (size_t)par * c->n_chunks * (kChunk / 32);
        ep.chunk_off = c->chunk_off;
        ep.events = c->events;
        ep.capacity = c->cfg.event_capacity;
        ep.ctrl = c->ctrl;
        // on the writer stream, so that the next frame's ingest and pass 1 run
        // beside it; while profiling, on the context's stream, so that every
        // kernel is timed alone
        const bool overlap = !c->prof_on;
        if (overlap && (cudaEventRecord(c->ev_solved, c->stream) != cudaSuccess ||
                        cudaStreamWaitEvent(c->writer_stream, c->ev_solved, 0) != cudaSuccess))
            return ESIM_AD_ECUDA;
        {
            const cudaStream_t ws = overlap ? c->writer_stream : c->stream;
            ProfScope ps(c, 2, ws);
            if (launch_event_write(ep, ws) != cudaSuccess) return ESIM_AD_ECUDA;
        }
        c->last_wr = (int)(c->t % kFrameEnds);
        if (cudaEventRecord(c->ev_wr[c->last_wr], overlap ? c->writer_stream : c->stream) != cudaSuccess)
            return ESIM_AD_ECUDA;
        c->writer_pending = true;
        c->prof_kernels += 1;
    } else {
        // frame 0 writes no events: its mark is the end of its solve
        c->last_wr = 0;
        if (cudaEventRecord(c->ev_wr[0], c->stream) != cudaSuccess) return ESIM_AD_ECUDA;
    }
    if (slot >= 0) {
        // the caller may reuse its host buffers once its copies are done
        if (cudaEventSynchronize(c->ev_copied[slot]) != cudaSuccess) return ESIM_AD_ECUDA;
    }
    c->t += 1;
    return ESIM_AD_OK;
}

// Copy n event records from ring position `from` (wrapping at the buffer's
// end: at most two pieces) and record them as drained.
static esim_ad_status copy_ring(esim_ad_ctx* c, esim_ad_event* dst, uint64_t from, uint64_t n,
                                int dst_is_device, cudaStream_t s)
{
    const uint64_t cap = c->cfg.event_capacity;
    const cudaMemcpyKind k = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (n > 0) {
        const uint64_t i0 = from % cap;
        const uint64_t first = n < cap - i0 ? n : cap - i0;
        if (cudaMemcpyAsync(dst, c->events + i0, first * sizeof(esim_ad_event), k, s) != cudaSuccess ||
            (n > first &&
             cudaMemcpyAsync(dst + first, c->events, (n - first) * sizeof(esim_ad_event), k, s) != cudaSuccess))
            return ESIM_AD_ECUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return ESIM_AD_ECUDA;
    c->drained = from + n;   // the next frames' writers see it as pushed
    return ESIM_AD_OK;
}

esim_ad_status esim_ad_events(esim_ad_ctx* c, esim_ad_event* dst, uint64_t cap, uint64_t* n_out,
                              int dst_is_device)
{
    if (!c || !n_out || (cap > 0 && !dst)) return ESIM_AD_EINVAL;
    if (c->sticky != ESIM_AD_OK) return ESIM_AD_ESTATE;
    DeviceGuard guard(c->device);
    Ctrl h;
    if (sync_and_check(c, &h) != ESIM_AD_OK) return ESIM_AD_ECUDA;
    const unsigned long long total = h.ev_total - c->drained;
    if (c->sticky == ESIM_AD_EOVERFLOW) {
        *n_out = total;
        return ESIM_AD_EOVERFLOW;
    }
    if (c->sticky != ESIM_AD_OK) return c->sticky;
    *n_out = total;
    if (cap < total) return ESIM_AD_ENOSPACE;
    if (total > 0) return copy_ring(c, dst, c->drained, total, dst_is_device, c->stream);
    return ESIM_AD_OK;
}

esim_ad_status esim_ad_events_frame(esim_ad_ctx* c, uint64_t frame, esim_ad_event* dst, uint64_t cap,
                                    uint64_t* n_out, int dst_is_device)
{
    if (!c || !n_out || (cap > 0 && !dst)) return ESIM_AD_EINVAL;
    if (c->sticky != ESIM_AD_OK) return ESIM_AD_ESTATE;
    if (frame >= c->t || c->t - 1 - frame >= (uint64_t)kFrameEnds) return ESIM_AD_EINVAL;
    DeviceGuard guard(c->device);
    // wait for that frame's writer only, on the drain stream; its end mark and
    // the status word land in pinned memory
    struct {
        unsigned long long end;
        uint32_t status;
    } h = {0, 0};
    const cudaStream_t s = c->drain_stream;
    c->hmark[1] = 0;
    if (cudaStreamWaitEvent(s, c->ev_wr[frame % kFrameEnds], 0) != cudaSuccess ||
        cudaMemcpyAsync(&c->hmark[0], &c->ctrl->frame_end[frame % kFrameEnds], sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&c->hmark[1], &c->ctrl->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return ESIM_AD_ECUDA;
    h.end = c->hmark[0];
    h.status = (uint32_t)c->hmark[1];
    if (frame == 0) h.end = c->drained;   // frame 0 writes no events (and no end mark)
    if (h.status & kStatusTimeout) c->sticky = ESIM_AD_ETIMEOUT;
    else if (h.status & kStatusOverflow) c->sticky = ESIM_AD_EOVERFLOW;
    const unsigned long long n = h.end > c->drained ? h.end - c->drained : 0ull;
    if (c->sticky == ESIM_AD_EOVERFLOW) {
        *n_out = n;
        return ESIM_AD_EOVERFLOW;
    }
    if (c->sticky != ESIM_AD_OK) return c->sticky;
    *n_out = n;
    if (cap < n) return ESIM_AD_ENOSPACE;
    return n > 0 ? copy_ring(c, dst, c->drained, n, dst_is_device, s) : ESIM_AD_OK;
}

esim_ad_status esim_ad_denoised(esim_ad_ctx* c, float* alpha, uint8_t* flags, int dst_is_device)
{
    if (!c) return ESIM_AD_EINVAL;
    if (c->sticky != ESIM_AD_OK) return ESIM_AD_ESTATE;
    DeviceGuard guard(c->device);
    const cudaMemcpyKind k = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (alpha && cudaMemcpyAsync(alpha, c->alpha, c->N * sizeof(float), k, c->stream) != cudaSuccess)
        return ESIM_AD_ECUDA;
    if (flags && cudaMemcpyAsync(flags, c->flag, c->N, k, c->stream) != cudaSuccess) return ESIM_AD_ECUDA;
    if (sync_and_check(c, nullptr) != ESIM_AD_OK) return ESIM_AD_ECUDA;
    return c->sticky == ESIM_AD_OK ? ESIM_AD_OK : c->sticky;
}

esim_ad_status esim_ad_get_state(esim_ad_ctx* c, float* l_last, float* beta, float* xc)
{
    if (!c) return ESIM_AD_EINVAL;
    if (c->sticky != ESIM_AD_OK) return ESIM_AD_ESTATE;
    DeviceGuard guard(c->device);
    const size_t N = c->N;
    float4* h = (float4*)malloc(4 * N * sizeof(float4));
    if (!h) return ESIM_AD_ENOMEM;
    if (cudaMemcpyAsync(h, c->state, 4 * N * sizeof(float4), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        sync_and_check(c, nullptr) != ESIM_AD_OK) {
        free(h);
        return ESIM_AD_ECUDA;
    }
    for (size_t i = 0; i < N; ++i) {
        const float4 b0 = h[i], b1 = h[N + i], x0 = h[2 * N + i], x1 = h[3 * N + i];
        if (l_last) l_last[i] = x1.w;
        if (beta) {
            float* b = beta + 7 * i;
            b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
            b[4] = b1.x; b[5] = b1.y; b[6] = b1.z;
        }
        if (xc) {
            float* x = xc + 7 * i;
            x[0] = x0.x; x[1] = x0.y; x[2] = x0.z; x[3] = x0.w;
            x[4] = x1.x; x[5] = x1.y; x[6] = x1.z;
        }
    }
    free(h);
    return ESIM_AD_OK;
}

esim_ad_status esim_ad_set_state(esim_ad_ctx* c, const float* l_last, const float* beta, const float* xc)
{
    if (!c) return ESIM_AD_EINVAL;
    if (c->sticky != ESIM_AD_OK) return ESIM_AD_ESTATE;
    DeviceGuard guard(c->device);
    const size_t N = c->N;
    float4* h = (float4*)malloc(4 * N * sizeof(float4));
    if (!h) return ESIM_AD_ENOMEM;
    if (cudaMemcpyAsync(h, c->state, 4 * N * sizeof(float4), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        sync_stream(c) != cudaSuccess) {
        free(h);
        return ESIM_AD_ECUDA;
    }
    for (size_t i = 0; i < N; ++i) {
        if (l_last) h[3 * N + i].w = l_last[i];
        if (beta) {
            const float* b = beta + 7 * i;
            h[i] = make_float4(b[0], b[1], b[2], b[3]);
            h[N + i].x = b[4]; h[N + i].y = b[5]; h[N + i].z = b[6];
        }
        if (xc) {
            const float* x = xc + 7 * i;
            const float lw = h[3 * N + i].w;
            h[2 * N + i] = make_float4(x[0], x[1], x[2], x[3]);
            h[3 * N + i] = make_float4(x[4], x[5], x[6], lw);
        }
        // keep sigma = beta . x^c consistent with the stored model
        const float4 x0 = h[2 * N + i], x1 = h[3 * N + i];
        h[N + i].w = dot7(h[i], h[N + i], x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z);
    }
    esim_ad_status st = ESIM_AD_OK;
    if (cudaMemcpyAsync(c->state, h, 4 * N * sizeof(float4), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        sync_stream(c) != cudaSuccess)
        st = ESIM_AD_ECUDA;
    free(h);
    return st;
}

esim_ad_status esim_ad_reset(esim_ad_ctx* c)
{
    if (!c) return ESIM_AD_EINVAL;
    DeviceGuard guard(c->device);
    if (sync_stream(c) != cudaSuccess) return ESIM_AD_ECUDA;
    if (cudaMemsetAsync(c->ctrl, 0, sizeof(Ctrl), c->stream) != cudaSuccess ||
        sync_stream(c) != cudaSuccess)
        return ESIM_AD_ECUDA;
    c->t = 0;
    c->drained = 0;
    c->staged_ingests = 0;
    c->sticky = ESIM_AD_OK;
    return ESIM_AD_OK;
}

esim_ad_status esim_ad_stats_get(esim_ad_ctx* c, esim_ad_stats* out)
{
    if (!c || !out) return ESIM_AD_EINVAL;
    DeviceGuard guard(c->device);
    Ctrl h;
    if (sync_and_check(c, &h) != ESIM_AD_OK) return ESIM_AD_ECUDA;
    out->frames = c->t;
    out->regressions = h.regressions;
    out->events = h.ev_cum;
    out->pixels = c->N;
    out->fp64_solves = h.fp64_solves;
    out->staged_ingests = c->staged_ingests;
    return ESIM_AD_OK;
}

esim_ad_status esim_ad_profile_enable(esim_ad_ctx* c, int on)
{
    if (!c) return ESIM_AD_EINVAL;
    DeviceGuard guard(c->device);
    if (sync_stream(c) != cudaSuccess) return ESIM_AD_ECUDA;
    c->prof_on = on != 0;
    c->prof_used = 0;
    c->prof_kernels = 0;
    return ESIM_AD_OK;
}

esim_ad_status esim_ad_profile_get(esim_ad_ctx* c, esim_ad_profile* out)
{
    if (!c || !out) return ESIM_AD_EINVAL;
    DeviceGuard guard(c->device);
    Ctrl h;
    if (sync_and_check(c, &h) != ESIM_AD_OK) return ESIM_AD_ECUDA;
    memset(out, 0, sizeof(*out));
    for (size_t k = 0; k < c->prof_used; ++k) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, c->prof_events[2 * k], c->prof_events[2 * k + 1]) != cudaSuccess)
            return ESIM_AD_ECUDA;
        out->launches[c->prof_class[k]] += 1;
        out->ms[c->prof_class[k]] += ms;
    }
    out->kernels = c->prof_kernels;
    out->neighbours = h.neighbours;
    out->regressions = h.regressions;
    return ESIM_AD_OK;
}

void esim_ad_destroy(esim_ad_ctx* c)
{
    if (!c) return;
    {
        DeviceGuard guard(c->device);
        sync_stream(c);
        if (c->writer_stream) cudaStreamSynchronize(c->writer_stream);
        if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
        release(c);
    }
    delete c;
}

}  // extern "C"
