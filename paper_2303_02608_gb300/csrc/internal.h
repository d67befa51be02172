// Internal declarations shared by the CUDA translation units of libesim_ad.
// Nothing here is part of the public ABI (include/esim_ad.h).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "esim_ad.h"

namespace esim {

// Pixel tile of one CTA in the ingest/test and regression kernels: 32 x 8
// pixels, one warp per tile row, so a warp's loads of a ring row are one
// contiguous 512-byte segment per half-plane.
constexpr int kTileX = 32;
constexpr int kTileY = 8;
constexpr int kTilePix = kTileX * kTileY;  // 256 threads per CTA
constexpr int kChunk = 2048;               // pixels per event-scan chunk (256 x 8)
constexpr int kMaxRadius = 15;
constexpr int kMaxFrames = 16;

// Sticky device status bits.
constexpr uint32_t kStatusOverflow = 1u;
constexpr uint32_t kStatusTimeout = 2u;

// Device control block.  The first 16 bytes are cleared before every frame.
struct Ctrl {
    uint32_t tile_count;            // active tiles queued by the test kernel
    uint32_t chunk_done;            // ticket of the event-count kernel
    uint32_t work_next;             // next work item of the persistent regression
    uint32_t flag_total;            // pixels flagged by the test kernel this frame
    uint32_t list_len;              // flagged-list length: each tile's run padded to a multiple of 4
    uint32_t tail_next;             // sparse regression: next single entry of the list's tail
    unsigned long long ev_total;    // record positions used: since init/reset (simulator: the event
                                    // buffer is a ring), or since the last drain (batching form)
    unsigned long long ev_cum;      // events since init/reset
    unsigned long long regressions; // pixels regressed since init/reset
    unsigned long long neighbours;  // (pixel, neighbour) pairs regressed
    unsigned long long fp64_solves; // mixed form: systems re-solved in FP64
    uint32_t status;                // sticky kStatus* bits
    uint32_t pad2;
    unsigned long long ev_base;     // ev_total before this frame's events (set by the solve kernel)
    unsigned long long frame_end[8];  // simulator: ev_total after frame f's writer, at f % 8
};
constexpr int kFrameEnds = 8;
constexpr size_t kCtrlPerFrameBytes = 24;   // the per-frame counters above ev_total
static_assert(offsetof(Ctrl, ev_total) == kCtrlPerFrameBytes, "per-frame part of Ctrl");
// Largest |signed event count| of one pixel in one frame: a 2048-pixel chunk then
// sums to at most 2^30 events, within the 32-bit chunk counts.
constexpr int kMaxCountPerPixel = 1 << 19;
constexpr uint32_t kStatusCountRange = 4u;   // a count map held |count| > kMaxCountPerPixel
constexpr size_t kGramRecordBytes = 272;   // one Gram record: 66 sums padded to 68 floats
constexpr uint32_t kPollLimit = 1u << 24;   // default bound on an mbarrier wait (polls)

// Ring of the last T frames.  FP32 form: float4 planes [2T][H][W]; plane
// 2*slot holds (y, normal xyz), plane 2*slot+1 holds (depth, albedo rgb).
// Mixed form: one 16-byte record per pixel, planes [T][H][W] of uint4
//   x = y (FP16) | n_x (BF16) << 16,  y = n_y | n_z << 16,
//   z = depth | a_r << 16,            w = a_g | a_b << 16
// where each BF16 feature q_j stores x_j / feature_scale_j.

__host__ __device__ __forceinline__ uint4 pack_mixed(unsigned short yh, const unsigned short (&q)[7])
{
    return make_uint4((uint32_t)yh | ((uint32_t)q[0] << 16), (uint32_t)q[1] | ((uint32_t)q[2] << 16),
                      (uint32_t)q[3] | ((uint32_t)q[4] << 16), (uint32_t)q[5] | ((uint32_t)q[6] << 16));
}

// Unpack a mixed record: y, then the seven stored feature values (still divided
// by their scales).  BF16 -> FP32 is exact (a 16-bit shift).
__device__ __forceinline__ void unpack_mixed(const uint4 v, float& y, float (&q)[7])
{
    y = __half2float(__ushort_as_half((unsigned short)(v.x & 0xffffu)));
    q[0] = __uint_as_float(v.x & 0xffff0000u);
    q[1] = __uint_as_float(v.y << 16);
    q[2] = __uint_as_float(v.y & 0xffff0000u);
    q[3] = __uint_as_float(v.z << 16);
    q[4] = __uint_as_float(v.z & 0xffff0000u);
    q[5] = __uint_as_float(v.w << 16);
    q[6] = __uint_as_float(v.w & 0xffff0000u);
}
// Model state: float4 planes [4][H][W]:
//   0: beta (normal xyz, depth)   1: beta (albedo rgb), sigma = beta . x^c
//   2: x^c (normal xyz, depth)    3: x^c (albedo rgb), L_last
// The test kernel reads planes 0-1 only: beta^T (x^c - xhat) = sigma - beta . xhat.

// beta . x over the seven features, in one fixed fma order so that the value
// stored at an event and the value recomputed by the test agree bit for bit
// when the features have not moved.
__host__ __device__ __forceinline__ float dot7(const float4 b0, const float4 b1, float n0, float n1,
                                               float n2, float d, float a0, float a1, float a2)
{
    float s = b0.x * n0;
    s = fmaf(b0.y, n1, s);
    s = fmaf(b0.z, n2, s);
    s = fmaf(b0.w, d, s);
    s = fmaf(b1.x, a0, s);
    s = fmaf(b1.y, a1, s);
    s = fmaf(b1.z, a2, s);
    return s;
}

struct IngestParams {
    const void* rad;       // [C][H][W] float32, or [H][W] FP16 log brightness
    const float* normal;   // [3][H][W] (FEAT_F32)
    const float* albedo;   // [3][H][W] (FEAT_F32)
    const float* depth;    // [H][W]    (FEAT_F32)
    const unsigned short* feat_bf16;  // [7][H][W] BF16 bits (FEAT_BF16)
    int rad_fmt;           // ESIM_AD_LUMA_F32 | RGB_F32 | LOGLUMA_F16
    int feat_fmt;          // ESIM_AD_FEAT_F32 | FEAT_BF16
    int mixed;             // ring in the mixed form
    float fscale[7];       // feature_scale
    float inv_fscale[7];
    int W, H, tiles_x;
    long long pitch;       // input row pitch in elements (>= W)
    int slot;              // ring slot of this frame
    int test;              // 1: Proposition-1 test; 0: flag every pixel
    float log_eps, C;
    float guard_kappa;     // > 0: also flag |y - L_last| >= C + guard_kappa * sigma_y
    const float* variance; // [H][W] Var[Y] for the guard, or NULL (sigma_y = 0)
    void* ring;
    const float4* state;
    uint8_t* flag;
    int32_t* nev;
    uint32_t* tile_queue;
    int32_t* tile_nflag;
    uint8_t* tile_pix;
    uint32_t* chunk_cnt;   // per event chunk, cleared here for the regression's counts
    int n_chunks;
    uint32_t* flag_list;   // frame-wide list of flagged pixel indices: each tile's run, in raster
                           // order, padded with 0xffffffff to a multiple of 4 entries
    uint32_t* tile_base;   // position of each queued tile's run in flag_list
    // one bit per pixel, set by the solve where the pixel emits; cleared here
    // (nullptr: the count map itself is cleared instead, for a dense writer)
    uint32_t* ev_mask = nullptr;
    int n_mask_words = 0;
    int n_tiles = 0;             // staged ingest: tiles of the frame
    uint32_t poll_limit = 0;     // staged ingest: bound of each mbarrier wait
    Ctrl* ctrl;
};

struct WlrParams {
    int W, H, r, T, t, n_tau, tiles_x, n_tiles;
    int mixed;             // ring in the mixed form (FP16/BF16), refined + FP64-fallback solve
    int nbuf;              // staged frames in flight per CTA (2 or 3)
    int dense;             // 1: every tile and pixel; 0: tiles from the queue
    int init;              // 1: frame 0 (initialise models, no events)
    int sw, sh;            // staged tile: (32 + 2r) x (8 + 2r) pixels
    float C;
    float s_coord_px;      // regressor scale of a one-pixel coordinate offset
    float s_coord;         // regressor scale of the coordinate unit (offset / r)
    float s_feat[7];       // regressor scale per feature: k / (h b_j)
    float q_scale[7];      // mixed form: regressor scale per stored value, s_feat * feature_scale
    float fscale[7];       // mixed form: feature_scale
    float ridge;
    const void* ring;
    float4* state;
    float* alpha;
    int32_t* nev;
    const uint32_t* tile_queue;
    const int32_t* tile_nflag;
    const uint8_t* tile_pix;
    uint32_t* chunk_cnt;             // events per 2048-pixel chunk (atomically summed)
    unsigned long long* chunk_off;   // exclusive offsets, written by the last CTA
    int n_chunks;
    int emit_events;                 // 0 on frame 0 (no events)
    uint32_t sparse_max;             // queue mode: at most this many flagged pixels -> sparse kernel
    const uint32_t* flag_list;       // flagged pixel indices per tile, each run padded to 4 entries
    int sparse_stage;                // sparse kernel: 1 stage window boxes in shared memory, 0 read via L1
    const uint32_t* tile_base;       // position of each queued tile's run in flag_list
    float* gram;                     // Gram records [entries][68]: entry = pixel index (dense) or
                                     // position in flag_list (adaptive frames)
    uint32_t poll_limit;             // bound on each mbarrier wait of the sparse kernel (polls)
    int withhold_copy;               // test only: the sparse kernel never issues its first box copy
    uint32_t* ev_mask = nullptr;     // bit per pixel, set where the pixel emits (nullptr: none kept)
    Ctrl* ctrl;
};

struct EventParams {
    const int32_t* nev;
    const uint32_t* ev_mask = nullptr;   // bit per pixel with events (nullptr: read every count)
    unsigned long long drained = 0;      // ring positions drained when the frame was pushed
    long long n_pix;
    int W;
    int n_chunks;
    uint32_t frame;
    uint32_t* chunk_cnt;
    unsigned long long* chunk_off;
    esim_ad_event* events;
    unsigned long long capacity;
    Ctrl* ctrl;
};

cudaError_t launch_ingest(const IngestParams& p, int n_tiles, cudaStream_t s);
// Staged ingest of FP16 log brightness + BF16 feature frames (precision form):
// persistent CTAs, each tile's inputs and model landed by TMA a tile ahead.
// map_y: {W, H} u16, map_f: {W, H, 7} u16, map_s: the model state as {4W, H, 4}
// f32; boxes {32, 8}, {32, 8, 7}, {128, 8, 2}.
constexpr int kIngestStageBytes = 12288;
constexpr int kIngestStages = 2;
cudaError_t launch_ingest_staged(const CUtensorMap& map_y, const CUtensorMap& map_f, const CUtensorMap& map_s,
                                 const IngestParams& p, int grid, cudaStream_t s);
int ingest_staged_grid(int sms);

// Autotuning cache (tune_cache.cu): value for key, or 0 if none.
int tune_cache_lookup(const char* key);
void tune_cache_store(const char* key, int value);
// Regression pass 1: dense frames (every tile) and adaptive frames (one launch
// choosing on the device between the sparse window-box form and the
// tile-staged queue form); the adaptive kernel's shared memory is the larger
// of the two forms'.
cudaError_t wlr_prepare(int smem_dense, int smem_adaptive, bool mixed);
size_t wlr_smem_bytes(int r, bool mixed, int max_smem_per_sm, int* nbuf);
int wlr_grid(int smem_bytes, int num_sms, bool mixed, bool adaptive);
int wlr_sparse_smem(int r, bool mixed);
cudaError_t launch_wlr(const CUtensorMap& tmap, const WlrParams& p, bool mixed, int grid,
                       int smem_bytes, cudaStream_t s);
cudaError_t launch_wlr_solve(const WlrParams& p, bool mixed, int grid, cudaStream_t s);
int wlr_solve_grid(int num_sms);
cudaError_t launch_events(const EventParams& p, cudaStream_t s);
cudaError_t launch_event_write(const EventParams& p, cudaStream_t s);

}  // namespace esim
