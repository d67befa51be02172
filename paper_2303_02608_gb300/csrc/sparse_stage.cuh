// Shared-memory window boxes of the sparse regression kernels (the
// single-sequence kernel and the batched one): per-warp buffer geometry and
// the dynamic shared-memory layout.
#pragma once

#include "internal.h"

namespace esim {

constexpr int kSparsePerWarp = 4;                  // list entries per work item (one warp)
constexpr uint32_t kListPad = 0xffffffffu;          // padding entry of the flagged list

// Window boxes of the single-sequence sparse regression: per warp one region
// of kBoxBytes, used either as two halves (double buffering over the frames
// of the temporal window: the copy of frame k+1 lands while frame k is
// summed) or whole (one frame at a time).  Rows of a box are kept at a fixed
// pitch so that one table of window offsets serves every box of that pitch.
//   mixed ring (16-byte records): halves of 20 x 20 records, whole 32 x 25
//   FP32 ring (two 16-byte half-planes): whole only, 20 x 20 per half-plane
constexpr int kBoxBytes = 12800;
constexpr int kPitchSmall = 20, kRowsSmall = 20;
constexpr int kPitchLarge = 32, kRowsLarge = 25;
constexpr int kBoxWarps = kTilePix / 32;

struct BoxLayout {
    int tab_small, tab_large, bar_off, buf_off, total;
};

// [table, pitch 20][table, pitch 32][mbarriers: 2 per warp][per-warp boxes]
__host__ __device__ inline BoxLayout box_layout(int r)
{
    const int side = 2 * r + 1, nq = side * side;
    BoxLayout L;
    L.tab_small = 0;
    L.tab_large = nq * 16;
    L.bar_off = 2 * nq * 16;
    L.buf_off = (L.bar_off + kBoxWarps * 2 * 8 + 127) & ~127;
    L.total = L.buf_off + kBoxWarps * kBoxBytes;
    return L;
}

}  // namespace esim
