// Shared-memory window boxes of the sparse regression kernels (the
// single-sequence kernel and the batched one): per-warp buffer geometry and
// the dynamic shared-memory layout.
#pragma once

#include "internal.h"

namespace esim {

template <bool kMixed>
struct SparseStage;
template <>
struct SparseStage<true> {   // one 16-byte record per pixel
    static constexpr int pitch = 32, rows = 24, rec = 16;
};
template <>
struct SparseStage<false> {  // two float4 half-planes per pixel
    static constexpr int pitch = 20, rows = 19, rec = 32;
};
constexpr int kSparsePerWarp = 4;                  // list entries per work item (one warp)
constexpr uint32_t kListPad = 0xffffffffu;          // padding entry of the flagged list

struct SparseLayout {
    int buf_off, buf_bytes, total;
};

// window table [(2r+1)^2] float4 (buffer offset, u_dx, u_dy, -(u_dx^2 + u_dy^2)) | 8 warp buffers
__host__ __device__ inline SparseLayout sparse_layout(int r, bool mixed)
{
    const int side = 2 * r + 1, nq = side * side;
    const int pitch = mixed ? SparseStage<true>::pitch : SparseStage<false>::pitch;
    const int rows = mixed ? SparseStage<true>::rows : SparseStage<false>::rows;
    const int rec = mixed ? SparseStage<true>::rec : SparseStage<false>::rec;
    const bool stage = side <= pitch && side <= rows;
    SparseLayout L;
    L.buf_bytes = stage ? pitch * rows * rec : 0;
    L.buf_off = nq * 16;
    L.total = L.buf_off + (kTilePix / 32) * L.buf_bytes;
    return L;
}

}  // namespace esim
