// Pass 1 in window-box form and the per-record solve, shared by the
// single-sequence regression (wlr.cu) and the batching form (batch.cu).
#pragma once

#include "internal.h"
#include "ptx.cuh"
#include "sparse_stage.cuh"
#include "wlr_math.cuh"

namespace esim {
namespace {

// The part of a sequence's parameters that varies between the sequences of a
// batch; a window-box item belongs to one sequence.
struct SeqView {
    int W, H, t, T, n_tau;
    const void* ring;
};

// One sequence: list entries are pixel indices.
struct SingleSeq {
    const WlrParams* p;
    __device__ __forceinline__ SeqView view(uint32_t) const { return {p->W, p->H, p->t, p->T, p->n_tau, p->ring}; }
    __device__ __forceinline__ uint32_t pixel(uint32_t e) const { return e; }
    __device__ __forceinline__ const WlrParams& params(uint32_t) const { return *p; }
};

constexpr int kSolveThreads = 128;

// Sum each pixel's partial sums over its g lanes through the warp's (idle)
// box buffer and store the Gram records.  Pixel q of the pass owns lanes
// q g .. q g + g - 1 and record entry0 + q.  Every lane writes its 66 sums as
// one row (pitch 67 floats, so the 32 rows of a column sit in distinct
// banks); the lanes then split the records' slots, consecutive lanes taking
// consecutive slots, and each adds its column over the pixel's rows in lane
// order.  Fewer instructions than a shuffle tree (3-5 levels of 65 shuffles
// and adds), and the stores come out coalesced.
constexpr int kRowPitch = 67;
static_assert(32 * kRowPitch * 4 <= kBoxBytes, "partial sums fit a box buffer");

__device__ __forceinline__ void store_records(const AccP& a, float* rows, float* __restrict__ gram, uint32_t entry0,
                                              int npix, int g)
{
    const int lane = threadIdx.x & 31;
    float v[kGramStride];
    accp_values(a, v);
    __syncwarp();   // every lane is past its reads of the box
#pragma unroll
    for (int s = 0; s < kGramFloats; ++s) rows[lane * kRowPitch + s] = v[s];
    __syncwarp();
    for (int k = lane; k < npix * kGramStride; k += 32) {
        const int q = k / kGramStride, s = k - q * kGramStride;
        float sum = 0.0f;
        if (s < kGramFloats) {
            const float* col = rows + q * g * kRowPitch + s;
            for (int i = 0; i < g; ++i) sum += col[i * kRowPitch];
        }
        gram[(size_t)(entry0 + (uint32_t)q) * kGramStride + s] = sum;
    }
    __syncwarp();   // the buffer is free for the next item's copies
}

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

// Window-box form of pass 1 (the solve kernel solves and emits).  Items are
// kItem consecutive list entries (4, 2 or 1: 8, 16 or 32 lanes per pixel).
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
template <int kItem, bool kMixed, class Src>
__device__ __forceinline__ void sparse_body(const WlrParams& p, const Src& src)
{
    extern __shared__ __align__(128) unsigned char sm[];
    const BoxLayout L = box_layout(p.r);
    __shared__ unsigned long long s_pairs, s_pix;
    const int side = 2 * p.r + 1, nq = side * side;
    const float spx = p.s_coord_px;
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
            base = atomicAdd(&p.ctrl->work_next, (uint32_t)kItem);
            if (base >= tail0) {
                base = tail0 + atomicAdd(&p.ctrl->tail_next, 1u);
                single = 1;
            }
        }
        base = __shfl_sync(0xffffffffu, base, 0);
        single = __shfl_sync(0xffffffffu, single, 0);
        if (base >= n_list) break;
        const int lim = single ? 1 : kItem;
        const uint32_t e4 = ((lane & 3) < lim) ? p.flag_list[base + (lane & 3)] : kListPad;
        // an item's m real entries come first (padding closes a tile's run);
        // 8 lanes per pixel for m = 3, 4, 16 for m = 2, 32 for m = 1
        const int m = __popc(__ballot_sync(0xffffffffu, e4 != kListPad) & 0xfu);
        if (m == 0) continue;   // a padding entry of the tail
        // the item's sequence (every entry of an item belongs to one: items never
        // straddle a tile's run, and entry 0 is real)
        const SeqView sv = src.view(__shfl_sync(0xffffffffu, e4, 0));
        const size_t N = (size_t)sv.W * sv.H;
        const float4* ringf = reinterpret_cast<const float4*>(sv.ring);
        const uint4* ringm = reinterpret_cast<const uint4*>(sv.ring);
        const int slot_t = sv.t % sv.T;
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
            const uint32_t px0 = src.pixel(__shfl_sync(0xffffffffu, e4, grp0));
            const int x0 = (int)(px0 % (uint32_t)sv.W), y0 = (int)(px0 / (uint32_t)sv.W);
            const int ux0 = __reduce_min_sync(0xffffffffu, act0 ? max(x0 - p.r, 0) : 0x7fffffff);
            const int uy0 = __reduce_min_sync(0xffffffffu, act0 ? max(y0 - p.r, 0) : 0x7fffffff);
            const int ux1 = __reduce_max_sync(0xffffffffu, act0 ? min(x0 + p.r, sv.W - 1) : -1);
            const int uy1 = __reduce_max_sync(0xffffffffu, act0 ? min(y0 + p.r, sv.H - 1) : -1);
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
        const uint32_t pix = active ? src.pixel(pix_e) : 0u;
        const uint32_t entry = base + (uint32_t)(split ? part : grp);
        const int cx = (int)(pix % (uint32_t)sv.W), cy = (int)(pix / (uint32_t)sv.W);
        const int dxlo = max(-p.r, -cx), dxhi = min(p.r, sv.W - 1 - cx);
        const int dylo = max(-p.r, -cy), dyhi = min(p.r, sv.H - 1 - cy);
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
        // the centre's features (frame t): from the ring (windows read through
        // L1) or from the first staged box, once it has landed
        PairConst kc;
        auto centre = [&](const uint4 vm, const float4 c0, const float4 c1) {
            float c[7];
            if (kMixed) {
                float yc;
                unpack_mixed(vm, yc, c);
            } else {
                c[0] = c0.y; c[1] = c0.z; c[2] = c0.w; c[3] = c1.x; c[4] = c1.y; c[5] = c1.z; c[6] = c1.w;
            }
            float cf[7];
#pragma unroll
            for (int j = 0; j < 7; ++j) cf[j] = c[j] * sf[j];
            kc = pair_const(sf, cf);
        };
        if (mode == 0 && active) {
            if (kMixed)
                centre(__ldg(ringm + (size_t)slot_t * N + pix), make_float4(0, 0, 0, 0), make_float4(0, 0, 0, 0));
            else
                centre(make_uint4(0, 0, 0, 0), __ldg(ringf + (size_t)(2 * slot_t) * N + pix),
                       __ldg(ringf + (size_t)(2 * slot_t + 1) * N + pix));
        }
        accp_zero(acc);
        // Copy frame k of the box into half b (mode 2) or the whole buffer
        // (mode 1).  Every lane is past its reads of that region first.
        auto issue = [&](int b, int k) {
            __syncwarp();
            fence_proxy_async_smem();
            if (p.withhold_copy && first_item && k == 0) return;   // test: this phase never completes
            const int slot = (sv.t - k) % sv.T;
            const uint32_t rowb = (uint32_t)bw * 16u;
            if (lane == 0) mbar_arrive_expect_tx(&bar[b], (uint32_t)bh * rowb * (kMixed ? 1u : 2u));
            __syncwarp();
            if (lane < bh) {
                const size_t gi = (size_t)(by0 + lane) * sv.W + bx0;
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
        for (int k = 0; k < sv.n_tau; ++k) {
            if (mode) {
                const int b = mode == 2 ? (k & 1) : 0;
                const bool ahead = mode == 2 && k + 1 < sv.n_tau;
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
                if (k == 0 && active) {   // frame t: the centre record is in this box
                    const int ci = (cy - by0) * P + (cx - bx0);
                    if (kMixed)
                        centre(reinterpret_cast<const uint4*>(buf)[ci], make_float4(0, 0, 0, 0), make_float4(0, 0, 0, 0));
                    else
                        centre(make_uint4(0, 0, 0, 0), reinterpret_cast<const float4*>(buf)[ci],
                               reinterpret_cast<const float4*>(buf + kBoxBytes / 2)[ci]);
                }
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
                if (mode == 1 && k + 1 < sv.n_tau) issue(0, k + 1);
            } else if (active) {
                // box too large for the buffer: read the windows through L1
                const int slot = (sv.t - k) % sv.T;
                const float4* __restrict__ R0 = ringf + (size_t)(2 * slot) * N + pix;
                const float4* __restrict__ R1 = ringf + (size_t)(2 * slot + 1) * N + pix;
                const uint4* __restrict__ RM = ringm + (size_t)slot * N + pix;
                const int nvalid = nx * ny;
                int ox = dxlo + sub % nx;
                int oy = dylo + sub / nx;
#pragma unroll 1
                for (int q = sub; q < nvalid; q += g) {
                    const float u1 = (float)ox * spx, u2 = (float)oy * spx;
                    const int d = oy * sv.W + ox;
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
        store_records(acc, reinterpret_cast<float*>(wbuf), p.gram, split ? base + (uint32_t)part : base,
                      split ? 1 : m, g);
        if (active && sub == 0) {
            atomicAdd(&s_pairs, (unsigned long long)(nx * ny * sv.n_tau));
            atomicAdd(&s_pix, 1ull);
        }
        }   // passes
        if (timed_out) break;
    }
    __syncthreads();
    finish(p, s_pairs, s_pix, 0ull, timed_out, false);
}

// Solve and emit every Gram record of the frame (entries [0, n) of the
// flagged list, or every pixel when p.dense): one thread per record.  Mixed
// form: systems whose condition estimate exceeds 1e6 are set aside and, after
// each pass of the block, re-accumulated by one warp each with compensated
// sums and solved in FP64.  Returns the block's count of such systems.
template <bool kMixed, class Src>
__device__ __forceinline__ unsigned long long solve_records(const WlrParams& p, const Src& src, uint32_t n)
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
    float s2[NZ];
    s2[0] = 0.0f;
    s2[1] = p.s_coord * p.s_coord;
    s2[2] = s2[1];
#pragma unroll
    for (int j = 0; j < 7; ++j) s2[3 + j] = p.s_feat[j] * p.s_feat[j];
    const uint32_t stride = gridDim.x * kSolveThreads;
    for (uint32_t b0 = blockIdx.x * kSolveThreads; b0 < n; b0 += stride) {   // same trip count in the block
        const uint32_t e = b0 + threadIdx.x;
        uint32_t v = kListPad;
        if (e < n) v = p.dense ? e : p.flag_list[e];
        bool ill = false;
        if (v != kListPad) {
            const WlrParams& sp = src.params(v);
            const uint32_t pix = src.pixel(v);
            const float* rec = p.gram + (size_t)e * kGramStride;
            float theta[NZ];
            if (kMixed) {
                ill = !solve_refined_rec(rec, s2, p.ridge, theta);
            } else {
                Acc acc;
                gram_load(rec, acc);
                solve(acc, s2, p.ridge, theta);
            }
            if (!ill) emit<kMixed>(sp, (int)(pix % (uint32_t)sp.W), (int)(pix / (uint32_t)sp.W), theta);
            else s_ill[atomicAdd(&s_nill, 1)] = v;
        }
        if (kMixed && __syncthreads_or(ill)) {
            const int nill = s_nill;
            for (int i = (int)(threadIdx.x >> 5); i < nill; i += kSolveThreads / 32)
                refine_fp64<kMixed>(src.params(s_ill[i]), src.pixel(s_ill[i]), s2, s_sys[threadIdx.x >> 5]);
            __syncthreads();
            if (threadIdx.x == 0) {
                s_fp64 += (unsigned long long)nill;
                s_nill = 0;
            }
            __syncthreads();
        }
    }
    __syncthreads();
    return s_fp64;
}

}  // namespace
}  // namespace esim
