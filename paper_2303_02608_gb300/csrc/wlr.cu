// Weighted local regression (Eqs. 3-5) with fused event emission (Eq. 1).
//
// One CTA owns a 32x8 pixel tile.  For each frame tau of the temporal window
// t-T+1..t it stages the tile plus an r-pixel halo of that frame's ring slot
// ((32+2r) x (8+2r) pixels x 2 float4 half-planes) in shared memory with one
// 4-D TMA load, double-buffered over tau on two mbarriers.  Pixels outside the
// image arrive zero-filled and are never read: each centre's offset range is
// clipped to the image instead.
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
#include "internal.h"
#include "ptx.cuh"

namespace esim {

namespace {

constexpr int NZ = 10;  // z = (1, u_dx, u_dy, u_feat[7])
constexpr int NG = NZ * (NZ + 1) / 2;

__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

struct Acc {
    float G[NG];
    float B[NZ];
};

// One neighbour: y and the raw features (h0 = y, normal xyz; h1 = depth, albedo rgb).
__device__ __forceinline__ void accumulate(Acc& a, const float4 h0, const float4 h1, float u1,
                                           float u2, float en0, const float (&sf)[7],
                                           const float (&cf)[7])
{
    float u[NZ];
    u[0] = 1.0f;
    u[1] = u1;
    u[2] = u2;
    u[3] = fmaf(h0.y, sf[0], -cf[0]);
    u[4] = fmaf(h0.z, sf[1], -cf[1]);
    u[5] = fmaf(h0.w, sf[2], -cf[2]);
    u[6] = fmaf(h1.x, sf[3], -cf[3]);
    u[7] = fmaf(h1.y, sf[4], -cf[4]);
    u[8] = fmaf(h1.z, sf[5], -cf[5]);
    u[9] = fmaf(h1.w, sf[6], -cf[6]);
    float en = en0;  // -(u1^2 + u2^2)
#pragma unroll
    for (int j = 3; j < NZ; ++j) en = fmaf(-u[j], u[j], en);
    const float w = ex2_approx(en);
    const float wy = w * h0.x;
    float wu[NZ];
    wu[0] = w;
#pragma unroll
    for (int j = 1; j < NZ; ++j) wu[j] = w * u[j];
    a.G[0] += w;
#pragma unroll
    for (int i = 1; i < NZ; ++i) {
        a.G[tri(i, 0)] += wu[i];
#pragma unroll
        for (int j = 1; j <= i; ++j) a.G[tri(i, j)] = fmaf(wu[i], u[j], a.G[tri(i, j)]);
    }
    a.B[0] += wy;
#pragma unroll
    for (int i = 1; i < NZ; ++i) a.B[i] = fmaf(wy, u[i], a.B[i]);
}

// Ridge, Jacobi equilibration and Cholesky solve of the packed 10x10 system.
// Returns theta in the scaled regressor basis.
__device__ __forceinline__ void solve(Acc& a, const float (&s2)[NZ], float ridge,
                                      float (&theta)[NZ])
{
    const float W = a.G[0];
#pragma unroll
    for (int j = 1; j < NZ; ++j) a.G[tri(j, j)] = fmaf(ridge * W, s2[j], a.G[tri(j, j)]);
    float dsc[NZ];
#pragma unroll
    for (int i = 0; i < NZ; ++i) dsc[i] = rsqrtf(a.G[tri(i, i)]);
#pragma unroll
    for (int i = 0; i < NZ; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) a.G[tri(i, j)] *= dsc[i] * dsc[j];
        a.B[i] *= dsc[i];
    }
    float inv[NZ];
#pragma unroll
    for (int j = 0; j < NZ; ++j) {
        float s = a.G[tri(j, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) s = fmaf(-a.G[tri(j, k)], a.G[tri(j, k)], s);
        s = fmaxf(s, 1e-20f);
        const float l = sqrtf(s);
        inv[j] = 1.0f / l;
#pragma unroll
        for (int i = j + 1; i < NZ; ++i) {
            float v = a.G[tri(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) v = fmaf(-a.G[tri(i, k)], a.G[tri(j, k)], v);
            a.G[tri(i, j)] = v * inv[j];
        }
    }
    float z[NZ];
#pragma unroll
    for (int i = 0; i < NZ; ++i) {
        float v = a.B[i];
#pragma unroll
        for (int k = 0; k < i; ++k) v = fmaf(-a.G[tri(i, k)], z[k], v);
        z[i] = v * inv[i];
    }
#pragma unroll
    for (int i = NZ - 1; i >= 0; --i) {
        float v = z[i];
#pragma unroll
        for (int k = i + 1; k < NZ; ++k) v = fmaf(-a.G[tri(k, i)], theta[k], v);
        theta[i] = v * inv[i];
    }
#pragma unroll
    for (int i = 0; i < NZ; ++i) theta[i] *= dsc[i];
}

}  // namespace

template <bool kDense>
__global__ void __launch_bounds__(kTilePix, 2)
    wlr_kernel(const __grid_constant__ CUtensorMap tmap, const WlrParams p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations must be 128-byte aligned; the allocation has 128 bytes of slack
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    const int plane = p.sw * p.sh;                      // float4 per half-plane
    const uint32_t stage_bytes = (uint32_t)(2 * plane * 16);
    const int buf_bytes = (int)((stage_bytes + 127u) & ~127u);
    float4* const buf0 = reinterpret_cast<float4*>(smem);
    float4* const buf1 = reinterpret_cast<float4*>(smem + buf_bytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * buf_bytes);

    uint32_t tile;
    int npix;
    if (kDense) {
        tile = blockIdx.x;
        npix = kTilePix;
    } else {
        if (blockIdx.x >= *(volatile uint32_t*)&p.ctrl->tile_count) return;
        tile = p.tile_queue[blockIdx.x];
        npix = p.tile_nflag[tile];
    }
    const int tx0 = (int)(tile % (uint32_t)p.tiles_x) * kTileX;
    const int ty0 = (int)(tile / (uint32_t)p.tiles_x) * kTileY;

    // lanes per regressed pixel
    int lg = 0;  // log2(g)
    if (!kDense) lg = npix > 128 ? 0 : npix > 64 ? 1 : npix > 32 ? 2 : npix > 16 ? 3 : npix > 8 ? 4 : 5;
    const int g = 1 << lg;
    const int item = threadIdx.x >> lg;
    const int sub = threadIdx.x & (g - 1);
    bool active = item < npix;
    const int lidx = kDense ? (int)threadIdx.x
                            : (active ? (int)p.tile_pix[(size_t)tile * kTilePix + item] : 0);
    const int lx = lidx & (kTileX - 1), ly = lidx / kTileX;
    const int cx = tx0 + lx, cy = ty0 + ly;
    if (cx >= p.W || cy >= p.H) active = false;

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar[0], stage_bytes);
        tma_load_4d(buf0, &tmap, &bar[0], 0, tx0 - p.r, ty0 - p.r, 2 * (p.t % p.T));
    }

    const int dxlo = max(-p.r, -cx), dxhi = min(p.r, p.W - 1 - cx);
    const int dylo = max(-p.r, -cy), dyhi = min(p.r, p.H - 1 - cy);
    const int nx = dxhi - dxlo + 1;
    const int nvalid = nx * (dyhi - dylo + 1);
    const int sx = lx + p.r, sy = ly + p.r;
    const float spx = p.s_coord_px;

    Acc acc;
#pragma unroll
    for (int i = 0; i < NG; ++i) acc.G[i] = 0.0f;
#pragma unroll
    for (int i = 0; i < NZ; ++i) acc.B[i] = 0.0f;
    float sf[7], cf[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        sf[j] = p.s_feat[j];
        cf[j] = 0.0f;
    }

    for (int k = 0; k < p.n_tau; ++k) {
        const int b = k & 1;
        if (k + 1 < p.n_tau && threadIdx.x == 0) {
            // the other buffer was released by the barrier that ended step k-1
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[b ^ 1], stage_bytes);
            const int slot = (p.t - k - 1) % p.T;
            tma_load_4d(b ? buf0 : buf1, &tmap, &bar[b ^ 1], 0, tx0 - p.r, ty0 - p.r, 2 * slot);
        }
        const bool ok = mbar_wait_bounded(&bar[b], (uint32_t)((k >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            // A staged copy never landed: record it, let the copies in flight
            // finish (bounded), and give up on this tile.
            if (threadIdx.x == 0) {
                atomicOr(&p.ctrl->status, kStatusTimeout);
                mbar_wait_bounded(&bar[b], (uint32_t)((k >> 1) & 1));
                if (k + 1 < p.n_tau) mbar_wait_bounded(&bar[b ^ 1], (uint32_t)(((k + 1) >> 1) & 1));
            }
            __syncthreads();
            return;
        }
        const float4* P0 = b ? buf1 : buf0;
        const float4* P1 = P0 + plane;
        if (active) {
            if (k == 0) {
                const float4 c0 = P0[sy * p.sw + sx];
                const float4 c1 = P1[sy * p.sw + sx];
                cf[0] = c0.y * sf[0];
                cf[1] = c0.z * sf[1];
                cf[2] = c0.w * sf[2];
                cf[3] = c1.x * sf[3];
                cf[4] = c1.y * sf[4];
                cf[5] = c1.z * sf[5];
                cf[6] = c1.w * sf[6];
            }
            if (g == 1) {
                for (int oy = dylo; oy <= dyhi; ++oy) {
                    const float u2 = (float)oy * spx;
                    const float en_row = -u2 * u2;
                    const int row = (sy + oy) * p.sw + sx;
                    float u1 = (float)dxlo * spx;
#pragma unroll 3
                    for (int ox = dxlo; ox <= dxhi; ++ox) {
                        const float4 h0 = P0[row + ox];
                        const float4 h1 = P1[row + ox];
                        accumulate(acc, h0, h1, u1, u2, fmaf(-u1, u1, en_row), sf, cf);
                        u1 += spx;
                    }
                }
            } else {
                int ox = dxlo + sub % nx;
                int oy = dylo + sub / nx;
                for (int q = sub; q < nvalid; q += g) {
                    const int si = (sy + oy) * p.sw + sx + ox;
                    const float4 h0 = P0[si];
                    const float4 h1 = P1[si];
                    const float u1 = (float)ox * spx;
                    const float u2 = (float)oy * spx;
                    accumulate(acc, h0, h1, u1, u2, -fmaf(u1, u1, u2 * u2), sf, cf);
                    ox += g;
                    while (ox > dxhi) {
                        ox -= nx;
                        ++oy;
                    }
                }
            }
        }
        __syncthreads();
    }

    {
        // work accounting: (pixel, neighbour) pairs of this tile
        __shared__ unsigned long long s_pairs;
        if (threadIdx.x == 0) s_pairs = 0ull;
        __syncthreads();
        if (active && sub == 0) atomicAdd(&s_pairs, (unsigned long long)nvalid * (unsigned long long)p.n_tau);
        __syncthreads();
        if (threadIdx.x == 0 && s_pairs) atomicAdd(&p.ctrl->neighbours, s_pairs);
    }

    if (!kDense && g > 1) {
        // lanes of one pixel are adjacent in the warp: butterfly-reduce
        for (int off = g >> 1; off >= 1; off >>= 1) {
#pragma unroll
            for (int i = 0; i < NG; ++i) acc.G[i] += __shfl_xor_sync(0xffffffffu, acc.G[i], off);
#pragma unroll
            for (int i = 0; i < NZ; ++i) acc.B[i] += __shfl_xor_sync(0xffffffffu, acc.B[i], off);
        }
    }

    if (threadIdx.x == 0) {
        int cnt = npix;
        if (kDense) cnt = min(kTileX, p.W - tx0) * min(kTileY, p.H - ty0);
        atomicAdd(&p.ctrl->regressions, (unsigned long long)cnt);
    }
    if (!active || sub != 0) return;

    float s2[NZ];
    s2[0] = 0.0f;
    s2[1] = p.s_coord * p.s_coord;
    s2[2] = s2[1];
#pragma unroll
    for (int j = 0; j < 7; ++j) s2[3 + j] = sf[j] * sf[j];
    float theta[NZ];
    solve(acc, s2, p.ridge, theta);

    const size_t N = (size_t)p.W * p.H;
    const size_t i = (size_t)cy * p.W + cx;
    const float alpha = theta[0];
    float bf[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) bf[j] = theta[3 + j] * sf[j];
    p.alpha[i] = alpha;

    float L;
    if (p.init) {
        L = alpha;
    } else {
        L = p.state[N + i].w;
        const float dl = alpha - L;
        const float n = floorf(fabsf(dl) / p.C);
        if (!(n >= 1.0f)) return;  // no event: keep the model (Fig. 1)
        const float pol = dl > 0.0f ? 1.0f : -1.0f;
        L = fmaf(pol * n, p.C, L);
        p.nev[i] = (int32_t)(pol * n);
    }
    const int slot = p.t % p.T;
    const float4 x0 = p.ring[(size_t)(2 * slot) * N + i];
    const float4 x1 = p.ring[(size_t)(2 * slot + 1) * N + i];
    p.state[i] = make_float4(bf[0], bf[1], bf[2], bf[3]);
    p.state[N + i] = make_float4(bf[4], bf[5], bf[6], L);
    p.state[2 * N + i] = make_float4(x0.y, x0.z, x0.w, x1.x);
    p.state[3 * N + i] = make_float4(x1.y, x1.z, x1.w, 0.0f);
}

size_t wlr_smem_bytes(int r)
{
    const size_t stage = (size_t)2 * (kTileX + 2 * r) * (kTileY + 2 * r) * 16;
    const size_t buf = (stage + 127) & ~(size_t)127;
    return 2 * buf + 2 * sizeof(uint64_t) + 128;
}

cudaError_t wlr_prepare(int smem_bytes)
{
    cudaError_t e = cudaFuncSetAttribute(wlr_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(wlr_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem_bytes);
}

cudaError_t launch_wlr(const CUtensorMap& tmap, const WlrParams& p, int grid, int smem_bytes,
                       cudaStream_t s)
{
    if (p.dense)
        wlr_kernel<true><<<grid, kTilePix, smem_bytes, s>>>(tmap, p);
    else
        wlr_kernel<false><<<grid, kTilePix, smem_bytes, s>>>(tmap, p);
    return cudaGetLastError();
}

}  // namespace esim
