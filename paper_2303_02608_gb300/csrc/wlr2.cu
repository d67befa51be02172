// Second-order form: the dense weighted local regression of Eqs. 4-5 with the
// Taylor expansion of Eq. 3 carried one order further (the non-linear
// regression that Section 4 names as the extension).  Per frame t and centre c
// the design row of neighbour i is built from the scaled offset u = s d
// (s_j = k / (h b_j), k = sqrt(log2(e) / 2), so w = 2^-|u|^2 is the product
// Gaussian of Eq. 5):
//
//     z = (u_a u_b for a <= b [45], u [9], 1),   55 unknowns,
//
// and the log brightness y rides along as a 56th entry, so one symmetric
// 56 x 56 Gram G = sum_i w_i [z;y][z;y]^T holds the normal matrix and the
// right-hand side.  The ridge lambda W |theta_k|^2 on every coefficient but the
// intercept is added in natural units (lambda W s_a^2 s_b^2 on the diagonal of
// a quadratic unknown, lambda W s_a^2 on a linear one).  With the intercept
// ordered last among the unknowns, the upper Cholesky factor U of the augmented
// (equilibrated) Gram gives alpha = U[54][55] / U[54][54] directly: no back
// substitution.
//
// Layout of the work: a CTA of 288 threads covers 8 slots.  The 56 x 56 Gram is
// cut into 8 x 8 blocks of 7; the 36 blocks on and above the block diagonal of
// each slot go one per thread, a 7 x 7 register tile (49 FP32 accumulators) fed
// by two 7-vectors from shared memory per neighbour.  A round builds sqrt(w) z
// for 32 neighbours per slot in shared memory, then every thread runs its tile
// over them.  G slots share one pixel, each summing an interleaved G-th of the
// window's neighbour batches (G grows with the window, so no accumulator sums
// more than a few hundred terms in FP32); their partial tiles are added in slot
// order, so results do not depend on scheduling.  The solve never leaves the
// tiles: ridge and Jacobi equilibration tile by tile, then a right-looking
// blocked Cholesky over the 8 block columns, panels passing through shared
// memory.
#include <stdlib.h>

#include "esim_ad.h"
#include "internal.h"
#include "ptx.cuh"

namespace esim {
namespace {

constexpr int kNQ = 55;                    // unknowns
constexpr int kNA = 56;                    // unknowns + log brightness
constexpr int kNB = 36;                    // 7 x 7 tiles on and above the block diagonal
constexpr int kSlots = 8;                  // 36-thread slots per CTA
constexpr int kThreads = kSlots * kNB;     // 288
constexpr int kBatch = 32;                 // neighbours per slot per round
constexpr int kRow4 = 17;                  // float4 per neighbour: [2 halves][8 blocks] + 1 pad
constexpr int kSlot4 = kBatch * kRow4 + 1; // float4 per slot: the +1 puts the 8 slots in 8 bank groups
constexpr int kUStride = 8 * 7 * 8 + 4;    // floats per slot of panel storage, same bank spread
constexpr size_t kSmemZ = (size_t)kSlots * kSlot4 * sizeof(float4);  // 69,760 B
static_assert((size_t)kSlots * kNB * 49 * sizeof(float) <= kSmemZ, "partial tiles must fit in the neighbour buffer");

constexpr float kExp2Scale = 0.84932180028801904272f;  // sqrt(log2(e) / 2)

// Quadratic unknown q (0..44) -> feature pair (a, b), a <= b, a-major order.
__host__ __device__ constexpr int pair_a(int q)
{
    int a = 0;
    while (q >= 9 - a) { q -= 9 - a; ++a; }
    return a;
}
__host__ __device__ constexpr int pair_b(int q)
{
    int a = 0;
    while (q >= 9 - a) { q -= 9 - a; ++a; }
    return a + q;
}

// Entry Z of the augmented row [z; y] (before the sqrt(w) factor).
template <int Z>
__device__ __forceinline__ float zval(const float (&u)[9], float y)
{
    if constexpr (Z < 45) return u[pair_a(Z)] * u[pair_b(Z)];
    else if constexpr (Z < 54) return u[Z - 45];
    else if constexpr (Z == 54) return 1.0f;
    else return y;
}

// Element m (0..7, 7 = pad) of block b sits in float4 slot (m / 4) * 8 + b,
// lane m % 4: the 8 blocks of one half fill a 128-byte row of banks.
template <int S>
__device__ __forceinline__ void store_row(float4* row, const float (&u)[9], float y, float sw)
{
    constexpr int h = S / 8, b = S % 8, z0 = 7 * b + 4 * h;
    float4 v;
    v.x = zval<z0>(u, y) * sw;
    v.y = zval<z0 + 1>(u, y) * sw;
    v.z = zval<z0 + 2>(u, y) * sw;
    if constexpr (h == 0) v.w = zval<z0 + 3>(u, y) * sw;
    else v.w = 0.0f;
    row[S] = v;
    if constexpr (S + 1 < 16) store_row<S + 1>(row, u, y, sw);
}

struct W2Params {
    int W, H, F, r, T, rgb, tiles_x;
    float h, log_eps, ridge;
    const float* radiance;   // [F][C][H][W]
    const float* features;   // [F][7][H][W]
    const float* bandwidth;  // [7]
    float4* packed;          // [F][2][H][W]: (y, normal xyz), (depth, albedo rgb)
    float* alpha;            // [F][H][W]
};

__global__ void __launch_bounds__(kTilePix) wlr2_pack_kernel(W2Params p)
{
    const size_t N = (size_t)p.W * p.H;
    const int f = blockIdx.y;
    const int x = (blockIdx.x % p.tiles_x) * kTileX + (threadIdx.x & 31);
    const int y = (blockIdx.x / p.tiles_x) * kTileY + (threadIdx.x >> 5);
    if (x >= p.W || y >= p.H) return;
    const size_t i = (size_t)y * p.W + x;
    const float* rad = p.radiance + (size_t)f * (p.rgb ? 3 : 1) * N;
    const float Y = p.rgb ? 0.2126f * rad[i] + 0.7152f * rad[N + i] + 0.0722f * rad[2 * N + i] : rad[i];
    const float* ft = p.features + (size_t)f * 7 * N;
    float4* out = p.packed + (size_t)f * 2 * N;
    out[i] = make_float4(logf(Y + p.log_eps), ft[i], ft[N + i], ft[2 * N + i]);
    out[N + i] = make_float4(ft[3 * N + i], ft[4 * N + i], ft[5 * N + i], ft[6 * N + i]);
}

// G slots per pixel, 8 / G pixels per CTA along one image row.  96 registers
// keep two 9-warp CTAs per SM (the register file is split over four
// sub-partitions); the few values that do not fit spill only in the panel solve.
template <int G>
__global__ void __maxnreg__(96) wlr2_kernel(W2Params p)
{
    constexpr int P = kSlots / G;              // pixels per CTA
    extern __shared__ float4 zbuf[];           // [kSlots][kSlot4]; then [kSlots][kNB][49] partial tiles
    __shared__ float s_s2[kNQ];                // squared natural-unit scale of each unknown
    __shared__ float s_sf[7];
    __shared__ float s_diag[kSlots][kNA + 1];  // Gram diagonal, for the equilibration
    __shared__ float s_lw[kSlots];             // lambda W
    __shared__ __align__(16) float s_u[kSlots * kUStride];  // panel U_J,K of the current block column
    __shared__ float s_inv[kSlots][7];         // 1 / diagonal of U_JJ
    __shared__ float s_cf[kSlots][7];          // scaled centre features of each slot's pixel

    const int tid = threadIdx.x;
    const size_t N = (size_t)p.W * p.H;
    const int nxc = (p.W + P - 1) / P;
    const int xc = (int)(blockIdx.x % (unsigned)nxc);
    const int cy = (int)((blockIdx.x / (unsigned)nxc) % (unsigned)p.H);
    const int f = (int)(blockIdx.x / ((unsigned)nxc * (unsigned)p.H));
    const int x0 = xc * P;

    if (tid < 7) s_sf[tid] = kExp2Scale / (p.h * p.bandwidth[tid]);
    __syncthreads();
    if (tid < kNQ) {
        const float sc = kExp2Scale / p.h;
        auto sdim = [&](int a) { return a < 2 ? sc : s_sf[a - 2]; };
        float s2 = 0.0f;
        if (tid < 45) {
            const float v = sdim(pair_a(tid)) * sdim(pair_b(tid));
            s2 = v * v;
        } else if (tid < 54) {
            const float v = sdim(tid - 45);
            s2 = v * v;
        }
        s_s2[tid] = s2;
    }

    // builder role: slot cs, neighbour j of each round
    const int cs = tid >> 5, j = tid & 31;
    const int b_pix = x0 + cs / G, b_sub = cs % G;
    const bool builder = tid < kSlots * kBatch;
    const bool b_ok = builder && b_pix < p.W;
    const float s_px = kExp2Scale / (p.h * (float)p.r);
    if (b_ok && j < 7) {   // scaled centre features of the slot's pixel
        const size_t ci = (size_t)cy * p.W + b_pix;
        const float4 c0 = p.packed[(size_t)f * 2 * N + ci];
        const float4 c1 = p.packed[((size_t)f * 2 + 1) * N + ci];
        const float xcv[7] = {c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
        float v = xcv[0];
#pragma unroll
        for (int k = 1; k < 7; ++k)
            if (j == k) v = xcv[k];
        s_cf[cs][j] = v * s_sf[j];
    }

    // accumulator role: 7 x 7 tile (bi, bj) of the block grid for one slot.  The
    // 8 slots' copies of a tile sit in adjacent lanes, so that each step of the
    // factorisation below runs in the few warps that hold its tiles.
    const int slot = tid % kSlots, tk = tid / kSlots;
    int bi = 0, bj = tk;
    while (bj >= 8 - bi) { bj -= 8 - bi; ++bi; }
    bj += bi;
    float acc[7][7];
#pragma unroll
    for (int i = 0; i < 7; ++i)
#pragma unroll
        for (int k = 0; k < 7; ++k) acc[i][k] = 0.0f;

    __syncthreads();   // s_cf, s_s2 ready
    const int S = 2 * p.r + 1;
    const int t_eff = min(p.T, f + 1);
    const int M = S * S * t_eff;
    const int n_batch = (M + kBatch - 1) / kBatch;
    const int rounds = (n_batch + G - 1) / G;
    for (int q = 0; q < rounds; ++q) {
        if (builder) {
            float4* row = zbuf + (size_t)cs * kSlot4 + j * kRow4;
            const int n = (q * G + b_sub) * kBatch + j;
            bool ok = b_ok && n < M;
            int qx = 0, qy = 0, tau = 0;
            if (ok) {
                const int ti = n / (S * S), rem = n - ti * S * S;
                const int oy = rem / S - p.r, ox = rem - (rem / S) * S - p.r;
                tau = f - t_eff + 1 + ti;
                qx = b_pix + ox;
                qy = cy + oy;
                ok = qx >= 0 && qx < p.W && qy >= 0 && qy < p.H;
                if (ok) {
                    const size_t qi = (size_t)qy * p.W + qx;
                    const float4 h0 = __ldg(p.packed + (size_t)tau * 2 * N + qi);
                    const float4 h1 = __ldg(p.packed + ((size_t)tau * 2 + 1) * N + qi);
                    const float xv[7] = {h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
                    float u[9];
                    u[0] = (float)ox * s_px;
                    u[1] = (float)oy * s_px;
                    float e = fmaf(u[0], u[0], u[1] * u[1]);
#pragma unroll
                    for (int k = 0; k < 7; ++k) {
                        u[2 + k] = fmaf(xv[k], s_sf[k], -s_cf[cs][k]);
                        e = fmaf(u[2 + k], u[2 + k], e);
                    }
                    store_row<0>(row, u, h0.x, ex2_approx(-0.5f * e));   // sqrt(w) = 2^(-|u|^2 / 2)
                }
            }
            if (!ok) {
#pragma unroll
                for (int k = 0; k < 16; ++k) row[k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
        }
        __syncthreads();
        const float4* base = zbuf + (size_t)slot * kSlot4;
#pragma unroll 2
        for (int n = 0; n < kBatch; ++n) {
            const float4* row = base + n * kRow4;
            const float4 r0 = row[bi], r1 = row[8 + bi], c0 = row[bj], c1 = row[8 + bj];
            const float rv[7] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z};
            const float cv[7] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z};
#pragma unroll
            for (int i = 0; i < 7; ++i)
#pragma unroll
                for (int k = 0; k < 7; ++k) acc[i][k] = fmaf(rv[i], cv[k], acc[i][k]);
        }
        __syncthreads();
    }

    // The G slots of a pixel add their tiles into the first slot's, in slot order.
    if constexpr (G > 1) {
        float* part = reinterpret_cast<float*>(zbuf) + ((size_t)slot * kNB + tk) * 49;
#pragma unroll
        for (int i = 0; i < 7; ++i)
#pragma unroll
            for (int k = 0; k < 7; ++k) part[i * 7 + k] = acc[i][k];
        __syncthreads();
        if (slot % G == 0) {
#pragma unroll
            for (int s = 1; s < G; ++s) {
                const float* o = part + (size_t)s * kNB * 49;
#pragma unroll
                for (int i = 0; i < 7; ++i)
#pragma unroll
                    for (int k = 0; k < 7; ++k) acc[i][k] += o[i * 7 + k];
            }
        }
    }
    const bool lead = slot % G == 0 && x0 + slot / G < p.W;

    // Ridge and Jacobi equilibration, tile by tile: A_ab <- A_ab / sqrt(A_aa A_bb)
    // (the log-brightness row keeps scale 1).
    if (lead && bi == bj) {
#pragma unroll
        for (int i = 0; i < 7; ++i) s_diag[slot][7 * bi + i] = acc[i][i];
        if (bi == 7) s_lw[slot] = p.ridge * acc[5][5];   // lambda W; W = sum w = A[54][54]
    }
    __syncthreads();
    float d54 = 1.0f;   // equilibration scale of the intercept (tile (7,7), row 5)
    if (lead) {
        const float lw = s_lw[slot];
        float dr[7], dc[7];
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            const int a = 7 * bi + i, c = 7 * bj + i;
            const float da = a < 54 ? fmaf(lw, s_s2[a], s_diag[slot][a]) : s_diag[slot][a];
            const float dcv = c < 54 ? fmaf(lw, s_s2[c], s_diag[slot][c]) : s_diag[slot][c];
            dr[i] = a < kNQ ? rsqrtf(da) : 1.0f;
            dc[i] = c < kNQ ? rsqrtf(dcv) : 1.0f;
            if (bi == bj && a < 54) acc[i][i] = fmaf(lw, s_s2[a], acc[i][i]);
        }
#pragma unroll
        for (int i = 0; i < 7; ++i)
#pragma unroll
            for (int k = 0; k < 7; ++k) acc[i][k] *= dr[i] * dc[k];
        d54 = dr[5];
    }

    // Right-looking blocked Cholesky A = U^T U over the 8 block columns, each
    // tile staying in its owner's registers: factor the diagonal tile, solve
    // the panel U_JK = U_JJ^-T A_JK, update the trailing tiles
    // A_KL -= U_JK^T U_JL.  Panels pass through shared memory.
    float* uf = s_u + slot * kUStride;         // [8 blocks][7 rows][8]
    for (int J = 0; J < 8; ++J) {
        if (lead && bi == J && bj == J) {
#pragma unroll
            for (int i = 0; i < 7; ++i) {
                float sd = acc[i][i];
#pragma unroll
                for (int m = 0; m < i; ++m) sd = fmaf(-acc[m][i], acc[m][i], sd);
                const float piv = sqrtf(fmaxf(sd, 1e-30f));
                const float inv = 1.0f / piv;
                acc[i][i] = piv;
#pragma unroll
                for (int k = i + 1; k < 7; ++k) {
                    float x = acc[i][k];
#pragma unroll
                    for (int m = 0; m < i; ++m) x = fmaf(-acc[m][i], acc[m][k], x);
                    acc[i][k] = x * inv;
                }
                s_inv[slot][i] = inv;
            }
#pragma unroll
            for (int i = 0; i < 7; ++i)
#pragma unroll
                for (int k = 0; k < 8; ++k) uf[(J * 7 + i) * 8 + k] = (k < 7 && k >= i) ? acc[i][k] : 0.0f;
        }
        __syncthreads();
        if (lead && bi == J && bj > J) {
#pragma unroll
            for (int i = 0; i < 7; ++i) {
                const float inv = s_inv[slot][i];
#pragma unroll
                for (int k = 0; k < 7; ++k) {
                    float x = acc[i][k];
#pragma unroll
                    for (int m = 0; m < i; ++m) x = fmaf(-uf[(J * 7 + m) * 8 + i], acc[m][k], x);
                    acc[i][k] = x * inv;
                }
            }
#pragma unroll
            for (int i = 0; i < 7; ++i)
#pragma unroll
                for (int k = 0; k < 8; ++k) uf[(bj * 7 + i) * 8 + k] = k < 7 ? acc[i][k] : 0.0f;
        }
        __syncthreads();
        if (lead && bi > J) {
            const float4* u4 = reinterpret_cast<const float4*>(uf);
#pragma unroll 1
            for (int m = 0; m < 7; ++m) {
                const float4 a0 = u4[(bi * 7 + m) * 2], a1 = u4[(bi * 7 + m) * 2 + 1];
                const float4 b0 = u4[(bj * 7 + m) * 2], b1 = u4[(bj * 7 + m) * 2 + 1];
                const float av[7] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z};
                const float bv[7] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z};
#pragma unroll
                for (int i = 0; i < 7; ++i)
#pragma unroll
                    for (int k = 0; k < 7; ++k) acc[i][k] = fmaf(-av[i], bv[k], acc[i][k]);
            }
        }
        __syncthreads();
    }
    // With the intercept last and y appended, U[54][55] = (U^-T b)_54 and
    // theta_54 = U[54][55] / U[54][54] in the equilibrated basis.
    if (lead && bi == 7 && bj == 7)
        p.alpha[(size_t)f * N + (size_t)cy * p.W + x0 + slot / G] = acc[5][6] / acc[5][5] * d54;
}

bool desc_ok(const esim_ad_wlr_desc* d)
{
    return d && d->struct_size == sizeof(esim_ad_wlr_desc) && d->width >= 1 && d->height >= 1 &&
           d->sequence >= 1 && d->radius >= 1 && d->radius <= kMaxRadius && d->frames >= 1 &&
           d->frames <= kMaxFrames && (d->radiance_fmt == ESIM_AD_LUMA_F32 || d->radiance_fmt == ESIM_AD_RGB_F32) &&
           d->h > 0.0f && d->ridge > 0.0f && d->log_eps >= 0.0f;
}

// Slots per pixel: the largest of 1, 2, 4, 8 that leaves each slot at least
// 128 of the window's neighbours.  ESIM_AD_WLR2_GROUPS overrides it.
int groups_for(const esim_ad_wlr_desc* d)
{
    if (const char* e = getenv("ESIM_AD_WLR2_GROUPS")) {
        const int g = atoi(e);
        if (g == 1 || g == 2 || g == 4 || g == 8) return g;
    }
    const int S = 2 * d->radius + 1, M = S * S * d->frames;
    int g = 1;
    while (g < 8 && M >= 2 * g * 128) g *= 2;
    return g;
}

template <int G>
cudaError_t launch(const W2Params& p, cudaStream_t s)
{
    constexpr int P = kSlots / G;
    cudaError_t e = cudaFuncSetAttribute(wlr2_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemZ);
    if (e != cudaSuccess) return e;
    // two CTAs per SM: about 175 KB of shared memory (the rest of the unified array stays L1)
    e = cudaFuncSetAttribute(wlr2_kernel<G>, cudaFuncAttributePreferredSharedMemoryCarveout, 80);
    if (e != cudaSuccess) return e;
    const unsigned long long n = (unsigned long long)p.F * p.H * ((p.W + P - 1) / P);
    if (n == 0 || n > 0x7fffffffull) return cudaErrorInvalidValue;
    wlr2_kernel<G><<<(unsigned)n, kThreads, kSmemZ, s>>>(p);
    return cudaGetLastError();
}

}  // namespace
}  // namespace esim

using namespace esim;

extern "C" size_t esim_ad_wlr2_workspace_size(const esim_ad_wlr_desc* d)
{
    if (!desc_ok(d)) return 0;
    return (size_t)d->sequence * 2 * (size_t)d->width * d->height * sizeof(float4);
}

extern "C" esim_ad_status esim_ad_wlr2_forward(const esim_ad_wlr_desc* d, const float* radiance,
                                               const float* features, const float* bandwidth, float* alpha,
                                               void* workspace, void* cuda_stream)
{
    if (!desc_ok(d) || !radiance || !features || !bandwidth || !alpha || !workspace) return ESIM_AD_EINVAL;
    W2Params p;
    p.W = d->width;
    p.H = d->height;
    p.F = d->sequence;
    p.r = d->radius;
    p.T = d->frames;
    p.rgb = d->radiance_fmt == ESIM_AD_RGB_F32 ? 1 : 0;
    p.tiles_x = (d->width + kTileX - 1) / kTileX;
    p.h = d->h;
    p.log_eps = d->log_eps;
    p.ridge = d->ridge;
    p.radiance = radiance;
    p.features = features;
    p.bandwidth = bandwidth;
    p.packed = static_cast<float4*>(workspace);
    p.alpha = alpha;
    if (d->sequence > 65535) return ESIM_AD_EINVAL;   // frames index the pack grid's y dimension
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const dim3 pack_grid(p.tiles_x * ((d->height + kTileY - 1) / kTileY), d->sequence);
    wlr2_pack_kernel<<<pack_grid, kTilePix, 0, s>>>(p);
    if (cudaGetLastError() != cudaSuccess) return ESIM_AD_ECUDA;
    cudaError_t e;
    switch (groups_for(d)) {
        case 1: e = launch<1>(p, s); break;
        case 2: e = launch<2>(p, s); break;
        case 4: e = launch<4>(p, s); break;
        default: e = launch<8>(p, s); break;
    }
    if (e == cudaErrorInvalidValue) return ESIM_AD_EINVAL;
    return e == cudaSuccess ? ESIM_AD_OK : ESIM_AD_ECUDA;
}
