// Differentiation form: dense weighted local regression over a sequence and its
// adjoint (backward) with respect to the noisy radiance and the seven feature
// bandwidths of Eq. 5.
//
// Forward, per frame t and centre c: the regression of Eqs. 3-5 over frames
// t-T+1..t (same arithmetic as the simulator: scaled regressors
// u = s * d with s = k / (h b), w = 2^-|u|^2, FP32 Gram, equilibrated Cholesky),
// keeping theta' and v' = A'^-1 e_0 in the scaled basis.
//
// Backward (adjoint of alpha = e_0^T A^-1 g):
//   d alpha / d y_i = w_i v^T z_i
//   d alpha / d w_i = v^T z_i r_i - lambda v^T P theta     (ridge lambda W |beta|^2)
//   d w_i / d b_j   = w_i d_ij^2 / (h^2 b_j^3) = w_i u_ij^2 / (k^2 b_j)
//   d y / d E_ch    = lum_ch / (Y + eps)
// where v^T z_i = v'^T u_i in the scaled basis and v^T P theta =
// sum_{j>=1} s_j^2 v'_j theta'_j.  The bandwidth gradient is a per-centre sum
// reduced per block into partials and then in a fixed order; the radiance
// gradient is a gather over the centres whose windows contain each pixel, so
// every result is deterministic.
#include "esim_ad.h"
#include "internal.h"
#include "wlr_math.cuh"

namespace esim {
namespace {

constexpr double kExp2ScaleD = 0.84932180028801904272;   // sqrt(log2(e) / 2)
constexpr float kExp2Scale = 0.84932180028801904272f;

struct AdjParams {
    int W, H, F, r, T, tiles_x, rgb;
    float h, log_eps, ridge;
    const float* radiance;   // [F][C][H][W]
    const float* features;   // [F][7][H][W]
    const float* bandwidth;  // [7]
    const float4* packed;    // [F][2][H][W]: (y, normal xyz), (depth, albedo rgb)
    float* alpha;            // [F][H][W]
    float* saved;            // [F][20][H][W]: theta' (10), v' (10)
    const float* g_alpha;    // [F][H][W]
    float4* gv;              // [F][3][H][W]: g_alpha * v' (10) + 2 pad
    float* partials;         // [blocks][8]
    float* g_radiance;       // [F][C][H][W]
    float* g_bandwidth;      // [7]
};

// Regressor scales from the bandwidths (device memory, read per block).
__device__ __forceinline__ void scales(const AdjParams& p, float (&sf)[7], float& s_c, float& s_px)
{
#pragma unroll
    for (int j = 0; j < 7; ++j) sf[j] = kExp2Scale / (p.h * p.bandwidth[j]);
    s_c = kExp2Scale / p.h;
    s_px = s_c / (float)p.r;
}

__global__ void __launch_bounds__(kTilePix) pack_kernel(AdjParams p)
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
    float4* out = const_cast<float4*>(p.packed) + (size_t)f * 2 * N;
    out[i] = make_float4(logf(Y + p.log_eps), ft[i], ft[N + i], ft[2 * N + i]);
    out[N + i] = make_float4(ft[3 * N + i], ft[4 * N + i], ft[5 * N + i], ft[6 * N + i]);
}

// Equilibrated Cholesky of the ridged system; theta' = A'^-1 g and v' = A'^-1 e_0.
__device__ __forceinline__ void solve_theta_v(Acc& a, const float (&s2)[NZ], float ridge,
                                              float (&theta)[NZ], float (&v)[NZ])
{
    const float Wsum = a.G[0];
#pragma unroll
    for (int j = 1; j < NZ; ++j) a.G[tri(j, j)] = fmaf(ridge * Wsum, s2[j], a.G[tri(j, j)]);
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
        float sj = a.G[tri(j, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) sj = fmaf(-a.G[tri(j, k)], a.G[tri(j, k)], sj);
        sj = fmaxf(sj, 1e-20f);
        const float l = sqrtf(sj);
        inv[j] = 1.0f / l;
#pragma unroll
        for (int i = j + 1; i < NZ; ++i) {
            float x = a.G[tri(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) x = fmaf(-a.G[tri(i, k)], a.G[tri(j, k)], x);
            a.G[tri(i, j)] = x * inv[j];
        }
    }
    float rhs[2][NZ];
#pragma unroll
    for (int i = 0; i < NZ; ++i) {
        rhs[0][i] = a.B[i];
        rhs[1][i] = i == 0 ? dsc[0] : 0.0f;
    }
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        float z[NZ], x[NZ];
#pragma unroll
        for (int i = 0; i < NZ; ++i) {
            float t = rhs[m][i];
#pragma unroll
            for (int k = 0; k < i; ++k) t = fmaf(-a.G[tri(i, k)], z[k], t);
            z[i] = t * inv[i];
        }
#pragma unroll
        for (int i = NZ - 1; i >= 0; --i) {
            float t = z[i];
#pragma unroll
            for (int k = i + 1; k < NZ; ++k) t = fmaf(-a.G[tri(k, i)], x[k], t);
            x[i] = t * inv[i];
        }
#pragma unroll
        for (int i = 0; i < NZ; ++i) {
            if (m == 0) theta[i] = x[i] * dsc[i];
            else v[i] = x[i] * dsc[i];
        }
    }
}

__global__ void __launch_bounds__(kTilePix, 2) fwd_kernel(AdjParams p)
{
    const size_t N = (size_t)p.W * p.H;
    const int f = blockIdx.y;
    const int cx = (blockIdx.x % p.tiles_x) * kTileX + (threadIdx.x & 31);
    const int cy = (blockIdx.x / p.tiles_x) * kTileY + (threadIdx.x >> 5);
    if (cx >= p.W || cy >= p.H) return;
    float sf[7], s_c, s_px;
    scales(p, sf, s_c, s_px);
    const size_t ci = (size_t)cy * p.W + cx;
    const float4 c0 = p.packed[(size_t)f * 2 * N + ci];
    const float4 c1 = p.packed[((size_t)f * 2 + 1) * N + ci];
    float cf[7] = {c0.y * sf[0], c0.z * sf[1], c0.w * sf[2], c1.x * sf[3], c1.y * sf[4], c1.z * sf[5],
                   c1.w * sf[6]};
    Acc acc;
#pragma unroll
    for (int i = 0; i < NG; ++i) acc.G[i] = 0.0f;
#pragma unroll
    for (int i = 0; i < NZ; ++i) acc.B[i] = 0.0f;
    const int dxlo = max(-p.r, -cx), dxhi = min(p.r, p.W - 1 - cx);
    const int dylo = max(-p.r, -cy), dyhi = min(p.r, p.H - 1 - cy);
    const int tau0 = max(0, f - p.T + 1);
    for (int tau = tau0; tau <= f; ++tau) {
        const float4* P0 = p.packed + (size_t)tau * 2 * N + ci;
        const float4* P1 = P0 + N;
        for (int oy = dylo; oy <= dyhi; ++oy) {
            const float u2 = (float)oy * s_px;
            for (int ox = dxlo; ox <= dxhi; ++ox) {
                const float u1 = (float)ox * s_px;
                const int d = oy * p.W + ox;
                accumulate(acc, __ldg(P0 + d), __ldg(P1 + d), u1, u2, -fmaf(u1, u1, u2 * u2), sf, cf);
            }
        }
    }
    float s2[NZ];
    s2[0] = 0.0f;
    s2[1] = s_c * s_c;
    s2[2] = s2[1];
#pragma unroll
    for (int j = 0; j < 7; ++j) s2[3 + j] = sf[j] * sf[j];
    float theta[NZ], v[NZ];
    solve_theta_v(acc, s2, p.ridge, theta, v);
    p.alpha[(size_t)f * N + ci] = theta[0];
    float* sv = p.saved + (size_t)f * 20 * N + ci;
#pragma unroll
    for (int k = 0; k < NZ; ++k) {
        sv[(size_t)k * N] = theta[k];
        sv[(size_t)(NZ + k) * N] = v[k];
    }
}

// Per centre: g_alpha v' for the radiance gather, and the centre's share of
// the bandwidth gradient (sum over its window of g_alpha (d alpha/d w_i) w_i u_ij^2).
// Each thread takes kCtrRows centres stacked in one column, so every neighbour
// record it loads (32 bytes) serves each of them whose window holds it; a
// 128-thread CTA covers one 32 x 8 tile.
constexpr int kCtrRows = 2;
constexpr int kCtrThreads = kTilePix / kCtrRows;

__global__ void __launch_bounds__(kCtrThreads, 4) bwd_center_kernel(AdjParams p)
{
    const size_t N = (size_t)p.W * p.H;
    const int f = blockIdx.y;
    const int cx = (blockIdx.x % p.tiles_x) * kTileX + (threadIdx.x & 31);
    const int cy0 = (blockIdx.x / p.tiles_x) * kTileY + kCtrRows * (threadIdx.x >> 5);
    float sf[7], s_c, s_px;
    scales(p, sf, s_c, s_px);
    float gb[7] = {0, 0, 0, 0, 0, 0, 0};
    float ga[kCtrRows], lvpt[kCtrRows], th[kCtrRows][NZ], v[kCtrRows][NZ], cf[kCtrRows][7];
    bool active[kCtrRows];
    bool any = false;
#pragma unroll
    for (int k = 0; k < kCtrRows; ++k) {
        const int cy = cy0 + k;
        active[k] = false;
        ga[k] = 0.0f;
        lvpt[k] = 0.0f;
#pragma unroll
        for (int i = 0; i < NZ; ++i) th[k][i] = v[k][i] = 0.0f;
#pragma unroll
        for (int j = 0; j < 7; ++j) cf[k][j] = 0.0f;
        if (cx >= p.W || cy >= p.H) continue;
        const size_t ci = (size_t)cy * p.W + cx;
        ga[k] = p.g_alpha[(size_t)f * N + ci];
        const float* sv = p.saved + (size_t)f * 20 * N + ci;
#pragma unroll
        for (int i = 0; i < NZ; ++i) {
            th[k][i] = sv[(size_t)i * N];
            v[k][i] = sv[(size_t)(NZ + i) * N];
        }
        float4* g = p.gv + (size_t)f * 3 * N + ci;
        g[0] = make_float4(ga[k] * v[k][0], ga[k] * v[k][1], ga[k] * v[k][2], ga[k] * v[k][3]);
        g[N] = make_float4(ga[k] * v[k][4], ga[k] * v[k][5], ga[k] * v[k][6], ga[k] * v[k][7]);
        g[2 * N] = make_float4(ga[k] * v[k][8], ga[k] * v[k][9], 0.0f, 0.0f);
        if (ga[k] == 0.0f) continue;
        // lambda v^T P theta in natural units
        float vpt = (s_c * s_c) * (v[k][1] * th[k][1] + v[k][2] * th[k][2]);
#pragma unroll
        for (int j = 0; j < 7; ++j) vpt = fmaf(sf[j] * sf[j], v[k][3 + j] * th[k][3 + j], vpt);
        lvpt[k] = p.ridge * vpt;
        const float4 c0 = p.packed[(size_t)f * 2 * N + ci];
        const float4 c1 = p.packed[((size_t)f * 2 + 1) * N + ci];
        cf[k][0] = c0.y * sf[0];
        cf[k][1] = c0.z * sf[1];
        cf[k][2] = c0.w * sf[2];
        cf[k][3] = c1.x * sf[3];
        cf[k][4] = c1.y * sf[4];
        cf[k][5] = c1.z * sf[5];
        cf[k][6] = c1.w * sf[6];
        active[k] = true;
        any = true;
    }
    if (any) {
        // neighbours (cx + ox, ny) inside the image, in the window of some centre row
        const int dxlo = max(-p.r, -cx), dxhi = min(p.r, p.W - 1 - cx);
        const int nylo = max(0, cy0 - p.r), nyhi = min(p.H - 1, cy0 + kCtrRows - 1 + p.r);
        for (int tau = max(0, f - p.T + 1); tau <= f; ++tau) {
            const float4* P0 = p.packed + (size_t)tau * 2 * N;
            const float4* P1 = P0 + N;
            for (int ny = nylo; ny <= nyhi; ++ny) {
                for (int ox = dxlo; ox <= dxhi; ++ox) {
                    const float u1 = (float)ox * s_px;
                    const size_t ni = (size_t)ny * p.W + cx + ox;
                    const float4 h0 = __ldg(P0 + ni), h1 = __ldg(P1 + ni);
                    const float fv[7] = {h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
#pragma unroll
                    for (int k = 0; k < kCtrRows; ++k) {
                        const int oy = ny - (cy0 + k);
                        if (!active[k] || oy < -p.r || oy > p.r) continue;
                        const float u2 = (float)oy * s_px;
                        float u[7];
                        float en = -fmaf(u1, u1, u2 * u2);
#pragma unroll
                        for (int j = 0; j < 7; ++j) {
                            u[j] = fmaf(fv[j], sf[j], -cf[k][j]);
                            en = fmaf(-u[j], u[j], en);
                        }
                        const float w = ex2_approx(en);
                        float fit = th[k][0] + th[k][1] * u1 + th[k][2] * u2;
                        float vz = v[k][0] + v[k][1] * u1 + v[k][2] * u2;
#pragma unroll
                        for (int j = 0; j < 7; ++j) {
                            fit = fmaf(th[k][3 + j], u[j], fit);
                            vz = fmaf(v[k][3 + j], u[j], vz);
                        }
                        const float dadw = fmaf(vz, h0.x - fit, -lvpt[k]);
                        const float c = ga[k] * dadw * w;
#pragma unroll
                        for (int j = 0; j < 7; ++j) gb[j] = fmaf(c, u[j] * u[j], gb[j]);
                    }
                }
            }
        }
    }
    // block tree sum in a fixed order -> one partial per block
    __shared__ float red[kCtrThreads][8];
#pragma unroll
    for (int j = 0; j < 7; ++j) red[threadIdx.x][j] = gb[j];
    __syncthreads();
    for (int s = kCtrThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int j = 0; j < 7; ++j) red[threadIdx.x][j] += red[threadIdx.x + s][j];
        __syncthreads();
    }
    if (threadIdx.x < 7)
        p.partials[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 8 + threadIdx.x] = red[0][threadIdx.x];
}

// Fixed-order reduction of the per-block partials; dL/db_j = sum / (k^2 b_j).
__global__ void __launch_bounds__(kTilePix) bwd_bandwidth_kernel(AdjParams p, int n_blocks)
{
    __shared__ double red[kTilePix];
    for (int j = 0; j < 7; ++j) {
        double acc = 0.0;
        for (int b = threadIdx.x; b < n_blocks; b += blockDim.x) acc += (double)p.partials[(size_t)b * 8 + j];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int s = kTilePix / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0)
            p.g_bandwidth[j] = (float)(red[0] / (kExp2ScaleD * kExp2ScaleD * (double)p.bandwidth[j]));
        __syncthreads();
    }
}

// Per source pixel q of frame tau: dL/dy = sum over centres c (|c - q| <= r) of
// frames t in [tau, tau + T - 1] of g_alpha_t(c) w v'_t(c)^T u, then dL/dE.
// Each thread gathers for kSrcRows sources stacked in one column, so every
// centre record it loads (two feature records and three g_alpha v' records,
// 80 bytes) serves each of those sources whose window holds it: 2.8 pairs per
// load at r = 3 instead of one.  A CTA covers 32 columns x 32 rows.
constexpr int kSrcRows = 4;
constexpr int kSrcTileY = kSrcRows * (kTilePix / 32);

__global__ void __launch_bounds__(kTilePix, 2) bwd_source_kernel(AdjParams p)
{
    const size_t N = (size_t)p.W * p.H;
    const int tau = blockIdx.y;
    const int qx = (blockIdx.x % p.tiles_x) * kTileX + (threadIdx.x & 31);
    const int qy0 = (blockIdx.x / p.tiles_x) * kSrcTileY + kSrcRows * (threadIdx.x >> 5);
    if (qx >= p.W || qy0 >= p.H) return;
    const int nrow = min(kSrcRows, p.H - qy0);
    float sf[7], s_c, s_px;
    scales(p, sf, s_c, s_px);
    float qf[kSrcRows][7], gy[kSrcRows];
#pragma unroll
    for (int s = 0; s < kSrcRows; ++s) {
        gy[s] = 0.0f;
        const size_t qi = (size_t)(qy0 + min(s, nrow - 1)) * p.W + qx;
        const float4 q0 = p.packed[(size_t)tau * 2 * N + qi];
        const float4 q1 = p.packed[((size_t)tau * 2 + 1) * N + qi];
        qf[s][0] = q0.y * sf[0];
        qf[s][1] = q0.z * sf[1];
        qf[s][2] = q0.w * sf[2];
        qf[s][3] = q1.x * sf[3];
        qf[s][4] = q1.y * sf[4];
        qf[s][5] = q1.z * sf[5];
        qf[s][6] = q1.w * sf[6];
    }
    // centres c = q - o (o the neighbour offset of q seen from c) inside the
    // image: columns qx - ox, rows cy with |qy - cy| <= r for some source row
    const int oxlo = max(-p.r, qx - (p.W - 1)), oxhi = min(p.r, qx);
    const int cylo = max(0, qy0 - p.r), cyhi = min(p.H - 1, qy0 + nrow - 1 + p.r);
    const int t1 = min(p.F - 1, tau + p.T - 1);
    for (int t = tau; t <= t1; ++t) {
        const float4* C0 = p.packed + (size_t)t * 2 * N;
        const float4* C1 = C0 + N;
        const float4* G = p.gv + (size_t)t * 3 * N;
        for (int cy = cylo; cy <= cyhi; ++cy) {
            for (int ox = oxlo; ox <= oxhi; ++ox) {
                const float u1 = (float)ox * s_px;
                const size_t ci = (size_t)cy * p.W + (qx - ox);
                const float4 c0 = __ldg(C0 + ci), c1 = __ldg(C1 + ci);
                const float4 g0 = __ldg(G + ci), g1 = __ldg(G + N + ci), g2 = __ldg(G + 2 * N + ci);
                const float cfv[7] = {c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                for (int s = 0; s < kSrcRows; ++s) {
                    const int oy = qy0 + s - cy;   // the same for the whole warp
                    if (s >= nrow || oy < -p.r || oy > p.r) continue;
                    const float u2 = (float)oy * s_px;
                    float u[7];
                    float en = -fmaf(u1, u1, u2 * u2);
#pragma unroll
                    for (int j = 0; j < 7; ++j) {
                        u[j] = fmaf(-cfv[j], sf[j], qf[s][j]);
                        en = fmaf(-u[j], u[j], en);
                    }
                    const float w = ex2_approx(en);
                    float vz = g0.x + g0.y * u1 + g0.z * u2;
                    vz = fmaf(g0.w, u[0], vz);
                    vz = fmaf(g1.x, u[1], vz);
                    vz = fmaf(g1.y, u[2], vz);
                    vz = fmaf(g1.z, u[3], vz);
                    vz = fmaf(g1.w, u[4], vz);
                    vz = fmaf(g2.x, u[5], vz);
                    vz = fmaf(g2.y, u[6], vz);
                    gy[s] = fmaf(w, vz, gy[s]);
                }
            }
        }
    }
    const float* rad = p.radiance + (size_t)tau * (p.rgb ? 3 : 1) * N;
    float* grad = p.g_radiance + (size_t)tau * (p.rgb ? 3 : 1) * N;
#pragma unroll
    for (int s = 0; s < kSrcRows; ++s) {
        if (s >= nrow) break;
        const size_t qi = (size_t)(qy0 + s) * p.W + qx;
        if (p.rgb) {
            const float Y = 0.2126f * rad[qi] + 0.7152f * rad[N + qi] + 0.0722f * rad[2 * N + qi];
            const float gY = gy[s] / (Y + p.log_eps);
            grad[qi] = 0.2126f * gY;
            grad[N + qi] = 0.7152f * gY;
            grad[2 * N + qi] = 0.0722f * gY;
        } else {
            grad[qi] = gy[s] / (rad[qi] + p.log_eps);
        }
    }
}

bool desc_ok(const esim_ad_wlr_desc* d)
{
    return d && d->struct_size == sizeof(esim_ad_wlr_desc) && d->width >= 1 && d->height >= 1 &&
           d->sequence >= 1 && d->radius >= 1 && d->radius <= kMaxRadius && d->frames >= 1 &&
           d->frames <= kMaxFrames && (d->radiance_fmt == ESIM_AD_LUMA_F32 || d->radiance_fmt == ESIM_AD_RGB_F32) &&
           d->h > 0.0f && d->ridge > 0.0f && d->log_eps >= 0.0f;
}

struct Layout {
    size_t packed, gv, partials, total;
    int tiles_x, n_tiles, n_blocks;
};

Layout layout(const esim_ad_wlr_desc* d)
{
    Layout L;
    const size_t N = (size_t)d->width * d->height, F = (size_t)d->sequence;
    L.tiles_x = (d->width + kTileX - 1) / kTileX;
    L.n_tiles = L.tiles_x * ((d->height + kTileY - 1) / kTileY);
    L.n_blocks = L.n_tiles * d->sequence;
    L.packed = 0;
    L.gv = L.packed + F * 2 * N * sizeof(float4);
    L.partials = L.gv + F * 3 * N * sizeof(float4);
    L.total = L.partials + (size_t)L.n_blocks * 8 * sizeof(float);
    return L;
}

AdjParams params(const esim_ad_wlr_desc* d, const Layout& L, void* ws)
{
    AdjParams p;
    p.W = d->width;
    p.H = d->height;
    p.F = d->sequence;
    p.r = d->radius;
    p.T = d->frames;
    p.tiles_x = L.tiles_x;
    p.rgb = d->radiance_fmt == ESIM_AD_RGB_F32 ? 1 : 0;
    p.h = d->h;
    p.log_eps = d->log_eps;
    p.ridge = d->ridge;
    unsigned char* base = static_cast<unsigned char*>(ws);
    p.packed = reinterpret_cast<const float4*>(base + L.packed);
    p.gv = reinterpret_cast<float4*>(base + L.gv);
    p.partials = reinterpret_cast<float*>(base + L.partials);
    p.radiance = p.features = p.bandwidth = p.g_alpha = nullptr;
    p.alpha = p.saved = p.g_radiance = p.g_bandwidth = nullptr;
    return p;
}

}  // namespace
}  // namespace esim

using namespace esim;

extern "C" size_t esim_ad_wlr_workspace_size(const esim_ad_wlr_desc* d)
{
    if (!desc_ok(d)) return 0;
    return layout(d).total;
}

extern "C" esim_ad_status esim_ad_wlr_forward(const esim_ad_wlr_desc* d, const float* radiance,
                                              const float* features, const float* bandwidth, float* alpha,
                                              float* saved, void* workspace, void* cuda_stream)
{
    if (!desc_ok(d) || !radiance || !features || !bandwidth || !alpha || !saved || !workspace)
        return ESIM_AD_EINVAL;
    const Layout L = layout(d);
    AdjParams p = params(d, L, workspace);
    p.radiance = radiance;
    p.features = features;
    p.bandwidth = bandwidth;
    p.alpha = alpha;
    p.saved = saved;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const dim3 grid(L.n_tiles, d->sequence);
    pack_kernel<<<grid, kTilePix, 0, s>>>(p);
    fwd_kernel<<<grid, kTilePix, 0, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? ESIM_AD_OK : ESIM_AD_ECUDA;
}

extern "C" esim_ad_status esim_ad_wlr_backward(const esim_ad_wlr_desc* d, const float* radiance,
                                               const float* features, const float* bandwidth,
                                               const float* saved, const float* g_alpha, float* g_radiance,
                                               float* g_bandwidth, void* workspace, void* cuda_stream)
{
    if (!desc_ok(d) || !radiance || !features || !bandwidth || !saved || !g_alpha || !g_radiance ||
        !g_bandwidth || !workspace)
        return ESIM_AD_EINVAL;
    const Layout L = layout(d);
    AdjParams p = params(d, L, workspace);
    p.radiance = radiance;
    p.features = features;
    p.bandwidth = bandwidth;
    p.saved = const_cast<float*>(saved);
    p.g_alpha = g_alpha;
    p.g_radiance = g_radiance;
    p.g_bandwidth = g_bandwidth;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const dim3 grid(L.n_tiles, d->sequence);
    bwd_center_kernel<<<grid, kCtrThreads, 0, s>>>(p);
    bwd_bandwidth_kernel<<<1, kTilePix, 0, s>>>(p, L.n_blocks);
    const dim3 grid_src(L.tiles_x * ((d->height + kSrcTileY - 1) / kSrcTileY), d->sequence);
    bwd_source_kernel<<<grid_src, kTilePix, 0, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? ESIM_AD_OK : ESIM_AD_ECUDA;
}
