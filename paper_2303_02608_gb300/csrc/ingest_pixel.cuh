// Per-pixel ingest and Proposition-1 test, shared by the single-sequence and
// the batched ingest kernels.
#pragma once

#include "internal.h"

namespace esim {
namespace {

// Store pixel i's ring record from its log brightness yv and features f
// (scaled to natural units), write its flag, and return 1 if the pixel is to
// be regressed this frame (always at frame 0 and in exhaustive mode).  Yeps is
// Y + eps when the input was linear radiance, else -1; ii is the pixel's index
// in the input planes (for the guard's variance); model() returns the pixel's
// first two model planes (beta, sigma), read only when the test runs.  For
// the mixed ring, frames already in its storage formats pass their bits
// through: with kRaw, qraw holds the BF16 features (f[j] = qraw[j] *
// fscale[j]); yraw is the FP16 log brightness, or -1; other values are
// rounded here.
template <bool kRaw, class ModelFn>
__device__ __forceinline__ int ingest_store_test(const IngestParams& p, size_t i, size_t ii, float yv, float Yeps,
                                                 float (&f)[7], const unsigned short (&qraw)[7], int yraw,
                                                 ModelFn model)
{
    const size_t N = (size_t)p.W * p.H;
    int flag = 0;
    if (p.mixed) {
        // FP16 log brightness and BF16 features; the test below sees the
        // stored (dequantised) values, as the regression will
        unsigned short q[7];
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            if (kRaw) {
                q[j] = qraw[j];
            } else {
                q[j] = __bfloat16_as_ushort(__float2bfloat16_rn(f[j] * p.inv_fscale[j]));
                f[j] = __uint_as_float((uint32_t)q[j] << 16) * p.fscale[j];
            }
        }
        const unsigned short yh = yraw >= 0 ? (unsigned short)yraw : __half_as_ushort(__float2half_rn(yv));
        reinterpret_cast<uint4*>(p.ring)[(size_t)p.slot * N + i] = pack_mixed(yh, q);
    } else {
        float4* ring = reinterpret_cast<float4*>(p.ring);
        ring[(size_t)(2 * p.slot) * N + i] = make_float4(yv, f[0], f[1], f[2]);
        ring[(size_t)(2 * p.slot + 1) * N + i] = make_float4(f[3], f[4], f[5], f[6]);
    }
    const float n0 = f[0], n1 = f[1], n2 = f[2], d = f[3], a0 = f[4], a1 = f[5], a2 = f[6];
    if (p.test) {
        // beta^T (x^c - xhat) = sigma - beta . xhat, sigma = beta . x^c kept in the model
        float4 b0, b1;
        model(b0, b1);
        const float s = b1.w - dot7(b0, b1, n0, n1, n2, d, a0, a1, a2);
        flag = (s * s >= p.C * p.C) ? 1 : 0;
        if (!flag && p.guard_kappa > 0.0f) {
            // optional guard: the log brightness itself has moved past C by
            // more than guard_kappa noise deviations (sigma_y by the delta method)
            float sigma = 0.0f;
            if (p.variance) {
                const float ye = Yeps > 0.0f ? Yeps : expf(yv);
                sigma = sqrtf(fmaxf(__ldg(p.variance + ii), 0.0f)) / ye;
            }
            const float L = p.state[3 * N + i].w;
            flag = fabsf(yv - L) >= fmaf(p.guard_kappa, sigma, p.C) ? 1 : 0;
        }
    } else {
        flag = 1;
    }
    p.flag[i] = (uint8_t)flag;
    if (!p.ev_mask) p.nev[i] = 0;   // with a mask, counts are read only where its bit is set
    return flag;
}

// Ingest pixel (x, y) of the frame described by p, reading its inputs from
// global memory: convert and store its ring record, clear its event count and
// flag, and return 1 if the pixel is to be regressed this frame.
__device__ __forceinline__ int ingest_pixel(const IngestParams& p, int x, int y)
{
    const bool inside = x < p.W && y < p.H;
    const size_t N = (size_t)p.W * p.H;
    int flag = 0;
    if (inside) {
        const size_t i = (size_t)y * p.W + x;                 // ring, model and maps (dense)
        const size_t ii = (size_t)y * p.pitch + x;            // inputs (row pitch p.pitch)
        const size_t NP = (size_t)p.H * p.pitch;              // input plane stride
        float yv;
        float Yeps = -1.0f;   // Y + eps when the input is linear radiance
        int yraw = -1;
        if (p.rad_fmt == ESIM_AD_LOGLUMA_F16) {
            const unsigned short h = reinterpret_cast<const unsigned short*>(p.rad)[ii];
            yv = __half2float(__ushort_as_half(h));
            yraw = h;
        } else {
            const float* rad = reinterpret_cast<const float*>(p.rad);
            float Y;
            if (p.rad_fmt == ESIM_AD_RGB_F32) {
                // Rec.709 luminance of the RGB radiance
                Y = 0.2126f * __ldg(rad + ii) + 0.7152f * __ldg(rad + NP + ii) + 0.0722f * __ldg(rad + 2 * NP + ii);
            } else {
                Y = __ldg(rad + ii);
            }
            Yeps = Y + p.log_eps;
            yv = logf(Yeps);
        }
        float f[7];   // normal xyz, depth, albedo rgb
        unsigned short qb[7];
        const bool bf16_in = p.feat_fmt == ESIM_AD_FEAT_BF16;
        if (bf16_in) {
#pragma unroll
            for (int j = 0; j < 7; ++j) {
                qb[j] = __ldg(p.feat_bf16 + j * NP + ii);
                f[j] = __uint_as_float((uint32_t)qb[j] << 16) * p.fscale[j];
            }
        } else {
            f[0] = __ldg(p.normal + ii);
            f[1] = __ldg(p.normal + NP + ii);
            f[2] = __ldg(p.normal + 2 * NP + ii);
            f[3] = __ldg(p.depth + ii);
            f[4] = __ldg(p.albedo + ii);
            f[5] = __ldg(p.albedo + NP + ii);
            f[6] = __ldg(p.albedo + 2 * NP + ii);
        }
        auto model = [&](float4& b0, float4& b1) {
            b0 = p.state[i];
            b1 = p.state[N + i];
        };
        if (bf16_in)
            flag = ingest_store_test<true>(p, i, ii, yv, Yeps, f, qb, yraw, model);
        else
            flag = ingest_store_test<false>(p, i, ii, yv, Yeps, f, qb, yraw, model);
    }
    return flag;
}

}  // namespace
}  // namespace esim
