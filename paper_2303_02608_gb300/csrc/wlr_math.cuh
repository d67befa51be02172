// Shared arithmetic of the weighted local regression (Eqs. 3-5): the
// per-neighbour accumulation of the Gram matrix of z = (1, u) and of the
// right-hand side, and the equilibrated Cholesky solves.  Included by the
// simulator's regression kernels and by the differentiation-form kernels.
#pragma once

#include "internal.h"
#include "ptx.cuh"

namespace esim {
// internal linkage: each translation unit gets its own copy
namespace {

constexpr int NZ = 10;  // z = (1, u_dx, u_dy, u_feat[7])
constexpr int NG = NZ * (NZ + 1) / 2;

__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

struct Acc {
    float G[NG];
    float B[NZ];
};

// One neighbour with log brightness y and seven feature values f (raw
// features, or the stored values of the mixed form); sc[j] turns a feature
// difference into its regressor, cf[j] = sc[j] * f_centre[j].
__device__ __forceinline__ void accum_core(Acc& a, float y, float f0, float f1, float f2, float f3,
                                           float f4, float f5, float f6, float u1, float u2,
                                           float en0, const float* __restrict__ sc,
                                           const float (&cf)[7])
{
    float u[NZ];
    u[0] = 1.0f;
    u[1] = u1;
    u[2] = u2;
    u[3] = fmaf(f0, sc[0], -cf[0]);
    u[4] = fmaf(f1, sc[1], -cf[1]);
    u[5] = fmaf(f2, sc[2], -cf[2]);
    u[6] = fmaf(f3, sc[3], -cf[3]);
    u[7] = fmaf(f4, sc[4], -cf[4]);
    u[8] = fmaf(f5, sc[5], -cf[5]);
    u[9] = fmaf(f6, sc[6], -cf[6]);
    float en = en0;  // -(u1^2 + u2^2)
#pragma unroll
    for (int j = 3; j < NZ; ++j) en = fmaf(-u[j], u[j], en);
    const float w = ex2_approx(en);
    const float wy = w * y;
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

// FP32 ring: h0 = (y, normal xyz), h1 = (depth, albedo rgb).
__device__ __forceinline__ void accumulate(Acc& a, const float4 h0, const float4 h1, float u1,
                                           float u2, float en0, const float* __restrict__ sf,
                                           const float (&cf)[7])
{
    accum_core(a, h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w, u1, u2, en0, sf, cf);
}

// Mixed ring: one 16-byte record (FP16 y, BF16 stored features).
__device__ __forceinline__ void accumulate(Acc& a, const uint4 v, float u1, float u2, float en0,
                                           const float* __restrict__ qs, const float (&cf)[7])
{
    float y, q[7];
    unpack_mixed(v, y, q);
    accum_core(a, y, q[0], q[1], q[2], q[3], q[4], q[5], q[6], u1, u2, en0, qs, cf);
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

// Mixed-form solve: FP32 Cholesky of the equilibrated system plus one step of
// iterative refinement (the residual taken against the unfactored matrix),
// and an FP64 Cholesky re-solve when the condition number estimated from the
// factor's diagonal, (max L_ii / min L_ii)^2, exceeds 1e6.  Returns 1 if the
// FP64 path ran.
__device__ __noinline__ int solve_mixed(Acc& a, const float (&s2)[NZ], float ridge,
                                        float (&theta)[NZ])
{
    const float W = a.G[0];
#pragma unroll
    for (int j = 1; j < NZ; ++j) a.G[tri(j, j)] = fmaf(ridge * W, s2[j], a.G[tri(j, j)]);
    float dsc[NZ];
#pragma unroll
    for (int i = 0; i < NZ; ++i) dsc[i] = rsqrtf(a.G[tri(i, i)]);
    float A[NG], b[NZ];
#pragma unroll
    for (int i = 0; i < NZ; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) A[tri(i, j)] = a.G[tri(i, j)] * (dsc[i] * dsc[j]);
        b[i] = a.B[i] * dsc[i];
    }
    // factor into a.G
    float inv[NZ];
    float lmin = 3.4e38f, lmax = 0.0f;
#pragma unroll
    for (int j = 0; j < NZ; ++j) {
        float sj = A[tri(j, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) sj = fmaf(-a.G[tri(j, k)], a.G[tri(j, k)], sj);
        sj = fmaxf(sj, 1e-20f);
        const float l = sqrtf(sj);
        lmin = fminf(lmin, l);
        lmax = fmaxf(lmax, l);
        a.G[tri(j, j)] = l;
        inv[j] = 1.0f / l;
#pragma unroll
        for (int i = j + 1; i < NZ; ++i) {
            float v = A[tri(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) v = fmaf(-a.G[tri(i, k)], a.G[tri(j, k)], v);
            a.G[tri(i, j)] = v * inv[j];
        }
    }
    auto llt_solve = [&](const float (&rhs)[NZ], float (&x)[NZ]) {
        float z[NZ];
#pragma unroll
        for (int i = 0; i < NZ; ++i) {
            float v = rhs[i];
#pragma unroll
            for (int k = 0; k < i; ++k) v = fmaf(-a.G[tri(i, k)], z[k], v);
            z[i] = v * inv[i];
        }
#pragma unroll
        for (int i = NZ - 1; i >= 0; --i) {
            float v = z[i];
#pragma unroll
            for (int k = i + 1; k < NZ; ++k) v = fmaf(-a.G[tri(k, i)], x[k], v);
            x[i] = v * inv[i];
        }
    };
    float th[NZ];
    llt_solve(b, th);
    // one refinement step: r = b - A th, th += (L L^T)^-1 r
    float r[NZ];
#pragma unroll
    for (int i = 0; i < NZ; ++i) {
        float v = b[i];
#pragma unroll
        for (int j = 0; j < NZ; ++j) v = fmaf(-A[i >= j ? tri(i, j) : tri(j, i)], th[j], v);
        r[i] = v;
    }
    float dth[NZ];
    llt_solve(r, dth);
#pragma unroll
    for (int i = 0; i < NZ; ++i) th[i] += dth[i];
    int used64 = 0;
    const float ratio = lmax / lmin;
    if (ratio * ratio > 1e6f) {
        // FP64 Cholesky of the same equilibrated FP32 system
        double L[NG];
        double dinv[NZ];
        for (int j = 0; j < NZ; ++j) {
            double sj = (double)A[tri(j, j)];
            for (int k = 0; k < j; ++k) sj -= L[tri(j, k)] * L[tri(j, k)];
            sj = sj > 1e-300 ? sj : 1e-300;
            const double l = sqrt(sj);
            L[tri(j, j)] = l;
            dinv[j] = 1.0 / l;
            for (int i = j + 1; i < NZ; ++i) {
                double v = (double)A[tri(i, j)];
                for (int k = 0; k < j; ++k) v -= L[tri(i, k)] * L[tri(j, k)];
                L[tri(i, j)] = v * dinv[j];
            }
        }
        double z[NZ], x[NZ];
        for (int i = 0; i < NZ; ++i) {
            double v = (double)b[i];
            for (int k = 0; k < i; ++k) v -= L[tri(i, k)] * z[k];
            z[i] = v * dinv[i];
        }
        for (int i = NZ - 1; i >= 0; --i) {
            double v = z[i];
            for (int k = i + 1; k < NZ; ++k) v -= L[tri(k, i)] * x[k];
            x[i] = v * dinv[i];
        }
        for (int i = 0; i < NZ; ++i) th[i] = (float)x[i];
        used64 = 1;
    }
#pragma unroll
    for (int i = 0; i < NZ; ++i) theta[i] = th[i] * dsc[i];
    return used64;
}


}  // namespace
}  // namespace esim
