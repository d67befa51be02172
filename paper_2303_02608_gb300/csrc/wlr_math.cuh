// Shared arithmetic of the weighted local regression (Eqs. 3-5): the
// per-neighbour accumulation of the Gram matrix of z = (1, u) and of the
// right-hand side, and the equilibrated Cholesky solves.  Included by the
// simulator's regression kernels and by the differentiation-form kernels.
#pragma once

#include "block_scan.cuh"
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

// FP64 Cholesky re-solve of the equilibrated FP32 system (rarely taken; kept
// out of line so that its arrays do not burden the callers' registers).
__device__ __noinline__ void solve_fp64(const float (&A)[NG], const float (&b)[NZ], float (&th)[NZ])
{
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
}

// Mixed-form solve: FP32 Cholesky of the equilibrated system plus one step of
// iterative refinement (the residual taken against the unfactored matrix),
// and an FP64 Cholesky re-solve when the condition number estimated from the
// factor's diagonal, (max L_ii / min L_ii)^2, exceeds 1e6.  Returns 1 if the
// FP64 path ran.
__device__ __forceinline__ int solve_mixed_inl(Acc& a, const float (&s2)[NZ], float ridge,
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
        solve_fp64(A, b, th);
        used64 = 1;
    }
#pragma unroll
    for (int i = 0; i < NZ; ++i) theta[i] = th[i] * dsc[i];
    return used64;
}


// Out-of-line copy for callers whose accumulation loop already holds the
// register budget (the solve then runs on the call's own frame).
__device__ __noinline__ int solve_mixed_call(Acc& a, const float (&s2)[NZ], float ridge, float (&theta)[NZ])
{
    return solve_mixed_inl(a, s2, ridge, theta);
}

// Eq. 1 at a fixed frame time, and the model update of Fig. 1.
template <bool kMixed>
__device__ __forceinline__ void emit(const WlrParams& p, int cx, int cy, const float (&theta)[NZ])
{
    const size_t N = (size_t)p.W * p.H;
    const size_t i = (size_t)cy * p.W + cx;
    const float alpha = theta[0];
    float bf[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) bf[j] = theta[3 + j] * p.s_feat[j];
    p.alpha[i] = alpha;
    float L;
    if (p.init) {
        L = alpha;
    } else {
        L = p.state[3 * N + i].w;
        const float dl = alpha - L;
        const float n = floorf(fabsf(dl) / p.C);
        if (!(n >= 1.0f)) return;  // no event: keep the model
        const float pol = dl > 0.0f ? 1.0f : -1.0f;
        L = fmaf(pol * n, p.C, L);
        p.nev[i] = (int32_t)(pol * n);
        atomicAdd(&p.chunk_cnt[i / kChunk], (uint32_t)n);
    }
    const int slot = p.t % p.T;
    float x[7];
    if (kMixed) {
        float y, q[7];
        unpack_mixed(reinterpret_cast<const uint4*>(p.ring)[(size_t)slot * N + i], y, q);
#pragma unroll
        for (int j = 0; j < 7; ++j) x[j] = q[j] * p.fscale[j];
    } else {
        const float4* ring = reinterpret_cast<const float4*>(p.ring);
        const float4 x0 = ring[(size_t)(2 * slot) * N + i];
        const float4 x1 = ring[(size_t)(2 * slot + 1) * N + i];
        x[0] = x0.y; x[1] = x0.z; x[2] = x0.w; x[3] = x1.x; x[4] = x1.y; x[5] = x1.z; x[6] = x1.w;
    }
    const float4 b0 = make_float4(bf[0], bf[1], bf[2], bf[3]);
    float4 b1 = make_float4(bf[4], bf[5], bf[6], 0.0f);
    b1.w = dot7(b0, b1, x[0], x[1], x[2], x[3], x[4], x[5], x[6]);
    p.state[i] = b0;
    p.state[N + i] = b1;
    p.state[2 * N + i] = make_float4(x[0], x[1], x[2], x[3]);
    p.state[3 * N + i] = make_float4(x[4], x[5], x[6], L);
}

// Regress one pixel from its reduced sums, then emit (both forms).  kInline:
// the mixed-form solve is inlined rather than called.
template <bool kMixed, bool kInline = false>
__device__ __forceinline__ void solve_and_emit(const WlrParams& p, Acc& acc, int cx, int cy,
                                               unsigned long long* fp64_count)
{
    float s2[NZ];
    s2[0] = 0.0f;
    s2[1] = p.s_coord * p.s_coord;
    s2[2] = s2[1];
#pragma unroll
    for (int j = 0; j < 7; ++j) s2[3 + j] = p.s_feat[j] * p.s_feat[j];
    float theta[NZ];
    if (kMixed) {
        const int used64 = kInline ? solve_mixed_inl(acc, s2, p.ridge, theta)
                                   : solve_mixed_call(acc, s2, p.ridge, theta);
        if (used64) atomicAdd(fp64_count, 1ull);
    } else {
        solve(acc, s2, p.ridge, theta);
    }
    emit<kMixed>(p, cx, cy, theta);
}

// End of a regression launch: add this CTA's work counters, record a timeout,
// and, when events are emitted, take a ticket; the last CTA to finish scans
// the per-chunk event counts into output offsets (no CTA waits on another).
__device__ __forceinline__ void finish(const WlrParams& p, unsigned long long pairs,
                                       unsigned long long pix, unsigned long long fp64, bool timed_out)
{
    __shared__ int s_timeout, s_last;
    __shared__ int s_warp[8];
    if (threadIdx.x == 0) {
        s_timeout = 0;
        s_last = 0;
    }
    __syncthreads();
    if (timed_out) s_timeout = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (pairs) atomicAdd(&p.ctrl->neighbours, pairs);
        if (pix) atomicAdd(&p.ctrl->regressions, pix);
        if (fp64) atomicAdd(&p.ctrl->fp64_solves, fp64);
        if (s_timeout) atomicOr(&p.ctrl->status, kStatusTimeout);
        if (p.emit_events) {
            __threadfence();
            const uint32_t ticket = atomicAdd(&p.ctrl->chunk_done, 1u);
            s_last = (ticket == gridDim.x - 1u) ? 1 : 0;
        }
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    unsigned long long running = *(volatile unsigned long long*)&p.ctrl->ev_total;
    const unsigned long long start = running;
    for (int base = 0; base < p.n_chunks; base += blockDim.x) {
        const int j = base + (int)threadIdx.x;
        const int v = (j < p.n_chunks) ? (int)*(volatile uint32_t*)&p.chunk_cnt[j] : 0;
        int seg;
        const int off = block_exclusive_scan(v, s_warp, seg);
        if (j < p.n_chunks) p.chunk_off[j] = running + (unsigned long long)off;
        running += (unsigned long long)seg;
    }
    if (threadIdx.x == 0) {
        p.ctrl->ev_total = running;
        p.ctrl->ev_cum += running - start;
    }
}

}  // namespace
}  // namespace esim
