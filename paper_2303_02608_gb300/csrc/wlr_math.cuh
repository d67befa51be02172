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

// ---------------------------------------------------------------------------
// Packed accumulation.  The 65 sums of the normal equations (the 55 entries of
// the Gram matrix of z = (1, u) and the 10 of the right-hand side) are held as
// float2 pairs, so that one packed FP32 instruction (two FMA lanes) updates two
// of them.  The regressors travel in five pairs
//     Q0 = (u_dx, u_dy)   Q1 = (u_ny, u_nz)   Q2 = (u_d, u_ar)
//     Q3 = (u_ag, u_ab)   Q4 = (y, u_nx)
// so that each pair comes straight out of one 8-byte half of a ring record,
// and the log brightness y rides in Q4: its products are the right-hand side.
// With wQ_k = w Q_k the sums are
//     g0 = sum w,  r_k = sum wQ_k,  s_k = sum wQ_k * Q_k,  x_k = sum wQ_k.x Q_k.y
//     d_b = sum wQ_k * Q_m,  c_b = sum wQ_k * swap(Q_m)      (k > m, b = k(k-1)/2 + m)
// (s_4.x = sum w y^2 is not needed: only s_4.y = sum w u_nx^2 is kept, as s4).
// A Gram record stores them in that order: g0, r[5], d[10], c[10], s[5] (with
// s_4.x = 0), x[5] = 66 floats, padded to 68.
struct AccP {
    float g0;
    float2 r[5];
    float2 d[10];
    float2 c[10];
    float2 s[4];
    float s4;
    float x[5];
};
constexpr int kGramFloats = 66;
constexpr int kGramStride = 68;   // floats per record (272 bytes, 16-byte aligned)
static_assert(kGramStride * 4 == kGramRecordBytes, "Gram record size");

// Per-pixel constants of the packed update: scales and negated centre terms
// of the feature pairs (a feature difference becomes f * scale - centre).
struct PairConst {
    float2 s1, s2, s3, n1, n2, n3;
    float snx, nnx;
};

__device__ __forceinline__ void accp_zero(AccP& a)
{
    a.g0 = 0.0f;
    a.s4 = 0.0f;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        a.r[k] = make_float2(0.0f, 0.0f);
        if (k < 4) a.s[k] = make_float2(0.0f, 0.0f);
        a.x[k] = 0.0f;
    }
#pragma unroll
    for (int b = 0; b < 10; ++b) {
        a.d[b] = make_float2(0.0f, 0.0f);
        a.c[b] = make_float2(0.0f, 0.0f);
    }
}

// sc[j] turns a stored feature value into its regressor scale, cf[j] = sc[j] * centre value.
__device__ __forceinline__ PairConst pair_const(const float* __restrict__ sc, const float (&cf)[7])
{
    PairConst k;
    k.snx = sc[0];
    k.nnx = -cf[0];
    k.s1 = make_float2(sc[1], sc[2]);
    k.n1 = make_float2(-cf[1], -cf[2]);
    k.s2 = make_float2(sc[3], sc[4]);
    k.n2 = make_float2(-cf[3], -cf[4]);
    k.s3 = make_float2(sc[5], sc[6]);
    k.n3 = make_float2(-cf[5], -cf[6]);
    return k;
}

// One neighbour: q0 = (u_dx, u_dy) and en0 = -(u_dx^2 + u_dy^2) of its offset,
// its log brightness y and its seven features as (n_x) and pairs (n_y, n_z),
// (d, a_r), (a_g, a_b).
__device__ __forceinline__ void accp_core(AccP& a, float2 q0, float en0, float y, float fnx, float2 f1,
                                          float2 f2, float2 f3, const PairConst& k)
{
    float2 Q[5];
    Q[0] = q0;
    Q[1] = __ffma2_rn(f1, k.s1, k.n1);
    Q[2] = __ffma2_rn(f2, k.s2, k.n2);
    Q[3] = __ffma2_rn(f3, k.s3, k.n3);
    const float unx = fmaf(fnx, k.snx, k.nnx);
    Q[4] = make_float2(y, unx);
    float2 sq = __fmul2_rn(Q[1], Q[1]);
    sq = __ffma2_rn(Q[2], Q[2], sq);
    sq = __ffma2_rn(Q[3], Q[3], sq);
    const float e = fmaf(unx, unx, sq.x) + sq.y;
    const float w = ex2_approx(en0 - e);
    const float2 w2 = make_float2(w, w);
    float2 wQ[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) wQ[i] = __fmul2_rn(w2, Q[i]);
    a.g0 += w;
#pragma unroll
    for (int i = 0; i < 5; ++i) a.r[i] = __fadd2_rn(a.r[i], wQ[i]);
#pragma unroll
    for (int i = 1; i < 5; ++i) {
#pragma unroll
        for (int m = 0; m < i; ++m) {
            const int b = i * (i - 1) / 2 + m;
            a.d[b] = __ffma2_rn(wQ[i], Q[m], a.d[b]);
            a.c[b] = __ffma2_rn(wQ[i], make_float2(Q[m].y, Q[m].x), a.c[b]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) a.s[i] = __ffma2_rn(wQ[i], Q[i], a.s[i]);
    a.s4 = fmaf(wQ[4].y, unx, a.s4);
#pragma unroll
    for (int i = 0; i < 5; ++i) a.x[i] = fmaf(wQ[i].x, Q[i].y, a.x[i]);
}

// FP32 ring: h0 = (y, n_x, n_y, n_z), h1 = (d, a_r, a_g, a_b).
__device__ __forceinline__ void accp(AccP& a, const float4 h0, const float4 h1, float2 q0, float en0,
                                     const PairConst& k)
{
    accp_core(a, q0, en0, h0.x, h0.y, make_float2(h0.z, h0.w), make_float2(h1.x, h1.y),
              make_float2(h1.z, h1.w), k);
}

// Mixed ring record (FP16 y, BF16 stored features).
__device__ __forceinline__ void accp(AccP& a, const uint4 v, float2 q0, float en0, const PairConst& k)
{
    const float y = __half2float(__ushort_as_half((unsigned short)(v.x & 0xffffu)));
    const float fnx = __uint_as_float(v.x & 0xffff0000u);
    accp_core(a, q0, en0, y, fnx, make_float2(__uint_as_float(v.y << 16), __uint_as_float(v.y & 0xffff0000u)),
              make_float2(__uint_as_float(v.z << 16), __uint_as_float(v.z & 0xffff0000u)),
              make_float2(__uint_as_float(v.w << 16), __uint_as_float(v.w & 0xffff0000u)), k);
}

// Butterfly sum over the g lanes (a power of two, aligned) that share a pixel.
__device__ __forceinline__ void accp_reduce(AccP& a, int g)
{
    for (int off = g >> 1; off >= 1; off >>= 1) {
        a.g0 += __shfl_xor_sync(0xffffffffu, a.g0, off);
        a.s4 += __shfl_xor_sync(0xffffffffu, a.s4, off);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            a.r[i].x += __shfl_xor_sync(0xffffffffu, a.r[i].x, off);
            a.r[i].y += __shfl_xor_sync(0xffffffffu, a.r[i].y, off);
            if (i < 4) {
                a.s[i].x += __shfl_xor_sync(0xffffffffu, a.s[i].x, off);
                a.s[i].y += __shfl_xor_sync(0xffffffffu, a.s[i].y, off);
            }
            a.x[i] += __shfl_xor_sync(0xffffffffu, a.x[i], off);
        }
#pragma unroll
        for (int b = 0; b < 10; ++b) {
            a.d[b].x += __shfl_xor_sync(0xffffffffu, a.d[b].x, off);
            a.d[b].y += __shfl_xor_sync(0xffffffffu, a.d[b].y, off);
            a.c[b].x += __shfl_xor_sync(0xffffffffu, a.c[b].x, off);
            a.c[b].y += __shfl_xor_sync(0xffffffffu, a.c[b].y, off);
        }
    }
}

// The sums in Gram-record order (kGramStride floats, the last two zero).
__device__ __forceinline__ void accp_values(const AccP& a, float (&v)[kGramStride])
{
    v[0] = a.g0;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        v[1 + 2 * i] = a.r[i].x;
        v[2 + 2 * i] = a.r[i].y;
        v[51 + 2 * i] = i < 4 ? a.s[i].x : 0.0f;
        v[52 + 2 * i] = i < 4 ? a.s[i].y : a.s4;
        v[61 + i] = a.x[i];
    }
#pragma unroll
    for (int b = 0; b < 10; ++b) {
        v[11 + 2 * b] = a.d[b].x;
        v[12 + 2 * b] = a.d[b].y;
        v[31 + 2 * b] = a.c[b].x;
        v[32 + 2 * b] = a.c[b].y;
    }
    v[66] = 0.0f;
    v[67] = 0.0f;
}

// Store the sums as one Gram record (rec: kGramStride floats, 16-byte aligned).
// The g lanes of a pixel (all holding the reduced sums) split the 17 16-byte
// pieces; sub is the lane's index among them.
__device__ __forceinline__ void accp_store(const AccP& a, float* __restrict__ rec, int sub, int g)
{
    float v[kGramStride];
    accp_values(a, v);
    float4* out = reinterpret_cast<float4*>(rec);
#pragma unroll
    for (int q = 0; q < kGramStride / 4; ++q)
        if ((q & (g - 1)) == sub) out[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// Natural index (0 = intercept, 1-2 = coordinates, 3-9 = features n_x, n_y,
// n_z, d, a_r, a_g, a_b, 10 = log brightness) of component h of pair k.
__host__ __device__ constexpr int pair_nat(int k, int h)
{
    return k == 0 ? 1 + h : k == 1 ? 4 + h : k == 2 ? 6 + h : k == 3 ? 8 + h : (h == 0 ? 10 : 3);
}

// Row and column (natural indices) of slot s of a Gram record.
__host__ __device__ constexpr int block_k(int b) { return b >= 6 ? 4 : b >= 3 ? 3 : b >= 1 ? 2 : 1; }
__host__ __device__ constexpr int block_m(int b) { return b - block_k(b) * (block_k(b) - 1) / 2; }

__host__ __device__ constexpr int slot_i(int s)
{
    return s == 0 ? 0
         : s < 11 ? pair_nat((s - 1) / 2, (s - 1) & 1)
         : s < 31 ? pair_nat(block_k((s - 11) / 2), (s - 11) & 1)
         : s < 51 ? pair_nat(block_k((s - 31) / 2), (s - 31) & 1)
         : s < 61 ? pair_nat((s - 51) / 2, (s - 51) & 1)
         : pair_nat(s - 61, 0);
}

__host__ __device__ constexpr int slot_j(int s)
{
    return s == 0 ? 0
         : s < 11 ? 0
         : s < 31 ? pair_nat(block_m((s - 11) / 2), (s - 11) & 1)
         : s < 51 ? pair_nat(block_m((s - 31) / 2), 1 - ((s - 31) & 1))
         : s < 61 ? pair_nat((s - 51) / 2, (s - 51) & 1)
         : pair_nat(s - 61, 1);
}

// Unpack a Gram record into the packed triangle and right-hand side.
__device__ __forceinline__ void gram_load(const float* __restrict__ rec, Acc& a)
{
    float v[kGramStride];
    const float4* in = reinterpret_cast<const float4*>(rec);
#pragma unroll
    for (int q = 0; q < kGramStride / 4; ++q) {
        const float4 t = in[q];
        v[4 * q] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
    }
#pragma unroll
    for (int s = 0; s < kGramFloats; ++s) {
        const int i = slot_i(s), j = slot_j(s);
        if (i == 10 && j == 10) continue;
        if (i == 10) a.B[j] = v[s];
        else if (j == 10) a.B[i] = v[s];
        else a.G[i >= j ? tri(i, j) : tri(j, i)] = v[s];
    }
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

// Mixed-form solve of one Gram record: FP32 Cholesky of the ridged,
// Jacobi-equilibrated system A plus one step of iterative refinement, whose
// residual is taken against the unfactored system re-read from the record,
// 16 bytes at a time (so that the factor can overwrite the matrix in
// registers).  The 2-norm condition number of A is estimated as
// lambda_max / lambda_min with lambda_max bounded by the largest absolute row
// sum (Gershgorin) and 1 / lambda_min by two steps of inverse iteration
// through the factor from a fixed start vector.  Returns false, leaving theta
// unset, when the estimate exceeds 1e6: such systems are accumulated again
// with compensated sums and solved in FP64.
__device__ __forceinline__ bool solve_refined_rec(const float* __restrict__ rec, const float (&s2)[NZ], float ridge,
                                                  float (&theta)[NZ])
{
    Acc a;
    gram_load(rec, a);
    const float rW = ridge * a.G[0];
#pragma unroll
    for (int j = 1; j < NZ; ++j) a.G[tri(j, j)] = fmaf(rW, s2[j], a.G[tri(j, j)]);
    float dsc[NZ], b[NZ];
#pragma unroll
    for (int i = 0; i < NZ; ++i) dsc[i] = rsqrtf(a.G[tri(i, i)]);
#pragma unroll
    for (int i = 0; i < NZ; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) a.G[tri(i, j)] *= dsc[i] * dsc[j];
        b[i] = a.B[i] * dsc[i];
    }
    float inv[NZ];
#pragma unroll
    for (int j = 0; j < NZ; ++j) {
        float sj = a.G[tri(j, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) sj = fmaf(-a.G[tri(j, k)], a.G[tri(j, k)], sj);
        sj = fmaxf(sj, 1e-20f);
        const float l = sqrtf(sj);
        a.G[tri(j, j)] = l;
        inv[j] = 1.0f / l;
#pragma unroll
        for (int i = j + 1; i < NZ; ++i) {
            float v = a.G[tri(i, j)];
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
    // 1 / lambda_min: two steps of inverse iteration from a fixed unit vector
    float x1[NZ], x2[NZ];
    {
        float v0[NZ];
#pragma unroll
        for (int i = 0; i < NZ; ++i) v0[i] = (i & 1) ? -0.31622777f : 0.31622777f;   // (+-1) / sqrt(10)
        llt_solve(v0, x1);
        float n1 = 0.0f;
#pragma unroll
        for (int i = 0; i < NZ; ++i) n1 = fmaf(x1[i], x1[i], n1);
        const float s1 = rsqrtf(fmaxf(n1, 1e-30f));
#pragma unroll
        for (int i = 0; i < NZ; ++i) x1[i] *= s1;
        llt_solve(x1, x2);
    }
    float inv_lmin = 0.0f;
#pragma unroll
    for (int i = 0; i < NZ; ++i) inv_lmin = fmaf(x2[i], x2[i], inv_lmin);
    inv_lmin = sqrtf(inv_lmin);
    float th[NZ];
    llt_solve(b, th);
    // r = b - A th with A re-read from the record; the same pass takes A's
    // absolute row sums (Gershgorin bound on lambda_max)
    float r[NZ], rowsum[NZ];
#pragma unroll
    for (int i = 0; i < NZ; ++i) {
        r[i] = b[i];
        rowsum[i] = 0.0f;
    }
    const float4* r4 = reinterpret_cast<const float4*>(rec);
#pragma unroll
    for (int q = 0; q < kGramStride / 4; ++q) {
        const float4 v4 = __ldg(r4 + q);
        const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int sl = 4 * q + k;
            if (sl >= kGramFloats) continue;
            const int i = slot_i(sl), j = slot_j(sl);
            if (i == 10 || j == 10) continue;   // right-hand side (already in b)
            float g = vv[k];
            if (i == j && i > 0) g = fmaf(rW, s2[i], g);
            const float aij = g * (dsc[i] * dsc[j]);
            r[i] = fmaf(-aij, th[j], r[i]);
            rowsum[i] += fabsf(aij);
            if (i != j) {
                r[j] = fmaf(-aij, th[i], r[j]);
                rowsum[j] += fabsf(aij);
            }
        }
    }
    float lmax = 0.0f;
#pragma unroll
    for (int i = 0; i < NZ; ++i) lmax = fmaxf(lmax, rowsum[i]);
    if (!(lmax * inv_lmin <= 1e6f)) return false;
    float dth[NZ];
    llt_solve(r, dth);
#pragma unroll
    for (int i = 0; i < NZ; ++i) theta[i] = (th[i] + dth[i]) * dsc[i];
    return true;
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
        float n = floorf(fabsf(dl) / p.C);
        if (!(n >= 1.0f)) return;  // no event: keep the model
        if (n > (float)kMaxCountPerPixel) {   // beyond what the writer's counts hold
            n = (float)kMaxCountPerPixel;
            atomicOr(&p.ctrl->status, kStatusOverflow);
        }
        const float pol = dl > 0.0f ? 1.0f : -1.0f;
        L = fmaf(pol * n, p.C, L);
        p.nev[i] = (int32_t)(pol * n);
        atomicAdd(&p.chunk_cnt[i / kChunk], (uint32_t)n);
        if (p.ev_mask) atomicOr(&p.ev_mask[i >> 5], 1u << (i & 31u));
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

// End of a regression launch: add this CTA's work counters, record a timeout,
// and, when events are emitted by this launch (scan), take a ticket; the last
// CTA to finish scans the per-chunk event counts into output offsets (no CTA
// waits on another).
__device__ __forceinline__ void finish(const WlrParams& p, unsigned long long pairs,
                                       unsigned long long pix, unsigned long long fp64, bool timed_out,
                                       bool scan = true)
{
    __shared__ int s_timeout, s_last;
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
        if (scan && p.emit_events) {
            __threadfence();
            const uint32_t ticket = atomicAdd(&p.ctrl->chunk_done, 1u);
            s_last = (ticket == gridDim.x - 1u) ? 1 : 0;
        }
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // last CTA: exclusive scan of the per-chunk event counts, in chunk order;
    // each thread takes a run of consecutive chunks (all its loads in flight at once)
    __shared__ unsigned long long s_warp64[8];
    const int per = (p.n_chunks + (int)blockDim.x - 1) / (int)blockDim.x;
    const int j0 = (int)threadIdx.x * per;
    const int j1 = min(j0 + per, p.n_chunks);
    unsigned long long mine = 0;
    for (int j = j0; j < j1; ++j) mine += *(volatile uint32_t*)&p.chunk_cnt[j];
    unsigned long long seg;
    const unsigned long long start = *(volatile unsigned long long*)&p.ctrl->ev_total;
    unsigned long long off = start + block_exclusive_scan64(mine, s_warp64, seg);
    for (int j = j0; j < j1; ++j) {
        p.chunk_off[j] = off;
        off += *(volatile uint32_t*)&p.chunk_cnt[j];
    }
    if (threadIdx.x == 0) {
        p.ctrl->ev_total = start + seg;
        p.ctrl->ev_cum += seg;
    }
}

}  // namespace
}  // namespace esim
