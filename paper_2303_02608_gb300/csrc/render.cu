// Monte Carlo renderer for analytic test scenes: produces the simulator's
// inputs (noisy radiance, variance of the luminance estimate, first-hit
// normal, depth and albedo) for an open-fronted room with an area light and
// moving spheres.  Every floating-point operation is an explicitly rounded
// IEEE FP32 operation (no fused multiply-add contraction), so each pixel is a
// fixed function of scene, frame and seed that a plain FP32 restatement can
// reproduce bit for bit.
//
// One thread per pixel; samples in order; per sample a jittered camera ray
// and up to max_bounces surface interactions, each with next-event estimation
// towards one uniform point of the light and a cosine-weighted bounce.
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key
// (seed, frame), counter (pixel, sample, call, 0); call 1 gives the pixel
// jitter, call 2b + 2 the light point and bounce direction of interaction b.
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace esim {
namespace {

// explicitly rounded FP32 arithmetic
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fd(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fq(float a) { return __fsqrt_rn(a); }

struct V3 {
    float x, y, z;
};
__device__ __forceinline__ V3 v3(float x, float y, float z) { return V3{x, y, z}; }
__device__ __forceinline__ V3 vsub(V3 a, V3 b) { return v3(fs(a.x, b.x), fs(a.y, b.y), fs(a.z, b.z)); }
__device__ __forceinline__ V3 vscale(V3 a, float s) { return v3(fm(a.x, s), fm(a.y, s), fm(a.z, s)); }
__device__ __forceinline__ float vdot(V3 a, V3 b) { return fa(fa(fm(a.x, b.x), fm(a.y, b.y)), fm(a.z, b.z)); }
// o + t d
__device__ __forceinline__ V3 vray(V3 o, float t, V3 d) { return v3(fa(o.x, fm(t, d.x)), fa(o.y, fm(t, d.y)), fa(o.z, fm(t, d.z))); }

// Philox4x32-10 bijection of a 128-bit counter under a 64-bit key.
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// uniform in [0, 1): the top 24 bits of a word, exactly representable
__device__ __forceinline__ float unit(uint32_t w) { return fm((float)(w >> 8), 5.9604644775390625e-8f); }

// cos and sin of 2 pi u, u in [0, 1): quarter-turn reduction, then the
// Taylor polynomials of sin and cos on [0, pi/2) (truncation below 1e-7).
__device__ __forceinline__ void sincos_turns(float u, float& c, float& s)
{
    const float u4 = fm(u, 4.0f);
    const float qf = floorf(u4);
    const int q = (int)qf;
    const float th = fm(fs(u4, qf), 1.57079637f);
    const float t2 = fm(th, th);
    float ps = -2.50521084e-8f;   // -1/11!
    ps = fa(fm(ps, t2), 2.75573188e-6f);
    ps = fa(fm(ps, t2), -1.98412701e-4f);
    ps = fa(fm(ps, t2), 8.33333377e-3f);
    ps = fa(fm(ps, t2), -1.66666672e-1f);
    ps = fa(fm(ps, t2), 1.0f);
    const float sn = fm(ps, th);
    float pc = 2.08767570e-9f;    // 1/12!
    pc = fa(fm(pc, t2), -2.75573188e-7f);
    pc = fa(fm(pc, t2), 2.48015876e-5f);
    pc = fa(fm(pc, t2), -1.38888892e-3f);
    pc = fa(fm(pc, t2), 4.16666679e-2f);
    pc = fa(fm(pc, t2), -0.5f);
    const float cs = fa(fm(pc, t2), 1.0f);
    if (q == 0) { c = cs; s = sn; }
    else if (q == 1) { c = -sn; s = cs; }
    else if (q == 2) { c = -cs; s = -sn; }
    else { c = sn; s = -cs; }
}

struct Hit {
    float t;
    int kind;   // 0..4 walls (left, right, floor, ceiling, back), 5 open front, 8 + j sphere j
};

// nearest sphere hit beyond eps (t = INF if none)
__device__ __forceinline__ Hit hit_spheres(const esim_ad_render_scene& sc, const V3* ctr, V3 o, V3 d)
{
    Hit h{INFINITY, -1};
    for (int j = 0; j < sc.n_spheres; ++j) {
        const V3 oc = vsub(o, ctr[j]);
        const float b = vdot(oc, d);
        const float cc = fs(vdot(oc, oc), fm(sc.spheres[j].radius, sc.spheres[j].radius));
        const float disc = fs(fm(b, b), cc);
        if (!(disc > 0.0f)) continue;
        const float sq = fq(disc);
        float t = fs(-b, sq);
        if (!(t > sc.eps)) t = fa(-b, sq);
        if (t > sc.eps && t < h.t) {
            h.t = t;
            h.kind = 8 + j;
        }
    }
    return h;
}

// the wall (or the open front) a ray from inside the room reaches
__device__ __forceinline__ Hit hit_walls(const esim_ad_render_scene& sc, V3 o, V3 d)
{
    Hit h{INFINITY, 5};
    if (d.x > 0.0f) { h.t = fd(fs(sc.box[0], o.x), d.x); h.kind = 1; }
    else if (d.x < 0.0f) { h.t = fd(fs(-sc.box[0], o.x), d.x); h.kind = 0; }
    float t;
    if (d.y > 0.0f) { t = fd(fs(sc.box[1], o.y), d.y); if (t < h.t) { h.t = t; h.kind = 3; } }
    else if (d.y < 0.0f) { t = fd(fs(-sc.box[1], o.y), d.y); if (t < h.t) { h.t = t; h.kind = 2; } }
    if (d.z < 0.0f) { t = fd(fs(-sc.box[2], o.z), d.z); if (t < h.t) { h.t = t; h.kind = 4; } }
    else if (d.z > 0.0f) { t = fd(fs(sc.box[2], o.z), d.z); if (t < h.t) { h.t = t; h.kind = 5; } }
    return h;
}

struct Surf {
    V3 n;
    float a[3];
    bool light;
};

__device__ __forceinline__ Surf surface(const esim_ad_render_scene& sc, const V3* ctr, int kind, V3 x)
{
    Surf s;
    s.light = false;
    if (kind >= 8) {
        const int j = kind - 8;
        const float inv_r = fd(1.0f, sc.spheres[j].radius);
        s.n = vscale(vsub(x, ctr[j]), inv_r);
        for (int c = 0; c < 3; ++c) s.a[c] = sc.spheres[j].albedo[c];
        return s;
    }
    const float nx[5] = {1.0f, -1.0f, 0.0f, 0.0f, 0.0f};
    const float ny[5] = {0.0f, 0.0f, 1.0f, -1.0f, 0.0f};
    const float nz[5] = {0.0f, 0.0f, 0.0f, 0.0f, 1.0f};
    s.n = v3(nx[kind], ny[kind], nz[kind]);
    for (int c = 0; c < 3; ++c) s.a[c] = sc.wall_albedo[kind][c];
    if (kind == 4 && sc.checker > 0.0f) {
        const float ix = floorf(fd(x.x, sc.checker)), iy = floorf(fd(x.y, sc.checker));
        if (((int)ix + (int)iy) & 1)
            for (int c = 0; c < 3; ++c) s.a[c] = sc.back_albedo2[c];
    }
    if (kind == 3 && x.x >= sc.light[0] && x.x <= sc.light[1] && x.z >= sc.light[2] && x.z <= sc.light[3])
        s.light = true;
    return s;
}

__global__ void render_kernel(const esim_ad_render_scene sc, int frame, float* __restrict__ radiance,
                              float* __restrict__ variance, float* __restrict__ normal,
                              float* __restrict__ albedo, float* __restrict__ depth)
{
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    const int py = blockIdx.y * blockDim.y + threadIdx.y;
    if (px >= sc.width || py >= sc.height) return;
    const size_t N = (size_t)sc.width * sc.height;
    const uint32_t pix = (uint32_t)py * (uint32_t)sc.width + (uint32_t)px;
    V3 ctr[8];
    const float tf = (float)frame;
    for (int j = 0; j < sc.n_spheres; ++j)
        ctr[j] = v3(fa(sc.spheres[j].center[0], fm(tf, sc.spheres[j].velocity[0])),
                    fa(sc.spheres[j].center[1], fm(tf, sc.spheres[j].velocity[1])),
                    fa(sc.spheres[j].center[2], fm(tf, sc.spheres[j].velocity[2])));
    const float tany = sc.tan_half_fov_y;
    const float tanx = fd(fm(tany, (float)sc.width), (float)sc.height);
    const float lw = fs(sc.light[1], sc.light[0]), lh = fs(sc.light[3], sc.light[2]);
    const float area = fm(lw, lh);
    const V3 cam = v3(sc.cam_pos[0], sc.cam_pos[1], sc.cam_pos[2]);
    float sum[3] = {0.0f, 0.0f, 0.0f}, sy = 0.0f, sy2 = 0.0f;
    float fn[3] = {0.0f, 0.0f, 0.0f}, fal[3] = {0.0f, 0.0f, 0.0f}, fdp = 0.0f;
    for (int smp = 0; smp < sc.spp; ++smp) {
        const uint4 jit = philox(pix, (uint32_t)smp, 1u, 0u, sc.seed, (uint32_t)frame);
        const float sxp = fm(fs(fm(fd(fa((float)px, unit(jit.x)), (float)sc.width), 2.0f), 1.0f), tanx);
        const float syp = fm(fs(1.0f, fm(fd(fa((float)py, unit(jit.y)), (float)sc.height), 2.0f)), tany);
        const float inv = fd(1.0f, fq(fa(fa(fm(sxp, sxp), fm(syp, syp)), 1.0f)));
        V3 o = cam;
        V3 d = v3(fm(sxp, inv), fm(syp, inv), -inv);
        float thr[3] = {1.0f, 1.0f, 1.0f};
        float L[3] = {0.0f, 0.0f, 0.0f};
        for (int b = 0; b < sc.max_bounces; ++b) {
            const Hit hw = hit_walls(sc, o, d);
            const Hit hsph = hit_spheres(sc, ctr, o, d);
            const Hit h = hsph.t < hw.t ? hsph : hw;
            if (h.kind == 5) break;   // out through the open front
            const V3 x = vray(o, h.t, d);
            const Surf s = surface(sc, ctr, h.kind, x);
            if (b == 0) {
                fn[0] = fa(fn[0], s.n.x);
                fn[1] = fa(fn[1], s.n.y);
                fn[2] = fa(fn[2], s.n.z);
                for (int c = 0; c < 3; ++c) fal[c] = fa(fal[c], s.a[c]);
                fdp = fa(fdp, h.t);
            }
            if (s.light) {
                if (b == 0)
                    for (int c = 0; c < 3; ++c) L[c] = fa(L[c], sc.light_radiance[c]);
                break;
            }
            const uint4 r = philox(pix, (uint32_t)smp, (uint32_t)(2 * b + 2), 0u, sc.seed, (uint32_t)frame);
            // next-event estimation: one uniform point of the light
            const V3 lp = v3(fa(sc.light[0], fm(unit(r.x), lw)), sc.box[1], fa(sc.light[2], fm(unit(r.y), lh)));
            const V3 w = vsub(lp, x);
            const float d2 = vdot(w, w);
            const float dist = fq(d2);
            const V3 wl = vscale(w, fd(1.0f, dist));
            const float cs = vdot(s.n, wl);
            const float cl = wl.y;
            if (cs > 0.0f && cl > 0.0f) {
                const Hit sh = hit_spheres(sc, ctr, x, wl);
                if (!(sh.t < fs(dist, sc.eps))) {
                    const float g = fd(fm(fm(cs, cl), area), fm(3.14159274f, d2));
                    for (int c = 0; c < 3; ++c)
                        L[c] = fa(L[c], fm(fm(fm(thr[c], s.a[c]), sc.light_radiance[c]), g));
                }
            }
            if (b + 1 >= sc.max_bounces) break;
            // cosine-weighted bounce around n (basis of Duff et al. 2017)
            float cph, sph;
            sincos_turns(unit(r.w), cph, sph);
            const float rr = fq(unit(r.z));
            const float lz = fq(fmaxf(fs(1.0f, unit(r.z)), 0.0f));
            const float lx = fm(rr, cph), ly = fm(rr, sph);
            const float sg = s.n.z >= 0.0f ? 1.0f : -1.0f;
            const float aa = fd(-1.0f, fa(sg, s.n.z));
            const float bb = fm(fm(s.n.x, s.n.y), aa);
            const V3 t1 = v3(fa(1.0f, fm(fm(sg, fm(s.n.x, s.n.x)), aa)), fm(sg, bb), -fm(sg, s.n.x));
            const V3 t2 = v3(bb, fa(sg, fm(fm(s.n.y, s.n.y), aa)), -s.n.y);
            d = v3(fa(fa(fm(t1.x, lx), fm(t2.x, ly)), fm(s.n.x, lz)),
                   fa(fa(fm(t1.y, lx), fm(t2.y, ly)), fm(s.n.y, lz)),
                   fa(fa(fm(t1.z, lx), fm(t2.z, ly)), fm(s.n.z, lz)));
            o = x;
            for (int c = 0; c < 3; ++c) thr[c] = fm(thr[c], s.a[c]);
        }
        for (int c = 0; c < 3; ++c) sum[c] = fa(sum[c], L[c]);
        const float Y = fa(fa(fm(0.2126f, L[0]), fm(0.7152f, L[1])), fm(0.0722f, L[2]));
        sy = fa(sy, Y);
        sy2 = fa(sy2, fm(Y, Y));
    }
    const float n = (float)sc.spp;
    for (int c = 0; c < 3; ++c) {
        radiance[c * N + pix] = fd(sum[c], n);
        normal[c * N + pix] = fd(fn[c], n);
        albedo[c * N + pix] = fd(fal[c], n);
    }
    depth[pix] = fd(fdp, n);
    float v = 0.0f;
    if (sc.spp > 1) v = fmaxf(fd(fs(sy2, fd(fm(sy, sy), n)), fm(n, fs(n, 1.0f))), 0.0f);
    variance[pix] = v;
}

}  // namespace
}  // namespace esim

using namespace esim;

extern "C" esim_ad_status esim_ad_render(const esim_ad_render_scene* scene, int32_t frame, float* radiance,
                                         float* variance, float* normal, float* albedo, float* depth,
                                         void* cuda_stream)
{
    if (!scene || !radiance || !variance || !normal || !albedo || !depth) return ESIM_AD_EINVAL;
    const esim_ad_render_scene& s = *scene;
    if (s.struct_size != sizeof(esim_ad_render_scene) || s.width < 1 || s.height < 1 ||
        (long long)s.width * s.height >= (1ll << 31) || s.spp < 1 || s.spp > 65536 || s.max_bounces < 1 ||
        s.max_bounces > 8 || s.n_spheres < 0 || s.n_spheres > 8 || !(s.tan_half_fov_y > 0.0f) ||
        !(s.box[0] > 0.0f) || !(s.box[1] > 0.0f) || !(s.box[2] > 0.0f) || !(s.light[1] > s.light[0]) ||
        !(s.light[3] > s.light[2]) || !(s.eps > 0.0f) || frame < 0)
        return ESIM_AD_EINVAL;
    for (int j = 0; j < s.n_spheres; ++j)
        if (!(s.spheres[j].radius > 0.0f)) return ESIM_AD_EINVAL;
    const dim3 block(16, 16);
    const dim3 grid((s.width + 15) / 16, (s.height + 15) / 16);
    render_kernel<<<grid, block, 0, (cudaStream_t)cuda_stream>>>(s, frame, radiance, variance, normal, albedo,
                                                                 depth);
    return cudaGetLastError() == cudaSuccess ? ESIM_AD_OK : ESIM_AD_ECUDA;
}
