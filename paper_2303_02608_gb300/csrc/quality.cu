// Evaluation kernels (Section 3, quantitative comparison): the plain ESIM
// simulator, and polarity-aware precision, recall, F-score and chamfer
// distance between two event sets with an exact nearest-neighbour search.
//
// Events are signed points (x / W, y / H, t / F).  For one set and each
// polarity, a column pass stores per pixel and frame the squared distance to
// the nearest event of that polarity in the pixel's column (g).  The nearest
// event of a query (x, y, t) is then
//     min over t', q of ((x - q) / W)^2 + g_t'(q, y) + ((t - t') / F)^2,
// searched outward in |t - t'| and |x - q| and cut off as soon as the
// separation alone reaches the best squared distance found.  Frames without
// any event of the polarity are skipped through a per-frame flag.  Sums of the
// chamfer terms are reduced per block in FP64 and then in a fixed order.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "internal.h"

namespace esim {
namespace {

constexpr int kQThreads = 256;
constexpr int kMaxTau = 16;

__global__ void esim_frame_kernel(const float* __restrict__ rad, int channels, float log_eps, float C,
                                  int init, float* __restrict__ l_last, int32_t* __restrict__ counts,
                                  long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float Y = channels == 3
            ? 0.2126f * __ldg(rad + i) + 0.7152f * __ldg(rad + n + i) + 0.0722f * __ldg(rad + 2 * n + i)
            : __ldg(rad + i);
        const float y = logf(Y + log_eps);
        if (init) {
            l_last[i] = y;
            counts[i] = 0;
            continue;
        }
        const float L = l_last[i];
        const float dl = y - L;
        const float nf = floorf(fabsf(dl) / C);
        if (nf >= 1.0f) {
            const float pol = dl > 0.0f ? 1.0f : -1.0f;
            l_last[i] = fmaf(pol * nf, C, L);
            counts[i] = (int32_t)(pol * nf);
        } else {
            counts[i] = 0;
        }
    }
}

struct QualParams {
    const int32_t* set[2];   // 0: generated, 1: reference; [F][H][W]
    float* g;                // [set][polarity][F][H][W] squared column distances (INF: none)
    uint32_t* frame_any;     // [set][polarity][F]: the frame holds an event of that polarity
    unsigned long long* hit; // [direction][kMaxTau] event counts within tau
    unsigned long long* n_ev;   // [direction] events queried
    uint32_t* unmatched;     // [direction] some event had no partner of its polarity
    double* partial;         // [direction][query blocks] sums of n * d^2
    int W, H, F, n_tau;
    float invW, invH, invF;
    float tau2[kMaxTau];
    int q_blocks;
};

// One thread per (column, frame, set): both polarities, downward then upward.
__global__ void column_kernel(QualParams p)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    const int s = blockIdx.z;
    if (x >= p.W) return;
    const size_t N = (size_t)p.W * p.H;
    const int32_t* c = p.set[s] + (size_t)t * N + x;
    float* g0 = p.g + ((size_t)(2 * s + 0) * p.F + t) * N + x;
    float* g1 = p.g + ((size_t)(2 * s + 1) * p.F + t) * N + x;
    const int kNone = -(1 << 30);
    int last0 = kNone, last1 = kNone;
    bool any0 = false, any1 = false;
    for (int y = 0; y < p.H; ++y) {
        const int32_t v = c[(size_t)y * p.W];
        if (v > 0) { last0 = y; any0 = true; }
        if (v < 0) { last1 = y; any1 = true; }
        const float d0 = last0 == kNone ? INFINITY : (float)(y - last0) * p.invH;
        const float d1 = last1 == kNone ? INFINITY : (float)(y - last1) * p.invH;
        g0[(size_t)y * p.W] = d0 * d0;
        g1[(size_t)y * p.W] = d1 * d1;
    }
    last0 = last1 = kNone;
    for (int y = p.H - 1; y >= 0; --y) {
        const int32_t v = c[(size_t)y * p.W];
        if (v > 0) last0 = y;
        if (v < 0) last1 = y;
        if (last0 != kNone) {
            const float d = (float)(last0 - y) * p.invH;
            g0[(size_t)y * p.W] = fminf(g0[(size_t)y * p.W], d * d);
        }
        if (last1 != kNone) {
            const float d = (float)(last1 - y) * p.invH;
            g1[(size_t)y * p.W] = fminf(g1[(size_t)y * p.W], d * d);
        }
    }
    if (any0) atomicOr(&p.frame_any[(2 * s + 0) * p.F + t], 1u);
    if (any1) atomicOr(&p.frame_any[(2 * s + 1) * p.F + t], 1u);
}

// Squared distance from (x, y, t) to the nearest event of polarity pol in set s.
__device__ float nearest2(const QualParams& p, int s, int pol, int x, int y, int t)
{
    const size_t N = (size_t)p.W * p.H;
    const uint32_t* any = p.frame_any + (2 * s + pol) * p.F;
    const float* gs = p.g + (size_t)(2 * s + pol) * p.F * N + (size_t)y * p.W;
    float best = INFINITY;
    for (int k = 0; k < p.F; ++k) {
        const float dt = (float)k * p.invF;
        const float dt2 = dt * dt;
        if (dt2 >= best) break;
        for (int side = 0; side < (k ? 2 : 1); ++side) {
            const int tt = side ? t + k : t - k;
            if (tt < 0 || tt >= p.F || !any[tt]) continue;
            const float* row = gs + (size_t)tt * N;
            for (int j = 0; j < p.W; ++j) {
                const float dx = (float)j * p.invW;
                const float sep = fmaf(dx, dx, dt2);
                if (sep >= best) break;
                float v = INFINITY;
                if (x - j >= 0) v = row[x - j];
                if (j && x + j < p.W) v = fminf(v, row[x + j]);
                best = fminf(best, sep + v);
            }
        }
    }
    return best;
}

// One thread per (pixel, frame) of the query set; blockIdx.y = direction
// (0: generated -> reference, 1: reference -> generated).
__global__ void __launch_bounds__(kQThreads) query_kernel(QualParams p)
{
    const int dir = blockIdx.y;
    const size_t N = (size_t)p.W * p.H;
    const size_t idx = (size_t)blockIdx.x * kQThreads + threadIdx.x;
    __shared__ unsigned long long s_hit[kMaxTau];
    __shared__ unsigned long long s_n;
    __shared__ uint32_t s_unmatched;
    __shared__ double s_sum[kQThreads / 32];
    if (threadIdx.x < kMaxTau) s_hit[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) {
        s_n = 0ull;
        s_unmatched = 0u;
    }
    __syncthreads();
    double sum = 0.0;
    if (idx < N * (size_t)p.F) {
        const int32_t c = p.set[dir][idx];
        if (c != 0) {
            const int t = (int)(idx / N);
            const int rem = (int)(idx - (size_t)t * N);
            const int y = rem / p.W, x = rem - (rem / p.W) * p.W;
            const int pol = c > 0 ? 0 : 1;
            const unsigned long long w = (unsigned long long)(c > 0 ? c : -c);
            const float d2 = nearest2(p, 1 - dir, pol, x, y, t);
            atomicAdd(&s_n, w);
            if (isinf(d2)) {
                s_unmatched = 1u;
            } else {
                sum = (double)w * (double)d2;
                for (int k = 0; k < p.n_tau; ++k)
                    if (d2 < p.tau2[k]) atomicAdd(&s_hit[k], w);
            }
        }
    }
    // block sum in a fixed order
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, off);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < kQThreads / 32; ++i) b += s_sum[i];
        p.partial[(size_t)dir * p.q_blocks + blockIdx.x] = b;
        if (s_n) atomicAdd(&p.n_ev[dir], s_n);
        if (s_unmatched) atomicOr(&p.unmatched[dir], 1u);
    }
    if (threadIdx.x < (unsigned)p.n_tau && s_hit[threadIdx.x])
        atomicAdd(&p.hit[dir * kMaxTau + threadIdx.x], s_hit[threadIdx.x]);
}

// Fixed-order sum of the per-block partials of both directions.
__global__ void __launch_bounds__(1024) reduce_kernel(QualParams p, double* out)
{
    __shared__ double s[1024];
    for (int dir = 0; dir < 2; ++dir) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < p.q_blocks; i += 1024) acc += p.partial[(size_t)dir * p.q_blocks + i];
        s[threadIdx.x] = acc;
        __syncthreads();
        for (int w = 512; w >= 1; w >>= 1) {
            if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[dir] = s[0];
        __syncthreads();
    }
}

struct QualLayout {
    size_t g, any, hit, n_ev, unmatched, partial, sums, total;
};

QualLayout qual_layout(int W, int H, int F)
{
    const size_t N = (size_t)W * H;
    const size_t q_blocks = (N * (size_t)F + kQThreads - 1) / kQThreads;
    QualLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return at;
    };
    L.g = take(4 * (size_t)F * N * sizeof(float));
    L.any = take(4 * (size_t)F * sizeof(uint32_t));
    L.hit = take(2 * kMaxTau * sizeof(unsigned long long));
    L.n_ev = take(2 * sizeof(unsigned long long));
    L.unmatched = take(2 * sizeof(uint32_t));
    L.partial = take(2 * q_blocks * sizeof(double));
    L.sums = take(2 * sizeof(double));
    L.total = off;
    return L;
}

}  // namespace
}  // namespace esim

using namespace esim;

extern "C" esim_ad_status esim_ad_esim_frame(const float* radiance, int32_t channels, float log_eps,
                                             float contrast, int32_t init, float* l_last, int32_t* counts,
                                             int64_t n_pix, void* cuda_stream)
{
    if (!radiance || !l_last || !counts || (channels != 1 && channels != 3) || n_pix < 0 ||
        !(contrast > 0.0f))
        return ESIM_AD_EINVAL;
    if (n_pix == 0) return ESIM_AD_OK;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return ESIM_AD_ECUDA;
    const long long blocks = (n_pix + 255) / 256;
    const int grid = (int)(blocks < (long long)sms * 16 ? blocks : (long long)sms * 16);
    esim_frame_kernel<<<grid, 256, 0, (cudaStream_t)cuda_stream>>>(radiance, channels, log_eps, contrast, init,
                                                                  l_last, counts, (long long)n_pix);
    return cudaGetLastError() == cudaSuccess ? ESIM_AD_OK : ESIM_AD_ECUDA;
}

extern "C" size_t esim_ad_quality_workspace_size(int32_t width, int32_t height, int32_t frames)
{
    if (width <= 0 || height <= 0 || frames <= 0) return 0;
    return qual_layout(width, height, frames).total;
}

extern "C" esim_ad_status esim_ad_quality(const int32_t* gen, const int32_t* ref, int32_t width, int32_t height,
                                          int32_t frames, const float* tau, int32_t n_tau, void* workspace,
                                          size_t workspace_bytes, esim_ad_quality_result* out, void* cuda_stream)
{
    if (!gen || !ref || !tau || !workspace || !out || width <= 0 || height <= 0 || frames <= 0 || frames > 65535 || n_tau < 1 ||
        n_tau > kMaxTau)
        return ESIM_AD_EINVAL;
    const QualLayout L = qual_layout(width, height, frames);
    if (workspace_bytes < L.total) return ESIM_AD_EINVAL;
    const size_t N = (size_t)width * height;
    const size_t q_blocks = (N * (size_t)frames + kQThreads - 1) / kQThreads;
    if (q_blocks > 0x7fffffffu) return ESIM_AD_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    QualParams p;
    p.set[0] = gen;
    p.set[1] = ref;
    p.g = reinterpret_cast<float*>(ws + L.g);
    p.frame_any = reinterpret_cast<uint32_t*>(ws + L.any);
    p.hit = reinterpret_cast<unsigned long long*>(ws + L.hit);
    p.n_ev = reinterpret_cast<unsigned long long*>(ws + L.n_ev);
    p.unmatched = reinterpret_cast<uint32_t*>(ws + L.unmatched);
    p.partial = reinterpret_cast<double*>(ws + L.partial);
    p.W = width;
    p.H = height;
    p.F = frames;
    p.n_tau = n_tau;
    p.invW = 1.0f / (float)width;
    p.invH = 1.0f / (float)height;
    p.invF = 1.0f / (float)frames;
    for (int k = 0; k < kMaxTau; ++k) p.tau2[k] = k < n_tau ? tau[k] * tau[k] : 0.0f;
    p.q_blocks = (int)q_blocks;
    // counters (everything between the flags and the partials) start at zero
    if (cudaMemsetAsync(ws + L.any, 0, L.partial - L.any, s) != cudaSuccess) return ESIM_AD_ECUDA;
    column_kernel<<<dim3((width + 127) / 128, frames, 2), 128, 0, s>>>(p);
    if (cudaGetLastError() != cudaSuccess) return ESIM_AD_ECUDA;
    query_kernel<<<dim3((unsigned)q_blocks, 2), kQThreads, 0, s>>>(p);
    if (cudaGetLastError() != cudaSuccess) return ESIM_AD_ECUDA;
    double* sums = reinterpret_cast<double*>(ws + L.sums);
    reduce_kernel<<<1, 1024, 0, s>>>(p, sums);
    if (cudaGetLastError() != cudaSuccess) return ESIM_AD_ECUDA;
    unsigned long long h_hit[2 * kMaxTau], h_n[2];
    uint32_t h_un[2];
    double h_sum[2];
    if (cudaMemcpyAsync(h_hit, p.hit, sizeof(h_hit), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(h_n, p.n_ev, sizeof(h_n), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(h_un, p.unmatched, sizeof(h_un), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(h_sum, sums, sizeof(h_sum), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return ESIM_AD_ECUDA;
    esim_ad_quality_result r;
    memset(&r, 0, sizeof(r));
    r.n_tau = n_tau;
    r.n_gen = h_n[0];
    r.n_ref = h_n[1];
    for (int k = 0; k < n_tau; ++k) {
        r.tau[k] = tau[k];
        const double P = h_n[0] ? (double)h_hit[k] / (double)h_n[0] : 0.0;
        const double R = h_n[1] ? (double)h_hit[kMaxTau + k] / (double)h_n[1] : 0.0;
        r.precision[k] = P;
        r.recall[k] = R;
        r.fscore[k] = P + R > 0.0 ? 2.0 * P * R / (P + R) : 0.0;
    }
    if (h_un[0] || h_un[1]) {
        r.chamfer = INFINITY;
    } else {
        r.chamfer = (h_n[0] ? h_sum[0] / (double)h_n[0] : 0.0) + (h_n[1] ? h_sum[1] / (double)h_n[1] : 0.0);
    }
    *out = r;
    return ESIM_AD_OK;
}
