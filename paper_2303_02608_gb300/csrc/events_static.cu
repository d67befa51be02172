// Ordered event writer that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they need
// events written: latency-critical loops where cudaMalloc's implicit
// device-wide synchronisation would stall other streams, and plugins hosted by
// a framework that owns every device allocation.  For them,
// esim_ad_write_events_noalloc runs the same two event-writer kernels as the
// simulator context, but their scratch (the control block and the per-chunk
// counts) lives in one fixed-size array of this file that every GPU loading
// the library holds until the process exits.
//
// The array's name in host code is only a host-side stand-in, not a device
// address, so its device address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernels.
#include <mutex>

#include "internal.h"

namespace esim {
namespace {

constexpr long long kNoAllocMaxPixels = 1ll << 24;                        // 16,777,216 pixels
constexpr int kNoAllocMaxChunks = (int)(kNoAllocMaxPixels / kChunk);      // 8192 chunks
constexpr size_t kCtrlBytes = 256;
constexpr size_t kCntBytes = (size_t)kNoAllocMaxChunks * sizeof(uint32_t);
constexpr size_t kScratchBytes = kCtrlBytes + kCntBytes;                  // 33,024 bytes
static_assert(sizeof(Ctrl) <= kCtrlBytes, "control block must fit its slot");

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) unsigned char g_event_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_dev[kMaxDevices] = {};

// Device address of the array on the current device (looked up on first use).
esim_ad_status scratch_on_current_device(unsigned char** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return ESIM_AD_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_event_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return ESIM_AD_ECUDA;
        }
        g_scratch_dev[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_dev[dev];
    return ESIM_AD_OK;
}

}  // namespace
}  // namespace esim

using namespace esim;

extern "C" esim_ad_status esim_ad_write_events_noalloc(const int32_t* counts, int32_t width,
                                                       int32_t height, uint32_t frame,
                                                       esim_ad_event* events, uint64_t capacity,
                                                       uint64_t* total_device, void* cuda_stream)
{
    if (!counts || !total_device || (capacity > 0 && !events)) return ESIM_AD_EINVAL;
    if (width < 1 || height < 1 || width > 65535 || height > 65535) return ESIM_AD_EINVAL;
    const long long n_pix = (long long)width * height;
    if (n_pix > kNoAllocMaxPixels) return ESIM_AD_EINVAL;
    unsigned char* base = nullptr;
    esim_ad_status st = scratch_on_current_device(&base);
    if (st != ESIM_AD_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(base);
    // the ticket, the running total and the status bits must start at zero
    if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s) != cudaSuccess) return ESIM_AD_ECUDA;
    EventParams p;
    p.nev = counts;
    p.n_pix = n_pix;
    p.W = width;
    p.n_chunks = (int)((n_pix + kChunk - 1) / kChunk);
    p.frame = frame;
    p.chunk_cnt = reinterpret_cast<uint32_t*>(base + kCtrlBytes);
    p.chunk_off = nullptr;   // the writer places each chunk from the counts alone
    p.events = events;
    p.capacity = capacity;
    p.ctrl = ctrl;
    if (launch_events(p, s) != cudaSuccess) return ESIM_AD_ECUDA;
    if (cudaMemcpyAsync(total_device, &ctrl->ev_total, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
        return ESIM_AD_ECUDA;
    return ESIM_AD_OK;
}
