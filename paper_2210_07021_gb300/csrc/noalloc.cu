// sfmm_sort_keys_static: the key computation and stable radix sort that every
// solve starts with, for callers that must not allocate device memory.
//
// Who needs this: code that runs where device allocation is not allowed or not
// affordable -- for instance a plugin inside a host application whose memory
// pool owns the whole device, or a latency-critical pipeline that cannot accept
// the device-wide synchronisation cudaMalloc/cudaFree may cause.  Such callers
// provide the outputs; all scratch memory (the sort's ping-pong buffers, the
// per-tile digit histograms and the scan's block sums) lives in one file-scope
// static device array of fixed size that every GPU loading this library holds
// until the process exits.
//
// The array's name in host code is only a host-side stand-in, not a device
// address, so on the first call on each device (with that device current) the
// device address is looked up once with cudaGetSymbolAddress and cached.  That
// first call should therefore come before any stream capture.
//
// Every call shares the one array.  Nothing in it has to start at zero: each
// radix pass writes the histogram, the offsets and the ping-pong buffers in
// full before reading them.  Calls that overlap on the GPU (for example on two
// streams at once) race on the array and must be serialised by the caller.
#include "common.cuh"

#include <cstdio>
#include <mutex>
#include <string>

namespace sfmm {
void set_process_error(const std::string& msg);

namespace {

constexpr int64_t STATIC_MAX_N = int64_t(1) << 18;                 // 262,144 points
constexpr size_t ALT_KEY_BYTES = size_t(STATIC_MAX_N) * 8;         // 2 MiB
constexpr size_t ALT_PERM_BYTES = size_t(STATIC_MAX_N) * 4;        // 1 MiB
constexpr size_t SORT_TMP_BYTES = size_t(1) << 19;                 // 512 KiB (histograms + scan sums)
constexpr size_t SCRATCH_BYTES = ALT_KEY_BYTES + ALT_PERM_BYTES + SORT_TMP_BYTES;

static __device__ __align__(256) unsigned char g_static_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace sfmm

using namespace sfmm;

extern "C" sfmm_status sfmm_sort_keys_static(const double* xyz, int64_t n, uint64_t* keys, uint32_t* perm,
                                             void* stream)
{
    if (n < 0 || n > STATIC_MAX_N) {
        char b[160];
        snprintf(b, sizeof b, "sfmm_sort_keys_static: n = %lld is outside 0..%lld (the size of its static scratch)",
                 (long long)n, (long long)STATIC_MAX_N);
        set_process_error(b);
        return SFMM_EINVAL;
    }
    if (n == 0) return SFMM_OK;
    if (!xyz || !keys || !perm) {
        set_process_error("sfmm_sort_keys_static: xyz, keys and perm must be non-NULL");
        return SFMM_EINVAL;
    }
    if (radix_tmp_bytes(STATIC_MAX_N) > SORT_TMP_BYTES) {
        set_process_error("sfmm_sort_keys_static: internal scratch layout too small");
        return SFMM_EINVAL;
    }
    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        set_process_error(std::string("sfmm_sort_keys_static: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
        return SFMM_ECUDA;
    }
    unsigned char* b = static_cast<unsigned char*>(base);
    uint64_t* alt_keys = reinterpret_cast<uint64_t*>(b);
    uint32_t* alt_perm = reinterpret_cast<uint32_t*>(b + ALT_KEY_BYTES);
    void* tmp = b + ALT_KEY_BYTES + ALT_PERM_BYTES;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((e = launch_keys(xyz, n, keys, perm, s)) != cudaSuccess) {
        set_process_error(std::string("sfmm_sort_keys_static: ") + cudaGetErrorString(e));
        return SFMM_ECUDA;
    }
    bool in_alt = false;
    // 62 key bits = 8 passes of 8 bits: an even number, so the result ends in (keys, perm)
    if ((e = radix_sort(keys, perm, alt_keys, alt_perm, n, 62, tmp, s, &in_alt)) != cudaSuccess || in_alt) {
        set_process_error(std::string("sfmm_sort_keys_static: ") +
                          (e != cudaSuccess ? cudaGetErrorString(e) : "odd number of sort passes"));
        return SFMM_ECUDA;
    }
    return SFMM_OK;
}
