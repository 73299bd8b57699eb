// sieve_static.cu -- prime-list compaction that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs where the allocator is
// off limits (a fixed memory arena, a real-time loop that must not take the
// allocator's locks, a plug-in whose host process owns all device memory).
// sieve_compact_static gives them the compaction of sieve_compact without a
// context: its scratch (per-tile popcounts, their prefix sums and the total)
// is a fixed array compiled into this library, so the call allocates nothing.
// The caller passes the bitmap and the output.  The paper has no counterpart.
//
// The array is a file-scope __device__ object of a fixed size, so every GPU
// that loads the library holds it until the process exits, and every call on
// that GPU shares it.  In host code its name is only a host-side stand-in,
// never a device address: the first call on each device, with that device
// current, asks the runtime for the real address once (cudaGetSymbolAddress)
// and later calls reuse it.  Make that first call before any stream capture.

#include <mutex>

#include "gbsieve.h"
#include "internal.h"

namespace {

using namespace gbs;

constexpr uint64_t kStaticTiles = SIEVE_STATIC_MAX_WORDS / kCompactTileWords;  // 32768
constexpr size_t kCountsBytes = kStaticTiles * sizeof(uint32_t);
constexpr size_t kOffsetsBytes = kStaticTiles * sizeof(uint64_t);
constexpr size_t kScratchBytes = kCountsBytes + kOffsetsBytes + 256;  // + the total, 256-aligned

// Layout: [tile counts (uint32) | tile offsets (uint64) | total (uint64)].
// Every word is written by a kernel before any kernel reads it, so nothing
// needs clearing between calls.
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (set up once per device).
cudaError_t scratch_on_current_device(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int sieve_compact_static(const uint32_t *bitmap_dev, uint64_t lo, uint64_t hi, uint32_t *out_dev,
                                    size_t cap, uint64_t *n, void *cuda_stream) {
    // argument checks in sieve_compact's order, all before any GPU work
    if (!n || lo > hi) return SIEVE_EINVAL;
    if (hi > (1ull << 32)) return SIEVE_ERANGE;
    const uint64_t o0 = lo | 1;
    const uint64_t nwords = o0 < hi ? ((hi - o0 + 1) / 2 + 31) / 32 : 0;
    if (nwords && !bitmap_dev) return SIEVE_EINVAL;
    if (!out_dev && cap) return SIEVE_EINVAL;
    // with hi <= 2^32 the bitmap has at most 2^26 words, so this cannot fire today; it
    // keeps the scratch array safe should SIEVE_STATIC_MAX_WORDS ever be made smaller
    if (nwords > SIEVE_STATIC_MAX_WORDS) return SIEVE_ERANGE;
    const uint32_t two = (lo <= 2 && 2 < hi) ? 1 : 0;
    const uint64_t ntiles = (nwords + kCompactTileWords - 1) / kCompactTileWords;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    unsigned char *base = nullptr;
    uint64_t total = 0;
    if (ntiles) {
        if (scratch_on_current_device(&base) != cudaSuccess) return SIEVE_ECUDA;
        uint32_t *tile_counts = reinterpret_cast<uint32_t *>(base);
        uint64_t *tile_offsets = reinterpret_cast<uint64_t *>(base + kCountsBytes);
        unsigned long long *d_total = reinterpret_cast<unsigned long long *>(base + kCountsBytes + kOffsetsBytes);
        int sms = 0, dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return SIEVE_ECUDA;
        if (launch_tile_popc(bitmap_dev, nwords, tile_counts, ntiles, sms * 8, stream) != cudaSuccess ||
            launch_tile_scan(tile_counts, tile_offsets, ntiles, d_total, stream) != cudaSuccess)
            return SIEVE_ECUDA;
        unsigned long long t = 0;
        if (cudaMemcpyAsync(&t, d_total, sizeof t, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess)
            return SIEVE_ECUDA;
        total = t;
        *n = total + two;
        if (*n > cap) return SIEVE_ETRUNC;
        if (*n && !out_dev) return SIEVE_EINVAL;
        if (two && launch_put_two(out_dev, 0, stream) != cudaSuccess) return SIEVE_ECUDA;
        if (launch_emit(bitmap_dev, nwords, tile_offsets, ntiles, o0, two, out_dev, 0, sms, stream) !=
            cudaSuccess)
            return SIEVE_ECUDA;
        return cudaStreamSynchronize(stream) == cudaSuccess ? SIEVE_OK : SIEVE_ECUDA;
    }
    *n = two;
    if (*n > cap) return SIEVE_ETRUNC;
    if (two) {
        if (!out_dev) return SIEVE_EINVAL;
        if (launch_put_two(out_dev, 0, stream) != cudaSuccess) return SIEVE_ECUDA;
        return cudaStreamSynchronize(stream) == cudaSuccess ? SIEVE_OK : SIEVE_ECUDA;
    }
    return SIEVE_OK;
}
