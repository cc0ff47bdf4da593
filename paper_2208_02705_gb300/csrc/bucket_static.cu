// roam_bucket_static: the field bucketing of roam_bucket for callers that
// cannot allocate device memory.  Some hosts forbid cudaMalloc/cudaFree
// outside their own allocator: an engine whose pool owns all device memory,
// or a per-frame loop that cannot take the device-wide synchronisation a
// cudaFree implies.  This entry point needs no context and allocates
// nothing: its scratch (histogram, cursors, per-field tile records and the
// device counters) is one file-scope device array of fixed size, which every
// GPU that loads the library keeps until the process exits.
#include <mutex>

#include "internal.cuh"

namespace roam {

namespace {

constexpr int kStaticMaxFields = 4096;
constexpr int kStaticMaxDevices = 64;
// hist[F] + cursor[F] + tiles[F] (4 words each) + counters (16 words)
constexpr size_t kScratchWords = (size_t)kStaticMaxFields * 6 + 16;
static_assert(sizeof(Tile) == 4 * sizeof(uint32_t), "tile record is 4 words");
static_assert(sizeof(Counters) <= 16 * sizeof(uint32_t), "counters fit their slot");

static __device__ __align__(256) uint32_t g_bucket_scratch[kScratchWords];

struct DeviceSetup {
    uint32_t *scratch = nullptr;   // device address of g_bucket_scratch on this device (set once found)
    int n_sm = 0;
};

DeviceSetup g_setup[kStaticMaxDevices];
std::mutex g_setup_mutex;

// failures are reported through roam_last_error(), like every entry point
roam_status static_fail(roam_status st, const char *msg)
{
    set_error_message(msg);
    return st;
}

}  // namespace

}  // namespace roam

using namespace roam;

extern "C" roam_status roam_bucket_static(const uint16_t *keys, int64_t n, int n_fields, uint32_t *perm,
                                          uint32_t *offsets, void *stream)
{
    if (n_fields < 1 || n_fields > kStaticMaxFields)
        return static_fail(ROAM_ERR_ARG, "roam_bucket_static: n_fields must be in [1, 4096] (fixed-size scratch)");
    if (n < 0 || n > 0x7fffffffLL) return static_fail(ROAM_ERR_ARG, "roam_bucket_static: n must be in [0, 2^31 - 1]");
    if (!offsets || (n > 0 && (!keys || !perm))) return static_fail(ROAM_ERR_ARG, "roam_bucket_static: null pointer");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) {
        cudaGetLastError();
        return static_fail(ROAM_ERR_CUDA, "roam_bucket_static: no usable current device");
    }
    // once per device, with that device current: the host-side name of the
    // array is not a device address, so look the address up (a failed lookup
    // is not remembered: the next call tries again)
    DeviceSetup &ds = g_setup[dev];
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!ds.scratch) {
            void *p = nullptr;
            int n_sm = 0;
            if (cudaGetSymbolAddress(&p, g_bucket_scratch) != cudaSuccess ||
                cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || !p) {
                cudaGetLastError();
                return static_fail(ROAM_ERR_CUDA,
                                   "roam_bucket_static: cudaGetSymbolAddress of the scratch array failed");
            }
            ds.n_sm = n_sm;
            ds.scratch = static_cast<uint32_t *>(p);
        }
    }

    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *hist = ds.scratch;
    uint32_t *cursor = ds.scratch + kStaticMaxFields;
    Tile *tiles = reinterpret_cast<Tile *>(ds.scratch + 2 * kStaticMaxFields);
    Counters *ctr = reinterpret_cast<Counters *>(ds.scratch + 6 * kStaticMaxFields);
    // the array keeps the previous call's contents: clear what must start at zero
    if (cudaMemsetAsync(hist, 0, (size_t)n_fields * sizeof(uint32_t), s) != cudaSuccess ||
        cudaMemsetAsync(ctr, 0, sizeof(Counters), s) != cudaSuccess) {
        cudaGetLastError();
        return static_fail(ROAM_ERR_CUDA, "roam_bucket_static: clearing the scratch failed");
    }
    BucketBufs b;
    b.hist = hist;
    b.offsets = offsets;
    b.cursor = cursor;
    b.tiles = tiles;
    b.sorted = perm;
    b.tile_off = nullptr;
    // one tile record per field at most (tile length 2^31 - 1 >= n)
    launch_bucket(nullptr, nullptr, nullptr, (uint32_t)n, 1, 1, keys, n_fields, 0x7fffffff, b, ctr, ds.n_sm * 2, s,
                  ClassBounds{{0, n_fields, n_fields, n_fields}, {0, 0, 0, 0}});
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(ROAM_ERR_CUDA, "roam_bucket_static: kernel launch failed");
    return ROAM_OK;
}
