// bsort_keys_noalloc: the plain sort with its scratch memory taken from a
// fixed array linked into the library instead of from cudaMalloc.
//
// Who needs it: callers that must not allocate device memory while they run,
// for example code being captured into a CUDA graph (allocation calls are
// not capturable and cudaMalloc / cudaFree synchronise the whole device),
// applications whose device memory is entirely owned by their own pool or
// caching allocator, and plugins hosted by an engine that forbids raw
// allocations after start-up.  They pass only their keys; the library
// neither allocates nor frees anything on this path.
//
// The array is BSORT_NOALLOC_SCRATCH_BYTES bytes of static device memory.
// Every GPU on which the entry point is first used keeps it until the
// process exits (the module holding it is loaded on that first use).
#include <mutex>

#include "bsort.h"
#include "bsort_handle.h"

namespace {

constexpr size_t kScratchBytes = BSORT_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 16;

// The scratch array.  In host code `g_scratch` only names a host-side stand-in
// for the symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};
bsort_handle g_handle[kMaxDevices];  // static storage: no allocation on any call

// Once per device, with that device current: resolve the array's device
// address.  Returns nullptr if the lookup fails.
void *scratch_for(int device) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[device]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        g_scratch_ptr[device] = ptr;
        g_handle[device].device = device;
    }
    return g_scratch_ptr[device];
}

}  // namespace

extern "C" bsort_status bsort_keys_noalloc(void *keys, size_t n, bsort_dtype dt, int descending, void *stream) {
    size_t need = 0;
    const bsort_status ws = bsort_workspace_bytes(n, dt, BSORT_MODE_PINGPONG, &need);
    if (ws != BSORT_OK) return ws;
    if (n <= 1) return BSORT_OK;
    if (!keys) return BSORT_ERR_INVALID_ARG;
    if (need > kScratchBytes) return BSORT_ERR_WORKSPACE_TOO_SMALL;  // n beyond the fixed array
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return BSORT_ERR_CUDA;
    if (device < 0 || device >= kMaxDevices) return BSORT_ERR_UNSUPPORTED;
    void *scratch = scratch_for(device);
    if (!scratch) return BSORT_ERR_CUDA;
    return bsort_keys_ws(&g_handle[device], keys, n, dt, descending, BSORT_MODE_PINGPONG, scratch, kScratchBytes,
                         stream);
}
