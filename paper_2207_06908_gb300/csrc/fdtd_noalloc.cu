// fdtd_noalloc.cu -- fdtd_step_noalloc(): the time step for callers that
// must not allocate device memory.
//
// The step kernel needs a little scratch memory besides the fields it reads
// and writes: two work-distribution counters per launch and a flag for a
// bounded wait that gave up.  fdtd_step() keeps them in the grid's arena;
// this entry point keeps them in a file-scope device array instead, so a
// caller that cannot allocate (and did not want that scratch carved from
// memory it handed over) can still run steps.  The array's device address
// is looked up once per device with cudaGetSymbolAddress(): host code only
// ever sees a host-side stand-in under the array's name, which a kernel must
// never be given.
#include <cuda_runtime.h>

#include <mutex>

#include "fdtd.h"
#include "fdtd_internal.h"

namespace {

// Step-kernel scratch shared by every fdtd_step_noalloc() call on a device:
// [0, 2 * launches) work counters of the grid being stepped; the last int is
// the error flag, a slot no grid uses as a counter.  Every GPU that loads the
// library holds these FDTD_NOALLOC_SCRATCH_INTS ints until the process exits.
static __device__ __align__(256) int g_step_scratch[FDTD_NOALLOC_SCRATCH_INTS];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
int *g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" int fdtd_step_noalloc(fdtd_grid *g, int n)
{
    if (!g) return FDTD_EINVAL;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fdtd::set_error(g, FDTD_ECUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return fdtd::set_error(g, FDTD_EINVAL, "device index too large");
    int *scratch;
    {
        std::lock_guard<std::mutex> lock(g_lock);
        if (!g_scratch_addr[dev]) {
            // first call on this device (with it current): the array's device address
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_step_scratch);
            if (e != cudaSuccess || !p)
                return fdtd::set_error(g, FDTD_ECUDA, "cudaGetSymbolAddress of the step scratch failed");
            g_scratch_addr[dev] = static_cast<int *>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    return fdtd::step_with_scratch(g, n, scratch, FDTD_NOALLOC_SCRATCH_INTS);
}
