// fdtd_watch.cu -- the divergence watchdog of the GB300 FDTD library: a
// streaming check of the six field arrays for values that are not finite
// (NaN or +-Inf).  The paper's explicit leapfrog (Sec. 2.1) is stable only
// under the Courant bound; a grid past it (or an unstable wire model) grows
// without bound, overflows FP32 and then spreads NaN, which this check turns
// into an error status the host reads (FDTD_EDIVERGED).
#include "fdtd_internal.h"

namespace fdtd {
namespace {

// IEEE 754 binary32: exponent field all ones = Inf or NaN
__device__ __forceinline__ bool not_finite(float v)
{
    return (__float_as_uint(v) & 0x7f800000u) == 0x7f800000u;
}

// Grid-stride over n4 float4 of each field (the arrays are 16-byte aligned
// and a whole number of float4 long, row padding included: padding stays
// zero).  Streaming loads, so the check does not evict the step's working
// set from L2.  One atomic per warp that saw a bad value.
__global__ void __launch_bounds__(256) finite_kernel(FieldPtrs f, long long n4, int *flag)
{
    if (*(volatile int *)flag) return;
    bool bad = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int c = 0; c < 6; ++c) {
        const float4 *p = reinterpret_cast<const float4 *>(f.p[c]);
        for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
            const float4 v = __ldcs(p + q);
            bad |= not_finite(v.x) | not_finite(v.y) | not_finite(v.z) | not_finite(v.w);
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(flag, 1);
}

}  // namespace

cudaError_t launch_finite_check(const FieldPtrs &f, long long n_elems, int *flag, int blocks, cudaStream_t s)
{
    finite_kernel<<<blocks, 256, 0, s>>>(f, n_elems / 4, flag);
    return cudaGetLastError();
}

}  // namespace fdtd
