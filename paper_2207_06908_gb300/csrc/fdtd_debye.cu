// fdtd_debye.cu -- dispersive (multi-term Debye) media: the part of the E
// update the step kernels leave out (Kuklin, arXiv 2207.06908, "Dispersive
// media": Debye permittivity by the auxiliary differential equation method
// of its references).
//
// For an edge with poles p the E half step is
//   E^{n+1} = ca E^n + cb curl H^{n+1/2} + sum_p cj_p J_p^n
// and the polarisation currents then advance by the trapezoidal rule
//   J_p^{n+1} = k_p J_p^n + be_p (E^{n+1} - E^n).
// The step kernels compute ca E + cb curl (ca, cb of dispersive edges
// already carry the poles); this kernel, launched after them and before the
// source / probe kernel, adds the current terms and advances the currents.
// It streams the planes that hold dispersive edges: per cell a record byte,
// E^n and E^{n+1} of the dispersive components and their currents.
#include <algorithm>

#include "fdtd_internal.h"

namespace fdtd {
namespace {

__device__ __forceinline__ float &el(float4 &v, int t) { return reinterpret_cast<float *>(&v)[t]; }

// Each thread takes four consecutive elements of the box (16-byte aligned:
// the plane is a multiple of 16 elements), issues every load of its
// dispersive components first (E^n, E^{n+1}, the currents, all float4),
// then updates and stores them.
template <int NP>
__global__ void __launch_bounds__(256) debye_kernel(const DebyeArgs a)
{
    extern __shared__ float tab[];          // [n_rec][kDebyeRec], then a component mask per record
    int *mask = reinterpret_cast<int *>(tab + a.n_rec * kDebyeRec);
    for (int q = threadIdx.x; q < a.n_rec * kDebyeRec; q += blockDim.x) tab[q] = __ldg(a.table + q);
    __syncthreads();
    constexpr int np = NP;
    for (int r = threadIdx.x; r < a.n_rec; r += blockDim.x) {
        int m = 0;
        for (int c = 0; c < 3; ++c)
            for (int p = 0; p < np; ++p)
                if (tab[r * kDebyeRec + c * kMaxPoles * 3 + 3 * p + 2] != 0.f) m |= 1 << c;
        mask[r] = m;
    }
    __syncthreads();
    const uchar4 *__restrict__ dcls4 = reinterpret_cast<const uchar4 *>(a.dcls);
    const long long n4 = a.jstride / 4;
    for (long long q4 = (long long)blockIdx.x * blockDim.x + threadIdx.x; q4 < n4;
         q4 += (long long)gridDim.x * blockDim.x) {
        const uchar4 rv = __ldg(dcls4 + q4);
        const int rec[4] = {rv.x, rv.y, rv.z, rv.w};
        const int comps = mask[rec[0]] | mask[rec[1]] | mask[rec[2]] | mask[rec[3]];
        if (!comps) continue;
        const long long q = 4 * q4, g = a.off + q;
        float4 e0[3], e1[3], jv[3][NP];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (!(comps >> c & 1)) continue;
            e0[c] = __ldg(reinterpret_cast<const float4 *>(a.Ein[c] + g));
            e1[c] = *reinterpret_cast<const float4 *>(a.Eout[c] + g);
#pragma unroll
            for (int p = 0; p < np; ++p)
                jv[c][p] = *reinterpret_cast<const float4 *>(a.J + (long long)(c * np + p) * a.jstride + q);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (!(comps >> c & 1)) continue;
            float4 e = e1[c];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const float *rc = tab + rec[t] * kDebyeRec + c * kMaxPoles * 3;
                float v = el(e, t);
#pragma unroll
                for (int p = 0; p < np; ++p) v += rc[3 * p] * el(jv[c][p], t);
#pragma unroll
                for (int p = 0; p < np; ++p)
                    el(jv[c][p], t) = rc[3 * p + 1] * el(jv[c][p], t) + rc[3 * p + 2] * (v - el(e0[c], t));
                el(e, t) = v;
            }
#pragma unroll
            for (int p = 0; p < np; ++p)
                *reinterpret_cast<float4 *>(a.J + (long long)(c * np + p) * a.jstride + q) = jv[c][p];
            *reinterpret_cast<float4 *>(a.Eout[c] + g) = e;
        }
    }
}

}  // namespace

cudaError_t launch_debye(const DebyeArgs &a, cudaStream_t s)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 148;
    }
    const long long blocks = std::min<long long>((a.jstride / 4 + 255) / 256, 8LL * sms);
    const dim3 grid((unsigned)std::max<long long>(blocks, 1));
    const size_t smem = (size_t)a.n_rec * (kDebyeRec * sizeof(float) + sizeof(int));
    switch (a.npoles) {
    case 1: debye_kernel<1><<<grid, 256, smem, s>>>(a); break;
    case 2: debye_kernel<2><<<grid, 256, smem, s>>>(a); break;
    case 3: debye_kernel<3><<<grid, 256, smem, s>>>(a); break;
    case 4: debye_kernel<4><<<grid, 256, smem, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace fdtd
