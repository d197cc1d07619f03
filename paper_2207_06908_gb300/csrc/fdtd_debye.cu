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

__global__ void __launch_bounds__(256) debye_kernel(const DebyeArgs a)
{
    extern __shared__ float tab[];          // [n_rec][kDebyeRec]
    for (int q = threadIdx.x; q < a.n_rec * kDebyeRec; q += blockDim.x) tab[q] = __ldg(a.table + q);
    __syncthreads();
    const int np = a.npoles;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < a.jstride;
         q += (long long)gridDim.x * blockDim.x) {
        const int rec = __ldg(a.dcls + q);
        if (rec == 0) continue;
        const float *r = tab + rec * kDebyeRec;
        const long long g = a.off + q;
        for (int c = 0; c < 3; ++c) {
            const float *rc = r + c * kMaxPoles * 3;
            bool disp = false;
            for (int p = 0; p < np; ++p) disp |= rc[3 * p + 2] != 0.f;
            if (!disp) continue;
            const float e0 = a.Ein[c][g];
            float e = a.Eout[c][g];
            float jv[kMaxPoles];
            for (int p = 0; p < np; ++p) jv[p] = a.J[(long long)(c * np + p) * a.jstride + q];
            for (int p = 0; p < np; ++p) e += rc[3 * p] * jv[p];
            for (int p = 0; p < np; ++p)
                a.J[(long long)(c * np + p) * a.jstride + q] = rc[3 * p + 1] * jv[p] + rc[3 * p + 2] * (e - e0);
            a.Eout[c][g] = e;
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
    const long long blocks = std::min<long long>((a.jstride + 255) / 256, 8LL * sms);
    debye_kernel<<<(unsigned)std::max<long long>(blocks, 1), 256, (size_t)a.n_rec * kDebyeRec * sizeof(float), s>>>(a);
    return cudaGetLastError();
}

}  // namespace fdtd
