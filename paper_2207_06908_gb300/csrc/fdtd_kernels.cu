// fdtd_kernels.cu -- CUDA kernels of the GB300 FDTD library (sm_103a, FP32).
//
// step_kernel: one fused Yee time step (Kuklin, arXiv 2207.06908, Sec. 2.1,
// Eq. fdtdhx then Eq. fdtdex with the loss term time-averaged) over the whole
// grid, CPML (Sec. 2.2) included.  Each CTA owns a TX x TY column of cells
// and marches up a chunk of z planes:
//   - E^n planes k and k+1 of the tile plus a one-cell halo sit in shared
//     memory (three rotating plane buffers);
//   - H^{n+1/2} of plane k is computed on the tile plus its low-x / low-y
//     halo (the halo values are recomputed, not exchanged), written for the
//     owned cells, and kept in shared memory;
//   - E^{n+1} of plane k follows at once from that H plane and the owned
//     column's H of plane k-1, held in registers.
// Fields ping-pong between two buffers, so E^n / H^{n-1/2} are read-only in
// the launch and the recomputed halo never races with its owner.  Each cell
// is read once and written once per step from DRAM (49 bytes with the class
// byte); the halos come from L2.
//
// edge_kernel: ideal current sources (Sec. 2.1, J = I/dx^2 on one edge) and
// the probes of the Sec. 4 model files, after the stencil of the same step.
#include "fdtd_internal.h"

namespace fdtd {
namespace {

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int NT = TX * TY;
constexpr int EW = TX + 2;   // E region: x0-1 .. x0+TX
constexpr int EH = TY + 2;   //           y0-1 .. y0+TY
constexpr int HW = TX + 1;   // H region: x0-1 .. x0+TX-1
constexpr int HH = TY + 1;   //           y0-1 .. y0+TY-1

struct __align__(16) Smem {
    float e[3][3][EH][EW];   // [plane buffer][component][ly][lx]
    float h[3][HH][HW];      // H^{n+1/2} of the current plane
    float tab[kMaxClasses * kNumCoef];
};

__device__ __forceinline__ long long fidx(const StepArgs &a, int i, int j, int k)
{
    return (long long)k * a.plane + (long long)j * a.pitch + i;
}

__device__ __forceinline__ int pbuf(int p) { return (p + 3) % 3; }

__device__ __forceinline__ bool in_slab(int i, int n, int d) { return i < d || i >= n - d; }
__device__ __forceinline__ int slab_idx(int i, int n, int d) { return i < d ? i : i - (n - 2 * d); }

// CPML convolution term: psi <- b psi + c dif; the curl term becomes
// dif / kappa + psi.  psi is written back only by the owner of the cell.
__device__ __forceinline__ float cpml(float dif, const float *prof, int n, int which, int i,
                                      const float *pin, float *pout, long long q, bool write)
{
    const float b = __ldg(prof + (which + 0) * n + i);
    const float c = __ldg(prof + (which + 1) * n + i);
    const float ki = __ldg(prof + (which + 2) * n + i);
    const float p = b * __ldg(pin + q) + c * dif;
    if (write) pout[q] = p;
    return dif * ki + p;
}

__device__ __forceinline__ void load_e_plane(const StepArgs &a, Smem &s, int buf, int k,
                                             int x0, int y0, int tid)
{
    const bool kin = k >= 0 && k < a.nz;
    for (int q = tid; q < EW * EH; q += NT) {
        const int ly = q / EW, lx = q - ly * EW;
        const int x = x0 - 1 + lx, y = y0 - 1 + ly;
        const bool in = kin && x >= 0 && x < a.nx && y >= 0 && y < a.ny;
        const long long g = in ? fidx(a, x, y, k) : 0;
        s.e[buf][0][ly][lx] = in ? __ldg(a.Ein[0] + g) : 0.f;
        s.e[buf][1][ly][lx] = in ? __ldg(a.Ein[1] + g) : 0.f;
        s.e[buf][2][ly][lx] = in ? __ldg(a.Ein[2] + g) : 0.f;
    }
}

// H^{n+1/2} at cell (i,j,k), region position (lx,ly); E planes k (bk) and
// k+1 (bk1) are in shared memory.
__device__ __forceinline__ void compute_h(const StepArgs &a, const Smem &s, int bk, int bk1,
                                          int lx, int ly, int i, int j, int k, int cl, bool own,
                                          float &hx, float &hy, float &hz)
{
    const float ex0 = s.e[bk][0][ly][lx], ey0 = s.e[bk][1][ly][lx], ez0 = s.e[bk][2][ly][lx];
    float hx_z = s.e[bk1][1][ly][lx] - ey0;        // Hx: dEy/dz - dEz/dy
    float hx_y = s.e[bk][2][ly + 1][lx] - ez0;
    float hy_x = s.e[bk][2][ly][lx + 1] - ez0;     // Hy: dEz/dx - dEx/dz
    float hy_z = s.e[bk1][0][ly][lx] - ex0;
    float hz_y = s.e[bk][0][ly + 1][lx] - ex0;     // Hz: dEx/dy - dEy/dx
    float hz_x = s.e[bk][1][ly][lx + 1] - ey0;
    const int d = a.d;
    if (d > 0) {
        if (in_slab(i, a.nx, d)) {
            const long long q = ((long long)k * a.ny + j) * (2 * d) + slab_idx(i, a.nx, d);
            hy_x = cpml(hy_x, a.prof[0], a.nx, PR_BH, i, a.psi_in[PSI_HY_X], a.psi_out[PSI_HY_X], q, own);
            hz_x = cpml(hz_x, a.prof[0], a.nx, PR_BH, i, a.psi_in[PSI_HZ_X], a.psi_out[PSI_HZ_X], q, own);
        }
        if (in_slab(j, a.ny, d)) {
            const long long q = ((long long)k * (2 * d) + slab_idx(j, a.ny, d)) * a.nx + i;
            hx_y = cpml(hx_y, a.prof[1], a.ny, PR_BH, j, a.psi_in[PSI_HX_Y], a.psi_out[PSI_HX_Y], q, own);
            hz_y = cpml(hz_y, a.prof[1], a.ny, PR_BH, j, a.psi_in[PSI_HZ_Y], a.psi_out[PSI_HZ_Y], q, own);
        }
        if (in_slab(k, a.nz, d)) {
            const long long q = ((long long)slab_idx(k, a.nz, d) * a.ny + j) * a.nx + i;
            hx_z = cpml(hx_z, a.prof[2], a.nz, PR_BH, k, a.psi_in[PSI_HX_Z], a.psi_out[PSI_HX_Z], q, own);
            hy_z = cpml(hy_z, a.prof[2], a.nz, PR_BH, k, a.psi_in[PSI_HY_Z], a.psi_out[PSI_HY_Z], q, own);
        }
    }
    const float *t = s.tab + cl * kNumCoef;
    const long long g = fidx(a, i, j, k);
    hx = __ldg(a.Hin[0] + g) + t[6] * (hx_z - hx_y);
    hy = __ldg(a.Hin[1] + g) + t[7] * (hy_x - hy_z);
    hz = __ldg(a.Hin[2] + g) + t[8] * (hz_y - hz_x);
    if (own) {
        a.Hout[0][g] = hx;
        a.Hout[1][g] = hy;
        a.Hout[2][g] = hz;
    }
}

__global__ void __launch_bounds__(NT) step_kernel(const StepArgs a)
{
    __shared__ Smem s;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * a.kz;
    const int z1 = min(z0 + a.kz, a.nz);
    const int i = x0 + tx, j = y0 + ty;
    const bool mine = i < a.nx && j < a.ny;
    const int lx = tx + 1, ly = ty + 1;

    for (int q = tid; q < a.n_classes * kNumCoef; q += NT) s.tab[q] = __ldg(a.table + q);

    // halo cell handled by this thread: the low-y row (threads 0..TX-1) or
    // the low-x column (threads TX..TX+TY-1); the corner is never needed
    const bool has_halo = tid < TX + TY;
    int hlx = 0, hly = 0, hi = -1, hj = -1;
    if (tid < TX) { hlx = tid + 1; hly = 0; hi = x0 + tid; hj = y0 - 1; }
    else if (has_halo) { hlx = 0; hly = tid - TX + 1; hi = x0 - 1; hj = y0 + (tid - TX); }
    const bool halo_ok = has_halo && hi >= 0 && hj >= 0 && hi < a.nx && hj < a.ny;

    float hx_prev = 0.f, hy_prev = 0.f;   // owned Hx, Hy of plane k-1 at n+1/2
    load_e_plane(a, s, pbuf(z0), z0, x0, y0, tid);
    if (z0 > 0) {
        // the plane below the chunk: recompute the owned Hx, Hy there
        load_e_plane(a, s, pbuf(z0 - 1), z0 - 1, x0, y0, tid);
        __syncthreads();
        if (mine) {
            float hz;
            const int cl = __ldg(a.cls + fidx(a, i, j, z0 - 1));
            compute_h(a, s, pbuf(z0 - 1), pbuf(z0), lx, ly, i, j, z0 - 1, cl, false, hx_prev, hy_prev, hz);
        }
    }
    for (int k = z0; k < z1; ++k) {
        const int bk = pbuf(k), bk1 = pbuf(k + 1);
        load_e_plane(a, s, bk1, k + 1, x0, y0, tid);
        __syncthreads();
        int cl_own = 0;
        float hx = 0.f, hy = 0.f, hz = 0.f;
        if (mine) {
            cl_own = __ldg(a.cls + fidx(a, i, j, k));
            compute_h(a, s, bk, bk1, lx, ly, i, j, k, cl_own, true, hx, hy, hz);
        }
        s.h[0][ly][lx] = hx;
        s.h[1][ly][lx] = hy;
        s.h[2][ly][lx] = hz;
        if (has_halo) {
            float gx = 0.f, gy = 0.f, gz = 0.f;
            if (halo_ok) {
                const int cl = __ldg(a.cls + fidx(a, hi, hj, k));
                compute_h(a, s, bk, bk1, hlx, hly, hi, hj, k, cl, false, gx, gy, gz);
            }
            s.h[0][hly][hlx] = gx;
            s.h[1][hly][hlx] = gy;
            s.h[2][hly][hlx] = gz;
        }
        __syncthreads();
        if (mine) {
            float ex_y = hz - s.h[2][ly - 1][lx];   // Ex: dHz/dy - dHy/dz
            float ex_z = hy - hy_prev;
            float ey_z = hx - hx_prev;              // Ey: dHx/dz - dHz/dx
            float ey_x = hz - s.h[2][ly][lx - 1];
            float ez_x = hy - s.h[1][ly][lx - 1];   // Ez: dHy/dx - dHx/dy
            float ez_y = hx - s.h[0][ly - 1][lx];
            const int d = a.d;
            if (d > 0) {
                if (in_slab(i, a.nx, d)) {
                    const long long q = ((long long)k * a.ny + j) * (2 * d) + slab_idx(i, a.nx, d);
                    ey_x = cpml(ey_x, a.prof[0], a.nx, PR_BE, i, a.psi_in[PSI_EY_X], a.psi_out[PSI_EY_X], q, true);
                    ez_x = cpml(ez_x, a.prof[0], a.nx, PR_BE, i, a.psi_in[PSI_EZ_X], a.psi_out[PSI_EZ_X], q, true);
                }
                if (in_slab(j, a.ny, d)) {
                    const long long q = ((long long)k * (2 * d) + slab_idx(j, a.ny, d)) * a.nx + i;
                    ex_y = cpml(ex_y, a.prof[1], a.ny, PR_BE, j, a.psi_in[PSI_EX_Y], a.psi_out[PSI_EX_Y], q, true);
                    ez_y = cpml(ez_y, a.prof[1], a.ny, PR_BE, j, a.psi_in[PSI_EZ_Y], a.psi_out[PSI_EZ_Y], q, true);
                }
                if (in_slab(k, a.nz, d)) {
                    const long long q = ((long long)slab_idx(k, a.nz, d) * a.ny + j) * a.nx + i;
                    ex_z = cpml(ex_z, a.prof[2], a.nz, PR_BE, k, a.psi_in[PSI_EX_Z], a.psi_out[PSI_EX_Z], q, true);
                    ey_z = cpml(ey_z, a.prof[2], a.nz, PR_BE, k, a.psi_in[PSI_EY_Z], a.psi_out[PSI_EY_Z], q, true);
                }
            }
            const float *t = s.tab + cl_own * kNumCoef;
            const long long g = fidx(a, i, j, k);
            a.Eout[0][g] = t[0] * s.e[bk][0][ly][lx] + t[3] * (ex_y - ex_z);
            a.Eout[1][g] = t[1] * s.e[bk][1][ly][lx] + t[4] * (ey_z - ey_x);
            a.Eout[2][g] = t[2] * s.e[bk][2][ly][lx] + t[5] * (ez_x - ez_y);
            hx_prev = hx;
            hy_prev = hy;
        }
    }
}

__device__ __forceinline__ long long eidx(const EdgeArgs &a, int i, int j, int k)
{
    return (long long)k * a.plane + (long long)j * a.pitch + i;
}

__global__ void edge_kernel(const EdgeArgs a)
{
    __shared__ long long n_s;
    if (threadIdx.x == 0) n_s = *a.step;
    __syncthreads();
    const long long n = n_s;
    for (int q = threadIdx.x; q < a.n_src; q += blockDim.x) {
        const SourceDesc sd = a.src[q];
        const float I = n < sd.n_samples ? a.samples[sd.sample_off + n] : 0.f;
        atomicAdd(a.E[sd.comp] + sd.idx, sd.coef * I);
    }
    __syncthreads();
    if (n < a.capacity) {
        for (int p = threadIdx.x; p < a.n_probes; p += blockDim.x) {
            const ProbeDesc pr = a.probes[p];
            float v = 0.f;
            if (pr.kind == 2) {
                v = a.E[pr.axis][eidx(a, pr.i, pr.j, pr.k)];
            } else if (pr.kind == 3) {
                v = a.H[pr.axis][eidx(a, pr.i, pr.j, pr.k)];
            } else if (pr.kind == 0) {
                int q[3] = {pr.i, pr.j, pr.k};
                for (int e = 0; e < pr.n_edges; ++e) {
                    v -= a.E[pr.axis][eidx(a, q[0], q[1], q[2])] * a.dx;
                    q[pr.axis]++;
                }
            } else {
                const float *Hx = a.H[0], *Hy = a.H[1], *Hz = a.H[2];
                const int i = pr.i, j = pr.j, k = pr.k;
                if (pr.axis == 2)
                    v = a.dx * ((Hy[eidx(a, i, j, k)] - Hy[eidx(a, i - 1, j, k)]) -
                                (Hx[eidx(a, i, j, k)] - Hx[eidx(a, i, j - 1, k)]));
                else if (pr.axis == 0)
                    v = a.dx * ((Hz[eidx(a, i, j, k)] - Hz[eidx(a, i, j - 1, k)]) -
                                (Hy[eidx(a, i, j, k)] - Hy[eidx(a, i, j, k - 1)]));
                else
                    v = a.dx * ((Hx[eidx(a, i, j, k)] - Hx[eidx(a, i, j, k - 1)]) -
                                (Hz[eidx(a, i, j, k)] - Hz[eidx(a, i - 1, j, k)]));
            }
            a.probe_out[(long long)p * a.capacity + n] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *a.step = n + 1;
}

}  // namespace

int step_tile_x() { return TX; }
int step_tile_y() { return TY; }

cudaError_t launch_step(const StepArgs &a, cudaStream_t s)
{
    dim3 block(TX, TY);
    dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (a.nz + a.kz - 1) / a.kz);
    step_kernel<<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_edges(const EdgeArgs &a, cudaStream_t s)
{
    edge_kernel<<<1, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace fdtd
