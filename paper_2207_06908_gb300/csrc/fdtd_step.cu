// fdtd_step.cu -- the fused Yee time step of the GB300 FDTD library
// (sm_103a, FP32): Kuklin, arXiv 2207.06908, Sec. 2.1, Eq. fdtdhx (H half
// step) then Eq. fdtdex (E half step, loss term time-averaged), with the
// CPML of Sec. 2.2, over the whole grid in one launch.
//
// Structure (one launch per time step; fields ping-pong between buffers):
//   - Work items are (z block, 32x16 column tile) pairs in z-block-major
//     order, handed out by an atomic counter to a persistent grid of
//     (SMs x resident CTAs); all CTAs march near the same z, so the halo
//     planes one CTA loads are still in L2 when its neighbours load them.
//     Within a z block the column tiles that meet a CPML layer come first:
//     the last items of a launch are the quick ones.
//   - One producer warp streams, plane by plane, TMA 3D boxes into two
//     shared-memory rings tracked by mbarriers: E^n (tile + 1-cell halo on
//     every side, x start rounded down to a 16-byte boundary) into a
//     4-slot ring (two planes in use, two in flight), and H^{n-1/2} (tile +
//     low halo), the class bytes and, in a CPML layer, the auxiliary fields
//     of one axis into a 3-slot ring (one in use, two in flight).
//   - Eight row warps: lane = x column, warp w owns rows w and w + 8 of the
//     tile (so a y layer's rows spread over all warps).  Per plane k they
//     form H^{n+1/2}(k) of their cells and store it, then E^{n+1}(k) from
//     that H plane and the owned column's H of plane k-1 kept in registers;
//     E^n(k+1) of the owned cells stays in registers for the next plane.  A ninth warp recomputes (never exchanges) H^{n+1/2} of
//     the low-y row and low-x column halo meanwhile, so every warp has the
//     same work between the two per-plane barriers.
//   - Items that touch no CPML layer run a variant compiled without any
//     CPML code; in the others the layer tests are hoisted per item, row
//     and plane.
// DRAM traffic per cell and step: 6 FP32 reads + 6 writes + 1 class byte
// (49 B) plus the CPML auxiliaries in the layer; every halo read is an L2
// hit.  Every wait is bounded; on a timeout the kernel records an error
// flag, drains its copies in flight and returns.
#include <cuda.h>

#include <algorithm>
#include <type_traits>

#include "fdtd.h"
#include "fdtd_internal.h"

namespace fdtd {
namespace {

using geom::TX;                        // tile width: one lane per column
using geom::TY;                        // tile height
constexpr int RW = 2;                  // rows per consumer warp (w and w + NCW)
constexpr int NCW = TY / RW;           // row warps
constexpr int NCONS = (NCW + 1) * 32;  // row warps + the halo warp
constexpr int NTHREADS = NCONS + 32;   // + the producer warp
constexpr int NE = 4;                  // E-plane ring: planes k, k+1 in use, two ahead
constexpr int NH_MAX = 3;              // H / class / CPML ring: plane k in use, up to two ahead
                                       // (a launch whose auxiliary region is large uses 2)

using geom::XO;
using geom::EBX;
using geom::EBY;
using geom::HBX;
using geom::HBY;
using geom::CXO;
using geom::CBX;
using geom::CBY;

constexpr int al128(int v) { return (v + 127) / 128 * 128; }

// Shared-memory copy of a class's coefficients: three float4 rows
// {db_x, db_y, db_z, 0}, {ca_x, ca_y, ca_z, 0}, {cb_x, cb_y, cb_z, 0}, so the
// H half step reads one 16-byte row and the E half step two (the global
// table keeps kNumCoef floats per class: ca[3], cb[3], db[3]).
constexpr int kTabStride = 12;
__device__ __forceinline__ int tab_src(int slot)
{
    const int r = slot >> 2, c = slot & 3;
    return c == 3 ? -1 : (r == 0 ? 6 + c : (r == 1 ? c : 3 + c));
}
constexpr int E_COMP = al128(EBX * EBY * 4);
constexpr int H_COMP = al128(HBX * HBY * 4);
constexpr int C_BYTES = al128(CBX * CBY);
constexpr int PE_BYTES = al128(TX * TY * 4);         // E-type psi box: the tile itself
// E slot: three E boxes and a header (item, plane, staged-layer flags,
// x-box start, y-box start)
constexpr int OFF_HDR = 3 * E_COMP;
constexpr int ESLOT = al128(OFF_HDR + 32);   // header: item, plane, flags, x start, y start, domain
// H slot: three H boxes, the class box, then the staged-auxiliary region
// (grid dependent size).  In a z-layer plane the region holds the z boxes
// (2 H-type with the H box, 2 E-type with the tile box); elsewhere the x
// boxes (4, narrowed along x) followed by the y boxes (4, narrowed along y).
constexpr int OFF_H = 0;
constexpr int OFF_C = 3 * H_COMP;
constexpr int OFF_PSI = OFF_C + C_BYTES;
constexpr int Z_BYTES = 2 * H_COMP + 2 * PE_BYTES;
constexpr uint32_t TX_E = 3u * EBX * EBY * 4;
constexpr uint32_t TX_H = 3u * HBX * HBY * 4 + CBX * CBY;
constexpr uint32_t TX_Z = 2u * HBX * HBY * 4 + 2u * TX * TY * 4;
constexpr int F_Z = 1, F_X = 2, F_Y = 4;              // staged-layer flags

__host__ __device__ constexpr int hslot_bytes(int region) { return al128(OFF_PSI + region); }

// block-level layout: E ring, H ring, H^{n+1/2} planes, barriers, misc,
// coefficient table, CPML profiles
constexpr int SM_EH = 0;
constexpr int SM_HH = NE * ESLOT;
constexpr int HNEW_PLANE = HBY * HBX;
constexpr int HNEW_BYTES = 2 * 3 * HNEW_PLANE * 4;     // [2][3][HBY][HBX]
constexpr int NBAR = 2 * NE + 2 * NH_MAX;             // fullE, emptyE, fullH, emptyH
struct Layout {
    int hslot, hnew, bar, misc, tab;
    __host__ __device__ Layout(int region, int nh)
    {
        hslot = hslot_bytes(region);
        hnew = SM_HH + nh * hslot;
        bar = hnew + HNEW_BYTES;
        misc = bar + NBAR * 8;
        tab = misc + 32;
    }
};

__host__ __device__ inline int smem_bytes(int n_classes, int d, int region, int nh)
{
    return Layout(region, nh).tab + al128(sizeof(StepArgs)) + n_classes * kTabStride * 4 + 3 * 2 * 2 * d * 16 +
           128;
}

constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s per wait

// ---- PTX helpers ----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait on one mbarrier phase; gives up on timeout (limit_ns) or when
// another warp of the CTA has already given up
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort,
                                          unsigned long long limit_ns = kWaitNs)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (*abort) return false;
        if (gtimer() - t0 > limit_ns) return false;
    }
}

// Self-test of the bounded wait: one thread waits, through mbar_wait, on an
// mbarrier phase that nothing will complete, gives up after limit_ns and
// records that in *flag (the step kernel's timeout path, without a step).
__global__ void wait_selftest_kernel(unsigned long long limit_ns, int *flag)
{
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        abort_flag = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool ok = mbar_wait(smem_u32(&bar), 0, &abort_flag, limit_ns);
        *flag = ok ? 2 : 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)) : "memory");
}

__device__ int g_selftest_flag;

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void consumer_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(NCONS) : "memory");
}

// ---- stencil cores ----------------------------------------------------------
// Layer membership of one cell, hoisted out of the per-cell work: slab
// index per axis (-1 outside the layer) and, per axis, the cell's entry in
// the staged boxes (null when not staged: read from global memory).
struct Slab {
    int sx, sy, sz;          // slab index along x, y, z or -1
    const float *base;       // staged-auxiliary region of the plane's H slot
    int xo, yo;              // float offsets of the cell in the first x / y box, or -1
    int zo, zeo;             // float offsets in the first z H-type / E-type box, or -1
};

__device__ __forceinline__ int slab_of(int i, int n, int d) { return i < d ? i : (i >= n - d ? i - (n - 2 * d) : -1); }

// CPML convolution of the two differences along one axis (Sec. 2.2): with
// the profile b, c, 1/kappa of the cell's slab entry s,
// psi <- b psi + c dif, dif <- dif / kappa + psi.  The profile row holds
// {b, c, 1/kappa, -} per slab entry, read with one 16-byte load for both
// differences, before any store.
template <bool WRITE>
__device__ __forceinline__ void cpml2(float &d0, float &d1, const float4 *pr, int s, float o0, float o1,
                                      float *out0, float *out1, int g, long long n, int *bounds)
{
    // g: the cell's element in its axis's compact auxiliary arrays (n elements)
    const float4 pv = pr[s];
    const float b = pv.x, c = pv.y, ki = pv.z;
    const float p0 = b * o0 + c * d0, p1 = b * o1 + c * d1;
    if (WRITE && in_bounds(g, n, 3, bounds)) {
        out0[g] = p0;
        out1[g] = p1;
    }
    d0 = d0 * ki + p0;
    d1 = d1 * ki + p1;
}

// Element of cell (i, j, k) in the compact auxiliaries of each axis, which
// hold only the layer: x [nz][ny][px] by slab column sx, y [nz][2d][pitch]
// by slab row sy, z [2d][ny][pitch] by slab plane sz (px = 2d rounded up to
// a multiple of 4, so rows stay 16-byte aligned for TMA).
// The host keeps every compact array below 2^31 elements, so 32-bit indices.
__device__ __forceinline__ int psi_x(const StepArgs &a, int sx, int j, int k) { return (k * a.ny + j) * a.px + sx; }
__device__ __forceinline__ int psi_y(const StepArgs &a, int i, int sy, int k)
{
    return (k * (2 * a.d) + sy) * a.pitch + i;
}
__device__ __forceinline__ int psi_z(const StepArgs &a, int i, int j, int sz)
{
    return (sz * a.ny + j) * a.pitch + i;
}
// elements of the compact x, y, z arrays (extents for the bounds-checked build)
__device__ __forceinline__ long long psi_n(const StepArgs &a, int u)
{
    return u == 0 ? (long long)a.nz * a.ny * a.px : (long long)(2 * a.d) * a.pitch * (u == 1 ? a.nz : a.ny);
}

// profile row of axis u at E (h = 0) or H (h = 1) positions in the staged
// profiles: [axis][E, H][2d slab entries] x {b, c, 1/kappa, -}
__device__ __forceinline__ const float4 *prow(const float *prof, int u, int h, int d2)
{
    return reinterpret_cast<const float4 *>(prof) + (u * 2 + h) * d2;
}

// H^{n+1/2} of cell (i,j,k) from E^n around it (Eq. fdtdhx and its cyclic
// analogues): Hx += db [dEy/dz - dEz/dy], Hy += db [dEz/dx - dEx/dz],
// Hz += db [dEx/dy - dEy/dx]; differences in field units, 1/dx in db.
// STAGED: every auxiliary the cell needs is in the staged boxes (true of
// the cells an item updates); otherwise one outside them is read from
// global memory.  WRITE: the cell is one the
// item updates, so the new auxiliaries are stored (halo and warm-up cells
// are recomputed only).
template <bool CPML, bool STAGED, bool WRITE>
__device__ __forceinline__ void h_core(const StepArgs &a, const float4 *t, const float *prof, const Slab &L,
                                       int i, int j, int k, float ex, float ey, float ez, float ey_x1, float ez_x1,
                                       float ex_y1, float ez_y1, float ex_z1, float ey_z1, float hx0, float hy0,
                                       float hz0, float &hx, float &hy, float &hz)
{
    float hx_z = ey_z1 - ey, hx_y = ez_y1 - ez;
    float hy_x = ez_x1 - ez, hy_z = ex_z1 - ex;
    float hz_y = ex_y1 - ex, hz_x = ey_x1 - ey;
    if (CPML) {
        const int d2 = 2 * a.d;
        if (L.sx >= 0) {
            const int q = a.pg.xb >> 2;
            const int g = psi_x(a, L.sx, j, k);
            const float o0 = (STAGED || L.xo >= 0) ? L.base[L.xo]
                                    : (in_bounds(g, psi_n(a, 0), 4, a.bounds) ? __ldg(a.psi_in[PSI_HY_X] + g) : 0.f);
            const float o1 = (STAGED || L.xo >= 0) ? L.base[L.xo + q]
                                    : (in_bounds(g, psi_n(a, 0), 4, a.bounds) ? __ldg(a.psi_in[PSI_HZ_X] + g) : 0.f);
            cpml2<WRITE>(hy_x, hz_x, prow(prof, 0, 1, d2), L.sx, o0, o1, a.psi_out[PSI_HY_X], a.psi_out[PSI_HZ_X], g,
                         psi_n(a, 0), a.bounds);
        }
        if (L.sy >= 0) {
            const int q = a.pg.yb >> 2;
            const int g = psi_y(a, i, L.sy, k);
            const float o0 = (STAGED || L.yo >= 0) ? L.base[L.yo]
                                    : (in_bounds(g, psi_n(a, 1), 4, a.bounds) ? __ldg(a.psi_in[PSI_HX_Y] + g) : 0.f);
            const float o1 = (STAGED || L.yo >= 0) ? L.base[L.yo + q]
                                    : (in_bounds(g, psi_n(a, 1), 4, a.bounds) ? __ldg(a.psi_in[PSI_HZ_Y] + g) : 0.f);
            cpml2<WRITE>(hx_y, hz_y, prow(prof, 1, 1, d2), L.sy, o0, o1, a.psi_out[PSI_HX_Y],
                         a.psi_out[PSI_HZ_Y], g, psi_n(a, 1), a.bounds);
        }
        if (L.sz >= 0) {
            const int g = psi_z(a, i, j, L.sz);
            const float o0 = (STAGED || L.zo >= 0) ? L.base[L.zo]
                                    : (in_bounds(g, psi_n(a, 2), 4, a.bounds) ? __ldg(a.psi_in[PSI_HX_Z] + g) : 0.f);
            const float o1 = (STAGED || L.zo >= 0) ? L.base[L.zo + H_COMP / 4]
                                    : (in_bounds(g, psi_n(a, 2), 4, a.bounds) ? __ldg(a.psi_in[PSI_HY_Z] + g) : 0.f);
            cpml2<WRITE>(hx_z, hy_z, prow(prof, 2, 1, d2), L.sz, o0, o1, a.psi_out[PSI_HX_Z],
                         a.psi_out[PSI_HY_Z], g, psi_n(a, 2), a.bounds);
        }
    }
    const float4 db = t[0];
    hx = hx0 + db.x * (hx_z - hx_y);
    hy = hy0 + db.y * (hy_x - hy_z);
    hz = hz0 + db.z * (hz_y - hz_x);
}

// E^{n+1} of cell (i,j,k) (Eq. fdtdex with sigma E time-averaged):
// E = ca E + cb [curl_h H^{n+1/2}], 1/dx in cb.  Only cells the item
// updates, whose auxiliaries are staged.
template <bool CPML>
__device__ __forceinline__ void e_core(const StepArgs &a, const float4 *t, const float *prof, const Slab &L,
                                       int i, int j, int k, float ex, float ey, float ez, float hx, float hy, float hz,
                                       float hz_ym, float hx_ym, float hz_xm, float hy_xm, float hx_zm,
                                       float hy_zm, float &ex1, float &ey1, float &ez1)
{
    float ex_y = hz - hz_ym, ex_z = hy - hy_zm;
    float ey_z = hx - hx_zm, ey_x = hz - hz_xm;
    float ez_x = hy - hy_xm, ez_y = hx - hx_ym;
    if (CPML) {
        const int d2 = 2 * a.d;
        if (L.sx >= 0) {
            const int q = a.pg.xb >> 2;
            cpml2<true>(ey_x, ez_x, prow(prof, 0, 0, d2), L.sx, L.base[L.xo + 2 * q], L.base[L.xo + 3 * q],
                        a.psi_out[PSI_EY_X], a.psi_out[PSI_EZ_X], psi_x(a, L.sx, j, k), psi_n(a, 0), a.bounds);
        }
        if (L.sy >= 0) {
            const int q = a.pg.yb >> 2;
            cpml2<true>(ex_y, ez_y, prow(prof, 1, 0, d2), L.sy, L.base[L.yo + 2 * q], L.base[L.yo + 3 * q],
                        a.psi_out[PSI_EX_Y], a.psi_out[PSI_EZ_Y], psi_y(a, i, L.sy, k), psi_n(a, 1), a.bounds);
        }
        if (L.sz >= 0)
            cpml2<true>(ex_z, ey_z, prow(prof, 2, 0, d2), L.sz, L.base[L.zeo],
                        L.base[L.zeo + PE_BYTES / 4], a.psi_out[PSI_EX_Z], a.psi_out[PSI_EY_Z], psi_z(a, i, j, L.sz),
                        psi_n(a, 2), a.bounds);
    }
    const float4 ca = t[1], cb = t[2];
    ex1 = ca.x * ex + cb.x * (ex_y - ex_z);
    ey1 = ca.y * ey + cb.y * (ey_z - ey_x);
    ez1 = ca.z * ez + cb.z * (ez_x - ez_y);
}

// Current sources of the grid whose edges lie in a finished work item (Sec.
// 2.1, J = I / dx^2 on one edge, I at t_{n+1/2}): E^{n+1} += coef I on each
// edge, rounded as a separate product and sum (the arithmetic of the source
// kernel's add to the stored E).  The item's consumers stored those E^{n+1}
// before the barrier that precedes this; no other CTA touches them in this
// step.  m: bit q set for each source q in the item.
__device__ __forceinline__ void add_sources(const StepArgs &a, uint32_t m)
{
    const long long n = __ldcg(a.step) + a.step_t;
    while (m) {
        const int q = __ffs(m) - 1;
        m &= m - 1;
        const SourceDesc &sd = a.src[q];
        const float I = n < sd.n_samples ? __ldg(a.samples + sd.sample_off + n) : 0.f;
        if (!in_bounds(sd.idx, (long long)a.plane * a.nz, 5, a.bounds)) continue;
        float *e = a.Eout[sd.comp] + sd.idx;
        *e = __fadd_rn(__ldcg(e), __fmul_rn(sd.coef, I));
    }
}

// sources that lie in work item `item` of launch `launch` (bit q: source q)
__device__ __forceinline__ uint32_t item_sources(const StepArgs &a, int launch, int item)
{
    uint32_t m = 0;
    for (int q = 0; q < a.n_isrc; ++q) {
        const int2 L = __ldg(a.isrc_loc + q);
        if (L.x == launch && L.y == item) m |= 1u << q;
    }
    return m;
}

// ---- shared-memory views ----------------------------------------------------
struct EView {
    char *p;
    __device__ float e(int c, int row, int col) const { return reinterpret_cast<const float *>(p + c * E_COMP)[row * EBX + col]; }
    __device__ int *hdr() const { return reinterpret_cast<int *>(p + OFF_HDR); }
};
struct HView {
    char *p;
    __device__ float h(int c, int row, int col) const { return reinterpret_cast<const float *>(p + OFF_H + c * H_COMP)[row * HBX + col]; }
    __device__ int cls(int row, int col) const { return reinterpret_cast<const uint8_t *>(p + OFF_C)[row * CBX + col]; }
    __device__ const float *psi() const { return reinterpret_cast<const float *>(p + OFF_PSI); }
};

// staging of one plane, copied out of its E-slot header (the E slot may be
// handed back to the producer before the plane's E half step)
struct Stg {
    int f, xs, ys;
    __device__ explicit Stg(const int *hdr) : f(hdr[2]), xs(hdr[3]), ys(hdr[4]) {}
    __device__ Stg(int f_, int xs_, int ys_) : f(f_), xs(xs_), ys(ys_) {}
};

// Offsets of cell (i, j) at H-box position (row, col) in the x / y boxes of
// an item (-1 when the cell is outside that layer or outside the box); they
// depend on the tile only, so they are formed once per item.
__device__ __forceinline__ int x_off(const StepArgs &a, const Stg &sg, int i, int row)
{
    const int sx = slab_of(i, a.nx, a.d);
    return (sx >= 0 && sx >= sg.xs && sx < sg.xs + a.pg.w) ? a.ox / 4 + row * a.pg.w + (sx - sg.xs) : -1;
}
__device__ __forceinline__ int y_off(const StepArgs &a, const Stg &sg, int x0, int i, int j)
{
    const int sy = slab_of(j, a.ny, a.d);
    return (sy >= 0 && sy >= sg.ys && sy < sg.ys + a.pg.hy) ? a.oy / 4 + (sy - sg.ys) * HBX + (i - (x0 - XO)) : -1;
}

// the staging of one plane applied to a cell's precomputed offsets
__device__ __forceinline__ Slab slab_in(const Stg &sg, const HView &hv, int sx, int sy, int sz, int xo, int yo,
                                        int zo, int zeo)
{
    const bool z = sg.f & F_Z;
    return Slab{sx, sy, sz, hv.psi(), (sg.f & F_X) ? xo : -1, (sg.f & F_Y) ? yo : -1, z ? zo : -1, z ? zeo : -1};
}

// x / y layer boxes of a tile (with its low halo): whether the tile touches
// the layer and where the box narrowed to the layer starts
__device__ __forceinline__ int tile_boxes(const StepArgs &a, int x0, int y0, int &xs, int &ys)
{
    // the layer cells among x0-1 .. x0+TX-1 (y0-1 .. y0+TY-1) form one run of
    // slab entries (the low layer's, then the high layer's, contiguous in
    // the compact arrays); the x box starts at the first, rounded down to a
    // 16-byte boundary, the y box at the first
    const int d = a.d;
    int f = 0;
    xs = 0;
    ys = 0;
    const int xl = max(x0 - 1, 0), xh = min(x0 + TX, a.nx) - 1;
    if (xl < d || xh >= a.nx - d) {
        f |= F_X;
        xs = slab_of(xl < d ? xl : max(xl, a.nx - d), a.nx, d) & ~3;
    }
    const int yl = max(y0 - 1, 0), yh = min(y0 + TY, a.ny) - 1;
    if (yl < d || yh >= a.ny - d) {
        f |= F_Y;
        ys = slab_of(yl < d ? yl : max(yl, a.ny - d), a.ny, d);
    }
    return f;
}

// staged-layer flags and box starts of plane z of a tile: the x and / or y
// layer boxes of the tile, and the z boxes when the plane is in the z
// layer (alone, unless the launch has room for all three)
__device__ __forceinline__ void staging(const StepArgs &a, int x0, int y0, int z, int &f, int &xs, int &ys)
{
    f = 0;
    xs = 0;
    ys = 0;
    if (a.d == 0 || z < 0 || z >= a.nz) return;
    const bool zs = z < a.d || z >= a.nz - a.d;
    if (zs && !a.zxy) {
        f = F_Z;
        return;
    }
    f = tile_boxes(a, x0, y0, xs, ys) | (zs ? F_Z : 0);
}

struct Item {
    int x0, y0, ka, kb;
};

__device__ __forceinline__ Item decode(const StepArgs &a, int item)
{
    const int ncols = a.ncx * a.ncy;
    const int zb = item / ncols;
    // within a z block the column tiles that meet a CPML layer (the slowest
    // items) come first, so the items handed out last in a launch are the
    // quickest and the launch's tail is short
    const int col = __ldg(a.col_order + (item - zb * ncols));
    Item it;
    it.x0 = (col % a.ncx) * TX;
    it.y0 = (col / a.ncx) * TY;
    const int nzb1 = (a.zhi - a.zlo + a.kz - 1) / a.kz;
    if (zb < nzb1) {
        it.ka = a.zlo + zb * a.kz;
        it.kb = min(it.ka + a.kz, a.zhi);
    } else {
        it.ka = a.zlo2 + (zb - nzb1) * a.kz;
        it.kb = min(it.ka + a.kz, a.zhi2);
    }
    return it;
}

// does any cell the item updates or recomputes lie in a CPML layer
__device__ __forceinline__ bool item_in_cpml(const StepArgs &a, const Item &it)
{
    const int d = a.d;
    if (d == 0) return false;
    if (it.ka - 1 < d || it.kb - 1 >= a.nz - d) return true;
    const int xl = max(it.x0 - 1, 0), xh = min(it.x0 + TX, a.nx) - 1;
    const int yl = max(it.y0 - 1, 0), yh = min(it.y0 + TY, a.ny) - 1;
    return xl < d || xh >= a.nx - d || yl < d || yh >= a.ny - d;
}

// shared state of the consumer warps
template <int NH>
struct Cons {
    const StepArgs *a;
    char *smem;
    const float *tab, *prof;
    float *hnew;
    uint64_t *bars;
    volatile int *abort;
    int warp, lane;
    bool halo;               // the halo warp
    int hslot;               // bytes per H slot
    __device__ uint32_t bar(int b) const { return (uint32_t)__cvta_generic_to_shared(&bars[b]); }
    __device__ const float4 *coef(int cls) const { return reinterpret_cast<const float4 *>(tab + cls * kTabStride); }
    __device__ uint32_t fullE(uint32_t q) const { return bar(q % NE); }
    __device__ uint32_t emptyE(uint32_t q) const { return bar(NE + q % NE); }
    __device__ uint32_t fullH(uint32_t q) const { return bar(2 * NE + q % NH); }
    __device__ uint32_t emptyH(uint32_t q) const { return bar(2 * NE + NH_MAX + q % NH); }
    __device__ EView ev(uint32_t q) const { return EView{smem + SM_EH + (q % NE) * ESLOT}; }
    __device__ HView hv(uint32_t q) const { return HView{smem + SM_HH + (q % NH) * hslot}; }
    __device__ float &hn(uint32_t b, int c, int row, int col) const { return hnew[(b * 3 + c) * HNEW_PLANE + row * HBX + col]; }
    __device__ void arrive(uint32_t b) const
    {
        __syncwarp();
        if (lane == 0) mbar_arrive(b);
    }
    __device__ bool waitE(uint32_t q) const { return mbar_wait(fullE(q), (q / NE) & 1, abort); }
    __device__ bool waitH(uint32_t q) const { return mbar_wait(fullH(q), (q / NH) & 1, abort); }
};

// one work item.  Its planes ka-1 .. kb occupy E slots qe0 .. qe0+kb-ka+1
// and planes ka-1 .. kb-1 H slots qh0 .. qh0+kb-ka.  Returns false when a
// wait gave up (the CTA then aborts).
// WIDE: 64-bit element indices for the field stores (grids of 2^31
// elements or more); 32-bit otherwise, fewer registers in the plane loop
template <bool CPML, int NH, bool WIDE>
__device__ __forceinline__ bool run_item(const Cons<NH> &C, const Item &it, uint32_t qe0, uint32_t qh0, uint32_t &hb)
{
    using Idx = typename std::conditional<WIDE, long long, int>::type;
    const StepArgs &a = *C.a;
    const int lane = C.lane;
    const int lx = XO + lane, clx = CXO + lane;
    const int i = it.x0 + lane;
    const int d = a.d;
    float ecur[3][RW], hxp[RW], hyp[RW];
    int sy[RW], xo[RW], yo[RW];
    const int sx = CPML ? slab_of(i, a.nx, d) : -1;
    Stg tb(0, 0, 0);                // the tile's x / y layer boxes
    if (CPML) tb.f = tile_boxes(a, it.x0, it.y0, tb.xs, tb.ys);
    for (int r = 0; r < RW; ++r) {
        const int row = 1 + C.warp + r * NCW, j = it.y0 + C.warp + r * NCW;
        sy[r] = CPML ? slab_of(j, a.ny, d) : -1;
        xo[r] = (CPML && (tb.f & F_X)) ? x_off(a, tb, i, row) : -1;
        yo[r] = (CPML && (tb.f & F_Y)) ? y_off(a, tb, it.x0, i, j) : -1;
        hxp[r] = 0.f;
        hyp[r] = 0.f;
    }
    // halo cells of the halo warp: pass 0 = (i, y0-1), pass 1 = (x0-1, y0+lane)
    int hxo[2] = {-1, -1}, hyo[2] = {-1, -1};
    if (CPML && C.halo) {
        if (tb.f & F_X) {
            hxo[0] = x_off(a, tb, i, 0);
            hxo[1] = x_off(a, tb, it.x0 - 1, 1 + lane);
        }
        if (tb.f & F_Y) {
            hyo[0] = y_off(a, tb, it.x0, i, it.y0 - 1);
            hyo[1] = y_off(a, tb, it.x0, it.x0 - 1, it.y0 + lane);
        }
    }
    bool ok = C.waitH(qh0);
    if (!ok) *C.abort = 1;
    if (ok && !C.halo) {
        const EView e0 = C.ev(qe0), e1 = C.ev(qe0 + 1);
        const HView h0 = C.hv(qh0);
        // owned E^n(ka) and, below the block, the owned Hx, Hy of plane ka-1
        for (int r = 0; r < RW; ++r) {
            const int row = 1 + C.warp + r * NCW;
            for (int c = 0; c < 3; ++c) ecur[c][r] = e1.e(c, row, lx);
        }
        if (it.ka > 0) {
            const int k = it.ka - 1;
            for (int r = 0; r < RW; ++r) {
                const int row = 1 + C.warp + r * NCW, j = it.y0 + C.warp + r * NCW;
                if (i < a.nx && j < a.ny) {
                    float hz;
                    const Slab L = CPML ? slab_in(Stg(e0.hdr()), h0, sx, sy[r], slab_of(k, a.nz, d), xo[r], yo[r],
                                                  row * HBX + lx, -1)
                                        : Slab{-1, -1, -1, nullptr, -1, -1, -1, -1};
                    h_core<CPML, false, false>(a, C.coef(h0.cls(row, clx)), C.prof, L, i, j, k, e0.e(0, row, lx),
                                 e0.e(1, row, lx), e0.e(2, row, lx), e0.e(1, row, lx + 1), e0.e(2, row, lx + 1),
                                 e0.e(0, row + 1, lx), e0.e(2, row + 1, lx), ecur[0][r], ecur[1][r],
                                 h0.h(0, row, lx), h0.h(1, row, lx), h0.h(2, row, lx), hxp[r], hyp[r], hz);
                }
            }
        }
    }
    C.arrive(C.emptyE(qe0));
    C.arrive(C.emptyH(qh0));
    if (!ok) return false;
    for (int k = it.ka; k < it.kb; ++k) {
        const uint32_t t = (uint32_t)(k - it.ka);
        const uint32_t qe = qe0 + 1 + t, qh = qh0 + 1 + t;     // plane k
        ok = C.waitE(qe + 1) && C.waitH(qh);
        if (!ok) *C.abort = 1;
        const EView ek = C.ev(qe), ek1 = C.ev(qe + 1);
        const HView hk = C.hv(qh);
        const int sz = CPML ? slab_of(k, a.nz, d) : -1;
        const Stg sg(ek.hdr());
        float hnw[3][RW], enx[3][RW];
        int cl[RW];
        if (ok && !C.halo) {
            for (int r = 0; r < RW; ++r) {
                const int row = 1 + C.warp + r * NCW, j = it.y0 + C.warp + r * NCW;
                for (int c = 0; c < 3; ++c) enx[c][r] = ek1.e(c, row, lx);
                cl[r] = hk.cls(row, clx);
                const float ex_y1 = ek.e(0, row + 1, lx);
                const float ez_y1 = ek.e(2, row + 1, lx);
                float hx = 0.f, hy = 0.f, hz = 0.f;
                if (i < a.nx && j < a.ny) {
                    const Idx g = (Idx)k * (Idx)a.plane + (Idx)j * a.pitch + i;
                    const Slab L = CPML ? slab_in(sg, hk, sx, sy[r], sz, xo[r], yo[r], row * HBX + lx,
                                                  (2 * H_COMP) / 4 + (row - 1) * TX + lane)
                                        : Slab{-1, -1, -1, nullptr, -1, -1, -1, -1};
                    h_core<CPML, true, true>(a, C.coef(cl[r]), C.prof, L, i, j, k, ecur[0][r], ecur[1][r],
                                 ecur[2][r], ek.e(1, row, lx + 1), ek.e(2, row, lx + 1), ex_y1, ez_y1, enx[0][r],
                                 enx[1][r], hk.h(0, row, lx), hk.h(1, row, lx), hk.h(2, row, lx), hx, hy, hz);
                    if (in_bounds(g, (long long)a.plane * a.nz, 1, a.bounds)) {
                        a.Hout[0][g] = hx;
                        a.Hout[1][g] = hy;
                        a.Hout[2][g] = hz;
                    }
                }
                hnw[0][r] = hx;
                hnw[1][r] = hy;
                hnw[2][r] = hz;
                C.hn(hb, 0, row, lx) = hx;
                C.hn(hb, 1, row, lx) = hy;
                C.hn(hb, 2, row, lx) = hz;
            }
        } else if (ok) {
            // halo warp: low-y row (all lanes), then low-x column (TY lanes)
            for (int pass = 0; pass < 2; ++pass) {
                int hrow, hcol, hi, hj;
                if (pass == 0) { hrow = 0; hcol = lx; hi = i; hj = it.y0 - 1; }
                else { hrow = 1 + lane; hcol = XO - 1; hi = it.x0 - 1; hj = it.y0 + lane; }
                if (pass == 1 && lane >= TY) break;
                float hx = 0.f, hy = 0.f, hz = 0.f;
                if (hi >= 0 && hj >= 0 && hi < a.nx && hj < a.ny) {
                    const Slab L = CPML ? slab_in(sg, hk, slab_of(hi, a.nx, d), slab_of(hj, a.ny, d), sz, hxo[pass],
                                                  hyo[pass], hrow * HBX + hcol, -1)
                                        : Slab{-1, -1, -1, nullptr, -1, -1, -1, -1};
                    h_core<CPML, false, false>(a, C.coef(hk.cls(hrow, hcol - XO + CXO)), C.prof, L, hi, hj, k,
                                 ek.e(0, hrow, hcol), ek.e(1, hrow, hcol), ek.e(2, hrow, hcol),
                                 ek.e(1, hrow, hcol + 1), ek.e(2, hrow, hcol + 1), ek.e(0, hrow + 1, hcol),
                                 ek.e(2, hrow + 1, hcol), ek1.e(0, hrow, hcol), ek1.e(1, hrow, hcol),
                                 hk.h(0, hrow, hcol), hk.h(1, hrow, hcol), hk.h(2, hrow, hcol), hx, hy, hz);
                }
                C.hn(hb, 0, hrow, hcol) = hx;
                C.hn(hb, 1, hrow, hcol) = hy;
                C.hn(hb, 2, hrow, hcol) = hz;
            }
        }
        consumer_sync();            // H^{n+1/2} of plane k complete (tile + halo)
        C.arrive(C.emptyE(qe));     // E(k) is not read again
        if (*C.abort) {
            C.arrive(C.emptyH(qh));
            return false;
        }
        if (!C.halo) {
            for (int r = 0; r < RW; ++r) {
                const int row = 1 + C.warp + r * NCW, j = it.y0 + C.warp + r * NCW;
                if (i < a.nx && j < a.ny) {
                    const float hz_ym = C.hn(hb, 2, row - 1, lx);
                    const float hx_ym = C.hn(hb, 0, row - 1, lx);
                    const Idx g = (Idx)k * (Idx)a.plane + (Idx)j * a.pitch + i;
                    const Slab L = CPML ? slab_in(sg, hk, sx, sy[r], sz, xo[r], yo[r], row * HBX + lx,
                                                  (2 * H_COMP) / 4 + (row - 1) * TX + lane)
                                        : Slab{-1, -1, -1, nullptr, -1, -1, -1, -1};
                    float ex1, ey1, ez1;
                    e_core<CPML>(a, C.coef(cl[r]), C.prof, L, i, j, k, ecur[0][r], ecur[1][r], ecur[2][r],
                                 hnw[0][r], hnw[1][r], hnw[2][r], hz_ym, hx_ym, C.hn(hb, 2, row, lx - 1),
                                 C.hn(hb, 1, row, lx - 1), hxp[r], hyp[r], ex1, ey1, ez1);
                    if (in_bounds(g, (long long)a.plane * a.nz, 2, a.bounds)) {
                        a.Eout[0][g] = ex1;
                        a.Eout[1][g] = ey1;
                        a.Eout[2][g] = ez1;
                    }
                }
                hxp[r] = hnw[0][r];
                hyp[r] = hnw[1][r];
                for (int c = 0; c < 3; ++c) ecur[c][r] = enx[c][r];
            }
        }
        C.arrive(C.emptyH(qh));     // this warp is done with plane k's H slot
        hb ^= 1u;
    }
    C.arrive(C.emptyE(qe0 + 1 + (uint32_t)(it.kb - it.ka)));   // plane kb (E only)
    return true;
}

// domain of global work item q: item_start[d] <= q < item_start[d + 1]
__device__ __forceinline__ int find_domain(const int *item_start, int n, int q)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(item_start + mid) <= q) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// BATCH = false: one domain whose arguments and descriptors are the kernel's
// own parameters (constant bank); BATCH = true: a table of domains in global
// memory, the current domain's arguments staged in shared memory.
template <int NH, bool BATCH, bool WIDE>
__global__ void __launch_bounds__(NTHREADS, 2) step_tma_kernel(const __grid_constant__ SingleArgs S,
                                                              const BatchArgs B)
{
    extern __shared__ __align__(128) char smem_raw[];
    // TMA destinations are kept 128-byte aligned
    char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Layout Lo(B.region, NH);
    StepArgs *sa = reinterpret_cast<StepArgs *>(smem + Lo.tab);          // current domain's arguments
    float *tab = reinterpret_cast<float *>(smem + Lo.tab + al128(sizeof(StepArgs)));
    float *prof = tab + B.max_classes * kTabStride;  // [axis][E, H][2d] x {b, c, 1/kappa, -}, slab entries only
    float *hnew = reinterpret_cast<float *>(smem + Lo.hnew);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + Lo.bar);
    volatile int *abort = reinterpret_cast<volatile int *>(smem + Lo.misc);
    int *cons_e = reinterpret_cast<int *>(smem + Lo.misc + 4);
    int *cons_h = reinterpret_cast<int *>(smem + Lo.misc + 8);
    int *iss_e = reinterpret_cast<int *>(smem + Lo.misc + 12);
    int *iss_h = reinterpret_cast<int *>(smem + Lo.misc + 16);
    Cons<NH> C{BATCH ? sa : &S.a, smem, tab, prof, hnew, bars, abort, warp, lane, warp == NCW, Lo.hslot};

    if (!BATCH) {
        // the one domain's coefficient table and CPML profiles, once
        const StepArgs &ga = S.a;
        for (int q = threadIdx.x; q < ga.n_classes * kTabStride; q += NTHREADS) {
            const int cl = q / kTabStride, src = tab_src(q - cl * kTabStride);
            tab[q] = src < 0 ? 0.f : __ldg(ga.table + cl * kNumCoef + src);
        }
        if (ga.d > 0) {
            const int d2 = 2 * ga.d, per = PR_COUNT * d2;
            for (int q = threadIdx.x; q < 3 * per; q += NTHREADS) {
                const int u = q / per, w = (q - u * per) / d2, sl = q - u * per - w * d2;
                const int n = u == 0 ? ga.nx : (u == 1 ? ga.ny : ga.nz);
                const int i = sl < ga.d ? sl : n - d2 + sl;
                prof[(((u * 2 + w / 3) * d2 + sl) << 2) + w % 3] = __ldg(ga.prof[u] + w * n + i);
            }
        }
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < NE; ++q) {
            mbar_init(C.fullE(q), 1);
            mbar_init(C.emptyE(q), NCW + 1);
        }
        for (int q = 0; q < NH; ++q) {
            mbar_init(C.fullH(q), 1);
            mbar_init(C.emptyH(q), NCW + 1);
        }
        *abort = 0;
        *cons_e = *cons_h = *iss_e = *iss_h = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == NCW + 1) {
        // ------------------------------ producer ------------------------------
        if (lane == 0) {
            uint32_t qe = 0, qh = 0;
            bool ok = true;
            while (ok) {
                const int gitem = atomicAdd(B.work, 1);
                if (gitem >= B.nitems) break;
                const int dom = BATCH ? find_domain(B.item_start, B.n_domains, gitem) : 0;
                const StepArgs &a = BATCH ? B.doms[dom].a[B.launch][B.parity] : S.a;
                const TmaMaps &m = BATCH ? B.doms[dom].m[B.parity] : S.m;
                const int item = BATCH ? gitem - __ldg(B.item_start + dom) : gitem;
                const Item it = decode(a, item);
                for (int z = it.ka - 1; z <= it.kb; ++z) {
                    const bool e_only = (z == it.kb);
                    int f = 0, xs = 0, ys = 0;
                    if (!e_only) staging(a, it.x0, it.y0, z, f, xs, ys);
                    if (!mbar_wait(C.emptyE(qe), ((qe / NE) & 1) ^ 1, abort)) { ok = false; break; }
                    char *es = smem + SM_EH + (qe % NE) * ESLOT;
                    int *hdr = reinterpret_cast<int *>(es + OFF_HDR);
                    hdr[0] = item;
                    hdr[1] = z;
                    hdr[2] = f;
                    hdr[3] = xs;
                    hdr[4] = ys;
                    hdr[5] = dom;
                    mbar_expect_tx(C.fullE(qe), TX_E);
                    for (int c = 0; c < 3; ++c)
                        tma_load_3d(smem_u32(es + c * E_COMP), &m.e[c], it.x0 - XO, it.y0 - 1, z, C.fullE(qe));
                    ++qe;
                    if (e_only) continue;
                    if (!mbar_wait(C.emptyH(qh), ((qh / NH) & 1) ^ 1, abort)) { ok = false; break; }
                    char *hs = smem + SM_HH + (qh % NH) * Lo.hslot;
                    const uint32_t txb = TX_H + ((f & F_Z) ? TX_Z : 0u) +
                                         ((f & F_X) ? 4u * a.pg.w * HBY * 4 : 0u) +
                                         ((f & F_Y) ? 4u * HBX * a.pg.hy * 4 : 0u);
                    const uint32_t fb = C.fullH(qh);
                    mbar_expect_tx(fb, txb);
                    for (int c = 0; c < 3; ++c)
                        tma_load_3d(smem_u32(hs + OFF_H + c * H_COMP), &m.h[c], it.x0 - XO, it.y0 - 1, z, fb);
                    tma_load_3d(smem_u32(hs + OFF_C), &m.c, it.x0 - CXO, it.y0 - 1, z, fb);
                    char *ps = hs + OFF_PSI;
                    if (f & F_Z) {
                        for (int q = 0; q < 2; ++q) {
                            const int sz = slab_of(z, a.nz, a.d);     // plane of the compact z arrays
                            tma_load_3d(smem_u32(ps + q * H_COMP), &m.zh[q], it.x0 - XO, it.y0 - 1, sz, fb);
                            tma_load_3d(smem_u32(ps + 2 * H_COMP + q * PE_BYTES), &m.ze[q], it.x0, it.y0, sz, fb);
                        }
                    }
                    if (f & F_X) {
                        for (int q = 0; q < 2; ++q) {
                            tma_load_3d(smem_u32(ps + a.ox + q * a.pg.xb), &m.xh[q], xs, it.y0 - 1, z, fb);
                            tma_load_3d(smem_u32(ps + a.ox + (2 + q) * a.pg.xb), &m.xe[q], xs, it.y0 - 1, z, fb);
                        }
                    }
                    if (f & F_Y) {
                        char *py = ps + a.oy;
                        for (int q = 0; q < 2; ++q) {
                            tma_load_3d(smem_u32(py + q * a.pg.yb), &m.yh[q], it.x0 - XO, ys, z, fb);
                            tma_load_3d(smem_u32(py + (2 + q) * a.pg.yb), &m.ye[q], it.x0 - XO, ys, z, fb);
                        }
                    }
                    ++qh;
                }
            }
            if (ok) {
                // end marker: an E slot whose header carries item -1
                if (mbar_wait(C.emptyE(qe), ((qe / NE) & 1) ^ 1, abort)) {
                    int *hdr = reinterpret_cast<int *>(smem + SM_EH + (qe % NE) * ESLOT + OFF_HDR);
                    hdr[0] = -1;
                    hdr[1] = 0;
                    hdr[2] = 0;
                    hdr[5] = -1;
                    mbar_arrive(C.fullE(qe));
                    ++qe;
                } else {
                    ok = false;
                }
            }
            if (!ok) {
                *abort = 1;
                atomicExch(B.err, 1);
            }
            *iss_e = (int)qe;
            *iss_h = (int)qh;
            // the last CTA to finish handing out work resets the counters
            __threadfence();
            if (atomicAdd(B.work + 1, 1) == (int)gridDim.x - 1) {
                B.work[0] = 0;
                B.work[1] = 0;
                __threadfence();
            }
        }
    } else {
        // ------------------------- row warps and halo warp -------------------------
        uint32_t ce = 0, ch = 0, hb = 0;
        int cur = -1;                   // domain whose arguments are staged
        const int tid = threadIdx.x;
        while (true) {
            // first plane of the next item (or the end marker)
            bool ok = C.waitE(ce);
            if (!ok) *abort = 1;
            consumer_sync();
            if (*abort) break;
            const int *hdr = C.ev(ce).hdr();
            const int item = hdr[0], dom = hdr[5];
            if (item < 0) break;
            if (BATCH && dom != cur) {
                // stage this domain's image -- its arguments, coefficient
                // table rows and CPML profile rows, which the host laid out
                // exactly as their shared-memory copy -- in one round of
                // independent 16-byte loads
                const int2 ref = __ldg(B.img_ref + (dom * 2 + B.launch) * 2 + B.parity);
                const int4 *src = B.img + ref.x;
                int4 *dst = reinterpret_cast<int4 *>(sa);
                for (int q = tid; q < ref.y; q += NCONS) dst[q] = __ldg(src + q);
                cur = dom;
                consumer_sync();
            }
            const StepArgs &a = *C.a;
            const Item it = decode(a, item);
            ok = C.waitE(ce + 1);
            if (!ok) *abort = 1;
            consumer_sync();
            if (*abort) break;
            const bool done = item_in_cpml(a, it) ? run_item<true, NH, WIDE>(C, it, ce, ch, hb)
                                                  : run_item<false, NH, WIDE>(C, it, ce, ch, hb);
            if (!done) break;
            if (!BATCH && a.n_isrc > 0) {
                // current sources on the item's edges, after all its E stores
                const uint32_t m = item_sources(a, B.launch, item);
                if (m) {
                    consumer_sync();
                    if (tid == 0) add_sources(a, m);
                }
            }
            ce += (uint32_t)(it.kb - it.ka) + 2;
            ch += (uint32_t)(it.kb - it.ka) + 1;
        }
        if (threadIdx.x == 0) {
            *cons_e = (int)ce;
            *cons_h = (int)ch;
        }
    }
    __syncthreads();
    // on an abort, wait (bounded) for copies still in flight before the
    // shared memory is given back
    if (threadIdx.x == 0 && *abort) {
        atomicExch(B.err, 1);
        const unsigned long long t0 = gtimer();
        for (int q = *cons_e; q < *iss_e; ++q)
            while (!mbar_try(C.fullE(q), (q / NE) & 1))
                if (gtimer() - t0 > kWaitNs) break;
        for (int q = *cons_h; q < *iss_h; ++q)
            while (!mbar_try(C.fullH(q), (q / NH) & 1))
                if (gtimer() - t0 > kWaitNs) break;
    }
}

}  // namespace

int step_tile_x() { return TX; }
int step_tile_y() { return TY; }
int step_threads() { return NTHREADS; }
int step_smem_bytes(int n_classes, int d, int region, int nh) { return smem_bytes(n_classes, d, region, nh); }
int step_tab_offset() { return al128(sizeof(StepArgs)); }

PsiGeom step_psi_geom(int d, int nx, int ny)
{
    PsiGeom pg{};
    if (d == 0) return pg;
    // the x (y) box of a tile spans the slab entries of the layer cells
    // among x0-1 .. x0+TX-1 (y0-1 .. y0+TY-1), from the first (rounded down
    // to a multiple of 4 along x) to the last: the largest span over the tiles
    auto slab = [d](int i, int n) { return i < d ? i : (i >= n - d ? i - (n - 2 * d) : -1); };
    int w = 0, hy = 0;
    for (int x0 = 0; x0 < nx; x0 += TX) {
        const int xl = std::max(x0 - 1, 0), xh = std::min(x0 + TX, nx) - 1;
        if (!(xl < d || xh >= nx - d)) continue;
        const int first = slab(xl < d ? xl : std::max(xl, nx - d), nx) & ~3;
        const int last = slab(xh >= nx - d ? xh : std::min(xh, d - 1), nx);
        w = std::max(w, (last - first + 1 + 3) / 4 * 4);
    }
    for (int y0 = 0; y0 < ny; y0 += TY) {
        const int yl = std::max(y0 - 1, 0), yh = std::min(y0 + TY, ny) - 1;
        if (!(yl < d || yh >= ny - d)) continue;
        const int first = slab(yl < d ? yl : std::max(yl, ny - d), ny);
        const int last = slab(yh >= ny - d ? yh : std::min(yh, d - 1), ny);
        hy = std::max(hy, last - first + 1);
    }
    pg.w = w;
    pg.hy = hy;
    pg.xb = al128(pg.w * HBY * 4);
    pg.yb = al128(HBX * pg.hy * 4);
    return pg;
}

void step_region(const PsiGeom &pg, int zxy, int *region, int *ox, int *oy)
{
    if (pg.w == 0) {
        *region = *ox = *oy = 0;
    } else if (zxy) {
        *ox = Z_BYTES;
        *oy = Z_BYTES + 4 * pg.xb;
        *region = *oy + 4 * pg.yb;
    } else {
        *ox = 0;
        *oy = 4 * pg.xb;
        *region = std::max(Z_BYTES, *oy + 4 * pg.yb);
    }
}
const void *step_kernel_ptr(int nh, bool batch, bool wide)
{
    if (batch) return nh == 2 ? (const void *)step_tma_kernel<2, true, false> : (const void *)step_tma_kernel<3, true, false>;
    if (wide) return nh == 2 ? (const void *)step_tma_kernel<2, false, true> : (const void *)step_tma_kernel<3, false, true>;
    return nh == 2 ? (const void *)step_tma_kernel<2, false, false> : (const void *)step_tma_kernel<3, false, false>;
}

cudaError_t launch_step(const SingleArgs &one, const BatchArgs &b, int grid, cudaStream_t s)
{
    const int smem = smem_bytes(b.max_classes, b.max_d, b.region, b.nh);
    const bool batch = b.doms != nullptr;
    if (b.nh == 2) {
        if (batch) step_tma_kernel<2, true, false><<<grid, NTHREADS, smem, s>>>(one, b);
        else if (b.wide) step_tma_kernel<2, false, true><<<grid, NTHREADS, smem, s>>>(one, b);
        else step_tma_kernel<2, false, false><<<grid, NTHREADS, smem, s>>>(one, b);
    } else {
        if (batch) step_tma_kernel<3, true, false><<<grid, NTHREADS, smem, s>>>(one, b);
        else if (b.wide) step_tma_kernel<3, false, true><<<grid, NTHREADS, smem, s>>>(one, b);
        else step_tma_kernel<3, false, false><<<grid, NTHREADS, smem, s>>>(one, b);
    }
    return cudaGetLastError();
}

}  // namespace fdtd

extern "C" int fdtd_selftest_wait(double seconds, void *cuda_stream)
{
    if (!(seconds > 0.0) || seconds > 10.0) return FDTD_EINVAL;
    int *flag = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&flag), fdtd::g_selftest_flag);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        fdtd::wait_selftest_kernel<<<1, 32, 0, s>>>((unsigned long long)(seconds * 1e9), flag);
        e = cudaGetLastError();
    }
    int v = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v, flag, sizeof v, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return FDTD_ECUDA;
    return v == 1 ? FDTD_ETIMEOUT : (v == 2 ? FDTD_OK : FDTD_ECUDA);
}
