// fdtd_mlp.cu -- surrogate-network kernels (BF16 operands, FP32 accumulate).
//
// Every contraction runs on the fifth-generation tensor cores
// (tcgen05.mma, BF16 x BF16 -> FP32 in TMEM).  Forward layers (x wt^T +
// bias, GELU) with k <= 256: one CTA per 128 x 64 output tile stages the
// whole K extent of both operands in shared memory (no-swizzle K-major
// core-matrix layout), one thread issues the MMA chain into a TMEM
// accumulator, and the eight warps read it back with tcgen05.ld for the
// bias / GELU epilogue.  The gradients (dz wt and dz^T x, whose operands
// are not K-major in memory) and forward layers with larger k use the same
// tile and epilogue with the reduction in chunks, each chunk staged through
// registers from operands addressed by element strides.  Inference runs a
// whole network in one launch (net_forward_kernel: a cluster of four CTAs per
// 128 rows, weights resident in shared memory, activations exchanged through
// distributed shared memory).  Small element-wise kernels form
// dz = dy * act'(z), the bias gradient, the losses and the Adam update.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "fdtd.h"
#include "fdtd_mlp.h"

namespace {


__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

struct Epi {
    int mode;                 // 0: forward (bias, act, bf16 / f32 / z outputs); 1: plain FP32 store
    const float *bias;
    int act;
    __nv_bfloat16 *yb;
    float *yf;
    float *zf;
    int ldc;
};

__global__ void act_grad_kernel(const float *__restrict__ dy, const float *__restrict__ z, float *__restrict__ dz,
                                long long count, int act)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x)
        dz[q] = act == FDTD_ACT_GELU ? dy[q] * gelu_grad(z[q]) : dy[q];
}

// db[n] = sum over rows of dz[row][n]
__global__ void colsum_kernel(const float *__restrict__ dz, int rows, int n, float *__restrict__ db)
{
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= n) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += dz[(long long)r * n + col];
    db[col] = s;
}

__global__ void adam_kernel(float *w, float *m, float *v, const float *g, __nv_bfloat16 *wb, int count, float lr,
                            float b1, float b2, float eps, float wd, float c1, float c2)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) {
        const float gq = g[q];
        const float mq = b1 * m[q] + (1.f - b1) * gq;
        const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        const float wq = w[q] - lr * (mq / c1) / (sqrtf(vq / c2) + eps) - lr * wd * w[q];
        w[q] = wq;
        if (wb) wb[q] = __float2bfloat16_rn(wq);
    }
}

// one block per row: loss += scale w_r sum_c e^2, dy = 2 scale w_r e
__global__ void mse_kernel(const float *y, const float *t, const float *row_w, int cols, float scale, float *dy,
                           float *loss)
{
    __shared__ float part[256];
    const size_t base = (size_t)blockIdx.x * cols;
    const float w = row_w ? row_w[blockIdx.x] : 1.f;
    float s = 0.f;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) {
        const float e = y[base + c] - t[base + c];
        if (dy) dy[base + c] = 2.f * scale * w * e;
        s += e * e;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) atomicAdd(loss, scale * w * part[0]);
}

// one block per row: err_r = ||y_r - t_r|| / ||t_r||
__global__ void row_rel_err_kernel(const float *y, const float *t, int cols, float *err)
{
    __shared__ float pe[256], pt[256];
    const size_t base = (size_t)blockIdx.x * cols;
    float se = 0.f, st = 0.f;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) {
        const float e = y[base + c] - t[base + c];
        se += e * e;
        st += t[base + c] * t[base + c];
    }
    pe[threadIdx.x] = se;
    pt[threadIdx.x] = st;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            pe[threadIdx.x] += pe[threadIdx.x + h];
            pt[threadIdx.x] += pt[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) err[blockIdx.x] = pt[0] > 0.f ? sqrtf(pe[0] / pt[0]) : sqrtf(pe[0]);
}

__global__ void gather_rows_kernel(const float *src, const int *idx, int rows, int cols, float *dst)
{
    const long long total = (long long)rows * cols;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long r = q / cols;
        dst[q] = src[(long long)idx[r] * cols + (q - r * cols)];
    }
}

// block row r = blockIdx.y (grid-strided), columns across the x dimension
__global__ void scale_rows_kernel(float *y, const float *s, int rows, int cols)
{
    for (int r = blockIdx.y; r < rows; r += gridDim.y) {
        const float f = __ldg(s + r);
        float *yr = y + (size_t)r * cols;
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) yr[c] *= f;
    }
}

__global__ void to_bf16_kernel(const float *src, __nv_bfloat16 *dst, int count)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x)
        dst[q] = __float2bfloat16_rn(src[q]);
}

// ---- tcgen05 forward layer ---------------------------------------------------
constexpr int TC_M = 128, TC_N = 64, TC_KMAX = 256, TC_THREADS = 256;   // 8 warps: 4 lane groups x 2 column halves
// dynamic shared memory: alignment slack, a 1 KB header (barrier, TMEM
// slot), then the A and B tiles (up to K = TC_KMAX); the epilogue's
// transpose buffers (8 x 32 x TC_TS floats) reuse the start of the tile
// area.  About 98 KB: two CTAs per SM.
constexpr int TC_SMEM = 1024 + 1024 + (TC_M + TC_N) * TC_KMAX * 2;
constexpr unsigned long long TC_WAIT_NS = 1000000000ull;      // 1 s per wait

__device__ int g_mlp_err;     // a bounded wait ran out (read and cleared by fdtd_mlp_check)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
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

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    const unsigned long long t0 = gtimer();
    while (!mbar_try(bar, parity))
        if (gtimer() - t0 > TC_WAIT_NS) return false;
    return true;
}

// shared-memory matrix descriptor: start, leading (K-direction) and stride
// (8-row-group) byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B both BF16 and
// K-major, M = TC_M, N = TC_N
constexpr uint32_t TC_IDESC =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// eight consecutive elements (k .. k+7) of row r of a rows x K matrix as
// BF16, zero outside it; vec: 16-byte loads are valid (BF16, K % 8 == 0,
// 16-byte aligned base)
template <typename T>
__device__ __forceinline__ uint4 load8(const T *M, int rows, int K, int r, int k, bool vec)
{
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (r >= rows || k >= K) return v;
    if (sizeof(T) == 2 && vec) return __ldg(reinterpret_cast<const uint4 *>(M + (size_t)r * K + k));
    float f[8];
    for (int j = 0; j < 8; ++j) {
        const int kk = k + j;
        f[j] = kk < K ? (sizeof(T) == 2 ? __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(M + (size_t)r * K + kk))
                                        : (float)*reinterpret_cast<const float *>(M + (size_t)r * K + kk))
                      : 0.f;
    }
    v.x = pack2(f[0], f[1]);
    v.y = pack2(f[2], f[3]);
    v.z = pack2(f[4], f[5]);
    v.w = pack2(f[6], f[7]);
    return v;
}

constexpr int TC_TS = 36;    // floats per row of a warp's 32 x 32 transpose buffer (16-byte rows, no conflicts)
static_assert(TC_THREADS / 32 * 32 * TC_TS * 4 <= (TC_M + TC_N) * TC_KMAX * 2, "transpose buffers fit the tile area");

__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// lane l holds columns n .. n+31 of row mrow + l; write them to out (row
// pitch N) as 128-byte row segments: pass i stores rows 4i + l/8, lane
// l % 8 covering four columns
__device__ __forceinline__ void store_f32(float *T, const float (&x)[32], float *out, int mrow, int rows, int n,
                                          int N, int lane)
{
    for (int j = 0; j < 32; j += 4)
        *reinterpret_cast<float4 *>(T + lane * TC_TS + j) = make_float4(x[j], x[j + 1], x[j + 2], x[j + 3]);
    __syncwarp();
    const int cc = (lane & 7) * 4;
    const bool vec = (N & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    for (int i = 0; i < 8; ++i) {
        const int rr = i * 4 + (lane >> 3), m = mrow + rr;
        if (m >= rows) continue;
        const float4 q = *reinterpret_cast<const float4 *>(T + rr * TC_TS + cc);
        float *o = out + (size_t)m * N + n + cc;
        if (vec && n + cc + 3 < N) {
            *reinterpret_cast<float4 *>(o) = q;
        } else {
            const float e[4] = {q.x, q.y, q.z, q.w};
            for (int u = 0; u < 4; ++u)
                if (n + cc + u < N) o[u] = e[u];
        }
    }
    __syncwarp();
}

// as store_f32 for BF16 outputs: 64-byte row segments, pass i stores rows
// 8i + l/4, lane l % 4 covering eight columns
__device__ __forceinline__ void store_bf16(float *T, const float (&x)[32], __nv_bfloat16 *out, int mrow, int rows,
                                           int n, int N, int lane)
{
    uint32_t *Tu = reinterpret_cast<uint32_t *>(T);
    for (int j = 0; j < 32; j += 8)
        *reinterpret_cast<uint4 *>(Tu + lane * TC_TS + j / 2) =
            make_uint4(pack2(x[j], x[j + 1]), pack2(x[j + 2], x[j + 3]), pack2(x[j + 4], x[j + 5]),
                       pack2(x[j + 6], x[j + 7]));
    __syncwarp();
    const int cc = (lane & 3) * 8;
    const bool vec = (N & 7) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    for (int i = 0; i < 4; ++i) {
        const int rr = i * 8 + (lane >> 2), m = mrow + rr;
        if (m >= rows) continue;
        const uint4 q = *reinterpret_cast<const uint4 *>(Tu + rr * TC_TS + cc / 2);
        __nv_bfloat16 *o = out + (size_t)m * N + n + cc;
        if (vec && n + cc + 7 < N) {
            *reinterpret_cast<uint4 *>(o) = q;
        } else {
            const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&q);
            for (int u = 0; u < 8; ++u)
                if (n + cc + u < N) o[u] = e[u];
        }
    }
    __syncwarp();
}

template <typename T>
__device__ __forceinline__ void stage_operand(char *dst, const T *M, int rows, int K, int r0, int tile_rows, int kgs,
                                              uint32_t sbo, bool vec, int tid)
{
    for (int q = tid; q < tile_rows * kgs; q += TC_THREADS) {
        const int r = q / kgs, g = q - r * kgs;
        char *d = dst + (r >> 3) * sbo + g * 128 + (r & 7) * 16;
        if (sizeof(T) == 2 && vec) {
            const bool in = r0 + r < rows && g * 8 < K;   // K % 8 == 0: a chunk is wholly in or out
            const T *src = in ? M + (size_t)(r0 + r) * K + g * 8 : M;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(d)), "l"(src),
                         "r"(in ? 16 : 0)
                         : "memory");
        } else {
            *reinterpret_cast<uint4 *>(d) = load8(M, rows, K, r0 + r, g * 8, false);
        }
    }
}

template <typename TA>
__global__ void __launch_bounds__(TC_THREADS, 2)
    tc_forward_kernel(const TA *__restrict__ X, int rows, int K, int Kp, bool xvec, const __nv_bfloat16 *__restrict__ Wt,
                      bool wvec, const float *__restrict__ bias, int N, int act, __nv_bfloat16 *yb, float *yf,
                      float *zf)
{
    extern __shared__ __align__(1024) char smraw[];
    char *sm = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + 8);
    char *As = sm + 1024;
    char *Bs = As + TC_M * Kp * 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_M, n0 = blockIdx.y * TC_N;
    const int kgs = Kp / 8;
    const uint32_t sbo = (uint32_t)Kp * 16;   // bytes between 8-row groups; k groups are 128 B apart
    // both operands into the core-matrix layout: chunk (row r, k group g)
    // = 8 elements of one row, 16 bytes at (r / 8) sbo + g 128 + (r % 8) 16.
    // BF16 rows that allow it are copied with asynchronous 16-byte copies,
    // all of a thread's in flight at once (zero-filled outside the matrix);
    // others are converted through registers.
    stage_operand(As, X, rows, K, m0, TC_M, kgs, sbo, xvec, tid);
    stage_operand(Bs, Wt, N, K, n0, TC_N, kgs, sbo, wvec, tid);
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
        for (int k0 = 0; k0 < Kp; k0 += 16) {
            const uint64_t ad = smem_desc(a0 + k0 * 16, 128, sbo), bd = smem_desc(b0 + k0 * 16, 128, sbo);
            const uint32_t acc = k0 > 0 ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(acc)
                : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                     : "memory");
    }
    bool ok = mbar_wait_bounded(smem_u32(bar), 0);
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (tid == 0) atomicExch(&g_mlp_err, 1);
        mbar_wait_bounded(smem_u32(bar), 0);   // the chain still in flight, bounded again
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (its 32 rows)
        // and accumulator columns 32 (w / 4) .. +31; bias and activation in
        // registers, then each output is transposed through the warp's
        // shared buffer in the (now idle) operand area and stored as whole
        // row segments
        const int lg = warp & 3, c = (warp >> 2) * 32;
        float *T = reinterpret_cast<float *>(As) + warp * 32 * TC_TS;
        const int mrow = m0 + lg * 32;
        if (n0 + c < N) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)c, v);
            float z[32], y[32];
            for (int j = 0; j < 32; ++j) {
                const int n = n0 + c + j;
                z[j] = __uint_as_float(v[j]) + ((bias && n < N) ? __ldg(bias + n) : 0.f);
                y[j] = act == FDTD_ACT_GELU ? gelu(z[j]) : z[j];
            }
            if (zf) store_f32(T, z, zf, mrow, rows, n0 + c, N, lane);
            if (yf) store_f32(T, y, yf, mrow, rows, n0 + c, N, lane);
            if (yb) store_bf16(T, y, yb, mrow, rows, n0 + c, N, lane);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N) : "memory");
    }
}

// ---- tcgen05 gradient GEMM ---------------------------------------------------
// C[M x N] (FP32, row pitch N) = sum_k A(m, k) B(k, n) with
// A(m, k) = A[m sam + k sak] and B(k, n) = B[k sbk + n sbn], FP32 or BF16
// operands with any element strides (the gradients dz^T x and dz wt read
// their operands transposed).  One CTA per 128 x 64 output tile; the
// reduction runs in chunks of GC_K: all threads stage a chunk of both
// operands into the K-major core-matrix layout (rounded to BF16 in
// registers; threads walk the operand's contiguous index so the loads
// coalesce), one thread issues its MMA chain into the TMEM accumulator and
// commits it to an mbarrier, and every thread waits (bounded) before the
// next chunk overwrites the tiles.  The epilogue is the forward layer's.
constexpr int GC_K = 128;
constexpr int GC_SMEM = 1024 + 1024 + (TC_M + TC_N) * GC_K * 2;

template <typename T>
__device__ __forceinline__ float elem(const T *p)
{
    if constexpr (sizeof(T) == 2) return __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(p));
    else return *reinterpret_cast<const float *>(p);
}

// rows r0 .. r0 + R - 1 (row index fast in memory when s_row == 1) and
// reduction indices k0 .. k0 + GC_K - 1 of X(row, k) = X[row s_row + k s_k]
// (zero outside rows x K) into the core-matrix layout of a GC_K chunk:
// 8 elements of one row at (r / 8) (GC_K 16) + (k / 8) 128 + (r % 8) 16
template <typename T>
__device__ __forceinline__ void stage_strided(char *dst, const T *X, long long s_row, long long s_k, int rows,
                                              int K, int r0, int R, int k0, int tid)
{
    constexpr int kgs = GC_K / 8;
    for (int q = tid; q < R * kgs; q += TC_THREADS) {
        int r, g;
        if (s_row == 1) { r = q % R; g = q / R; }
        else { r = q / kgs; g = q % kgs; }
        const int row = r0 + r, k = k0 + g * 8;
        float f[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            f[j] = (row < rows && k + j < K) ? elem(X + row * s_row + (long long)(k + j) * s_k) : 0.f;
        *reinterpret_cast<uint4 *>(dst + (r >> 3) * (GC_K * 16) + g * 128 + (r & 7) * 16) =
            make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
    }
}

template <typename TA, typename TB>
__global__ void __launch_bounds__(TC_THREADS, 2)
    tc_grad_kernel(const TA *__restrict__ A, long long sam, long long sak, const TB *__restrict__ B, long long sbk,
                   long long sbn, int M, int N, int K, Epi ep)
{
    extern __shared__ __align__(1024) char smraw[];
    char *sm = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + 8);
    char *As = sm + 1024;
    char *Bs = As + TC_M * GC_K * 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_M, n0 = blockIdx.y * TC_N;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t sbo = GC_K * 16;
    bool ok = true;
    const int nchunk = (K + GC_K - 1) / GC_K;
    for (int c = 0; c < nchunk && ok; ++c) {
        const int k0 = c * GC_K;
        // A rows are m, B rows are n (B(k, n) read as row n of B^T)
        stage_strided(As, A, sam, sak, M, K, m0, TC_M, k0, tid);
        stage_strided(Bs, B, sbn, sbk, N, K, n0, TC_N, k0, tid);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
            for (int kk = 0; kk < GC_K; kk += 16) {
                const uint64_t ad = smem_desc(a0 + kk * 16, 128, sbo), bd = smem_desc(b0 + kk * 16, 128, sbo);
                const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(bar))
                         : "memory");
        }
        // the tiles are free again (and, after the last chunk, the accumulator complete)
        bool done = mbar_wait_bounded(smem_u32(bar), (uint32_t)(c & 1));
        ok = __syncthreads_and(done);
        if (!ok) {
            if (tid == 0) atomicExch(&g_mlp_err, 1);
            mbar_wait_bounded(smem_u32(bar), (uint32_t)(c & 1));   // the chain still in flight, bounded again
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (ok) {
        const int lg = warp & 3, cc = (warp >> 2) * 32;
        float *T = reinterpret_cast<float *>(As) + warp * 32 * TC_TS;
        const int mrow = m0 + lg * 32;
        if (n0 + cc < N) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)cc, v);
            if (ep.mode == 1) {
                float y[32];
                for (int j = 0; j < 32; ++j) y[j] = __uint_as_float(v[j]);
                store_f32(T, y, ep.yf, mrow, M, n0 + cc, N, lane);
            } else {
                float z[32], y[32];
                for (int j = 0; j < 32; ++j) {
                    const int n = n0 + cc + j;
                    z[j] = __uint_as_float(v[j]) + ((ep.bias && n < N) ? __ldg(ep.bias + n) : 0.f);
                    y[j] = ep.act == FDTD_ACT_GELU ? gelu(z[j]) : z[j];
                }
                if (ep.zf) store_f32(T, z, ep.zf, mrow, M, n0 + cc, N, lane);
                if (ep.yf) store_f32(T, y, ep.yf, mrow, M, n0 + cc, N, lane);
                if (ep.yb) store_bf16(T, y, ep.yb, mrow, M, n0 + cc, N, lane);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N) : "memory");
    }
}

static_assert(TC_THREADS / 32 * 32 * TC_TS * 4 <= (TC_M + TC_N) * GC_K * 2, "transpose buffers fit the tile area");

template <typename TA, typename TB>
cudaError_t tc_grad(const TA *A, long long sam, long long sak, const TB *B, long long sbk, long long sbn, int M, int N,
                    int K, const Epi &ep, cudaStream_t s)
{
    static std::mutex mu;
    static bool ready[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!ready[dev]) {
            e = cudaFuncSetAttribute(tc_grad_kernel<TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, GC_SMEM);
            if (e != cudaSuccess) return e;
            ready[dev] = true;
        }
    }
    dim3 grid((M + TC_M - 1) / TC_M, (N + TC_N - 1) / TC_N);
    tc_grad_kernel<TA, TB><<<grid, TC_THREADS, GC_SMEM, s>>>(A, sam, sak, B, sbk, sbn, M, N, K, ep);
    return cudaGetLastError();
}

template <typename TA>
cudaError_t tc_forward(const TA *x, int rows, int K, const __nv_bfloat16 *wt, const float *bias, int N, int act,
                       __nv_bfloat16 *yb, float *yf, float *zf, cudaStream_t s)
{
    static std::mutex mu;
    static bool ready[2][64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(mu);
        bool &r = ready[sizeof(TA) == 2][dev];
        if (!r) {
            e = cudaFuncSetAttribute(tc_forward_kernel<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
            if (e != cudaSuccess) return e;
            r = true;
        }
    }
    const int Kp = (K + 15) / 16 * 16;
    const bool xvec = sizeof(TA) == 2 && K % 8 == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0;
    const bool wvec = K % 8 == 0 && (reinterpret_cast<uintptr_t>(wt) & 15) == 0;
    dim3 grid((rows + TC_M - 1) / TC_M, (N + TC_N - 1) / TC_N);
    tc_forward_kernel<TA><<<grid, TC_THREADS, TC_SMEM, s>>>(x, rows, K, Kp, xvec, wt, wvec, bias, N, act, yb, yf, zf);
    return cudaGetLastError();
}

// ---- whole network in one launch: a cluster of four CTAs per 128 rows ------
// Each CTA of a cluster owns a quarter of every layer's outputs (ns columns,
// a multiple of 16) and keeps its slices of all weight matrices resident in
// shared memory (one bulk copy per layer from a packed image, issued at
// launch).  Per layer one thread issues the MMA chain (A = the cluster's
// shared activations of the 128 rows, B = the CTA's weight slice, D = TMEM),
// the sixteen warps read the accumulator back (bias, activation, BF16) and
// store their columns, in the next layer's K-major core-matrix layout,
// into the activation buffer of every CTA of the cluster (distributed
// shared memory); two cluster barriers per layer separate the MMAs that
// read a buffer from the stores that overwrite it.  The last layer writes
// FP32 rows to global memory.  The arithmetic of each output element is the
// per-layer kernel's (same BF16 roundings, same K = 16 MMA steps, bias then
// activation in FP32), so the two paths agree bit for bit.
constexpr int NF_MAX_LAYERS = 6;
constexpr int NF_CLUSTER = 4;
constexpr int NF_WARPS = 16;                         // 4 TMEM lane groups x 4 column quarters
constexpr int NF_THREADS = NF_WARPS * 32;
constexpr int NF_SMEM_MAX = 227 * 1024;

struct NetArgs {
    int n_layers;
    int k[NF_MAX_LAYERS + 1];      // sizes: k[0] inputs, k[l + 1] outputs of layer l
    int kp[NF_MAX_LAYERS + 1];     // sizes rounded up to 16 (the K extent of the layer they feed)
    int ns[NF_MAX_LAYERS];         // output columns of layer l per cluster rank (multiple of 16)
    long long woff[NF_MAX_LAYERS]; // byte offset of layer l's rank-0 slice in the packed image
    int wsm[NF_MAX_LAYERS];        // byte offset of layer l's slice in shared memory
    int act[NF_MAX_LAYERS];
    const float *bias[NF_MAX_LAYERS];
    const char *image;
    int boff[NF_MAX_LAYERS];       // first float of layer l's bias slice in the staged biases
    int bias_bytes;                // staged biases of this rank's columns, all layers
    int act_bytes;                 // activation buffer: 128 rows x the largest K, BF16
    int tmem_cols;
    float out_scale;
};

// byte offset of element (n, k) of a rows x kp matrix in the K-major
// core-matrix layout: 8 x 8 blocks of 128 bytes, k blocks adjacent
__host__ __device__ __forceinline__ long long core_off(int n, int k, int kp)
{
    return (long long)(n >> 3) * (kp * 16) + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
}

// the image: per layer, per rank, the rank's ns x kp slice of wt (zero
// outside n x k) in the core-matrix layout
__global__ void net_pack_kernel(const __nv_bfloat16 *__restrict__ wt, int n, int k, int ns, int kp, char *dst)
{
    const long long per = (long long)ns * kp, total = per * NF_CLUSTER;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(q / per);
        const int nl = (int)((q - r * per) / kp), kk = (int)(q - r * per - (long long)nl * kp);
        const int ng = r * ns + nl;
        const __nv_bfloat16 v = (ng < n && kk < k) ? wt[(long long)ng * k + kk] : __float2bfloat16_rn(0.f);
        *reinterpret_cast<__nv_bfloat16 *>(dst + r * per * 2 + core_off(nl, kk, kp)) = v;
    }
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t addr, uint32_t (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(NF_THREADS, 1)
    net_forward_kernel(const float *__restrict__ x, int rows, const __grid_constant__ NetArgs P, float *__restrict__ y)
{
    extern __shared__ __align__(1024) char smraw[];
    char *sm = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
    uint64_t *wbar = reinterpret_cast<uint64_t *>(sm);        // weight slices landed
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + 8);    // a layer's MMA chain done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + 16);
    float *bsm = reinterpret_cast<float *>(sm + 1024);
    char *act = sm + 1024 + P.bias_bytes;
    char *wsm = act + P.act_bytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t rank = cluster_rank();
    const int m0 = (blockIdx.x / NF_CLUSTER) * TC_M;
    const int L = P.n_layers;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(P.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(wbar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 32) {
        // this CTA's weight slices, one bulk copy per layer
        uint32_t bytes = 0;
        for (int l = 0; l < L; ++l) bytes += (uint32_t)P.ns[l] * P.kp[l] * 2;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(wbar)), "r"(bytes)
                     : "memory");
        for (int l = 0; l < L; ++l) {
            const uint32_t sz = (uint32_t)P.ns[l] * P.kp[l] * 2;
            const char *src = P.image + P.woff[l] + (long long)rank * sz;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(wsm + P.wsm[l])),
                "l"(src), "r"(sz), "r"(smem_u32(wbar))
                : "memory");
        }
    }
    // this rank's bias columns of every layer (zero past the layer's outputs)
    for (int l = 0; l < L; ++l)
        for (int c = tid; c < P.ns[l]; c += NF_THREADS) {
            const int n = (int)rank * P.ns[l] + c;
            bsm[P.boff[l] + c] = (P.bias[l] && n < P.k[l + 1]) ? __ldg(P.bias[l] + n) : 0.f;
        }
    // the 128 input rows, rounded to BF16, as layer 0's A operand (every CTA
    // of the cluster stages its own copy)
    {
        const int kgs = P.kp[0] / 8;
        for (int q = tid; q < TC_M * kgs; q += NF_THREADS) {
            const int r = q / kgs, g = q - r * kgs;
            *reinterpret_cast<uint4 *>(act + core_off(r, g * 8, P.kp[0])) = load8(x, rows, P.k[0], m0 + r, g * 8, false);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    cluster_sync();                 // every CTA of the cluster runs (its shared memory may be written)
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    bool ok = true;
    if (tid == 0) ok = mbar_wait_bounded(smem_u32(wbar), 0);
    ok = __syncthreads_and(ok);
    const bool loaded = ok;
    int fail = -1;                  // layer whose MMA chain a wait gave up on
    if (!ok && tid == 0) atomicExch(&g_mlp_err, 1);
    // warp: TMEM lane group lg (its 32 tile rows) and column chunks of 8
    // starting at 8 quarter, every fourth chunk
    const int lg = warp & 3, quarter = warp >> 2, r = lg * 32 + lane;
    uint32_t dst[NF_CLUSTER];       // the activation buffer in each CTA of the cluster
    for (int c = 0; c < NF_CLUSTER; ++c)
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(dst[c]) : "r"(smem_u32(act)), "r"(c));
    for (int l = 0; l < L; ++l) {
        const int ns = P.ns[l], kp = P.kp[l], N = P.k[l + 1];
        const bool last = l == L - 1;
        if (ok && tid == 0) {
            const uint32_t idesc =
                (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(ns >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
            const uint32_t a0 = smem_u32(act), b0 = smem_u32(wsm + P.wsm[l]), sbo = (uint32_t)kp * 16;
            // the activations stored through the generic proxy (this CTA's
            // or, across the cluster barrier, the other CTAs') are read by
            // the tensor cores' asynchronous proxy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int k0 = 0; k0 < kp; k0 += 16) {
                const uint64_t ad = smem_desc(a0 + k0 * 16, 128, sbo), bd = smem_desc(b0 + k0 * 16, 128, sbo);
                const uint32_t acc = k0 > 0 ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(mbar))
                         : "memory");
        }
        bool done = !ok || mbar_wait_bounded(smem_u32(mbar), (uint32_t)(l & 1));
        done = __syncthreads_and(done);
        if (ok && !done) {
            ok = false;
            fail = l;
            if (tid == 0) atomicExch(&g_mlp_err, 1);
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int n0 = (int)rank * ns;
        const float *bl = bsm + P.boff[l];
        if (!last) {
            cluster_sync();         // every CTA's MMAs of this layer have read its activation buffer
            const int kpn = P.kp[l + 1];
            for (int c = quarter * 8; ok && c < ns; c += 32) {
                const int nb = n0 + c;          // first of the 8 columns (a multiple of 8)
                if (nb >= kpn) break;
                uint32_t v[8];
                tmem_ld8(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)c, v);
                float f[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float z = __uint_as_float(v[j]) + bl[c + j];
                    f[j] = P.act[l] == FDTD_ACT_GELU ? gelu(z) : z;
                }
                const uint4 q = make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
                const uint32_t off = (uint32_t)core_off(r, nb, kpn);
                for (int t = 0; t < NF_CLUSTER; ++t)
                    asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(dst[t] + off), "r"(q.x),
                                 "r"(q.y), "r"(q.z), "r"(q.w)
                                 : "memory");
            }
            asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            cluster_sync();         // the next layer's A operand is complete in every CTA
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        } else if (ok) {
            const int m = m0 + r;
            for (int c = quarter * 8; c < ns; c += 32) {
                const int nb = n0 + c;
                if (nb >= N) break;
                uint32_t v[8];
                tmem_ld8(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)c, v);
                if (m >= rows) continue;
                float f[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float z = __uint_as_float(v[j]) + bl[c + j];
                    f[j] = (P.act[l] == FDTD_ACT_GELU ? gelu(z) : z) * P.out_scale;
                }
                float *o = y + (long long)m * N + nb;
                if (nb + 8 <= N && (N & 3) == 0 && (reinterpret_cast<uintptr_t>(y) & 15) == 0) {
                    reinterpret_cast<float4 *>(o)[0] = make_float4(f[0], f[1], f[2], f[3]);
                    reinterpret_cast<float4 *>(o)[1] = make_float4(f[4], f[5], f[6], f[7]);
                } else {
                    for (int j = 0; j < 8 && nb + j < N; ++j) o[j] = f[j];
                }
            }
        }
    }
    // copies or an MMA chain still in flight after a wait gave up: wait
    // (bounded) before the shared memory and TMEM are given back
    if (tid == 0 && !loaded) mbar_wait_bounded(smem_u32(wbar), 0);
    if (tid == 0 && fail >= 0) mbar_wait_bounded(smem_u32(mbar), (uint32_t)(fail & 1));
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P.tmem_cols) : "memory");
    }
    cluster_sync();                 // no CTA leaves while another may still address its shared memory
}

// layout of a network's packed image and of the kernel's shared memory;
// false when the sizes are outside what the kernel supports
bool net_layout(const int *sizes, int L, NetArgs &P, size_t &image_bytes, int &smem)
{
    if (!sizes || L < 1 || L > NF_MAX_LAYERS) return false;
    P = NetArgs{};
    P.n_layers = L;
    int kmax = 0, nsmax = 0, nbias = 0;
    long long off = 0;
    int wbytes = 0;
    for (int l = 0; l <= L; ++l) {
        if (sizes[l] < 1) return false;
        P.k[l] = sizes[l];
        P.kp[l] = (sizes[l] + 15) / 16 * 16;
    }
    for (int l = 0; l < L; ++l) {
        if (P.k[l] > TC_KMAX) return false;                 // every layer's K fits the activation buffer
        const int q = (P.k[l + 1] + NF_CLUSTER - 1) / NF_CLUSTER;
        P.ns[l] = (q + 15) / 16 * 16;
        if (P.ns[l] > 256) return false;                    // one MMA N extent
        P.woff[l] = off;
        P.wsm[l] = wbytes;
        P.boff[l] = nbias;
        nbias += P.ns[l];
        off += (long long)NF_CLUSTER * P.ns[l] * P.kp[l] * 2;
        wbytes += P.ns[l] * P.kp[l] * 2;
        kmax = std::max(kmax, P.kp[l]);
        nsmax = std::max(nsmax, P.ns[l]);
    }
    P.act_bytes = TC_M * kmax * 2;
    P.bias_bytes = (nbias * 4 + 1023) / 1024 * 1024;
    P.tmem_cols = 32;
    while (P.tmem_cols < nsmax) P.tmem_cols *= 2;
    image_bytes = (size_t)off;
    smem = 1024 + 1024 + P.bias_bytes + P.act_bytes + wbytes;
    return smem <= NF_SMEM_MAX;
}

int rc(cudaError_t e) { return e == cudaSuccess ? FDTD_OK : FDTD_ECUDA; }
int grid1d(long long n) { return (int)std::min<long long>((n + 255) / 256, 4096); }

}  // namespace

extern "C" {

int fdtd_mlp_forward(const void *x, int x_is_bf16, int rows, int k, const void *wt, const float *bias, int n,
                     int act, void *y_bf16, float *y_f32, float *z_f32, void *cuda_stream)
{
    if (!x || !wt || rows < 0 || k < 1 || n < 1 || (act != FDTD_ACT_NONE && act != FDTD_ACT_GELU)) return FDTD_EINVAL;
    if (rows == 0) return FDTD_OK;
    Epi ep{0, bias, act, static_cast<__nv_bfloat16 *>(y_bf16), y_f32, z_f32, n};
    const auto *w = static_cast<const __nv_bfloat16 *>(wt);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (k <= TC_KMAX) {       // tensor-core path (every layer of the surrogate networks)
        if (x_is_bf16)
            return rc(tc_forward(static_cast<const __nv_bfloat16 *>(x), rows, k, w, bias, n, act,
                                 static_cast<__nv_bfloat16 *>(y_bf16), y_f32, z_f32, s));
        return rc(tc_forward(static_cast<const float *>(x), rows, k, w, bias, n, act,
                             static_cast<__nv_bfloat16 *>(y_bf16), y_f32, z_f32, s));
    }
    // larger k: the chunked tensor-core GEMM, B(k, n) = wt[n * k + k']
    if (x_is_bf16)
        return rc(tc_grad(static_cast<const __nv_bfloat16 *>(x), k, 1, w, 1, k, rows, n, k, ep, s));
    return rc(tc_grad(static_cast<const float *>(x), k, 1, w, 1, k, rows, n, k, ep, s));
}

int fdtd_mlp_net_pack_bytes(const int *sizes, int n_layers, size_t *bytes)
{
    NetArgs P;
    size_t b = 0;
    int smem = 0;
    if (!bytes || !net_layout(sizes, n_layers, P, b, smem)) return FDTD_EINVAL;
    *bytes = b;
    return FDTD_OK;
}

int fdtd_mlp_net_pack(const int *sizes, int n_layers, const void *const *wt, void *image, void *cuda_stream)
{
    NetArgs P;
    size_t b = 0;
    int smem = 0;
    if (!wt || !image || (reinterpret_cast<uintptr_t>(image) & 15) || !net_layout(sizes, n_layers, P, b, smem))
        return FDTD_EINVAL;
    for (int l = 0; l < n_layers; ++l)
        if (!wt[l]) return FDTD_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    for (int l = 0; l < n_layers; ++l) {
        const long long total = (long long)NF_CLUSTER * P.ns[l] * P.kp[l];
        net_pack_kernel<<<grid1d(total), 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(wt[l]), P.k[l + 1], P.k[l],
                                                      P.ns[l], P.kp[l], static_cast<char *>(image) + P.woff[l]);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return FDTD_ECUDA;
    }
    return FDTD_OK;
}

int fdtd_mlp_net_forward(const float *x, int rows, const int *sizes, int n_layers, const int *acts,
                         const void *image, const float *const *bias, float out_scale, float *y, void *cuda_stream)
{
    NetArgs P;
    size_t b = 0;
    int smem = 0;
    if (!x || !y || !image || !acts || rows < 0 || (reinterpret_cast<uintptr_t>(image) & 15) ||
        !net_layout(sizes, n_layers, P, b, smem))
        return FDTD_EINVAL;
    for (int l = 0; l < n_layers; ++l) {
        if (acts[l] != FDTD_ACT_NONE && acts[l] != FDTD_ACT_GELU) return FDTD_EINVAL;
        P.act[l] = acts[l];
        P.bias[l] = bias ? bias[l] : nullptr;
    }
    if (rows == 0) return FDTD_OK;
    P.image = static_cast<const char *>(image);
    P.out_scale = out_scale;
    static std::mutex mu;
    static int ready_smem[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev >= 64) return FDTD_ECUDA;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (ready_smem[dev] < smem) {
            e = cudaFuncSetAttribute(net_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, NF_SMEM_MAX);
            if (e != cudaSuccess) return FDTD_ECUDA;
            ready_smem[dev] = NF_SMEM_MAX;
        }
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(((rows + TC_M - 1) / TC_M) * NF_CLUSTER));
    cfg.blockDim = dim3(NF_THREADS);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = (cudaStream_t)cuda_stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = NF_CLUSTER;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return rc(cudaLaunchKernelEx(&cfg, net_forward_kernel, x, rows, P, y));
}

int fdtd_mlp_check(void *cuda_stream)
{
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return FDTD_ECUDA;
    int flag = 0;
    e = cudaMemcpyFromSymbol(&flag, g_mlp_err, sizeof flag);
    if (e != cudaSuccess) return FDTD_ECUDA;
    if (flag) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_mlp_err, &zero, sizeof zero);
        return e == cudaSuccess ? FDTD_ETIMEOUT : FDTD_ECUDA;
    }
    return FDTD_OK;
}

int fdtd_mlp_backward(const void *x, int x_is_bf16, const float *z, const float *dy, int rows, int k, int n,
                      int act, const void *wt, float *dz, float *dw, float *db, float *dx, void *cuda_stream)
{
    if (!dy || !dz || rows < 0 || k < 1 || n < 1 || (act == FDTD_ACT_GELU && !z)) return FDTD_EINVAL;
    if ((dw && !x) || (dx && !wt)) return FDTD_EINVAL;
    if (rows == 0) return FDTD_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const long long cnt = (long long)rows * n;
    act_grad_kernel<<<grid1d(cnt), 256, 0, s>>>(dy, z, dz, cnt, act);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && db) {
        colsum_kernel<<<(n + 127) / 128, 128, 0, s>>>(dz, rows, n, db);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && dw) {
        // dw[n x k] = dz^T x: A(m=o, kk=r) = dz[r * n + o]; B(kk=r, c) = x[r * k + c]
        Epi ep{1, nullptr, 0, nullptr, dw, nullptr, k};
        if (x_is_bf16)
            e = tc_grad(dz, 1, n, static_cast<const __nv_bfloat16 *>(x), k, 1, n, k, rows, ep, s);
        else
            e = tc_grad(dz, 1, n, static_cast<const float *>(x), k, 1, n, k, rows, ep, s);
    }
    if (e == cudaSuccess && dx) {
        // dx[rows x k] = dz wt: A(r, o) = dz[r * n + o]; B(o, c) = wt[o * k + c]
        Epi ep{1, nullptr, 0, nullptr, dx, nullptr, k};
        e = tc_grad(dz, n, 1, static_cast<const __nv_bfloat16 *>(wt), k, 1, rows, k, n, ep, s);
    }
    return rc(e);
}

int fdtd_mlp_adam(float *w, float *m, float *v, const float *g, void *w_bf16, int count, float lr, float beta1,
                  float beta2, float eps, float weight_decay, int t, void *cuda_stream)
{
    if (!w || !m || !v || !g || count < 0 || t < 1) return FDTD_EINVAL;
    if (count == 0) return FDTD_OK;
    const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
    adam_kernel<<<grid1d(count), 256, 0, (cudaStream_t)cuda_stream>>>(
        w, m, v, g, static_cast<__nv_bfloat16 *>(w_bf16), count, lr, beta1, beta2, eps, weight_decay, c1, c2);
    return rc(cudaGetLastError());
}

int fdtd_mlp_mse(const float *y, const float *target, const float *row_weight, int rows, int cols, float scale,
                 float *dy, float *loss, void *cuda_stream)
{
    if (!y || !target || rows < 0 || cols < 0) return FDTD_EINVAL;
    if (rows == 0 || cols == 0) return FDTD_OK;
    mse_kernel<<<rows, 256, 0, (cudaStream_t)cuda_stream>>>(y, target, row_weight, cols, scale, dy, loss);
    return rc(cudaGetLastError());
}

int fdtd_mlp_row_rel_err(const float *y, const float *target, int rows, int cols, float *err, void *cuda_stream)
{
    if (!y || !target || !err || rows < 0 || cols < 0) return FDTD_EINVAL;
    if (rows == 0) return FDTD_OK;
    row_rel_err_kernel<<<rows, 256, 0, (cudaStream_t)cuda_stream>>>(y, target, cols, err);
    return rc(cudaGetLastError());
}

int fdtd_mlp_gather_rows(const float *src, const int *idx, int rows, int cols, float *dst, void *cuda_stream)
{
    if (!src || !idx || !dst || rows < 0 || cols < 0) return FDTD_EINVAL;
    if ((long long)rows * cols == 0) return FDTD_OK;
    gather_rows_kernel<<<grid1d((long long)rows * cols), 256, 0, (cudaStream_t)cuda_stream>>>(src, idx, rows, cols,
                                                                                            dst);
    return rc(cudaGetLastError());
}

int fdtd_mlp_scale_rows(float *y, const float *scale, int rows, int cols, void *cuda_stream)
{
    if (!y || !scale || rows < 0 || cols < 0) return FDTD_EINVAL;
    if ((long long)rows * cols == 0) return FDTD_OK;
    const dim3 grid((unsigned)std::min((cols + 255) / 256, 64), (unsigned)std::min(rows, 65535));
    scale_rows_kernel<<<grid, 256, 0, (cudaStream_t)cuda_stream>>>(y, scale, rows, cols);
    return rc(cudaGetLastError());
}

int fdtd_mlp_to_bf16(const float *src, void *dst, int count, void *cuda_stream)
{
    if (!src || !dst || count < 0) return FDTD_EINVAL;
    if (count == 0) return FDTD_OK;
    to_bf16_kernel<<<grid1d(count), 256, 0, (cudaStream_t)cuda_stream>>>(src, static_cast<__nv_bfloat16 *>(dst),
                                                                         count);
    return rc(cudaGetLastError());
}

}  // extern "C"
