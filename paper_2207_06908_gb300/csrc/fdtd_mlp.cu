// fdtd_mlp.cu -- surrogate-network kernels (BF16 operands, FP32 accumulate).
//
// One tiled GEMM serves the forward layer (x wt^T), the input gradient
// (dz wt) and the weight gradient (dz^T x): operands are addressed through
// element strides, staged into shared memory as BF16 with k contiguous, and
// multiplied with mma.sync m16n8k16 (BF16 x BF16 -> FP32).  The forward
// epilogue adds the bias and applies GELU (erf form, CUDA's erff).  Small
// element-wise kernels form dz = dy * act'(z), the bias gradient, the MSE
// loss and the Adam update.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "fdtd.h"
#include "fdtd_mlp.h"

namespace {

constexpr int BM = 64, BN = 64, BK = 32, PAD = 8;
constexpr int GT = 128;                       // 4 warps, 2 x 2, each 32 x 32

template <typename T>
__device__ __forceinline__ __nv_bfloat16 to_bf16(T v);
template <>
__device__ __forceinline__ __nv_bfloat16 to_bf16<__nv_bfloat16>(__nv_bfloat16 v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_bf16<float>(float v) { return __float2bfloat16_rn(v); }

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

// C[M x N] = A[M x K] B[K x N] with A(m,k) = A[m*sam + k*sak],
// B(k,n) = B[k*sbk + n*sbn]
template <typename TA, typename TB>
__global__ void __launch_bounds__(GT) gemm_kernel(const TA *__restrict__ A, long long sam, long long sak,
                                                  const TB *__restrict__ B, long long sbk, long long sbn, int M,
                                                  int N, int K, Epi ep)
{
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PAD];   // n-major: k contiguous
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 4; ++b)
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    const bool a_kfast = (sak == 1), b_kfast = (sbk == 1);
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int q = tid; q < BM * BK; q += GT) {
            int i, j;
            if (a_kfast) { i = q / BK; j = q % BK; }
            else { j = q / BM; i = q % BM; }
            const int m = m0 + i, k = k0 + j;
            As[i][j] = (m < M && k < K) ? to_bf16(A[m * sam + k * sak]) : __float2bfloat16_rn(0.f);
        }
        for (int q = tid; q < BN * BK; q += GT) {
            int jj, j;
            if (b_kfast) { jj = q / BK; j = q % BK; }
            else { j = q / BN; jj = q % BN; }
            const int n = n0 + jj, k = k0 + j;
            Bs[jj][j] = (n < N && k < K) ? to_bf16(B[k * sbk + n * sbn]) : __float2bfloat16_rn(0.f);
        }
        __syncthreads();
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
            for (int mi = 0; mi < 2; ++mi) {
                const int r = wm + mi * 16 + g, c = kk + 2 * t;
                af[mi][0] = *reinterpret_cast<const uint32_t *>(&As[r][c]);
                af[mi][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][c]);
                af[mi][2] = *reinterpret_cast<const uint32_t *>(&As[r][c + 8]);
                af[mi][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][c + 8]);
            }
            for (int ni = 0; ni < 4; ++ni) {
                const int n = wn + ni * 8 + g, c = kk + 2 * t;
                bf[ni][0] = *reinterpret_cast<const uint32_t *>(&Bs[n][c]);
                bf[ni][1] = *reinterpret_cast<const uint32_t *>(&Bs[n][c + 8]);
            }
            for (int mi = 0; mi < 2; ++mi)
                for (int ni = 0; ni < 4; ++ni)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(acc[mi][ni][0]), "+f"(acc[mi][ni][1]), "+f"(acc[mi][ni][2]), "+f"(acc[mi][ni][3])
                        : "r"(af[mi][0]), "r"(af[mi][1]), "r"(af[mi][2]), "r"(af[mi][3]), "r"(bf[ni][0]),
                          "r"(bf[ni][1]));
        }
        __syncthreads();
    }
    for (int mi = 0; mi < 2; ++mi)
        for (int ni = 0; ni < 4; ++ni)
            for (int h = 0; h < 2; ++h)
                for (int e = 0; e < 2; ++e) {
                    const int m = m0 + wm + mi * 16 + g + 8 * h;
                    const int n = n0 + wn + ni * 8 + 2 * t + e;
                    if (m >= M || n >= N) continue;
                    const float v = acc[mi][ni][2 * h + e];
                    const long long o = (long long)m * ep.ldc + n;
                    if (ep.mode == 1) {
                        ep.yf[o] = v;
                    } else {
                        const float z = v + (ep.bias ? ep.bias[n] : 0.f);
                        const float y = ep.act == FDTD_ACT_GELU ? gelu(z) : z;
                        if (ep.zf) ep.zf[o] = z;
                        if (ep.yf) ep.yf[o] = y;
                        if (ep.yb) ep.yb[o] = __float2bfloat16_rn(y);
                    }
                }
}

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

__global__ void scale_rows_kernel(float *y, const float *s, int rows, int cols)
{
    const long long total = (long long)rows * cols;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x)
        y[q] *= s[q / cols];
}

__global__ void to_bf16_kernel(const float *src, __nv_bfloat16 *dst, int count)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x)
        dst[q] = __float2bfloat16_rn(src[q]);
}

template <typename TA, typename TB>
cudaError_t gemm(const TA *A, long long sam, long long sak, const TB *B, long long sbk, long long sbn, int M, int N,
                 int K, const Epi &ep, cudaStream_t s)
{
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    gemm_kernel<TA, TB><<<grid, GT, 0, s>>>(A, sam, sak, B, sbk, sbn, M, N, K, ep);
    return cudaGetLastError();
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
    // B(k, n) = wt[n * k + k']
    if (x_is_bf16)
        return rc(gemm(static_cast<const __nv_bfloat16 *>(x), k, 1, w, 1, k, rows, n, k, ep, s));
    return rc(gemm(static_cast<const float *>(x), k, 1, w, 1, k, rows, n, k, ep, s));
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
            e = gemm(dz, 1, n, static_cast<const __nv_bfloat16 *>(x), k, 1, n, k, rows, ep, s);
        else
            e = gemm(dz, 1, n, static_cast<const float *>(x), k, 1, n, k, rows, ep, s);
    }
    if (e == cudaSuccess && dx) {
        // dx[rows x k] = dz wt: A(r, o) = dz[r * n + o]; B(o, c) = wt[o * k + c]
        Epi ep{1, nullptr, 0, nullptr, dx, nullptr, k};
        e = gemm(dz, n, 1, static_cast<const __nv_bfloat16 *>(wt), k, 1, rows, k, n, ep, s);
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
    scale_rows_kernel<<<grid1d((long long)rows * cols), 256, 0, (cudaStream_t)cuda_stream>>>(y, scale, rows, cols);
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
