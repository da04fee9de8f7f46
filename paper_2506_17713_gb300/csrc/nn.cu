// Kernels of the warm-start network (include/lbm_nn.h): periodic 3x3x3
// convolution forward / adjoint / weight gradient, leaky-ReLU backward, 2x pooling and
// upsampling, relative squared loss and Adam. FP32 throughout; every reduction
// runs in a fixed order.
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm_nn.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCoChunk = 8;    // output channels per CTA (blockIdx.y)
constexpr int kCiChunk = 16;   // input channels staged in shared memory at a time
constexpr float kLeak = 0.01f; // slope of the leaky ReLU for negative inputs

// y[o][p] = b[o] + sum_{i, t} w[o][i][t] x[i][p + offset(t)], periodic; one thread per
// voxel, 8 output channels per CTA
__global__ void __launch_bounds__(kThreads) k_conv3d(const float* __restrict__ x, int cin, int D, int H, int W,
                                                     const float* __restrict__ wt, const float* __restrict__ bias,
                                                     int cout, int relu, float* __restrict__ y)
{
    __shared__ float ws[kCiChunk][27][kCoChunk];
    const int co0 = blockIdx.y * kCoChunk;
    const long long P = (long long)D * H * W;
    const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
    const bool active = p < P;
    int xo[3] = {0, 0, 0}, yo[3] = {0, 0, 0}, zo[3] = {0, 0, 0};
    if (active) {
        const int xx = (int)(p % W), yy = (int)((p / W) % H), zz = (int)(p / ((long long)W * H));
        xo[0] = xx == 0 ? W - 1 : xx - 1;
        xo[1] = xx;
        xo[2] = xx == W - 1 ? 0 : xx + 1;
        yo[0] = (yy == 0 ? H - 1 : yy - 1) * W;
        yo[1] = yy * W;
        yo[2] = (yy == H - 1 ? 0 : yy + 1) * W;
        zo[0] = (zz == 0 ? D - 1 : zz - 1) * W * H;
        zo[1] = zz * W * H;
        zo[2] = (zz == D - 1 ? 0 : zz + 1) * W * H;
    }
    float acc[kCoChunk];
#pragma unroll
    for (int c = 0; c < kCoChunk; ++c) acc[c] = (bias && co0 + c < cout) ? bias[co0 + c] : 0.0f;
    for (int ci0 = 0; ci0 < cin; ci0 += kCiChunk) {
        const int nci = cin - ci0 < kCiChunk ? cin - ci0 : kCiChunk;
        __syncthreads();
        for (int e = threadIdx.x; e < nci * 27 * kCoChunk; e += kThreads) {
            const int c = e % kCoChunk, t = (e / kCoChunk) % 27, i = e / (kCoChunk * 27);
            ws[i][t][c] = co0 + c < cout ? wt[((long long)(co0 + c) * cin + ci0 + i) * 27 + t] : 0.0f;
        }
        __syncthreads();
        if (active) {
            for (int i = 0; i < nci; ++i) {
                const float* __restrict__ xi = x + (long long)(ci0 + i) * P;
#pragma unroll
                for (int t = 0; t < 27; ++t) {
                    const float v = xi[zo[t / 9] + yo[(t / 3) % 3] + xo[t % 3]];
#pragma unroll
                    for (int c = 0; c < kCoChunk; ++c) acc[c] = fmaf(ws[i][t][c], v, acc[c]);
                }
            }
        }
    }
    if (!active) return;
#pragma unroll
    for (int c = 0; c < kCoChunk; ++c)
        if (co0 + c < cout) y[(long long)(co0 + c) * P + p] = relu && acc[c] < 0.0f ? kLeak * acc[c] : acc[c];
}

// wt[i][o][26 - t] = w[o][i][t]: the adjoint convolution's weights
__global__ void k_flip_transpose(const float* __restrict__ w, int cout, int cin, float* __restrict__ wt)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)cout * cin * 27) return;
    const int t = (int)(e % 27), i = (int)((e / 27) % cin), o = (int)(e / (27LL * cin));
    wt[((long long)i * cout + o) * 27 + (26 - t)] = w[e];
}

// partial sums of gw[o][i][:] and gb[o] over one segment of the voxels: CTA (o*cin + i, seg)
__global__ void __launch_bounds__(kThreads) k_conv3d_gw_partial(const float* __restrict__ x, int cin,
                                                                const float* __restrict__ gy, int cout, int D,
                                                                int H, int W, float* __restrict__ part)
{
    __shared__ float red[28][kThreads];
    const int o = blockIdx.x / cin, i = blockIdx.x % cin, seg = blockIdx.y;
    const long long P = (long long)D * H * W;
    const long long per = (P + LBM_NN_GW_SEGMENTS - 1) / LBM_NN_GW_SEGMENTS;
    const long long p0 = seg * per, p1 = p0 + per < P ? p0 + per : P;
    float acc[28];
#pragma unroll
    for (int t = 0; t < 28; ++t) acc[t] = 0.0f;
    const float* __restrict__ xi = x + (long long)i * P;
    const float* __restrict__ go = gy + (long long)o * P;
    for (long long p = p0 + threadIdx.x; p < p1; p += kThreads) {
        const int xx = (int)(p % W), yy = (int)((p / W) % H), zz = (int)(p / ((long long)W * H));
        const int xo[3] = {xx == 0 ? W - 1 : xx - 1, xx, xx == W - 1 ? 0 : xx + 1};
        const int yo[3] = {(yy == 0 ? H - 1 : yy - 1) * W, yy * W, (yy == H - 1 ? 0 : yy + 1) * W};
        const int zo[3] = {(zz == 0 ? D - 1 : zz - 1) * W * H, zz * W * H, (zz == D - 1 ? 0 : zz + 1) * W * H};
        const float g = go[p];
#pragma unroll
        for (int t = 0; t < 27; ++t) acc[t] = fmaf(g, xi[zo[t / 9] + yo[(t / 3) % 3] + xo[t % 3]], acc[t]);
        acc[27] += g;
    }
#pragma unroll
    for (int t = 0; t < 28; ++t) red[t][threadIdx.x] = acc[t];
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int t = 0; t < 28; ++t) red[t][threadIdx.x] += red[t][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 28)
        part[(((long long)seg * cout + o) * cin + i) * 28 + threadIdx.x] = red[threadIdx.x][0];
}

// gw, gb from the partial sums, segments added in order
__global__ void k_conv3d_gw_final(const float* __restrict__ part, int cout, int cin, float* __restrict__ gw,
                                  float* __restrict__ gb, int accumulate)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)cout * cin * 28) return;
    const int t = (int)(e % 28), oi = (int)(e / 28), i = oi % cin, o = oi / cin;
    if (t == 27 && (i != 0 || !gb)) return;   // bias once per output channel (from input channel 0)
    float s = 0.0f;
    for (int seg = 0; seg < LBM_NN_GW_SEGMENTS; ++seg) s += part[((long long)seg * cout * cin + oi) * 28 + t];
    if (t == 27) gb[o] = accumulate ? gb[o] + s : s;
    else gw[((long long)o * cin + i) * 27 + t] = accumulate ? gw[((long long)o * cin + i) * 27 + t] + s : s;
}

__global__ void k_axpy(float* __restrict__ y, const float* __restrict__ x, long long n, float a)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) y[e] = fmaf(a, x[e], y[e]);
}

__global__ void k_relu_grad(const float* __restrict__ y, float* __restrict__ g, long long n)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n && !(y[e] > 0.0f)) g[e] *= kLeak;
}

// y[c][z][y][x] = mean of x over the 2x2x2 block; d, h, w: sizes of x
__global__ void k_pool2(const float* __restrict__ x, int c, int d, int h, int w, float* __restrict__ y)
{
    const int d2 = d / 2, h2 = h / 2, w2 = w / 2;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)c * d2 * h2 * w2) return;
    const int xx = (int)(e % w2), yy = (int)((e / w2) % h2), zz = (int)((e / ((long long)w2 * h2)) % d2);
    const int ch = (int)(e / ((long long)w2 * h2 * d2));
    const float* b = x + (long long)ch * d * h * w;
    float s = 0.0f;
    for (int a = 0; a < 2; ++a)
        for (int bb = 0; bb < 2; ++bb)
            for (int cc = 0; cc < 2; ++cc) s += b[((long long)(2 * zz + a) * h + 2 * yy + bb) * w + 2 * xx + cc];
    y[e] = 0.125f * s;
}

__global__ void k_pool2_grad(const float* __restrict__ gy, int c, int d, int h, int w, float* __restrict__ gx)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)c * d * h * w) return;
    const int xx = (int)(e % w), yy = (int)((e / w) % h), zz = (int)((e / ((long long)w * h)) % d);
    const int ch = (int)(e / ((long long)w * h * d));
    gx[e] = 0.125f * gy[(((long long)ch * (d / 2) + zz / 2) * (h / 2) + yy / 2) * (w / 2) + xx / 2];
}

// y[c][Z][Y][X] = x[c][Z/2][Y/2][X/2]; d, h, w: sizes of x
__global__ void k_up2(const float* __restrict__ x, int c, int d, int h, int w, float* __restrict__ y)
{
    const int D = 2 * d, Hh = 2 * h, Ww = 2 * w;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)c * D * Hh * Ww) return;
    const int xx = (int)(e % Ww), yy = (int)((e / Ww) % Hh), zz = (int)((e / ((long long)Ww * Hh)) % D);
    const int ch = (int)(e / ((long long)Ww * Hh * D));
    y[e] = x[(((long long)ch * d + zz / 2) * h + yy / 2) * w + xx / 2];
}

__global__ void k_up2_grad(const float* __restrict__ gy, int c, int d, int h, int w, float* __restrict__ gx)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)c * d * h * w) return;
    const int xx = (int)(e % w), yy = (int)((e / w) % h), zz = (int)((e / ((long long)w * h)) % d);
    const int ch = (int)(e / ((long long)w * h * d));
    const int Hh = 2 * h, Ww = 2 * w;
    const float* b = gy + (long long)ch * 8 * d * h * w;
    float s = 0.0f;
    for (int a = 0; a < 2; ++a)
        for (int bb = 0; bb < 2; ++bb)
            for (int cc = 0; cc < 2; ++cc) s += b[((long long)(2 * zz + a) * Hh + 2 * yy + bb) * Ww + 2 * xx + cc];
    gx[e] = s;
}

// one CTA: sums[0] = sum (p - t)^2, sums[1] = sum t^2 (FP64, fixed order)
__global__ void __launch_bounds__(1024) k_loss_sums(const float* __restrict__ p, const float* __restrict__ t,
                                                    long long n, double* __restrict__ sums,
                                                    double* __restrict__ loss)
{
    __shared__ double r0[1024], r1[1024];
    double a = 0.0, b = 0.0;
    for (long long e = threadIdx.x; e < n; e += 1024) {
        const double d = (double)p[e] - (double)t[e];
        a += d * d;
        b += (double)t[e] * (double)t[e];
    }
    r0[threadIdx.x] = a;
    r1[threadIdx.x] = b;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            r0[threadIdx.x] += r0[threadIdx.x + s];
            r1[threadIdx.x] += r1[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sums[0] = r0[0];
        sums[1] = r1[0];
        if (loss) *loss = r1[0] > 0.0 ? r0[0] / r1[0] : 0.0;
    }
}

__global__ void k_loss_grad(const float* __restrict__ p, const float* __restrict__ t, long long n,
                            const double* __restrict__ sums, float* __restrict__ g)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double s = sums[1] > 0.0 ? sums[1] : 1.0;
    g[e] = (float)(2.0 * ((double)p[e] - (double)t[e]) / s);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.0f - b1) * gg;
    const float vv = b2 * v[e] + (1.0f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

unsigned blocks_for(long long n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

lbm_status launched()
{
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

}  // namespace

extern "C" {

lbm_status lbm_nn_conv3d(const float* x, int cin, int d, int h, int w, const float* weight, const float* bias,
                         int cout, int relu, float* y, void* stream)
{
    if (!x || !weight || !y || cin < 1 || cout < 1 || d < 1 || h < 1 || w < 1) return LBM_ERR_INVALID_ARG;
    const long long P = (long long)d * h * w;
    const dim3 grid(blocks_for(P), (unsigned)((cout + kCoChunk - 1) / kCoChunk));
    k_conv3d<<<grid, kThreads, 0, (cudaStream_t)stream>>>(x, cin, d, h, w, weight, bias, cout, relu, y);
    return launched();
}

lbm_status lbm_nn_conv3d_grad_input(const float* gy, int cout, int d, int h, int w, const float* weight, int cin,
                                    float* wt_scratch, float* gx, void* stream)
{
    if (!gy || !weight || !wt_scratch || !gx || cin < 1 || cout < 1 || d < 1 || h < 1 || w < 1)
        return LBM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    k_flip_transpose<<<blocks_for((long long)cout * cin * 27), kThreads, 0, st>>>(weight, cout, cin, wt_scratch);
    const long long P = (long long)d * h * w;
    const dim3 grid(blocks_for(P), (unsigned)((cin + kCoChunk - 1) / kCoChunk));
    k_conv3d<<<grid, kThreads, 0, st>>>(gy, cout, d, h, w, wt_scratch, nullptr, cin, 0, gx);
    return launched();
}

lbm_status lbm_nn_conv3d_grad_weight(const float* x, int cin, const float* gy, int cout, int d, int h, int w,
                                     float* gw, float* gb, int accumulate, float* scratch, void* stream)
{
    if (!x || !gy || !gw || !scratch || cin < 1 || cout < 1 || d < 1 || h < 1 || w < 1) return LBM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const dim3 grid((unsigned)(cout * cin), LBM_NN_GW_SEGMENTS);
    k_conv3d_gw_partial<<<grid, kThreads, 0, st>>>(x, cin, gy, cout, d, h, w, scratch);
    k_conv3d_gw_final<<<blocks_for((long long)cout * cin * 28), kThreads, 0, st>>>(scratch, cout, cin, gw, gb,
                                                                                  accumulate);
    return launched();
}

lbm_status lbm_nn_axpy(float* y, const float* x, long long n, float a, void* stream)
{
    if (!y || !x || n < 1) return LBM_ERR_INVALID_ARG;
    k_axpy<<<blocks_for(n), kThreads, 0, (cudaStream_t)stream>>>(y, x, n, a);
    return launched();
}

lbm_status lbm_nn_relu_grad(const float* y, float* g, long long n, void* stream)
{
    if (!y || !g || n < 1) return LBM_ERR_INVALID_ARG;
    k_relu_grad<<<blocks_for(n), kThreads, 0, (cudaStream_t)stream>>>(y, g, n);
    return launched();
}

lbm_status lbm_nn_avg_pool2(const float* x, int c, int d, int h, int w, float* y, void* stream)
{
    if (!x || !y || c < 1 || d < 2 || h < 2 || w < 2 || (d | h | w) & 1) return LBM_ERR_INVALID_ARG;
    k_pool2<<<blocks_for((long long)c * d * h * w / 8), kThreads, 0, (cudaStream_t)stream>>>(x, c, d, h, w, y);
    return launched();
}

lbm_status lbm_nn_avg_pool2_grad(const float* gy, int c, int d, int h, int w, float* gx, void* stream)
{
    if (!gy || !gx || c < 1 || d < 2 || h < 2 || w < 2 || (d | h | w) & 1) return LBM_ERR_INVALID_ARG;
    k_pool2_grad<<<blocks_for((long long)c * d * h * w), kThreads, 0, (cudaStream_t)stream>>>(gy, c, d, h, w, gx);
    return launched();
}

lbm_status lbm_nn_up2(const float* x, int c, int d, int h, int w, float* y, void* stream)
{
    if (!x || !y || c < 1 || d < 1 || h < 1 || w < 1) return LBM_ERR_INVALID_ARG;
    k_up2<<<blocks_for(8LL * c * d * h * w), kThreads, 0, (cudaStream_t)stream>>>(x, c, d, h, w, y);
    return launched();
}

lbm_status lbm_nn_up2_grad(const float* gy, int c, int d, int h, int w, float* gx, void* stream)
{
    if (!gy || !gx || c < 1 || d < 1 || h < 1 || w < 1) return LBM_ERR_INVALID_ARG;
    k_up2_grad<<<blocks_for((long long)c * d * h * w), kThreads, 0, (cudaStream_t)stream>>>(gy, c, d, h, w, gx);
    return launched();
}

lbm_status lbm_nn_rel_loss(const float* p, const float* t, long long n, float* grad, double* sums, double* loss,
                           void* stream)
{
    if (!p || !t || !sums || n < 1) return LBM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    k_loss_sums<<<1, 1024, 0, st>>>(p, t, n, sums, loss);
    if (grad) k_loss_grad<<<blocks_for(n), kThreads, 0, st>>>(p, t, n, sums, grad);
    return launched();
}

lbm_status lbm_nn_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2, void* stream)
{
    if (!p || !g || !m || !v || n < 1) return LBM_ERR_INVALID_ARG;
    k_adam<<<blocks_for(n), kThreads, 0, (cudaStream_t)stream>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return launched();
}

}  // extern "C"
