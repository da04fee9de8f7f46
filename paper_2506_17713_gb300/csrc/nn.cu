// Kernels of the warm-start network (include/lbm_nn.h): periodic 3x3x3
// convolution forward / adjoint / weight gradient, leaky-ReLU backward, 2x pooling and
// upsampling, relative squared loss and Adam. FP32 on the CUDA cores, and the three
// convolution passes again as BF16 implicit GEMMs on the tcgen05 tensor cores with FP32
// accumulators in tensor memory. Every reduction runs in a fixed order.
#include <cuda_bf16.h>
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

// ---------------------------------------------------------------------------------
// Tensor-core convolutions (tcgen05, kind::f16 with BF16 operands, FP32 accumulate).
//
// Both GEMMs take M = 128 rows, one per tensor-memory lane, and N = output columns
// rounded up to 16. Operands sit in shared memory in the no-swizzle K-major layout:
// core matrices of 8 rows x 16 bytes (8 BF16 along K), neighbours along K 128 bytes
// apart (LBO), neighbouring 8-row groups SBO bytes apart. CUDA-core threads build the
// operand tiles (gather, periodic wrap, FP32 -> BF16 round to nearest even), one
// elected thread issues the MMAs and commits them to an mbarrier per stage, and the
// next stage is gathered while the tensor cores work on the previous one.

constexpr int kRows = 128;                          // MMA M, tensor-memory lanes
constexpr long long kWaitCycles = 4000000000LL;     // ~2 s at 2 GHz: an mbarrier wait gives up after this

__device__ unsigned g_tc_error;                     // set once a wait gave up

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, LBO, SBO (bytes, multiples of 16),
// descriptor version 1 (bits 46-48), base offset 0, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_bf16(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// wait for the completion of phase `parity`; false (and the error flag) after `limit`
// SM clock cycles (~2 s by default)
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit = kWaitCycles)
{
    const long long t0 = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > limit) {
            atomicOr(&g_tc_error, 1u);
            return false;
        }
    return true;
}

// Failure-detection check of the bounded wait: one thread initialises an mbarrier that
// expects one arrival, never arrives on it and waits for its first phase with the given
// limit. No tensor memory is allocated and no MMA or copy is in flight, so giving up is
// the only way out and nothing is left behind. The outcome goes to g_wait_result.
__device__ int g_wait_result;

__global__ void k_wait_selftest(long long limit)
{
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = smem_addr(&bar);
    mbar_init(b);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    g_wait_result = mbar_wait(b, 0, limit) ? 1 : 0;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

// D (+)= A B^T for one K step of 16
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// the mbarrier receives one arrival once every MMA issued so far by this thread is done
__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's lane (warp w reads lanes 32w .. 32w + 31)
__device__ __forceinline__ void tmem_load16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&b);
}

// 8 FP32 values -> one 16-byte core-matrix row of BF16
__device__ __forceinline__ void store_row8(uint8_t* dst, const float (&v)[8])
{
    *reinterpret_cast<uint4*>(dst) =
        make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
}

// voxel coordinates, and the index of the periodic neighbour at tap t (volumes of
// fewer than 2^31 voxels)
struct Vox {
    int x, y, z;
};

__device__ __forceinline__ Vox voxel(int p, int H, int W)
{
    const int r = p / W;
    return {p - r * W, r % H, r / H};
}

__device__ __forceinline__ int wrap(int c, int n) { return c < 0 ? n - 1 : (c == n ? 0 : c); }

__device__ __forceinline__ int tap_index(const Vox& v, int t, int D, int H, int W)
{
    return (wrap(v.z + t / 9 - 1, D) * H + wrap(v.y + (t / 3) % 3 - 1, H)) * W + wrap(v.x + t % 3 - 1, W);
}

// the u-th commit (u = 0, 1, ...) goes to stage u & 1 and completes that stage's
// barrier phase (u >> 1) & 1
__device__ __forceinline__ uint32_t commit_parity(uint32_t u) { return (u >> 1) & 1; }

struct TcConv {
    int cin, cp;        // input channels, rounded up to 16 (the K of one tap)
    int cout, npad;     // output channels, rounded up to 16 (the MMA N)
    int D, H, W;
    int P;              // voxels
    int tiles;          // ceil(P / 128)
    int taps;           // taps per pipeline stage: 3 (the x offsets of one (dz, dy)) or 1
    uint32_t tcols;     // tensor-memory columns allocated (power of two >= 32)
};

// forward: y[o][p] = b[o] + sum_{t, i} w[o][i][t] x[i][p + offset(t)] (leaky ReLU if relu).
// Implicit GEMM with rows = 128 voxels, K = (tap, channel) with channel fastest, N = o.
// Shared memory: [barriers | B = weights, whole K | A stage 0 | A stage 1]; a stage holds
// s.taps taps of 128 x cp BF16. Thread m builds row m; CP16 = cp / 16 when fixed at
// compile time (0: read from s); FULL: cin = cp, no padded channels to zero.
template <int CP16, bool FULL>
__global__ void __launch_bounds__(kRows, 1) k_conv3d_tc(const float* __restrict__ x, const float* __restrict__ wt,
                                                        const float* __restrict__ bias, TcConv s, int relu,
                                                        float* __restrict__ y)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const int cp = CP16 ? 16 * CP16 : s.cp;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    uint32_t* slot = reinterpret_cast<uint32_t*>(smem + 16);
    uint8_t* bsm = smem + 1024;
    const uint32_t kch = 27 * cp / 8;                         // 16-byte chunks along K
    const uint32_t b_bytes = (uint32_t)s.npad * kch * 16, tap_bytes = kRows * cp * 2;
    const uint32_t stage_bytes = (uint32_t)s.taps * tap_bytes;
    uint8_t* ast0 = bsm + b_bytes;                            // stage k at ast0 + k * stage_bytes
    const uint32_t sbo_b = kch * 128, sbo_a = cp / 8 * 128;
    const int m = threadIdx.x, warp = m >> 5;
    const size_t P = (size_t)s.P;

    for (uint32_t e = m; e < (uint32_t)s.npad * kch; e += kRows) {
        const int n = (int)(e / kch), c = (int)(e % kch);
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = c * 8 + q, t = k / cp, i = k % cp;
            v[q] = n < s.cout && i < s.cin ? wt[((size_t)n * s.cin + i) * 27 + t] : 0.0f;
        }
        store_row8(bsm + (n / 8) * sbo_b + c * 128 + (n % 8) * 16, v);
    }
    if (m == 0) {
        mbar_init(smem_addr(&bars[0]));
        mbar_init(smem_addr(&bars[1]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_addr(slot), s.tcols);
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *slot, idesc = idesc_bf16(s.npad);
    const uint32_t bars0 = smem_addr(&bars[0]);               // stage k's barrier at bars0 + 8 k
    uint32_t u = 0;                                           // commits so far
    bool ok = true;
    for (int tile = blockIdx.x; tile < s.tiles && ok; tile += gridDim.x) {
        const int p = tile * kRows + m;
        const bool active = p < s.P;                          // rows past the end are computed, not stored
        const Vox vx = voxel(active ? p : 0, s.H, s.W);
        for (int t0 = 0; t0 < 27; t0 += s.taps) {
            const uint32_t st = u & 1;
            if (u >= 2) {                                     // the stage's previous MMAs must be done
                const bool w = mbar_wait(bars0 + 8 * st, commit_parity(u - 2));
                if (__syncthreads_or(!w)) {
                    ok = false;
                    break;
                }
            }
            uint8_t* stage = ast0 + st * stage_bytes;
            for (int g = 0; g < s.taps; ++g) {
                const float* src = x + tap_index(vx, t0 + g, s.D, s.H, s.W);
                uint8_t* row = stage + g * tap_bytes + (m / 8) * sbo_a + (m % 8) * 16;
#pragma unroll
                for (int c = 0; c < cp / 8; ++c) {
                    float v[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        v[e] = FULL || c * 8 + e < s.cin ? *src : 0.0f;
                        src += P;
                    }
                    store_row8(row + c * 128, v);
                }
            }
            fence_async_smem();
            __syncthreads();
            if (m == 0) {
                tc_after_sync();
                for (int g = 0; g < s.taps; ++g) {
                    const uint32_t a0 = smem_addr(stage) + g * tap_bytes;
                    const uint32_t b0 = smem_addr(bsm) + (uint32_t)(t0 + g) * (cp / 8) * 128;
                    for (int j = 0; j < cp / 16; ++j)
                        mma_bf16(tmem, smem_desc(a0 + j * 256, 128, sbo_a), smem_desc(b0 + j * 256, 128, sbo_b),
                                 idesc, t0 + g > 0 || j > 0);
                }
                mma_commit(bars0 + 8 * st);
            }
            ++u;
        }
        if (!ok) break;
        const bool w = mbar_wait(bars0 + 8 * ((u - 1) & 1), commit_parity(u - 1));
        if (__syncthreads_or(!w)) {
            ok = false;
            break;
        }
        tc_after_sync();
        for (int n0 = 0; n0 < s.npad; n0 += 16) {
            float acc[16];
            tmem_load16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)n0, acc);
            if (active)
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int o = n0 + q;
                    if (o < s.cout) {
                        const float v = acc[q] + (bias ? bias[o] : 0.0f);
                        y[(size_t)o * P + p] = relu && v < 0.0f ? kLeak * v : v;
                    }
                }
        }
        tc_before_sync();      // the next tile's first MMA (after a barrier) overwrites the accumulator
    }
    if (!ok)                   // give MMAs still in flight a bounded chance to finish
        for (uint32_t k = u >= 2 ? u - 2 : 0; k < u; ++k) mbar_wait(bars0 + 8 * (k & 1), commit_parity(k));
    tc_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_after_sync();
        tmem_free(tmem, s.tcols);
    }
}

constexpr int kGwK = 64;   // voxels per K stage of the weight gradient (4 MMA steps)

struct TcGw {
    int cin, cout, npad;
    int D, H, W;
    int P;
    int rows;           // 27 cin weight rows (r = t cin + i) and one row of ones (bias gradient)
    int chunks;         // 64-voxel K stages per segment
    int segs;           // voxel segments (grid x)
    uint32_t tcols;
};

// partial weight gradient of one voxel segment (blockIdx.x) and one tile of 128 rows
// (blockIdx.y): D[r][o] = sum_p x[i][p + offset(t)] gy[o][p] for r = t cin + i, and
// D[27 cin][o] = sum_p gy[o][p]. K = voxels, 64 per stage. Shared memory:
// [barriers | neighbour table x 2 | B (gy) x 2 | A x 2], operands 8 core matrices deep in K.
__global__ void __launch_bounds__(kRows) k_conv3d_gw_tc(const float* __restrict__ x, const float* __restrict__ gy,
                                                        TcGw s, float* __restrict__ part)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    uint32_t* slot = reinterpret_cast<uint32_t*>(smem + 16);
    constexpr int kTab = 27 * kGwK;                           // neighbour table entries per stage
    int* nbr0 = reinterpret_cast<int*>(smem + 1024);
    const uint32_t b_bytes = (uint32_t)s.npad * kGwK * 2, a_bytes = kRows * kGwK * 2;
    uint8_t* bst0 = smem + 1024 + 2 * kTab * 4;               // stage k at bst0 + k * b_bytes
    uint8_t* ast0 = bst0 + 2 * b_bytes;                       // stage k at ast0 + k * a_bytes
    const int m = threadIdx.x, warp = m >> 5;
    const int seg = blockIdx.x, r0 = blockIdx.y * kRows, r = r0 + m;
    const bool wrow = r < 27 * s.cin, ones = r == 27 * s.cin;
    // taps met by the weight rows of this tile: the neighbour table holds only these
    const int t_lo = r0 / s.cin, t_hi = (r0 + kRows - 1) / s.cin < 26 ? (r0 + kRows - 1) / s.cin : 26;
    const int ntab = t_lo <= t_hi ? (t_hi - t_lo + 1) * kGwK : 0;
    const int t = wrow ? r / s.cin : t_lo;
    const float* xi = x + (size_t)(wrow ? r % s.cin : 0) * s.P;
    if (m == 0) {
        mbar_init(smem_addr(&bars[0]));
        mbar_init(smem_addr(&bars[1]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_addr(slot), s.tcols);
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *slot, idesc = idesc_bf16(s.npad), bars0 = smem_addr(&bars[0]);
    const int nsteps = (s.P + kGwK - 1) / kGwK;
    const int c0 = seg * s.chunks, c1 = c0 + s.chunks < nsteps ? c0 + s.chunks : nsteps;
    uint32_t u = 0;
    bool ok = true;
    for (int c = c0; c < c1; ++c) {
        const uint32_t st = u & 1;
        if (u >= 2) {
            const bool w = mbar_wait(bars0 + 8 * st, commit_parity(u - 2));
            if (__syncthreads_or(!w)) {
                ok = false;
                break;
            }
        }
        const int p0 = c * kGwK;
        int* nbr = nbr0 + st * kTab;
        uint8_t* bst = bst0 + st * b_bytes;
        uint8_t* ast = ast0 + st * a_bytes;
        for (int e = m; e < ntab; e += kRows) {               // neighbour of voxel p0 + k at tap tt, or -1
            const int k = e % kGwK, tt = t_lo + e / kGwK, p = p0 + k;
            nbr[e] = p < s.P ? tap_index(voxel(p, s.H, s.W), tt, s.D, s.H, s.W) : -1;
        }
        for (int e = m; e < s.npad * (kGwK / 8); e += kRows) {  // B: gy rows, 8 voxels per core-matrix row
            const int n = e / (kGwK / 8), h = e % (kGwK / 8);
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int p = p0 + h * 8 + q;
                v[q] = n < s.cout && p < s.P ? gy[(size_t)n * s.P + p] : 0.0f;
            }
            store_row8(bst + (n / 8) * (kGwK * 16) + h * 128 + (n % 8) * 16, v);
        }
        __syncthreads();
        {                                                      // A: this thread's row
            const int* nt = nbr + (wrow ? (t - t_lo) * kGwK : 0);
            uint8_t* row = ast + (m / 8) * (kGwK * 16) + (m % 8) * 16;
#pragma unroll
            for (int h = 0; h < kGwK / 8; ++h) {
                float v[8];
                if (wrow) {
                    const int4 a = *reinterpret_cast<const int4*>(nt + h * 8);
                    const int4 b = *reinterpret_cast<const int4*>(nt + h * 8 + 4);
                    const int nq[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[q] = nq[q] >= 0 ? xi[nq[q]] : 0.0f;
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[q] = ones && p0 + h * 8 + q < s.P ? 1.0f : 0.0f;
                }
                store_row8(row + h * 128, v);
            }
        }
        fence_async_smem();
        __syncthreads();
        if (m == 0) {
            tc_after_sync();
            for (int j = 0; j < kGwK / 16; ++j)
                mma_bf16(tmem, smem_desc(smem_addr(ast) + j * 256, 128, kGwK * 16),
                         smem_desc(smem_addr(bst) + j * 256, 128, kGwK * 16), idesc, c > c0 || j > 0);
            mma_commit(bars0 + 8 * st);
        }
        ++u;
    }
    if (ok && u > 0) {
        const bool w = mbar_wait(bars0 + 8 * ((u - 1) & 1), commit_parity(u - 1));
        ok = !__syncthreads_or(!w);
    }
    if (ok) {
        tc_after_sync();
        const int rr = blockIdx.y * kRows + warp * 32 + (m & 31);   // the row of this thread's lane
        for (int n0 = 0; n0 < s.npad; n0 += 16) {
            float acc[16];
            if (u > 0) {
                tmem_load16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)n0, acc);
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
            }
            if (rr < s.rows)
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (n0 + q < s.cout) part[((size_t)seg * s.rows + rr) * s.cout + n0 + q] = acc[q];
        }
    } else {
        for (uint32_t k = u >= 2 ? u - 2 : 0; k < u; ++k) mbar_wait(bars0 + 8 * (k & 1), commit_parity(k));
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_after_sync();
        tmem_free(tmem, s.tcols);
    }
}

// gw[o][i][t] (+)= sum over segments of part[seg][t cin + i][o], gb[o] (+)= ... [27 cin][o],
// segments added in order
__global__ void k_conv3d_gw_tc_final(const float* __restrict__ part, int segs, int cin, int cout,
                                     float* __restrict__ gw, float* __restrict__ gb, int accumulate)
{
    const int rows = 27 * cin + 1;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)rows * cout) return;
    const int o = (int)(e % cout), r = (int)(e / cout);
    if (r == 27 * cin && !gb) return;
    float s = 0.0f;
    for (int g = 0; g < segs; ++g) s += part[((long long)g * rows + r) * cout + o];
    if (r == 27 * cin) {
        gb[o] = accumulate ? gb[o] + s : s;
        return;
    }
    const int t = r / cin, i = r % cin;
    float& dst = gw[((long long)o * cin + i) * 27 + t];
    dst = accumulate ? dst + s : s;
}

uint32_t tmem_columns(int n)
{
    uint32_t c = 32;
    while ((int)c < n) c <<= 1;
    return c;
}

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return n;
}

constexpr size_t kMaxSmem = 227 * 1024;
constexpr size_t kSmPerSm = 228 * 1024;                 // shared memory of one SM (1 KB of it reserved per CTA)

// CTAs of `kernel` that fit on one SM: registers (256 per warp granule), shared memory,
// threads, and the tensor-memory columns each CTA allocates
template <class K>
int resident_ctas(K kernel, size_t smem_bytes, uint32_t tcols)
{
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return 0;
    const int warps = kRows / 32;
    const int regs_cta = warps * ((fa.numRegs * 32 + 255) / 256) * 256;
    int n = 65536 / (regs_cta > 0 ? regs_cta : 1);
    const int by_smem = (int)(kSmPerSm / (smem_bytes + 1024));
    const int by_tmem = (int)(512 / tcols);
    n = n < by_smem ? n : by_smem;
    n = n < by_tmem ? n : by_tmem;
    n = n < 2048 / kRows ? n : 2048 / kRows;
    return n;
}

size_t conv_tc_smem(const TcConv& s)
{
    return 1024 + (size_t)s.npad * 27 * s.cp * 2 + 2 * (size_t)s.taps * kRows * s.cp * 2 + 1024;
}

// shape of a forward launch; LBM_ERR_INVALID_ARG beyond the limits (no device call).
// Three taps per stage when that still leaves room for three CTAs per SM, else one.
lbm_status conv_tc_shape(int cin, int d, int h, int w, int cout, TcConv& s, size_t& bytes)
{
    s.cin = cin;
    s.cp = (cin + 15) / 16 * 16;
    s.cout = cout;
    s.npad = (cout + 15) / 16 * 16;
    s.D = d;
    s.H = h;
    s.W = w;
    const long long P = (long long)d * h * w;
    if (s.npad > 256 || P > 0x7fffffffLL - kRows) return LBM_ERR_INVALID_ARG;
    s.P = (int)P;
    s.tiles = (s.P + kRows - 1) / kRows;
    s.tcols = tmem_columns(s.npad);
    s.taps = 3;
    bytes = conv_tc_smem(s);
    if (bytes + 1024 > kSmPerSm / 3) {
        s.taps = 1;
        bytes = conv_tc_smem(s);
    }
    return bytes > kMaxSmem ? LBM_ERR_INVALID_ARG : LBM_OK;
}

template <int CP16, bool FULL>
lbm_status conv_tc_launch(const float* x, const TcConv& s, size_t bytes, const float* wt, const float* bias,
                          int relu, float* y, cudaStream_t st)
{
    if (cudaFuncSetAttribute(k_conv3d_tc<CP16, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return LBM_ERR_CUDA;
    const int per_sm = resident_ctas(k_conv3d_tc<CP16, FULL>, bytes, s.tcols), sms = sm_count();
    if (per_sm < 1 || sms < 1) return LBM_ERR_CUDA;
    const long long grid = (long long)sms * per_sm;
    k_conv3d_tc<CP16, FULL>
        <<<(unsigned)(grid < s.tiles ? grid : s.tiles), kRows, bytes, st>>>(x, wt, bias, s, relu, y);
    return launched();
}

lbm_status conv_tc(const float* x, const TcConv& s, size_t bytes, const float* wt, const float* bias, int relu,
                   float* y, cudaStream_t st)
{
    const bool full = s.cin == s.cp;
    switch (s.cp / 16) {
    case 1: return full ? conv_tc_launch<1, true>(x, s, bytes, wt, bias, relu, y, st)
                        : conv_tc_launch<1, false>(x, s, bytes, wt, bias, relu, y, st);
    case 2: return full ? conv_tc_launch<2, true>(x, s, bytes, wt, bias, relu, y, st)
                        : conv_tc_launch<2, false>(x, s, bytes, wt, bias, relu, y, st);
    case 3: return full ? conv_tc_launch<3, true>(x, s, bytes, wt, bias, relu, y, st)
                        : conv_tc_launch<3, false>(x, s, bytes, wt, bias, relu, y, st);
    case 4: return full ? conv_tc_launch<4, true>(x, s, bytes, wt, bias, relu, y, st)
                        : conv_tc_launch<4, false>(x, s, bytes, wt, bias, relu, y, st);
    default: return conv_tc_launch<0, false>(x, s, bytes, wt, bias, relu, y, st);
    }
}

size_t gw_tc_smem(const TcGw& s)
{
    return 1024 + 2 * 27 * kGwK * 4 + 2 * (size_t)s.npad * kGwK * 2 + 2 * (size_t)kRows * kGwK * 2 + 1024;
}

lbm_status gw_tc(const float* x, int cin, const float* gy, int cout, int d, int h, int w, float* gw, float* gb,
                 int accumulate, float* scratch, cudaStream_t st)
{
    TcGw s;
    s.cin = cin;
    s.cout = cout;
    s.npad = (cout + 15) / 16 * 16;
    s.D = d;
    s.H = h;
    s.W = w;
    const long long P = (long long)d * h * w;
    if (s.npad > 256 || P > 0x7fffffffLL - kGwK || 27LL * cin + 1 > 0x7fffffffLL / 2) return LBM_ERR_INVALID_ARG;
    s.P = (int)P;
    s.rows = 27 * cin + 1;
    s.tcols = tmem_columns(s.npad);
    const int nsteps = (s.P + kGwK - 1) / kGwK;
    s.segs = nsteps < LBM_NN_GW_TC_SEGMENTS ? nsteps : LBM_NN_GW_TC_SEGMENTS;
    s.chunks = (nsteps + s.segs - 1) / s.segs;
    const size_t bytes = gw_tc_smem(s);
    if (bytes > kMaxSmem) return LBM_ERR_INVALID_ARG;
    if (cudaFuncSetAttribute(k_conv3d_gw_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return LBM_ERR_CUDA;
    const dim3 grid((unsigned)s.segs, (unsigned)((s.rows + kRows - 1) / kRows));
    k_conv3d_gw_tc<<<grid, kRows, bytes, st>>>(x, gy, s, scratch);
    k_conv3d_gw_tc_final<<<blocks_for((long long)s.rows * cout), kThreads, 0, st>>>(scratch, s.segs, cin, cout, gw,
                                                                                     gb, accumulate);
    return launched();
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

lbm_status lbm_nn_conv3d_tc(const float* x, int cin, int d, int h, int w, const float* weight, const float* bias,
                            int cout, int relu, float* y, void* stream)
{
    if (!x || !weight || !y || cin < 1 || cout < 1 || d < 1 || h < 1 || w < 1) return LBM_ERR_INVALID_ARG;
    TcConv s;
    size_t bytes = 0;
    const lbm_status e = conv_tc_shape(cin, d, h, w, cout, s, bytes);
    return e != LBM_OK ? e : conv_tc(x, s, bytes, weight, bias, relu, y, (cudaStream_t)stream);
}

lbm_status lbm_nn_conv3d_tc_grad_input(const float* gy, int cout, int d, int h, int w, const float* weight, int cin,
                                       float* wt_scratch, float* gx, void* stream)
{
    if (!gy || !weight || !wt_scratch || !gx || cin < 1 || cout < 1 || d < 1 || h < 1 || w < 1)
        return LBM_ERR_INVALID_ARG;
    TcConv s;
    size_t bytes = 0;
    lbm_status e = conv_tc_shape(cout, d, h, w, cin, s, bytes);     // the adjoint maps cout channels to cin
    if (e != LBM_OK) return e;
    cudaStream_t st = (cudaStream_t)stream;
    k_flip_transpose<<<blocks_for((long long)cout * cin * 27), kThreads, 0, st>>>(weight, cout, cin, wt_scratch);
    e = launched();
    return e != LBM_OK ? e : conv_tc(gy, s, bytes, wt_scratch, nullptr, 0, gx, st);
}

lbm_status lbm_nn_conv3d_tc_grad_weight(const float* x, int cin, const float* gy, int cout, int d, int h, int w,
                                        float* gw, float* gb, int accumulate, float* scratch, void* stream)
{
    if (!x || !gy || !gw || !scratch || cin < 1 || cout < 1 || d < 1 || h < 1 || w < 1) return LBM_ERR_INVALID_ARG;
    return gw_tc(x, cin, gy, cout, d, h, w, gw, gb, accumulate, scratch, (cudaStream_t)stream);
}

lbm_status lbm_nn_wait_selftest(long long limit_cycles, int* completed, void* stream)
{
    if (!completed || limit_cycles < 1 || limit_cycles > kWaitCycles) return LBM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int v = -1;
    if (cudaMemcpyToSymbolAsync(g_wait_result, &v, sizeof v, 0, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return LBM_ERR_CUDA;
    k_wait_selftest<<<1, 1, 0, st>>>(limit_cycles);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    if (cudaMemcpyFromSymbolAsync(&v, g_wait_result, sizeof v, 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return LBM_ERR_CUDA;
    *completed = v;
    return LBM_OK;
}

lbm_status lbm_nn_tc_error(int* flag)
{
    if (!flag) return LBM_ERR_INVALID_ARG;
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_error, sizeof v) != cudaSuccess) return LBM_ERR_CUDA;
    *flag = (int)v;
    v = 0;
    return cudaMemcpyToSymbol(g_tc_error, &v, sizeof v) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

}  // extern "C"
