// lbm_mass_noalloc: total mass per component with no memory allocation at all.
//
// Some callers cannot allocate device memory: host processes that hand the GPU to a
// framework owning every allocation, or callers whose memory pool is exhausted by the
// lattice itself. This entry point computes the same mass sums as lbm_diagnostics
// from populations the caller already holds, and keeps its scratch (the per-block FP64
// partial sums of the two-stage reduction) in a file-scope device array instead of a
// caller workspace. That array lives on every GPU that loads the library until the
// process exits. The call copies the totals to host memory and synchronises its
// stream, which a stream being captured into a CUDA graph cannot do: on such a stream
// it returns LBM_ERR_INVALID_ARG before enqueuing anything, so the capture stays valid.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "lbm.h"

namespace {

constexpr int kThreads = 256;                       // threads per block
constexpr int kNodesPerThread = 64;                 // nodes one thread sums
constexpr long long kNodesPerBlock = (long long)kThreads * kNodesPerThread;   // 16384
constexpr int kMaxBlocks = LBM_NOALLOC_MAX_NODES / (int)kNodesPerBlock;        // 1024
constexpr int kMaxDevices = 64;

static_assert(LBM_NOALLOC_MAX_NODES % kNodesPerBlock == 0, "max nodes must fill whole blocks");

// Scratch shared by every call: [kMaxBlocks][2] partial sums, then the 2 totals.
static __device__ __align__(256) double g_mass_scratch[kMaxBlocks * 2 + 2];

// Device address of g_mass_scratch per device ordinal (host code cannot use the
// symbol itself: in host code its name stands for a host-side shadow object). Atomic,
// because host threads making their first call on a device may fill the same entry at
// once (with the same value).
std::atomic<void*> g_scratch_ptr[kMaxDevices] = {};

template <typename T>
__global__ void __launch_bounds__(kThreads) k_mass_partials(const T* __restrict__ f, int K, int Q, long long N,
                                                          double* __restrict__ scratch)
{
    // block b sums nodes [b*kNodesPerBlock, (b+1)*kNodesPerBlock), thread t every
    // kThreads-th node from b*kNodesPerBlock + t: a fixed order, so results are
    // reproducible bit for bit
    __shared__ double sh[kThreads / 32][2];
    const long long base = (long long)blockIdx.x * kNodesPerBlock + threadIdx.x;
    double acc[2] = {0.0, 0.0};
    for (int k = 0; k < K; ++k) {
        const T* fk = f + (long long)k * Q * N;
        for (int m = 0; m < kNodesPerThread; ++m) {
            const long long n = base + (long long)m * kThreads;
            if (n >= N) break;
            double r = 0.0;
            for (int i = 0; i < Q; ++i) r += (double)fk[(long long)i * N + n];
            acc[k] += r;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 2; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[warp][k] = v;
    }
    __syncthreads();
    if (warp == 0) {
        for (int k = 0; k < 2; ++k) {
            double v = lane < kThreads / 32 ? sh[lane][k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) scratch[2 * blockIdx.x + k] = v;
        }
    }
}

__global__ void k_mass_total(int nblocks, double* __restrict__ scratch)
{
    // one warp; lane l sums blocks l, l+32, ... in order, then a fixed shuffle tree.
    // Every total is written, so nothing from an earlier call survives into this one.
    const int lane = threadIdx.x;
    for (int k = 0; k < 2; ++k) {
        double v = 0.0;
        for (int b = lane; b < nblocks; b += 32) v += scratch[2 * b + k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) scratch[2 * kMaxBlocks + k] = v;
    }
}

// Once per device, with that device current: the device address of the scratch.
lbm_status scratch_of_current_device(double** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return LBM_ERR_INVALID_ARG;
    void* p = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        if (cudaGetSymbolAddress(&p, g_mass_scratch) != cudaSuccess || !p) return LBM_ERR_CUDA;
        g_scratch_ptr[dev].store(p, std::memory_order_release);
    }
    *out = (double*)p;
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_mass_noalloc(const lbm_params* p, const void* d_f, double* mass, void* stream)
{
    if (!p || !d_f || !mass) return LBM_ERR_INVALID_ARG;
    if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D3Q19) return LBM_ERR_INVALID_ARG;
    if (p->ncomp != 1 && p->ncomp != 2) return LBM_ERR_INVALID_ARG;
    if (p->real != LBM_FP32 && p->real != LBM_FP64) return LBM_ERR_INVALID_ARG;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return LBM_ERR_INVALID_ARG;
    const long long N = (long long)p->nx * p->ny * p->nz;
    if (N > LBM_NOALLOC_MAX_NODES) return LBM_ERR_INVALID_ARG;  // scratch holds this many nodes
    const int Q = p->lattice == LBM_D2Q9 ? 9 : 19;
    cudaStream_t st = (cudaStream_t)stream;
    // the copy to host memory and the synchronisation below are not allowed on a stream
    // that is being captured: refuse it before anything is enqueued
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return LBM_ERR_CUDA;
    if (cs != cudaStreamCaptureStatusNone) return LBM_ERR_INVALID_ARG;
    double* scratch = nullptr;
    const lbm_status s = scratch_of_current_device(&scratch);
    if (s != LBM_OK) return s;
    const int nblocks = (int)((N + kNodesPerBlock - 1) / kNodesPerBlock);
    if (p->real == LBM_FP64)
        k_mass_partials<double><<<nblocks, kThreads, 0, st>>>((const double*)d_f, p->ncomp, Q, N, scratch);
    else
        k_mass_partials<float><<<nblocks, kThreads, 0, st>>>((const float*)d_f, p->ncomp, Q, N, scratch);
    k_mass_total<<<1, 32, 0, st>>>(nblocks, scratch);
    double tot[2];
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tot, scratch + 2 * kMaxBlocks, sizeof(tot), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    for (int k = 0; k < p->ncomp; ++k) mass[k] = tot[k];
    return LBM_OK;
}
