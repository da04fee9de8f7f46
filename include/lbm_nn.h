/*
 * Kernels of the warm-start network (a learned initial velocity field for
 * steady-state runs; the paper cites the idea in Section 1, the project builds it as
 * its row f3). The paper defines no network: everything here is the project's own.
 *
 * Conventions:
 *   - Fields are FP32, channel-major [C][D][H][W] (x = W fastest) on a periodic box:
 *     3x3x3 convolutions wrap around, like the lattices they are trained on.
 *   - Weights are [Cout][Cin][27], tap t = 9 (dz + 1) + 3 (dy + 1) + (dx + 1) for the
 *     offset (dz, dy, dx) in {-1, 0, 1}^3, so
 *       y[o][p] = b[o] + sum_{i, t} w[o][i][t] x[i][p + offset(t)].
 *   - All pointers are device pointers of the current device; the caller owns them.
 *     Work is enqueued on `stream` (cudaStream_t as void*); nothing synchronises.
 *   - Returns LBM_ERR_INVALID_ARG for null pointers or non-positive sizes (and for odd
 *     sizes in the 2x pooling / upsampling entry points), LBM_ERR_CUDA if a launch
 *     fails. Reductions use a fixed order, so results are reproducible bit for bit.
 */
#ifndef GB300_LBM_NN_H
#define GB300_LBM_NN_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* y = conv(x, w) + b, then the leaky ReLU (y < 0 -> 0.01 y) if relu; bias may be NULL. */
lbm_status lbm_nn_conv3d(const float* x, int cin, int d, int h, int w, const float* weight,
                         const float* bias, int cout, int relu, float* y, void* stream);

/* gx = d/dx sum(gy * conv(x, w)): the adjoint convolution. wt_scratch: cin*cout*27 floats
 * (the flipped, transposed weights). */
lbm_status lbm_nn_conv3d_grad_input(const float* gy, int cout, int d, int h, int w, const float* weight,
                                    int cin, float* wt_scratch, float* gx, void* stream);

/* gw[o][i][t] (+)= sum_p gy[o][p] x[i][p + offset(t)], gb[o] (+)= sum_p gy[o][p]
 * (accumulate != 0 adds to the existing values; gb may be NULL). The voxels are split
 * into LBM_NN_GW_SEGMENTS segments whose partial sums go to scratch
 * (LBM_NN_GW_SEGMENTS * cout * cin * 28 floats) and are then added in segment order. */
#define LBM_NN_GW_SEGMENTS 64
lbm_status lbm_nn_conv3d_grad_weight(const float* x, int cin, const float* gy, int cout, int d, int h, int w,
                                     float* gw, float* gb, int accumulate, float* scratch, void* stream);

/* y += a x over n values (gradients meeting at a skip connection). */
lbm_status lbm_nn_axpy(float* y, const float* x, long long n, float a, void* stream);

/* g *= (y > 0 ? 1 : 0.01), elementwise over n values (leaky-ReLU backward from its output y). */
lbm_status lbm_nn_relu_grad(const float* y, float* g, long long n, void* stream);

/* 2x2x2 average pooling of x [c][d][h][w] (d, h, w even) into y [c][d/2][h/2][w/2], and
 * its gradient gx from gy. */
lbm_status lbm_nn_avg_pool2(const float* x, int c, int d, int h, int w, float* y, void* stream);
lbm_status lbm_nn_avg_pool2_grad(const float* gy, int c, int d, int h, int w, float* gx, void* stream);

/* nearest 2x upsampling of x [c][d][h][w] into y [c][2d][2h][2w], and its gradient gx
 * [c][d][h][w] from gy (sum of the 8 children). */
lbm_status lbm_nn_up2(const float* x, int c, int d, int h, int w, float* y, void* stream);
lbm_status lbm_nn_up2_grad(const float* gy, int c, int d, int h, int w, float* gx, void* stream);

/* loss = sum (p - t)^2 / sum t^2 over n values, grad = 2 (p - t) / sum t^2.
 * sums: device, 2 doubles (scratch; sums[0] = sum (p-t)^2, sums[1] = sum t^2 on return);
 * loss: device double (may be NULL). */
lbm_status lbm_nn_rel_loss(const float* p, const float* t, long long n, float* grad, double* sums,
                           double* loss, void* stream);

/* Adam step over n parameters: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr (m / c1) / (sqrt(v / c2) + eps), with c1 = 1 - b1^t, c2 = 1 - b2^t. */
lbm_status lbm_nn_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2, void* stream);

/*
 * The three convolution passes on the tcgen05 tensor cores (same arguments and layouts
 * as the FP32 entry points above; the weight gradient splits the voxels into up to
 * LBM_NN_GW_TC_SEGMENTS segments and takes scratch of LBM_NN_GW_TC_SEGMENTS * cout *
 * (27 cin + 1) floats). Each is an implicit GEMM with M = 128
 * voxels (forward, adjoint) or 128 (tap, channel) rows (weight gradient), N = output
 * channels rounded up to 16, and BF16 operands: x, the weights and gy are rounded from
 * FP32 to BF16 (to nearest, ties to even) as they are staged in shared memory, and the
 * products are accumulated in FP32 in tensor memory. Bias, leaky ReLU and the segment
 * sums stay FP32. Limits (LBM_ERR_INVALID_ARG beyond them): d h w < 2^31 - 128 voxels,
 * cout <= 256, and the forward pass needs 54 Np Cp + 512 Cp + 2048 bytes of shared
 * memory <= 227 KB, with Np = cout and Cp = cin rounded up to 16 (for the adjoint, cout
 * and cin swap roles).
 * A wait on the tensor cores that does not end within about 2 s makes the kernel stop,
 * free its tensor memory and set a flag that lbm_nn_tc_error reads.
 */
#define LBM_NN_GW_TC_SEGMENTS 512
lbm_status lbm_nn_conv3d_tc(const float* x, int cin, int d, int h, int w, const float* weight,
                            const float* bias, int cout, int relu, float* y, void* stream);
lbm_status lbm_nn_conv3d_tc_grad_input(const float* gy, int cout, int d, int h, int w, const float* weight,
                                       int cin, float* wt_scratch, float* gx, void* stream);
lbm_status lbm_nn_conv3d_tc_grad_weight(const float* x, int cin, const float* gy, int cout, int d, int h, int w,
                                        float* gw, float* gb, int accumulate, float* scratch, void* stream);

/* *flag = 1 if a tensor-core wait gave up since the last call, else 0; clears the flag.
 * Synchronises the device. */
lbm_status lbm_nn_tc_error(int* flag);

/* Check of the failure detection above (no counterpart in the paper): one GPU thread waits,
 * with the same bounded wait the tensor-core kernels use, on an mbarrier that nothing
 * arrives on, and gives up after limit_cycles SM clock cycles (1 .. 4e9; ~2e6 is about a
 * millisecond at 2 GHz). *completed receives 1 if the wait ended normally (it cannot
 * here), 0 if it gave up; a wait that gives up also sets the flag that lbm_nn_tc_error
 * reads. No tensor memory is allocated and no MMA is in flight. Synchronises the stream;
 * LBM_ERR_INVALID_ARG for a NULL result or a limit out of range. */
lbm_status lbm_nn_wait_selftest(long long limit_cycles, int* completed, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GB300_LBM_NN_H */
