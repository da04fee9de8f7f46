// Kernel instantiations for the D2Q9 lattice: FP32 compute, BF16 shifted population
// storage (one translation unit per lattice and type, compiled in parallel).
#include "kernels.cuh"

namespace lbm {
template cudaError_t run<D2Q9, float, __nv_bfloat16>(int op, const KArgs<float>& a);
template cudaError_t run_batch<D2Q9, float, __nv_bfloat16>(int bop, const KArgs<float>& shape, const BatchItem<float>* items,
                                              int n_items, const BatchLaunch& launch, int parity,
                                              cudaStream_t stream);
}  // namespace lbm
