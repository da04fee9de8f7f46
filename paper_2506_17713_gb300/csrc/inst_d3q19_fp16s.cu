// Kernel instantiations for the D3Q19 lattice: FP32 compute, FP16 shifted population
// storage (one translation unit per lattice and type, compiled in parallel).
#include "kernels.cuh"

namespace lbm {
template cudaError_t run<D3Q19, float, __half>(int op, const KArgs<float>& a);
template cudaError_t run_batch<D3Q19, float, __half>(int bop, const KArgs<float>& shape, const BatchItem<float>* items,
                                              int n_items, const BatchLaunch& launch, int parity,
                                              cudaStream_t stream);
}  // namespace lbm
