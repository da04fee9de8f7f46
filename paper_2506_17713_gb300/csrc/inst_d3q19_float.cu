// Kernel instantiations for the D3Q19 lattice in float (one translation unit per
// lattice and type so that the build compiles them in parallel).
#include "kernels.cuh"

namespace lbm {
template cudaError_t run<D3Q19, float, float>(int op, const KArgs<float>& a);
template cudaError_t run_batch<D3Q19, float, float>(int bop, const KArgs<float>& shape, const BatchItem<float>* items,
                                              int n_items, const BatchLaunch& launch, int parity,
                                              cudaStream_t stream);
}  // namespace lbm
