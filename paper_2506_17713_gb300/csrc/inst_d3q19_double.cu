// Kernel instantiations for the D3Q19 lattice in double (one translation unit per
// lattice and type so that the build compiles them in parallel).
#include "kernels.cuh"

namespace lbm {
template cudaError_t run<D3Q19, double, double>(int op, const KArgs<double>& a);
template cudaError_t run_batch<D3Q19, double, double>(int bop, const KArgs<double>& shape, const BatchItem<double>* items,
                                              int n_items, const BatchLaunch& launch, int parity,
                                              cudaStream_t stream);
}  // namespace lbm
