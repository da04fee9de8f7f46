// Kernel instantiations for the D3Q19 lattice in double (one translation unit per
// lattice and type so that the build compiles them in parallel).
#include "kernels.cuh"

namespace lbm {
template cudaError_t run<D3Q19, double, double>(int op, const KArgs<double>& a);
}  // namespace lbm
