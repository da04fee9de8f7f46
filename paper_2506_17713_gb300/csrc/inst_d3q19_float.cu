// Kernel instantiations for the D3Q19 lattice in float (one translation unit per
// lattice and type so that the build compiles them in parallel).
#include "kernels.cuh"

namespace lbm {
template cudaError_t run<D3Q19, float, float>(int op, const KArgs<float>& a);
}  // namespace lbm
