// Kernel instantiations for the D2Q9 lattice: FP32 compute, FP16 shifted population
// storage (one translation unit per lattice and type, compiled in parallel).
#include "kernels.cuh"

namespace lbm {
template cudaError_t run<D2Q9, float, __half>(int op, const KArgs<float>& a);
}  // namespace lbm
