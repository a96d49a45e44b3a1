// Kernels of the coupled lattice Boltzmann step for storage precision LBPC_FP16S.
#include "lbpc_kernels.cuh"

namespace lbpc {
const Launchers& launchers_f16() { return Impl<LBPC_FP16S>::table(); }
}  // namespace lbpc
