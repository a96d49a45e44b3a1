// Kernels of the coupled lattice Boltzmann step for storage precision LBPC_FP64.
#include "lbpc_kernels.cuh"

namespace lbpc {
const Launchers& launchers_f64() { return Impl<LBPC_FP64>::table(); }
}  // namespace lbpc
