// Kernels of the coupled lattice Boltzmann step for storage precision LBPC_FP32.
#include "lbpc_kernels.cuh"

namespace lbpc {
const Launchers& launchers_f32() { return Impl<LBPC_FP32>::table(); }
}  // namespace lbpc
