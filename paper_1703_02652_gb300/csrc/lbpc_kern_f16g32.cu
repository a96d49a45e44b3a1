// Kernels of the coupled lattice Boltzmann step for storage mode LBPC_FP16S_G32.
#include "lbpc_kernels.cuh"

namespace lbpc {
const Launchers& launchers_f16g32() { return Impl<LBPC_FP16S_G32>::table(); }
}  // namespace lbpc
