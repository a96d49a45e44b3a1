// Kernels of the coupled lattice Boltzmann step for storage mode LBPC_BF16S_G32.
#include "lbpc_kernels.cuh"

namespace lbpc {
const Launchers& launchers_bf16g32() { return Impl<LBPC_BF16S_G32>::table(); }
}  // namespace lbpc
