// Kernels of the coupled lattice Boltzmann step for storage precision LBPC_BF16S.
#include "lbpc_kernels.cuh"

namespace lbpc {
const Launchers& launchers_bf16() { return Impl<LBPC_BF16S>::table(); }
}  // namespace lbpc
