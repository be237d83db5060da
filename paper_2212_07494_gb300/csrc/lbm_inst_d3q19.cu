// Instantiation of the lattice Boltzmann kernels for D3Q19.
#include "lbm_kernels.cuh"

namespace lbm {
const Launchers &launchers_d3q19() { return Dispatch<D3Q19>::table(); }
}  // namespace lbm
