// Instantiation of the lattice Boltzmann kernels for D3Q27.
#include "lbm_kernels.cuh"

namespace lbm {
const Launchers &launchers_d3q27() { return Dispatch<D3Q27>::table(); }
}  // namespace lbm
