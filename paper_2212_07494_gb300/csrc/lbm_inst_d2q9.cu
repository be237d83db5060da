// Instantiation of the lattice Boltzmann kernels for D2Q9.
#include "lbm_kernels.cuh"

namespace lbm {
const Launchers &launchers_d2q9() { return Dispatch<D2Q9>::table(); }
}  // namespace lbm
