// k_step_vec instantiated for D3Q27 with F32 storage.
#include "lbm_step_vec.cuh"

namespace lbm {
cudaError_t step_vec_d3q27_f32(int coll, StepCfg cfg, const KParams &p, const void *fin, void *fout, cudaStream_t s) {
    return VecDispatch<D3Q27, ST_F32>::step(coll, cfg, p, fin, fout, s);
}
}  // namespace lbm
