// k_step_vec instantiated for D2Q9 with F64 storage.
#include "lbm_step_vec.cuh"

namespace lbm {
cudaError_t step_vec_d2q9_f64(int coll, StepCfg cfg, const KParams &p, const void *fin, void *fout, cudaStream_t s) {
    return VecDispatch<D2Q9, ST_F64>::step(coll, cfg, p, fin, fout, s);
}
}  // namespace lbm
