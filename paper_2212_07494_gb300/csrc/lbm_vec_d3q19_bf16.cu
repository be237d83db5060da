// k_step_vec instantiated for D3Q19 with BF16 storage.
#include "lbm_step_vec.cuh"

namespace lbm {
cudaError_t step_vec_d3q19_bf16(int coll, StepCfg cfg, const KParams &p, const void *fin, void *fout, cudaStream_t s) {
    return VecDispatch<D3Q19, ST_BF16>::step(coll, cfg, p, fin, fout, s);
}
}  // namespace lbm
