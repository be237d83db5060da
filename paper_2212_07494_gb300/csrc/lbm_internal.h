// lbm_internal.h -- interface between the C ABI runtime and the
// per-lattice kernel launchers, and the collision dispatch that every step
// kernel shares (collide_any, collide_one).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "lbm_device.cuh"
#include "lbm_f32x2.cuh"

namespace lbm {

// the collision selected by COLL on one node's grid G (or two nodes' with F2)
template <int L, int COLL, typename R>
__device__ __forceinline__ void collide_any(R *G, R gx, R gy, R gz, R om2, R om3, R om4, R omb) {
    if constexpr (COLL == SMRT) collide_smrt<L>(G, gx, gy, gz, om2, om3, om4, omb);
    else if constexpr (COLL == SMRT_TRIM) collide_smrt_trim<L>(G, gx, gy, gz, om2);
    else if constexpr (COLL == SMRT_FNEQ) collide_smrt_fneq<L>(G, gx, gy, gz, om2, om3, om4, omb);
    else if constexpr (COLL == MRT_RAW) collide_mrt_raw<L>(G, gx, gy, gz, om2, om3, om4);
    else collide_bgk<L>(G, gx, gy, gz, om2);
}

// One node's collision.  In FP32 the node runs through the pair type with
// its values in both lanes (lbm_f32x2.cuh) and keeps the first: the same
// template instantiation and the same instructions as two paired nodes, so
// a node's result does not depend on whether the launch shape collides it
// alone or paired.  FP64 as written.
template <int L, int COLL, typename R>
__device__ __forceinline__ void collide_one(R *G, R gx, R gy, R gz, R om2, R om3, R om4, R omb) {
    if constexpr (sizeof(R) == 4) {
        constexpr int NG = Grid<Lat<L>::D>::N;
        F2 H[NG];
#pragma unroll
        for (int g = 0; g < NG; ++g) H[g] = F2(G[g]);
        collide_any<L, COLL>(H, F2(gx), F2(gy), F2(gz), F2(om2), F2(om3), F2(om4), F2(omb));
#pragma unroll
        for (int g = 0; g < NG; ++g) G[g] = H[g].lo();
    } else {
        collide_any<L, COLL>(G, gx, gy, gz, om2, om3, om4, omb);
    }
}

// number of doubles each moments block writes to the partial-sum scratch:
// {sum (rho - 1), Px, Py, Pz, residual numerator, residual denominator,
//  non-finite count, fluid-node count}
constexpr int kPartials = 8;
constexpr int kMomBlock = 128;
constexpr int kMomNpt = 2;          // nodes per thread per work item
constexpr int kMomGridMax = 1216;   // 8 blocks per SM on 152 SMs: one wave

struct StepCfg {
    int bdx;  // threads per block along x
    int npt;  // nodes per thread: strided by bdx (vec = 0), or consecutive (vec = 1)
    int vec;  // 1: k_step_vec, each population of a thread's npt nodes moved as one vector
};

// vector widths (nodes per thread) k_step_vec is built for, per lattice and
// storage: D2Q9 moves 16 bytes per population and thread at the upper width;
// the 3-D lattices, with 19 or 27 populations in registers, 4 or 8 bytes
__host__ __device__ constexpr int vec_width_lo(int L, int ST) {
    return L == D2Q9 ? (ST == ST_F64 ? 1 : (ST == ST_F32 ? 2 : 4)) : (ST == ST_F64 || ST == ST_F32 ? 1 : 2);
}
__host__ __device__ constexpr int vec_width_hi(int L, int ST) {
    return L == D2Q9 ? (ST == ST_F64 ? 2 : (ST == ST_F32 ? 4 : 8)) : (ST == ST_F64 ? 1 : (ST == ST_F32 ? 2 : 4));
}

// k_step_vec launcher of one lattice and storage (collision and width from
// the arguments); cudaErrorInvalidValue for a width it is not built for
typedef cudaError_t (*StepVecFn)(int coll, StepCfg cfg, const KParams &p, const void *fin, void *fout,
                                 cudaStream_t s);
cudaError_t step_vec_d2q9_f64(int, StepCfg, const KParams &, const void *, void *, cudaStream_t);
cudaError_t step_vec_d2q9_f32(int, StepCfg, const KParams &, const void *, void *, cudaStream_t);
cudaError_t step_vec_d2q9_f16(int, StepCfg, const KParams &, const void *, void *, cudaStream_t);
cudaError_t step_vec_d2q9_bf16(int, StepCfg, const KParams &, const void *, void *, cudaStream_t);
cudaError_t step_vec_d3q19_f64(int, StepCfg, const KParams &, const void *, void *, cudaStream_t);
cudaError_t step_vec_d3q19_f32(int, StepCfg, const KParams &, const void *, void *, cudaStream_t);
cudaError_t step_vec_d3q19_f16(int, StepCfg, const KParams &, const void *, void *, cudaStream_t);
cudaError_t step_vec_d3q19_bf16(int, StepCfg, const KParams &, const void *, void *, cudaStream_t);
cudaError_t step_vec_d3q27_f64(int, StepCfg, const KParams &, const void *, void *, cudaStream_t);
cudaError_t step_vec_d3q27_f32(int, StepCfg, const KParams &, const void *, void *, cudaStream_t);
cudaError_t step_vec_d3q27_f16(int, StepCfg, const KParams &, const void *, void *, cudaStream_t);
cudaError_t step_vec_d3q27_bf16(int, StepCfg, const KParams &, const void *, void *, cudaStream_t);

inline StepVecFn step_vec_fn(int lattice, int storage) {
    static const StepVecFn t[3][4] = {
        {step_vec_d2q9_f64, step_vec_d2q9_f32, step_vec_d2q9_f16, step_vec_d2q9_bf16},
        {step_vec_d3q19_f64, step_vec_d3q19_f32, step_vec_d3q19_f16, step_vec_d3q19_bf16},
        {step_vec_d3q27_f64, step_vec_d3q27_f32, step_vec_d3q27_f16, step_vec_d3q27_bf16}};
    return t[lattice][storage];
}

struct Launchers {
    cudaError_t (*step)(int coll, int st, bool mask, StepCfg cfg, const KParams &p, const void *fin,
                        void *fout, cudaStream_t s);
    // rho/u (unpadded FP64, nullable), partials [nblocks * kPartials];
    // uprev (unpadded D planes of the arithmetic type, nullable): residual
    // against it, then updated
    cudaError_t (*moments)(int st, bool mask, const KParams &p, const void *f, double *rho, double *u,
                           double *partials, void *uprev, cudaStream_t s, int *nblocks);
    cudaError_t (*init)(int coll, int st, bool mask, const KParams &p, const double *rho0,
                        const double *u0, void *target, cudaStream_t s);
    cudaError_t (*unstream)(int st, bool mask, const KParams &p, const void *target, void *state,
                            cudaStream_t s);
    cudaError_t (*get_pops)(int st, bool mask, const KParams &p, const void *state, double *out,
                            cudaStream_t s);
    cudaError_t (*put_pops)(int st, const KParams &p, const double *in, void *target, cudaStream_t s);
};

const Launchers &launchers_d2q9();
const Launchers &launchers_d3q19();
const Launchers &launchers_d3q27();

cudaError_t launch_finalize(const double *partials, int nblocks, double *out, cudaStream_t s);

// record a message for lbm_last_error(NULL) (thread-local)
void set_thread_error(const char *msg);

inline int moments_grid(const KParams &p, int resident) {
    const long long items = (long long)((p.nx + kMomBlock * kMomNpt - 1) / (kMomBlock * kMomNpt)) *
                            (p.ny - (p.halo_ax == 1 ? 2 : 0)) * (p.nz - (p.halo_ax == 2 ? 2 : 0));
    long long g = items < kMomGridMax ? items : kMomGridMax;
    if (resident > 0 && g > resident) g = resident;
    return (int)g;
}

// totals out[0..6] = {M, Px, Py, Pz, residual num, residual den, non-finite}
// from per-block partials in a fixed order
inline dim3 node_grid(const KParams &p, int bdx, int npt) {
    return dim3((unsigned)((p.nx + bdx * npt - 1) / (bdx * npt)), (unsigned)p.ny, (unsigned)p.nz);
}
// the step kernels' grid: the layers they update (a slab's halo layers excluded)
inline dim3 step_grid(const KParams &p, int bdx, int npt) {
    return dim3((unsigned)((p.nx + bdx * npt - 1) / (bdx * npt)), (unsigned)(p.ny - (p.halo_ax == 1 ? 2 : 0)),
                (unsigned)(p.nz - (p.halo_ax == 2 ? 2 : 0)));
}

}  // namespace lbm
