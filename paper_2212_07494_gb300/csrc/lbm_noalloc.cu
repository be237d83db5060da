// lbm_noalloc.cu -- lbm_check_noalloc: the FP64 check without any device
// allocation, for callers that may not call cudaMalloc (see include/lbm.h).
// Its scratch is the static device array below; host code only ever passes
// the address that cudaGetSymbolAddress returns for the current device.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace lbm;

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // per device
constexpr size_t kForceOffset = 80 * 1024;          // after kMomGridMax * kPartials doubles
constexpr size_t kSnapOffset = 128 * 1024;
constexpr size_t kSnapBytes = kScratchBytes - kSnapOffset;
static_assert((size_t)kMomGridMax * kPartials * sizeof(double) <= kForceOffset, "partials overflow");
constexpr int kMaxDevices = 64;

}  // namespace

// Scratch of lbm_check_noalloc: [0, 80 KiB) per-block partial sums,
// [80 KiB, +64 B) the uniform force (4 doubles, 4 floats), [128 KiB, 16 MiB)
// the velocity snapshot.  In host code this name is only a handle for
// cudaGetSymbolAddress, never a device address.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_mu;
unsigned char *g_dev_ptr[kMaxDevices] = {};

__global__ void k_noalloc_force(double *gd, float *gf, double gx, double gy, double gz) {
    gd[0] = gx;
    gd[1] = gy;
    gd[2] = gz;
    gf[0] = (float)gx;
    gf[1] = (float)gy;
    gf[2] = (float)gz;
}

lbm_status err(lbm_status st, const std::string &m) {
    set_thread_error(m.c_str());
    return st;
}

// once per device, with that device current: resolve the array's device
// address and clear it (the snapshot starts at zero)
lbm_status device_scratch(unsigned char **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(LBM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return err(LBM_ERR_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return err(LBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        e = cudaMemset(p, 0, kScratchBytes);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return err(LBM_ERR_CUDA, std::string("scratch clear: ") + cudaGetErrorString(e));
        g_dev_ptr[dev] = (unsigned char *)p;
    }
    *out = g_dev_ptr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_check_noalloc(const lbm_desc *d, const void *state_dev, double *out_dev, void *stream) {
    if (!d || !state_dev || !out_dev) return err(LBM_ERR_ARG, "lbm_check_noalloc: NULL argument");
    if (d->lattice < LBM_D2Q9 || d->lattice > LBM_D3Q27) return err(LBM_ERR_ARG, "bad lattice");
    if (d->storage < LBM_F64 || d->storage > LBM_BF16_SHIFT) return err(LBM_ERR_ARG, "bad storage");
    const int D = d->lattice == LBM_D2Q9 ? 2 : 3;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || (D == 2 && d->nz != 1) || d->ny > 65535 || d->nz > 65535)
        return err(LBM_ERR_ARG, "bad sizes");
    if (d->solid) return err(LBM_ERR_ARG, "lbm_check_noalloc: solid masks are not supported (use lbm_check_device)");
    if (d->force_kind != LBM_G_NONE && d->force_kind != LBM_G_UNIFORM)
        return err(LBM_ERR_ARG, "lbm_check_noalloc: only LBM_G_NONE and LBM_G_UNIFORM forces are supported");
    if (d->force_kind == LBM_G_UNIFORM && !d->g) return err(LBM_ERR_ARG, "uniform force values are NULL");
    const size_t N = (size_t)d->nx * d->ny * d->nz;
    const size_t snap = (size_t)D * N * (d->storage == LBM_F64 ? 8 : 4);
    if (snap > kSnapBytes)
        return err(LBM_ERR_ARG, "lbm_check_noalloc: the velocity snapshot needs " + std::to_string(snap) +
                                    " bytes, more than the " + std::to_string(kSnapBytes) +
                                    " bytes of static scratch; use lbm_check_device");

    unsigned char *scratch = nullptr;
    lbm_status st = device_scratch(&scratch);
    if (st != LBM_OK) return st;

    KParams kp{};
    kp.nx = d->nx;
    kp.ny = d->ny;
    kp.nz = d->nz;
    kp.nxp = (d->nx + 31) / 32 * 32;
    kp.plane = (long long)kp.nxp * d->ny * d->nz;
    for (int k = 0; k < 3; ++k) kp.per[k] = d->periodic[k] ? 1 : 0;
    kp.force_kind = d->force_kind;
    kp.g = (const double *)(scratch + kForceOffset);
    kp.g32 = (const float *)(scratch + kForceOffset + 4 * sizeof(double));
    kp.solid = nullptr;
    if (d->lattice == LBM_D2Q9) fill_offsets<D2Q9>(kp);
    else if (d->lattice == LBM_D3Q19) fill_offsets<D3Q19>(kp);
    else fill_offsets<D3Q27>(kp);

    cudaStream_t s = (cudaStream_t)stream;
    if (d->force_kind == LBM_G_UNIFORM) {
        k_noalloc_force<<<1, 1, 0, s>>>((double *)(scratch + kForceOffset),
                                        (float *)(scratch + kForceOffset + 4 * sizeof(double)), d->g[0], d->g[1],
                                        D == 3 ? d->g[2] : 0.0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return err(LBM_ERR_CUDA, std::string("force launch: ") + cudaGetErrorString(e));
    }
    const Launchers &L = d->lattice == LBM_D2Q9 ? launchers_d2q9()
                       : (d->lattice == LBM_D3Q19 ? launchers_d3q19() : launchers_d3q27());
    int nb = 0;
    cudaError_t e = L.moments(d->storage, false, kp, state_dev, nullptr, nullptr, (double *)scratch,
                              scratch + kSnapOffset, s, &nb);
    if (e == cudaSuccess && nb > kMomGridMax) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) e = launch_finalize((const double *)scratch, nb, out_dev, s);
    if (e != cudaSuccess) return err(LBM_ERR_CUDA, std::string("lbm_check_noalloc: ") + cudaGetErrorString(e));
    return LBM_OK;
}
