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

// layout of the snapshot the last call on each device left in the scratch:
// a call with another layout would read those bytes as its own velocities
struct SnapLayout {
    int lattice = -1, storage = -1, nx = 0, ny = 0, nz = 0;
    bool operator==(const SnapLayout &o) const {
        return lattice == o.lattice && storage == o.storage && nx == o.nx && ny == o.ny && nz == o.nz;
    }
};
SnapLayout g_layout[kMaxDevices];

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
lbm_status device_scratch(unsigned char **out, int *dev_out) {
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
    *dev_out = dev;
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
    int dev = -1;
    lbm_status st = device_scratch(&scratch, &dev);
    if (st != LBM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    // a snapshot left by a call with another layout is not this state's
    // velocity: clear the bytes this call reads, so the residual entries
    // then compare with zero, as on the first call
    {
        SnapLayout now;
        now.lattice = d->lattice;
        now.storage = d->storage;
        now.nx = d->nx;
        now.ny = d->ny;
        now.nz = d->nz;
        std::lock_guard<std::mutex> lock(g_mu);
        if (!(g_layout[dev] == now)) {
            cudaError_t e = cudaMemsetAsync(scratch + kSnapOffset, 0, snap, s);
            if (e != cudaSuccess)
                return err(LBM_ERR_CUDA, std::string("snapshot clear: ") + cudaGetErrorString(e));
            g_layout[dev] = now;
        }
    }

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

    if (d->force_kind == LBM_G_UNIFORM) {
        k_noalloc_force<<<1, 1, 0, s>>>((double *)(scratch + kForceOffset),
                                        (float *)(scratch + kForceOffset + 4 * sizeof(double)), d->g[0], d->g[1],
                                        D == 3 ? d->g[2] : 0.0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return err(LBM_ERR_CUDA, std::string("force launch: ") + cudaGetErrorString(e));
    }
    const Launchers &L = d->lattice == LBM_D2Q9 ? launchers_d2q9()
                       : (d->lattice == LBM_D3Q19 ? launchers_d3q19() : launchers_d3q27());
    // the moments launcher caps its grid at kMomGridMax blocks (moments_grid),
    // and the static_assert above keeps that many partial sums below the
    // force region
    int nb = 0;
    cudaError_t e = L.moments(d->storage, false, kp, state_dev, nullptr, nullptr, (double *)scratch,
                              scratch + kSnapOffset, s, &nb);
    if (e == cudaSuccess) e = launch_finalize((const double *)scratch, nb, out_dev, s);
    if (e != cudaSuccess) return err(LBM_ERR_CUDA, std::string("lbm_check_noalloc: ") + cudaGetErrorString(e));
    return LBM_OK;
}
