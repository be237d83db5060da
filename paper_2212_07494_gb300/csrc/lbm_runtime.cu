// lbm_runtime.cu -- the C ABI (include/lbm.h): handle, buffers, stream and
// CUDA-graph management, FP64 reductions and error reporting around the
// fused stream-collide kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace lbm;

namespace {

thread_local std::string g_thread_err;

int lattice_D(int lat) { return lat == LBM_D2Q9 ? 2 : 3; }
int lattice_Q(int lat) { return lat == LBM_D2Q9 ? 9 : (lat == LBM_D3Q19 ? 19 : 27); }
size_t storage_bytes(int st) { return st == LBM_F64 ? 8 : (st == LBM_F32 ? 4 : 2); }
size_t arith_bytes(int st) { return st == LBM_F64 ? 8 : 4; }

// 2^(p+1) max|g|, p the significand bits of the storage format (see
// lbm_force_resolution)
double stall_speed(int st, double gmax) {
    const int p = st == LBM_F64 ? 53 : (st == LBM_F32 ? 24 : (st == LBM_F16_SHIFT ? 11 : 8));
    return gmax > 0.0 ? std::ldexp(gmax, p + 1) : INFINITY;
}

const Launchers &launchers_for(int lat) {
    return lat == LBM_D2Q9 ? launchers_d2q9() : (lat == LBM_D3Q19 ? launchers_d3q19() : launchers_d3q27());
}

}  // namespace

// finalize: one block sums the per-block partials in a fixed order
namespace lbm {
__global__ void k_finalize(const double *__restrict__ partials, int nblocks, double *__restrict__ out) {
    __shared__ double sh[256][kPartials];
    double v[kPartials];
#pragma unroll
    for (int k = 0; k < kPartials; ++k) v[k] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < kPartials; ++k) v[k] += partials[(long long)b * kPartials + k];
#pragma unroll
    for (int k = 0; k < kPartials; ++k) sh[threadIdx.x][k] = v[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < kPartials; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + s][k];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sh[0][7] + sh[0][0];  // M = fluid nodes + sum (rho - 1)
#pragma unroll
        for (int k = 1; k < 7; ++k) out[k] = sh[0][k];
    }
}

// Force schedules.  The step kernels read the force buffers as always; after
// each step k_sched_apply writes the force of the next step into them, from
// the schedule's entry (*t + off): a uniform g (table of 3 per step), or the
// saved base force times a factor (table of 1 per step), over `count` values
// of the device layout.  The tables hold period + 64 entries, entry i being
// the schedule's entry i mod period, and *t < period, off <= 64, so no modulo
// is taken on the device.  k_sched_advance moves the counter on (one
// thread) and keeps it below the period.
__global__ void k_sched_advance(long long *t, long long n, long long period) { *t = (*t + n) % period; }

__global__ void k_sched_apply(const double *table, const long long *t, int off, int scale, const double *base,
                              long long count, double *g, float *g32) {
    const long long idx = *t + off;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (!scale) {
        if (i < 3) {
            g[i] = table[3 * idx + i];
            g32[i] = (float)table[3 * idx + i];
        }
        return;
    }
    if (i < count) {
        const double v = table[idx] * base[i];
        g[i] = v;
        g32[i] = (float)v;
    }
}

cudaError_t launch_finalize(const double *partials, int nblocks, double *out, cudaStream_t s) {
    k_finalize<<<1, 256, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

void set_thread_error(const char *msg) { g_thread_err = msg; }
}  // namespace lbm

struct lbm_handle {
    int lattice = 0, collision = 0, storage = 0;
    int D = 2, Q = 9;
    int nx = 0, ny = 0, nz = 0;
    int force_kind = 0;
    bool mask = false;
    KParams kp{};
    StepCfg cfg{128, 1, 0};
    size_t state_bytes = 0;   // one population buffer
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;              // buffer holding the state
    double *g_dev = nullptr;
    size_t g_count = 0;       // doubles in the host layout of g
    unsigned char *solid_dev = nullptr;
    double *partials = nullptr;
    int max_blocks = 0;
    double *red_dev = nullptr;   // 8 doubles: M, Px, Py, Pz, res num, res den, non-finite
    void *uprev = nullptr;       // D * N values of the arithmetic type: u at the last check
    float *g32_dev = nullptr;    // FP32 copy of the force
    int64_t uprev_step = -1;
    double *fields = nullptr;    // (1 + D) * N doubles for lbm_moments
    double gmax = 0.0;           // largest |g| component of the constant force (lbm_force_resolution)
    double gmax_sched = 0.0;     // the same over a force schedule, while one is set
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // graph_steps steps starting from buf[0] / buf[1]
    double *gs_dev = nullptr;    // force schedule [period + 64][3] or scale schedule [period + 64]
    double *gbase_dev = nullptr; // the force a scale schedule multiplies (device layout of g_dev)
    size_t gdev_count = 0;       // doubles of g_dev
    bool gs_scale = false;       // gs_dev holds a scale schedule
    long long *gs_t_dev = nullptr;
    int64_t gs_period = 0;
    int graph_steps = 0;
    int64_t step = 0;
    void *(*alloc)(size_t, void *) = nullptr;
    void (*free_)(void *, void *) = nullptr;
    void *alloc_ctx = nullptr;
    std::string err;

    size_t N() const { return (size_t)nx * ny * nz; }
};

namespace {

lbm_status fail(lbm_handle *h, lbm_status st, const std::string &msg) {
    if (h) h->err = msg;
    else g_thread_err = msg;
    return st;
}

lbm_status cuda_fail(lbm_handle *h, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, m);
}

#define LBM_CUDA(h, call)                                          \
    do {                                                           \
        cudaError_t e__ = (call);                                  \
        if (e__ != cudaSuccess) return cuda_fail((h), e__, #call); \
    } while (0)

void *dev_alloc(lbm_handle *h, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (h->alloc) return h->alloc(bytes, h->alloc_ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(lbm_handle *h, void *p) {
    if (!p) return;
    if (h->free_) h->free_(p, h->alloc_ctx);
    else cudaFree(p);
}

template <typename T>
lbm_status alloc_into(lbm_handle *h, T **out, size_t bytes, const char *what) {
    *out = (T *)dev_alloc(h, bytes);
    if (!*out) return fail(h, LBM_ERR_OOM, std::string("device allocation failed: ") + what);
    return LBM_OK;
}

size_t g_count_for(const lbm_handle *h) {
    switch (h->force_kind) {
    case LBM_G_UNIFORM: return (size_t)h->D;
    case LBM_G_ROWS: return (size_t)h->ny * h->D;
    case LBM_G_FIELD: return (size_t)h->D * h->N();
    default: return 0;
    }
}

// device layout of g: uniform [3], rows [ny][D], field [D][plane] (padded rows)
lbm_status upload_force(lbm_handle *h, const double *g) {
    if (h->force_kind == LBM_G_NONE) return LBM_OK;
    if (!g) return fail(h, LBM_ERR_ARG, "force array is NULL");
    std::vector<double> tmp;
    if (h->force_kind == LBM_G_UNIFORM) {
        tmp.assign(3, 0.0);
        for (int a = 0; a < h->D; ++a) tmp[a] = g[a];
    } else if (h->force_kind == LBM_G_ROWS) {
        tmp.assign(g, g + (size_t)h->ny * h->D);
    } else {
        const size_t plane = (size_t)h->kp.plane;
        tmp.assign((size_t)h->D * plane, 0.0);
        for (int a = 0; a < h->D; ++a)
            for (size_t zy = 0; zy < (size_t)h->ny * h->nz; ++zy)
                std::memcpy(&tmp[a * plane + zy * h->kp.nxp], &g[a * h->N() + zy * h->nx],
                            sizeof(double) * h->nx);
    }
    double gmax = 0.0;
    for (double v : tmp) {
        if (!std::isfinite(v)) return fail(h, LBM_ERR_ARG, "force contains a non-finite value");
        gmax = std::max(gmax, std::fabs(v));
    }
    h->gmax = gmax;
    std::vector<float> tmp32(tmp.begin(), tmp.end());
    LBM_CUDA(h, cudaMemcpyAsync(h->g_dev, tmp.data(), tmp.size() * sizeof(double), cudaMemcpyHostToDevice,
                                h->stream));
    LBM_CUDA(h, cudaMemcpyAsync(h->g32_dev, tmp32.data(), tmp32.size() * sizeof(float), cudaMemcpyHostToDevice,
                                h->stream));
    // the staging vector dies on return: wait for the copy
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status sched_apply(lbm_handle *h, int off) {
    const long long count = h->gs_scale ? (long long)h->gdev_count : 3;
    k_sched_apply<<<(unsigned)((count + 255) / 256), 256, 0, h->stream>>>(
        h->gs_dev, h->gs_t_dev, off, h->gs_scale ? 1 : 0, h->gbase_dev, count, h->g_dev, h->g32_dev);
    LBM_CUDA(h, cudaGetLastError());
    return LBM_OK;
}

// k_step_vec takes 32-bit element offsets and no obstacle mask
bool vec_ok(const lbm_handle *h) { return !h->mask && (long long)h->Q * h->kp.plane < (1LL << 32); }

// one step from fin to fout with launch shape c
cudaError_t launch_step(lbm_handle *h, StepCfg c, const void *fin, void *fout) {
    if (c.vec) return step_vec_fn(h->lattice, h->storage)(h->collision, c, h->kp, fin, fout, h->stream);
    return launchers_for(h->lattice).step(h->collision, h->storage, h->mask, c, h->kp, fin, fout, h->stream);
}

// launch shape check: strided 1 or 2 nodes, or a vector width built for
// this lattice and storage
bool shape_ok(const lbm_handle *h, StepCfg c) {
    if (!(c.bdx == 32 || c.bdx == 64 || c.bdx == 128 || c.bdx == 256)) return false;
    if (!c.vec) return c.npt == 1 || c.npt == 2;
    if (!vec_ok(h)) return false;
    return c.npt == vec_width_lo(h->lattice, h->storage) || c.npt == vec_width_hi(h->lattice, h->storage);
}

lbm_status launch_steps(lbm_handle *h, int64_t n) {
    int since = 0;   // with a force schedule: steps since the counter last advanced (< 64)
    for (int64_t s = 0; s < n; ++s) {
        cudaError_t e = launch_step(h, h->cfg, h->buf[h->cur], h->buf[1 - h->cur]);
        if (e != cudaSuccess) return cuda_fail(h, e, "stream-collide launch");
        h->cur = 1 - h->cur;
        if (h->gs_dev) {
            // the force of the next step
            lbm_status st = sched_apply(h, since + 1);
            if (st != LBM_OK) return st;
        }
        if (h->gs_dev && ++since == 64) {
            k_sched_advance<<<1, 1, 0, h->stream>>>(h->gs_t_dev, 64LL, (long long)h->gs_period);
            LBM_CUDA(h, cudaGetLastError());
            since = 0;
        }
    }
    if (h->gs_dev && since > 0) {
        k_sched_advance<<<1, 1, 0, h->stream>>>(h->gs_t_dev, (long long)since, (long long)h->gs_period);
        LBM_CUDA(h, cudaGetLastError());
    }
    return LBM_OK;
}

// graphs bake kernel parameters: drop them when those change
void drop_graphs(lbm_handle *h) {
    for (cudaGraphExec_t &ge : h->graph)
        if (ge) {
            cudaGraphExecDestroy(ge);
            ge = nullptr;
        }
}

// drop a schedule; the force it replaced goes back into the force buffers
// (the force set last by lbm_set_force or at creation applies again).  The
// copies run on the handle's stream, which need not synchronise with the
// legacy default stream, and are waited for before the buffers are freed.
void free_schedule(lbm_handle *h) {
    if (h->gbase_dev) {
        const size_t n = h->gdev_count;
        std::vector<double> base(n);
        cudaError_t e = cudaMemcpyAsync(h->g_dev, h->gbase_dev, n * sizeof(double), cudaMemcpyDeviceToDevice,
                                        h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base.data(), h->gbase_dev, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess) {
            std::vector<float> base32(base.begin(), base.end());
            e = cudaMemcpyAsync(h->g32_dev, base32.data(), n * sizeof(float), cudaMemcpyHostToDevice, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        }
        cudaGetLastError();
    }
    dev_free(h, h->gs_dev);
    dev_free(h, h->gbase_dev);
    dev_free(h, h->gs_t_dev);
    h->gs_dev = nullptr;
    h->gbase_dev = nullptr;
    h->gs_t_dev = nullptr;
    h->gs_period = 0;
    h->gs_scale = false;
}

// the graph of graph_steps steps that starts from the buffer holding the
// state now (a graph has its buffers baked in; after an odd number of single
// steps the state lives in the other buffer, so each parity has its graph)
lbm_status ensure_graph(lbm_handle *h) {
    if (h->graph[h->cur]) return LBM_OK;
    const int steps = h->graph_steps;
    const int saved = h->cur;
    cudaGraph_t g = nullptr;
    LBM_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    lbm_status st = launch_steps(h, steps);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    h->cur = saved;  // capture does not execute; steps is even anyway
    if (st != LBM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->graph[saved], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->graph[saved] = nullptr;
        return cuda_fail(h, e, "cudaGraphInstantiate");
    }
    return LBM_OK;
}

// rho/u into device pointers (nullable), partial sums, finalize into `out`
// (default: red_dev)
lbm_status run_moments(lbm_handle *h, double *rho, double *u, void *uprev, double *out = nullptr) {
    const Launchers &L = launchers_for(h->lattice);
    int nb = 0;
    cudaError_t e = L.moments(h->storage, h->mask, h->kp, h->buf[h->cur], rho, u, h->partials, uprev,
                              h->stream, &nb);
    if (e != cudaSuccess) return cuda_fail(h, e, "moments launch");
    if (nb > h->max_blocks) return fail(h, LBM_ERR_STATE, "partial-sum scratch too small");
    e = launch_finalize(h->partials, nb, out ? out : h->red_dev, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "finalize launch");
    return LBM_OK;
}

// upload a schedule of `width` doubles per step (3: a uniform force, 1: a
// scale) and arm it from the next step on
lbm_status set_schedule(lbm_handle *h, const std::vector<double> &table, int64_t period, bool scale) {
    // in-flight steps may still read the old schedule
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    free_schedule(h);
    if (period == 0) return LBM_OK;
    double m = 0.0;
    for (double v : table) m = std::max(m, std::fabs(v));
    h->gmax_sched = scale ? m * h->gmax : m;
    // extended by 64 wrapped entries: the kernels index it at counter + offset
    const size_t width = scale ? 1 : 3;
    std::vector<double> tmp(width * (size_t)(period + 64));
    for (int64_t i = 0; i < period + 64; ++i)
        for (size_t a = 0; a < width; ++a) tmp[(size_t)i * width + a] = table[(size_t)(i % period) * width + a];
    lbm_status st = alloc_into(h, &h->gs_dev, tmp.size() * sizeof(double), "force schedule");
    if (st == LBM_OK) st = alloc_into(h, &h->gs_t_dev, sizeof(long long), "force schedule counter");
    if (st == LBM_OK) st = alloc_into(h, &h->gbase_dev, h->gdev_count * sizeof(double), "force schedule base");
    if (st != LBM_OK) {
        free_schedule(h);
        return st;
    }
    // the base force first: free_schedule restores the force buffers from it
    cudaError_t e = cudaMemcpyAsync(h->gbase_dev, h->g_dev, h->gdev_count * sizeof(double),
                                    cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) {
        dev_free(h, h->gbase_dev);
        h->gbase_dev = nullptr;
        free_schedule(h);
        return cuda_fail(h, e, "force schedule upload");
    }
    e = cudaMemcpyAsync(h->gs_dev, tmp.data(), tmp.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->gs_t_dev, 0, sizeof(long long), h->stream);
    if (e != cudaSuccess) {
        free_schedule(h);
        return cuda_fail(h, e, "force schedule upload");
    }
    h->gs_period = period;
    h->gs_scale = scale;
    // the force of the first step
    if ((st = sched_apply(h, 0)) != LBM_OK) {
        free_schedule(h);
        return st;
    }
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

}  // namespace

// Library-internal entry points of the batch handoff: a handle created for
// one channel of a batched run takes over that channel's state and residual
// snapshot at a step boundary, and gives its state back at the end.  The
// batch stores a D2Q9 channel exactly as a handle does ([Q][ny][nxp],
// nxp = 32 ceil(nx / 32), deviations; snapshot [D][nx * ny] of the arithmetic
// type), so both copies are plain device-to-device copies on the handle's
// stream.
namespace lbm {

lbm_status handle_adopt(lbm_handle *h, const void *state_dev, const void *snap_dev, int64_t step,
                        int64_t snap_step) {
    const size_t sb = (size_t)h->D * h->N() * arith_bytes(h->storage);
    if (!h->uprev) {
        lbm_status st = alloc_into(h, &h->uprev, sb, "residual velocity");
        if (st != LBM_OK) return st;
    }
    LBM_CUDA(h, cudaMemcpyAsync(h->buf[h->cur], state_dev, h->state_bytes, cudaMemcpyDeviceToDevice, h->stream));
    LBM_CUDA(h, cudaMemcpyAsync(h->uprev, snap_dev, sb, cudaMemcpyDeviceToDevice, h->stream));
    h->step = step;
    h->uprev_step = snap_step;
    return LBM_OK;
}

lbm_status handle_export_state(lbm_handle *h, void *state_dev) {
    LBM_CUDA(h, cudaMemcpyAsync(state_dev, h->buf[h->cur], h->state_bytes, cudaMemcpyDeviceToDevice, h->stream));
    return LBM_OK;
}

cudaStream_t handle_stream(const lbm_handle *h) { return h->stream; }

// Library-internal entry points of split domains (lbm_split.cu): a handle
// created for one slab of a domain split along its outermost axis becomes a
// slab (halo layers at both ends of that axis, see KParams), and the split
// reaches its two population buffers and which of them holds the state.
lbm_status handle_make_slab(lbm_handle *h, int ax, int g0, int gn) {
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    h->kp.halo_ax = ax;
    h->kp.hg0 = g0;
    h->kp.hgn = gn;
    drop_graphs(h);
    return LBM_OK;
}

void handle_buffers(const lbm_handle *h, void **b0, void **b1, int *cur, size_t *bytes) {
    *b0 = h->buf[0];
    *b1 = h->buf[1];
    *cur = h->cur;
    *bytes = h->state_bytes;
}

}  // namespace lbm

extern "C" {

const char *lbm_last_error(const lbm_handle *h) { return h ? h->err.c_str() : g_thread_err.c_str(); }

void lbm_destroy(lbm_handle *h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (cudaGraphExec_t &ge : h->graph)
        if (ge) cudaGraphExecDestroy(ge);
    dev_free(h, h->buf[0]);
    dev_free(h, h->buf[1]);
    dev_free(h, h->g_dev);
    dev_free(h, h->g32_dev);
    dev_free(h, h->solid_dev);
    dev_free(h, h->partials);
    dev_free(h, h->red_dev);
    dev_free(h, h->uprev);
    dev_free(h, h->fields);
    dev_free(h, h->gs_dev);
    dev_free(h, h->gbase_dev);
    dev_free(h, h->gs_t_dev);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

lbm_status lbm_create(const lbm_desc *d, lbm_handle **out) {
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!d) return fail(nullptr, LBM_ERR_ARG, "desc is NULL");
    if (d->lattice < LBM_D2Q9 || d->lattice > LBM_D3Q27) return fail(nullptr, LBM_ERR_ARG, "bad lattice");
    if (d->collision < LBM_BGK || d->collision > LBM_MRT_RAW)
        return fail(nullptr, LBM_ERR_ARG, "bad collision");
    if (d->storage < LBM_F64 || d->storage > LBM_BF16_SHIFT) return fail(nullptr, LBM_ERR_ARG, "bad storage");
    if (d->force_kind < LBM_G_NONE || d->force_kind > LBM_G_FIELD) return fail(nullptr, LBM_ERR_ARG, "bad force kind");
    const int D = lattice_D(d->lattice), Q = lattice_Q(d->lattice);
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return fail(nullptr, LBM_ERR_ARG, "sizes must be >= 1");
    if (D == 2 && d->nz != 1) return fail(nullptr, LBM_ERR_ARG, "nz must be 1 for D2Q9");
    if (d->ny > 65535 || d->nz > 65535) return fail(nullptr, LBM_ERR_ARG, "ny and nz must be <= 65535");
    if (d->collision == LBM_BGK && !(d->tau[2] > 0.5)) return fail(nullptr, LBM_ERR_ARG, "tau[2] must be > 1/2");
    if (d->collision != LBM_BGK)
        for (int n = 2; n <= 4; ++n)
            if (!(d->tau[n] > 0.5)) return fail(nullptr, LBM_ERR_ARG, "tau[2..4] must be > 1/2");
    if (d->tau_bulk != 0.0) {
        if (!(d->tau_bulk > 0.5)) return fail(nullptr, LBM_ERR_ARG, "tau_bulk must be 0 or > 1/2");
        if (d->tau_bulk != d->tau[2] && d->collision != LBM_SMRT && d->collision != LBM_SMRT_FNEQ)
            return fail(nullptr, LBM_ERR_ARG, "tau_bulk applies to the SMRT collisions only");
    }
    if ((d->alloc == nullptr) != (d->free_ == nullptr))
        return fail(nullptr, LBM_ERR_ARG, "alloc and free_ must be given together");

    lbm_handle *h = new (std::nothrow) lbm_handle();
    if (!h) return fail(nullptr, LBM_ERR_OOM, "host allocation failed");
    h->lattice = d->lattice;
    h->collision = d->collision;
    h->storage = d->storage;
    h->D = D;
    h->Q = Q;
    h->nx = d->nx;
    h->ny = d->ny;
    h->nz = d->nz;
    h->force_kind = d->force_kind;
    h->mask = d->solid != nullptr;
    h->alloc = d->alloc;
    h->free_ = d->free_;
    h->alloc_ctx = d->alloc_ctx;

    const int nxp = (d->nx + 31) / 32 * 32;
    const long long plane = (long long)nxp * d->ny * d->nz;
    if (plane * Q >= (1LL << 40) || plane >= (1LL << 31)) {
        delete h;
        return fail(nullptr, LBM_ERR_ARG, "domain too large");
    }
    KParams &kp = h->kp;
    kp.nx = d->nx;
    kp.ny = d->ny;
    kp.nz = d->nz;
    kp.nxp = nxp;
    kp.plane = plane;
    for (int k = 0; k < 3; ++k) kp.per[k] = d->periodic[k] ? 1 : 0;
    kp.force_kind = d->force_kind;
    for (int n = 0; n < 5; ++n) {
        kp.om[n] = d->tau[n] > 0.0 ? 1.0 / d->tau[n] : 0.0;
        kp.om32[n] = (float)kp.om[n];
    }
    kp.omb = d->tau_bulk != 0.0 ? 1.0 / d->tau_bulk : kp.om[2];
    kp.omb32 = (float)kp.omb;
    if (d->lattice == LBM_D2Q9) fill_offsets<D2Q9>(kp);
    else if (d->lattice == LBM_D3Q19) fill_offsets<D3Q19>(kp);
    else fill_offsets<D3Q27>(kp);

    // launch shape, from the measured rates on GB300 (D2Q9 4096^2, 256^3):
    // without an obstacle mask, 2-byte storage and D3Q27 in FP32 take the
    // vector kernel; everything else the strided kernel, wide 2-D rows and
    // D3Q19 in FP32 with two nodes per thread
    h->cfg.bdx = D == 2 ? 128 : 64;
    h->cfg.npt = (D == 2 && d->nx >= 512) ? 2 : 1;
    h->cfg.vec = 0;
    if (d->nx <= 64) h->cfg.bdx = 64;
    if (D == 3 && d->storage == LBM_F32 && d->lattice == LBM_D3Q19) h->cfg.npt = 2;
    const bool vec_fits = !h->mask && (long long)Q * plane < (1LL << 32);
    if (vec_fits && storage_bytes(d->storage) == 2) {
        // 2-byte storage without a mask: the vector layout at its wider width
        // (D2Q9 8 nodes, 16 bytes; the 3-D lattices 4 nodes, 8 bytes)
        h->cfg.vec = 1;
        h->cfg.npt = vec_width_hi(d->lattice, d->storage);
        h->cfg.bdx = d->lattice == LBM_D3Q27 ? 64 : 32;
    } else if (vec_fits && d->lattice == LBM_D3Q27 && d->storage == LBM_F32) {
        h->cfg.vec = 1;
        h->cfg.npt = vec_width_hi(d->lattice, d->storage);
        h->cfg.bdx = 128;
    }
    h->graph_steps = 64;

    lbm_status st;
    if (d->stream) {
        h->stream = (cudaStream_t)d->stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            lbm_status s2 = cuda_fail(nullptr, e, "cudaStreamCreate");
            delete h;
            return s2;
        }
        h->own_stream = true;
    }
    h->state_bytes = (size_t)plane * Q * storage_bytes(d->storage);
    h->max_blocks = kMomGridMax;
    const size_t N = h->N();
    h->g_count = g_count_for(h);
    h->gdev_count = std::max<size_t>(3, h->force_kind == LBM_G_FIELD ? (size_t)D * plane : h->g_count);
    if ((st = alloc_into(h, &h->buf[0], h->state_bytes, "population buffer A")) ||
        (st = alloc_into(h, &h->buf[1], h->state_bytes, "population buffer B")) ||
        (st = alloc_into(h, &h->partials, (size_t)h->max_blocks * kPartials * sizeof(double), "partials")) ||
        (st = alloc_into(h, &h->red_dev, 8 * sizeof(double), "reduction")) ||
        (st = alloc_into(h, &h->g_dev,
                         std::max<size_t>(3, h->force_kind == LBM_G_FIELD ? (size_t)D * plane : h->g_count) *
                             sizeof(double),
                         "force")) ||
        (st = alloc_into(h, &h->g32_dev,
                         std::max<size_t>(3, h->force_kind == LBM_G_FIELD ? (size_t)D * plane : h->g_count) *
                             sizeof(float),
                         "force (FP32)"))) {
        *out = nullptr;
        std::string m = h->err;
        lbm_destroy(h);
        return fail(nullptr, st, m);
    }
    kp.g = h->g_dev;
    kp.g32 = h->g32_dev;
    // zero both buffers (padding included) so every byte is defined
    cudaError_t e = cudaMemsetAsync(h->buf[0], 0, h->state_bytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->buf[1], 0, h->state_bytes, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->g_dev, 0, 3 * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->g32_dev, 0, 3 * sizeof(float), h->stream);
    if (e != cudaSuccess) {
        lbm_status s2 = cuda_fail(nullptr, e, "cudaMemsetAsync");
        lbm_destroy(h);
        return s2;
    }
    if ((st = upload_force(h, d->g)) != LBM_OK) {
        std::string m = h->err;
        lbm_destroy(h);
        return fail(nullptr, st, m);
    }
    if (h->mask) {
        if ((st = alloc_into(h, &h->solid_dev, (size_t)plane, "solid mask")) != LBM_OK) {
            std::string m = h->err;
            lbm_destroy(h);
            return fail(nullptr, st, m);
        }
        std::vector<unsigned char> tmp((size_t)plane, 0);
        for (size_t zy = 0; zy < (size_t)d->ny * d->nz; ++zy)
            for (int x = 0; x < d->nx; ++x) tmp[zy * nxp + x] = d->solid[zy * d->nx + x] ? 1 : 0;
        e = cudaMemcpyAsync(h->solid_dev, tmp.data(), tmp.size(), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) {
            lbm_status s2 = cuda_fail(nullptr, e, "solid upload");
            lbm_destroy(h);
            return s2;
        }
        kp.solid = h->solid_dev;
    }
    // initial state: target fbar in buffer B, unstreamed into buffer A
    double *rho0_dev = nullptr, *u0_dev = nullptr;
    if (d->rho0 || d->u0) {
        if ((st = alloc_into(h, &h->fields, (size_t)(1 + D) * N * sizeof(double), "fields")) != LBM_OK) {
            std::string m = h->err;
            lbm_destroy(h);
            return fail(nullptr, st, m);
        }
        if (d->rho0) {
            rho0_dev = h->fields;
            e = cudaMemcpyAsync(rho0_dev, d->rho0, N * sizeof(double), cudaMemcpyHostToDevice, h->stream);
        }
        if (e == cudaSuccess && d->u0) {
            u0_dev = h->fields + N;
            e = cudaMemcpyAsync(u0_dev, d->u0, (size_t)D * N * sizeof(double), cudaMemcpyHostToDevice, h->stream);
        }
        if (e != cudaSuccess) {
            lbm_status s2 = cuda_fail(nullptr, e, "initial field upload");
            lbm_destroy(h);
            return s2;
        }
    }
    const Launchers &L = launchers_for(h->lattice);
    e = L.init(h->collision, h->storage, h->mask, kp, rho0_dev, u0_dev, h->buf[1], h->stream);
    if (e == cudaSuccess) e = L.unstream(h->storage, h->mask, kp, h->buf[1], h->buf[0], h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        lbm_status s2 = cuda_fail(nullptr, e, "initialisation");
        lbm_destroy(h);
        return s2;
    }
    h->cur = 0;
    if (d->u0 && h->gmax > 0.0) {
        double umax = 0.0;
        for (size_t k = 0; k < (size_t)D * N; ++k) umax = std::max(umax, std::fabs(d->u0[k]));
        const double us = stall_speed(h->storage, h->gmax);
        if (umax > us)
            h->err = "note: the initial speed " + std::to_string(umax) + " exceeds " + std::to_string(us) +
                     ", above which one step of the body force rounds away in this storage format "
                     "(lbm_force_resolution)";
    }
    *out = h;
    return LBM_OK;
}

lbm_status lbm_step(lbm_handle *h, int64_t nsteps) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (nsteps < 0) return fail(h, LBM_ERR_ARG, "nsteps < 0");
    int64_t left = nsteps;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    LBM_CUDA(h, cudaStreamIsCapturing(h->stream, &cs));
    if (cs == cudaStreamCaptureStatusNone && left >= h->graph_steps) {
        lbm_status st = ensure_graph(h);
        if (st != LBM_OK) return st;
        while (left >= h->graph_steps) {
            LBM_CUDA(h, cudaGraphLaunch(h->graph[h->cur], h->stream));
            left -= h->graph_steps;
        }
    }
    lbm_status st = launch_steps(h, left);
    if (st != LBM_OK) return st;
    h->step += nsteps;
    return LBM_OK;
}

lbm_status lbm_moments_device(lbm_handle *h, double *rho_dev, double *u_dev, double *totals_dev) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    lbm_status st = run_moments(h, rho_dev, u_dev, nullptr);
    if (st != LBM_OK) return st;
    if (totals_dev)
        LBM_CUDA(h, cudaMemcpyAsync(totals_dev, h->red_dev, 4 * sizeof(double), cudaMemcpyDeviceToDevice,
                                    h->stream));
    return LBM_OK;
}

lbm_status lbm_moments(lbm_handle *h, double *rho, double *u, double *totals) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    const size_t N = h->N();
    if ((rho || u) && !h->fields) {
        lbm_status st = alloc_into(h, &h->fields, (size_t)(1 + h->D) * N * sizeof(double), "fields");
        if (st != LBM_OK) return st;
    }
    double *rd = rho ? h->fields : nullptr;
    double *ud = u ? h->fields + N : nullptr;
    lbm_status st = run_moments(h, rd, ud, nullptr);
    if (st != LBM_OK) return st;
    double red[7];
    LBM_CUDA(h, cudaMemcpyAsync(red, h->red_dev, sizeof(red), cudaMemcpyDeviceToHost, h->stream));
    if (rho) LBM_CUDA(h, cudaMemcpyAsync(rho, rd, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (u) LBM_CUDA(h, cudaMemcpyAsync(u, ud, (size_t)h->D * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    if (totals) {
        totals[0] = red[0];
        totals[1] = red[1];
        totals[2] = red[2];
        totals[3] = h->D == 3 ? red[3] : 0.0;
    }
    if (red[6] > 0.0) return fail(h, LBM_ERR_UNSTABLE, "non-finite density or velocity");
    return LBM_OK;
}

lbm_status lbm_residual(lbm_handle *h, int K, double *r) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (K < 1 || !r) return fail(h, LBM_ERR_ARG, "K must be >= 1 and r non-NULL");
    const size_t N = h->N();
    if (!h->uprev) {
        const size_t bytes = (size_t)h->D * N * arith_bytes(h->storage);
        lbm_status st = alloc_into(h, &h->uprev, bytes, "residual velocity");
        if (st != LBM_OK) return st;
        LBM_CUDA(h, cudaMemsetAsync(h->uprev, 0, bytes, h->stream));
    }
    lbm_status st;
    if (h->uprev_step != h->step) {
        // velocity at the current step into uprev
        if ((st = run_moments(h, nullptr, nullptr, h->uprev)) != LBM_OK) return st;
    }
    if ((st = lbm_step(h, K)) != LBM_OK) return st;
    if ((st = run_moments(h, nullptr, nullptr, h->uprev)) != LBM_OK) return st;
    double red[7];
    LBM_CUDA(h, cudaMemcpyAsync(red, h->red_dev, sizeof(red), cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    h->uprev_step = h->step;
    if (red[6] > 0.0 || !std::isfinite(red[4]) || !std::isfinite(red[5])) {
        *r = NAN;
        return fail(h, LBM_ERR_UNSTABLE, "non-finite velocity");
    }
    *r = red[5] > 0.0 ? std::sqrt(red[4]) / ((double)K * std::sqrt(red[5])) : (red[4] > 0.0 ? INFINITY : 0.0);
    return LBM_OK;
}

lbm_status lbm_check_device(lbm_handle *h, double *out_dev) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (!out_dev) return fail(h, LBM_ERR_ARG, "out_dev is NULL");
    if (!h->uprev) {
        const size_t bytes = (size_t)h->D * h->N() * arith_bytes(h->storage);
        lbm_status st = alloc_into(h, &h->uprev, bytes, "residual velocity");
        if (st != LBM_OK) return st;
        LBM_CUDA(h, cudaMemsetAsync(h->uprev, 0, bytes, h->stream));
    }
    lbm_status st = run_moments(h, nullptr, nullptr, h->uprev, out_dev);
    if (st != LBM_OK) return st;
    h->uprev_step = h->step;
    return LBM_OK;
}

lbm_status lbm_set_force(lbm_handle *h, const double *g) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (h->force_kind == LBM_G_NONE) return fail(h, LBM_ERR_STATE, "created without a force");
    if (h->gs_dev) {
        // a constant force replaces the schedule
        LBM_CUDA(h, cudaStreamSynchronize(h->stream));
        drop_graphs(h);
        free_schedule(h);
    }
    return upload_force(h, g);
}


lbm_status lbm_set_force_schedule(lbm_handle *h, const double *table, int64_t period) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (h->force_kind != LBM_G_UNIFORM) return fail(h, LBM_ERR_STATE, "a force schedule needs LBM_G_UNIFORM");
    if (period < 0 || (period > 0 && !table)) return fail(h, LBM_ERR_ARG, "bad schedule");
    if (period > (int64_t)1 << 30) return fail(h, LBM_ERR_ARG, "schedule period too long");
    std::vector<double> tmp((size_t)period * 3, 0.0);
    for (int64_t t = 0; t < period; ++t)
        for (int a = 0; a < h->D; ++a) {
            const double v = table[t * h->D + a];
            if (!std::isfinite(v)) return fail(h, LBM_ERR_ARG, "schedule contains a non-finite value");
            tmp[(size_t)t * 3 + a] = v;
        }
    return set_schedule(h, tmp, period, false);
}

lbm_status lbm_set_force_scale_schedule(lbm_handle *h, const double *scale, int64_t period) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (h->force_kind == LBM_G_NONE) return fail(h, LBM_ERR_STATE, "created without a force");
    if (period < 0 || (period > 0 && !scale)) return fail(h, LBM_ERR_ARG, "bad schedule");
    if (period > (int64_t)1 << 30) return fail(h, LBM_ERR_ARG, "schedule period too long");
    std::vector<double> tmp(scale, scale + period);
    for (double v : tmp)
        if (!std::isfinite(v)) return fail(h, LBM_ERR_ARG, "schedule contains a non-finite value");
    return set_schedule(h, tmp, period, true);
}

lbm_status lbm_get_populations(lbm_handle *h, double *f) {
    if (!h || !f) return fail(h, LBM_ERR_ARG, "NULL argument");
    const size_t n = (size_t)h->Q * h->N();
    double *tmp = nullptr;
    lbm_status st = alloc_into(h, &tmp, n * sizeof(double), "population export");
    if (st != LBM_OK) return st;
    cudaError_t e = launchers_for(h->lattice).get_pops(h->storage, h->mask, h->kp, h->buf[h->cur], tmp, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, tmp, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dev_free(h, tmp);
    if (e != cudaSuccess) return cuda_fail(h, e, "population export");
    return LBM_OK;
}

lbm_status lbm_set_populations(lbm_handle *h, const double *f) {
    if (!h || !f) return fail(h, LBM_ERR_ARG, "NULL argument");
    const size_t n = (size_t)h->Q * h->N();
    double *tmp = nullptr;
    lbm_status st = alloc_into(h, &tmp, n * sizeof(double), "population import");
    if (st != LBM_OK) return st;
    const Launchers &L = launchers_for(h->lattice);
    void *spare = h->buf[1 - h->cur];
    cudaError_t e = cudaMemcpyAsync(tmp, f, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = L.put_pops(h->storage, h->kp, tmp, spare, h->stream);
    if (e == cudaSuccess) e = L.unstream(h->storage, h->mask, h->kp, spare, h->buf[h->cur], h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dev_free(h, tmp);
    if (e != cudaSuccess) return cuda_fail(h, e, "population import");
    h->uprev_step = -1;
    return LBM_OK;
}

size_t lbm_state_bytes(const lbm_handle *h) { return h ? h->state_bytes : 0; }

lbm_status lbm_get_state(lbm_handle *h, void *host, size_t bytes, int64_t *step) {
    if (!h || !host) return fail(h, LBM_ERR_ARG, "NULL argument");
    if (bytes != h->state_bytes) return fail(h, LBM_ERR_STATE, "state size mismatch");
    LBM_CUDA(h, cudaMemcpyAsync(host, h->buf[h->cur], bytes, cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    if (step) *step = h->step;
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_handle *h, const void *host, size_t bytes, int64_t step) {
    if (!h || !host) return fail(h, LBM_ERR_ARG, "NULL argument");
    if (bytes != h->state_bytes) return fail(h, LBM_ERR_STATE, "state size mismatch");
    LBM_CUDA(h, cudaMemcpyAsync(h->buf[h->cur], host, bytes, cudaMemcpyHostToDevice, h->stream));
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    h->step = step;
    h->uprev_step = -1;
    return LBM_OK;
}

lbm_status lbm_set_launch_layout(lbm_handle *h, int block_x, int nodes_per_thread, int layout) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (layout != LBM_LAYOUT_STRIDED && layout != LBM_LAYOUT_VECTOR) return fail(h, LBM_ERR_ARG, "bad layout");
    const StepCfg c{block_x, nodes_per_thread, layout == LBM_LAYOUT_VECTOR ? 1 : 0};
    if (!shape_ok(h, c)) {
        if (layout == LBM_LAYOUT_VECTOR && !vec_ok(h))
            return fail(h, LBM_ERR_ARG, "the vector layout takes no obstacle mask and Q * plane < 2^32");
        return fail(h, LBM_ERR_ARG,
                    layout == LBM_LAYOUT_VECTOR
                        ? "block_x must be 32, 64, 128 or 256 and nodes_per_thread a vector width built for this "
                          "lattice and storage (lbm_launch_widths)"
                        : "block_x must be 32, 64, 128 or 256 and nodes_per_thread 1 or 2");
    }
    LBM_CUDA(h, cudaStreamSynchronize(h->stream));
    h->cfg = c;
    drop_graphs(h);
    return LBM_OK;
}

lbm_status lbm_set_launch(lbm_handle *h, int block_x, int nodes_per_thread) {
    return lbm_set_launch_layout(h, block_x, nodes_per_thread, LBM_LAYOUT_STRIDED);
}

lbm_status lbm_get_launch(const lbm_handle *h, int *block_x, int *nodes_per_thread, int *layout) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (block_x) *block_x = h->cfg.bdx;
    if (nodes_per_thread) *nodes_per_thread = h->cfg.npt;
    if (layout) *layout = h->cfg.vec ? LBM_LAYOUT_VECTOR : LBM_LAYOUT_STRIDED;
    return LBM_OK;
}

lbm_status lbm_launch_widths(int lattice, int storage, int *lo, int *hi) {
    if (lattice < LBM_D2Q9 || lattice > LBM_D3Q27 || storage < LBM_F64 || storage > LBM_BF16_SHIFT)
        return fail(nullptr, LBM_ERR_ARG, "bad lattice or storage");
    if (lo) *lo = vec_width_lo(lattice, storage);
    if (hi) *hi = vec_width_hi(lattice, storage);
    return LBM_OK;
}

lbm_status lbm_autotune(lbm_handle *h, int trials, int *block_x, int *nodes_per_thread, double *ms) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (trials < 1) return fail(h, LBM_ERR_ARG, "trials must be >= 1");
    // strided shapes, then (without a mask) the vector widths
    std::vector<StepCfg> shapes = {{32, 1, 0}, {64, 1, 0}, {64, 2, 0}, {128, 1, 0}, {128, 2, 0}, {256, 1, 0}, {256, 2, 0}};
    if (vec_ok(h)) {
        const int wl = vec_width_lo(h->lattice, h->storage), wh = vec_width_hi(h->lattice, h->storage);
        for (int bx : {32, 64, 128}) {
            shapes.push_back({bx, wl, 1});
            if (wh != wl) shapes.push_back({bx, wh, 1});
        }
    }
    cudaEvent_t e0, e1;
    LBM_CUDA(h, cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(h, e, "cudaEventCreate");
    }
    double best = 1e300;
    StepCfg best_cfg = h->cfg;
    for (const StepCfg &c : shapes) {
        // one untimed launch, then the timed ones; all read the state and
        // write the spare buffer
        e = launch_step(h, c, h->buf[h->cur], h->buf[1 - h->cur]);
        if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
        for (int t = 0; t < trials && e == cudaSuccess; ++t) e = launch_step(h, c, h->buf[h->cur], h->buf[1 - h->cur]);
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t_ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t_ms, e0, e1);
        if (e != cudaSuccess) break;
        const double per = (double)t_ms / trials;
        if (per < best) {
            best = per;
            best_cfg = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(h, e, "autotune");
    lbm_status st = lbm_set_launch_layout(h, best_cfg.bdx, best_cfg.npt,
                                          best_cfg.vec ? LBM_LAYOUT_VECTOR : LBM_LAYOUT_STRIDED);
    if (st != LBM_OK) return st;
    if (block_x) *block_x = best_cfg.bdx;
    if (nodes_per_thread) *nodes_per_thread = best_cfg.npt;
    if (ms) *ms = best;
    return LBM_OK;
}

lbm_status lbm_force_resolution(const lbm_handle *h, double *u_stall) {
    if (!h || !u_stall) return fail(nullptr, LBM_ERR_ARG, "NULL argument");
    *u_stall = stall_speed(h->storage, h->gs_dev ? h->gmax_sched : h->gmax);
    return LBM_OK;
}

lbm_status lbm_info(const lbm_handle *h, int *D, int *Q, int64_t *step, size_t *bytes_per_node) {
    if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
    if (D) *D = h->D;
    if (Q) *Q = h->Q;
    if (step) *step = h->step;
    if (bytes_per_node) *bytes_per_node = 2 * (size_t)h->Q * storage_bytes(h->storage);
    return LBM_OK;
}

}  // extern "C"
