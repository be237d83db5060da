// lbm_split.cu -- a domain split into slabs along its outermost axis (y in
// 2-D, z in 3-D), each slab in its own population buffers with one halo
// layer at each end of that axis.  One time step is the stream-collide step
// of every slab, then one exchange: the pull of Sec. II.C reads, at a slab's
// first and last layer, the populations that cross the cut, which the
// neighbouring slab wrote; they are copied into the halo layers (those with
// c = +1 along the axis into the lower halo, c = -1 into the upper).  The
// FP64 check is each slab's partial sums, added in slab order (the
// all-reduce of 1 + D doubles and the residual terms).
//
// Here all slabs live on one device and share one stream, so the steps and
// the exchange are ordered by the stream; the exchange is one kernel over a
// table of layer copies.  The layout (which layers a slab owns) and the
// schedule (which copy fills which halo) are host functions, exported as
// lbm_split_schedule so that other transports can run the same schedule.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace lbm;

namespace lbm {
lbm_status handle_make_slab(lbm_handle *h, int ax, int g0, int gn);
void handle_buffers(const lbm_handle *h, void **b0, void **b1, int *cur, size_t *bytes);
cudaStream_t handle_stream(const lbm_handle *h);
}  // namespace lbm

namespace {

int lat_D(int lat) { return lat == LBM_D2Q9 ? 2 : 3; }
int lat_Q(int lat) { return lat == LBM_D2Q9 ? 9 : (lat == LBM_D3Q19 ? 19 : 27); }
size_t st_bytes(int st) { return st == LBM_F64 ? 8 : (st == LBM_F32 ? 4 : 2); }

// velocity component of population i along axis a, in the population order
// of include/lbm.h
int pop_c(int lat, int i, int a) {
    if (lat == LBM_D2Q9) return a == 0 ? Lat<D2Q9>::cx(i) : (a == 1 ? Lat<D2Q9>::cy(i) : 0);
    return C3::c(i, a);
}

// slab p owns the global layers [g0, g0 + n) of an axis of extent n_all:
// the first n_all % parts slabs one layer more
void layout(int n_all, int parts, int p, int *g0, int *n) {
    const int base = n_all / parts, rem = n_all % parts;
    *n = base + (p < rem ? 1 : 0);
    *g0 = p * base + std::min(p, rem);
}

struct Copy {
    int dst_part, dst_layer, src_part, src_layer, pop;
};

// the halo copies of one exchange, slab by slab: the lower halo (local layer
// 0) takes the populations with c = +1 along the axis from the top owned
// layer of the slab below, the upper halo (local layer n + 1) those with
// c = -1 from the first owned layer of the slab above; across the domain's
// ends only when the axis is periodic (a wall there bounces back instead)
std::vector<Copy> schedule(int lat, int n_all, int parts, int periodic) {
    const int D = lat_D(lat), Q = lat_Q(lat), ax = D - 1;
    std::vector<Copy> out;
    for (int p = 0; p < parts; ++p) {
        int g0, n;
        layout(n_all, parts, p, &g0, &n);
        const int below = p > 0 ? p - 1 : (periodic ? parts - 1 : -1);
        const int above = p < parts - 1 ? p + 1 : (periodic ? 0 : -1);
        if (below >= 0) {
            int bg0, bn;
            layout(n_all, parts, below, &bg0, &bn);
            for (int i = 0; i < Q; ++i)
                if (pop_c(lat, i, ax) == 1) out.push_back({p, 0, below, bn, i});
        }
        if (above >= 0)
            for (int i = 0; i < Q; ++i)
                if (pop_c(lat, i, ax) == -1) out.push_back({p, n + 1, above, 1, i});
    }
    return out;
}

struct HaloCopy {
    const uint4 *src;
    uint4 *dst;
    unsigned n16;   // 16-byte words
};

// every copy of the exchange in one launch: block b takes copies b,
// b + gridDim.x, ...
__global__ void k_halo(const HaloCopy *__restrict__ t, int n) {
    for (int c = blockIdx.x; c < n; c += gridDim.x) {
        const HaloCopy h = t[c];
        for (unsigned k = threadIdx.x; k < h.n16; k += blockDim.x) h.dst[k] = h.src[k];
    }
}

// the all-reduce of the slabs' checks: 7 doubles each, added in slab order
__global__ void k_sum_parts(const double *__restrict__ parts, int n, double *__restrict__ out) {
    const int k = threadIdx.x;
    if (k >= 7) return;
    double s = 0.0;
    for (int p = 0; p < n; ++p) s += parts[8 * p + k];
    out[k] = s;
}

thread_local std::string g_split_err;

}  // namespace

struct lbm_split {
    int lattice = 0, storage = 0, D = 2, Q = 9, parts = 0, ax = 1;
    int n_all = 0;                 // global extent of the split axis
    int periodic = 0;              // along the split axis
    size_t layer_elems = 0;        // elements of one population layer: nxp (2-D), nxp * ny (3-D)
    lbm_handle *global = nullptr;  // the whole domain: initial state, and reads
    std::vector<lbm_handle *> h;   // the slabs
    std::vector<int> g0, n;
    cudaStream_t stream = nullptr;
    HaloCopy *table[2] = {nullptr, nullptr};   // device tables, by the buffer that holds the state
    int ncopies = 0;
    double *tmp = nullptr;         // 8 doubles per slab: the slabs' checks
    int64_t step = 0;
    std::string err;
};

namespace {

lbm_status sfail(lbm_split *s, lbm_status st, const std::string &m) {
    if (s) s->err = m;
    else g_split_err = m;
    return st;
}

lbm_status scuda(lbm_split *s, cudaError_t e, const char *what) {
    return sfail(s, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

// global layer of local layer l of a slab starting at g0, wrapped on a
// periodic axis; -1 beyond a wall
int global_layer(int g0, int l, int n_all, int periodic) {
    int g = g0 + l - 1;
    if (g < 0 || g >= n_all) {
        if (!periodic) return -1;
        g = (g + n_all) % n_all;
    }
    return g;
}

// copy layers [l0, l1) of a slab from (to) the whole-domain buffer, all
// populations; runs of consecutive global layers are one copy each
cudaError_t move_layers(lbm_split *s, int p, int l0, int l1, void *slab_buf, void *glob_buf, bool to_slab) {
    const size_t es = st_bytes(s->storage);
    const size_t lay = s->layer_elems * es;
    // the plane of a population: 2-D [ny][nxp], 3-D [nz][ny][nxp]: both are
    // (layers of the split axis) x (layer), the split axis outermost
    const size_t gplane = (size_t)s->n_all * lay;
    const size_t lplane = (size_t)(s->n[p] + 2) * lay;
    for (int i = 0; i < s->Q; ++i) {
        int l = l0;
        while (l < l1) {
            const int g = global_layer(s->g0[p], l, s->n_all, s->periodic);
            if (g < 0) {
                ++l;
                continue;
            }
            int run = 1;
            while (l + run < l1 && global_layer(s->g0[p], l + run, s->n_all, s->periodic) == g + run) ++run;
            char *sl = (char *)slab_buf + (size_t)i * lplane + (size_t)l * lay;
            char *gl = (char *)glob_buf + (size_t)i * gplane + (size_t)g * lay;
            cudaError_t e = to_slab ? cudaMemcpyAsync(sl, gl, run * lay, cudaMemcpyDeviceToDevice, s->stream)
                                    : cudaMemcpyAsync(gl, sl, run * lay, cudaMemcpyDeviceToDevice, s->stream);
            if (e != cudaSuccess) return e;
            l += run;
        }
    }
    return cudaSuccess;
}

// the slabs' owned layers into the whole-domain handle's state buffer
lbm_status gather(lbm_split *s) {
    void *b0, *b1;
    int cur;
    size_t bytes;
    handle_buffers(s->global, &b0, &b1, &cur, &bytes);
    void *gbuf = cur ? b1 : b0;
    for (int p = 0; p < s->parts; ++p) {
        void *c0, *c1;
        int ccur;
        size_t cb;
        handle_buffers(s->h[p], &c0, &c1, &ccur, &cb);
        cudaError_t e = move_layers(s, p, 1, s->n[p] + 1, ccur ? c1 : c0, gbuf, false);
        if (e != cudaSuccess) return scuda(s, e, "gather");
    }
    return LBM_OK;
}

void destroy(lbm_split *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (lbm_handle *h : s->h) lbm_destroy(h);
    for (HaloCopy *t : s->table)
        if (t) cudaFree(t);
    if (s->tmp) cudaFree(s->tmp);
    if (s->global) lbm_destroy(s->global);
    delete s;
}

}  // namespace

extern "C" {

lbm_status lbm_split_schedule(int lattice, int n_all, int parts, int periodic, int *layers, int *copies,
                              int max_copies, int *n_copies) {
    if (lattice < LBM_D2Q9 || lattice > LBM_D3Q27) return sfail(nullptr, LBM_ERR_ARG, "bad lattice");
    if (parts < 1 || n_all < parts) return sfail(nullptr, LBM_ERR_ARG, "need 1 <= parts <= the axis's extent");
    if (layers)
        for (int p = 0; p < parts; ++p) layout(n_all, parts, p, &layers[2 * p], &layers[2 * p + 1]);
    const std::vector<Copy> sc = schedule(lattice, n_all, parts, periodic);
    if (n_copies) *n_copies = (int)sc.size();
    if (copies) {
        if (max_copies < (int)sc.size()) return sfail(nullptr, LBM_ERR_ARG, "copies array too small");
        for (size_t k = 0; k < sc.size(); ++k) {
            copies[5 * k + 0] = sc[k].dst_part;
            copies[5 * k + 1] = sc[k].dst_layer;
            copies[5 * k + 2] = sc[k].src_part;
            copies[5 * k + 3] = sc[k].src_layer;
            copies[5 * k + 4] = sc[k].pop;
        }
    }
    return LBM_OK;
}

lbm_status lbm_split_create(const lbm_desc *d, int parts, lbm_split **out) {
    if (!d || !out) return sfail(nullptr, LBM_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (d->lattice < LBM_D2Q9 || d->lattice > LBM_D3Q27) return sfail(nullptr, LBM_ERR_ARG, "bad lattice");
    const int D = lat_D(d->lattice);
    const int n_all = D == 2 ? d->ny : d->nz;
    if (parts < 1 || parts > n_all) return sfail(nullptr, LBM_ERR_ARG, "need 1 <= parts <= the split axis's extent");
    lbm_split *s = new (std::nothrow) lbm_split();
    if (!s) return sfail(nullptr, LBM_ERR_OOM, "host allocation failed");
    s->lattice = d->lattice;
    s->storage = d->storage;
    s->D = D;
    s->Q = lat_Q(d->lattice);
    s->parts = parts;
    s->ax = D - 1;
    s->n_all = n_all;
    s->periodic = d->periodic[D - 1] ? 1 : 0;
    const int nxp = (d->nx + 31) / 32 * 32;
    s->layer_elems = D == 2 ? (size_t)nxp : (size_t)nxp * d->ny;

    // the whole domain: its creation computes the initial state
    lbm_status st = lbm_create(d, &s->global);
    if (st != LBM_OK) {
        std::string m = lbm_last_error(nullptr);
        destroy(s);
        return sfail(nullptr, st, m);
    }
    s->stream = handle_stream(s->global);

    // the slabs: the same description over their layers plus the halo
    // layers, with the force and mask of those layers (zero beyond a wall)
    const size_t row = (size_t)d->nx;                       // elements of an unpadded row
    const size_t lay = D == 2 ? row : row * d->ny;          // of an unpadded layer
    for (int p = 0; p < parts; ++p) {
        int g0, n;
        layout(n_all, parts, p, &g0, &n);
        s->g0.push_back(g0);
        s->n.push_back(n);
        lbm_desc ld = *d;
        if (D == 2) ld.ny = n + 2;
        else ld.nz = n + 2;
        ld.rho0 = nullptr;
        ld.u0 = nullptr;
        ld.stream = s->stream;
        std::vector<double> g;
        std::vector<uint8_t> solid;
        const size_t layers = (size_t)n + 2;
        if (d->force_kind == LBM_G_ROWS && D == 2) {
            // one row of the table per y: the slab's rows
            g.assign(layers * D, 0.0);
            for (size_t l = 0; l < layers; ++l) {
                const int gl = global_layer(g0, (int)l, n_all, s->periodic);
                const int src = gl < 0 ? (l == 0 ? 0 : n_all - 1) : gl;
                for (int a = 0; a < D; ++a) g[l * D + a] = d->g[(size_t)src * D + a];
            }
            ld.g = g.data();
        } else if (d->force_kind == LBM_G_FIELD) {
            const size_t N = (size_t)d->nx * d->ny * d->nz;
            g.assign((size_t)D * layers * lay, 0.0);
            for (int a = 0; a < D; ++a)
                for (size_t l = 0; l < layers; ++l) {
                    const int gl = global_layer(g0, (int)l, n_all, s->periodic);
                    if (gl < 0) continue;
                    std::memcpy(&g[(size_t)a * layers * lay + l * lay], &d->g[(size_t)a * N + (size_t)gl * lay],
                                lay * sizeof(double));
                }
            ld.g = g.data();
        }
        if (d->solid) {
            solid.assign(layers * lay, 0);
            for (size_t l = 0; l < layers; ++l) {
                const int gl = global_layer(g0, (int)l, n_all, s->periodic);
                if (gl < 0) continue;
                std::memcpy(&solid[l * lay], &d->solid[(size_t)gl * lay], lay);
            }
            ld.solid = solid.data();
        }
        lbm_handle *h = nullptr;
        st = lbm_create(&ld, &h);
        if (st != LBM_OK) {
            std::string m = lbm_last_error(nullptr);
            destroy(s);
            return sfail(nullptr, st, m);
        }
        s->h.push_back(h);
        if ((st = handle_make_slab(h, D == 2 ? 1 : 2, g0, n_all)) != LBM_OK) {
            std::string m = lbm_last_error(h);
            destroy(s);
            return sfail(nullptr, st, m);
        }
    }

    // the initial state, halo layers included, from the whole domain
    void *gb0, *gb1;
    int gcur;
    size_t gbytes;
    handle_buffers(s->global, &gb0, &gb1, &gcur, &gbytes);
    for (int p = 0; p < parts; ++p) {
        void *b0, *b1;
        int cur;
        size_t bytes;
        handle_buffers(s->h[p], &b0, &b1, &cur, &bytes);
        cudaError_t e = move_layers(s, p, 0, s->n[p] + 2, cur ? b1 : b0, gcur ? gb1 : gb0, true);
        if (e != cudaSuccess) {
            lbm_status r = scuda(nullptr, e, "initial slab state");
            destroy(s);
            return r;
        }
    }

    // the exchange tables, one per buffer that holds the state after a step
    const std::vector<Copy> sc = schedule(d->lattice, n_all, parts, s->periodic);
    s->ncopies = (int)sc.size();
    const size_t es = st_bytes(d->storage);
    const size_t lay_b = s->layer_elems * es;   // a multiple of 64 bytes (nxp is a multiple of 32)
    for (int c = 0; c < 2; ++c) {
        std::vector<HaloCopy> t;
        for (const Copy &k : sc) {
            void *d0, *d1, *q0, *q1;
            int cur;
            size_t bytes;
            handle_buffers(s->h[k.dst_part], &d0, &d1, &cur, &bytes);
            handle_buffers(s->h[k.src_part], &q0, &q1, &cur, &bytes);
            const size_t dplane = (size_t)(s->n[k.dst_part] + 2) * lay_b;
            const size_t splane = (size_t)(s->n[k.src_part] + 2) * lay_b;
            HaloCopy hc;
            hc.src = (const uint4 *)((const char *)(c ? q1 : q0) + (size_t)k.pop * splane + (size_t)k.src_layer * lay_b);
            hc.dst = (uint4 *)((char *)(c ? d1 : d0) + (size_t)k.pop * dplane + (size_t)k.dst_layer * lay_b);
            hc.n16 = (unsigned)(lay_b / 16);
            t.push_back(hc);
        }
        if (!t.empty()) {
            cudaError_t e = cudaMalloc(&s->table[c], t.size() * sizeof(HaloCopy));
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s->table[c], t.data(), t.size() * sizeof(HaloCopy), cudaMemcpyHostToDevice,
                                    s->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
            if (e != cudaSuccess) {
                lbm_status r = scuda(nullptr, e, "exchange table");
                destroy(s);
                return r;
            }
        }
    }
    cudaError_t e = cudaMalloc(&s->tmp, (size_t)8 * parts * sizeof(double));
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        lbm_status r = scuda(nullptr, e, "check scratch");
        destroy(s);
        return r;
    }
    *out = s;
    return LBM_OK;
}

lbm_status lbm_split_step(lbm_split *s, int64_t nsteps) {
    if (!s) return sfail(nullptr, LBM_ERR_ARG, "split is NULL");
    if (nsteps < 0) return sfail(s, LBM_ERR_ARG, "nsteps < 0");
    for (int64_t t = 0; t < nsteps; ++t) {
        for (int p = 0; p < s->parts; ++p) {
            lbm_status st = lbm_step(s->h[p], 1);
            if (st != LBM_OK) return sfail(s, st, lbm_last_error(s->h[p]));
        }
        void *b0, *b1;
        int cur;
        size_t bytes;
        handle_buffers(s->h[0], &b0, &b1, &cur, &bytes);
        if (s->ncopies) {
            k_halo<<<std::min(s->ncopies, 1024), 256, 0, s->stream>>>(s->table[cur], s->ncopies);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return scuda(s, e, "halo exchange");
        }
        ++s->step;
    }
    return LBM_OK;
}

lbm_status lbm_split_check_device(lbm_split *s, double *out_dev) {
    if (!s || !out_dev) return sfail(s, LBM_ERR_ARG, "NULL argument");
    for (int p = 0; p < s->parts; ++p) {
        lbm_status st = lbm_check_device(s->h[p], s->tmp + 8 * p);
        if (st != LBM_OK) return sfail(s, st, lbm_last_error(s->h[p]));
    }
    k_sum_parts<<<1, 32, 0, s->stream>>>(s->tmp, s->parts, out_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return scuda(s, e, "check all-reduce");
    return LBM_OK;
}

lbm_status lbm_split_moments(lbm_split *s, double *rho, double *u, double *totals) {
    if (!s) return sfail(nullptr, LBM_ERR_ARG, "split is NULL");
    lbm_status st = gather(s);
    if (st != LBM_OK) return st;
    st = lbm_moments(s->global, rho, u, totals);
    if (st != LBM_OK) return sfail(s, st, lbm_last_error(s->global));
    return LBM_OK;
}

size_t lbm_split_state_bytes(const lbm_split *s) { return s ? lbm_state_bytes(s->global) : 0; }

lbm_status lbm_split_get_state(lbm_split *s, void *host, size_t bytes, int64_t *step) {
    if (!s) return sfail(nullptr, LBM_ERR_ARG, "split is NULL");
    lbm_status st = gather(s);
    if (st != LBM_OK) return st;
    st = lbm_get_state(s->global, host, bytes, nullptr);
    if (st != LBM_OK) return sfail(s, st, lbm_last_error(s->global));
    if (step) *step = s->step;
    return LBM_OK;
}

lbm_status lbm_split_get_populations(lbm_split *s, double *f) {
    if (!s) return sfail(nullptr, LBM_ERR_ARG, "split is NULL");
    lbm_status st = gather(s);
    if (st != LBM_OK) return st;
    st = lbm_get_populations(s->global, f);
    if (st != LBM_OK) return sfail(s, st, lbm_last_error(s->global));
    return LBM_OK;
}

lbm_status lbm_split_set_launch_layout(lbm_split *s, int block_x, int nodes_per_thread, int layout) {
    if (!s) return sfail(nullptr, LBM_ERR_ARG, "split is NULL");
    for (int p = 0; p < s->parts; ++p) {
        lbm_status st = lbm_set_launch_layout(s->h[p], block_x, nodes_per_thread, layout);
        if (st != LBM_OK) return sfail(s, st, lbm_last_error(s->h[p]));
    }
    return LBM_OK;
}

const char *lbm_split_last_error(const lbm_split *s) { return s ? s->err.c_str() : g_split_err.c_str(); }

void lbm_split_destroy(lbm_split *s) { destroy(s); }

}  // extern "C"
