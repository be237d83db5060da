// lbm_batch.cu -- many independent D2Q9 lattices (channels of uneven size and
// parameters) advanced by ONE persistent kernel until each reaches its
// steady-state residual.
//
// Work unit: a tile = a band of rows of one channel for one time step.  A CTA
// claims a tile through the channel's packed claim word (step | tiles of the
// step | next tile), pulls, collides and stores it, then counts it done; the
// CTA finishing the last tile of a step closes the step: at check steps it
// sums the tiles' FP64 residual partials in tile order, decides convergence,
// and publishes the next step (or retires the channel).  The tile count of
// the next step follows the work left: active nodes / (2 x resident CTAs),
// clamped to [2 x CTA size, the tuned maximum] -- large tiles while many
// channels run, small ones when few channels (the slowest) remain, so a
// lone channel's step is spread over many CTAs.  Steps of one channel are thus ordered by the
// done counter; different channels run independently.  No CTA waits for a
// particular other CTA: a CTA that finds nothing to claim scans again, and the
// scan is bounded by a no-progress counter that sets an error flag and exits.
// Population data written during the kernel by other CTAs is read through L2
// (ld.global.cg), never through the non-coherent read-only path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace lbm;

namespace lbm {

// the handoff of the tail to plain lattices (lbm_runtime.cu)
lbm_status handle_adopt(lbm_handle *h, const void *state_dev, const void *snap_dev, int64_t step, int64_t snap_step);
lbm_status handle_export_state(lbm_handle *h, void *state_dev);
cudaStream_t handle_stream(const lbm_handle *h);

struct BatchChan {
    long long off;       // element offset of the channel's Q planes in each population arena
    long long plane;     // nxp * ny
    long long snap_off;  // offset (elements of the arithmetic type) of its velocity snapshot, 2 * nx * ny
    long long part_off;  // offset (doubles) of its tile partials, 2 per tile, room for ny tiles
    long long solid_off; // offset of its obstacle mask (nxp * ny bytes) in the mask arena, -1: none
    int nx, ny, nxp;
    int per_x, per_y;
    double om2, om3, om4;
    double gx, gy;
};

// claim word: bits [0,13) next tile, [13,26) tiles of this step (<= 4096),
// [26,64) step.  Claimers only add when the tile field is below the tile
// count, so it overshoots by at most the number of CTAs (< 4096).
constexpr int kTileBits = 13;
constexpr unsigned long long kTileMask = (1ull << kTileBits) - 1;
constexpr int kMaxTiles = 4096;
__host__ __device__ inline unsigned long long claim_word(long long step, int tiles) {
    return ((unsigned long long)step << (2 * kTileBits)) | ((unsigned long long)tiles << kTileBits);
}

struct BatchCtl {
    unsigned long long claim;  // claim_word(step, tiles) + next tile index
    unsigned int done;         // tiles finished in the current step
    int active;
    long long steps;           // steps completed
    long long start;           // steps completed when the run began
    int status;
    double r;                  // last residual
    int parked;                // 1: left the kernel at a step boundary for the handoff
};

struct BatchRun {
    const BatchChan *ch;
    BatchCtl *ctl;
    int n;
    const unsigned char *solid;  // mask arena
    int grid;                  // resident CTAs
    int tile_min, tile_max;    // nodes per tile
    long long *active_nodes;   // nodes of channels still running
    unsigned *active_bits;     // bit c: channel c still running
    void *fa, *fb;  // the state after s steps lives in fa for even s, fb for odd s
    void *snap;
    double *part;
    int *active_count;
    unsigned long long *progress;
    int *error;
    double tol;     // < 0: never converge (fixed number of steps)
    int park_below; // > 0: once at most this many channels run, each parks at its next step boundary
    int K;
    long long max_steps;   // per channel, counted from the run's start
    long long spin_limit;  // scans without any progress anywhere before giving up
};

template <typename T> __device__ __forceinline__ T ld_cg(const T *p);
template <> __device__ __forceinline__ double ld_cg<double>(const double *p) { return __ldcg(p); }
template <> __device__ __forceinline__ float ld_cg<float>(const float *p) { return __ldcg(p); }

template <typename T>
__device__ __forceinline__ T vload(const T *p) { return *(const volatile T *)p; }

// pull of one D2Q9 node of a channel (walls or periodic per axis, halfway
// bounce-back at solid nodes when the channel has a mask); f is the channel's
// base, all offsets within a channel fit in 32 bits
template <int ST>
__device__ __forceinline__ void gather_chan(const BatchChan &C, const typename Store<ST>::T *f,
                                            const unsigned char *solid, int x, int y,
                                            typename Store<ST>::R *G) {
    typedef typename Store<ST>::R R;
    typedef typename Store<ST>::T T;
    const int plane = (int)C.plane;
    const int own = y * C.nxp + x;
    // no wall or wrap along y, and x inside the row or periodic (the row's
    // first and last nodes then take their x - c_x across the periodic face)
    const bool interior = ((x > 0 && x < C.nx - 1) || C.per_x) && y > 0 && y < C.ny - 1;
    const int xl = x == 0 ? C.nx - 1 : -1, xr = x == C.nx - 1 ? 1 - C.nx : 1;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int cx = Lat<D2Q9>::cx(i), cy = Lat<D2Q9>::cy(i);
        int src;
        bool wall = false;
        if (interior) {
            src = own + (cx == 1 ? xl : (cx == -1 ? xr : 0)) - cy * C.nxp;
        } else {
            int sx = x - cx, sy = y - cy;
            if (sx < 0) { if (C.per_x) sx += C.nx; else wall = true; }
            else if (sx >= C.nx) { if (C.per_x) sx -= C.nx; else wall = true; }
            if (sy < 0) { if (C.per_y) sy += C.ny; else wall = true; }
            else if (sy >= C.ny) { if (C.per_y) sy -= C.ny; else wall = true; }
            src = sy * C.nxp + sx;
        }
        if (solid && i != 0 && !wall) wall = solid[src] != 0;
        const int idx = wall ? opp<D2Q9>(i) * plane + own : i * plane + src;
        G[gpos<D2Q9>(i)] = (R)ld_cg<T>(f + idx);
    }
}

// sum of two doubles over the block (blockDim.x <= 256); thread 0 gets it
__device__ __forceinline__ void block_sum_batch(double (&v)[2]) {
    __shared__ double sh[8][2];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[wid][0] = v[0];
        sh[wid][1] = v[1];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += sh[w][0];
            b += sh[w][1];
        }
        v[0] = a;
        v[1] = b;
    }
}

// the channel's collision on one node's grid (R = double) or two nodes'
// (R = F2); SMRT with tau_3 = tau_4 = 1 takes the trimmed collision, as
// k_step does, and the bulk relaxes with tau_2
template <int COLL, typename R>
__device__ __forceinline__ void batch_collide(R *G, R gx, R gy, R om2, R om3, R om4, bool trim) {
    const R z = R(0);
    if constexpr (COLL == SMRT_TRIM) collide_smrt_trim<D2Q9>(G, gx, gy, z, om2);
    else if constexpr (COLL == SMRT) {
        if (trim) collide_smrt_trim<D2Q9>(G, gx, gy, z, om2);
        else collide_smrt<D2Q9>(G, gx, gy, z, om2, om3, om4, om2);
    } else if constexpr (COLL == SMRT_FNEQ) collide_smrt_fneq<D2Q9>(G, gx, gy, z, om2, om3, om4, om2);
    else if constexpr (COLL == MRT_RAW) collide_mrt_raw<D2Q9>(G, gx, gy, z, om2, om3, om4);
    else collide_bgk<D2Q9>(G, gx, gy, z, om2);
}

// One FP32 node of a channel on the pair instructions (both lanes), out of
// line: the node of a pass whose partner lies past the tile, so that the
// kernel keeps one inlined pair collision per collision kind
template <int COLL>
__device__ __noinline__ void batch_node_alone(const BatchChan C, const float *fin, float *fout,
                                              const unsigned char *solid, int x, int y, float gx, float gy,
                                              float om2, float om3, float om4, bool trim) {
    float G[9];
    gather_chan<ST_F32>(C, fin, solid, x, y, G);
    F2 G2[9];
#pragma unroll
    for (int g = 0; g < 9; ++g) G2[g] = F2(G[g]);
    batch_collide<COLL>(G2, F2(gx), F2(gy), F2(om2), F2(om3), F2(om4), trim);
    float *dst = fout + (y * C.nxp + x);
#pragma unroll
    for (int i = 0; i < 9; ++i) Store<ST_F32>::st(dst + i * (int)C.plane, G2[gpos<D2Q9>(i)].lo());
}

// tiles per step for a channel of nx x ny with `active` nodes still running
__host__ __device__ inline int tiles_for(int nx, int ny, long long active, int grid, int tile_min, int tile_max) {
    long long target = active / (2LL * grid);
    if (target < tile_min) target = tile_min;
    if (target > tile_max) target = tile_max;
    int rows = (int)((target + nx - 1) / nx);
    const int min_rows = (ny + kMaxTiles - 1) / kMaxTiles;
    if (rows < min_rows) rows = min_rows;
    if (rows < 1) rows = 1;
    if (rows > ny) rows = ny;
    return (ny + rows - 1) / rows;
}

// batch storage is FP32 or FP64 (loads through L2: ld.global.cg).  The
// launch bounds cap the kernel at 64 registers (no spills in FP32), so 8
// blocks of 128 threads share an SM instead of 6.
template <int COLL, int ST>
__global__ void __launch_bounds__(256, 4) k_batch(const BatchRun r) {
    typedef typename Store<ST>::T T;
    typedef typename Store<ST>::R R;
    __shared__ int s_c, s_tile, s_tiles, s_quit;
    __shared__ long long s_step;
    long long empty = 0;
    unsigned long long seen = 0;
    for (;;) {
        // warp 0 looks for a claimable tile: the active-channel bitmap is read
        // 32 words per load, the claim words of a word's channels in one round,
        // and the lowest-index (highest-priority) claimable channel is claimed
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            int fc = -1, ft = 0, fn = 0;
            long long fs = 0;
            const int nwords = (r.n + 31) >> 5;
            for (int wb = 0; wb < nwords && fc < 0; wb += 32) {
                const int wi = wb + lane;
                const unsigned bits = wi < nwords ? vload(r.active_bits + wi) : 0u;
                unsigned nz = __ballot_sync(0xffffffffu, bits != 0u);
                while (nz != 0u && fc < 0) {
                    const int src = __ffs(nz) - 1;
                    nz &= nz - 1u;
                    const unsigned wbits = __shfl_sync(0xffffffffu, bits, src);
                    const int c = (wb + src) * 32 + lane;
                    bool ok = (wbits >> lane) & 1u;
                    if (ok) {
                        const unsigned long long w = vload(&r.ctl[c].claim);
                        ok = (int)(w & kTileMask) < (int)((w >> kTileBits) & kTileMask);
                    }
                    unsigned m = __ballot_sync(0xffffffffu, ok);
                    while (m != 0u) {
                        const int pick = __ffs(m) - 1;
                        m &= m - 1u;
                        unsigned long long w2 = 0ull;
                        if (lane == pick) w2 = atomicAdd(&r.ctl[c].claim, 1ull);
                        w2 = __shfl_sync(0xffffffffu, w2, pick);
                        const int t2 = (int)(w2 & kTileMask), n2 = (int)((w2 >> kTileBits) & kTileMask);
                        if (t2 < n2) {
                            fc = (wb + src) * 32 + pick;
                            fs = (long long)(w2 >> (2 * kTileBits));
                            ft = t2;
                            fn = n2;
                            break;
                        }
                    }
                }
            }
            if (lane == 0) {
                s_c = fc;
                s_step = fs;
                s_tile = ft;
                s_tiles = fn;
                s_quit = 0;
                if (fc < 0) {
                    if (vload(r.active_count) == 0 || vload(r.error) != 0) {
                        s_quit = 1;
                    } else {
                        const unsigned long long pg = vload(r.progress);
                        if (pg != seen) {
                            seen = pg;
                            empty = 0;
                        } else if (++empty > r.spin_limit) {
                            atomicExch(r.error, (int)LBM_ERR_TIMEOUT);
                            s_quit = 1;
                        }
                        __nanosleep(100);
                    }
                } else {
                    empty = 0;
                }
                __threadfence();
            }
        }
        __syncthreads();
        if (s_quit) break;
        const int c = s_c;
        if (c >= 0) {
            const BatchChan C = r.ch[c];
            const long long step = s_step;
            const int tile = s_tile;
            const int ntiles = s_tiles;
            const int rows = (C.ny + ntiles - 1) / ntiles;
            const T *fin = (const T *)((step & 1) ? r.fb : r.fa) + C.off;
            T *fout = (T *)((step & 1) ? r.fa : r.fb) + C.off;
            const long long start = r.ctl[c].start;
            const bool check = ((step - start) % r.K) == 0;
            const int y0 = tile * rows;
            const int y1 = min(y0 + rows, C.ny);
            const int nn = y1 > y0 ? (y1 - y0) * C.nx : 0;  // the last tiles may be empty
            R *snap = (R *)r.snap + C.snap_off;
            const unsigned char *solid = C.solid_off >= 0 ? r.solid + C.solid_off : nullptr;
            const int N = C.nx * C.ny;
            const R om2 = R(C.om2), om3 = R(C.om3), om4 = R(C.om4), gx = R(C.gx), gy = R(C.gy);
            const bool trim = C.om3 == 1.0 && C.om4 == 1.0;
            double v[2] = {0.0, 0.0};
            // two nodes per thread per pass, all loads issued first.  The
            // tile's nodes are numbered row by row; a thread's two nodes
            // (numbers base and base + blockDim.x) advance by 2 blockDim.x a
            // pass, i.e. by (dy, dx) rows and columns with one carry, so no
            // node needs a division
            const int stride = 2 * (int)blockDim.x;
            const int step_dy = stride / C.nx, step_dx = stride - step_dy * C.nx;
            int xs[2], ys[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int idx = (int)threadIdx.x + k * (int)blockDim.x;
                const int yy = idx / C.nx;
                xs[k] = idx - yy * C.nx;
                ys[k] = y0 + yy;
            }
            for (int base = threadIdx.x; base < nn; base += stride) {
                R G[2][9];
                bool on[2];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    on[k] = base + k * (int)blockDim.x < nn;
                    if (on[k] && solid) on[k] = solid[ys[k] * C.nxp + xs[k]] == 0;
                    if (on[k]) gather_chan<ST>(C, fin, solid, xs[k], ys[k], G[k]);
                }
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (!on[k]) continue;
                    const int x = xs[k], y = ys[k];
                    if (check) {
                        R drho = 0, jx = 0, jy = 0;
#pragma unroll
                        for (int i = 0; i < 9; ++i) {
                            const R w = G[k][gpos<D2Q9>(i)];
                            drho += w;
                            jx += Lat<D2Q9>::cx(i) * w;
                            jy += Lat<D2Q9>::cy(i) * w;
                        }
                        const R rho = R(1) + drho;
                        const R ux = jx / rho + R(0.5) * gx, uy = jy / rho + R(0.5) * gy;
                        const int n = y * C.nx + x;
                        const R dx = ux - ld_cg<R>(snap + n), dy = uy - ld_cg<R>(snap + N + n);
                        v[0] += (double)(dx * dx + dy * dy);
                        v[1] += (double)(ux * ux + uy * uy);
                        snap[n] = ux;
                        snap[N + n] = uy;
                    }
                }
                if constexpr (ST == ST_F32) {
                    if (on[0] && on[1]) {
                        // both nodes: one collision in packed FP32, as k_step
                        // pairs its nodes
                        F2 G2[9];
#pragma unroll
                        for (int g = 0; g < 9; ++g) G2[g] = F2::pair(G[0][g], G[1][g]);
                        batch_collide<COLL>(G2, F2(gx), F2(gy), F2(om2), F2(om3), F2(om4), trim);
                        T *d0 = fout + (ys[0] * C.nxp + xs[0]), *d1 = fout + (ys[1] * C.nxp + xs[1]);
#pragma unroll
                        for (int i = 0; i < 9; ++i) {
                            Store<ST>::st(d0 + i * (int)C.plane, G2[gpos<D2Q9>(i)].lo());
                            Store<ST>::st(d1 + i * (int)C.plane, G2[gpos<D2Q9>(i)].hi());
                        }
                    } else {
                        // a node alone (the tile's last pass): out of line
                        if (on[0]) batch_node_alone<COLL>(C, fin, fout, solid, xs[0], ys[0], gx, gy, om2, om3, om4, trim);
                        if (on[1]) batch_node_alone<COLL>(C, fin, fout, solid, xs[1], ys[1], gx, gy, om2, om3, om4, trim);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        if (!on[k]) continue;
                        const int x = xs[k], y = ys[k];
                        batch_collide<COLL>(G[k], gx, gy, om2, om3, om4, trim);
                        T *dst = fout + (y * C.nxp + x);
#pragma unroll
                        for (int i = 0; i < 9; ++i) Store<ST>::st(dst + i * (int)C.plane, G[k][gpos<D2Q9>(i)]);
                    }
                }
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    xs[k] += step_dx;
                    ys[k] += step_dy;
                    if (xs[k] >= C.nx) {
                        xs[k] -= C.nx;
                        ++ys[k];
                    }
                }
            }
            if (check) {
                block_sum_batch(v);
                if (threadIdx.x == 0) {
                    r.part[C.part_off + 2 * tile + 0] = v[0];
                    r.part[C.part_off + 2 * tile + 1] = v[1];
                }
            }
            // every thread orders its stores (populations, snapshot) at GPU
            // scope before the tile is counted done
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                const unsigned prev = atomicAdd(&r.ctl[c].done, 1u);
                if (prev == (unsigned)(ntiles - 1)) {
                    // last tile of this step: close it
                    __threadfence();
                    const long long done_steps = step + 1;
                    bool retire = false;
                    int status = 0;
                    if (check && step > start) {
                        double num = 0.0, den = 0.0;
                        for (int t = 0; t < ntiles; ++t) {
                            num += ld_cg<double>(r.part + C.part_off + 2 * t);
                            den += ld_cg<double>(r.part + C.part_off + 2 * t + 1);
                        }
                        const double rr = den > 0.0 ? sqrt(num) / ((double)r.K * sqrt(den)) : (num > 0.0 ? INFINITY : 0.0);
                        r.ctl[c].r = rr;
                        if (!isfinite(num) || !isfinite(den)) {
                            retire = true;
                            status = (int)LBM_ERR_UNSTABLE;
                        } else if (r.tol >= 0.0 && rr <= r.tol) {
                            retire = true;
                            status = (int)LBM_OK;
                        }
                    }
                    if (!retire && done_steps - start >= r.max_steps) {
                        retire = true;
                        status = r.tol >= 0.0 ? (int)LBM_NOT_CONVERGED : (int)LBM_OK;
                    }
                    r.ctl[c].steps = done_steps;
                    atomicExch(&r.ctl[c].done, 0u);
                    // the tail: few channels left, each would take a whole
                    // scheduling round per step here; they leave at this step
                    // boundary and the host continues them as plain lattices
                    const bool park = !retire && r.park_below > 0 && vload(r.active_count) <= r.park_below;
                    if (retire || park) {
                        if (retire) r.ctl[c].status = status;
                        else r.ctl[c].parked = 1;
                        __threadfence();
                        atomicExch(&r.ctl[c].active, 0);
                        atomicAnd(r.active_bits + (c >> 5), ~(1u << (c & 31)));
                        atomicAdd((unsigned long long *)r.active_nodes, (unsigned long long)(-(long long)C.nx * C.ny));
                        atomicSub(r.active_count, 1);
                    } else {
                        const int nt = tiles_for(C.nx, C.ny, vload(r.active_nodes), r.grid, r.tile_min, r.tile_max);
                        __threadfence();
                        atomicExch(&r.ctl[c].claim, claim_word(done_steps, nt));
                    }
                    atomicAdd(r.progress, 1ull);
                }
            }
        }
        __syncthreads();
    }
}

// start of a run: every channel active from its current step
__global__ void k_batch_reset(BatchRun r, long long total_nodes) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < r.n) {
        BatchCtl *ctl = r.ctl;
        const long long s = ctl[c].steps;
        ctl[c].claim = claim_word(s, tiles_for(r.ch[c].nx, r.ch[c].ny, total_nodes, r.grid, r.tile_min, r.tile_max));
        ctl[c].done = 0u;
        ctl[c].active = 1;
        ctl[c].start = s;
        ctl[c].status = 1;
        ctl[c].r = -1.0;
        ctl[c].parked = 0;
        atomicOr(r.active_bits + (c >> 5), 1u << (c & 31));
    }
    if (c == 0) {
        *r.active_count = r.n;
        *r.active_nodes = total_nodes;
        *r.progress = 0ull;
        *r.error = 0;
    }
}

}  // namespace lbm

// ----------------------------------------------------------------- host side
struct lbm_batch {
    int n = 0;
    int collision = 0, storage = 0;
    std::vector<lbm_desc> desc;
    std::vector<KParams> kp;    // per channel, pointing into the arenas
    std::vector<BatchChan> ch;
    std::vector<long long> steps;
    void *fa = nullptr, *fb = nullptr, *snap = nullptr;
    double *part = nullptr;
    double *g_dev = nullptr;    // per channel 4 doubles
    float *g32_dev = nullptr;   // per channel 4 floats
    double *fields = nullptr;   // initial rho0 / u0, per channel, when given
    unsigned char *solid = nullptr;  // obstacle masks of the channels that have one
    std::vector<long long> field_off;
    BatchChan *ch_dev = nullptr;
    BatchCtl *ctl_dev = nullptr;
    int *active_count = nullptr, *error = nullptr;
    unsigned long long *progress = nullptr;
    long long *active_nodes = nullptr;
    unsigned *active_bits = nullptr;
    long long total_nodes = 0;
    std::vector<int> order;     // position -> channel index given by the caller
    std::vector<int> pos_of;    // channel index -> position (priority order)
    int last_grid = 0;
    double *partials = nullptr, *red = nullptr, *tmp = nullptr;
    size_t tmp_bytes = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int block = 128, tile_nodes = 2048;
    int handoff = 8;           // channels left when the tail moves to plain lattices (0: never)
    long long spin_limit = 1ll << 26;
    size_t arena_elems = 0;
    std::string err;
};

namespace {

size_t elem_bytes(int st) { return st == LBM_F64 ? 8 : 4; }

lbm_status bfail(lbm_batch *b, lbm_status st, const std::string &m) {
    if (b) b->err = m;
    set_thread_error(m.c_str());
    return st;
}

#define B_CUDA(b, call)                                                                       \
    do {                                                                                      \
        cudaError_t e__ = (call);                                                             \
        if (e__ != cudaSuccess)                                                               \
            return bfail((b), e__ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,  \
                         std::string(#call) + ": " + cudaGetErrorString(e__));                \
    } while (0)

// a blocking copy in the batch stream's order: the stream need not
// synchronise with the legacy default stream, and a plain cudaMemcpy from
// pageable memory may return before its data reaches the device
cudaError_t bcopy(lbm_batch *b, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, b->stream);
    return e == cudaSuccess ? cudaStreamSynchronize(b->stream) : e;
}

template <typename T>
lbm_status balloc(lbm_batch *b, T **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *q = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, LBM_ERR_OOM, "device allocation failed");
    }
    *p = (T *)q;
    return LBM_OK;
}

lbm_status build_tiles(lbm_batch *b) {
    long long part_off = 0;
    b->total_nodes = 0;
    for (int c = 0; c < b->n; ++c) {
        BatchChan &C = b->ch[c];
        C.part_off = part_off;
        part_off += 2LL * C.ny;  // room for the finest tiling (one row per tile)
        b->total_nodes += (long long)C.nx * C.ny;
    }
    B_CUDA(b, cudaMemcpyAsync(b->ch_dev, b->ch.data(), sizeof(BatchChan) * b->n, cudaMemcpyHostToDevice, b->stream));
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

typedef void (*BatchKernel)(const BatchRun);

// SMRT with every channel at tau_3 = tau_4 = 1 takes the kernel built for the
// trimmed collision alone
BatchKernel batch_kernel(int coll, int st, bool all_trim) {
    if (coll == LBM_SMRT && all_trim) return st == LBM_F64 ? k_batch<SMRT_TRIM, ST_F64> : k_batch<SMRT_TRIM, ST_F32>;
    if (coll == LBM_SMRT) return st == LBM_F64 ? k_batch<SMRT, ST_F64> : k_batch<SMRT, ST_F32>;
    if (coll == LBM_SMRT_FNEQ) return st == LBM_F64 ? k_batch<SMRT_FNEQ, ST_F64> : k_batch<SMRT_FNEQ, ST_F32>;
    if (coll == LBM_MRT_RAW) return st == LBM_F64 ? k_batch<MRT_RAW, ST_F64> : k_batch<MRT_RAW, ST_F32>;
    return st == LBM_F64 ? k_batch<BGK, ST_F64> : k_batch<BGK, ST_F32>;
}

bool all_trim(const lbm_batch *b) {
    for (const BatchChan &C : b->ch)
        if (!(C.om3 == 1.0 && C.om4 == 1.0)) return false;
    return true;
}

// one run: reset + persistent kernel, captured in a graph and launched once
lbm_status batch_run(lbm_batch *b, double tol, int K, int64_t max_steps) {
    BatchKernel kern = batch_kernel(b->collision, b->storage, all_trim(b));
    int dev = 0, sms = 0, per_sm = 0;
    B_CUDA(b, cudaGetDevice(&dev));
    B_CUDA(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    B_CUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, b->block, 0));
    if (per_sm < 1) return bfail(b, LBM_ERR_ARG, "batch block size does not fit on an SM");
    BatchRun r;
    r.ch = b->ch_dev;
    r.ctl = b->ctl_dev;
    r.n = b->n;
    r.solid = b->solid;
    // at most 4000 CTAs: the tile field of the claim word overshoots the tile
    // count (<= 4096) by at most the number of concurrent claimers (< 8192 - 4096)
    r.grid = std::min(sms * per_sm, 4000);
    r.tile_min = 2 * b->block;
    r.tile_max = std::max(b->tile_nodes, 2 * b->block);
    r.active_nodes = b->active_nodes;
    r.active_bits = b->active_bits;
    b->last_grid = r.grid;
    r.fa = b->fa;
    r.fb = b->fb;
    r.snap = b->snap;
    r.part = b->part;
    r.active_count = b->active_count;
    r.progress = b->progress;
    r.error = b->error;
    r.tol = tol;
    r.park_below = tol >= 0.0 ? b->handoff : 0;
    r.K = K;
    r.max_steps = max_steps;
    r.spin_limit = b->spin_limit;
    const int grid = r.grid;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    B_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(b->active_bits, 0, (size_t)((b->n + 31) / 32) * 4, b->stream);
    k_batch_reset<<<(b->n + 127) / 128, 128, 0, b->stream>>>(r, b->total_nodes);
    kern<<<grid, b->block, 0, b->stream>>>(r);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    e = cudaGraphLaunch(ge, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaGraphExecDestroy(ge);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("batch run: ") + cudaGetErrorString(e));
    int errflag = 0;
    B_CUDA(b, bcopy(b, &errflag, b->error, sizeof(int), cudaMemcpyDeviceToHost));
    std::vector<BatchCtl> ctl(b->n);
    B_CUDA(b, bcopy(b, ctl.data(), b->ctl_dev, sizeof(BatchCtl) * b->n, cudaMemcpyDeviceToHost));
    for (int c = 0; c < b->n; ++c) b->steps[c] = ctl[c].steps;
    if (errflag) return bfail(b, (lbm_status)errflag, "batch kernel stopped: no progress within the scan limit");
    return LBM_OK;
}

lbm_status init_channels(lbm_batch *b) {
    const Launchers &L = launchers_d2q9();
    std::vector<BatchCtl> ctl(b->n);
    for (int c = 0; c < b->n; ++c) {
        const lbm_desc &d = b->desc[c];
        const double *rho0 = d.rho0 ? b->fields + b->field_off[c] : nullptr;
        const double *u0 = d.u0 ? b->fields + b->field_off[c] + (size_t)d.nx * d.ny : nullptr;
        const size_t eb = elem_bytes(b->storage);
        void *A = (char *)b->fa + b->ch[c].off * eb;
        void *B = (char *)b->fb + b->ch[c].off * eb;
        const bool mask = b->kp[c].solid != nullptr;
        cudaError_t e = L.init(b->collision, b->storage, mask, b->kp[c], rho0, u0, B, b->stream);
        if (e == cudaSuccess) e = L.unstream(b->storage, mask, b->kp[c], B, A, b->stream);
        if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("batch init: ") + cudaGetErrorString(e));
        b->steps[c] = 0;
        ctl[c] = BatchCtl{};
    }
    size_t snap_elems = 0;
    for (int c = 0; c < b->n; ++c) snap_elems += 2ull * b->ch[c].nx * b->ch[c].ny;
    B_CUDA(b, cudaMemsetAsync(b->snap, 0, snap_elems * elem_bytes(b->storage), b->stream));
    B_CUDA(b, cudaMemcpyAsync(b->ctl_dev, ctl.data(), sizeof(BatchCtl) * b->n, cudaMemcpyHostToDevice, b->stream));
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

const void *channel_state(const lbm_batch *b, int c) {
    const size_t eb = elem_bytes(b->storage);
    return (const char *)((b->steps[c] & 1) ? b->fb : b->fa) + b->ch[c].off * eb;
}

// Continue the channels that parked in the tail of a run, each as a plain
// lattice (its own handle and stream, graph-launched steps), all of them
// concurrently, with the batch's residual cadence and rules:
//  - a check at every step s with (s - start) % K == 0 and s - start below
//    max_steps, r = |u(s) - u(s - K)| / (K |u(s)|) over the fluid nodes;
//  - r <= tol: converged, and (as in the kernel, which finishes the step it
//    checked) one more step; non-finite: unstable, likewise;
//  - s - start reaching max_steps: not converged.
// The final state goes back into the batch's arena, so the channel reads
// as if the kernel had run it to the end.
lbm_status run_parked(lbm_batch *b, double tol, int K, int64_t max_steps) {
    std::vector<BatchCtl> ctl(b->n);
    B_CUDA(b, bcopy(b, ctl.data(), b->ctl_dev, sizeof(BatchCtl) * b->n, cudaMemcpyDeviceToHost));
    struct Run {
        int p;
        lbm_handle *h;
        int64_t s0;      // step of the velocity snapshot (the last check)
        bool running;
        bool check;      // a check was issued this round
    };
    std::vector<Run> runs;
    for (int p = 0; p < b->n; ++p)
        if (ctl[p].parked) runs.push_back({p, nullptr, 0, true, false});
    if (runs.empty()) return LBM_OK;
    const size_t eb = elem_bytes(b->storage);
    double *red = nullptr;
    lbm_status st = balloc(b, &red, runs.size() * 8 * sizeof(double));
    auto cleanup = [&]() {
        for (Run &q : runs)
            if (q.h) lbm_destroy(q.h);
        if (red) cudaFree(red);
    };
    if (st != LBM_OK) return st;
    for (Run &q : runs) {
        const int p = q.p;
        const BatchChan &C = b->ch[p];
        lbm_desc d = b->desc[p];
        double g[3] = {C.gx, C.gy, 0.0};
        d.g = d.force_kind == LBM_G_UNIFORM ? g : nullptr;
        std::vector<unsigned char> mask;
        if (C.solid_off >= 0) {
            std::vector<unsigned char> pad((size_t)C.plane);
            cudaError_t e = bcopy(b, pad.data(), b->solid + C.solid_off, (size_t)C.plane, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                cleanup();
                return bfail(b, LBM_ERR_CUDA, std::string("handoff mask: ") + cudaGetErrorString(e));
            }
            mask.resize((size_t)C.nx * C.ny);
            for (int y = 0; y < C.ny; ++y)
                for (int x = 0; x < C.nx; ++x) mask[(size_t)y * C.nx + x] = pad[(size_t)y * C.nxp + x];
            d.solid = mask.data();
        } else {
            d.solid = nullptr;
        }
        d.rho0 = d.u0 = nullptr;
        d.stream = nullptr;
        d.alloc = nullptr;
        d.free_ = nullptr;
        d.alloc_ctx = nullptr;
        if ((st = lbm_create(&d, &q.h)) != LBM_OK) {
            q.h = nullptr;
            cleanup();
            return bfail(b, st, std::string("handoff: ") + lbm_last_error(nullptr));
        }
        const long long steps = ctl[p].steps, start = ctl[p].start;
        q.s0 = start + (long long)K * ((steps - 1 - start) / K);
        st = handle_adopt(q.h, channel_state(b, p), (const char *)b->snap + C.snap_off * eb, steps, q.s0);
        if (st != LBM_OK) {
            cleanup();
            return bfail(b, st, "handoff: state copy failed");
        }
    }
    int left = (int)runs.size();
    while (left > 0) {
        for (size_t k = 0; k < runs.size(); ++k) {
            Run &q = runs[k];
            if (!q.running) continue;
            const long long start = ctl[q.p].start, steps = b->steps[q.p] = ctl[q.p].steps;
            const long long next = q.s0 + K, end = start + max_steps;
            const long long target = std::min(next, end);
            q.check = target == next && next - start < max_steps;
            st = lbm_step(q.h, target - steps);
            if (st == LBM_OK && q.check) st = lbm_check_device(q.h, red + 8 * k);
            if (st != LBM_OK) {
                cleanup();
                return bfail(b, st, "handoff: step failed");
            }
            ctl[q.p].steps = target;
        }
        for (size_t k = 0; k < runs.size(); ++k) {
            Run &q = runs[k];
            if (!q.running) continue;
            double v[8] = {0};
            cudaError_t e = cudaStreamSynchronize(handle_stream(q.h));
            if (e == cudaSuccess && q.check) e = bcopy(b, v, red + 8 * k, 7 * sizeof(double), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                cleanup();
                return bfail(b, LBM_ERR_CUDA, std::string("handoff: ") + cudaGetErrorString(e));
            }
            BatchCtl &c = ctl[q.p];
            bool finish = false, extra = false;
            if (q.check) {
                q.s0 = c.steps;
                const double rr = v[5] > 0.0 ? sqrt(v[4]) / ((double)K * sqrt(v[5])) : (v[4] > 0.0 ? INFINITY : 0.0);
                c.r = rr;
                if (v[6] > 0.0 || !std::isfinite(v[4]) || !std::isfinite(v[5])) {
                    c.status = (int)LBM_ERR_UNSTABLE;
                    finish = extra = true;
                } else if (rr <= tol) {
                    c.status = (int)LBM_OK;
                    finish = extra = true;
                }
            }
            if (!finish && c.steps - c.start >= max_steps) {
                c.status = (int)LBM_NOT_CONVERGED;
                finish = true;
            }
            if (!finish) continue;
            if (extra) {
                if ((st = lbm_step(q.h, 1)) != LBM_OK) {
                    cleanup();
                    return bfail(b, st, "handoff: step failed");
                }
                c.steps += 1;
            }
            void *dst = (char *)((c.steps & 1) ? b->fb : b->fa) + b->ch[q.p].off * eb;
            st = handle_export_state(q.h, dst);
            e = st == LBM_OK ? cudaStreamSynchronize(handle_stream(q.h)) : cudaErrorUnknown;
            if (e != cudaSuccess) {
                cleanup();
                return bfail(b, LBM_ERR_CUDA, "handoff: state copy back failed");
            }
            b->steps[q.p] = c.steps;
            c.parked = 0;
            c.active = 0;
            lbm_destroy(q.h);
            q.h = nullptr;
            q.running = false;
            --left;
        }
    }
    cleanup();
    B_CUDA(b, bcopy(b, b->ctl_dev, ctl.data(), sizeof(BatchCtl) * b->n, cudaMemcpyHostToDevice));
    return LBM_OK;
}

lbm_status ensure_tmp(lbm_batch *b, size_t bytes) {
    if (b->tmp_bytes >= bytes) return LBM_OK;
    if (b->tmp) cudaFree(b->tmp);
    b->tmp = nullptr;
    b->tmp_bytes = 0;
    lbm_status st = balloc(b, &b->tmp, bytes);
    if (st == LBM_OK) b->tmp_bytes = bytes;
    return st;
}

}  // namespace

extern "C" {

void lbm_batch_destroy(lbm_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    void *ptrs[] = {b->fa,      b->fb,       b->snap,         b->part,  b->g_dev,    b->g32_dev,
                    b->fields,  b->ch_dev,   b->ctl_dev,      b->active_count, b->error, b->progress,
                    b->active_nodes, b->active_bits, b->partials, b->red, b->tmp, b->solid};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

lbm_status lbm_batch_create(const lbm_desc *descs, int n, lbm_batch **out) {
    if (!out) return bfail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!descs || n < 1) return bfail(nullptr, LBM_ERR_ARG, "need at least one description");
    const lbm_desc &d0 = descs[0];
    if (d0.lattice != LBM_D2Q9) return bfail(nullptr, LBM_ERR_ARG, "batches are D2Q9");
    if (d0.storage != LBM_F32 && d0.storage != LBM_F64) return bfail(nullptr, LBM_ERR_ARG, "batch storage is F32 or F64");
    if (d0.collision < LBM_BGK || d0.collision > LBM_MRT_RAW) return bfail(nullptr, LBM_ERR_ARG, "bad collision");
    for (int c = 0; c < n; ++c) {
        const lbm_desc &d = descs[c];
        if (d.lattice != d0.lattice || d.collision != d0.collision || d.storage != d0.storage)
            return bfail(nullptr, LBM_ERR_ARG, "channels must share lattice, collision and storage");
        if (d.nx < 1 || d.ny < 1 || d.nz != 1 || d.ny > 65535) return bfail(nullptr, LBM_ERR_ARG, "bad channel sizes");
        if (d.force_kind != LBM_G_NONE && d.force_kind != LBM_G_UNIFORM)
            return bfail(nullptr, LBM_ERR_ARG, "batch channels take a uniform force or none");
        if (d.force_kind == LBM_G_UNIFORM && !d.g) return bfail(nullptr, LBM_ERR_ARG, "force values are NULL");
        if (d.collision == LBM_BGK && !(d.tau[2] > 0.5)) return bfail(nullptr, LBM_ERR_ARG, "tau[2] must be > 1/2");
        if (d.tau_bulk != 0.0 && d.tau_bulk != d.tau[2])
            return bfail(nullptr, LBM_ERR_ARG, "batches relax the second order with one tau (tau_bulk 0 or tau[2])");
        if (d.collision != LBM_BGK)
            for (int k = 2; k <= 4; ++k)
                if (!(d.tau[k] > 0.5)) return bfail(nullptr, LBM_ERR_ARG, "tau[2..4] must be > 1/2");
    }
    lbm_batch *b = new lbm_batch();
    b->n = n;
    b->collision = d0.collision;
    b->storage = d0.storage;
    // priority order: longest diffusive time scale L^2 / nu first (L: the
    // extent between walls, else the largest extent), so that the channels
    // needing the most steps are always served first
    b->order.resize(n);
    b->pos_of.resize(n);
    {
        std::vector<std::pair<double, int>> key(n);
        for (int c = 0; c < n; ++c) {
            const lbm_desc &d = descs[c];
            const double L = !d.periodic[1] ? d.ny : (!d.periodic[0] ? d.nx : std::max(d.nx, d.ny));
            const double nu = (d.tau[2] - 0.5) / 3.0;
            key[c] = {-(L * L / nu), c};
        }
        std::stable_sort(key.begin(), key.end());
        for (int p = 0; p < n; ++p) {
            b->order[p] = key[p].second;
            b->pos_of[key[p].second] = p;
        }
    }
    b->desc.resize(n);
    for (int p = 0; p < n; ++p) b->desc[p] = descs[b->order[p]];
    descs = b->desc.data();
    b->ch.resize(n);
    b->kp.resize(n);
    b->steps.assign(n, 0);
    b->field_off.assign(n, 0);
    lbm_status st = LBM_OK;
    if (d0.stream) {
        b->stream = (cudaStream_t)d0.stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return bfail(nullptr, LBM_ERR_CUDA, "cudaStreamCreate failed");
        }
        b->own_stream = true;
    }
    long long off = 0, snap_off = 0, parts = 0, fields = 0, solid_bytes = 0;
    for (int c = 0; c < n; ++c) {
        const lbm_desc &d = descs[c];
        BatchChan &C = b->ch[c];
        C.nx = d.nx;
        C.ny = d.ny;
        C.nxp = (d.nx + 31) / 32 * 32;
        C.plane = (long long)C.nxp * d.ny;
        C.off = off;
        off += 9LL * C.plane;
        C.snap_off = snap_off;
        snap_off += 2LL * d.nx * d.ny;
        parts += 2LL * d.ny;
        C.per_x = d.periodic[0] ? 1 : 0;
        C.per_y = d.periodic[1] ? 1 : 0;
        C.om2 = 1.0 / d.tau[2];
        C.om3 = d.collision != LBM_BGK ? 1.0 / d.tau[3] : 0.0;
        C.om4 = d.collision != LBM_BGK ? 1.0 / d.tau[4] : 0.0;
        C.gx = d.force_kind == LBM_G_UNIFORM ? d.g[0] : 0.0;
        C.gy = d.force_kind == LBM_G_UNIFORM ? d.g[1] : 0.0;
        b->field_off[c] = fields;
        if (d.rho0 || d.u0) fields += 3LL * d.nx * d.ny;
        C.solid_off = d.solid ? solid_bytes : -1;
        if (d.solid) solid_bytes += C.plane;
    }
    b->arena_elems = (size_t)off;
    const size_t eb = elem_bytes(b->storage);
    if ((st = balloc(b, &b->fa, (size_t)off * eb)) || (st = balloc(b, &b->fb, (size_t)off * eb)) ||
        (st = balloc(b, &b->snap, (size_t)snap_off * eb)) || (st = balloc(b, &b->part, (size_t)parts * 8)) ||
        (st = balloc(b, &b->g_dev, (size_t)n * 4 * 8)) || (st = balloc(b, &b->g32_dev, (size_t)n * 4 * 4)) ||
        (st = balloc(b, &b->ch_dev, sizeof(BatchChan) * n)) || (st = balloc(b, &b->ctl_dev, sizeof(BatchCtl) * n)) ||
        (st = balloc(b, &b->active_count, 16)) || (st = balloc(b, &b->error, 16)) ||
        (st = balloc(b, &b->progress, 16)) || (st = balloc(b, &b->active_nodes, 16)) ||
        (st = balloc(b, &b->active_bits, (size_t)((n + 31) / 32) * 4)) ||
        (st = balloc(b, &b->partials, (size_t)kMomGridMax * kPartials * 8)) || (st = balloc(b, &b->red, 64)) ||
        (fields && (st = balloc(b, &b->fields, (size_t)fields * 8))) ||
        (solid_bytes && (st = balloc(b, &b->solid, (size_t)solid_bytes)))) {
        std::string m = b->err;
        lbm_batch_destroy(b);
        return bfail(nullptr, st, m);
    }
    // per-channel force copies and launch parameters for the shared kernels
    std::vector<double> g(4 * (size_t)n, 0.0);
    std::vector<float> g32(4 * (size_t)n, 0.f);
    for (int c = 0; c < n; ++c) {
        g[4 * c + 0] = b->ch[c].gx;
        g[4 * c + 1] = b->ch[c].gy;
        g32[4 * c + 0] = (float)b->ch[c].gx;
        g32[4 * c + 1] = (float)b->ch[c].gy;
        const lbm_desc &d = descs[c];
        KParams &k = b->kp[c];
        k = KParams{};
        k.nx = d.nx;
        k.ny = d.ny;
        k.nz = 1;
        k.nxp = b->ch[c].nxp;
        k.plane = b->ch[c].plane;
        k.per[0] = b->ch[c].per_x;
        k.per[1] = b->ch[c].per_y;
        k.per[2] = 1;
        k.force_kind = d.force_kind == LBM_G_UNIFORM ? G_UNIFORM : G_NONE;
        k.solid = d.solid ? b->solid + b->ch[c].solid_off : nullptr;
        k.g = b->g_dev + 4 * c;
        k.g32 = b->g32_dev + 4 * c;
        for (int m = 0; m < 5; ++m) {
            k.om[m] = d.tau[m] > 0.0 ? 1.0 / d.tau[m] : 0.0;
            k.om32[m] = (float)k.om[m];
        }
        fill_offsets<D2Q9>(k);
    }
    cudaError_t e = cudaMemcpyAsync(b->g_dev, g.data(), g.size() * 8, cudaMemcpyHostToDevice, b->stream);
    for (int c = 0; c < n && e == cudaSuccess; ++c) {
        const lbm_desc &d = descs[c];
        if (!d.solid) continue;
        std::vector<unsigned char> m((size_t)b->ch[c].plane, 0);
        for (int y = 0; y < d.ny; ++y)
            for (int x = 0; x < d.nx; ++x) m[(size_t)y * b->ch[c].nxp + x] = d.solid[(size_t)y * d.nx + x] ? 1 : 0;
        e = cudaMemcpyAsync(b->solid + b->ch[c].solid_off, m.data(), m.size(), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->g32_dev, g32.data(), g32.size() * 4, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->fa, 0, (size_t)off * eb, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->fb, 0, (size_t)off * eb, b->stream);
    for (int c = 0; c < n && e == cudaSuccess; ++c) {
        const lbm_desc &d = descs[c];
        const size_t N = (size_t)d.nx * d.ny;
        if (d.rho0 || d.u0) {
            std::vector<double> f(3 * N, 0.0);
            for (size_t i = 0; i < N; ++i) f[i] = d.rho0 ? d.rho0[i] : 1.0;
            if (d.u0)
                for (size_t i = 0; i < 2 * N; ++i) f[N + i] = d.u0[i];
            e = cudaMemcpyAsync(b->fields + b->field_off[c], f.data(), f.size() * 8, cudaMemcpyHostToDevice, b->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        lbm_batch_destroy(b);
        return bfail(nullptr, LBM_ERR_CUDA, std::string("batch upload: ") + cudaGetErrorString(e));
    }
    if ((st = build_tiles(b)) != LBM_OK || (st = init_channels(b)) != LBM_OK) {
        std::string m = b->err;
        lbm_batch_destroy(b);
        return bfail(nullptr, st, m);
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_reset(lbm_batch *b) {
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
    return init_channels(b);
}

lbm_status lbm_batch_set_tiles(lbm_batch *b, int block, int tile_nodes) {
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
    if (!(block == 64 || block == 128 || block == 256)) return bfail(b, LBM_ERR_ARG, "block must be 64, 128 or 256");
    if (tile_nodes < 32 || tile_nodes > (1 << 20)) return bfail(b, LBM_ERR_ARG, "tile_nodes out of range");
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    b->block = block;
    b->tile_nodes = tile_nodes;
    return build_tiles(b);
}

lbm_status lbm_batch_set_spin_limit(lbm_batch *b, int64_t scans) {
    if (!b || scans < 1) return bfail(b, LBM_ERR_ARG, "bad spin limit");
    b->spin_limit = scans;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch *b, int64_t nsteps) {
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
    if (nsteps < 0) return bfail(b, LBM_ERR_ARG, "nsteps < 0");
    if (nsteps == 0) return LBM_OK;
    return batch_run(b, -1.0, 1 << 30, nsteps);
}

lbm_status lbm_batch_run_to_steady(lbm_batch *b, double tol, int K, int64_t max_steps, int64_t *steps_out,
                                   int *st_out, double *r_out) {
    if (!b) return bfail(nullptr, LBM_ERR_ARG, "batch is NULL");
    if (!(tol >= 0.0) || K < 1 || max_steps < 1) return bfail(b, LBM_ERR_ARG, "need tol >= 0, K >= 1, max_steps >= 1");
    lbm_status st = batch_run(b, tol, K, max_steps);
    if (st != LBM_OK && st != LBM_ERR_TIMEOUT) return st;
    if (st == LBM_OK && (st = run_parked(b, tol, K, max_steps)) != LBM_OK) return st;
    std::vector<BatchCtl> ctl(b->n);
    B_CUDA(b, bcopy(b, ctl.data(), b->ctl_dev, sizeof(BatchCtl) * b->n, cudaMemcpyDeviceToHost));
    for (int p = 0; p < b->n; ++p) {
        const int c = b->order[p];
        if (steps_out) steps_out[c] = ctl[p].steps;
        if (st_out) st_out[c] = ctl[p].status;
        if (r_out) r_out[c] = ctl[p].r;
    }
    return st;
}

lbm_status lbm_batch_set_handoff(lbm_batch *b, int channels) {
    if (!b || channels < 0) return bfail(b, LBM_ERR_ARG, "need a batch and channels >= 0");
    b->handoff = channels;
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch *b, int steps, int *block, int *tile_nodes, double *ms) {
    if (!b || steps < 1) return bfail(b, LBM_ERR_ARG, "bad arguments");
    // the largest tile (used while many channels run); tiles shrink on their
    // own as channels retire
    static const int blocks[] = {64, 128, 256};
    static const int tiles[] = {1024, 2048, 4096, 8192};
    cudaEvent_t e0, e1;
    B_CUDA(b, cudaEventCreate(&e0));
    B_CUDA(b, cudaEventCreate(&e1));
    double best = 1e300;
    int bb = b->block, bt = b->tile_nodes;
    lbm_status st = LBM_OK;
    for (int bl : blocks)
        for (int tn : tiles) {
            if ((st = lbm_batch_set_tiles(b, bl, tn)) != LBM_OK) break;
            if (cudaEventRecord(e0, b->stream) != cudaSuccess) { st = LBM_ERR_CUDA; break; }
            if ((st = lbm_batch_step(b, steps)) != LBM_OK) break;
            float t = 0.f;
            if (cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
                st = LBM_ERR_CUDA;
                break;
            }
            if (t < best) {
                best = t;
                bb = bl;
                bt = tn;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LBM_OK) return st;
    if ((st = lbm_batch_set_tiles(b, bb, bt)) != LBM_OK) return st;
    if ((st = init_channels(b)) != LBM_OK) return st;  // tuning advanced the state: start again
    if (block) *block = bb;
    if (tile_nodes) *tile_nodes = bt;
    if (ms) *ms = best / steps;
    return LBM_OK;
}

lbm_status lbm_batch_moments(lbm_batch *b, int i, double *rho, double *u) {
    if (!b || i < 0 || i >= b->n) return bfail(b, LBM_ERR_ARG, "bad channel index");
    i = b->pos_of[i];
    const lbm_desc &d = b->desc[i];
    const size_t N = (size_t)d.nx * d.ny;
    lbm_status st = ensure_tmp(b, 3 * N * 8);
    if (st != LBM_OK) return st;
    int nb = 0;
    cudaError_t e = launchers_d2q9().moments(b->storage, b->kp[i].solid != nullptr, b->kp[i], channel_state(b, i),
                                             b->tmp, b->tmp + N, b->partials, nullptr, b->stream, &nb);
    if (e == cudaSuccess && rho) e = cudaMemcpyAsync(rho, b->tmp, N * 8, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, b->tmp + N, 2 * N * 8, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("batch moments: ") + cudaGetErrorString(e));
    return LBM_OK;
}

lbm_status lbm_batch_get_populations(lbm_batch *b, int i, double *f) {
    if (!b || i < 0 || i >= b->n || !f) return bfail(b, LBM_ERR_ARG, "bad arguments");
    i = b->pos_of[i];
    const lbm_desc &d = b->desc[i];
    const size_t N = (size_t)d.nx * d.ny;
    lbm_status st = ensure_tmp(b, 9 * N * 8);
    if (st != LBM_OK) return st;
    cudaError_t e = launchers_d2q9().get_pops(b->storage, b->kp[i].solid != nullptr, b->kp[i], channel_state(b, i),
                                              b->tmp, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, b->tmp, 9 * N * 8, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, std::string("batch export: ") + cudaGetErrorString(e));
    return LBM_OK;
}

lbm_status lbm_batch_info(const lbm_batch *b, int i, int64_t *steps, int *tiles, int *rows) {
    if (!b || i < 0 || i >= b->n) return bfail(nullptr, LBM_ERR_ARG, "bad channel index");
    i = b->pos_of[i];
    if (steps) *steps = b->steps[i];
    // tiling a run starts with (all channels active)
    const int grid = b->last_grid > 0 ? b->last_grid : 1;
    const int t = tiles_for(b->ch[i].nx, b->ch[i].ny, b->total_nodes, grid, 2 * b->block,
                            std::max(b->tile_nodes, 2 * b->block));
    if (tiles) *tiles = t;
    if (rows) *rows = (b->ch[i].ny + t - 1) / t;
    return LBM_OK;
}

const char *lbm_batch_last_error(const lbm_batch *b) { return b ? b->err.c_str() : ""; }

}  // extern "C"
