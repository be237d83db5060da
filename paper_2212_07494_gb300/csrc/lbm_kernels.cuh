// lbm_kernels.cuh -- the fused stream-collide kernel and its companions
// (initialisation, moments with FP64 reductions, population import/export),
// templated on lattice, collision, storage and obstacle mask.  Each lattice
// instantiates them in its own translation unit.
#pragma once
#include "lbm_internal.h"

namespace lbm {

// Fused pull-stream + collide + store for NPT nodes per thread along x
// (strided by blockDim.x so every load instruction of a warp is a contiguous
// row segment).  Loads for all NPT nodes are issued before any arithmetic.
// In 2-byte storage the kernel is bound by instruction issue and latency:
// at most 64 registers (launch bounds of 4 blocks of 256 threads) buys
// occupancy (measured on GB300, 256^3 Taylor-Green in FP16: D3Q27 31.5
// against 29.9 GLUPS, D3Q19 46.5 against 44.1); FP32 and FP64 keep the
// compiler's choice.
template <int ST> constexpr int step_min_blocks() { return ST == ST_F16 || ST == ST_BF16 ? 4 : 1; }

// One node on the pair instructions (collide_one), out of line: the node of
// a two-node thread whose partner is past the row's end or solid, so that
// the kernel keeps one inlined collision (the pair's).  The kernel's
// parameters are __grid_constant__: the reference copies nothing.
template <int L, int COLL, int ST, bool MASK>
__device__ __noinline__ void step_node_alone(const KParams &p, const typename Store<ST>::T *__restrict__ fin,
                                             typename Store<ST>::T *__restrict__ fout, int x, int y, int z) {
    typedef typename Store<ST>::R R;
    constexpr int NG = Grid<Lat<L>::D>::N;
    R G[NG];
    gather<L, ST, MASK>(p, fin, x, y, z, G);
    const long long own = node_index(p, x, y, z);
    R gx, gy, gz;
    load_force<L>(p, y, own, gx, gy, gz);
    collide_one<L, COLL>(G, gx, gy, gz, omega<R>(p, 2), omega<R>(p, 3), omega<R>(p, 4), omega_bulk<R>(p));
    typename Store<ST>::T *dst = fout + own;
#pragma unroll
    for (int i = 0; i < Lat<L>::Q; ++i) Store<ST>::st(dst + p.poff[i], G[gpos<L>(i)]);
}

template <int L, int COLL, int ST, bool MASK, int NPT>
__global__ void __launch_bounds__(256, step_min_blocks<ST>()) k_step(const __grid_constant__ KParams p, const typename Store<ST>::T *__restrict__ fin,
                                              typename Store<ST>::T *__restrict__ fout) {
    typedef typename Store<ST>::R R;
    constexpr int NG = Grid<Lat<L>::D>::N;
    const int y = blockIdx.y + (p.halo_ax == 1), z = blockIdx.z + (p.halo_ax == 2);
    const int x0 = blockIdx.x * blockDim.x * NPT + threadIdx.x;
    R G[NPT][NG];
    bool act[NPT];
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
        const int x = x0 + k * blockDim.x;
        act[k] = x < p.nx;
        if (MASK && act[k]) act[k] = p.solid[node_index(p, x, y, z)] == 0;
        if (act[k]) gather<L, ST, MASK>(p, fin, x, y, z, G[k]);
    }
    const R om2 = omega<R>(p, 2), om3 = omega<R>(p, 3), om4 = omega<R>(p, 4), omb = omega_bulk<R>(p);
    R gx, gy, gz;
    const bool per_node_force = p.force_kind == G_FIELD;
    if (!per_node_force) load_force<L>(p, y, 0, gx, gy, gz);
    if constexpr (NPT == 2 && sizeof(R) == 4) {
        if (act[0] && act[1]) {
            // both nodes: one collision for the pair in packed FP32
            const long long own0 = node_index(p, x0, y, z), own1 = own0 + blockDim.x;
            F2 G2[NG];
#pragma unroll
            for (int g = 0; g < NG; ++g) G2[g] = F2::pair(G[0][g], G[1][g]);
            F2 gx2 = F2(gx), gy2 = F2(gy), gz2 = F2(gz);
            if (per_node_force) {
                R ax, ay, az, bx, by, bz;
                load_force<L>(p, y, own0, ax, ay, az);
                load_force<L>(p, y, own1, bx, by, bz);
                gx2 = F2::pair(ax, bx);
                gy2 = F2::pair(ay, by);
                gz2 = F2::pair(az, bz);
            }
            collide_any<L, COLL>(G2, gx2, gy2, gz2, F2(om2), F2(om3), F2(om4), F2(omb));
            typename Store<ST>::T *d0 = fout + own0, *d1 = fout + own1;
#pragma unroll
            for (int i = 0; i < Lat<L>::Q; ++i) {
                Store<ST>::st(d0 + p.poff[i], G2[gpos<L>(i)].lo());
                Store<ST>::st(d1 + p.poff[i], G2[gpos<L>(i)].hi());
            }
            return;
        }
        // a node whose partner is past the row's end or solid: out of line
        if (act[0]) step_node_alone<L, COLL, ST, MASK>(p, fin, fout, x0, y, z);
        if (act[1]) step_node_alone<L, COLL, ST, MASK>(p, fin, fout, x0 + (int)blockDim.x, y, z);
    } else {
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            if (!act[k]) continue;
            const int x = x0 + k * blockDim.x;
            const long long own = node_index(p, x, y, z);
            if (per_node_force) load_force<L>(p, y, own, gx, gy, gz);
            collide_one<L, COLL>(G[k], gx, gy, gz, om2, om3, om4, omb);
            typename Store<ST>::T *dst = fout + own;
#pragma unroll
            for (int i = 0; i < Lat<L>::Q; ++i) Store<ST>::st(dst + p.poff[i], G[k][gpos<L>(i)]);
        }
    }
}

// warp + block reduction of NV doubles; thread 0 of the block gets the sums
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double sh[kMomBlock / 32][NV];
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[wid][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w][k];
            v[k] = s;
        }
    }
}

// Running sum of per-thread values in the arithmetic type.  FP32 uses a
// compensated pair (Knuth's TwoSum: the rounding error of every addition is
// kept in lo), which carries the sum to about twice FP32's precision without
// FP64 instructions per work item (GB300's FP64 pipe is narrow); FP64 sums
// plainly.  Plain additions and subtractions only, so contraction cannot
// change the result.
template <typename R> struct Acc {
    R s = R(0);
    __device__ __forceinline__ void add(R x) { s += x; }
    __device__ __forceinline__ double value() const { return (double)s; }
};
template <> struct Acc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float s = hi + x;
        const float bp = s - hi;
        lo += (hi - (s - bp)) + (x - bp);
        hi = s;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Macroscopic fields of the current state (Eq. half_F) and the FP64 check.
// A fixed grid walks the work items (row segments of kMomBlock * kMomNpt
// nodes; grid-stride, so the partial sums and their order do not depend on
// how the hardware schedules blocks); each thread takes kMomNpt nodes of a
// segment and issues all their loads before any arithmetic.  Per-node
// arithmetic runs in the storage's arithmetic type; each thread keeps its
// running sums in Acc of that type and converts them to FP64 once, for the
// FP64 block and grid reductions; node counts are integers.  Partials per
// block: {sum (rho - 1), sum rho u_x, sum rho u_y, sum rho u_z,
// sum |u - uprev|^2, sum |u|^2, non-finite count, fluid count}.
// rho/u outputs (unpadded FP64) and uprev (unpadded, arithmetic type; read
// for the residual, then overwritten with u) are optional.
template <int L, int ST, bool MASK>
__global__ void __launch_bounds__(kMomBlock) k_moments(const KParams p, const typename Store<ST>::T *__restrict__ f,
                                                       double *__restrict__ rho_out, double *__restrict__ u_out,
                                                       double *__restrict__ partials,
                                                       typename Store<ST>::R *__restrict__ uprev) {
    typedef typename Store<ST>::R R;
    constexpr int D = Lat<L>::D;
    constexpr int NG = Grid<D>::N;
    constexpr int SEG = kMomBlock * kMomNpt;
    // work items (row segment, row) walked with 32-bit counters: a row is
    // (y, z), at most 65535^2 of them, and segments per row are few
    const int segs = (p.nx + SEG - 1) / SEG;
    // a slab's halo layers are not its nodes
    const int ylo = p.halo_ax == 1 ? 1 : 0, zlo = p.halo_ax == 2 ? 1 : 0;
    const unsigned nyc = (unsigned)(p.ny - 2 * ylo);
    const unsigned rows = nyc * (unsigned)(p.nz - 2 * zlo);
    const long long N = (long long)p.nx * p.ny * p.nz;
    Acc<R> a_drho, a_j[3], a_dd, a_uu;
    int fluid = 0, nonfinite = 0;
    unsigned row = blockIdx.x / segs;
    int seg = blockIdx.x % segs;
    const unsigned drow = gridDim.x / segs;
    const int dseg = gridDim.x % segs;
    for (; row < rows; row += drow, seg += dseg) {
        if (seg >= segs) {
            seg -= segs;
            ++row;
            if (row >= rows) break;
        }
        const int y = ylo + (int)(row % nyc), z = zlo + (int)(row / nyc);
        R G[kMomNpt][NG];
        bool on[kMomNpt], fl[kMomNpt];
        R up[kMomNpt][3];
#pragma unroll
        for (int k = 0; k < kMomNpt; ++k) {
            const int x = seg * SEG + k * kMomBlock + threadIdx.x;
            on[k] = x < p.nx;
            fl[k] = on[k] && (!MASK || p.solid[node_index(p, x, y, z)] == 0);
            if (fl[k]) gather<L, ST, MASK>(p, f, x, y, z, G[k]);
        }
        // the snapshot is read for all nodes of the work item before any of
        // it is overwritten, so these loads overlap the gathers
        if (uprev) {
#pragma unroll
            for (int k = 0; k < kMomNpt; ++k) {
                const long long n = ((long long)z * p.ny + y) * p.nx + seg * SEG + k * kMomBlock + threadIdx.x;
#pragma unroll
                for (int a = 0; a < D; ++a) up[k][a] = fl[k] ? uprev[a * N + n] : R(0);
            }
        }
        R g3[3];
        const bool per_node_force = p.force_kind == G_FIELD;
        if (!per_node_force) load_force<L>(p, y, 0, g3[0], g3[1], g3[2]);
        // the kMomNpt nodes of this work item are summed plainly, then added
        // to the running sums once per work item
        R sdrho = R(0), sj[3] = {R(0), R(0), R(0)}, sdd = R(0), suu = R(0);
#pragma unroll
        for (int k = 0; k < kMomNpt; ++k) {
            if (!on[k]) continue;
            const int x = seg * SEG + k * kMomBlock + threadIdx.x;
            const long long own = node_index(p, x, y, z);
            const long long n = ((long long)z * p.ny + y) * p.nx + x;
            R drho = R(0), u[3] = {R(0), R(0), R(0)};
            if (fl[k]) {
                R j[3] = {R(0), R(0), R(0)};
#pragma unroll
                for (int i = 0; i < Lat<L>::Q; ++i) {
                    const R w = G[k][gpos<L>(i)];
                    drho += w;
                    if (Lat<L>::cx(i)) j[0] += Lat<L>::cx(i) > 0 ? w : -w;
                    if (Lat<L>::cy(i)) j[1] += Lat<L>::cy(i) > 0 ? w : -w;
                    if (D == 3 && Lat<L>::cz(i)) j[2] += Lat<L>::cz(i) > 0 ? w : -w;
                }
                const R rho = R(1) + drho;
                if (per_node_force) load_force<L>(p, y, own, g3[0], g3[1], g3[2]);
                bool finite = isfinite(rho);
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    u[a] = j[a] / rho + R(0.5) * g3[a];
                    finite = finite && isfinite(u[a]);
                    sj[a] += j[a] + R(0.5) * rho * g3[a];   // rho u
                }
                sdrho += drho;
                nonfinite += finite ? 0 : 1;
                ++fluid;
                if (uprev) {
#pragma unroll
                    for (int a = 0; a < D; ++a) {
                        const R d = u[a] - up[k][a];
                        sdd += d * d;
                        suu += u[a] * u[a];
                        uprev[a * N + n] = u[a];
                    }
                }
            }
            if (rho_out) rho_out[n] = fl[k] ? 1.0 + (double)drho : 1.0;
            if (u_out)
#pragma unroll
                for (int a = 0; a < D; ++a) u_out[a * N + n] = (double)u[a];
        }
        a_drho.add(sdrho);
#pragma unroll
        for (int a = 0; a < D; ++a) a_j[a].add(sj[a]);
        a_dd.add(sdd);
        a_uu.add(suu);
    }
    double v[kPartials];
    v[0] = a_drho.value();
    v[1] = a_j[0].value();
    v[2] = a_j[1].value();
    v[3] = D == 3 ? a_j[2].value() : 0.0;
    v[4] = a_dd.value();
    v[5] = a_uu.value();
    v[6] = (double)nonfinite;
    v[7] = (double)fluid;
    block_sum(v);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < kPartials; ++k) partials[(long long)blockIdx.x * kPartials + k] = v[k];
}

// Target pre-collision state at every node (fbar = f_eq - F/2, deviations),
// written at the node's own position; solid nodes get zero deviation.
template <int L, int COLL, int ST, bool MASK>
__global__ void k_init(const KParams p, const double *__restrict__ rho0, const double *__restrict__ u0,
                       typename Store<ST>::T *__restrict__ target) {
    typedef typename Store<ST>::R R;
    constexpr int D = Lat<L>::D;
    const int y = blockIdx.y, z = blockIdx.z;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
    const long long own = node_index(p, x, y, z);
    const long long n = ((long long)z * p.ny + y) * p.nx + x;
    const long long N = (long long)p.nx * p.ny * p.nz;
    R G[Grid<D>::N];
    if (MASK && p.solid[own]) {
#pragma unroll
        for (int g = 0; g < Grid<D>::N; ++g) G[g] = R(0);
    } else {
        const R drho = rho0 ? R(rho0[n] - 1.0) : R(0);
        const R ux = u0 ? R(u0[n]) : R(0);
        const R uy = u0 ? R(u0[N + n]) : R(0);
        const R uz = (u0 && D == 3) ? R(u0[2 * N + n]) : R(0);
        R gx, gy, gz;
        load_force<L>(p, y, own, gx, gy, gz);
        initial_state<L, COLL>(G, drho, ux, uy, uz, gx, gy, gz);
    }
#pragma unroll
    for (int i = 0; i < Lat<L>::Q; ++i) Store<ST>::st(target + (long long)i * p.plane + own, G[gpos<L>(i)]);
}

// Inverse of the pull: state P such that pulling it reproduces the target T,
//   P_j(y) = T_j(y + c_j)   or   T_opp(j)(y) when y + c_j is a wall or solid.
template <int L, int ST, bool MASK>
__global__ void k_unstream(const KParams p, const typename Store<ST>::T *__restrict__ T,
                           typename Store<ST>::T *__restrict__ P) {
    const int y = blockIdx.y, z = blockIdx.z;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
    const long long own = node_index(p, x, y, z);
    if (MASK && p.solid[own]) return;
    NodeNbr nb;
    node_nbr(p, x, y, z, nb);
#pragma unroll
    for (int j = 0; j < Lat<L>::Q; ++j) {
        // destination x + c_j is the source entry for c = -c_j: index 1 - c_j
        const int kx = 1 - Lat<L>::cx(j), ky = 1 - Lat<L>::cy(j), kz = 1 - Lat<L>::cz(j);
        bool wall = nb.xw[kx] || nb.yw[ky] || (Lat<L>::D == 3 && nb.zw[kz]);
        const long long dst = node_index(p, nb.xs[kx], nb.ys[ky], Lat<L>::D == 3 ? nb.zs[kz] : z);
        if (MASK && j != 0 && !wall) wall = p.solid[dst] != 0;
        const long long idx = wall ? (long long)opp<L>(j) * p.plane + own : (long long)j * p.plane + dst;
        P[(long long)j * p.plane + own] = T[idx];
    }
}

// Pre-collision populations fbar = w + delta in FP64, unpadded [Q][N]
template <int L, int ST, bool MASK>
__global__ void k_get_pops(const KParams p, const typename Store<ST>::T *__restrict__ f, double *__restrict__ out) {
    typedef typename Store<ST>::R R;
    constexpr int D = Lat<L>::D;
    const int y = blockIdx.y, z = blockIdx.z;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
    const long long own = node_index(p, x, y, z);
    const long long n = ((long long)z * p.ny + y) * p.nx + x;
    const long long N = (long long)p.nx * p.ny * p.nz;
    R G[Grid<D>::N];
    const bool fluid = !MASK || p.solid[own] == 0;
    if (fluid) gather<L, ST, MASK>(p, f, x, y, z, G);
#pragma unroll
    for (int i = 0; i < Lat<L>::Q; ++i)
        out[(long long)i * N + n] = weight<L>(i) + (fluid ? (double)G[gpos<L>(i)] : 0.0);
}

// Encode FP64 populations (unpadded [Q][N]) as storage deviations at their
// own position (a target for k_unstream)
template <int L, int ST>
__global__ void k_put_pops(const KParams p, const double *__restrict__ in, typename Store<ST>::T *__restrict__ T) {
    typedef typename Store<ST>::R R;
    const int y = blockIdx.y, z = blockIdx.z;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
    const long long own = node_index(p, x, y, z);
    const long long n = ((long long)z * p.ny + y) * p.nx + x;
    const long long N = (long long)p.nx * p.ny * p.nz;
#pragma unroll
    for (int i = 0; i < Lat<L>::Q; ++i)
        Store<ST>::st(T + (long long)i * p.plane + own, R(in[(long long)i * N + n] - weight<L>(i)));
}

// ------------------------------------------------------------ host dispatch
template <int L> struct Dispatch {
    template <int COLL, int ST, bool MASK, int NPT>
    static cudaError_t step_t(StepCfg cfg, const KParams &p, const void *fin, void *fout, cudaStream_t s) {
        typedef typename Store<ST>::T T;
        k_step<L, COLL, ST, MASK, NPT><<<step_grid(p, cfg.bdx, NPT), cfg.bdx, 0, s>>>(
            p, (const T *)fin, (T *)fout);
        return cudaGetLastError();
    }
    template <int COLL, int ST, bool MASK>
    static cudaError_t step_n(StepCfg cfg, const KParams &p, const void *fin, void *fout, cudaStream_t s) {
        if (cfg.npt == 2) return step_t<COLL, ST, MASK, 2>(cfg, p, fin, fout, s);
        return step_t<COLL, ST, MASK, 1>(cfg, p, fin, fout, s);
    }
    template <int COLL, int ST>
    static cudaError_t step_m(bool mask, StepCfg cfg, const KParams &p, const void *fin, void *fout, cudaStream_t s) {
        return mask ? step_n<COLL, ST, true>(cfg, p, fin, fout, s) : step_n<COLL, ST, false>(cfg, p, fin, fout, s);
    }
    template <int COLL>
    static cudaError_t step_s(int st, bool mask, StepCfg cfg, const KParams &p, const void *fin, void *fout,
                              cudaStream_t s) {
        switch (st) {
        case ST_F64: return step_m<COLL, ST_F64>(mask, cfg, p, fin, fout, s);
        case ST_F32: return step_m<COLL, ST_F32>(mask, cfg, p, fin, fout, s);
        case ST_F16: return step_m<COLL, ST_F16>(mask, cfg, p, fin, fout, s);
        case ST_BF16: return step_m<COLL, ST_BF16>(mask, cfg, p, fin, fout, s);
        }
        return cudaErrorInvalidValue;
    }
    static cudaError_t step(int coll, int st, bool mask, StepCfg cfg, const KParams &p, const void *fin,
                            void *fout, cudaStream_t s) {
        // tau_3 = tau_4 = 1 exactly, one second-order tau: the trimmed
        // collision, the same arithmetic on the moments that stay non-zero
        if (coll == SMRT && p.om[3] == 1.0 && p.om[4] == 1.0 && p.omb == p.om[2])
            return step_s<SMRT_TRIM>(st, mask, cfg, p, fin, fout, s);
        if (coll == SMRT_FNEQ) return step_s<SMRT_FNEQ>(st, mask, cfg, p, fin, fout, s);
        if (coll == MRT_RAW) return step_s<MRT_RAW>(st, mask, cfg, p, fin, fout, s);
        return coll == SMRT ? step_s<SMRT>(st, mask, cfg, p, fin, fout, s)
                            : step_s<BGK>(st, mask, cfg, p, fin, fout, s);
    }

    template <int ST, bool MASK>
    static cudaError_t moments_t(const KParams &p, const void *f, double *rho, double *u, double *partials,
                                 void *uprev, cudaStream_t s, int *nb) {
        typedef typename Store<ST>::T T;
        typedef typename Store<ST>::R R;
        // one wave of resident blocks (fixed for a device and build, so the
        // partial sums keep a fixed order), at most kMomGridMax
        static int resident = 0;
        if (resident == 0) {
            int dev = 0, sms = 0, per_sm = 0;
            cudaError_t e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_moments<L, ST, MASK>, kMomBlock, 0);
            if (e != cudaSuccess) return e;
            resident = sms * (per_sm > 0 ? per_sm : 1);
        }
        *nb = moments_grid(p, resident);
        k_moments<L, ST, MASK><<<*nb, kMomBlock, 0, s>>>(p, (const T *)f, rho, u, partials, (R *)uprev);
        return cudaGetLastError();
    }
    static cudaError_t moments(int st, bool mask, const KParams &p, const void *f, double *rho, double *u,
                               double *partials, void *uprev, cudaStream_t s, int *nb) {
#define LBM_MOM(S)                                                                               \
    case S:                                                                                      \
        return mask ? moments_t<S, true>(p, f, rho, u, partials, uprev, s, nb)                   \
                    : moments_t<S, false>(p, f, rho, u, partials, uprev, s, nb);
        switch (st) { LBM_MOM(ST_F64) LBM_MOM(ST_F32) LBM_MOM(ST_F16) LBM_MOM(ST_BF16) }
#undef LBM_MOM
        return cudaErrorInvalidValue;
    }

    template <int COLL, int ST, bool MASK>
    static cudaError_t init_t(const KParams &p, const double *rho0, const double *u0, void *target, cudaStream_t s) {
        typedef typename Store<ST>::T T;
        k_init<L, COLL, ST, MASK><<<node_grid(p, 128, 1), 128, 0, s>>>(p, rho0, u0, (T *)target);
        return cudaGetLastError();
    }
    template <int COLL>
    static cudaError_t init_c(int st, bool mask, const KParams &p, const double *rho0, const double *u0,
                              void *target, cudaStream_t s) {
#define LBM_INIT(S)                                                                                   \
    case S:                                                                                           \
        return mask ? init_t<COLL, S, true>(p, rho0, u0, target, s) : init_t<COLL, S, false>(p, rho0, u0, target, s);
        switch (st) { LBM_INIT(ST_F64) LBM_INIT(ST_F32) LBM_INIT(ST_F16) LBM_INIT(ST_BF16) }
#undef LBM_INIT
        return cudaErrorInvalidValue;
    }
    static cudaError_t init(int coll, int st, bool mask, const KParams &p, const double *rho0, const double *u0,
                            void *target, cudaStream_t s) {
        // the moment models all start from zero non-equilibrium with the same
        // equilibrium and force expansions (d_F^(n>=2) = 0 there)
        return coll == BGK ? init_c<BGK>(st, mask, p, rho0, u0, target, s)
                           : init_c<SMRT>(st, mask, p, rho0, u0, target, s);
    }

    static cudaError_t unstream(int st, bool mask, const KParams &p, const void *T, void *P, cudaStream_t s) {
#define LBM_UNS(S)                                                                                         \
    case S: {                                                                                              \
        typedef typename Store<S>::T TT;                                                                   \
        if (mask) k_unstream<L, S, true><<<node_grid(p, 128, 1), 128, 0, s>>>(p, (const TT *)T, (TT *)P);   \
        else k_unstream<L, S, false><<<node_grid(p, 128, 1), 128, 0, s>>>(p, (const TT *)T, (TT *)P);      \
        return cudaGetLastError();                                                                         \
    }
        switch (st) { LBM_UNS(ST_F64) LBM_UNS(ST_F32) LBM_UNS(ST_F16) LBM_UNS(ST_BF16) }
#undef LBM_UNS
        return cudaErrorInvalidValue;
    }
    static cudaError_t get_pops(int st, bool mask, const KParams &p, const void *f, double *out, cudaStream_t s) {
#define LBM_GET(S)                                                                                   \
    case S: {                                                                                        \
        typedef typename Store<S>::T TT;                                                             \
        if (mask) k_get_pops<L, S, true><<<node_grid(p, 128, 1), 128, 0, s>>>(p, (const TT *)f, out); \
        else k_get_pops<L, S, false><<<node_grid(p, 128, 1), 128, 0, s>>>(p, (const TT *)f, out);    \
        return cudaGetLastError();                                                                   \
    }
        switch (st) { LBM_GET(ST_F64) LBM_GET(ST_F32) LBM_GET(ST_F16) LBM_GET(ST_BF16) }
#undef LBM_GET
        return cudaErrorInvalidValue;
    }
    static cudaError_t put_pops(int st, const KParams &p, const double *in, void *T, cudaStream_t s) {
#define LBM_PUT(S)                                                                  \
    case S: {                                                                       \
        typedef typename Store<S>::T TT;                                            \
        k_put_pops<L, S><<<node_grid(p, 128, 1), 128, 0, s>>>(p, in, (TT *)T);       \
        return cudaGetLastError();                                                  \
    }
        switch (st) { LBM_PUT(ST_F64) LBM_PUT(ST_F32) LBM_PUT(ST_F16) LBM_PUT(ST_BF16) }
#undef LBM_PUT
        return cudaErrorInvalidValue;
    }

    static const Launchers &table() {
        static const Launchers t = {&step, &moments, &init, &unstream, &get_pops, &put_pops};
        return t;
    }
};

}  // namespace lbm
