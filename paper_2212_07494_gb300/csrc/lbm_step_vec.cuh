// lbm_step_vec.cuh -- the fused pull-stream + collide + store kernel with
// vector loads: each thread takes V consecutive nodes of a row and moves each
// population of them as one aligned vector of V storage elements (16 bytes
// for D2Q9 in every storage type, 4 or 8 bytes on the 3-D lattices).
//
// The pull f_i(x) <- f_i,p(x - c_i) reads, for the V nodes of a thread, the
// elements x0 - cx .. x0 + V - 1 - cx of population i's row y - cy (z - cz).
// For cx = 0 that is the thread's own aligned vector of the source row; for
// cx = +1 it is that vector shifted by one element, whose first element is
// the last element of the neighbouring lane's vector (one warp shuffle), and
// for cx = -1 the last element is the next lane's first.  Only the first and
// last lane of a warp load that edge element themselves.  Decoding picks the
// element out of its 32-bit word (the 2-byte types hold two per word), so
// the shift costs no extra instruction per node.
//
// Rows are resolved once per block: a source row across a periodic face
// wraps; a row next to a wall takes the per-node path (gather of
// lbm_device.cuh with halfway bounce-back).  At the row's ends the element
// before or after a thread's vector wraps across a periodic x face (the
// thread loads it from the other end of the row); with walls in x, and for
// a last thread whose vector the row does not fill, the thread takes the
// per-node path.  Obstacle masks use the strided kernel k_step.
//
// Element offsets are 32-bit: the host launches this kernel only when
// Q * plane < 2^32.
#pragma once
#include "lbm_kernels.cuh"

namespace lbm {

template <int ST> struct Bits;
template <> struct Bits<ST_F64> { typedef unsigned long long E; };
template <> struct Bits<ST_F32> { typedef unsigned int E; };
template <> struct Bits<ST_F16> { typedef unsigned int E; };    // element in the low 16 bits
template <> struct Bits<ST_BF16> { typedef unsigned int E; };   // element in the low 16 bits

// storage element bits -> arithmetic type
template <int ST> __device__ __forceinline__ typename Store<ST>::R dec(typename Bits<ST>::E e);
template <> __device__ __forceinline__ double dec<ST_F64>(unsigned long long e) { return __longlong_as_double((long long)e); }
template <> __device__ __forceinline__ float dec<ST_F32>(unsigned int e) { return __uint_as_float(e); }
template <> __device__ __forceinline__ float dec<ST_F16>(unsigned int e) {
    return __half2float(__ushort_as_half((unsigned short)(e & 0xffffu)));
}
template <> __device__ __forceinline__ float dec<ST_BF16>(unsigned int e) { return __uint_as_float(e << 16); }

// one vector of V elements as NW 32-bit words
template <int ST, int V> struct Vec {
    typedef typename Store<ST>::T T;
    typedef typename Store<ST>::R R;
    typedef typename Bits<ST>::E E;
    static constexpr int BYTES = V * (int)sizeof(T);
    static constexpr int NW = BYTES / 4;
    static_assert(BYTES % 4 == 0 && BYTES >= 4 && BYTES <= 32, "vector of 4 to 32 bytes");

    // element e (0 <= e < V) of the words
    __device__ __forceinline__ static E elem(const unsigned (&w)[NW], int e) {
        if constexpr (sizeof(T) == 2) return (e & 1) ? (w[e >> 1] >> 16) : (w[e >> 1] & 0xffffu);
        else if constexpr (sizeof(T) == 4) return w[e];
        else return (unsigned long long)w[2 * e] | ((unsigned long long)w[2 * e + 1] << 32);
    }
    // BF16 decodes straight from either half of a word
    __device__ __forceinline__ static R delem(const unsigned (&w)[NW], int e) {
        if constexpr (ST == ST_BF16) return __uint_as_float((e & 1) ? (w[e >> 1] & 0xffff0000u) : (w[e >> 1] << 16));
        else return dec<ST>(elem(w, e));
    }
    __device__ __forceinline__ static void load(const T *p, unsigned (&w)[NW]) {
        if constexpr (NW >= 4) {
#pragma unroll
            for (int k = 0; k < NW / 4; ++k) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p) + k);
                w[4 * k] = v.x;
                w[4 * k + 1] = v.y;
                w[4 * k + 2] = v.z;
                w[4 * k + 3] = v.w;
            }
        } else if constexpr (NW == 2) {
            const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
            w[0] = v.x;
            w[1] = v.y;
        } else {
            w[0] = __ldg(reinterpret_cast<const unsigned *>(p));
        }
    }
    __device__ __forceinline__ static void store(T *p, const unsigned (&w)[NW]) {
        if constexpr (NW >= 4) {
#pragma unroll
            for (int k = 0; k < NW / 4; ++k)
                reinterpret_cast<uint4 *>(p)[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
        } else if constexpr (NW == 2) {
            *reinterpret_cast<uint2 *>(p) = make_uint2(w[0], w[1]);
        } else {
            *reinterpret_cast<unsigned *>(p) = w[0];
        }
    }
    // one element loaded on its own (the lane at a warp's edge)
    __device__ __forceinline__ static E load1(const T *p) {
        if constexpr (sizeof(T) == 2) return (unsigned)__ldg(reinterpret_cast<const unsigned short *>(p));
        else if constexpr (sizeof(T) == 4) return __ldg(reinterpret_cast<const unsigned *>(p));
        else return __ldg(reinterpret_cast<const unsigned long long *>(p));
    }
    // the last element of the previous lane, the first of the next lane
    __device__ __forceinline__ static E from_prev_lane(const unsigned (&w)[NW]) {
        if constexpr (sizeof(T) == 2) return __shfl_up_sync(0xffffffffu, w[NW - 1], 1) >> 16;
        else if constexpr (sizeof(T) == 4) return __shfl_up_sync(0xffffffffu, w[NW - 1], 1);
        else
            return (unsigned long long)__shfl_up_sync(0xffffffffu, w[NW - 2], 1) |
                   ((unsigned long long)__shfl_up_sync(0xffffffffu, w[NW - 1], 1) << 32);
    }
    __device__ __forceinline__ static E from_next_lane(const unsigned (&w)[NW]) {
        if constexpr (sizeof(T) == 2) return __shfl_down_sync(0xffffffffu, w[0], 1) & 0xffffu;
        else if constexpr (sizeof(T) == 4) return __shfl_down_sync(0xffffffffu, w[0], 1);
        else
            return (unsigned long long)__shfl_down_sync(0xffffffffu, w[0], 1) |
                   ((unsigned long long)__shfl_down_sync(0xffffffffu, w[1], 1) << 32);
    }
    // put the result of node k into the output words; the 2-byte types pack
    // the results of nodes k - 1 and k (round to nearest even) at odd k
    __device__ __forceinline__ static void put(unsigned (&o)[NW], int k, R v, R &held) {
        if constexpr (ST == ST_F16) {
            if (k & 1) {
                const __half2 h = __floats2half2_rn(held, v);
                o[k >> 1] = *reinterpret_cast<const unsigned *>(&h);
            } else {
                held = v;
            }
        } else if constexpr (ST == ST_BF16) {
            if (k & 1) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(held, v);
                o[k >> 1] = *reinterpret_cast<const unsigned *>(&h);
            } else {
                held = v;
            }
        } else if constexpr (ST == ST_F32) {
            o[k] = __float_as_uint(v);
        } else {
            const unsigned long long b = (unsigned long long)__double_as_longlong(v);
            o[2 * k] = (unsigned)b;
            o[2 * k + 1] = (unsigned)(b >> 32);
        }
    }
};


// source row index along one axis for c = -1, 0, +1 (entry c + 1): the
// coordinate minus c, wrapped on a periodic axis; false if it lies beyond a
// wall
__device__ __forceinline__ bool row_src(int v, int n, int per, int (&s)[3]) {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int t = v - (k - 1);
        if (t < 0) { if (per) t += n; else { ok = false; t = 0; } }
        else if (t >= n) { if (per) t -= n; else { ok = false; t = n - 1; } }
        s[k] = t;
    }
    return ok;
}

// the same along the split axis of a slab (axis_src_halo): the source layer
// is in the buffer unless it lies beyond a wall of the whole domain
__device__ __forceinline__ bool row_src_halo(const KParams &p, int ax, int v, int (&s)[3]) {
    int t[3];
    bool w[3];
    axis_src_halo(v, p.per[ax], p.hg0, p.hgn, t, w);
#pragma unroll
    for (int k = 0; k < 3; ++k) s[k] = t[k];
    return !(w[0] || w[1] || w[2]);
}

// Register caps (launch bounds of n blocks of 256 threads: at most
// 65536 / (256 n) registers, 64 for n = 4, 85 for n = 3, 128 for n = 2), so
// that more warps keep loads in flight.  Measured on GB300 (D2Q9 4096^2 Kolmogorov, 256^3
// Taylor-Green): D2Q9 2-byte at 64 registers 147 against 141 GLUPS; D3Q27
// and D3Q19 2-byte at 128 registers 49.8 and 70.0 against 36.1 and 49.6;
// D3Q27 FP32 at 85 registers 32.2 against 28.1.  FP64 keeps the compiler's
// choice.
template <int L, int ST> constexpr int vec_min_blocks() {
    return L == D2Q9 ? (ST == ST_F64 ? 1 : 4) : (ST == ST_F64 ? 1 : (ST == ST_F32 ? 3 : 2));
}

// The per-node path of k_step_vec: rows next to a wall, and the row ends
// (the SLOW launch).
template <int L, int COLL, int ST, int V>
__device__ __forceinline__ void step_vec_nodes(const KParams &p, const typename Store<ST>::T *__restrict__ fin,
                                            typename Store<ST>::T *__restrict__ fout, int x0, int y, int z) {
    typedef typename Store<ST>::R R;
    constexpr int D = Lat<L>::D, Q = Lat<L>::Q, NG = Grid<D>::N;
    const R om2 = omega<R>(p, 2), om3 = omega<R>(p, 3), om4 = omega<R>(p, 4), omb = omega_bulk<R>(p);
    const bool per_node_force = p.force_kind == G_FIELD;
    R gx = R(0), gy = R(0), gz = R(0);
    if (!per_node_force) load_force<L>(p, y, 0, gx, gy, gz);
    if constexpr (sizeof(R) == 4) {
        // two of the thread's nodes per collision in packed FP32, gathered
        // node by node; a lone last node fills both lanes and only its lane
        // is stored (every node on the pair instructions)
#pragma unroll 1
        for (int k = 0; k < V; k += 2) {
            const int xa = x0 + k;
            if (xa >= p.nx) break;
            const bool two = k + 1 < V && xa + 1 < p.nx;
            R Ga[NG], Gb[NG];
            gather<L, ST, false>(p, fin, xa, y, z, Ga);
            if (two) gather<L, ST, false>(p, fin, xa + 1, y, z, Gb);
            F2 G2[NG];
#pragma unroll
            for (int g = 0; g < NG; ++g) G2[g] = F2::pair(Ga[g], two ? Gb[g] : Ga[g]);
            const long long own = node_index(p, xa, y, z);
            F2 gx2 = F2(gx), gy2 = F2(gy), gz2 = F2(gz);
            if (per_node_force) {
                R ax, ay, az, bx, by, bz;
                load_force<L>(p, y, own, ax, ay, az);
                load_force<L>(p, y, two ? own + 1 : own, bx, by, bz);
                gx2 = F2::pair(ax, bx);
                gy2 = F2::pair(ay, by);
                gz2 = F2::pair(az, bz);
            }
            collide_any<L, COLL>(G2, gx2, gy2, gz2, F2(om2), F2(om3), F2(om4), F2(omb));
            typename Store<ST>::T *dst = fout + own;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                Store<ST>::st(dst + p.poff[i], G2[gpos<L>(i)].lo());
                if (two) Store<ST>::st(dst + 1 + p.poff[i], G2[gpos<L>(i)].hi());
            }
        }
    } else {
#pragma unroll 1
        for (int k = 0; k < V; ++k) {
            const int x = x0 + k;
            if (x >= p.nx) break;
            R G[NG];
            gather<L, ST, false>(p, fin, x, y, z, G);
            const long long own = node_index(p, x, y, z);
            if (per_node_force) load_force<L>(p, y, own, gx, gy, gz);
            collide_one<L, COLL>(G, gx, gy, gz, om2, om3, om4, omb);
            typename Store<ST>::T *dst = fout + own;
#pragma unroll
            for (int i = 0; i < Q; ++i) Store<ST>::st(dst + p.poff[i], G[gpos<L>(i)]);
        }
    }
}

// SLOW = false: the threads whose nodes take the vector path ("fast"); the
// others return.  SLOW = true: the other nodes (rows next to a wall, the
// row ends), node by node, in a launch of their own that the host adds only
// when the domain has such nodes.  Two kernels, so that the per-node path's
// collision and register needs stay out of the vector path's allocation.
template <int L, int COLL, int ST, int V, bool SLOW>
__global__ void __launch_bounds__(256, vec_min_blocks<L, ST>()) k_step_vec(const KParams p, const typename Store<ST>::T *__restrict__ fin,
                                                  typename Store<ST>::T *__restrict__ fout) {
    typedef Vec<ST, V> VT;
    typedef typename Store<ST>::R R;
    typedef typename Bits<ST>::E E;
    constexpr int D = Lat<L>::D, Q = Lat<L>::Q, NG = Grid<D>::N, NW = VT::NW;
    const int y = blockIdx.y + (p.halo_ax == 1), z = blockIdx.z + (p.halo_ax == 2);
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const R om2 = omega<R>(p, 2), om3 = omega<R>(p, 3), om4 = omega<R>(p, 4), omb = omega_bulk<R>(p);
    const bool per_node_force = p.force_kind == G_FIELD;
    R gx, gy, gz;
    if (!per_node_force) load_force<L>(p, y, 0, gx, gy, gz);

    int ys[3], zs[3] = {0, 0, 0};
    bool row_ok = p.halo_ax == 1 ? row_src_halo(p, 1, y, ys) : row_src(y, p.ny, p.per[1], ys);
    if (D == 3) row_ok = (p.halo_ax == 2 ? row_src_halo(p, 2, z, zs) : row_src(z, p.nz, p.per[2], zs)) && row_ok;
    // fast: every source of the thread's V nodes is in this row band's
    // interior or wraps across a periodic face of y or z
    // x: the thread's V nodes all lie in the row, and the elements just
    // before and after them exist (inside the row, or across a periodic x
    // face, where they wrap to the other end of the row)
    const bool first = x0 == 0, last = x0 + V == p.nx;
    const bool fast = row_ok && x0 + V <= p.nx && (p.per[0] || (!first && !last));
    if constexpr (SLOW) {
        if (!fast && x0 < p.nx) step_vec_nodes<L, COLL, ST, V>(p, fin, fout, x0, y, z);
        return;
    }

    if (row_ok) {
        // the whole block is one row band: every lane takes part in the loads
        // and shuffles; threads past the row's end load nothing
        const bool on = x0 < p.nx;
        const int lane = threadIdx.x & 31;
        unsigned w[Q][NW];
        E edge[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int cx = Lat<L>::cx(i), cy = Lat<L>::cy(i), cz = Lat<L>::cz(i);
            const unsigned src = (unsigned)i * (unsigned)p.plane +
                                 ((unsigned)(D == 3 ? zs[cz + 1] : 0) * (unsigned)p.ny + (unsigned)ys[cy + 1]) *
                                     (unsigned)p.nxp + (unsigned)x0;
            if (on) VT::load(fin + src, w[i]);
            else
#pragma unroll
                for (int k = 0; k < NW; ++k) w[i][k] = 0u;
            if (cx == 1) {
                // element x0 - 1 (x = nx - 1 across the periodic face)
                edge[i] = VT::from_prev_lane(w[i]);
                if ((lane == 0 || first) && fast) edge[i] = VT::load1(fin + (first ? src + (unsigned)(p.nx - 1) : src - 1u));
            } else if (cx == -1) {
                // element x0 + V (x = 0 across the periodic face)
                edge[i] = VT::from_next_lane(w[i]);
                if ((lane == 31 || last) && fast) edge[i] = VT::load1(fin + (last ? src - (unsigned)x0 : src + (unsigned)V));
            } else {
                edge[i] = 0;
            }
        }
        if (fast) {
            const unsigned own = ((unsigned)z * (unsigned)p.ny + (unsigned)y) * (unsigned)p.nxp + (unsigned)x0;
            unsigned o[Q][NW];
            R held[Q];
            if constexpr (sizeof(R) == 4 && V % 2 == 0) {
                // nodes k and k + 1 collide together in packed FP32
#pragma unroll
                for (int k = 0; k < V; k += 2) {
                    F2 G2[NG];
#pragma unroll
                    for (int g = 0; g < NG; ++g) G2[g] = F2(0.0f);
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        const int e0 = k - Lat<L>::cx(i), e1 = e0 + 1;
                        const R v0 = (e0 < 0 || e0 >= V) ? dec<ST>(edge[i]) : VT::delem(w[i], e0);
                        const R v1 = (e1 < 0 || e1 >= V) ? dec<ST>(edge[i]) : VT::delem(w[i], e1);
                        G2[gpos<L>(i)] = F2::pair(v0, v1);
                    }
                    F2 gx2 = F2(gx), gy2 = F2(gy), gz2 = F2(gz);
                    if (per_node_force) {
                        R ax, ay, az, bx, by, bz;
                        load_force<L>(p, y, (long long)own + k, ax, ay, az);
                        load_force<L>(p, y, (long long)own + k + 1, bx, by, bz);
                        gx2 = F2::pair(ax, bx);
                        gy2 = F2::pair(ay, by);
                        gz2 = F2::pair(az, bz);
                    }
                    collide_any<L, COLL>(G2, gx2, gy2, gz2, F2(om2), F2(om3), F2(om4), F2(omb));
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        VT::put(o[i], k, G2[gpos<L>(i)].lo(), held[i]);
                        VT::put(o[i], k + 1, G2[gpos<L>(i)].hi(), held[i]);
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    R G[NG];
#pragma unroll
                    for (int g = 0; g < NG; ++g) G[g] = R(0);
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        const int e = k - Lat<L>::cx(i);   // element of the source vector
                        G[gpos<L>(i)] = (e < 0 || e >= V) ? dec<ST>(edge[i]) : VT::delem(w[i], e);
                    }
                    if (per_node_force) load_force<L>(p, y, (long long)own + k, gx, gy, gz);
                    collide_one<L, COLL>(G, gx, gy, gz, om2, om3, om4, omb);
#pragma unroll
                    for (int i = 0; i < Q; ++i) VT::put(o[i], k, G[gpos<L>(i)], held[i]);
                }
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) VT::store(fout + ((unsigned)i * (unsigned)p.plane + own), o[i]);
            return;
        }
    }
    // the other nodes are the SLOW launch's
}

// host launcher of one (lattice, storage) pair: the collision and vector
// width are template arguments, the supported widths listed by vec_widths
template <int L, int ST> struct VecDispatch {
    // a node can leave the vector path only across a wall (some axis not
    // periodic) or at a ragged row end (nx not a multiple of V); otherwise
    // the per-node launch would find nothing to do and is left out
    template <int V> static bool has_slow_nodes(const KParams &p) {
        return !(p.per[0] && p.per[1] && (Lat<L>::D == 2 || p.per[2]) && p.nx % V == 0);
    }
    template <int COLL, int V>
    static cudaError_t go(StepCfg cfg, const KParams &p, const void *fin, void *fout, cudaStream_t s) {
        typedef typename Store<ST>::T T;
        const dim3 grid = step_grid(p, cfg.bdx, V);
        k_step_vec<L, COLL, ST, V, false><<<grid, cfg.bdx, 0, s>>>(p, (const T *)fin, (T *)fout);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && has_slow_nodes<V>(p)) {
            k_step_vec<L, COLL, ST, V, true><<<grid, cfg.bdx, 0, s>>>(p, (const T *)fin, (T *)fout);
            e = cudaGetLastError();
        }
        return e;
    }
    template <int COLL>
    static cudaError_t by_width(StepCfg cfg, const KParams &p, const void *fin, void *fout, cudaStream_t s) {
        constexpr int W0 = vec_width_lo(L, ST), W1 = vec_width_hi(L, ST);
        if (cfg.npt == W0) return go<COLL, W0>(cfg, p, fin, fout, s);
        if constexpr (W1 != W0)
            if (cfg.npt == W1) return go<COLL, W1>(cfg, p, fin, fout, s);
        return cudaErrorInvalidValue;
    }
    static cudaError_t step(int coll, StepCfg cfg, const KParams &p, const void *fin, void *fout, cudaStream_t s) {
        if (coll == SMRT && p.om[3] == 1.0 && p.om[4] == 1.0 && p.omb == p.om[2])
            return by_width<SMRT_TRIM>(cfg, p, fin, fout, s);
        switch (coll) {
        case SMRT: return by_width<SMRT>(cfg, p, fin, fout, s);
        case SMRT_FNEQ: return by_width<SMRT_FNEQ>(cfg, p, fin, fout, s);
        case MRT_RAW: return by_width<MRT_RAW>(cfg, p, fin, fout, s);
        case BGK: return by_width<BGK>(cfg, p, fin, fout, s);
        }
        return cudaErrorInvalidValue;
    }
};

}  // namespace lbm
