// lbm_device.cuh -- device building blocks of the fused lattice Boltzmann
// update with the second-order force scheme (arXiv:2212.07494).
//
// Populations are kept as deviations delta_i = fbar_i - w_i, structure of
// arrays f[i][z][y][xp] with rows padded to nxp elements.  The SMRT collision
// works on the 3 x 3 (x 3) velocity grid of the tensor-product lattices
// (D2Q9 = D1Q3^2, D3Q27 = D1Q3^3; D3Q19 = D3Q27 without its 8 corners) and
// runs every moment transform as three-point passes along one axis at a time:
//   project  (Hermite moments h0 = 1, h1 = c, h2 = c^2 - 1/3; Eq. dft)
//   shift by -u   (raw -> central moments, the Hermite addition theorem)
//   relax    (order by order, d_p^(n) = (1 - 1/tau_n) d_1^(n); d_p^(1) = F/2)
//   shift by +u   (central -> raw, Eq. bbd1 in closed binomial form)
//   truncate to the retained components and reconstruct (Sec. II.C).
// In lattice units the reconstruction coefficients per axis are
// r0 = 1, r1 = 3c, r2 = 4.5 c^2 - 1.5.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbm {

enum { D2Q9 = 0, D3Q19 = 1, D3Q27 = 2 };
// BGK, SMRT, SMRT_FNEQ and MRT_RAW carry the values of the C ABI's
// lbm_collision; SMRT_TRIM is SMRT with tau_3 = tau_4 = 1 (a kernel choice only)
enum { BGK = 0, SMRT = 1, SMRT_FNEQ = 2, MRT_RAW = 3, SMRT_TRIM = 4 };
enum { ST_F64 = 0, ST_F32 = 1, ST_F16 = 2, ST_BF16 = 3 };
enum { G_NONE = 0, G_UNIFORM = 1, G_ROWS = 2, G_FIELD = 3 };

// ---------------------------------------------------------------- lattices
template <int L> struct Lat;

template <> struct Lat<D2Q9> {
    static constexpr int D = 2, Q = 9, NG = 9;
    __host__ __device__ static constexpr int cx(int i) {
        return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
    }
    __host__ __device__ static constexpr int cy(int i) {
        return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
};

// D3Q27 order: rest; 6 faces; 12 edges; 8 corners, opposite pairs adjacent.
struct C3 {
    __host__ __device__ static constexpr int c(int i, int a) {
        // rows of the table (cx, cy, cz)
        return i == 0 ? 0
             : i == 1 ? (a == 0 ? 1 : 0)
             : i == 2 ? (a == 0 ? -1 : 0)
             : i == 3 ? (a == 1 ? 1 : 0)
             : i == 4 ? (a == 1 ? -1 : 0)
             : i == 5 ? (a == 2 ? 1 : 0)
             : i == 6 ? (a == 2 ? -1 : 0)
             : i == 7 ? (a == 2 ? 0 : 1)
             : i == 8 ? (a == 2 ? 0 : -1)
             : i == 9 ? (a == 0 ? 1 : (a == 1 ? -1 : 0))
             : i == 10 ? (a == 0 ? -1 : (a == 1 ? 1 : 0))
             : i == 11 ? (a == 1 ? 0 : 1)
             : i == 12 ? (a == 1 ? 0 : -1)
             : i == 13 ? (a == 0 ? 1 : (a == 2 ? -1 : 0))
             : i == 14 ? (a == 0 ? -1 : (a == 2 ? 1 : 0))
             : i == 15 ? (a == 0 ? 0 : 1)
             : i == 16 ? (a == 0 ? 0 : -1)
             : i == 17 ? (a == 1 ? 1 : (a == 2 ? -1 : 0))
             : i == 18 ? (a == 1 ? -1 : (a == 2 ? 1 : 0))
             : i == 19 ? 1
             : i == 20 ? -1
             : i == 21 ? (a == 2 ? -1 : 1)
             : i == 22 ? (a == 2 ? 1 : -1)
             : i == 23 ? (a == 1 ? -1 : 1)
             : i == 24 ? (a == 1 ? 1 : -1)
             : i == 25 ? (a == 0 ? -1 : 1)
             : (a == 0 ? 1 : -1);
    }
};

template <> struct Lat<D3Q19> {
    static constexpr int D = 3, Q = 19, NG = 27;
    __host__ __device__ static constexpr int cx(int i) { return C3::c(i, 0); }
    __host__ __device__ static constexpr int cy(int i) { return C3::c(i, 1); }
    __host__ __device__ static constexpr int cz(int i) { return C3::c(i, 2); }
};
template <> struct Lat<D3Q27> {
    static constexpr int D = 3, Q = 27, NG = 27;
    __host__ __device__ static constexpr int cx(int i) { return C3::c(i, 0); }
    __host__ __device__ static constexpr int cy(int i) { return C3::c(i, 1); }
    __host__ __device__ static constexpr int cz(int i) { return C3::c(i, 2); }
};

template <int L> __host__ __device__ constexpr int opp(int i) {
    // opposite pairs: D2Q9 (1,3) (2,4) (5,7) (6,8); 3-D: (2k-1, 2k)
    return L == D2Q9 ? (i == 0 ? 0 : (i <= 4 ? (i <= 2 ? i + 2 : i - 2) : (i <= 6 ? i + 2 : i - 2)))
                     : (i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1));
}

__host__ __device__ constexpr double w1d(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }

template <int L> __host__ __device__ constexpr double weight(int i) {
    return L == D3Q19
        ? ((Lat<L>::cx(i) != 0) + (Lat<L>::cy(i) != 0) + (Lat<L>::cz(i) != 0) == 0 ? 1.0 / 3.0
           : (Lat<L>::cx(i) != 0) + (Lat<L>::cy(i) != 0) + (Lat<L>::cz(i) != 0) == 1 ? 1.0 / 18.0
                                                                                    : 1.0 / 36.0)
        : w1d(Lat<L>::cx(i)) * w1d(Lat<L>::cy(i)) * (Lat<L>::D == 3 ? w1d(Lat<L>::cz(i)) : 1.0);
}

// grid position of population i on the 3^D velocity grid: (c + 1) per axis
template <int L> __host__ __device__ constexpr int gpos(int i) {
    return (Lat<L>::cx(i) + 1) + 3 * (Lat<L>::cy(i) + 1) + (Lat<L>::D == 3 ? 9 * (Lat<L>::cz(i) + 1) : 0);
}

// moment index digits on the grid (order m_a per axis)
template <int D> __host__ __device__ constexpr int mdig(int g, int a) { return (a == 0 ? g : (a == 1 ? g / 3 : g / 9)) % 3; }
template <int D> __host__ __device__ constexpr int morder(int g) {
    return mdig<D>(g, 0) + mdig<D>(g, 1) + (D == 3 ? mdig<D>(g, 2) : 0);
}
template <int D> __host__ __device__ constexpr int maxdig(int g) {
    return mdig<D>(g, 0) > mdig<D>(g, 1)
               ? (D == 3 && mdig<D>(g, 2) > mdig<D>(g, 0) ? mdig<D>(g, 2) : mdig<D>(g, 0))
               : (D == 3 && mdig<D>(g, 2) > mdig<D>(g, 1) ? mdig<D>(g, 2) : mdig<D>(g, 1));
}
// retained Hermite components: D2Q9 all nine; D3Q27 total order <= 4;
// D3Q19 orders <= 2 and the (2,1,0)-type third-order components
template <int L> __host__ __device__ constexpr bool retained(int g) {
    return L == D2Q9 ? true
         : L == D3Q27 ? morder<3>(g) <= 4
                      : (morder<3>(g) <= 2 || (morder<3>(g) == 3 && maxdig<3>(g) == 2));
}
template <int L> __host__ __device__ constexpr bool on_lattice(int g) {
    // D3Q19 has no (+-1, +-1, +-1) velocities
    return L != D3Q19 || !((g % 3) != 1 && ((g / 3) % 3) != 1 && (g / 9) != 1);
}

// ------------------------------------------------------------- storage codec
template <int ST> struct Store;
template <> struct Store<ST_F64> {
    typedef double T;
    typedef double R;
    __device__ static R ld(const T *p) { return __ldg(p); }
    __device__ static void st(T *p, R v) { *p = v; }
};
template <> struct Store<ST_F32> {
    typedef float T;
    typedef float R;
    __device__ static R ld(const T *p) { return __ldg(p); }
    __device__ static void st(T *p, R v) { *p = v; }
};
template <> struct Store<ST_F16> {
    typedef __half T;
    typedef float R;
    __device__ static R ld(const T *p) { return __half2float(__ldg(p)); }
    __device__ static void st(T *p, R v) { *p = __float2half_rn(v); }
};
template <> struct Store<ST_BF16> {
    typedef __nv_bfloat16 T;
    typedef float R;
    __device__ static R ld(const T *p) { return __bfloat162float(__ldg(p)); }
    __device__ static void st(T *p, R v) { *p = __float2bfloat16_rn(v); }
};

// ------------------------------------------------------------ kernel params
struct KParams {
    int nx, ny, nz, nxp;
    long long plane;               // elements per population plane (nxp*ny*nz)
    int per[3];                    // periodic flags
    int force_kind;                // G_*
    const double *g;               // uniform [3] | rows [ny][D] | field [D][plane]
    const float *g32;              // the same force in FP32 (for FP32 arithmetic)
    const unsigned char *solid;    // [plane] or null
    double om[5];                  // 1 / tau_n
    float om32[5];
    double omb;                    // 1 / tau of the trace (bulk) part of order 2; om[2] unless split
    float omb32;
    // A slab of a domain split along its outermost axis (halo_ax = 1: y in
    // 2-D, 2: z in 3-D; 0: a whole domain).  That axis then holds one halo
    // layer at each end, which the caller fills with the neighbouring slabs'
    // layers; the step and moments kernels work on layers 1 .. n - 2, and
    // the pull reads the halo layers without wrapping.  hg0 is the global
    // index of layer 1 and hgn the global extent, which place the domain's
    // walls on that axis.
    int halo_ax, hg0, hgn;
    // per population i, relative to a node's element index:
    // per population i, relative to the element index of a node's x - c_x
    // (the node itself, or its neighbour along x, wrapped on a periodic x):
    long long doff[27];            // i*plane - (cy*nxp + cz*nxp*ny): pull source
    long long poff[27];            // i*plane: the node's own entry (relative to the node)
    int noff[27];                  // -(cy*nxp + cz*nxp*ny): neighbour x - c_i
};

// fill the per-population offsets of KParams for lattice L (host side)
template <int L> inline void fill_offsets(KParams &p) {
    for (int i = 0; i < 27; ++i) p.doff[i] = p.poff[i] = p.noff[i] = 0;
    for (int i = 0; i < Lat<L>::Q; ++i) {
        const long long nb = (long long)Lat<L>::cy(i) * p.nxp + (long long)Lat<L>::cz(i) * p.nxp * p.ny;
        p.poff[i] = (long long)i * p.plane;
        p.doff[i] = p.poff[i] - nb;
        p.noff[i] = (int)(-nb);
    }
}

// --------------------------------------------------------- moment-space passes
// All passes act in place on a 3^D array indexed by grid position / moment
// order, along axis AX (stride 3^AX).
template <int D> struct Grid { static constexpr int N = D == 2 ? 9 : 27; };

template <int D, int AX, typename R, typename F>
__host__ __device__ __forceinline__ void for_lines(R *a, F f) {
    constexpr int S = AX == 0 ? 1 : (AX == 1 ? 3 : 9);
#pragma unroll
    for (int g = 0; g < Grid<D>::N; ++g) {
        if ((g / S) % 3 == 0) f(a[g], a[g + S], a[g + 2 * S]);
    }
}

// populations (c = -1, 0, +1) -> moments (h0, h1, h2) on one line
template <typename R> __host__ __device__ __forceinline__ void proj_line(R &m, R &z, R &p) {
    const R s = p + m, d = p - m;
    const R m0 = s + z;
    const R m2 = (R(2) * s - z) * R(1.0 / 3.0);
    m = m0;
    z = d;
    p = m2;
}
// shift a line of moments (h0, h1, h2) by velocity v: Hermite addition theorem
template <typename R> __host__ __device__ __forceinline__ void shift_line(R &a0, R &a1, R &a2, R v) {
    a2 = a2 + v * (R(2) * a1 + v * a0);
    a1 = a1 + v * a0;
}
// moments (t0, t1, t2) -> populations with the D1Q3 weight folded in
template <typename R> __host__ __device__ __forceinline__ void recon_line_w(R &t0, R &t1, R &t2) {
    const R a = t0 + R(3) * t2, b = R(3) * t1;
    const R fz = R(2.0 / 3.0) * (t0 - R(1.5) * t2);
    t0 = R(1.0 / 6.0) * (a - b);
    t2 = R(1.0 / 6.0) * (a + b);
    t1 = fz;
}
template <typename R> __host__ __device__ __forceinline__ void recon_line(R &t0, R &t1, R &t2) {
    const R a = t0 + R(3) * t2, b = R(3) * t1;
    const R fz = t0 - R(1.5) * t2;
    t0 = a - b;
    t2 = a + b;
    t1 = fz;
}

template <int D, typename R> __host__ __device__ __forceinline__ void project(R *a) {
    for_lines<D, 0>(a, [](R &x, R &y, R &z) { proj_line(x, y, z); });
    for_lines<D, 1>(a, [](R &x, R &y, R &z) { proj_line(x, y, z); });
    if (D == 3) for_lines<D, 2>(a, [](R &x, R &y, R &z) { proj_line(x, y, z); });
}
template <int D, typename R> __host__ __device__ __forceinline__ void shift(R *a, R ux, R uy, R uz) {
    for_lines<D, 0>(a, [ux](R &x, R &y, R &z) { shift_line(x, y, z, ux); });
    for_lines<D, 1>(a, [uy](R &x, R &y, R &z) { shift_line(x, y, z, uy); });
    if (D == 3) for_lines<D, 2>(a, [uz](R &x, R &y, R &z) { shift_line(x, y, z, uz); });
}
template <int L, typename R> __host__ __device__ __forceinline__ void reconstruct(R *a) {
    constexpr int D = Lat<L>::D;
    if (L == D3Q19) {
        for_lines<D, 0>(a, [](R &x, R &y, R &z) { recon_line(x, y, z); });
        for_lines<D, 1>(a, [](R &x, R &y, R &z) { recon_line(x, y, z); });
        for_lines<D, 2>(a, [](R &x, R &y, R &z) { recon_line(x, y, z); });
    } else {
        for_lines<D, 0>(a, [](R &x, R &y, R &z) { recon_line_w(x, y, z); });
        for_lines<D, 1>(a, [](R &x, R &y, R &z) { recon_line_w(x, y, z); });
        if (D == 3) for_lines<D, 2>(a, [](R &x, R &y, R &z) { recon_line_w(x, y, z); });
    }
}

// ------------------------------------------------------------------ collisions
// Second-order central moments scaled by (1 - a) in their traceless (shear)
// part and (1 - b) in their trace (bulk) part, Eq. (domg) with tau_{2,2} and
// tau_{2,0}: G <- (1 - a) G + (a - b) delta tr(G)/D.  The grid entries with
// per-axis orders 2e_k are the diagonal components; with a = b the added
// term is an exact zero.
template <int D, typename R> __host__ __device__ __forceinline__ void relax_order2(R *G, R a, R b) {
    constexpr int N = Grid<D>::N;
    R tr = G[2] + G[6];
    if constexpr (D == 3) tr += G[18];
    const R iso = tr * R(1.0 / D) * (a - b);
#pragma unroll
    for (int g = 0; g < N; ++g) {
        if (morder<D>(g) != 2) continue;
        const bool diag = g == 2 || g == 6 || g == 18;
        G[g] = diag ? (R(1) - a) * G[g] + iso : (R(1) - a) * G[g];
    }
}

// G holds the deviations delta on the velocity grid (zeros off-lattice) and is
// overwritten with the post-collision deviations.  g: acceleration (lattice
// units).  Returns nothing; rho/u are recomputed by the moments kernel.
template <int L, typename R>
__host__ __device__ __forceinline__ void collide_smrt(R *G, R gx, R gy, R gz, R om2, R om3, R om4, R omb) {
    constexpr int D = Lat<L>::D;
    constexpr int N = Grid<D>::N;
    constexpr int EX = 1, EY = 3, EZ = 9;
    project<D>(G);
    const R drho = G[0];                 // rho - 1 (moments of w vanish beyond order 0)
    const R rho = R(1) + drho;
    const R inv = R(1) / rho;
    const R ux = G[EX] * inv + R(0.5) * gx;   // Eq. (half_F)
    const R uy = G[EY] * inv + R(0.5) * gy;
    const R uz = D == 3 ? G[EZ] * inv + R(0.5) * gz : R(0);
    G[0] = rho;
    shift<D>(G, -ux, -uy, -uz);           // central moments of fbar
    // relaxation of the non-equilibrium central moments (equilibrium ones are
    // rho delta_{n0}); the force enters at first order only: d_p^(1) = rho g/2
    relax_order2<D>(G, om2, omb);
#pragma unroll
    for (int g = 0; g < N; ++g) {
        const int n = morder<D>(g);
        if (n == 3) G[g] *= (R(1) - om3);
        else if (n == 4) G[g] *= (R(1) - om4);
        else if (n >= 5) G[g] = R(0);
    }
    G[0] = rho;
    G[EX] = R(0.5) * rho * gx;
    G[EY] = R(0.5) * rho * gy;
    if (D == 3) G[EZ] = R(0.5) * rho * gz;
    shift<D>(G, ux, uy, uz);              // back to raw moments: a_0 + a_p
#pragma unroll
    for (int g = 0; g < N; ++g)
        if (!retained<L>(g)) G[g] = R(0);
    G[0] = drho;                          // deviation from the weights
    reconstruct<L>(G);
    if (L == D3Q19) {
#pragma unroll
        for (int i = 0; i < Lat<L>::Q; ++i) G[gpos<L>(i)] *= R(weight<L>(i));
    }
}

// ------------------------------------------------- sparse passes (trimmed SMRT)
// With tau_3 = tau_4 = 1 the factors (1 - 1/tau_n) of orders 3 and 4 vanish:
// after relaxation only the central moments of orders <= 2 are non-zero, so
// only the raw moments of orders <= 2 need projecting and shifting.  The
// passes below are the same per-axis line operations as above, restricted
// at compile time by masks over the 3^D grid (bit g): NEED, the entries a
// later step reads (an unneeded output is not computed), and NZ, the entries
// that may be non-zero (a known zero is not read).
template <int D> __host__ __device__ constexpr unsigned grid_mask() { return D == 2 ? 0x1FFu : 0x7FFFFFFu; }
__host__ __device__ constexpr int ax_stride(int ax) { return ax == 0 ? 1 : (ax == 1 ? 3 : 9); }
__host__ __device__ constexpr int line_pos(int g, int ax) { return (g / ax_stride(ax)) % 3; }
template <int D> __host__ __device__ constexpr unsigned orders_upto(int n) {
    unsigned m = 0;
    for (int g = 0; g < Grid<D>::N; ++g)
        if (morder<D>(g) <= n) m |= 1u << g;
    return m;
}
template <int L> __host__ __device__ constexpr unsigned retained_mask() {
    unsigned m = 0;
    for (int g = 0; g < Grid<Lat<L>::D>::N; ++g)
        if (retained<L>(g)) m |= 1u << g;
    return m;
}
// inputs read by a projection pass along ax for the outputs `need`: whole lines
template <int D> __host__ __device__ constexpr unsigned need_proj(unsigned need, int ax) {
    unsigned m = 0;
    const int S = ax_stride(ax);
    for (int g = 0; g < Grid<D>::N; ++g)
        if ((need >> g) & 1u) {
            const int b = g - line_pos(g, ax) * S;
            m |= (1u << b) | (1u << (b + S)) | (1u << (b + 2 * S));
        }
    return m;
}
// inputs read by a shift pass along ax for the outputs `need`: output k of a
// line reads entries 0..k of it
template <int D> __host__ __device__ constexpr unsigned need_shift(unsigned need, int ax) {
    unsigned m = 0;
    const int S = ax_stride(ax);
    for (int g = 0; g < Grid<D>::N; ++g)
        if ((need >> g) & 1u) {
            const int b = g - line_pos(g, ax) * S;
            for (int j = 0; j <= line_pos(g, ax); ++j) m |= 1u << (b + j * S);
        }
    return m;
}
// entries that may be non-zero after a shift pass along ax
template <int D> __host__ __device__ constexpr unsigned nz_shift(unsigned nz, int ax) {
    unsigned m = 0;
    const int S = ax_stride(ax);
    for (int g = 0; g < Grid<D>::N; ++g) {
        const int b = g - line_pos(g, ax) * S;
        for (int j = 0; j <= line_pos(g, ax); ++j)
            if ((nz >> (b + j * S)) & 1u) m |= 1u << g;
    }
    return m;
}

template <int I> struct Idx { static constexpr int value = I; };
template <int N, typename F, int I = 0> __host__ __device__ __forceinline__ void static_for(F &&f) {
    if constexpr (I < N) {
        f(Idx<I>{});
        static_for<N, F, I + 1>(static_cast<F &&>(f));
    }
}

// projection pass (proj_line) computing only the outputs in NEED
template <int D, int AX, unsigned NEED, typename R> __host__ __device__ __forceinline__ void proj_pass(R *a) {
    constexpr int S = ax_stride(AX);
    static_for<Grid<D>::N>([&](auto I) {
        constexpr int g = decltype(I)::value;
        if constexpr (line_pos(g, AX) == 0) {
            constexpr bool n0 = (NEED >> g) & 1u, n1 = (NEED >> (g + S)) & 1u, n2 = (NEED >> (g + 2 * S)) & 1u;
            if constexpr (n0 || n1 || n2) {
                const R m = a[g], z = a[g + S], p = a[g + 2 * S];
                const R s = p + m;
                if constexpr (n0) a[g] = s + z;
                if constexpr (n1) a[g + S] = p - m;
                if constexpr (n2) a[g + 2 * S] = (R(2) * s - z) * R(1.0 / 3.0);
            }
        }
    });
}

// shift pass (shift_line) computing only the outputs in NEED from inputs of
// which only those in NZ may be non-zero
template <int D, int AX, unsigned NZ, unsigned NEED, typename R>
__host__ __device__ __forceinline__ void shift_pass(R *a, R v) {
    constexpr int S = ax_stride(AX);
    static_for<Grid<D>::N>([&](auto I) {
        constexpr int g = decltype(I)::value;
        if constexpr (line_pos(g, AX) == 0) {
            constexpr bool z0 = (NZ >> g) & 1u, z1 = (NZ >> (g + S)) & 1u, z2 = (NZ >> (g + 2 * S)) & 1u;
            constexpr bool n0 = (NEED >> g) & 1u, n1 = (NEED >> (g + S)) & 1u, n2 = (NEED >> (g + 2 * S)) & 1u;
            const R a0 = z0 ? a[g] : R(0);
            const R a1 = z1 ? a[g + S] : R(0);
            if constexpr (n2) {
                if constexpr (z0 && z1 && z2) a[g + 2 * S] = a[g + 2 * S] + v * (R(2) * a1 + v * a0);
                else if constexpr (z0 && z1) a[g + 2 * S] = v * (R(2) * a1 + v * a0);
                else if constexpr (z0 && z2) a[g + 2 * S] = a[g + 2 * S] + v * (v * a0);
                else if constexpr (z1 && z2) a[g + 2 * S] = a[g + 2 * S] + v * (R(2) * a1);
                else if constexpr (z0) a[g + 2 * S] = v * (v * a0);
                else if constexpr (z1) a[g + 2 * S] = v * (R(2) * a1);
                else if constexpr (!z2) a[g + 2 * S] = R(0);
            }
            if constexpr (n1) {
                if constexpr (z0 && z1) a[g + S] = a1 + v * a0;
                else if constexpr (z0) a[g + S] = v * a0;
                else if constexpr (!z1) a[g + S] = R(0);
            }
            if constexpr (n0 && !z0) a[g] = R(0);
        }
    });
}

// SMRT with tau_3 = tau_4 = 1 (om3 = om4 = 1): the same collision as
// collide_smrt, whose orders-3/4 factors (1 - om) are then exactly zero,
// with the passes restricted to what is non-zero or read.
template <int L, typename R>
__host__ __device__ __forceinline__ void collide_smrt_trim(R *G, R gx, R gy, R gz, R om2) {
    constexpr int D = Lat<L>::D;
    constexpr int N = Grid<D>::N;
    constexpr int EX = 1, EY = 3, EZ = 9;
    constexpr unsigned LOW = orders_upto<D>(2);
    constexpr unsigned RET = retained_mask<L>();
    // projection: raw moments of orders <= 2 (a downward-closed set, so the
    // central shift below reads nothing else)
    constexpr unsigned P3 = LOW;
    constexpr unsigned P2 = D == 3 ? need_proj<D>(P3, 2) : LOW;
    constexpr unsigned P1 = need_proj<D>(P2, 1);
    proj_pass<D, 0, P1>(G);
    proj_pass<D, 1, P2>(G);
    if constexpr (D == 3) proj_pass<D, 2, P3>(G);
    const R drho = G[0];
    const R rho = R(1) + drho;
    const R inv = R(1) / rho;
    const R ux = G[EX] * inv + R(0.5) * gx;   // Eq. (half_F)
    const R uy = G[EY] * inv + R(0.5) * gy;
    const R uz = D == 3 ? G[EZ] * inv + R(0.5) * gz : R(0);
    G[0] = rho;
    constexpr unsigned ALL = grid_mask<D>();
    shift_pass<D, 0, ALL, LOW>(G, -ux);
    shift_pass<D, 1, ALL, LOW>(G, -uy);
    if constexpr (D == 3) shift_pass<D, 2, ALL, LOW>(G, -uz);
    // one relaxation time for the whole second order: a split bulk time runs
    // the general collision
    static_for<N>([&](auto I) {
        constexpr int g = decltype(I)::value;
        if constexpr (((LOW >> g) & 1u) && morder<D>(g) == 2) G[g] *= (R(1) - om2);
    });
    G[0] = rho;
    G[EX] = R(0.5) * rho * gx;
    G[EY] = R(0.5) * rho * gy;
    if constexpr (D == 3) G[EZ] = R(0.5) * rho * gz;
    // back to raw moments on the retained set: only orders <= 2 are non-zero
    constexpr unsigned S3 = RET;
    constexpr unsigned S2 = D == 3 ? need_shift<D>(S3, 2) : RET;
    constexpr unsigned S1 = need_shift<D>(S2, 1);
    constexpr unsigned Z1 = nz_shift<D>(LOW, 0) & S1;
    constexpr unsigned Z2 = nz_shift<D>(Z1, 1) & S2;
    shift_pass<D, 0, LOW, S1>(G, ux);
    shift_pass<D, 1, Z1, S2>(G, uy);
    if constexpr (D == 3) shift_pass<D, 2, Z2, S3>(G, uz);
    static_for<N>([&](auto I) {
        constexpr int g = decltype(I)::value;
        if constexpr (!((RET >> g) & 1u)) G[g] = R(0);
    });
    G[0] = drho;                          // deviation from the weights
    reconstruct<L>(G);
    if (L == D3Q19) {
#pragma unroll
        for (int i = 0; i < Lat<L>::Q; ++i) G[gpos<L>(i)] *= R(weight<L>(i));
    }
}

// SMRT with the force's non-equilibrium contributions (Eq. Frc, third and
// fourth terms): d_F^(n) = n g d^(n-1) in the co-moving frame for n <= 4, the
// product summed over the n positions of g, which on the grid of per-axis
// orders reads d_F[m] = sum_a m_a g_a d[m - e_a] (the monic per-axis
// polynomials satisfy h_k' = k h_(k-1), so this holds in lattice units).  d
// are the central moments of f itself, not of fbar: d^(1) = 0, and for n >= 2
// Eq. (newf) inverts to d^(n) = (1 - om_n/2)(dbar_1^(n) + d_F^(n)/2).  Hence
// d_F^(2) = 0, d_F^(3) = 3 g d^(2) and d_F^(4) = 4 g d^(3), each order needing
// the one below it.  Relaxation as in collide_smrt with these d_F added.
template <int L, typename R>
__host__ __device__ __forceinline__ void collide_smrt_fneq(R *G, R gx, R gy, R gz, R om2, R om3, R om4, R omb) {
    constexpr int D = Lat<L>::D;
    constexpr int N = Grid<D>::N;
    constexpr int EX = 1, EY = 3, EZ = 9;
    project<D>(G);
    const R drho = G[0];
    const R rho = R(1) + drho;
    const R inv = R(1) / rho;
    const R ux = G[EX] * inv + R(0.5) * gx;   // Eq. (half_F)
    const R uy = G[EY] * inv + R(0.5) * gy;
    const R uz = D == 3 ? G[EZ] * inv + R(0.5) * gz : R(0);
    G[0] = rho;
    shift<D>(G, -ux, -uy, -uz);           // central moments of fbar
    const R ga[3] = {gx, gy, gz};
    R d2[N], F3[N], d3[N];                // second- and third-order central moments of f, d_F^(3)
#pragma unroll
    for (int g = 0; g < N; ++g) d2[g] = morder<D>(g) == 2 ? G[g] : R(0);
    relax_order2<D>(d2, R(R(0.5) * om2), R(R(0.5) * omb));   // d^(2) = (1 - om/2) dbar_1^(2) per part
#pragma unroll
    for (int g = 0; g < N; ++g) {
        F3[g] = R(0);
        if (morder<D>(g) == 3) {
#pragma unroll
            for (int a = 0; a < D; ++a)
                if (mdig<D>(g, a) > 0) F3[g] += R(mdig<D>(g, a)) * ga[a] * d2[g - ax_stride(a)];
        }
        d3[g] = morder<D>(g) == 3 ? (R(1) - R(0.5) * om3) * (G[g] + R(0.5) * F3[g]) : R(0);
    }
    relax_order2<D>(G, om2, omb);
#pragma unroll
    for (int g = 0; g < N; ++g) {
        const int n = morder<D>(g);
        if (n == 3) G[g] = (R(1) - om3) * G[g] + (R(1) - R(0.5) * om3) * F3[g];
        else if (n == 4) {
            R F4 = R(0);
#pragma unroll
            for (int a = 0; a < D; ++a)
                if (mdig<D>(g, a) > 0) F4 += R(mdig<D>(g, a)) * ga[a] * d3[g - ax_stride(a)];
            G[g] = (R(1) - om4) * G[g] + (R(1) - R(0.5) * om4) * F4;
        } else if (n >= 5) G[g] = R(0);
    }
    G[0] = rho;
    G[EX] = R(0.5) * rho * gx;
    G[EY] = R(0.5) * rho * gy;
    if (D == 3) G[EZ] = R(0.5) * rho * gz;
    shift<D>(G, ux, uy, uz);              // back to raw moments: a_0 + a_p
#pragma unroll
    for (int g = 0; g < N; ++g)
        if (!retained<L>(g)) G[g] = R(0);
    G[0] = drho;                          // deviation from the weights
    reconstruct<L>(G);
    if (L == D3Q19) {
#pragma unroll
        for (int i = 0; i < Lat<L>::Q; ++i) G[gpos<L>(i)] *= R(weight<L>(i));
    }
}

// Raw-moment MRT of the appendix: the raw (not co-moving) non-equilibrium
// moments relax order by order,
//   a_p^(n) = a_0^(n) + (1 - om_n) a_1^(n) + (1 - om_n/2) a_F^(n),
// with a_1^(1) = -F/2, orders 2 and 3 projected, the fourth order from the
// appendix's recursion, and the force's equilibrium part
// a_F[m] = sum_a m_a rho g_a u^(m - e_a) (a_F^(n) = n F u^(n-1)).  The
// recursion is the statement that the fourth-order central moment of the
// non-equilibrium part vanishes, so it is applied as a round trip through
// the co-moving frame with the orders >= 4 dropped.
template <int L, typename R>
__host__ __device__ __forceinline__ void collide_mrt_raw(R *G, R gx, R gy, R gz, R om2, R om3, R om4) {
    constexpr int D = Lat<L>::D;
    constexpr int N = Grid<D>::N;
    constexpr int EX = 1, EY = 3, EZ = 9;
    project<D>(G);
    const R drho = G[0];
    const R rho = R(1) + drho;
    const R inv = R(1) / rho;
    const R ux = G[EX] * inv + R(0.5) * gx;   // Eq. (half_F)
    const R uy = G[EY] * inv + R(0.5) * gy;
    const R uz = D == 3 ? G[EZ] * inv + R(0.5) * gz : R(0);
    G[0] = rho;
    shift<D>(G, -ux, -uy, -uz);           // central moments of fbar; the equilibrium's are rho e_0
    G[0] = R(0);
    G[EX] = R(-0.5) * rho * gx;           // a_1^(1) = -F/2
    G[EY] = R(-0.5) * rho * gy;
    if (D == 3) G[EZ] = R(-0.5) * rho * gz;
#pragma unroll
    for (int g = 0; g < N; ++g)
        if (morder<D>(g) >= 4) G[g] = R(0);
    shift<D>(G, ux, uy, uz);              // raw non-equilibrium moments, recursive fourth order
    const R up[3][3] = {{R(1), ux, ux * ux}, {R(1), uy, uy * uy}, {R(1), uz, uz * uz}};
    const R ga[3] = {gx, gy, gz};
#pragma unroll
    for (int g = 0; g < N; ++g) {
        const int n = morder<D>(g);
        if (n == 0) {
            G[g] = drho;                  // deviation from the weights
        } else if (n <= 4 && retained<L>(g)) {
            R a0 = rho, aF = R(0);
#pragma unroll
            for (int a = 0; a < D; ++a) a0 *= up[a][mdig<D>(g, a)];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                if (mdig<D>(g, a) == 0) continue;
                R t = R(mdig<D>(g, a)) * rho * ga[a] * up[a][mdig<D>(g, a) - 1];
#pragma unroll
                for (int b = 0; b < D; ++b)
                    if (b != a) t *= up[b][mdig<D>(g, b)];
                aF += t;
            }
            const R om = n == 1 ? R(1) : (n == 2 ? om2 : (n == 3 ? om3 : om4));
            G[g] = n == 1 ? a0 + R(0.5) * aF : a0 + (R(1) - om) * G[g] + (R(1) - R(0.5) * om) * aF;
        } else {
            G[g] = R(0);
        }
    }
    reconstruct<L>(G);
    if (L == D3Q19) {
#pragma unroll
        for (int i = 0; i < Lat<L>::Q; ++i) G[gpos<L>(i)] *= R(weight<L>(i));
    }
}

// BGK with the second-order equilibrium and Guo-form force, Eq. (explict_eq)
template <int L, typename R>
__host__ __device__ __forceinline__ void collide_bgk(R *G, R gx, R gy, R gz, R om) {
    constexpr int Q = Lat<L>::Q;
    constexpr int D = Lat<L>::D;
    R drho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const R v = G[gpos<L>(i)];
        drho += v;
        if (Lat<L>::cx(i)) jx += Lat<L>::cx(i) > 0 ? v : -v;
        if (Lat<L>::cy(i)) jy += Lat<L>::cy(i) > 0 ? v : -v;
        if (D == 3 && Lat<L>::cz(i)) jz += Lat<L>::cz(i) > 0 ? v : -v;
    }
    const R rho = R(1) + drho;
    const R inv = R(1) / rho;
    const R ux = jx * inv + R(0.5) * gx, uy = jy * inv + R(0.5) * gy;
    const R uz = D == 3 ? jz * inv + R(0.5) * gz : R(0);
    const R uu15 = R(1.5) * (ux * ux + uy * uy + uz * uz);
    const R gu = gx * ux + gy * uy + gz * uz;
    const R fk = (R(1) - R(0.5) * om) * rho;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = Lat<L>::cx(i), cy = Lat<L>::cy(i), cz = Lat<L>::cz(i);
        const R cu = R(cx) * ux + R(cy) * uy + R(cz) * uz;
        const R cg = R(cx) * gx + R(cy) * gy + R(cz) * gz;
        const R w = R(weight<L>(i));
        const R deq = w * (drho + rho * (R(3) * cu + R(4.5) * cu * cu - uu15));
        const R Fi = w * fk * (R(3) * (cg - gu) + R(9) * cu * cg);
        R &v = G[gpos<L>(i)];
        v = v + om * (deq - v) + Fi;
    }
}

// initial deviations fbar - w = f_eq(rho, u) - F/2 - w for the model's own
// equilibrium and force; G receives the grid values
template <int L, int COLL, typename R>
__device__ __forceinline__ void initial_state(R *G, R drho, R ux, R uy, R uz, R gx, R gy, R gz) {
    constexpr int D = Lat<L>::D;
    constexpr int N = Grid<D>::N;
    const R rho = R(1) + drho;
    if (COLL == BGK) {
        const R uu15 = R(1.5) * (ux * ux + uy * uy + uz * uz);
        const R gu = gx * ux + gy * uy + gz * uz;
#pragma unroll
        for (int g = 0; g < N; ++g) G[g] = R(0);
#pragma unroll
        for (int i = 0; i < Lat<L>::Q; ++i) {
            const int cx = Lat<L>::cx(i), cy = Lat<L>::cy(i), cz = Lat<L>::cz(i);
            const R cu = R(cx) * ux + R(cy) * uy + R(cz) * uz;
            const R cg = R(cx) * gx + R(cy) * gy + R(cz) * gz;
            const R w = R(weight<L>(i));
            G[gpos<L>(i)] = w * (drho + rho * (R(3) * cu + R(4.5) * cu * cu - uu15)) -
                            R(0.5) * w * rho * (R(3) * (cg - gu) + R(9) * cu * cg);
        }
    } else {
#pragma unroll
        for (int g = 0; g < N; ++g) G[g] = R(0);
        G[0] = rho;
        G[1] = -R(0.5) * rho * gx;
        G[3] = -R(0.5) * rho * gy;
        if (D == 3) G[9] = -R(0.5) * rho * gz;
        shift<D>(G, ux, uy, uz);
#pragma unroll
        for (int g = 0; g < N; ++g)
            if (!retained<L>(g)) G[g] = R(0);
        G[0] = drho;
        reconstruct<L>(G);
        if (L == D3Q19) {
#pragma unroll
            for (int i = 0; i < Lat<L>::Q; ++i) G[gpos<L>(i)] *= R(weight<L>(i));
        }
    }
}

// ------------------------------------------------------------------ indexing
struct NodeNbr {
    int xs[3], ys[3], zs[3];   // source coordinate for c = -1, 0, +1 (x - c)
    bool xw[3], yw[3], zw[3];  // true when x - c lies beyond a wall
};

__device__ __forceinline__ void axis_src(int x, int n, int per, int *s, bool *w) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int c = k - 1;
        int v = x - c;
        bool wall = false;
        if (v < 0) { if (per) v += n; else { wall = true; v = 0; } }
        else if (v >= n) { if (per) v -= n; else { wall = true; v = n - 1; } }
        s[k] = v;
        w[k] = wall;
    }
}

// the same along the split axis of a slab: the source layer is always in
// the buffer (halo layers at both ends), and a wall only where the global
// layer leaves a domain that is not periodic on that axis
__device__ __forceinline__ void axis_src_halo(int v, int per, int g0, int gn, int *s, bool *w) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int t = v - (k - 1);
        const int g = g0 + t - 1;
        const bool wall = !per && (g < 0 || g >= gn);
        s[k] = wall ? v : t;
        w[k] = wall;
    }
}

__device__ __forceinline__ void node_nbr(const KParams &p, int x, int y, int z, NodeNbr &nb) {
    axis_src(x, p.nx, p.per[0], nb.xs, nb.xw);
    if (p.halo_ax == 1) axis_src_halo(y, p.per[1], p.hg0, p.hgn, nb.ys, nb.yw);
    else axis_src(y, p.ny, p.per[1], nb.ys, nb.yw);
    if (p.halo_ax == 2) axis_src_halo(z, p.per[2], p.hg0, p.hgn, nb.zs, nb.zw);
    else axis_src(z, p.nz, p.per[2], nb.zs, nb.zw);
}

// v is not at a face of axis ax (1: y, 2: z) of extent n: all three sources
// along it lie inside the buffer without wrap or wall
__device__ __forceinline__ bool inner(const KParams &p, int ax, int v, int n) {
    if (p.halo_ax == ax) {
        const int g = p.hg0 + v - 1;
        return p.per[ax] || (g > 0 && g < p.hgn - 1);
    }
    return v > 0 && v < n - 1;
}

__device__ __forceinline__ long long node_index(const KParams &p, int x, int y, int z) {
    return ((long long)z * p.ny + y) * p.nxp + x;
}

// pull the pre-collision deviations of node (x,y,z) onto the velocity grid:
// delta_i(x) = P_i(x - c_i), or P_opp(i)(x) across a wall or a solid node.
// Interior nodes use the precomputed per-population offsets; nodes on the
// domain faces resolve periodic wrap and walls per axis.
template <int L, int ST, bool MASK>
__device__ __forceinline__ void gather(const KParams &p, const typename Store<ST>::T *__restrict__ f,
                                       int x, int y, int z, typename Store<ST>::R *G) {
    typedef typename Store<ST>::R R;
    constexpr int D = Lat<L>::D;
    const long long own = node_index(p, x, y, z);
#pragma unroll
    for (int g = 0; g < Grid<D>::N; ++g) G[g] = R(0);
    // no wall and no wrap along y and z, and x inside the row or periodic: the
    // sources are fixed offsets from the node, from its left neighbour
    // (c_x = +1) or its right one (c_x = -1), those wrapped across a periodic
    // x face, so the first and last nodes of a row take this path too
    const bool interior = ((x > 0 && x < p.nx - 1) || p.per[0]) && inner(p, 1, y, p.ny) &&
                          (D == 2 || inner(p, 2, z, p.nz));
    if (interior) {
        const long long xl = x == 0 ? p.nx - 1 : -1;          // to x - 1
        const long long xr = x == p.nx - 1 ? 1 - p.nx : 1;    // to x + 1
        const typename Store<ST>::T *base = f + own, *basel = base + xl, *baser = base + xr;
#pragma unroll
        for (int i = 0; i < Lat<L>::Q; ++i) {
            const int cx = Lat<L>::cx(i);
            const long long sx = cx == 1 ? xl : (cx == -1 ? xr : 0);
            const typename Store<ST>::T *src = cx == 1 ? basel : (cx == -1 ? baser : base);
            if (MASK && i != 0 && p.solid[own + sx + p.noff[i]] != 0)
                G[gpos<L>(i)] = Store<ST>::ld(base + p.poff[opp<L>(i)]);
            else
                G[gpos<L>(i)] = Store<ST>::ld(src + p.doff[i]);
        }
        return;
    }
    NodeNbr nb;
    node_nbr(p, x, y, z, nb);
#pragma unroll
    for (int i = 0; i < Lat<L>::Q; ++i) {
        const int kx = Lat<L>::cx(i) + 1, ky = Lat<L>::cy(i) + 1, kz = Lat<L>::cz(i) + 1;
        bool wall = nb.xw[kx] || nb.yw[ky] || (D == 3 && nb.zw[kz]);
        const long long src = node_index(p, nb.xs[kx], nb.ys[ky], D == 3 ? nb.zs[kz] : z);
        if (MASK && i != 0 && !wall) wall = p.solid[src] != 0;
        const long long idx = wall ? p.poff[opp<L>(i)] + own : p.poff[i] + src;
        G[gpos<L>(i)] = Store<ST>::ld(f + idx);
    }
}

template <typename R> __device__ __forceinline__ const R *force_ptr(const KParams &p);
template <> __device__ __forceinline__ const double *force_ptr<double>(const KParams &p) { return p.g; }
template <> __device__ __forceinline__ const float *force_ptr<float>(const KParams &p) { return p.g32; }

// body-force acceleration at a node; `node` is the element index within a plane
template <int L, typename R>
__device__ __forceinline__ void load_force(const KParams &p, int y, long long node, R &gx, R &gy, R &gz) {
    constexpr int D = Lat<L>::D;
    const R *g = force_ptr<R>(p);
    gx = gy = gz = R(0);
    if (p.force_kind == G_UNIFORM) {
        gx = __ldg(g + 0);
        gy = __ldg(g + 1);
        if (D == 3) gz = __ldg(g + 2);
    } else if (p.force_kind == G_ROWS) {
        gx = __ldg(g + (long long)y * D + 0);
        gy = __ldg(g + (long long)y * D + 1);
        if (D == 3) gz = __ldg(g + (long long)y * D + 2);
    } else if (p.force_kind == G_FIELD) {
        gx = __ldg(g + node);
        gy = __ldg(g + p.plane + node);
        if (D == 3) gz = __ldg(g + 2 * p.plane + node);
    }
}

template <typename R> __device__ __forceinline__ R omega(const KParams &p, int n);
template <> __device__ __forceinline__ double omega<double>(const KParams &p, int n) { return p.om[n]; }
template <> __device__ __forceinline__ float omega<float>(const KParams &p, int n) { return p.om32[n]; }
template <typename R> __device__ __forceinline__ R omega_bulk(const KParams &p);
template <> __device__ __forceinline__ double omega_bulk<double>(const KParams &p) { return p.omb; }
template <> __device__ __forceinline__ float omega_bulk<float>(const KParams &p) { return p.omb32; }

}  // namespace lbm
