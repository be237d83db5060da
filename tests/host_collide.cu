// Host build of the fused kernel's per-node collision, for CPU tests: the
// __host__ __device__ collision functions the stream-collide kernel calls,
// applied to one node's stored deviations delta_i = fbar_i - w_i in double
// or float arithmetic, exactly as the kernel applies them after its gather.
// Test infrastructure only; nothing in the library calls it.
#include "../paper_2212_07494_gb300/csrc/lbm_device.cuh"

using namespace lbm;

namespace {

template <int L, typename R>
int run(int coll, const double *din, const double *g, const double *tau, double tau_bulk, double *dout) {
    R G[Grid<Lat<L>::D>::N];
    for (int k = 0; k < Grid<Lat<L>::D>::N; ++k) G[k] = R(0);
    for (int i = 0; i < Lat<L>::Q; ++i) G[gpos<L>(i)] = R(din[i]);
    // the kernel's relaxation rates: 1 / tau in FP64, rounded to the
    // arithmetic type (KParams om / om32)
    const R om2 = R(1.0 / tau[2]), om3 = R(1.0 / tau[3]), om4 = R(1.0 / tau[4]);
    const R omb = R(tau_bulk != 0.0 ? 1.0 / tau_bulk : 1.0 / tau[2]);
    const R gx = R(g[0]), gy = R(g[1]), gz = R(Lat<L>::D == 3 ? g[2] : 0.0);
    switch (coll) {
    case BGK: collide_bgk<L>(G, gx, gy, gz, om2); break;
    case SMRT: collide_smrt<L>(G, gx, gy, gz, om2, om3, om4, omb); break;
    case SMRT_FNEQ: collide_smrt_fneq<L>(G, gx, gy, gz, om2, om3, om4, omb); break;
    case MRT_RAW: collide_mrt_raw<L>(G, gx, gy, gz, om2, om3, om4); break;
    case SMRT_TRIM: collide_smrt_trim<L>(G, gx, gy, gz, om2); break;
    default: return -1;
    }
    for (int i = 0; i < Lat<L>::Q; ++i) dout[i] = (double)G[gpos<L>(i)];
    return 0;
}

// An arithmetic type that counts the additions (and subtractions),
// multiplications and divisions done on it: the collision templates
// instantiated with it give their operation counts per node, as written in
// the source, before the compiler fuses or hoists anything.
struct Cnt {
    double v;
    static long long add, mul, div;
    __host__ __device__ Cnt() : v(0) {}
    __host__ __device__ Cnt(double x) : v(x) {}
    __host__ __device__ explicit operator double() const { return v; }
};
long long Cnt::add = 0, Cnt::mul = 0, Cnt::div = 0;
#ifndef __CUDA_ARCH__
#define HC_COUNT(k) (++Cnt::k)
#else
#define HC_COUNT(k) ((void)0)
#endif
__host__ __device__ inline Cnt operator+(Cnt a, Cnt b) { HC_COUNT(add); return Cnt(a.v + b.v); }
__host__ __device__ inline Cnt operator-(Cnt a, Cnt b) { HC_COUNT(add); return Cnt(a.v - b.v); }
__host__ __device__ inline Cnt operator*(Cnt a, Cnt b) { HC_COUNT(mul); return Cnt(a.v * b.v); }
__host__ __device__ inline Cnt operator/(Cnt a, Cnt b) { HC_COUNT(div); return Cnt(a.v / b.v); }
__host__ __device__ inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
__host__ __device__ inline Cnt &operator+=(Cnt &a, Cnt b) { return a = a + b; }
__host__ __device__ inline Cnt &operator-=(Cnt &a, Cnt b) { return a = a - b; }
__host__ __device__ inline Cnt &operator*=(Cnt &a, Cnt b) { return a = a * b; }

template <int L> int count_ops(int coll, long long *out) {
    double din[Lat<L>::Q], dout[Lat<L>::Q];
    for (int i = 0; i < Lat<L>::Q; ++i) din[i] = 1e-3 * (i + 1);
    const double g[3] = {1e-6, -2e-6, 3e-6}, tau[5] = {1.0, 1.0, 0.8, 1.1, 1.2};
    Cnt::add = Cnt::mul = Cnt::div = 0;
    const int st = run<L, Cnt>(coll, din, g, tau, coll == SMRT_TRIM ? 0.0 : 0.9, dout);
    out[0] = Cnt::add;
    out[1] = Cnt::mul;
    out[2] = Cnt::div;
    return st;
}

template <int L> void velocities(int *c) {
    for (int i = 0; i < Lat<L>::Q; ++i) {
        c[3 * i + 0] = Lat<L>::cx(i);
        c[3 * i + 1] = Lat<L>::cy(i);
        c[3 * i + 2] = Lat<L>::cz(i);
    }
}

}  // namespace

// lat: 0 D2Q9, 1 D3Q19, 2 D3Q27; coll: 0 BGK, 1 SMRT, 2 SMRT_FNEQ,
// 3 MRT_RAW, 4 the trimmed SMRT (tau_3 = tau_4 = 1); fp32: float arithmetic.
// din/dout: Q deviations in the kernel's population order; g: 3 values in
// lattice units; tau: tau-hat per Hermite order (5 values).  0 or -1.
extern "C" int host_collide(int lat, int coll, int fp32, const double *din, const double *g, const double *tau,
                            double tau_bulk, double *dout) {
    if (lat == D2Q9) return fp32 ? run<D2Q9, float>(coll, din, g, tau, tau_bulk, dout)
                                 : run<D2Q9, double>(coll, din, g, tau, tau_bulk, dout);
    if (lat == D3Q19) return fp32 ? run<D3Q19, float>(coll, din, g, tau, tau_bulk, dout)
                                  : run<D3Q19, double>(coll, din, g, tau, tau_bulk, dout);
    if (lat == D3Q27) return fp32 ? run<D3Q27, float>(coll, din, g, tau, tau_bulk, dout)
                                  : run<D3Q27, double>(coll, din, g, tau, tau_bulk, dout);
    return -1;
}

// operations one collision of one node performs, as written: out[0]
// additions and subtractions, out[1] multiplications, out[2] divisions
extern "C" int host_collide_ops(int lat, int coll, long long *out) {
    if (lat == D2Q9) return count_ops<D2Q9>(coll, out);
    if (lat == D3Q19) return count_ops<D3Q19>(coll, out);
    if (lat == D3Q27) return count_ops<D3Q27>(coll, out);
    return -1;
}

// the kernel's velocity table: Q rows of (cx, cy, cz)
extern "C" int host_velocities(int lat, int *c) {
    if (lat == D2Q9) velocities<D2Q9>(c);
    else if (lat == D3Q19) velocities<D3Q19>(c);
    else if (lat == D3Q27) velocities<D3Q27>(c);
    else return -1;
    return 0;
}
