// lbm_f32x2.cuh -- two FP32 values that every arithmetic operation treats
// together, through the packed f32x2 instructions of sm_100 and later
// (add/sub/mul/fma.rn.f32x2 on a 64-bit register pair): one instruction issue
// for two nodes' worth of FP32 arithmetic.  The collision templates of
// lbm_device.cuh take it as their arithmetic type R, so one call collides
// two nodes; each lane of the pair gets exactly the IEEE round-to-nearest
// result of the corresponding scalar instruction.
//
// A product is kept unevaluated until it is used (F2Mul), so that a product
// added to or subtracted from a value becomes one fused multiply-add.  Which
// products fuse can differ from the compiler's choice for plain floats, so
// a node collided alone also runs through F2, with its values in both lanes
// (collide_one): every FP32 node then gets the same bits alone or paired,
// whatever the launch shape pairs it with.  That matters beyond
// reproducibility: a periodic row whose nodes all run one arithmetic keeps
// its translation symmetry exactly, whereas nodes rounding two ways break it
// at the last bit and the slow shear modes along the row keep FP32 noise
// alive, so a run to a tight steady-state residual stalls (measured: a
// 502 x 126 channel that settles in 50,000 steps stalled at r_K = 2e-8 with
// half its nodes paired and half alone).
#pragma once

namespace lbm {

struct F2 {
    unsigned long long v;   // low 32 bits: the first value, high 32 bits: the second
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ F2(double s) { set((float)s, (float)s); }
    __device__ __forceinline__ F2(float s) { set(s, s); }
    __device__ __forceinline__ F2(int s) { set((float)s, (float)s); }
    __device__ __forceinline__ static F2 pair(float a, float b) {
        F2 r;
        r.set(a, b);
        return r;
    }
    __device__ __forceinline__ static F2 bits(unsigned long long b) {
        F2 r;
        r.v = b;
        return r;
    }
    __device__ __forceinline__ void set(float a, float b) { asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(a), "f"(b)); }
    __device__ __forceinline__ void split(float &a, float &b) const {
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    }
    __device__ __forceinline__ float lo() const { return __uint_as_float((unsigned)v); }
    __device__ __forceinline__ float hi() const { return __uint_as_float((unsigned)(v >> 32)); }
};

__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 f2_sub(F2 a, F2 b) {
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 f2_fma(F2 a, F2 b, F2 c) {
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
// -a: both sign bits flipped (exact, like a scalar negation)
__device__ __forceinline__ F2 f2_neg(F2 a) { return F2::bits(a.v ^ 0x8000000080000000ull); }

// an unevaluated product a * b
struct F2Mul {
    F2 a, b;
    __device__ __forceinline__ operator F2() const { return f2_mul(a, b); }
};

__device__ __forceinline__ F2Mul operator*(F2 a, F2 b) { return {a, b}; }
__device__ __forceinline__ F2Mul operator*(F2Mul m, F2 c) { return {F2(m), c}; }
__device__ __forceinline__ F2Mul operator*(F2 c, F2Mul m) { return {c, F2(m)}; }
__device__ __forceinline__ F2Mul operator*(F2Mul m, F2Mul n) { return {F2(m), F2(n)}; }

__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return f2_add(a, b); }
__device__ __forceinline__ F2 operator+(F2Mul m, F2 c) { return f2_fma(m.a, m.b, c); }
__device__ __forceinline__ F2 operator+(F2 c, F2Mul m) { return f2_fma(m.a, m.b, c); }
__device__ __forceinline__ F2 operator+(F2Mul m, F2Mul n) { return f2_fma(m.a, m.b, F2(n)); }

__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return f2_sub(a, b); }
__device__ __forceinline__ F2 operator-(F2Mul m, F2 c) { return f2_fma(m.a, m.b, f2_neg(c)); }
__device__ __forceinline__ F2 operator-(F2 c, F2Mul m) { return f2_fma(f2_neg(m.a), m.b, c); }
__device__ __forceinline__ F2 operator-(F2Mul m, F2Mul n) { return f2_fma(m.a, m.b, f2_neg(F2(n))); }

__device__ __forceinline__ F2 operator-(F2 a) { return f2_neg(a); }
__device__ __forceinline__ F2Mul operator-(F2Mul m) { return F2Mul{f2_neg(m.a), m.b}; }

__device__ __forceinline__ F2 &operator+=(F2 &a, F2 b) { return a = f2_add(a, b); }
__device__ __forceinline__ F2 &operator+=(F2 &a, F2Mul m) { return a = f2_fma(m.a, m.b, a); }
__device__ __forceinline__ F2 &operator-=(F2 &a, F2 b) { return a = f2_sub(a, b); }
__device__ __forceinline__ F2 &operator*=(F2 &a, F2 b) { return a = f2_mul(a, b); }

// the IEEE quotient of one lane (div.rn.f32; inline PTX like the pair
// instructions, so that the compiler neither folds nor rewrites it)
__device__ __forceinline__ float f1_div(float a, float b) {
    float r;
    asm("div.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
// a / b per lane, each correctly rounded
__device__ __forceinline__ F2 operator/(F2 a, F2 b) { return F2::pair(f1_div(a.lo(), b.lo()), f1_div(a.hi(), b.hi())); }

}  // namespace lbm
