// lbm_unet.cu -- the steady-flow surrogate: a 4-level U-Net (widths
// 32/64/128/256, 3x3 convolutions with ReLU, 2x2 average pooling, nearest 2x
// upsampling followed by a convolution, skip concatenation, linear 3x3 head)
// trained with a weighted mean-squared error and Adam, entirely in this file's
// kernels.
//
// Activations are NHWC bfloat16; every contraction accumulates in FP32 on the
// tensor cores (mma.sync m16n8k16 BF16, operands staged by cp.async and read
// with ldmatrix).  Convolutions are implicit GEMMs:
//   forward      y[p][co]  = sum_{tap,ci} x[p+tap][ci] W[co][tap][ci]
//   input grad   dx[p][ci] = sum_{tap,co} dz[p-tap][co] W[co][tap][ci]
//                (the same kernel with the flipped, transposed weights)
//   weight grad  dW[co][tap][ci] = sum_p dz[p][co] x[p+tap][ci]
//                (split over pixel chunks, FP32 atomics; tcgen05 with
//                MN-major operands where the shape allows, else mma.sync)
// Concatenation is free: producers write into channel slices of one buffer.
// Master weights and Adam moments are FP32; each update repacks the BF16
// copies used by the forward and input-gradient kernels.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace unet {

typedef __nv_bfloat16 bf16;

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// 16-byte global -> shared copy; zero-filled when !valid (no bytes are read)
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst)), "l"(src), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// --------------------------------------------------------------- convolution
struct ConvArgs {
    const bf16 *x;
    int xc, xo;          // input channel stride / offset (multiples of 8)
    const bf16 *w;       // [wrows][9][cin]
    const float *bias;   // [cout] or null
    bf16 *y;             // output (null: only yf)
    int yc, yo;
    float *yf;           // optional FP32 output [pixel][yfc], channels < yfc
    int yfc;
    const bf16 *gate;    // optional: result *= (gate[p][go + co] > 0)
    int gc, go;
    int N, H, W, cin, cout, wrows;
    int relu;
    int wrapx;           // 1: periodic padding along x (the width), else zero padding
};

constexpr int CBM = 128, CBN = 64, CPAD = 8;

template <int BK>
__global__ void __launch_bounds__(256) k_conv(const ConvArgs a) {
    __shared__ __align__(16) bf16 As[2][CBM][BK + CPAD];
    __shared__ __align__(16) bf16 Bs[2][CBN][BK + CPAD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 3, wn = warp >> 2;
    const long long M = (long long)a.N * a.H * a.W;
    const long long m0 = (long long)blockIdx.x * CBM;
    const int co0 = blockIdx.y * CBN;
    constexpr int ACH = BK / 8;                 // 16-byte chunks per tile row
    constexpr int AREP = CBM * ACH / 256;       // A chunks per thread
    constexpr int BCH = CBN * ACH;              // B chunks per tile
    // pixel coordinates of this thread's A rows (fixed over the K loop)
    int an[AREP], ay[AREP], ax[AREP], arow[AREP], acc_[AREP];
#pragma unroll
    for (int i = 0; i < AREP; ++i) {
        const int q = tid + i * 256;
        arow[i] = q / ACH;
        acc_[i] = q % ACH;
        const long long m = m0 + arow[i];
        if (m < M) {
            const int hw = a.H * a.W;
            an[i] = (int)(m / hw);
            const int r = (int)(m - (long long)an[i] * hw);
            ay[i] = r / a.W;
            ax[i] = r - ay[i] * a.W;
        } else {
            an[i] = -1;
            ay[i] = ax[i] = 0;
        }
    }
    const int cblocks = a.cin / BK;
    const int KB = 9 * cblocks;
    auto load = [&](int kb, int buf) {
        const int tap = kb / cblocks, c0 = (kb - tap * cblocks) * BK;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
#pragma unroll
        for (int i = 0; i < AREP; ++i) {
            const int yy = ay[i] + dy;
            int xx = ax[i] + dx;
            if (a.wrapx) xx = xx < 0 ? xx + a.W : (xx >= a.W ? xx - a.W : xx);
            const bool ok = an[i] >= 0 && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
            const bf16 *src = ok ? a.x + ((long long)(an[i] * a.H + yy) * a.W + xx) * a.xc + a.xo + c0 + acc_[i] * 8 : a.x;
            cp_async16(&As[buf][arow[i]][acc_[i] * 8], src, ok);
        }
        for (int q = tid; q < BCH; q += 256) {
            const int r = q / ACH, cc = q % ACH;
            const int co = co0 + r;
            const bool ok = co < a.wrows;
            const bf16 *src = ok ? a.w + (long long)co * 9 * a.cin + tap * a.cin + c0 + cc * 8 : a.w;
            cp_async16(&Bs[buf][r][cc * 8], src, ok);
        }
        cp_async_commit();
    };
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;
    load(0, 0);
    for (int kb = 0; kb < KB; ++kb) {
        const int buf = kb & 1;
        if (kb + 1 < KB) {
            load(kb + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK / 16; ++ks) {
            unsigned af[2][4], bfr[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
                ldsm_x4(af[mt], &As[buf][wm * 32 + mt * 16 + (lane & 15)][ks * 16 + (lane >> 4) * 8]);
#pragma unroll
            for (int p = 0; p < 2; ++p)
                ldsm_x4(bfr[p], &Bs[buf][wn * 32 + p * 16 + (lane & 7) + (lane >> 4) * 8][ks * 16 + ((lane >> 3) & 1) * 8]);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
                    mma16816(acc[mt][nt], af[mt], bfr[nt >> 1][(nt & 1) * 2], bfr[nt >> 1][(nt & 1) * 2 + 1]);
        }
        __syncthreads();
    }
    // epilogue: bias, ReLU, gate, store
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long m = m0 + wm * 32 + mt * 16 + (lane >> 2) + h * 8;
                const int co = co0 + wn * 32 + nt * 8 + (lane & 3) * 2;
                if (m >= M || co >= a.cout) continue;
                float v[2] = {acc[mt][nt][h * 2], acc[mt][nt][h * 2 + 1]};
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    if (co + e >= a.cout) continue;
                    if (a.bias) v[e] += a.bias[co + e];
                    if (a.relu) v[e] = fmaxf(v[e], 0.f);
                    if (a.gate && !(__bfloat162float(a.gate[m * a.gc + a.go + co + e]) > 0.f)) v[e] = 0.f;
                    if (a.yf && co + e < a.yfc) a.yf[m * a.yfc + co + e] = v[e];
                }
                if (a.y) {
                    bf16 *dst = a.y + m * a.yc + a.yo + co;
                    if (co + 1 < a.cout) {
                        *reinterpret_cast<__nv_bfloat162 *>(dst) = __floats2bfloat162_rn(v[0], v[1]);
                    } else {
                        dst[0] = __float2bfloat16_rn(v[0]);
                    }
                }
            }
}

// ------------------------------------------- convolution on tcgen05 (TMEM)
// The same implicit GEMM as k_conv on the 5th-generation tensor cores: a CTA
// computes 128 pixels x NT output channels, accumulating in TMEM (128 lanes x
// NT FP32 columns).  Operand tiles are staged by cp.async into shared memory
// in the swizzled K-major layout the MMA reads through matrix descriptors.
// A tile row (one pixel, or one output channel of the weights) is the K
// block's BK channels, ROWB = 2 BK bytes; rows follow each other at ROWB, and
// the 16-byte chunk c of row r sits at chunk position c XOR sw(r), with
// sw(r) = r mod 8 (BK 64, 128-byte swizzle), (r / 2) mod 4 (BK 32, 64-byte)
// or (r / 4) mod 2 (BK 16, 32-byte): the address bits 4.. XORed with bits
// 7.., which is the pattern of the descriptor's swizzle modes.  Eight rows
// form one swizzle atom, so 8-row groups are 8 ROWB apart (the descriptor's
// stride offset); a whole row is one atom wide, so the MMA's K slices of 16
// channels start 32 bytes apart within it.  The pattern lets a warp copy
// whole pixel rows (coalesced global reads) into shared memory without bank
// conflicts.
constexpr long TC_SPIN = 1L << 22;

template <int BK> __host__ __device__ constexpr int sw_rowbytes() { return 2 * BK; }
// descriptor swizzle mode for a row of 2 BK bytes: 2 = 128B, 4 = 64B, 6 = 32B
template <int BK> __host__ __device__ constexpr uint64_t sw_mode() { return BK == 64 ? 2 : (BK == 32 ? 4 : 6); }
template <int BK> __device__ __forceinline__ int sw_off(int r, int c) {
    const int x = BK == 64 ? (r & 7) : (BK == 32 ? ((r >> 1) & 3) : ((r >> 2) & 1));
    return r * sw_rowbytes<BK>() + ((c ^ x) << 4);
}

template <int BK> __device__ __forceinline__ uint64_t tc_desc_sw(unsigned saddr) {
    constexpr unsigned SBO = 8 * sw_rowbytes<BK>();
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                    // leading offset: unused by the swizzled K-major layout
    d |= (uint64_t)((SBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;                    // descriptor version of the sm_100 family; base offset 0
    d |= sw_mode<BK>() << 61;
    return d;
}
// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// k_conv_ws: the convolution, warp-specialised, 5 warps.  Warps 0-3
// are producers, warp w owning stage w (K blocks kb = w, w + 4, ...): it
// waits until the MMAs that last read its stage are done (empty[w]), fills
// the stage with cp.async, waits for its own copies only, fences them into
// the async proxy and arrives on full[w].  Warp 4 issues the MMAs: for each
// K block it waits full[s], issues BK / 16 MMAs and commits them to empty[s];
// after the last block it commits to done.  Then warps 0-3 read their TMEM
// lane quarter for the epilogue.  Four stages are in flight, and no thread
// waits on copies it did not issue.  Every wait is bounded and gives up when
// another thread has failed (s_fail).
constexpr int WS_S = 4;

__device__ __forceinline__ bool ws_wait(unsigned long long *mbar, unsigned parity, volatile int *fail) {
    for (long it = 0; it < TC_SPIN; ++it) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t"
            "}\n"
            : "=r"(ok)
            : "r"(smem_addr(mbar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (*fail) return false;
        if (it > 64) __nanosleep(32);
    }
    *fail = 1;
    return false;
}

// Epilogue of the tcgen05 convolutions: warp w (0-3) reads TMEM lanes
// 32w .. 32w + 31, one output pixel per thread (m; -1: none), NT FP32
// columns, adds the bias, applies ReLU and the gate, and stores bf16.
template <int NT>
__device__ __forceinline__ void conv_epilogue(const ConvArgs &a, unsigned tmem, int warp, int lane, long long m,
                                              int co0) {
#pragma unroll
    for (int c = 0; c < NT; c += 16) {
        unsigned r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
            "[%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15])
            : "r"(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int cb = co0 + c;
        if (m < 0 || cb >= a.cout) continue;
        float v[16];
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
            v[jj] = __uint_as_float(r[jj]);
            if (a.bias && cb + jj < a.cout) v[jj] += a.bias[cb + jj];
            if (a.relu) v[jj] = fmaxf(v[jj], 0.f);
        }
        if (a.gate) {
#pragma unroll
            for (int jj = 0; jj < 16; ++jj)
                if (cb + jj < a.cout && !(__bfloat162float(a.gate[m * a.gc + a.go + cb + jj]) > 0.f)) v[jj] = 0.f;
        }
        bf16 *dst = a.y + m * a.yc + a.yo + cb;
        if (cb + 16 <= a.cout) {
            __align__(16) __nv_bfloat162 o[8];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) o[jj] = __floats2bfloat162_rn(v[2 * jj], v[2 * jj + 1]);
            reinterpret_cast<uint4 *>(dst)[0] = reinterpret_cast<const uint4 *>(o)[0];
            reinterpret_cast<uint4 *>(dst)[1] = reinterpret_cast<const uint4 *>(o)[1];
        } else {
            for (int jj = 0; jj < 16 && cb + jj < a.cout; ++jj) dst[jj] = __float2bfloat16_rn(v[jj]);
        }
    }
}

template <int BK, int NT>
__global__ void __launch_bounds__(160) k_conv_ws(const ConvArgs a, int *err) {
    constexpr int ABYTES = 128 * BK * 2, BBYTES = NT * BK * 2, STAGE = ABYTES + BBYTES;
    constexpr int NCOL = NT < 32 ? 32 : NT;
    constexpr int CH = BK / 8;    // 16-byte chunks per tile row
    constexpr int RPW = 32 / CH;  // tile rows per warp-wide copy
    // every stage and both tiles start on a swizzle atom (8 rows)
    static_assert(NT % RPW == 0 && STAGE % (16 * BK) == 0 && ABYTES % (16 * BK) == 0, "tile shape");
    extern __shared__ __align__(1024) unsigned char ws_smem[];
    __shared__ __align__(8) unsigned long long full[WS_S], empty[WS_S], done;
    __shared__ unsigned tmem_base;
    __shared__ volatile int s_fail;
    __shared__ int s_rows[128][3];  // (image, y, x) of the tile's pixels; image -1 past the end
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *sm = (unsigned char *)(((uintptr_t)ws_smem + 1023) & ~(uintptr_t)1023);
    const long long M = (long long)a.N * a.H * a.W;
    const long long m0 = (long long)blockIdx.x * 128;
    const int co0 = blockIdx.y * NT;
    const int cblocks = a.cin / BK;
    const int KB = 9 * cblocks;
    if (tid < 128) {
        const long long m = m0 + tid;
        int an = -1, ay = 0, ax = 0;
        if (m < M) {
            const int hw = a.H * a.W;
            an = (int)(m / hw);
            const int r = (int)(m - (long long)an * hw);
            ay = r / a.W;
            ax = r - ay * a.W;
        }
        s_rows[tid][0] = an;
        s_rows[tid][1] = ay;
        s_rows[tid][2] = ax;
    }
    if (tid == 0) {
        s_fail = 0;
        for (int s = 0; s < WS_S; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&full[s])), "r"(32));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&empty[s])), "r"(1));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&done)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(NCOL));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = tmem_base;
    if (warp < WS_S) {
        // ---- producer of stage `warp`: each warp-wide copy moves RPW whole
        // tile rows, lane l taking chunk l % CH of row l / CH (pixel
        // coordinates from s_rows), then the same for the weight rows
        unsigned char *sa = sm + warp * STAGE, *sb = sa + ABYTES;
        const int lr = lane / CH, lc = lane % CH;
        for (int kb = warp, j = 0; kb < KB; kb += WS_S, ++j) {
            if (j >= 1 && !ws_wait(&empty[warp], (j - 1) & 1, &s_fail)) break;
            const int tap = kb / cblocks, c0 = (kb - tap * cblocks) * BK;
            const int dy = tap / 3 - 1, dx = tap % 3 - 1;
#pragma unroll 4
            for (int r0 = 0; r0 < 128; r0 += RPW) {
                const int r = r0 + lr;
                const int an = s_rows[r][0];
                const int yy = s_rows[r][1] + dy;
                int xx = s_rows[r][2] + dx;
                if (a.wrapx) xx = xx < 0 ? xx + a.W : (xx >= a.W ? xx - a.W : xx);
                const bool ok = an >= 0 && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
                const bf16 *src = ok ? a.x + ((long long)(an * a.H + yy) * a.W + xx) * a.xc + a.xo + c0 + lc * 8 : a.x;
                cp_async16(sa + sw_off<BK>(r, lc), src, ok);
            }
#pragma unroll 4
            for (int r0 = 0; r0 < NT; r0 += RPW) {
                const int r = r0 + lr;
                const int co = co0 + r;
                const bool ok = co < a.wrows;
                const bf16 *src = ok ? a.w + (long long)co * 9 * a.cin + tap * a.cin + c0 + lc * 8 : a.w;
                cp_async16(sb + sw_off<BK>(r, lc), src, ok);
            }
            cp_async_commit();
            cp_async_wait<0>();
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                smem_addr(&full[warp]))
                         : "memory");
        }
        cp_async_wait<0>();
    } else if (lane == 0) {
        // ---- MMA issuer
        constexpr uint32_t IDESC = tc_idesc(128, NT);
        int kb = 0;
        for (; kb < KB; ++kb) {
            const int s = kb % WS_S;
            if (!ws_wait(&full[s], (kb / WS_S) & 1, &s_fail)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const unsigned sa = smem_addr(sm + s * STAGE), sb = sa + ABYTES;
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
                const uint64_t da = tc_desc_sw<BK>(sa + ks * 32);
                const uint64_t db = tc_desc_sw<BK>(sb + ks * 32);
                const unsigned acc = (kb > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t"
                    "}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(IDESC), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(&empty[s])));
        }
        // done completes when every MMA issued above has (after a failure: the
        // ones issued before it)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(&done)));
    }
    if (warp < WS_S) {
        const bool ok = ws_wait(&done, 0, &s_fail) && !s_fail;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (ok) conv_epilogue<NT>(a, tmem, warp, lane, m0 + warp * 32 + lane < M ? m0 + warp * 32 + lane : -1, co0);
    }
    if (tid == 0 && s_fail) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL));
}

// k_conv_tma: the same convolution with the operand tiles fetched by the
// Tensor Memory Accelerator.  A tile is one x column: its 128 pixels are HB
// consecutive rows y of NB images at one x (HB = min(H, 128), NB = 128 / HB).
// A tap's shift dx moves the whole box to column x + dx (periodic padding:
// modulo W; zero padding: a column outside the image reads as zeros), and dy
// shifts its rows, those outside the image reading as zeros (the walls'
// zero padding).  The activation box is channels c0 .. c0 + BK of
// (x, rows, images) in a 4-D tensor map over [N][H][W][xc]; the weight box
// is BK taps-and-channels of NT output channels in a 2-D map over
// [wrows][9 cin].  Both land in the swizzled K-major layout of k_conv_ws.
// One thread issues a stage's two copies after announcing their bytes on
// full[s] (arrive.expect_tx), so every stage can be in flight at once; the
// MMA warp and the epilogue are k_conv_ws's.  Every wait is bounded; after a
// failure the producer waits (bounded) for the copies it still has in flight
// before the TMEM is freed and the CTA exits.  Four stages by default, so
// several CTAs share an SM; DEEP (for grids of under two CTAs per SM, where
// nothing else hides a stage's latency) fills about 192 KB with up to 8.
template <int BK, int NT> constexpr int tma_stage_bytes() { return (128 * BK * 2 + NT * BK * 2 + 1023) & ~1023; }
template <int BK, int NT, bool DEEP> constexpr int tma_stages() {
    return !DEEP ? 4
         : (196608 / tma_stage_bytes<BK, NT>() < 4 ? 4
         : (196608 / tma_stage_bytes<BK, NT>() > 8 ? 8 : 196608 / tma_stage_bytes<BK, NT>()));
}

template <int BK, int NT, bool DEEP>
__global__ void __launch_bounds__(160) k_conv_tma(const ConvArgs a, const __grid_constant__ CUtensorMap tmA,
                                                  const __grid_constant__ CUtensorMap tmB, int HB, int NB, int *err) {
    constexpr int ABYTES = 128 * BK * 2, BBYTES = NT * BK * 2;
    constexpr int STAGE = tma_stage_bytes<BK, NT>();
    constexpr int TMA_S = tma_stages<BK, NT, DEEP>();
    constexpr int NCOL = NT < 32 ? 32 : NT;
    extern __shared__ __align__(1024) unsigned char tm_smem[];
    __shared__ __align__(8) unsigned long long full[TMA_S], empty[TMA_S], done;
    __shared__ unsigned tmem_base;
    __shared__ volatile int s_fail;
    __shared__ int s_consumed;  // K blocks the MMA warp received
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *sm = (unsigned char *)(((uintptr_t)tm_smem + 1023) & ~(uintptr_t)1023);
    const int ytiles = a.H / HB;
    const int xcol = blockIdx.x % a.W;
    const int rest = blockIdx.x / a.W;
    const int yt = rest % ytiles, ng = rest / ytiles;
    const int co0 = blockIdx.y * NT;
    const int cblocks = a.cin / BK;
    const int KB = 9 * cblocks;
    if (tid == 0) {
        s_fail = 0;
        s_consumed = 0;
        for (int s = 0; s < TMA_S; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&full[s])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&empty[s])), "r"(1));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&done)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(NCOL));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = tmem_base;
    int issued = 0;
    if (tid == 0) {
        // ---- producer
        const uint64_t pa = reinterpret_cast<uint64_t>(&tmA), pb = reinterpret_cast<uint64_t>(&tmB);
        for (int kb = 0; kb < KB; ++kb) {
            const int s = kb % TMA_S;
            if (kb >= TMA_S && !ws_wait(&empty[s], (kb / TMA_S - 1) & 1, &s_fail)) break;
            const int tap = kb / cblocks, c0 = (kb - tap * cblocks) * BK;
            const int dy = tap / 3 - 1, dx = tap % 3 - 1;
            int xx = xcol + dx;
            if (a.wrapx) xx = xx < 0 ? xx + a.W : (xx >= a.W ? xx - a.W : xx);
            const unsigned sa = smem_addr(sm + s * STAGE), sb = sa + ABYTES, mb = smem_addr(&full[s]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(ABYTES + BBYTES)
                         : "memory");
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                "%4, %5}], [%6];" ::"r"(sa),
                "l"(pa), "r"(c0), "r"(xx), "r"(yt * HB + dy), "r"(ng * NB), "r"(mb)
                : "memory");
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                "[%4];" ::"r"(sb),
                "l"(pb), "r"(tap * a.cin + c0), "r"(co0), "r"(mb)
                : "memory");
            issued = kb + 1;
        }
    } else if (warp == 4 && lane == 0) {
        // ---- MMA issuer
        constexpr uint32_t IDESC = tc_idesc(128, NT);
        int kb = 0;
        for (; kb < KB; ++kb) {
            const int s = kb % TMA_S;
            if (!ws_wait(&full[s], (kb / TMA_S) & 1, &s_fail)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const unsigned sa = smem_addr(sm + s * STAGE), sb = sa + ABYTES;
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
                const uint64_t da = tc_desc_sw<BK>(sa + ks * 32);
                const uint64_t db = tc_desc_sw<BK>(sb + ks * 32);
                const unsigned acc = (kb > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t"
                    "}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(IDESC), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(&empty[s])));
        }
        s_consumed = kb;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(&done)));
    }
    if (warp < 4) {
        // warp-uniform: the epilogue's TMEM loads are warp-aligned
        const bool ok = __all_sync(0xffffffffu, ws_wait(&done, 0, &s_fail) && !s_fail);
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (ok) {
            const int r = warp * 32 + lane;
            const long long n = (long long)ng * NB + r / HB;
            const int y = yt * HB + r % HB;
            conv_epilogue<NT>(a, tmem, warp, lane, (n * a.H + y) * a.W + xcol, co0);
        }
    }
    __syncthreads();
    if (tid == 0 && s_fail) {
        // copies still in flight land, and issued MMAs finish, before the
        // CTA frees its TMEM and leaves
        volatile int never = 0;
        for (int kb = s_consumed; kb < issued; ++kb) ws_wait(&full[kb % TMA_S], (kb / TMA_S) & 1, &never);
        ws_wait(&done, 0, &never);
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL));
}

// ------------------------------------------------------------ weight gradient
struct WgradArgs {
    const bf16 *dz;
    int dzc, dzo;   // gradient with respect to the conv output (pre-activation)
    const bf16 *x;
    int xc, xo;     // conv input
    float *dw;      // [wrows][9][cin]
    int N, H, W, cin, cout;
    int pix;        // pixels per block
    int wrapx;      // periodic padding along x
};

constexpr int WBM = 64, WBN = 32, WBK = 32, WPAD = 8;

__global__ void __launch_bounds__(128) k_wgrad(const WgradArgs a) {
    __shared__ __align__(16) bf16 As[2][WBK][WBM + WPAD];  // [pixel][co]
    __shared__ __align__(16) bf16 Bs[2][WBK][WBN + WPAD];  // [pixel][ci]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const long long P = (long long)a.N * a.H * a.W;
    const long long p_begin = (long long)blockIdx.x * a.pix;
    const long long p_end = p_begin + a.pix < P ? p_begin + a.pix : P;
    const int co0 = blockIdx.y * WBM;
    const int cblocks = (a.cin + WBN - 1) / WBN;
    const int tap = blockIdx.z / cblocks, ci0 = (blockIdx.z % cblocks) * WBN;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const int hw = a.H * a.W;
    auto load = [&](long long p0, int buf) {
        // A: 32 pixels x 64 co = 256 chunks, two per thread
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int q = tid + i * 128;
            const int r = q >> 3, cc = q & 7;
            const long long p = p0 + r;
            const int co = co0 + cc * 8;
            const bool ok = p < p_end && co < a.cout;
            const bf16 *src = ok ? a.dz + p * a.dzc + a.dzo + co : a.dz;
            cp_async16(&As[buf][r][cc * 8], src, ok);
        }
        // B: 32 pixels x 32 ci = 128 chunks, one per thread (input shifted by the tap)
        {
            const int r = tid >> 2, cc = tid & 3;
            const long long p = p0 + r;
            bool ok = p < p_end && ci0 + cc * 8 < a.cin;
            const bf16 *src = a.x;
            if (ok) {
                const int n = (int)(p / hw);
                const int rr = (int)(p - (long long)n * hw);
                const int yy = rr / a.W + dy;
                int xx = rr % a.W + dx;
                if (a.wrapx) xx = xx < 0 ? xx + a.W : (xx >= a.W ? xx - a.W : xx);
                ok = yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
                if (ok) src = a.x + ((long long)(n * a.H + yy) * a.W + xx) * a.xc + a.xo + ci0 + cc * 8;
            }
            cp_async16(&Bs[buf][r][cc * 8], src, ok);
        }
        cp_async_commit();
    };
    float acc[2][2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;
    const int KB = (int)((p_end - p_begin + WBK - 1) / WBK);
    if (KB > 0) load(p_begin, 0);
    for (int kb = 0; kb < KB; ++kb) {
        const int buf = kb & 1;
        if (kb + 1 < KB) {
            load(p_begin + (long long)(kb + 1) * WBK, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < WBK / 16; ++ks) {
            unsigned af[2][4], bfr[4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
                ldsm_x4_t(af[mt], &As[buf][ks * 16 + (lane & 7) + (lane >> 4) * 8][wm * 32 + mt * 16 + ((lane >> 3) & 1) * 8]);
            ldsm_x4_t(bfr, &Bs[buf][ks * 16 + (lane & 7) + ((lane >> 3) & 1) * 8][wn * 16 + (lane >> 4) * 8]);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) mma16816(acc[mt][nt], af[mt], bfr[nt * 2], bfr[nt * 2 + 1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int co = co0 + wm * 32 + mt * 16 + (lane >> 2) + (e >> 1) * 8;
                const int ci = ci0 + wn * 16 + nt * 8 + (lane & 3) * 2 + (e & 1);
                if (co < a.cout && ci < a.cin) atomicAdd(a.dw + ((long long)co * 9 + tap) * a.cin + ci, acc[mt][nt][e]);
            }
}

// ------------------------------------------- weight gradient on tcgen05 (TMEM)
// dW[co][tap][ci] = sum_p dz[p][co] x[p + tap][ci] as one GEMM per CTA on the
// 5th-generation tensor cores, D[m][co] += sum_p A[m][p] B[co][p]: a row m of
// D is one input channel of one (tap, channel block) pair, 128 rows per CTA
// (128 / CA pairs of CA channels), and N = the layer's padded output
// channels.  The contraction runs over pixels in blocks of 64 along one x
// column: HB rows y of NB images (HB NB = 64), as the forward kernel's column
// tiles.  The x operand of pair (tap, block) for a pixel block is the TMA box
// at column x + dx (modulo W, or reading zeros outside the image) and rows
// y + dy (zeros outside), the dz operand the unshifted box, so every operand
// is one plain 4-D box per atom.
// Both operands arrive channel-contiguous, i.e. MN-major: an atom is CA (A)
// or CB (B) channels wide -- the swizzle width, 64 -> 128 B, 32 -> 64 B,
// 16 -> 32 B -- and 64 pixel rows deep; the atoms of an operand lie one atom
// apart (the descriptor's leading offset), 8-row pixel groups 8 rows apart
// (its stride offset), and the MMA's K slices of 16 pixels start 16 rows
// apart.  The instruction descriptor marks both operands MN-major.  CTAs
// split the pixel blocks between them and add their 128 x N partial sums to
// dW with FP32 atomics.  One thread issues the copies, one the MMAs; four
// stages; every wait is bounded, as in k_conv_tma.
struct WgTcArgs {
    float *dw;           // [cout][9][cin]
    int cin, cout;       // padded channels (cout = the MMA's N)
    int H, W;
    int HB, NB;          // a pixel block: HB rows of NB images at one x
    int wrapx;
    int CA, CB;          // atom widths of the x and dz operands (channels)
    int pairs;           // 9 cin / CA (tap, channel block) pairs
    long long kb_total;  // pixel blocks
    int kb_per;          // pixel blocks per CTA
    unsigned ncol;       // TMEM columns (power of two >= 32, >= cout)
};
constexpr int WG_S = 4;
constexpr unsigned WG_ABYTES = 128 * 64 * 2;  // the x operand: 128 rows of 64 pixels
constexpr unsigned wg_stage_bytes(int cout) { return WG_ABYTES + (unsigned)cout * 64 * 2; }

__device__ __forceinline__ uint64_t sw_mode_bytes(int rowbytes) { return rowbytes == 128 ? 2 : (rowbytes == 64 ? 4 : 6); }

// shared memory descriptor of an MN-major swizzled operand
__device__ __forceinline__ uint64_t tc_desc_mn(unsigned saddr, unsigned lbo, unsigned sbo, uint64_t mode) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= mode << 61;
    return d;
}

__device__ __forceinline__ void tma_load4(unsigned dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                          unsigned mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
        : "memory");
}

__global__ void __launch_bounds__(160) k_wgrad_tc(const WgTcArgs a, const __grid_constant__ CUtensorMap tmX,
                                                  const __grid_constant__ CUtensorMap tmZ, int *err) {
    extern __shared__ __align__(1024) unsigned char wg_smem[];
    __shared__ __align__(8) unsigned long long full[WG_S], empty[WG_S], done;
    __shared__ unsigned tmem_base;
    __shared__ volatile int s_fail;
    __shared__ int s_consumed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *sm = (unsigned char *)(((uintptr_t)wg_smem + 1023) & ~(uintptr_t)1023);
    const unsigned STAGE = wg_stage_bytes(a.cout);
    const int per_tile = 128 / a.CA;                // pairs per CTA
    const int p0 = blockIdx.y * per_tile;
    const int np = min(per_tile, a.pairs - p0);     // pairs this CTA loads (>= 1)
    const int cblocks = a.cin / a.CA;
    const int ytiles = a.H / a.HB;
    const int nb_atoms = a.cout / a.CB;
    const unsigned arow = 2u * a.CA, brow = 2u * a.CB;      // bytes of one pixel row of an atom
    const unsigned aatom = 64u * arow, batom = 64u * brow;  // bytes of one atom
    const long long kb0 = (long long)blockIdx.x * a.kb_per;
    const int KB = (int)min((long long)a.kb_per, a.kb_total - kb0);  // >= 1
    if (tid == 0) {
        s_fail = 0;
        s_consumed = 0;
        for (int s = 0; s < WG_S; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&full[s])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&empty[s])), "r"(1));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&done)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(a.ncol));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = tmem_base;
    int issued = 0;
    if (tid == 0) {
        // ---- producer: np x boxes and nb_atoms dz boxes per pixel block
        const unsigned tx = (unsigned)np * aatom + (unsigned)nb_atoms * batom;
        for (int i = 0; i < KB; ++i) {
            const int s = i % WG_S;
            if (i >= WG_S && !ws_wait(&empty[s], (i / WG_S - 1) & 1, &s_fail)) break;
            const long long kb = kb0 + i;
            const int xcol = (int)(kb % a.W);
            const long long rest = kb / a.W;
            const int y0 = (int)(rest % ytiles) * a.HB, n0 = (int)(rest / ytiles) * a.NB;
            const unsigned sa = smem_addr(sm + (size_t)s * STAGE), sb = sa + WG_ABYTES, mb = smem_addr(&full[s]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(tx) : "memory");
            for (int j = 0; j < np; ++j) {
                const int pr = p0 + j;
                const int tap = pr / cblocks, c0 = (pr - tap * cblocks) * a.CA;
                const int dy = tap / 3 - 1, dx = tap % 3 - 1;
                int xx = xcol + dx;
                if (a.wrapx) xx = xx < 0 ? xx + a.W : (xx >= a.W ? xx - a.W : xx);
                tma_load4(sa + j * aatom, &tmX, c0, xx, y0 + dy, n0, mb);
            }
            for (int j = 0; j < nb_atoms; ++j) tma_load4(sb + j * batom, &tmZ, j * a.CB, xcol, y0, n0, mb);
            issued = i + 1;
        }
    } else if (warp == 4 && lane == 0) {
        // ---- MMA issuer: M = 128, N = cout, both operands MN-major
        const uint32_t idesc = tc_idesc(128, a.cout) | (1u << 15) | (1u << 16);
        const uint64_t amode = sw_mode_bytes(arow), bmode = sw_mode_bytes(brow);
        int i = 0;
        for (; i < KB; ++i) {
            const int s = i % WG_S;
            if (!ws_wait(&full[s], (i / WG_S) & 1, &s_fail)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const unsigned sa = smem_addr(sm + (size_t)s * STAGE), sb = sa + WG_ABYTES;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint64_t da = tc_desc_mn(sa + ks * 16 * arow, aatom, 8 * arow, amode);
                const uint64_t db = tc_desc_mn(sb + ks * 16 * brow, batom, 8 * brow, bmode);
                const unsigned acc = (i > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t"
                    "}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(&empty[s])));
        }
        s_consumed = i;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(&done)));
    }
    if (warp < 4) {
        // epilogue: warp w holds rows 32w .. 32w + 31; rows of pairs this CTA
        // did not load are never written
        const bool ok = __all_sync(0xffffffffu, ws_wait(&done, 0, &s_fail) && !s_fail);
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (ok) {
            const int m = warp * 32 + lane;
            const int j = m / a.CA;
            const int pr = p0 + j;
            const int tap = pr / cblocks;
            const int ci = (pr - tap * cblocks) * a.CA + (m - j * a.CA);
            const bool valid = j < np;
            float *dst = a.dw + (long long)tap * a.cin + ci;
            const long long co_stride = 9LL * a.cin;
            for (int c = 0; c < a.cout; c += 16) {
                unsigned r[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (valid) {
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) atomicAdd(dst + (c + jj) * co_stride, __uint_as_float(r[jj]));
                }
            }
        }
    }
    __syncthreads();
    if (tid == 0 && s_fail) {
        // copies still in flight land, and issued MMAs finish, before the
        // CTA frees its TMEM and leaves
        volatile int never = 0;
        for (int i = s_consumed; i < issued; ++i) ws_wait(&full[i % WG_S], (i / WG_S) & 1, &never);
        ws_wait(&done, 0, &never);
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.ncol));
}

// ------------------------------------------------------------- small kernels
// bias gradient: db[c] += sum_p dz[p][c].  A block of 256 threads takes all
// C channels of a chunk of pixels.  Thread t reads the 8 channels of group
// t mod G (G = ceil(C / 8)) 16 bytes at a time, in R = 256 / G pixel rows
// (row t / G takes pixels p0 + row, p0 + row + R, ...); the rows meet in
// shared memory and each channel's sum goes out in one atomic.  Channels
// C .. 8 G - 1 are read (the buffer has them: its stride is a multiple of 8)
// but never written.
constexpr int kBiasLoads = 16;  // loads per thread and block
__global__ void __launch_bounds__(256) k_bias_grad(const bf16 *dz, int dzc, int C, long long P, int chunk, float *db) {
    __shared__ float sh[256 * 8];
    const int G = (C + 7) >> 3, R = 256 / G;
    const int t = threadIdx.x, g = t % G, r = t / G;
    const long long p0 = (long long)blockIdx.x * chunk;
    const long long p1 = p0 + chunk < P ? p0 + chunk : P;
    if (r < R) {
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (long long p = p0 + r; p < p1; p += R) {
            const uint4 v = *reinterpret_cast<const uint4 *>(dz + p * dzc + g * 8);
            const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = __bfloat1622float2(h[k]);
                s[2 * k] += f.x;
                s[2 * k + 1] += f.y;
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) sh[(r * G + g) * 8 + k] = s[k];
    }
    __syncthreads();
    for (int c = t; c < C; c += 256) {
        float tot = 0.f;
        for (int rr = 0; rr < R; ++rr) tot += sh[rr * G * 8 + c];
        atomicAdd(db + c, tot);
    }
}

// 2x2 average pooling: y[n][i][j] = mean of x[n][2i..2i+1][2j..2j+1]
__global__ void k_pool(const bf16 *x, int xc, int xo, bf16 *y, int yc, int yo, int N, int H, int W, int C) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int Ho = H / 2, Wo = W / 2;
    const long long total = (long long)N * Ho * Wo * C;
    if (idx >= total) return;
    const int c = (int)(idx % C);
    const long long q = idx / C;
    const int j = (int)(q % Wo), i = (int)((q / Wo) % Ho), n = (int)(q / ((long long)Wo * Ho));
    auto at = [&](int yy, int xx) {
        return __bfloat162float(x[((long long)(n * H + yy) * W + xx) * xc + xo + c]);
    };
    const float s = 0.25f * (at(2 * i, 2 * j) + at(2 * i, 2 * j + 1) + at(2 * i + 1, 2 * j) + at(2 * i + 1, 2 * j + 1));
    y[((long long)(n * Ho + i) * Wo + j) * yc + yo + c] = __float2bfloat16_rn(s);
}

// pooling backward at the fine resolution, gated by the fine activation:
// dst[n][y][x][c] (+)= 0.25 dy[n][y/2][x/2][c] * (gate > 0)
__global__ void k_pool_back(const bf16 *dy, int dyc, int dyo, const bf16 *gate, int gc, int go, bf16 *dst, int dc, int dof,
                            int N, int H, int W, int C, int accumulate) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)N * H * W * C;
    if (idx >= total) return;
    const int c = (int)(idx % C);
    const long long p = idx / C;
    const int x = (int)(p % W), yv = (int)((p / W) % H), n = (int)(p / ((long long)W * H));
    const long long pc = ((long long)(n * (H / 2) + yv / 2) * (W / 2) + x / 2);
    float v = 0.25f * __bfloat162float(dy[pc * dyc + dyo + c]);
    if (!(__bfloat162float(gate[p * gc + go + c]) > 0.f)) v = 0.f;
    bf16 *d = dst + p * dc + dof + c;
    if (accumulate) v += __bfloat162float(*d);
    *d = __float2bfloat16_rn(v);
}

// nearest 2x upsampling: y[n][i][j] = x[n][i/2][j/2]
// grid (ceil(W * C / 8 / 256), N * H): blockIdx.y is an output row, a thread
// moves 8 channels (16 bytes; C, xc, yc, xo, yo multiples of 8)
__global__ void k_up(const bf16 *x, int xc, int xo, bf16 *y, int yc, int yo, int N, int H, int W, int C) {
    // H, W: fine (output) sizes
    const int C8 = C >> 3;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= W * C8) return;
    const int row = blockIdx.y, n = row / H, i = row - n * H;
    const int j = t / C8, c = (t - j * C8) * 8;
    const long long p = (long long)row * W + j;
    const long long q = ((long long)(n * (H / 2) + i / 2) * (W / 2) + j / 2);
    *reinterpret_cast<uint4 *>(y + p * yc + yo + c) = *reinterpret_cast<const uint4 *>(x + q * xc + xo + c);
}

// upsampling backward at the coarse resolution, gated by the coarse activation
__global__ void k_up_back(const bf16 *dy, int dyc, int dyo, const bf16 *gate, int gc, int go, bf16 *dst, int dc, int dof,
                          int N, int H, int W, int C) {
    // H, W: coarse sizes
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)N * H * W * C;
    if (idx >= total) return;
    const int c = (int)(idx % C);
    const long long p = idx / C;
    const int j = (int)(p % W), i = (int)((p / W) % H), n = (int)(p / ((long long)W * H));
    const int W2 = 2 * W, H2 = 2 * H;
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
            s += __bfloat162float(dy[((long long)(n * H2 + 2 * i + a) * W2 + 2 * j + b) * dyc + dyo + c]);
    if (!(__bfloat162float(gate[p * gc + go + c]) > 0.f)) s = 0.f;
    dst[p * dc + dof + c] = __float2bfloat16_rn(s);
}

// inputs [p][cin] FP32 -> [p][16] BF16 (channels cin..15 zero), cin <= 16
__global__ void k_pack_input(const float *x, int cin, bf16 *y, long long P) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
#pragma unroll
    for (int c = 0; c < 16; ++c) y[p * 16 + c] = __float2bfloat16_rn(c < cin ? x[p * cin + c] : 0.f);
}

// weighted MSE: loss += sum m (y - t)^2 * scale; dz[p][c] = 2 m (y - t) scale
// (c < 3; channels 3..dzc-1 zero), scale = 1 / (3 sum m)
__global__ void k_loss(const float *y, const float *t, const float *m, long long P, float scale, bf16 *dz, int dzc,
                       double *loss) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (p < P) {
        const float w = m[p];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float d = y[p * 3 + c] - t[p * 3 + c];
            l += (double)(w * d * d) * scale;
            dz[p * dzc + c] = __float2bfloat16_rn(2.f * w * d * scale);
        }
        for (int c = 3; c < dzc; ++c) dz[p * dzc + c] = __float2bfloat16_rn(0.f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}

// Adam on the FP32 master parameters (Kingma & Ba, bias-corrected)
__global__ void k_adam(float *p, float *m, float *v, const float *g, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 copies of one layer: w[co][tap][ci] and wt[ci][8 - tap][co]
__global__ void k_pack_weights(const float *wf, bf16 *w, bf16 *wt, int coutp, int cinp) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)coutp * 9 * cinp;
    if (i >= n) return;
    const int ci = (int)(i % cinp);
    const int tap = (int)((i / cinp) % 9);
    const int co = (int)(i / (9LL * cinp));
    const bf16 v = __float2bfloat16_rn(wf[i]);
    w[i] = v;
    wt[((long long)ci * 9 + (8 - tap)) * coutp + co] = v;
}

}  // namespace unet

// ====================================================================== host
using namespace unet;

namespace {

struct Layer {
    const char *name;
    int cin, cout, relu;
    int cinp, coutp;          // padded: input 16 for the 3-channel input, head 32 outputs
    size_t woff, boff;        // offsets in the FP32 master buffer (padded layout)
    size_t canon_w, canon_b;  // offsets in the canonical layout
    bf16 *w = nullptr, *wt = nullptr;
};

const struct { const char *name; int cin, cout, relu; } kArch[] = {
    {"enc1a", 3, 32, 1},   {"enc1b", 32, 32, 1},   {"enc2a", 32, 64, 1},   {"enc2b", 64, 64, 1},
    {"enc3a", 64, 128, 1}, {"enc3b", 128, 128, 1}, {"bota", 128, 256, 1},  {"botb", 256, 256, 1},
    {"up3", 256, 128, 1},  {"dec3a", 256, 128, 1}, {"dec3b", 128, 128, 1}, {"up2", 128, 64, 1},
    {"dec2a", 128, 64, 1}, {"dec2b", 64, 64, 1},   {"up1", 64, 32, 1},     {"dec1a", 64, 32, 1},
    {"dec1b", 32, 32, 1},  {"head", 32, 3, 0},
};
constexpr int kL = sizeof(kArch) / sizeof(kArch[0]);
enum { E1A, E1B, E2A, E2B, E3A, E3B, BA, BB, U3, D3A, D3B, U2, D2A, D2B, U1, D1A, D1B, HEAD };

}  // namespace

struct lbm_unet {
    int H = 0, W = 0, B = 0;
    int cin = 3;        // input channels of the first layer
    int wrapx = 0;      // periodic padding along x in every convolution
    int sms = 152;      // multiprocessors of the device
    int wgrad_kind = LBM_UNET_WGRAD_AUTO;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Layer L[kL];
    size_t nparam = 0, ncanon = 0;
    float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;  // padded FP32
    int adam_t = 0;
    // activations (bf16, NHWC) and gradients
    bf16 *x0, *e1a, *cat1, *p1, *e2a, *cat2, *p2, *e3a, *cat3, *p3, *ba, *bb, *u3in, *d3a, *d3, *u2in, *d2a, *d2, *u1in,
        *d1a, *d1;
    bf16 *g_head, *g_d1, *g_d1a, *g_cat1, *g_u1in, *g_d2, *g_d2a, *g_cat2, *g_u2in, *g_d3, *g_d3a, *g_cat3, *g_u3in, *g_bb,
        *g_ba, *g_p3, *g_e3a, *g_p2, *g_e2a, *g_p1, *g_e1a;
    float *yf = nullptr;
    double *loss = nullptr;
    int *tc_err = nullptr;     // set by a tcgen05 convolution whose bounded wait expired
    std::vector<void *> allocs;
    std::string err;
};

namespace {

lbm_status ufail(lbm_unet *u, lbm_status st, const std::string &m) {
    if (u) u->err = m;
    lbm::set_thread_error(m.c_str());
    return st;
}

#define U_CUDA(u, call)                                                                           \
    do {                                                                                          \
        cudaError_t e__ = (call);                                                                 \
        if (e__ != cudaSuccess)                                                                   \
            return ufail((u), e__ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,      \
                         std::string(#call) + ": " + cudaGetErrorString(e__));                    \
    } while (0)

template <typename T>
lbm_status ualloc(lbm_unet *u, T **p, size_t count) {
    void *q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T) + 16) != cudaSuccess) {
        cudaGetLastError();
        return ufail(u, LBM_ERR_OOM, "device allocation failed");
    }
    u->allocs.push_back(q);
    *p = (T *)q;
    return LBM_OK;
}

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// dynamic shared memory of k_conv_ws<BK, NT>: WS_S stages plus alignment
// slack, and at least enough that no more CTAs fit on an SM than its 512
// TMEM columns serve (tcgen05.alloc of a CTA beyond them would wait)
template <int BK, int NT> size_t tc_smem_bytes() {
    const size_t need = WS_S * (size_t)(128 * BK + NT * BK) * 2 + 1024;
    const int ncol = NT < 32 ? 32 : NT;
    const size_t floor_ = 233472 / (512 / ncol + 1) - 1024 + 1;
    return need > floor_ ? need : floor_;
}

template <int BK, int NT> lbm_status launch_tc(lbm_unet *u, const ConvArgs &a, long long M) {
    static bool attr = false;
    const size_t smem = tc_smem_bytes<BK, NT>();
    if (!attr) {
        U_CUDA(u, cudaFuncSetAttribute(k_conv_ws<BK, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    dim3 grid(nblk(M, 128), nblk(a.cout, NT));
    k_conv_ws<BK, NT><<<grid, 160, smem, u->stream>>>(a, u->tc_err);
    U_CUDA(u, cudaGetLastError());
    return LBM_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once (null: unavailable)
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    }
    return fn;
}

template <int BK, int NT, bool DEEP>
cudaError_t launch_tma_kernel(lbm_unet *u, const ConvArgs &a, const CUtensorMap &ta, const CUtensorMap &tb, int HB,
                              int NB, dim3 grid) {
    constexpr size_t STAGE = tma_stage_bytes<BK, NT>();
    const int ncol = NT < 32 ? 32 : NT;
    const size_t need = tma_stages<BK, NT, DEEP>() * STAGE + 1024, floor_ = 233472 / (512 / ncol + 1) - 1024 + 1;
    const size_t smem = need > floor_ ? need : floor_;
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(k_conv_tma<BK, NT, DEEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_conv_tma<BK, NT, DEEP><<<grid, 160, smem, u->stream>>>(a, ta, tb, HB, NB, u->tc_err);
    return cudaSuccess;
}

// The TMA convolution when the shape suits its column tiles: H <= 128
// dividing 128 with N a multiple of 128 / H, or H a multiple of 128; every
// global address and stride a multiple of 16 bytes.  Returns false (nothing
// launched) otherwise, and when a tensor map cannot be made.
template <int BK, int NT> bool launch_tma(lbm_unet *u, const ConvArgs &a, lbm_status *st) {
    const int H = a.H, W = a.W, N = a.N;
    const int HB = H <= 128 ? H : 128;
    const int NB = H <= 128 ? 128 / H : 1;
    if (H <= 128 ? (128 % H != 0 || N % NB != 0) : (H % 128 != 0)) return false;
    if (a.cin % BK != 0 || a.xc % 8 != 0 || a.xo % 8 != 0 || ((uintptr_t)a.x) % 16 != 0 || ((uintptr_t)a.w) % 16 != 0 ||
        (9 * a.cin) % 8 != 0)
        return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return false;
    const CUtensorMapSwizzle swz =
        BK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : (BK == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
    alignas(64) CUtensorMap ta, tb;
    const cuuint64_t gdA[4] = {(cuuint64_t)a.cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t rowb = (cuuint64_t)a.xc * 2;
    const cuuint64_t gsA[3] = {rowb, rowb * W, rowb * W * H};
    const cuuint32_t boxA[4] = {(cuuint32_t)BK, 1u, (cuuint32_t)HB, (cuuint32_t)NB};
    const cuuint32_t es[4] = {1u, 1u, 1u, 1u};
    if (enc(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)(a.x + a.xo), gdA, gsA, boxA, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const cuuint64_t gdB[2] = {(cuuint64_t)9 * a.cin, (cuuint64_t)a.wrows};
    const cuuint64_t gsB[1] = {(cuuint64_t)9 * a.cin * 2};
    const cuuint32_t boxB[2] = {(cuuint32_t)BK, (cuuint32_t)NT};
    if (enc(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)a.w, gdB, gsB, boxB, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    dim3 grid((unsigned)(W * (H / HB) * (N / NB)), (unsigned)nblk(a.cout, NT));
    const bool deep = (long long)grid.x * grid.y < 2LL * u->sms;
    cudaError_t e = deep ? launch_tma_kernel<BK, NT, true>(u, a, ta, tb, HB, NB, grid)
                         : launch_tma_kernel<BK, NT, false>(u, a, ta, tb, HB, NB, grid);
    if (e == cudaSuccess) e = cudaGetLastError();
    *st = e == cudaSuccess ? LBM_OK : ufail(u, LBM_ERR_CUDA, std::string("k_conv_tma: ") + cudaGetErrorString(e));
    return true;
}

template <int BK> lbm_status launch_conv_n(lbm_unet *u, const ConvArgs &a, long long M) {
    lbm_status st = LBM_OK;
    if (a.cout <= 16) return launch_tma<BK, 16>(u, a, &st) ? st : launch_tc<BK, 16>(u, a, M);
    if (a.cout <= 32) return launch_tma<BK, 32>(u, a, &st) ? st : launch_tc<BK, 32>(u, a, M);
    if (a.cout <= 64) return launch_tma<BK, 64>(u, a, &st) ? st : launch_tc<BK, 64>(u, a, M);
    return launch_tma<BK, 128>(u, a, &st) ? st : launch_tc<BK, 128>(u, a, M);
}

// convolutions with N = cout a multiple of 16 (every layer but the head):
// TMA-fed where the shape allows, else cp.async-fed
lbm_status conv_tc(lbm_unet *u, const ConvArgs &a, long long M) {
    if (a.cin % 64 == 0) return launch_conv_n<64>(u, a, M);
    if (a.cin % 32 == 0) return launch_conv_n<32>(u, a, M);
    return launch_conv_n<16>(u, a, M);
}

lbm_status conv(lbm_unet *u, int li, const bf16 *x, int xc, int xo, int n, int H, int W, bf16 *y, int yc, int yo,
                bool forward, const bf16 *gate = nullptr, int gc = 0, int go = 0, float *yf = nullptr, int yfc = 0) {
    const Layer &l = u->L[li];
    ConvArgs a{};
    a.x = x;
    a.xc = xc;
    a.xo = xo;
    a.N = n;
    a.H = H;
    a.W = W;
    a.y = y;
    a.yc = yc;
    a.yo = yo;
    a.yf = yf;
    a.yfc = yfc;
    a.gate = gate;
    a.gc = gc;
    a.go = go;
    a.wrapx = u->wrapx;
    if (forward) {
        a.w = l.w;
        a.bias = u->p + l.boff;
        a.cin = l.cinp;
        a.cout = l.cout;
        a.wrows = l.coutp;
        a.relu = l.relu;
    } else {
        // input gradient: conv of dz (coutp channels) with the flipped transpose
        a.w = l.wt;
        a.bias = nullptr;
        a.cin = l.coutp;
        a.cout = l.cinp;
        a.wrows = l.cinp;
        a.relu = 0;
    }
    const long long M = (long long)n * H * W;
    if (!yf && a.cout % 16 == 0 && a.cin % 16 == 0) return conv_tc(u, a, M);
    dim3 grid(nblk(M, CBM), nblk(a.cout, CBN));
    if (a.cin % 32 == 0) k_conv<32><<<grid, 256, 0, u->stream>>>(a);
    else k_conv<16><<<grid, 256, 0, u->stream>>>(a);
    U_CUDA(u, cudaGetLastError());
    return LBM_OK;
}

// db += the per-channel sums of dz (C <= 256 channels of a buffer whose
// channel stride dzc is a multiple of 8 and at least 8 ceil(C / 8), 16-byte
// aligned: every gradient buffer of the network is)
lbm_status bias_grad(lbm_unet *u, const bf16 *dz, int dzc, int C, long long P, float *db) {
    const int G = (C + 7) / 8;
    if (C < 1 || C > 256 || dzc % 8 != 0 || dzc < 8 * G || ((uintptr_t)dz) % 16 != 0)
        return ufail(u, LBM_ERR_STATE, "bias gradient: unsupported gradient buffer layout");
    const int chunk = (256 / G) * kBiasLoads;
    k_bias_grad<<<nblk(P, chunk), 256, 0, u->stream>>>(dz, dzc, C, P, chunk, db);
    U_CUDA(u, cudaGetLastError());
    return LBM_OK;
}

// The tcgen05 weight gradient when the shape suits its pixel blocks (64
// pixels of one column: H <= 64 dividing 64 with n a multiple of 64 / H, or H
// a multiple of 64) and every global address and stride is a multiple of 16
// bytes.  Returns false (nothing launched) otherwise, and when a tensor map
// cannot be made.  The pixel blocks are split so that about two CTAs per SM
// run, each taking at least 8 blocks (its 128 x N atomics stay small against
// its MMA work).
bool launch_wgrad_tc(lbm_unet *u, const Layer &l, const bf16 *dz, int dzc, const bf16 *x, int xc, int xo, int n,
                     int H, int W, lbm_status *st) {
    const int HB = H <= 64 ? H : 64;
    const int NB = H <= 64 ? 64 / H : 1;
    if (H <= 64 ? (64 % H != 0 || n % NB != 0) : (H % 64 != 0)) return false;
    const int cin = l.cinp, cout = l.coutp;
    // atom widths are swizzle widths: 16, 32 or 64 channels
    if ((cin < 64 ? (cin != 16 && cin != 32) : cin % 64 != 0) || cout > 256 || (cout < 64 ? cout != 32 : cout % 64 != 0))
        return false;
    if (xc % 8 != 0 || xo % 8 != 0 || dzc % 8 != 0 || xc < xo + cin || dzc < cout ||
        ((uintptr_t)(x + xo)) % 16 != 0 || ((uintptr_t)dz) % 16 != 0)
        return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return false;
    const int CA = cin >= 64 ? 64 : cin, CB = cout >= 64 ? 64 : cout;
    auto swz = [](int ch) {
        return ch == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : (ch == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
    };
    alignas(64) CUtensorMap tx, tz;
    const cuuint32_t es[4] = {1u, 1u, 1u, 1u};
    const cuuint64_t gdX[4] = {(cuuint64_t)cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)n};
    const cuuint64_t rx = (cuuint64_t)xc * 2;
    const cuuint64_t gsX[3] = {rx, rx * W, rx * W * H};
    const cuuint32_t boxX[4] = {(cuuint32_t)CA, 1u, (cuuint32_t)HB, (cuuint32_t)NB};
    if (enc(&tx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)(x + xo), gdX, gsX, boxX, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swz(CA), CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const cuuint64_t gdZ[4] = {(cuuint64_t)cout, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)n};
    const cuuint64_t rz = (cuuint64_t)dzc * 2;
    const cuuint64_t gsZ[3] = {rz, rz * W, rz * W * H};
    const cuuint32_t boxZ[4] = {(cuuint32_t)CB, 1u, (cuuint32_t)HB, (cuuint32_t)NB};
    if (enc(&tz, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)dz, gdZ, gsZ, boxZ, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            swz(CB), CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    WgTcArgs a{};
    a.dw = u->g + l.woff;
    a.cin = cin;
    a.cout = cout;
    a.H = H;
    a.W = W;
    a.HB = HB;
    a.NB = NB;
    a.wrapx = u->wrapx;
    a.CA = CA;
    a.CB = CB;
    a.pairs = 9 * cin / CA;
    a.kb_total = (long long)n * H * W / 64;
    a.ncol = cout <= 32 ? 32u : (cout <= 64 ? 64u : (cout <= 128 ? 128u : 256u));
    const int mtiles = (a.pairs + 128 / CA - 1) / (128 / CA);
    long long splits = (2LL * u->sms + mtiles - 1) / mtiles;
    const long long cap = a.kb_total / 8 > 0 ? a.kb_total / 8 : 1;
    if (splits > cap) splits = cap;
    a.kb_per = (int)((a.kb_total + splits - 1) / splits);
    splits = (a.kb_total + a.kb_per - 1) / a.kb_per;  // every CTA gets at least one block
    const size_t smem = (size_t)WG_S * wg_stage_bytes(256) + 1024;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            *st = ufail(u, LBM_ERR_CUDA, std::string("k_wgrad_tc attribute: ") + cudaGetErrorString(e));
            return true;
        }
        attr = true;
    }
    const size_t need = (size_t)WG_S * wg_stage_bytes(cout) + 1024;
    k_wgrad_tc<<<dim3((unsigned)splits, (unsigned)mtiles), 160, need, u->stream>>>(a, tx, tz, u->tc_err);
    cudaError_t e = cudaGetLastError();
    *st = e == cudaSuccess ? LBM_OK : ufail(u, LBM_ERR_CUDA, std::string("k_wgrad_tc: ") + cudaGetErrorString(e));
    return true;
}

lbm_status wgrad(lbm_unet *u, int li, const bf16 *dz, int dzc, const bf16 *x, int xc, int xo, int n, int H, int W) {
    const Layer &l = u->L[li];
    const long long P = (long long)n * H * W;
    lbm_status st = LBM_OK;
    if (u->wgrad_kind == LBM_UNET_WGRAD_AUTO && launch_wgrad_tc(u, l, dz, dzc, x, xc, xo, n, H, W, &st)) {
        if (st != LBM_OK) return st;
        return bias_grad(u, dz, dzc, l.cout, P, u->g + l.boff);
    }
    WgradArgs a{};
    a.dz = dz;
    a.dzc = dzc;
    a.dzo = 0;
    a.x = x;
    a.xc = xc;
    a.xo = xo;
    a.dw = u->g + l.woff;
    a.N = n;
    a.H = H;
    a.W = W;
    a.cin = l.cinp;
    a.cout = l.coutp;
    a.wrapx = u->wrapx;
    a.pix = 2048;
    dim3 grid(nblk(P, a.pix), nblk(l.coutp, WBM), 9 * ((l.cinp + WBN - 1) / WBN));
    k_wgrad<<<grid, 128, 0, u->stream>>>(a);
    U_CUDA(u, cudaGetLastError());
    return bias_grad(u, dz, dzc, l.cout, P, u->g + l.boff);
}

lbm_status repack(lbm_unet *u) {
    for (int i = 0; i < kL; ++i) {
        const Layer &l = u->L[i];
        const long long n = (long long)l.coutp * 9 * l.cinp;
        k_pack_weights<<<nblk(n, 256), 256, 0, u->stream>>>(u->p + l.woff, l.w, l.wt, l.coutp, l.cinp);
        U_CUDA(u, cudaGetLastError());
    }
    return LBM_OK;
}

lbm_status forward(lbm_unet *u, const float *xin, int n) {
    const int H = u->H, W = u->W;
    const int H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4, H8 = H / 8, W8 = W / 8;
    lbm_status st;
    const long long P = (long long)n * H * W;
    k_pack_input<<<nblk(P, 256), 256, 0, u->stream>>>(xin, u->cin, u->x0, P);
    U_CUDA(u, cudaGetLastError());
#define FW(li, x, xc, xo, h, w, y, yc, yo) \
    if ((st = conv(u, li, x, xc, xo, n, h, w, y, yc, yo, true)) != LBM_OK) return st;
    FW(E1A, u->x0, 16, 0, H, W, u->e1a, 32, 0);
    FW(E1B, u->e1a, 32, 0, H, W, u->cat1, 64, 32);
    k_pool<<<nblk((long long)n * H2 * W2 * 32, 256), 256, 0, u->stream>>>(u->cat1, 64, 32, u->p1, 32, 0, n, H, W, 32);
    FW(E2A, u->p1, 32, 0, H2, W2, u->e2a, 64, 0);
    FW(E2B, u->e2a, 64, 0, H2, W2, u->cat2, 128, 64);
    k_pool<<<nblk((long long)n * H4 * W4 * 64, 256), 256, 0, u->stream>>>(u->cat2, 128, 64, u->p2, 64, 0, n, H2, W2, 64);
    FW(E3A, u->p2, 64, 0, H4, W4, u->e3a, 128, 0);
    FW(E3B, u->e3a, 128, 0, H4, W4, u->cat3, 256, 128);
    k_pool<<<nblk((long long)n * H8 * W8 * 128, 256), 256, 0, u->stream>>>(u->cat3, 256, 128, u->p3, 128, 0, n, H4, W4, 128);
    FW(BA, u->p3, 128, 0, H8, W8, u->ba, 256, 0);
    FW(BB, u->ba, 256, 0, H8, W8, u->bb, 256, 0);
    k_up<<<dim3(nblk((long long)W4 * 256 / 8, 256), n * H4), 256, 0, u->stream>>>(u->bb, 256, 0, u->u3in, 256, 0, n, H4, W4, 256);
    FW(U3, u->u3in, 256, 0, H4, W4, u->cat3, 256, 0);
    FW(D3A, u->cat3, 256, 0, H4, W4, u->d3a, 128, 0);
    FW(D3B, u->d3a, 128, 0, H4, W4, u->d3, 128, 0);
    k_up<<<dim3(nblk((long long)W2 * 128 / 8, 256), n * H2), 256, 0, u->stream>>>(u->d3, 128, 0, u->u2in, 128, 0, n, H2, W2, 128);
    FW(U2, u->u2in, 128, 0, H2, W2, u->cat2, 128, 0);
    FW(D2A, u->cat2, 128, 0, H2, W2, u->d2a, 64, 0);
    FW(D2B, u->d2a, 64, 0, H2, W2, u->d2, 64, 0);
    k_up<<<dim3(nblk((long long)W * 64 / 8, 256), n * H), 256, 0, u->stream>>>(u->d2, 64, 0, u->u1in, 64, 0, n, H, W, 64);
    FW(U1, u->u1in, 64, 0, H, W, u->cat1, 64, 0);
    FW(D1A, u->cat1, 64, 0, H, W, u->d1a, 32, 0);
    FW(D1B, u->d1a, 32, 0, H, W, u->d1, 32, 0);
#undef FW
    if ((st = conv(u, HEAD, u->d1, 32, 0, n, H, W, nullptr, 0, 0, true, nullptr, 0, 0, u->yf, 3)) != LBM_OK) return st;
    U_CUDA(u, cudaGetLastError());
    return LBM_OK;
}

// gradients of the weighted MSE into u->g (zeroed first); loss into u->loss
lbm_status backward(lbm_unet *u, const float *t, const float *m, int n, float scale) {
    const int H = u->H, W = u->W;
    const int H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4, H8 = H / 8, W8 = W / 8;
    const long long P = (long long)n * H * W;
    lbm_status st;
    U_CUDA(u, cudaMemsetAsync(u->g, 0, u->nparam * sizeof(float), u->stream));
    U_CUDA(u, cudaMemsetAsync(u->loss, 0, sizeof(double), u->stream));
    k_loss<<<nblk(P, 256), 256, 0, u->stream>>>(u->yf, t, m, P, scale, u->g_head, 32, u->loss);
    U_CUDA(u, cudaGetLastError());
#define WG(li, dz, dzc, x, xc, xo, h, w) \
    if ((st = wgrad(u, li, dz, dzc, x, xc, xo, n, h, w)) != LBM_OK) return st;
#define DG(li, dz, dzc, h, w, y, yc, yo, gate, gc, go) \
    if ((st = conv(u, li, dz, dzc, 0, n, h, w, y, yc, yo, false, gate, gc, go)) != LBM_OK) return st;
    // head and decoder level 1
    WG(HEAD, u->g_head, 32, u->d1, 32, 0, H, W);
    DG(HEAD, u->g_head, 32, H, W, u->g_d1, 32, 0, u->d1, 32, 0);
    WG(D1B, u->g_d1, 32, u->d1a, 32, 0, H, W);
    DG(D1B, u->g_d1, 32, H, W, u->g_d1a, 32, 0, u->d1a, 32, 0);
    WG(D1A, u->g_d1a, 32, u->cat1, 64, 0, H, W);
    DG(D1A, u->g_d1a, 32, H, W, u->g_cat1, 64, 0, u->cat1, 64, 0);  // [dz up1 | dz enc1b (decoder part)]
    WG(U1, u->g_cat1, 64, u->u1in, 64, 0, H, W);
    DG(U1, u->g_cat1, 64, H, W, u->g_u1in, 64, 0, nullptr, 0, 0);
    k_up_back<<<nblk((long long)n * H2 * W2 * 64, 256), 256, 0, u->stream>>>(u->g_u1in, 64, 0, u->d2, 64, 0, u->g_d2, 64, 0,
                                                                            n, H2, W2, 64);
    // decoder level 2
    WG(D2B, u->g_d2, 64, u->d2a, 64, 0, H2, W2);
    DG(D2B, u->g_d2, 64, H2, W2, u->g_d2a, 64, 0, u->d2a, 64, 0);
    WG(D2A, u->g_d2a, 64, u->cat2, 128, 0, H2, W2);
    DG(D2A, u->g_d2a, 64, H2, W2, u->g_cat2, 128, 0, u->cat2, 128, 0);
    WG(U2, u->g_cat2, 128, u->u2in, 128, 0, H2, W2);
    DG(U2, u->g_cat2, 128, H2, W2, u->g_u2in, 128, 0, nullptr, 0, 0);
    k_up_back<<<nblk((long long)n * H4 * W4 * 128, 256), 256, 0, u->stream>>>(u->g_u2in, 128, 0, u->d3, 128, 0, u->g_d3,
                                                                             128, 0, n, H4, W4, 128);
    // decoder level 3
    WG(D3B, u->g_d3, 128, u->d3a, 128, 0, H4, W4);
    DG(D3B, u->g_d3, 128, H4, W4, u->g_d3a, 128, 0, u->d3a, 128, 0);
    WG(D3A, u->g_d3a, 128, u->cat3, 256, 0, H4, W4);
    DG(D3A, u->g_d3a, 128, H4, W4, u->g_cat3, 256, 0, u->cat3, 256, 0);
    WG(U3, u->g_cat3, 256, u->u3in, 256, 0, H4, W4);
    DG(U3, u->g_cat3, 256, H4, W4, u->g_u3in, 256, 0, nullptr, 0, 0);
    k_up_back<<<nblk((long long)n * H8 * W8 * 256, 256), 256, 0, u->stream>>>(u->g_u3in, 256, 0, u->bb, 256, 0, u->g_bb,
                                                                             256, 0, n, H8, W8, 256);
    // bottleneck
    WG(BB, u->g_bb, 256, u->ba, 256, 0, H8, W8);
    DG(BB, u->g_bb, 256, H8, W8, u->g_ba, 256, 0, u->ba, 256, 0);
    WG(BA, u->g_ba, 256, u->p3, 128, 0, H8, W8);
    DG(BA, u->g_ba, 256, H8, W8, u->g_p3, 128, 0, nullptr, 0, 0);
    // encoder level 3: dz of enc3b = decoder part + pooling path (gated by enc3b > 0)
    k_pool_back<<<nblk((long long)n * H4 * W4 * 128, 256), 256, 0, u->stream>>>(u->g_p3, 128, 0, u->cat3, 256, 128,
                                                                               u->g_cat3, 256, 128, n, H4, W4, 128, 1);
    WG(E3B, u->g_cat3 + 128, 256, u->e3a, 128, 0, H4, W4);
    DG(E3B, u->g_cat3 + 128, 256, H4, W4, u->g_e3a, 128, 0, u->e3a, 128, 0);
    WG(E3A, u->g_e3a, 128, u->p2, 64, 0, H4, W4);
    DG(E3A, u->g_e3a, 128, H4, W4, u->g_p2, 64, 0, nullptr, 0, 0);
    k_pool_back<<<nblk((long long)n * H2 * W2 * 64, 256), 256, 0, u->stream>>>(u->g_p2, 64, 0, u->cat2, 128, 64, u->g_cat2,
                                                                              128, 64, n, H2, W2, 64, 1);
    WG(E2B, u->g_cat2 + 64, 128, u->e2a, 64, 0, H2, W2);
    DG(E2B, u->g_cat2 + 64, 128, H2, W2, u->g_e2a, 64, 0, u->e2a, 64, 0);
    WG(E2A, u->g_e2a, 64, u->p1, 32, 0, H2, W2);
    DG(E2A, u->g_e2a, 64, H2, W2, u->g_p1, 32, 0, nullptr, 0, 0);
    k_pool_back<<<nblk((long long)n * H * W * 32, 256), 256, 0, u->stream>>>(u->g_p1, 32, 0, u->cat1, 64, 32, u->g_cat1, 64,
                                                                            32, n, H, W, 32, 1);
    WG(E1B, u->g_cat1 + 32, 64, u->e1a, 32, 0, H, W);
    DG(E1B, u->g_cat1 + 32, 64, H, W, u->g_e1a, 32, 0, u->e1a, 32, 0);
    WG(E1A, u->g_e1a, 32, u->x0, 16, 0, H, W);
#undef WG
#undef DG
    U_CUDA(u, cudaGetLastError());
    return LBM_OK;
}

}  // namespace

extern "C" {

void lbm_unet_destroy(lbm_unet *u) {
    if (!u) return;
    if (u->stream) cudaStreamSynchronize(u->stream);
    for (void *p : u->allocs) cudaFree(p);
    if (u->own_stream && u->stream) cudaStreamDestroy(u->stream);
    delete u;
}

lbm_status lbm_unet_create(int H, int W, int cin, int periodic_x, int max_batch, void *stream, lbm_unet **out) {
    if (!out) return ufail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (H < 8 || W < 8 || H % 8 || W % 8 || max_batch < 1)
        return ufail(nullptr, LBM_ERR_ARG, "H and W must be multiples of 8 (>= 8), max_batch >= 1");
    if (cin < 1 || cin > 16) return ufail(nullptr, LBM_ERR_ARG, "cin must be in [1, 16]");
    if ((long long)max_batch * H > 65535) return ufail(nullptr, LBM_ERR_ARG, "max_batch * H must be <= 65535");
    if (periodic_x != 0 && periodic_x != 1) return ufail(nullptr, LBM_ERR_ARG, "periodic_x must be 0 or 1");
    lbm_unet *u = new lbm_unet();
    u->H = H;
    u->W = W;
    u->B = max_batch;
    u->cin = cin;
    u->wrapx = periodic_x;
    {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
            u->sms = n;
        cudaGetLastError();
    }
    if (stream) {
        u->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&u->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete u;
            return ufail(nullptr, LBM_ERR_CUDA, "cudaStreamCreate failed");
        }
        u->own_stream = true;
    }
    size_t off = 0, coff = 0;
    for (int i = 0; i < kL; ++i) {
        Layer &l = u->L[i];
        l.name = kArch[i].name;
        l.cin = i == E1A ? cin : kArch[i].cin;
        l.cout = kArch[i].cout;
        l.relu = kArch[i].relu;
        l.cinp = l.cin < 16 ? 16 : l.cin;
        l.coutp = l.cout < 32 ? 32 : l.cout;
        l.woff = off;
        off += (size_t)l.coutp * 9 * l.cinp;
        l.boff = off;
        off += (size_t)l.coutp;
        l.canon_w = coff;
        coff += (size_t)l.cout * 9 * l.cin;
        l.canon_b = coff;
        coff += (size_t)l.cout;
    }
    u->nparam = off;
    u->ncanon = coff;
    const size_t B = max_batch;
    const size_t P1 = B * H * W, P2 = P1 / 4, P3 = P1 / 16, P4 = P1 / 64;
    lbm_status st = LBM_OK;
    auto A = [&](bf16 **p, size_t n) {
        if (st == LBM_OK) st = ualloc(u, p, n);
    };
    if ((st = ualloc(u, &u->p, off)) || (st = ualloc(u, &u->m, off)) || (st = ualloc(u, &u->v, off)) ||
        (st = ualloc(u, &u->g, off)) || (st = ualloc(u, &u->yf, P1 * 3)) || (st = ualloc(u, &u->loss, 1)) ||
        (st = ualloc(u, &u->tc_err, 1))) {
        lbm_unet_destroy(u);
        return ufail(nullptr, st, "device allocation failed");
    }
    for (int i = 0; i < kL; ++i) {
        A(&u->L[i].w, (size_t)u->L[i].coutp * 9 * u->L[i].cinp);
        A(&u->L[i].wt, (size_t)u->L[i].coutp * 9 * u->L[i].cinp);
    }
    A(&u->x0, P1 * 16); A(&u->e1a, P1 * 32); A(&u->cat1, P1 * 64); A(&u->p1, P2 * 32); A(&u->e2a, P2 * 64);
    A(&u->cat2, P2 * 128); A(&u->p2, P3 * 64); A(&u->e3a, P3 * 128); A(&u->cat3, P3 * 256); A(&u->p3, P4 * 128);
    A(&u->ba, P4 * 256); A(&u->bb, P4 * 256); A(&u->u3in, P3 * 256); A(&u->d3a, P3 * 128); A(&u->d3, P3 * 128);
    A(&u->u2in, P2 * 128); A(&u->d2a, P2 * 64); A(&u->d2, P2 * 64); A(&u->u1in, P1 * 64); A(&u->d1a, P1 * 32);
    A(&u->d1, P1 * 32);
    A(&u->g_head, P1 * 32); A(&u->g_d1, P1 * 32); A(&u->g_d1a, P1 * 32); A(&u->g_cat1, P1 * 64);
    A(&u->g_u1in, P1 * 64); A(&u->g_d2, P2 * 64); A(&u->g_d2a, P2 * 64); A(&u->g_cat2, P2 * 128);
    A(&u->g_u2in, P2 * 128); A(&u->g_d3, P3 * 128); A(&u->g_d3a, P3 * 128); A(&u->g_cat3, P3 * 256);
    A(&u->g_u3in, P3 * 256); A(&u->g_bb, P4 * 256); A(&u->g_ba, P4 * 256); A(&u->g_p3, P4 * 128);
    A(&u->g_e3a, P3 * 128); A(&u->g_p2, P3 * 64); A(&u->g_e2a, P2 * 64); A(&u->g_p1, P2 * 32); A(&u->g_e1a, P1 * 32);
    if (st != LBM_OK) {
        lbm_unet_destroy(u);
        return ufail(nullptr, st, "device allocation failed");
    }
    cudaError_t e = cudaMemsetAsync(u->p, 0, off * 4, u->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(u->m, 0, off * 4, u->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(u->v, 0, off * 4, u->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(u->tc_err, 0, sizeof(int), u->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(u->stream);
    if (e != cudaSuccess) {
        lbm_unet_destroy(u);
        return ufail(nullptr, LBM_ERR_CUDA, "initialisation failed");
    }
    *out = u;
    return LBM_OK;
}

int64_t lbm_unet_num_params(const lbm_unet *u) { return u ? (int64_t)u->ncanon : 0; }

// canonical layout (per layer W[co][ky][kx][ci], b[co]) <-> padded master buffer
lbm_status lbm_unet_set_params(lbm_unet *u, const float *host) {
    if (!u || !host) return ufail(u, LBM_ERR_ARG, "NULL argument");
    std::vector<float> pad(u->nparam, 0.f);
    for (int i = 0; i < kL; ++i) {
        const Layer &l = u->L[i];
        for (int co = 0; co < l.cout; ++co) {
            for (int t = 0; t < 9; ++t)
                for (int ci = 0; ci < l.cin; ++ci)
                    pad[l.woff + ((size_t)co * 9 + t) * l.cinp + ci] = host[l.canon_w + ((size_t)co * 9 + t) * l.cin + ci];
            pad[l.boff + co] = host[l.canon_b + co];
        }
    }
    U_CUDA(u, cudaMemcpyAsync(u->p, pad.data(), pad.size() * 4, cudaMemcpyHostToDevice, u->stream));
    U_CUDA(u, cudaMemsetAsync(u->m, 0, u->nparam * 4, u->stream));
    U_CUDA(u, cudaMemsetAsync(u->v, 0, u->nparam * 4, u->stream));
    u->adam_t = 0;
    lbm_status st = repack(u);
    if (st != LBM_OK) return st;
    U_CUDA(u, cudaStreamSynchronize(u->stream));
    return LBM_OK;
}

// a tcgen05 convolution whose bounded wait expired (reported at the next
// synchronising call)
static lbm_status check_tc(lbm_unet *u) {
    int flag = 0;
    U_CUDA(u, cudaMemcpyAsync(&flag, u->tc_err, sizeof(int), cudaMemcpyDeviceToHost, u->stream));
    U_CUDA(u, cudaStreamSynchronize(u->stream));
    if (flag) return ufail(u, LBM_ERR_TIMEOUT, "tensor-core convolution: a bounded wait expired");
    return LBM_OK;
}

static lbm_status copy_out(lbm_unet *u, const float *dev, float *host) {
    std::vector<float> pad(u->nparam);
    U_CUDA(u, cudaMemcpyAsync(pad.data(), dev, pad.size() * 4, cudaMemcpyDeviceToHost, u->stream));
    U_CUDA(u, cudaStreamSynchronize(u->stream));
    for (int i = 0; i < kL; ++i) {
        const Layer &l = u->L[i];
        for (int co = 0; co < l.cout; ++co) {
            for (int t = 0; t < 9; ++t)
                for (int ci = 0; ci < l.cin; ++ci)
                    host[l.canon_w + ((size_t)co * 9 + t) * l.cin + ci] = pad[l.woff + ((size_t)co * 9 + t) * l.cinp + ci];
            host[l.canon_b + co] = pad[l.boff + co];
        }
    }
    return LBM_OK;
}

lbm_status lbm_unet_get_params(lbm_unet *u, float *host) {
    if (!u || !host) return ufail(u, LBM_ERR_ARG, "NULL argument");
    lbm_status st = check_tc(u);
    if (st != LBM_OK) return st;
    return copy_out(u, u->p, host);
}

lbm_status lbm_unet_forward(lbm_unet *u, const float *x_dev, float *y_dev, int n) {
    if (!u || !x_dev || !y_dev) return ufail(u, LBM_ERR_ARG, "NULL argument");
    if (n < 1 || n > u->B) return ufail(u, LBM_ERR_ARG, "batch size out of range");
    lbm_status st = forward(u, x_dev, n);
    if (st != LBM_OK) return st;
    U_CUDA(u, cudaMemcpyAsync(y_dev, u->yf, (size_t)n * u->H * u->W * 3 * 4, cudaMemcpyDeviceToDevice, u->stream));
    return LBM_OK;
}

lbm_status lbm_unet_grad(lbm_unet *u, const float *x_dev, const float *t_dev, const float *m_dev, int n, float scale,
                         double *loss_host, float *grad_host) {
    if (!u || !x_dev || !t_dev || !m_dev) return ufail(u, LBM_ERR_ARG, "NULL argument");
    if (n < 1 || n > u->B) return ufail(u, LBM_ERR_ARG, "batch size out of range");
    lbm_status st = forward(u, x_dev, n);
    if (st == LBM_OK) st = backward(u, t_dev, m_dev, n, scale);
    if (st != LBM_OK) return st;
    if ((st = check_tc(u)) != LBM_OK) return st;
    if (loss_host) {
        U_CUDA(u, cudaMemcpyAsync(loss_host, u->loss, sizeof(double), cudaMemcpyDeviceToHost, u->stream));
        U_CUDA(u, cudaStreamSynchronize(u->stream));
    }
    if (grad_host) return copy_out(u, u->g, grad_host);
    return LBM_OK;
}

lbm_status lbm_unet_adam(lbm_unet *u, float lr, float beta1, float beta2, float eps) {
    if (!u) return ufail(nullptr, LBM_ERR_ARG, "NULL argument");
    u->adam_t += 1;
    const float c1 = 1.f - powf(beta1, (float)u->adam_t), c2 = 1.f - powf(beta2, (float)u->adam_t);
    k_adam<<<nblk((long long)u->nparam, 256), 256, 0, u->stream>>>(u->p, u->m, u->v, u->g, (long long)u->nparam, lr,
                                                                   beta1, beta2, eps, c1, c2);
    U_CUDA(u, cudaGetLastError());
    return repack(u);
}

lbm_status lbm_unet_train_step(lbm_unet *u, const float *x_dev, const float *t_dev, const float *m_dev, int n,
                               float scale, float lr, double *loss_dev) {
    if (!u || !x_dev || !t_dev || !m_dev) return ufail(u, LBM_ERR_ARG, "NULL argument");
    if (n < 1 || n > u->B) return ufail(u, LBM_ERR_ARG, "batch size out of range");
    lbm_status st = forward(u, x_dev, n);
    if (st == LBM_OK) st = backward(u, t_dev, m_dev, n, scale);
    if (st == LBM_OK) st = lbm_unet_adam(u, lr, 0.9f, 0.999f, 1e-8f);
    if (st != LBM_OK) return st;
    if (loss_dev) U_CUDA(u, cudaMemcpyAsync(loss_dev, u->loss, sizeof(double), cudaMemcpyDeviceToDevice, u->stream));
    return LBM_OK;
}

lbm_status lbm_unet_set_wgrad(lbm_unet *u, int kind) {
    if (!u) return ufail(nullptr, LBM_ERR_ARG, "network is NULL");
    if (kind != LBM_UNET_WGRAD_AUTO && kind != LBM_UNET_WGRAD_MMA_SYNC)
        return ufail(u, LBM_ERR_ARG, "kind must be LBM_UNET_WGRAD_AUTO or LBM_UNET_WGRAD_MMA_SYNC");
    U_CUDA(u, cudaStreamSynchronize(u->stream));
    u->wgrad_kind = kind;
    return LBM_OK;
}

const char *lbm_unet_last_error(const lbm_unet *u) { return u ? u->err.c_str() : ""; }

}  // extern "C"
