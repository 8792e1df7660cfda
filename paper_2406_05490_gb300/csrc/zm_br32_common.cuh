// zm_br32_common.cuh -- device pieces shared by the two FP32C Birkhoff-Rott kernels (the
// CUDA-core one of zm_br32.cu and the tensor-core one of zm_br32tc.cu): packed FP32x2
// arithmetic (two adjacent sources per instruction, even sources in the low word), the
// per-interface fixed-point scale, and the near-pair terms of one source tile (paper Sec. 2
// BRSolver, Sec. 3.2.1 ExactBRSolver; the masked form for the cutoff sum of Sec. 3.2.2).
#pragma once

#include "zm_internal.cuh"

namespace zm {
namespace {

constexpr int kTs = 256;  // sources per tile (and targets per target tile)

typedef unsigned long long u64;  // two packed floats (low word first)

__device__ __forceinline__ u64 ffma2(u64 a, u64 b, u64 c)
{
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 fmul2(u64 a, u64 b)
{
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 fadd2(u64 a, u64 b)
{
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 fsub2(u64 a, u64 b)
{
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 neg2(u64 a) { return a ^ 0x8000000080000000ull; }
__device__ __forceinline__ u64 pack2(float lo, float hi)
{
    u64 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ void unpack2(u64 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ float sum2(u64 v)
{
    float lo, hi;
    unpack2(v, lo, hi);
    return lo + hi;
}
__device__ __forceinline__ u64 rsqrt2(u64 v)
{
    float lo, hi;
    unpack2(v, lo, hi);
    return pack2(dev::rsqrt_approx(lo), dev::rsqrt_approx(hi));
}

// Fixed-point scale of one interface: |sum| <= N max|gamma'| * 0.385 / delta^2 < 2^(e+1); keep
// the scaled sum below 2^61.
__device__ __forceinline__ int fix_scale(const Inst &I)
{
    const float gm = __uint_as_float(*I.gmax);
    const double bound = (double)gm * (double)I.geom.N * 0.385 / (I.delta * I.delta) + 1e-300;
    return max(0, min(100, 60 - ilogb(bound)));
}

// Near pair terms of one source tile (record in shared memory `s`: hi/lo positions and scaled
// strengths, rows of kTs) for this thread's R targets, T threads apart in the target tile (near
// record row pointer `tr0`): the FP32 hi/lo difference r = (s_hi - t_hi) + (s_lo - t_lo),
// K = (|r|^2 + delta^2)^(-3/2), r x gamma, two adjacent sources per packed FP32x2 instruction
// (added at the end).  kMask: keep only pairs with |r|^2 <= c2 (the cutoff sum's per-pair
// decision, taken in FP32 on that difference: exact to about 2^-22 in the distance).
template <bool kMask, int R, int T>
__device__ __forceinline__ void near_tile(const float *s, const float *__restrict__ tr0, float d2, float c2,
                                          float mult, long long (*acc)[R][T], int tid)
{
    u64 hx[R], hy[R], hz[R], lx[R], ly[R], lz[R], px[R], py[R], pz[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float *tr = tr0 + r * T;
        float v;
        v = __ldg(tr);
        hx[r] = pack2(v, v);
        v = __ldg(tr + kTs);
        hy[r] = pack2(v, v);
        v = __ldg(tr + 2 * kTs);
        hz[r] = pack2(v, v);
        v = __ldg(tr + 3 * kTs);
        lx[r] = pack2(v, v);
        v = __ldg(tr + 4 * kTs);
        ly[r] = pack2(v, v);
        v = __ldg(tr + 5 * kTs);
        lz[r] = pack2(v, v);
        px[r] = py[r] = pz[r] = 0ull;
    }
    const u64 d22 = pack2(d2, d2);
    const u64 *s2 = reinterpret_cast<const u64 *>(s);  // row k at s2[k * kTs / 2]
    constexpr int H = kTs / 2;
#pragma unroll 2
    for (int m = 0; m < H; ++m) {
        const u64 shx = s2[m], shy = s2[H + m], shz = s2[2 * H + m];
        const u64 slx = s2[3 * H + m], sly = s2[4 * H + m], slz = s2[5 * H + m];
        const u64 gx = s2[6 * H + m], gy = s2[7 * H + m], gz = s2[8 * H + m];
        const u64 ngx = neg2(gx), ngy = neg2(gy), ngz = neg2(gz);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const u64 rx = fadd2(fsub2(shx, hx[r]), fsub2(slx, lx[r]));
            const u64 ry = fadd2(fsub2(shy, hy[r]), fsub2(sly, ly[r]));
            const u64 rz = fadd2(fsub2(shz, hz[r]), fsub2(slz, lz[r]));
            const u64 q = ffma2(rx, rx, ffma2(ry, ry, ffma2(rz, rz, d22)));
            const u64 iq = rsqrt2(q);
            u64 kk = fmul2(fmul2(iq, iq), iq);
            if (kMask) {
                const u64 r2 = ffma2(rx, rx, ffma2(ry, ry, fmul2(rz, rz)));
                float r2a, r2b, ka, kb;
                unpack2(r2, r2a, r2b);
                unpack2(kk, ka, kb);
                kk = pack2(r2a <= c2 ? ka : 0.0f, r2b <= c2 ? kb : 0.0f);
            }
            px[r] = ffma2(kk, ffma2(ry, gz, fmul2(rz, ngy)), px[r]);
            py[r] = ffma2(kk, ffma2(rz, gx, fmul2(rx, ngz)), py[r]);
            pz[r] = ffma2(kk, ffma2(rx, gy, fmul2(ry, ngx)), pz[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        acc[0][r][tid] += __float2ll_rn(sum2(px[r]) * mult);
        acc[1][r][tid] += __float2ll_rn(sum2(py[r]) * mult);
        acc[2][r][tid] += __float2ll_rn(sum2(pz[r]) * mult);
    }
}

}  // namespace
}  // namespace zm
