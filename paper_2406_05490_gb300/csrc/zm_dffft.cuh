// zm_dffft.cuh -- device building blocks of the double-word FFT Riesz passes (ZM_PREC_DF64),
// shared by the power-of-two passes (zm_lowdf.cu) and the passes over sides R 2^A
// (zm_lowdf_mix.cu).  Paper Sec. 2 (low-order model: FFT Riesz-transform velocity).
#pragma once

#include <algorithm>
#include <type_traits>

#include "zm_df64.cuh"
#include "zm_internal.cuh"

namespace zm {
namespace {

using namespace dw;

// A double-word constant prepared on the host.
struct Dc {
    float hi, lo;
};

inline Dc split(double v)
{
    const float h = (float)v;
    return Dc{h, (float)(v - (double)h)};
}

__device__ __forceinline__ df dc(Dc c) { return df{c.hi, c.lo}; }
// Node offsets are 32-bit: meshes hold at most 2^26 nodes, so 5N < 2^31.
__device__ __forceinline__ df ldf(const float2 *__restrict__ f, int k) { return from_f2(f[k]); }

// ---- FFT Riesz velocity --------------------------------------------------------------------------
// The same three passes as the FP64 path (rows forward with a transposed write; columns
// forward, Riesz multiplier, inverse, transposed write; rows inverse with the velocity
// epilogue), on complex double words in packed FP32x2 instructions.
//
// Each pass holds `rows` complete rows (rows * L up to 4096 complex values, 68 KiB with padding;
// a single row of 4096 at the largest side) in shared memory.  The log2 L radix-2 stages are done in chunks of K <= 4 stages: a thread
// loads a group of 2^K values spaced h apart into registers, applies the chunk's stages there
// and writes the group back, so shared memory is traversed once per chunk rather than once per
// stage.  Inside a chunk, pairs of stages are fused as radix-2^2 butterflies (three twiddle
// products per four values instead of four, bit-reversed order kept).  The first chunk of a
// pass reads its group straight from global memory; in pass B the last forward chunk, the
// Riesz multiplier and the first inverse chunk share one register group (the forward
// transform's last chunk and the inverse transform's first chunk both act on 2^K consecutive
// bit-reversed positions).  Shared memory is padded by one entry per 16 so that groups of
// consecutive values (h = 1) do not collide in banks.
// Twiddles W_L^k = exp(-2 pi i k / L) come from a half table (k < L/2), the upper range by
// W_L^(k + L/2) = -W_L^k, conjugated for the inverse.

#ifndef ZM_DF_KMAX
#define ZM_DF_KMAX 4  // most radix-2 stages per register group (group of 2^K values)
#endif
#ifndef ZM_DF_REGS
#define ZM_DF_REGS 128  // register budget per thread the FFT passes are compiled for
#endif
#ifndef ZM_DF_ELEMS
#define ZM_DF_ELEMS 4096  // complex values per CTA of an FFT pass (rows * row length)
#endif
constexpr int kKmax = ZM_DF_KMAX;
constexpr int kFftElems = ZM_DF_ELEMS;

__device__ __forceinline__ int bitrev(int j, int logL) { return (int)(__brev((unsigned)j) >> (32 - logL)); }
__device__ __forceinline__ int phys(int i) { return i + (i >> 4); }

__device__ __forceinline__ C2 tw_get(const ulonglong2 *__restrict__ tw, int k, int half, int sgn)
{
    const bool up = k >= half;
    const ulonglong2 v = __ldg(tw + (up ? k - half : k));
    u64 flip = up ? (kSign0 | kSign1) : 0ull;
    if (sgn > 0) flip ^= kSign1;  // conjugate: negate the imaginary lane
    return C2{v.x ^ flip, v.y ^ flip};
}

// Radix-2^2 decimation-in-frequency butterfly on v[m], v[m+Q], v[m+2Q], v[m+3Q] (positions
// p, p + S, p + 2S, p + 3S of a block of 4S); e1 = exponent of W_{4S}^p on W_L.
template <int Q>
__device__ __forceinline__ void bfly_dif(C2 *v, int m, int e1, int half, const ulonglong2 *__restrict__ tw, int sgn)
{
    const C2 a0 = v[m], a1 = v[m + Q], a2 = v[m + 2 * Q], a3 = v[m + 3 * Q];
    const C2 s02 = cadd2_lazy(a0, a2), d02 = csub2_lazy(a0, a2), s13 = cadd2_lazy(a1, a3);
    const C2 d13 = cmul_i2(csub2_lazy(a1, a3), sgn);
    v[m] = cadd2(s02, s13);
    const C2 x2 = csub2(s02, s13), x1 = cadd2(d02, d13), x3 = csub2(d02, d13);
    if (e1 == 0) {
        v[m + Q] = x2;
        v[m + 2 * Q] = x1;
        v[m + 3 * Q] = x3;
    } else {
        v[m + Q] = cmul2(x2, tw_get(tw, 2 * e1, half, sgn));
        v[m + 2 * Q] = cmul2(x1, tw_get(tw, e1, half, sgn));
        v[m + 3 * Q] = cmul2(x3, tw_get(tw, 3 * e1, half, sgn));
    }
}

// Radix-2^2 decimation-in-time butterfly (spans S, then 2S).
template <int Q>
__device__ __forceinline__ void bfly_dit(C2 *v, int m, int e1, int half, const ulonglong2 *__restrict__ tw, int sgn)
{
    const C2 a0 = v[m];
    C2 c1 = v[m + Q], c2 = v[m + 2 * Q], c3 = v[m + 3 * Q];
    if (e1 != 0) {
        c1 = cmul2(c1, tw_get(tw, 2 * e1, half, sgn));
        c2 = cmul2(c2, tw_get(tw, e1, half, sgn));
        c3 = cmul2(c3, tw_get(tw, 3 * e1, half, sgn));
    }
    const C2 s01 = cadd2_lazy(a0, c1), d01 = csub2_lazy(a0, c1), s23 = cadd2_lazy(c2, c3);
    const C2 d23 = cmul_i2(csub2_lazy(c2, c3), sgn);
    v[m] = cadd2(s01, s23);
    v[m + 2 * Q] = csub2(s01, s23);
    v[m + Q] = cadd2(d01, d23);
    v[m + 3 * Q] = csub2(d01, d23);
}

// The K decimation-in-frequency stages of one chunk on a register group: v[m] is the value at
// position base + m h of its row (h = 2^lh, pos = base mod h); spans h 2^(K-1) down to h.
template <int K>
__device__ __forceinline__ void dif_chunk(C2 *v, int pos, int lh, int logL, const ulonglong2 *__restrict__ tw, int sgn)
{
    constexpr int R = 1 << K;
    const int half = 1 << (logL - 1);
    if (K & 1) {  // one radix-2 stage at the top span S = h 2^(K-1): W_{2S}^(pos + m h)
#pragma unroll
        for (int m = 0; m < R / 2; ++m) {
            const C2 a = v[m], b = v[m + R / 2];
            v[m] = cadd2(a, b);
            const C2 d = csub2(a, b);
            const int e = (pos + (m << lh)) << (logL - lh - K);
            v[m + R / 2] = e ? cmul2(d, tw_get(tw, e, half, sgn)) : d;
        }
    }
#pragma unroll
    for (int jj = (K & 1) ? K - 3 : K - 2; jj >= 0; jj -= 2) {  // spans (2S, S), S = h 2^jj
#pragma unroll
        for (int m = 0; m < R; ++m) {
            if ((m & (4 << jj) - 1) >= (1 << jj)) continue;  // quadruple leaders only
            const int r = m & ((1 << jj) - 1);
            const int e1 = (pos + (r << lh)) << (logL - lh - jj - 2);
            if (jj == 0) bfly_dif<1>(v, m, e1, half, tw, sgn);
            else bfly_dif<4>(v, m, e1, half, tw, sgn);
        }
    }
}

// The K decimation-in-time stages of one chunk: spans h up to h 2^(K-1).
template <int K>
__device__ __forceinline__ void dit_chunk(C2 *v, int pos, int lh, int logL, const ulonglong2 *__restrict__ tw, int sgn)
{
    constexpr int R = 1 << K;
    const int half = 1 << (logL - 1);
#pragma unroll
    for (int jj = 0; jj + 2 <= K; jj += 2) {  // spans (S, 2S), S = h 2^jj
#pragma unroll
        for (int m = 0; m < R; ++m) {
            if ((m & (4 << jj) - 1) >= (1 << jj)) continue;
            const int r = m & ((1 << jj) - 1);
            const int e1 = (pos + (r << lh)) << (logL - lh - jj - 2);
            if (jj == 0) bfly_dit<1>(v, m, e1, half, tw, sgn);
            else bfly_dit<4>(v, m, e1, half, tw, sgn);
        }
    }
    if (K & 1) {  // one radix-2 stage at the top span
#pragma unroll
        for (int m = 0; m < R / 2; ++m) {
            const C2 a = v[m];
            C2 b = v[m + R / 2];
            const int e = (pos + (m << lh)) << (logL - lh - K);
            if (e) b = cmul2(b, tw_get(tw, e, half, sgn));
            v[m] = cadd2(a, b);
            v[m + R / 2] = csub2(a, b);
        }
    }
}

// Chunk plan, fixed at compile time per row length 2^l: ceil(l / kKmax) chunks of near-equal
// size, the larger ones last (so that the last forward chunk of pass B, which the first inverse
// chunk mirrors, is the largest).  Chunk c of the forward transform, and chunk c of the inverse
// one, act on values spaced 2^lh_of(l, c) apart.
constexpr int nc_of(int l) { return (l + kKmax - 1) / kKmax; }
constexpr int k_of(int l, int c) { return l / nc_of(l) + (c >= nc_of(l) - l % nc_of(l) ? 1 : 0); }
constexpr int lh_of(int l, int c) { return c < 0 ? l : lh_of(l, c - 1) - k_of(l, c); }

// Group g of a chunk with 2^K values per group and spacing h = 2^lh, in a pass over `rows`
// rows of length 2^l: its row, pos and base position.
struct Grp {
    int row, pos, base;
};

__device__ __forceinline__ Grp group_of(int g, int K, int lh, int l)
{
    const int per_row = 1 << (l - K);
    const int gi = g & (per_row - 1);
    const int pos = gi & ((1 << lh) - 1);
    return Grp{g >> (l - K), pos, ((gi >> lh) << (lh + K)) + pos};
}

// One chunk: load each group with ld(row, index), run the K stages, store with st(row, index).
template <int K, bool kDif, int L, int LH, class Ld, class St>
__device__ __forceinline__ void chunk_pass(int rows, const ulonglong2 *__restrict__ tw, int sgn, Ld ld, St st)
{
    constexpr int R = 1 << K;
    const int ngroups = rows << (L - K);
    for (int g = threadIdx.x; g < ngroups; g += blockDim.x) {
        const Grp q = group_of(g, K, LH, L);
        C2 v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = ld(q.row, q.base + (m << LH));
        if (kDif) dif_chunk<K>(v, q.pos, LH, L, tw, sgn);
        else dit_chunk<K>(v, q.pos, LH, L, tw, sgn);
#pragma unroll
        for (int m = 0; m < R; ++m) st(q.row, q.base + (m << LH), v[m]);
    }
}

// Forward chunks C .. CEnd of `rows` rows of length 2^L in shared memory `sx` (padded); chunk 0
// reads its groups with ld0 (global memory) instead.
template <int L, int C, int CEnd, class Ld0>
__device__ __forceinline__ void dif_seq(ulonglong2 *sx, const ulonglong2 *__restrict__ tw, int rows, int sgn, Ld0 ld0)
{
    if constexpr (C <= CEnd) {
        constexpr int K = k_of(L, C), LH = lh_of(L, C);
        auto sts = [&](int row, int i, C2 v) { sx[phys((row << L) + i)] = st2(v); };
        if constexpr (C == 0) {
            chunk_pass<K, true, L, LH>(rows, tw, sgn, ld0, sts);
        } else {
            auto lds = [&](int row, int i) { return ld2(sx[phys((row << L) + i)]); };
            chunk_pass<K, true, L, LH>(rows, tw, sgn, lds, sts);
        }
        __syncthreads();
        dif_seq<L, C + 1, CEnd>(sx, tw, rows, sgn, ld0);
    }
}

// Inverse chunks C, C - 1, .., 0 (spans growing) in shared memory.
template <int L, int C>
__device__ __forceinline__ void dit_seq(ulonglong2 *sx, const ulonglong2 *__restrict__ tw, int rows, int sgn)
{
    if constexpr (C >= 0) {
        constexpr int K = k_of(L, C), LH = lh_of(L, C);
        auto lds = [&](int row, int i) { return ld2(sx[phys((row << L) + i)]); };
        auto sts = [&](int row, int i, C2 v) { sx[phys((row << L) + i)] = st2(v); };
        chunk_pass<K, false, L, LH>(rows, tw, sgn, lds, sts);
        __syncthreads();
        dit_seq<L, C - 1>(sx, tw, rows, sgn);
    }
}

__device__ __forceinline__ ulonglong2 c2_pack(float2 re, float2 im)
{
    return make_ulonglong2(pk(re.x, im.x), pk(re.y, im.y));
}

// Threads per CTA and resident CTAs per SM of the passes over rows of length 2^L: one group of
// 16 values per thread over the CTA's kFftElems values (a single row when it is longer), as many
// CTAs per SM as a budget of ZM_DF_REGS registers per thread allows.
constexpr int elems_for(int L) { return (1 << L) > kFftElems ? (1 << L) : kFftElems; }
constexpr int threads_for(int L) { return elems_for(L) / 16; }
constexpr int minb_for(int L) { return 65536 / (threads_for(L) * ZM_DF_REGS); }

// The Riesz multiplier -(k2 + i k1)/|k| at frequency (i, j) as a complex double word, zero at
// k = 0 and on the Nyquist row and column; k_l/|k| is formed from t_l = m_l / L_l (2 pi cancels).
__device__ __forceinline__ C2 riesz_mult(int i, int j, int n1, int n2, Dc invL1, Dc invL2)
{
    const int m1 = (2 * i < n1) ? i : i - n1;
    const int m2 = (2 * j < n2) ? j : j - n2;
    if ((m1 == 0 && m2 == 0) || 2 * i == n1 || 2 * j == n2) return C2{0ull, 0ull};
    const df t1 = mul_f(dc(invL1), (float)m1), t2 = mul_f(dc(invL2), (float)m2);
    const df rs = rsqrt(add(sqr(t1), sqr(t2)));
    return c2_from(neg(mul(t2, rs)), neg(mul(t1, rs)));
}

// Pass B's middle: the last forward chunk, the multiplier and the first inverse chunk on one
// register group of 2^K consecutive (bit-reversed) positions of a column of length 2^L.
// kMix: the rows are the sub-rows of columns of length n1 = RR 2^L (RR odd, > 1): sub-row
// q.row = r RR + k2 of column j0 + r holds the frequencies RR k1 + k2.
template <int L, bool kMix = false>
__device__ __forceinline__ void mid_b(ulonglong2 *sx, int rows, int j0, int n2, Dc invL1, Dc invL2,
                                      const ulonglong2 *__restrict__ tw1, int RR = 1)
{
    constexpr int K = k_of(L, nc_of(L) - 1), R = 1 << K;
    const int ngroups = rows << (L - K);
    for (int g = threadIdx.x; g < ngroups; g += blockDim.x) {
        const Grp q = group_of(g, K, 0, L);
        C2 v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = ld2(sx[phys((q.row << L) + q.base + m)]);
        dif_chunk<K>(v, 0, 0, L, tw1, -1);
        const int ib = bitrev(q.base, L);
        int col = j0 + q.row, k2 = 0;
        if (kMix) {
            const int r = q.row / RR;
            col = j0 + r;
            k2 = q.row - r * RR;
        }
#pragma unroll
        for (int m = 0; m < R; ++m) {
            const int k1 = ib | (bitrev(m, K) << (L - K));  // natural frequency index of base + m
            const int i = kMix ? RR * k1 + k2 : k1;
            v[m] = cmul2(v[m], riesz_mult(i, col, kMix ? (RR << L) : (1 << L), n2, invL1, invL2));
        }
        dit_chunk<K>(v, 0, 0, L, tw1, +1);
#pragma unroll
        for (int m = 0; m < R; ++m) sx[phys((q.row << L) + q.base + m)] = st2(v[m]);
    }
}

// padded shared-memory entries for `count` complex values (one pad entry per 16)
int phys_host(int count) { return count + count / 16; }

int ilog2(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

bool pow2_side(int n) { return (n & (n - 1)) == 0; }

// Calls f(std::integral_constant<int, l>) for the row-length exponents the FFT supports.
template <class F>
int with_log2(int l, F &&f)
{
    switch (l) {
    case 3: return f(std::integral_constant<int, 3>{});
    case 4: return f(std::integral_constant<int, 4>{});
    case 5: return f(std::integral_constant<int, 5>{});
    case 6: return f(std::integral_constant<int, 6>{});
    case 7: return f(std::integral_constant<int, 7>{});
    case 8: return f(std::integral_constant<int, 8>{});
    case 9: return f(std::integral_constant<int, 9>{});
    case 10: return f(std::integral_constant<int, 10>{});
    case 11: return f(std::integral_constant<int, 11>{});
    case 12: return f(std::integral_constant<int, 12>{});
    default: return set_error(ZM_ERR_UNSUPPORTED, "double-word FFT: side must be 2^3 .. 2^12");
    }
}

// Sets a kernel's dynamic shared-memory limit (a host-side attribute, legal during stream capture).
inline int smem_attr(const void *fn, size_t smem)
{
    return cuda_check(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                      "double-word FFT shared-memory attribute");
}

}  // namespace

// Passes over rows of length R 2^A (R odd, 3 .. 19; 3 <= A <= 12), in zm_lowdf_mix.cu.  Arguments
// as the power-of-two passes; lr = log2 of the rows per CTA, smem = its dynamic shared memory.
int df_mix_pass_a(int A, int n1, int R, int lr, size_t smem, cudaStream_t s, const float2 *w,
                  const ulonglong2 *tw2, const ulonglong2 *twl2, ulonglong2 *out);
int df_mix_pass_b(int A, int n2, int R, int lr, size_t smem, cudaStream_t s, double invL1, double invL2,
                  const ulonglong2 *in, const ulonglong2 *tw1, const ulonglong2 *twl1, ulonglong2 *out);
int df_mix_pass_c(int A, int n1, int R, int lr, size_t smem, cudaStream_t s, double scale, const ulonglong2 *in,
                  const ulonglong2 *tw2, const ulonglong2 *twl2, const float2 *nrm, const float2 *q, float2 *u,
                  float2 *phi);
// Radices the double-word passes take.
#define ZM_DF_RADICES(X) X(3) X(5) X(7) X(9) X(11) X(13) X(15) X(17) X(19)

}  // namespace zm
