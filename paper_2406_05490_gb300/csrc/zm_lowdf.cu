// zm_lowdf.cu -- the low-order Z-Model derivative and RK3 stage in double-word arithmetic
// (ZM_PREC_DF64): the same equations as the FP64 low-order path (paper Sec. 2 low-order
// model: FFT Riesz-transform velocity along the normal; Sec. 3.1 SurfaceMesh stencils,
// BoundaryCondition periodic ghosts, TimeIntegrator SSP-RK3), computed in FP32-pair
// ("double-float", zm_df64.cuh) arithmetic instead of FP64 instructions.
//
// Device-resident state and every intermediate field are double words (float2, 8 bytes per
// value, the same footprint as FP64).  z1 and z2 are stored as displacements from the mesh
// coordinates, d1 = z1 - i dx1, d2 = z2 - j dx2: the displacement is periodic (the seam shift
// disappears), and the 4th-order difference of the mesh coordinate is exactly 1, so
// a1 = (1 + D1 d1, D1 d2, D1 d3) and a2 = (D2 d1, 1 + D2 d2, D2 d3).  Storing displacements keeps
// the 2^-48 relative rounding of the stored values proportional to the perturbation, not to
// the coordinate, before the stencil divides by dx.
// Conversions between the FP64 API arrays and this storage run only at set/get/velocity calls.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "zm_df64.cuh"
#include "zm_internal.cuh"

namespace zm {
namespace {

using namespace dw;

constexpr int kTpb = 256;

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
// Node offsets are 32-bit: low order is limited to 4096^2 = 2^24 nodes, so 5N < 2^31.
__device__ __forceinline__ df ldf(const float2 *__restrict__ f, int k) { return from_f2(f[k]); }

struct DfGeo {
    int n1, n2, l2;
    int N;
    Dc i12a, i12b;    // 1 / (12 dx1), 1 / (12 dx2)
    Dc i12a2, i12b2;  // 1 / (12 dx1^2), 1 / (12 dx2^2)
    Dc d12a, d12b;    // 12 dx1, 12 dx2
    Dc c8det;         // (144 dx1 dx2)^2 / 8
    Dc grav;          // g
    Dc m2a;           // -2 A
    Dc mu;
};

// Periodic 4th-order first difference along one axis at node p: the four neighbours are
// p + k * stride for k = -2, -1, 1, 2 after wrapping the axis index c0 + k into [0, n).
struct Nb {
    int m2, m1, p1, p2;
};

__device__ __forceinline__ Nb nb_axis0(int i, int j, const DfGeo &g)
{
    const int m = g.n1 - 1;
    return Nb{(((i - 2) & m) << g.l2) + j, (((i - 1) & m) << g.l2) + j, (((i + 1) & m) << g.l2) + j,
              (((i + 2) & m) << g.l2) + j};
}

__device__ __forceinline__ Nb nb_axis1(int i, int j, const DfGeo &g)
{
    const int m = g.n2 - 1;
    const int r = i << g.l2;
    return Nb{r + ((j - 2) & m), r + ((j - 1) & m), r + ((j + 1) & m), r + ((j + 2) & m)};
}

// (f-2 - f+2) + 8 (f+1 - f-1): 12 dx times the 4th-order first difference
__device__ __forceinline__ df diff1_s(const float2 *__restrict__ f, const Nb &n)
{
    return stencil_s(ldf(f, n.m2), ldf(f, n.m1), ldf(f, n.p1), ldf(f, n.p2));
}

// ((f-2 - f+2) + 8 (f+1 - f-1)) / (12 dx)
__device__ __forceinline__ df diff1_df(const float2 *__restrict__ f, const Nb &n, df inv12)
{
    return mul(diff1_s(f, n), inv12);
}

// (16 (f-1 + f+1) - (f-2 + f+2) - 30 f0) / (12 dx^2), accurate sums: the three groups cancel
// to O(dx^2) of their size.
__device__ __forceinline__ df diff2_df(const float2 *__restrict__ f, const Nb &n, int p0, df inv12sq)
{
    const df s1 = add_acc(ldf(f, n.m1), ldf(f, n.p1));
    const df s2 = add_acc(ldf(f, n.m2), ldf(f, n.p2));
    const df t = sub_acc(sub_acc(scale2(s1, 16.0f), s2), mul_f(ldf(f, p0), 30.0f));
    return mul(t, inv12sq);
}

// Geometry pass: unit normal N = a1 x a2 / |a1 x a2| and q = g z3 + 1/8 w^T h^-1 w.
// The tangents are kept scaled, b_l = 12 dx_l a_l (the stencil sums without the division), since
// the unit normal does not depend on their lengths; with gamma = w1 a2 - w2 a1 (formed from b and
// w_l / (12 dx)), w^T h^-1 w = |gamma|^2 / det and det = |a1 x a2|^2 = |b1 x b2|^2 / (144 dx1 dx2)^2
// (Lagrange's identity), so one rsqrt of |b1 x b2|^2 serves both.
__global__ void __launch_bounds__(kTpb)
    geometry_df(DfGeo g, const float2 *__restrict__ y, float2 *__restrict__ q, float2 *__restrict__ nrm)
{
    const int p = blockIdx.x * kTpb + threadIdx.x;
    if (p >= g.N) return;
    const int i = p >> g.l2, j = p & (g.n2 - 1);
    const int N = g.N;
    const Nb na = nb_axis0(i, j, g), nb = nb_axis1(i, j, g);
    df b1[3], b2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        b1[c] = diff1_s(y + c * N, na);
        b2[c] = diff1_s(y + c * N, nb);
    }
    b1[0] = add(dc(g.d12a), b1[0]);  // the mesh coordinate's share: 12 dx1 along alpha1
    b2[1] = add(dc(g.d12b), b2[1]);
    const df nx = mul_sub(b1[1], b2[2], b1[2], b2[1]);
    const df ny = mul_sub(b1[2], b2[0], b1[0], b2[2]);
    const df nz = mul_sub(b1[0], b2[1], b1[1], b2[0]);
    const df rs = rsqrt(sum_sq3(nx, ny, nz));
    nrm[p] = to_f2(mul(nx, rs));
    nrm[N + p] = to_f2(mul(ny, rs));
    nrm[2 * N + p] = to_f2(mul(nz, rs));

    // gamma = (w1 / (12 dx2)) b2 - (w2 / (12 dx1)) b1
    const df s1 = mul(ldf(y, 3 * N + p), dc(g.i12b)), s2 = mul(ldf(y, 4 * N + p), dc(g.i12a));
    const df gx = mul_sub(s1, b2[0], s2, b1[0]);
    const df gy = mul_sub(s1, b2[1], s2, b1[1]);
    const df gz = mul_sub(s1, b2[2], s2, b1[2]);
    const df g2 = sum_sq3(gx, gy, gz);
    // 1/8 |gamma|^2 / det = 1/8 |gamma|^2 rs^2 (144 dx1 dx2)^2
    const df jump = mul(mul(g2, sqr(rs)), dc(g.c8det));
    q[p] = to_f2(add(mul(dc(g.grav), ldf(y, 2 * N + p)), jump));
}

// Vorticity pass: dw_l/dt = -2 A D_l Phi + mu Lap w_l.  Mode 0 writes dw/dt; mode 1 the SSP-RK3
// stage yout = ca y0 + cb (y + dt (u, dw/dt)).
template <bool kVisc, int kMode>
__global__ void __launch_bounds__(kTpb)
    vorticity_df(DfGeo g, const float2 *__restrict__ phi, const float2 *__restrict__ y,
                 const float2 *__restrict__ u, Dc dt, Dc ca, Dc cb, const float2 *y0, float2 *yout,
                 float2 *__restrict__ wdot)
{
    const int p = blockIdx.x * kTpb + threadIdx.x;
    if (p >= g.N) return;
    const int i = p >> g.l2, j = p & (g.n2 - 1);
    const int N = g.N;
    const Nb na = nb_axis0(i, j, g), nb = nb_axis1(i, j, g);
    const df m2a = dc(g.m2a);
    df f1 = mul(m2a, diff1_df(phi, na, dc(g.i12a)));
    df f2 = mul(m2a, diff1_df(phi, nb, dc(g.i12b)));
    if (kVisc) {
        const float2 *w1 = y + 3 * N, *w2 = y + 4 * N;
        const df l1 = add(diff2_df(w1, na, p, dc(g.i12a2)), diff2_df(w1, nb, p, dc(g.i12b2)));
        const df l2 = add(diff2_df(w2, na, p, dc(g.i12a2)), diff2_df(w2, nb, p, dc(g.i12b2)));
        f1 = add(f1, mul(dc(g.mu), l1));
        f2 = add(f2, mul(dc(g.mu), l2));
    }
    if (kMode == 0) {
        wdot[p] = to_f2(f1);
        wdot[N + p] = to_f2(f2);
        return;
    }
    const df d[5] = {ldf(u, p), ldf(u, N + p), ldf(u, 2 * N + p), f1, f2};
    float2 out[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        const df s = add(ldf(y, c * N + p), mul(dc(dt), d[c]));
        out[c] = to_f2(add(mul(dc(ca), ldf(y0, c * N + p)), mul(dc(cb), s)));
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) yout[c * N + p] = out[c];
}

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

// pass A: rows i (length n2 = 2^L) of c = w1 + i w2; forward; write out[j][i] (transposed).
template <int L>
__global__ void __launch_bounds__(threads_for(L), minb_for(L))
    pass_a_df(int n1, int lr, const float2 *__restrict__ w, const ulonglong2 *__restrict__ tw2,
              ulonglong2 *__restrict__ out)
{
    extern __shared__ ulonglong2 sx[];
    const int rows = 1 << lr;
    const int i0 = blockIdx.x * rows;
    const size_t N = (size_t)n1 << L;
    const float2 *w1 = w + ((size_t)i0 << L), *w2 = w1 + N;
    auto ldg = [&](int row, int i) { return ld2(c2_pack(w1[(row << L) + i], w2[(row << L) + i])); };
    dif_seq<L, 0, nc_of(L) - 1>(sx, tw2, rows, -1, ldg);
    for (int e = threadIdx.x; e < (rows << L); e += blockDim.x) {
        const int j = e >> lr, r = e & (rows - 1);
        out[(size_t)j * n1 + i0 + r] = sx[phys((r << L) + bitrev(j, L))];
    }
}

// The Riesz multiplier -(k2 + i k1)/|k| at frequency (i, j) as a complex double word, zero at
// k = 0 and on the Nyquist row and column; k_l/|k| is formed from t_l = m_l / L_l (2 pi cancels).
__device__ __forceinline__ C2 riesz_mult(int i, int j, int n1, int n2, Dc invL1, Dc invL2)
{
    const int m1 = (i < n1 / 2) ? i : i - n1;
    const int m2 = (j < n2 / 2) ? j : j - n2;
    if ((m1 == 0 && m2 == 0) || 2 * i == n1 || 2 * j == n2) return C2{0ull, 0ull};
    const df t1 = mul_f(dc(invL1), (float)m1), t2 = mul_f(dc(invL2), (float)m2);
    const df rs = rsqrt(add(sqr(t1), sqr(t2)));
    return c2_from(neg(mul(t2, rs)), neg(mul(t1, rs)));
}

// Pass B's middle: the last forward chunk, the multiplier and the first inverse chunk on one
// register group of 2^K consecutive (bit-reversed) positions of a column of length 2^L.
template <int L>
__device__ __forceinline__ void mid_b(ulonglong2 *sx, int rows, int j0, int n2, Dc invL1, Dc invL2,
                                      const ulonglong2 *__restrict__ tw1)
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
#pragma unroll
        for (int m = 0; m < R; ++m) {
            const int i = ib | (bitrev(m, K) << (L - K));  // natural frequency index of base + m
            v[m] = cmul2(v[m], riesz_mult(i, j0 + q.row, 1 << L, n2, invL1, invL2));
        }
        dit_chunk<K>(v, 0, 0, L, tw1, +1);
#pragma unroll
        for (int m = 0; m < R; ++m) sx[phys((q.row << L) + q.base + m)] = st2(v[m]);
    }
}

// pass B: rows j (length n1 = 2^L) of the transpose; forward; multiply; inverse; write out[i][j].
template <int L>
__global__ void __launch_bounds__(threads_for(L), minb_for(L))
    pass_b_df(int n2, int lr, Dc invL1, Dc invL2, const ulonglong2 *__restrict__ in,
              const ulonglong2 *__restrict__ tw1, ulonglong2 *__restrict__ out)
{
    extern __shared__ ulonglong2 sx[];
    constexpr int NC = nc_of(L);
    const int rows = 1 << lr;
    const int j0 = blockIdx.x * rows;
    const ulonglong2 *src = in + ((size_t)j0 << L);
    if constexpr (NC == 1) {  // the whole transform is the middle group: stage the rows first
        for (int e = threadIdx.x; e < (rows << L); e += blockDim.x) sx[phys(e)] = src[e];
        __syncthreads();
    } else {
        auto ldg = [&](int row, int i) { return ld2(src[(row << L) + i]); };
        dif_seq<L, 0, NC - 2>(sx, tw1, rows, -1, ldg);
    }
    mid_b<L>(sx, rows, j0, n2, invL1, invL2, tw1);
    __syncthreads();
    dit_seq<L, NC - 2>(sx, tw1, rows, +1);
    for (int e = threadIdx.x; e < (rows << L); e += blockDim.x) {
        const int i = e >> lr, r = e & (rows - 1);
        out[(size_t)i * n2 + j0 + r] = sx[phys((r << L) + i)];
    }
}

// pass C: rows i (length n2 = 2^L); inverse; s = Re / (n1 n2); u = -s/2 N; Phi = q + |u|^2 / 2.
template <int L>
__global__ void __launch_bounds__(threads_for(L), minb_for(L))
    pass_c_df(int n1, int lr, float scale, const ulonglong2 *__restrict__ in,
              const ulonglong2 *__restrict__ tw2, const float2 *__restrict__ nrm,
              const float2 *__restrict__ q, float2 *__restrict__ u, float2 *__restrict__ phi)
{
    extern __shared__ ulonglong2 sx[];
    const int rows = 1 << lr;
    const int i0 = blockIdx.x * rows;
    const size_t N = (size_t)n1 << L;
    const size_t o = (size_t)i0 << L;
    const ulonglong2 *src = in + o;
    auto ldg = [&](int row, int i) { return ld2(src[(row << L) + i]); };
    dif_seq<L, 0, nc_of(L) - 1>(sx, tw2, rows, +1, ldg);
#pragma unroll 4
    for (int e = threadIdx.x; e < (rows << L); e += blockDim.x) {
        const int r = e >> L, j = e & ((1 << L) - 1);
        const size_t p = o + e;
        const df s = scale2(c2_re(ld2(sx[phys((r << L) + bitrev(j, L))])), scale);  // scale = -1/(2 n1 n2)
        const df ux = mul(s, ldf(nrm, p)), uy = mul(s, ldf(nrm, N + p)), uz = mul(s, ldf(nrm, 2 * N + p));
        u[p] = to_f2(ux);
        u[N + p] = to_f2(uy);
        u[2 * N + p] = to_f2(uz);
        const df k2 = add(add(sqr(ux), sqr(uy)), sqr(uz));
        phi[p] = to_f2(add(ldf(q, p), scale2(k2, 0.5f)));
    }
}

// twiddle table entry k < L/2: {cos.hi, sin.hi, cos.lo, sin.lo} of -2 pi k / L
__global__ void twiddle_df_kernel(int L, float4 *tw)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L / 2) return;
    double s, c;
    sincospi(-2.0 * (double)k / (double)L, &s, &c);
    const float ch = __double2float_rn(c), sh = __double2float_rn(s);
    tw[k] = make_float4(ch, sh, __double2float_rn(c - (double)ch), __double2float_rn(s - (double)sh));
}

// ---- conversions between the FP64 API arrays and double-word storage -----------------------------
// to_df: dst[k] = split(src[k] - alpha), alpha = the mesh coordinate for z1 and z2 when `state`
// (src holds the 5N state), else 0.  from_df: the inverse.  Element k is read and written by the
// same thread, so src and dst may be the same buffer.
__global__ void to_df_kernel(int l2, int n2, size_t N, size_t count, double dx1, double dx2, int state,
                             const double *src, float2 *dst)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < count;
         k += (size_t)gridDim.x * blockDim.x) {
        double v = src[k];
        if (state && k < 2 * N) {
            const size_t p = k < N ? k : k - N;
            v -= k < N ? (double)(p >> l2) * dx1 : (double)(p & (n2 - 1)) * dx2;
        }
        const float hi = __double2float_rn(v);
        dst[k] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
}

__global__ void from_df_kernel(int l2, int n2, size_t N, size_t count, double dx1, double dx2, int state,
                               const float2 *src, double *dst)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < count;
         k += (size_t)gridDim.x * blockDim.x) {
        const float2 f = src[k];
        double v = (double)f.x + (double)f.y;
        if (state && k < 2 * N) {
            const size_t p = k < N ? k : k - N;
            v += k < N ? (double)(p >> l2) * dx1 : (double)(p & (n2 - 1)) * dx2;
        }
        dst[k] = v;
    }
}

__global__ void finite_f32_kernel(size_t n, const float *__restrict__ y, int *bad)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        if (!isfinite(y[k])) {
            atomicOr(bad, 1);
            return;
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

// log2 of the rows per CTA of an FFT pass over rows of length 2^l, and no more rows than the
// pass has (`avail`).
int lrows_for(int l, int avail) { return ilog2(std::max(1, std::min(elems_for(l) >> l, avail))); }

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

DfGeo make_geo(const zm_ctx *c)
{
    const Geom &G = c->geom;
    DfGeo g;
    g.n1 = G.n1;
    g.n2 = G.n2;
    g.l2 = ilog2(G.n2);
    g.N = G.N;
    g.i12a = split(1.0 / (12.0 * G.dx1));
    g.i12b = split(1.0 / (12.0 * G.dx2));
    g.i12a2 = split(1.0 / (12.0 * G.dx1 * G.dx1));
    g.i12b2 = split(1.0 / (12.0 * G.dx2 * G.dx2));
    g.d12a = split(12.0 * G.dx1);
    g.d12b = split(12.0 * G.dx2);
    g.c8det = split((144.0 * G.dx1 * G.dx2) * (144.0 * G.dx1 * G.dx2) / 8.0);
    g.grav = split(c->g);
    g.m2a = split(-2.0 * c->atwood);
    g.mu = split(c->mu);
    return g;
}

inline const float2 *F2(const double *p) { return reinterpret_cast<const float2 *>(p); }
inline float2 *F2(double *p) { return reinterpret_cast<float2 *>(p); }
inline ulonglong2 *U2(double2 *p) { return reinterpret_cast<ulonglong2 *>(p); }

// Launches of the three passes for rows of length 2^L.  Each sets the kernel's dynamic shared
// memory limit (a host-side attribute, legal during stream capture) and checks its own launch.
template <int L>
struct FftLaunch {
    static int prep(const void *fn, size_t smem)
    {
        return cuda_check(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                          "double-word FFT shared-memory attribute");
    }
    static int a(int n1, int lr, size_t smem, cudaStream_t s, const float2 *w, const ulonglong2 *tw2, ulonglong2 *out)
    {
        int rc = prep((const void *)pass_a_df<L>, smem);
        if (rc) return rc;
        pass_a_df<L><<<n1 >> lr, threads_for(L), smem, s>>>(n1, lr, w, tw2, out);
        return cuda_check(cudaGetLastError(), "double-word FFT pass A launch");
    }
    static int b(int n2, int lr, size_t smem, cudaStream_t s, Dc invL1, Dc invL2, const ulonglong2 *in,
                 const ulonglong2 *tw1, ulonglong2 *out)
    {
        int rc = prep((const void *)pass_b_df<L>, smem);
        if (rc) return rc;
        pass_b_df<L><<<n2 >> lr, threads_for(L), smem, s>>>(n2, lr, invL1, invL2, in, tw1, out);
        return cuda_check(cudaGetLastError(), "double-word FFT pass B launch");
    }
    static int c(int n1, int lr, size_t smem, cudaStream_t s, float scale, const ulonglong2 *in,
                 const ulonglong2 *tw2, const float2 *nrm, const float2 *q, float2 *u, float2 *phi)
    {
        int rc = prep((const void *)pass_c_df<L>, smem);
        if (rc) return rc;
        pass_c_df<L><<<n1 >> lr, threads_for(L), smem, s>>>(n1, lr, scale, in, tw2, nrm, q, u, phi);
        return cuda_check(cudaGetLastError(), "double-word FFT pass C launch");
    }
};

}  // namespace

int df_setup(zm_ctx *c)
{
    const Geom &g = c->geom;
    const size_t N = g.N;
    if (cudaMalloc(&c->fa, N * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&c->fb, N * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&c->tw1, (g.n1 / 2) * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&c->tw2, (g.n2 / 2) * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ZM_ERR_NOMEM, "df_setup: device allocation failed");
    }
    twiddle_df_kernel<<<(g.n1 / 2 + 255) / 256, 256>>>(g.n1, reinterpret_cast<float4 *>(c->tw1));
    twiddle_df_kernel<<<(g.n2 / 2 + 255) / 256, 256>>>(g.n2, reinterpret_cast<float4 *>(c->tw2));
    int rc = ZM_OK;
    if (!rc) rc = cuda_check(cudaGetLastError(), "df twiddle kernel");
    return rc;
}

int df_derivative(zm_ctx *c, const double *y)
{
    if (!y || !c->q || !c->nrm || !c->u || !c->phi || !c->fa || !c->fb || !c->tw1 || !c->tw2)
        return set_error(ZM_ERR_INVALID, "double-word derivative: missing buffer");
    const Geom &G = c->geom;
    const DfGeo g = make_geo(c);
    cudaEvent_t ev = nullptr;
    prof_begin(c, ZM_K_GEOMETRY, &ev);
    geometry_df<<<(G.N + kTpb - 1) / kTpb, kTpb, 0, c->stream>>>(g, F2(y), F2(c->q), F2(c->nrm));
    prof_end(c, ZM_K_GEOMETRY, ev);
    int rc = cuda_check(cudaGetLastError(), "double-word geometry launch");
    if (rc) return rc;

    const int l1 = ilog2(G.n1), l2 = ilog2(G.n2);
    const int ra = lrows_for(l2, G.n1), rb = lrows_for(l1, G.n2);
    const size_t sa = (size_t)phys_host(G.n2 << ra) * sizeof(ulonglong2);
    const size_t sb = (size_t)phys_host(G.n1 << rb) * sizeof(ulonglong2);
    const float scale = (float)(-0.5 / ((double)G.n1 * (double)G.n2));
    prof_begin(c, ZM_K_FFT, &ev);
    rc = with_log2(l2, [&](auto lc) {
        return FftLaunch<decltype(lc)::value>::a(G.n1, ra, sa, c->stream, F2(y) + 3 * (size_t)G.N, U2(c->tw2),
                                                 U2(c->fa));
    });
    if (!rc) rc = with_log2(l1, [&](auto lc) {
        return FftLaunch<decltype(lc)::value>::b(G.n2, rb, sb, c->stream, split(1.0 / G.L1), split(1.0 / G.L2),
                                                 U2(c->fa), U2(c->tw1), U2(c->fb));
    });
    if (!rc) rc = with_log2(l2, [&](auto lc) {
        return FftLaunch<decltype(lc)::value>::c(G.n1, ra, sa, c->stream, scale, U2(c->fb), U2(c->tw2), F2(c->nrm),
                                                 F2(c->q), F2(c->u), F2(c->phi));
    });
    prof_end(c, ZM_K_FFT, ev);
    c->prof.acc.launches[ZM_K_FFT] += 2;  // three kernels per Riesz evaluation
    if (rc) return rc;
    return cuda_check(cudaGetLastError(), "double-word Riesz launch");
}

int df_vorticity(zm_ctx *c, const double *y, double *wdot_out, const double *y0, double *yout, double dt,
                 double ca, double cb, int mode)
{
    if (!y || !c->phi || !c->u || (mode == 0 && !wdot_out) || (mode == 1 && (!y0 || !yout)))
        return set_error(ZM_ERR_INVALID, "double-word vorticity pass: missing buffer");
    const DfGeo g = make_geo(c);
    const int grid = (c->geom.N + kTpb - 1) / kTpb;
    cudaEvent_t ev = nullptr;
    prof_begin(c, ZM_K_VORT, &ev);
    const bool visc = (c->mu != 0.0);
#define ZM_VDF(V, M)                                                                                      \
    vorticity_df<V, M><<<grid, kTpb, 0, c->stream>>>(g, F2(c->phi), F2(y), F2(c->u), split(dt), split(ca), \
                                                     split(cb), F2(y0), F2(yout), F2(wdot_out))
    if (mode == 0) {
        if (visc) ZM_VDF(true, 0); else ZM_VDF(false, 0);
    } else {
        if (visc) ZM_VDF(true, 1); else ZM_VDF(false, 1);
    }
#undef ZM_VDF
    prof_end(c, ZM_K_VORT, ev);
    return cuda_check(cudaGetLastError(), "double-word vorticity launch");
}

int df_convert(zm_ctx *c, const double *src, double *dst, size_t count, int state, int to_df)
{
    if (!src || !dst) return set_error(ZM_ERR_INVALID, "double-word conversion: missing buffer");
    const Geom &G = c->geom;
    const int l2 = ilog2(G.n2);
    const int grid = (int)std::min<size_t>((count + kTpb - 1) / kTpb, 4 * 152);
    if (to_df)
        to_df_kernel<<<grid, kTpb, 0, c->stream>>>(l2, G.n2, G.N, count, G.dx1, G.dx2, state, src, F2(dst));
    else
        from_df_kernel<<<grid, kTpb, 0, c->stream>>>(l2, G.n2, G.N, count, G.dx1, G.dx2, state, F2(src), dst);
    return cuda_check(cudaGetLastError(), "double-word conversion launch");
}

int df_check_finite(zm_ctx *c, const double *y, size_t nvalues, int *dev_flag)
{
    int rc = cuda_check(cudaMemsetAsync(dev_flag, 0, sizeof(int), c->stream), "finite flag clear");
    if (rc) return rc;
    finite_f32_kernel<<<4 * 152, kTpb, 0, c->stream>>>(2 * nvalues, reinterpret_cast<const float *>(y), dev_flag);
    return cuda_check(cudaGetLastError(), "finite check launch");
}

}  // namespace zm
