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

#include "zm_dffft.cuh"

namespace zm {
namespace {

constexpr int kTpb = 256;

struct DfGeo {
    int n1, n2, l2;  // l2 = log2 n2 when n2 is a power of two
    int N;
    unsigned long long divm;  // floor(2^40 / n2) + 1: p / n2 = (p divm) >> 40 for p < 2^26
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

// (a + d) mod n for |d| <= 2 < n
__device__ __forceinline__ int wrap(int a, int d, int n)
{
    const int b = a + d;
    return b < 0 ? b + n : (b >= n ? b - n : b);
}

// Mesh indices of node p; kP2: both sides are powers of two (shift and mask), else a
// multiply-shift division exact for p < 2^26 and n2 <= 2^13.
template <bool kP2>
__device__ __forceinline__ void node_ij(int p, const DfGeo &g, int &i, int &j)
{
    if (kP2) {
        i = p >> g.l2;
        j = p & (g.n2 - 1);
    } else {
        i = (int)(((unsigned long long)p * g.divm) >> 40);
        j = p - i * g.n2;
    }
}

template <bool kP2>
__device__ __forceinline__ Nb nb_axis0(int i, int j, const DfGeo &g)
{
    if (kP2) {
        const int m = g.n1 - 1;
        return Nb{(((i - 2) & m) << g.l2) + j, (((i - 1) & m) << g.l2) + j, (((i + 1) & m) << g.l2) + j,
                  (((i + 2) & m) << g.l2) + j};
    }
    return Nb{wrap(i, -2, g.n1) * g.n2 + j, wrap(i, -1, g.n1) * g.n2 + j, wrap(i, 1, g.n1) * g.n2 + j,
              wrap(i, 2, g.n1) * g.n2 + j};
}

template <bool kP2>
__device__ __forceinline__ Nb nb_axis1(int i, int j, const DfGeo &g)
{
    if (kP2) {
        const int m = g.n2 - 1;
        const int r = i << g.l2;
        return Nb{r + ((j - 2) & m), r + ((j - 1) & m), r + ((j + 1) & m), r + ((j + 2) & m)};
    }
    const int r = i * g.n2;
    return Nb{r + wrap(j, -2, g.n2), r + wrap(j, -1, g.n2), r + wrap(j, 1, g.n2), r + wrap(j, 2, g.n2)};
}

// Checked build: every neighbour index lies in the mesh.
__device__ __forceinline__ bool nb_ok(const Nb &n, int N)
{
    return ZM_IDX_OK(n.m2, N) && ZM_IDX_OK(n.m1, N) && ZM_IDX_OK(n.p1, N) && ZM_IDX_OK(n.p2, N);
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
template <bool kP2>
__global__ void __launch_bounds__(kTpb)
    geometry_df(DfGeo g, const float2 *__restrict__ y, float2 *__restrict__ q, float2 *__restrict__ nrm)
{
    const int p = blockIdx.x * kTpb + threadIdx.x;
    if (p >= g.N) return;
    int i, j;
    node_ij<kP2>(p, g, i, j);
    const int N = g.N;
    const Nb na = nb_axis0<kP2>(i, j, g), nb = nb_axis1<kP2>(i, j, g);
    if (!nb_ok(na, N) || !nb_ok(nb, N)) return;  // checked build only
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
template <bool kVisc, int kMode, bool kP2>
__global__ void __launch_bounds__(kTpb)
    vorticity_df(DfGeo g, const float2 *__restrict__ phi, const float2 *__restrict__ y,
                 const float2 *__restrict__ u, Dc dt, Dc ca, Dc cb, const float2 *y0, float2 *yout,
                 float2 *__restrict__ wdot)
{
    const int p = blockIdx.x * kTpb + threadIdx.x;
    if (p >= g.N) return;
    int i, j;
    node_ij<kP2>(p, g, i, j);
    const int N = g.N;
    const Nb na = nb_axis0<kP2>(i, j, g), nb = nb_axis1<kP2>(i, j, g);
    if (!nb_ok(na, N) || !nb_ok(nb, N)) return;  // checked build only
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

// pass A: rows i (length n2 = 2^L) of c = w1 + i w2; forward; write out[j][i] (transposed).
template <int L>
__global__ void __launch_bounds__(threads_for(L), minb_for(L))
    pass_a_df(int n1, int lr, const float2 *__restrict__ w, const ulonglong2 *__restrict__ tw2,
              ulonglong2 *__restrict__ out)
{
    extern __shared__ ulonglong2 sx[];
    const int rows = 1 << lr;
    const int i0 = blockIdx.x * rows;
    if (!ZM_IDX_OK(i0 + rows - 1, n1)) return;  // checked build: the CTA's rows exist
    const size_t N = (size_t)n1 << L;
    const float2 *w1 = w + ((size_t)i0 << L), *w2 = w1 + N;
    auto ldg = [&](int row, int i) { return ld2(c2_pack(w1[(row << L) + i], w2[(row << L) + i])); };
    dif_seq<L, 0, nc_of(L) - 1>(sx, tw2, rows, -1, ldg);
    for (int e = threadIdx.x; e < (rows << L); e += blockDim.x) {
        const int j = e >> lr, r = e & (rows - 1);
        out[(size_t)j * n1 + i0 + r] = sx[phys((r << L) + bitrev(j, L))];
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
    if (!ZM_IDX_OK(j0 + rows - 1, n2)) return;  // checked build: the CTA's columns exist
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
    pass_c_df(int n1, int lr, Dc scale, const ulonglong2 *__restrict__ in,
              const ulonglong2 *__restrict__ tw2, const float2 *__restrict__ nrm,
              const float2 *__restrict__ q, float2 *__restrict__ u, float2 *__restrict__ phi)
{
    extern __shared__ ulonglong2 sx[];
    const int rows = 1 << lr;
    const int i0 = blockIdx.x * rows;
    if (!ZM_IDX_OK(i0 + rows - 1, n1)) return;  // checked build: the CTA's rows exist
    const size_t N = (size_t)n1 << L;
    const size_t o = (size_t)i0 << L;
    const ulonglong2 *src = in + o;
    auto ldg = [&](int row, int i) { return ld2(src[(row << L) + i]); };
    dif_seq<L, 0, nc_of(L) - 1>(sx, tw2, rows, +1, ldg);
#pragma unroll 4
    for (int e = threadIdx.x; e < (rows << L); e += blockDim.x) {
        const int r = e >> L, j = e & ((1 << L) - 1);
        const size_t p = o + e;
        // scale = -1/(2 n1 n2) as a double word (a power of two only when both sides are)
        const df s = mul(c2_re(ld2(sx[phys((r << L) + bitrev(j, L))])), dc(scale));
        const df ux = mul(s, ldf(nrm, p)), uy = mul(s, ldf(nrm, N + p)), uz = mul(s, ldf(nrm, 2 * N + p));
        u[p] = to_f2(ux);
        u[N + p] = to_f2(uy);
        u[2 * N + p] = to_f2(uz);
        const df k2 = add(add(sqr(ux), sqr(uy)), sqr(uz));
        phi[p] = to_f2(add(ldf(q, p), scale2(k2, 0.5f)));
    }
}

// ---- Hermitian inverse (both sides powers of two) ------------------------------------------------
// The spectrum of the real field s is Hermitian, S(-k) = conj S(k), and with Q = (m1 - i m2) P
// (P the spectrum of w1 + i w2) it is S(k) = (Q(k) + conj Q(-k)) / 2, so only the columns
// k2 = 0 .. n2/2 need the inverse along alpha1, and each row then holds a Hermitian sequence
// whose real inverse of length n2 is one complex inverse of length n2/2 (the even and odd
// samples as real and imaginary parts).  The Nyquist column k2 = n2/2 has a zero multiplier.
// This halves the inverse transforms against the full complex inverse of the passes above.
//
// Pass B_h: a CTA takes rows/2 column pairs (q, n2 - q), q = q0 .. q0 + rows/2 - 1, the pair
// q = 0 being (0, n2/2): columns q in local rows 0 .. rows/2 - 1, their mirrors in the rest.  It
// transforms all of them forward, forms 2 S(., q) = Q(., q) + conj Q(-., mirror) in the local
// row of q, transforms those rows back and writes G(i, q) = 2 x (the alpha1 inverse of S) to
// out[i][q], n2/2 columns.
__device__ __forceinline__ C2 conj2(C2 a) { return C2{a.h ^ kSign1, a.l ^ kSign1}; }

template <int L>
__global__ void __launch_bounds__(threads_for(L), minb_for(L))
    pass_b_h(int n2, int lr, Dc invL1, Dc invL2, const ulonglong2 *__restrict__ in,
             const ulonglong2 *__restrict__ tw1, ulonglong2 *__restrict__ out)
{
    extern __shared__ ulonglong2 sx[];
    constexpr int n1 = 1 << L;
    const int rows = 1 << lr, hr = rows >> 1;
    const int q0 = blockIdx.x * hr;
    if (!ZM_IDX_OK(q0 + hr - 1, n2 / 2)) return;  // checked build: the CTA's pairs exist
    auto col = [&](int row) {
        const int q = q0 + (row < hr ? row : row - hr);
        return row < hr ? q : (q == 0 ? n2 / 2 : n2 - q);
    };
    auto ldg = [&](int row, int i) { return ld2(in[(size_t)col(row) * n1 + i]); };
    dif_seq<L, 0, nc_of(L) - 1>(sx, tw1, rows, -1, ldg);
    // 2 S at frequencies k1 and -k1 of column q from Q of column q and of its mirror
    for (int e = threadIdx.x; e < hr * (n1 / 2 + 1); e += blockDim.x) {
        const int t = e / (n1 / 2 + 1), k1 = e - t * (n1 / 2 + 1);
        const int km = (n1 - k1) & (n1 - 1);
        const int q = q0 + t, cm = (q == 0) ? 0 : n2 - q;  // the mirror column of q
        const int ra = t << L, rm = ((q == 0 ? t : hr + t) << L);
        const int pk = bitrev(k1, L), pkm = bitrev(km, L);
        const C2 qa = cmul2(ld2(sx[phys(ra + pk)]), riesz_mult(k1, q, n1, n2, invL1, invL2));
        const C2 qam = cmul2(ld2(sx[phys(ra + pkm)]), riesz_mult(km, q, n1, n2, invL1, invL2));
        const C2 qb = cmul2(ld2(sx[phys(rm + pk)]), riesz_mult(k1, cm, n1, n2, invL1, invL2));
        const C2 qbm = cmul2(ld2(sx[phys(rm + pkm)]), riesz_mult(km, cm, n1, n2, invL1, invL2));
        const C2 s0 = cadd2(qa, conj2(qbm)), s1 = cadd2(qam, conj2(qb));
        sx[phys(ra + pk)] = st2(s0);
        if (km != k1) sx[phys(ra + pkm)] = st2(s1);
    }
    __syncthreads();
    dit_seq<L, nc_of(L) - 1>(sx, tw1, hr, +1);
    for (int e = threadIdx.x; e < (hr << L); e += blockDim.x) {
        const int i = e >> (lr - 1), t = e & (hr - 1);
        out[(size_t)i * (n2 / 2) + q0 + t] = sx[phys((t << L) + i)];
    }
}

// Pass C_h: rows i of G (length M = n2/2 = 2^L); the real inverse of length n2 as the complex
// inverse of Z[k] = (G[k] + conj G[M - k]) + i W_n2^(-k) (G[k] - conj G[M - k]) (G[M] = 0), whose
// output m holds s[2m] + i s[2m + 1]; then u = -s/2 N and Phi = q + |u|^2 / 2.  twn: half table
// of W_n2, twm: of W_M.  scale = -1 / (4 n1 n2) (the 1/2 of S and of u, the 1/(n1 n2) of the
// inverse).
template <int L>
__global__ void __launch_bounds__(threads_for(L), minb_for(L))
    pass_c_h(int n1, int lr, Dc scale, const ulonglong2 *__restrict__ in, const ulonglong2 *__restrict__ twm,
             const ulonglong2 *__restrict__ twn, const float2 *__restrict__ nrm, const float2 *__restrict__ q,
             float2 *__restrict__ u, float2 *__restrict__ phi)
{
    extern __shared__ ulonglong2 sx[];
    constexpr int M = 1 << L, n2 = 2 * M;
    const int rows = 1 << lr;
    const int i0 = blockIdx.x * rows;
    if (!ZM_IDX_OK(i0 + rows - 1, n1)) return;  // checked build: the CTA's rows exist
    const size_t N = (size_t)n1 * n2;
    const ulonglong2 *src = in + (size_t)i0 * M;
    auto ldz = [&](int row, int k) {
        const C2 g = ld2(src[row * M + k]);
        const C2 gm = k ? conj2(ld2(src[row * M + M - k])) : C2{0ull, 0ull};
        const C2 a = cadd2(g, gm), b = csub2(g, gm);
        return cadd2(a, cmul_i2(k ? cmul2(b, tw_get(twn, k, M, +1)) : b, +1));
    };
    dif_seq<L, 0, nc_of(L) - 1>(sx, twm, rows, +1, ldz);
    const df sc = dc(scale);
    for (int e = threadIdx.x; e < rows * M; e += blockDim.x) {
        const int r = e >> L, m = e & (M - 1);
        const C2 z = ld2(sx[phys((r << L) + bitrev(m, L))]);
        const size_t p0 = (size_t)(i0 + r) * n2 + 2 * m;
        const df s2[2] = {mul(df{lane0(z.h), lane0(z.l)}, sc), mul(df{lane1(z.h), lane1(z.l)}, sc)};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const size_t p = p0 + h;
            const df ux = mul(s2[h], ldf(nrm, p)), uy = mul(s2[h], ldf(nrm, N + p)), uz = mul(s2[h], ldf(nrm, 2 * N + p));
            u[p] = to_f2(ux);
            u[N + p] = to_f2(uy);
            u[2 * N + p] = to_f2(uz);
            const df k2 = add(add(sqr(ux), sqr(uy)), sqr(uz));
            phi[p] = to_f2(add(ldf(q, p), scale2(k2, 0.5f)));
        }
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
__global__ void to_df_kernel(int n2, size_t N, size_t count, double dx1, double dx2, int state,
                             const double *src, float2 *dst)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < count;
         k += (size_t)gridDim.x * blockDim.x) {
        double v = src[k];
        if (state && k < 2 * N) {
            const size_t p = k < N ? k : k - N;
            v -= k < N ? (double)(p / n2) * dx1 : (double)(p % n2) * dx2;
        }
        const float hi = __double2float_rn(v);
        dst[k] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
}

__global__ void from_df_kernel(int n2, size_t N, size_t count, double dx1, double dx2, int state,
                               const float2 *src, double *dst)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < count;
         k += (size_t)gridDim.x * blockDim.x) {
        const float2 f = src[k];
        double v = (double)f.x + (double)f.y;
        if (state && k < 2 * N) {
            const size_t p = k < N ? k : k - N;
            v += k < N ? (double)(p / n2) * dx1 : (double)(p % n2) * dx2;
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

// log2 of the rows per CTA of an FFT pass over rows of length 2^l: a power of two dividing the
// number of rows the pass has (`avail`), at most elems_for(l) / 2^l.
int lrows_for(int l, int avail)
{
    const int cap = std::max(1, std::min(elems_for(l) >> l, avail & -avail));
    int r = 0;
    while ((2 << r) <= cap) ++r;
    return r;
}

// Fewer rows per CTA (down to one) while the pass would have fewer than `floor` CTAs: small
// meshes then fill the GPU with more, smaller CTAs (pass_threads gives each one thread per group
// of 16 values).  Measured A/B on GB300 (FFT ms per evaluation; floors 0 / 304 / 456 / 608):
// 512^2 0.0587 / 0.0444 / 0.0449 / 0.0446, 1024^2 0.0969 / 0.0972 / 0.0976 / 0.1015; at 2048^2
// only the Hermitian pass C gains (floor 608: 512 -> 1024 CTAs, 0.310 -> 0.302 ms).
#ifndef ZM_DF_MINGRID
#define ZM_DF_MINGRID 304  // two CTAs per SM of the 152
#endif
#ifndef ZM_DF_MINGRID_CH
#define ZM_DF_MINGRID_CH 608  // the Hermitian pass C: four per SM
#endif
int lrows_grid(int l, int avail, int floor = ZM_DF_MINGRID)
{
    int r = lrows_for(l, avail);
    while (r > 0 && (avail >> r) < floor) --r;
    return r;
}

// Threads per CTA of a pass over 2^lr rows of length 2^L: one per group of 16 values, at most
// threads_for(L) (the launch bound).
int pass_threads(int L, int lr) { return std::max(32, std::min(threads_for(L), ((1 << L) << lr) / 16)); }

// The same for rows of length L = R 2^A (not a power of two): rows * L <= kFftElems.
int lrows_mix(int L, int avail)
{
    const int cap = std::max(1, std::min(kFftElems / L, avail & -avail));
    int r = 0;
    while ((2 << r) <= cap) ++r;
    return r;
}

DfGeo make_geo(const zm_ctx *c)
{
    const Geom &G = c->geom;
    DfGeo g;
    g.n1 = G.n1;
    g.n2 = G.n2;
    g.l2 = ilog2(G.n2);
    g.N = G.N;
    g.divm = (1ull << 40) / (unsigned long long)G.n2 + 1;
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
    static int a(int n1, int lr, size_t smem, cudaStream_t s, const float2 *w, const ulonglong2 *tw2, ulonglong2 *out)
    {
        int rc = smem_attr((const void *)pass_a_df<L>, smem);
        if (rc) return rc;
        pass_a_df<L><<<n1 >> lr, pass_threads(L, lr), smem, s>>>(n1, lr, w, tw2, out);
        return cuda_check(cudaGetLastError(), "double-word FFT pass A launch");
    }
    static int b(int n2, int lr, size_t smem, cudaStream_t s, Dc invL1, Dc invL2, const ulonglong2 *in,
                 const ulonglong2 *tw1, ulonglong2 *out)
    {
        int rc = smem_attr((const void *)pass_b_df<L>, smem);
        if (rc) return rc;
        pass_b_df<L><<<n2 >> lr, pass_threads(L, lr), smem, s>>>(n2, lr, invL1, invL2, in, tw1, out);
        return cuda_check(cudaGetLastError(), "double-word FFT pass B launch");
    }
    static int b_h(int n2, int lr, size_t smem, cudaStream_t s, Dc invL1, Dc invL2, const ulonglong2 *in,
                   const ulonglong2 *tw1, ulonglong2 *out)
    {
        int rc = smem_attr((const void *)pass_b_h<L>, smem);
        if (rc) return rc;
        pass_b_h<L><<<n2 >> lr, pass_threads(L, lr), smem, s>>>(n2, lr, invL1, invL2, in, tw1, out);
        return cuda_check(cudaGetLastError(), "double-word FFT pass B (Hermitian) launch");
    }
    static int c_h(int n1, int lr, size_t smem, cudaStream_t s, Dc scale, const ulonglong2 *in,
                   const ulonglong2 *twm, const ulonglong2 *twn, const float2 *nrm, const float2 *q, float2 *u,
                   float2 *phi)
    {
        int rc = smem_attr((const void *)pass_c_h<L>, smem);
        if (rc) return rc;
        pass_c_h<L><<<n1 >> lr, pass_threads(L, lr), smem, s>>>(n1, lr, scale, in, twm, twn, nrm, q, u, phi);
        return cuda_check(cudaGetLastError(), "double-word FFT pass C (Hermitian) launch");
    }
    static int c(int n1, int lr, size_t smem, cudaStream_t s, Dc scale, const ulonglong2 *in,
                 const ulonglong2 *tw2, const float2 *nrm, const float2 *q, float2 *u, float2 *phi)
    {
        int rc = smem_attr((const void *)pass_c_df<L>, smem);
        if (rc) return rc;
        pass_c_df<L><<<n1 >> lr, pass_threads(L, lr), smem, s>>>(n1, lr, scale, in, tw2, nrm, q, u, phi);
        return cuda_check(cudaGetLastError(), "double-word FFT pass C launch");
    }
};

// One side of the double-word transform: L = R 2^A.
struct DfSide {
    int L, R, A;
};

DfSide df_side(int L)
{
    const int M = L & -L;
    return DfSide{L, L / M, ilog2(M)};
}

}  // namespace

// Meshes whose double-word Riesz pass uses the Hermitian inverse: both sides powers of two,
// n2 >= 16 (the half-length row transform has at least 8 values) and columns of 2048.  Measured
// on GB300 against the full inverse (FFT ms per evaluation): 512^2 0.0634 vs 0.0587, 1024^2
// 0.0961 vs 0.0969, 2048^2 0.3098 vs 0.3311; at 4096^2 the column pair of pass B_h needs 139 KB
// of shared memory (one CTA per SM) and gained nothing.  Below 2048 the unfused middle of pass
// B_h (the fused last-forward / multiplier / first-inverse group of pass B is lost) outweighs
// the halved inverse.
#ifndef ZM_DF_HERM
#define ZM_DF_HERM 1  // 0: the full complex inverse everywhere
#endif
bool herm_sides(int n1, int n2)
{
    return ZM_DF_HERM && pow2_side(n1) && pow2_side(n2) && n2 >= 16 && n1 == 2048;
}

bool df_side_ok(int L)
{
    if (L < 8 || L > 8192) return false;
    const DfSide s = df_side(L);
    if (s.R == 1) return L <= 4096;
    if (s.A < 3 || s.A > 12) return false;
    switch (s.R) {
#define ZM_CASE(r) case r:
        ZM_DF_RADICES(ZM_CASE)
#undef ZM_CASE
        return true;
    default: return false;
    }
}

int df_setup(zm_ctx *c)
{
    const Geom &g = c->geom;
    const size_t N = g.N;
    const DfSide s1 = df_side(g.n1), s2 = df_side(g.n2);
    const int m1 = 1 << s1.A, m2 = 1 << s2.A;
    if (cudaMalloc(&c->fa, N * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&c->fb, N * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&c->tw1, (m1 / 2) * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&c->tw2, (m2 / 2) * sizeof(double2)) != cudaSuccess ||
        (s1.R > 1 && cudaMalloc(&c->twl1, (g.n1 / 2) * sizeof(double2)) != cudaSuccess) ||
        (s2.R > 1 && cudaMalloc(&c->twl2, (g.n2 / 2) * sizeof(double2)) != cudaSuccess)) {
        cudaGetLastError();
        return set_error(ZM_ERR_NOMEM, "df_setup: device allocation failed");
    }
    twiddle_df_kernel<<<(m1 / 2 + 255) / 256, 256>>>(m1, reinterpret_cast<float4 *>(c->tw1));
    twiddle_df_kernel<<<(m2 / 2 + 255) / 256, 256>>>(m2, reinterpret_cast<float4 *>(c->tw2));
    if (c->twl1) twiddle_df_kernel<<<(g.n1 / 2 + 255) / 256, 256>>>(g.n1, reinterpret_cast<float4 *>(c->twl1));
    if (c->twl2) twiddle_df_kernel<<<(g.n2 / 2 + 255) / 256, 256>>>(g.n2, reinterpret_cast<float4 *>(c->twl2));
    if (herm_sides(g.n1, g.n2)) {  // the Hermitian inverse's half-length row transform
        if (cudaMalloc(&c->twh, (g.n2 / 4) * sizeof(double2)) != cudaSuccess) {
            cudaGetLastError();
            return set_error(ZM_ERR_NOMEM, "df_setup: device allocation failed");
        }
        twiddle_df_kernel<<<(g.n2 / 4 + 255) / 256, 256>>>(g.n2 / 2, reinterpret_cast<float4 *>(c->twh));
    }
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
    const int grid = (G.N + kTpb - 1) / kTpb;
    if (pow2_side(G.n1) && pow2_side(G.n2))  // shift-and-mask indexing needs both sides
        geometry_df<true><<<grid, kTpb, 0, c->stream>>>(g, F2(y), F2(c->q), F2(c->nrm));
    else
        geometry_df<false><<<grid, kTpb, 0, c->stream>>>(g, F2(y), F2(c->q), F2(c->nrm));
    prof_end(c, ZM_K_GEOMETRY, ev);
    int rc = cuda_check(cudaGetLastError(), "double-word geometry launch");
    if (rc) return rc;

    const DfSide s1 = df_side(G.n1), s2 = df_side(G.n2);
    if ((s1.R > 1 && !c->twl1) || (s2.R > 1 && !c->twl2))
        return set_error(ZM_ERR_INVALID, "double-word derivative: missing twiddle table");
    const int ra = s2.R > 1 ? lrows_mix(G.n2, G.n1) : lrows_grid(s2.A, G.n1);
    const int rb = s1.R > 1 ? lrows_mix(G.n1, G.n2) : lrows_grid(s1.A, G.n2);
    if (G.n1 % (1 << ra) || G.n2 % (1 << rb))
        return set_error(ZM_ERR_INVALID, "double-word derivative: rows per CTA do not divide the side");
    const size_t sa = (size_t)phys_host(G.n2 << ra) * sizeof(ulonglong2);
    const size_t sb = (size_t)phys_host(G.n1 << rb) * sizeof(ulonglong2);
    const double scale = -0.5 / ((double)G.n1 * (double)G.n2);
    const float2 *w = F2(y) + 3 * (size_t)G.N;
    const Dc iL1 = split(1.0 / G.L1), iL2 = split(1.0 / G.L2);
    prof_begin(c, ZM_K_FFT, &ev);
    rc = with_log2(s2.A, [&](auto lc) {
        constexpr int A = decltype(lc)::value;
        return s2.R > 1 ? df_mix_pass_a(A, G.n1, s2.R, ra, sa, c->stream, w, U2(c->tw2), U2(c->twl2), U2(c->fa))
                        : FftLaunch<A>::a(G.n1, ra, sa, c->stream, w, U2(c->tw2), U2(c->fa));
    });
    if (c->twh) {  // Hermitian inverse: half the columns back along alpha1, then real rows
        const int rbh = std::max(1, lrows_grid(s1.A, G.n2));  // a column pair: rows >= 2
        const int rch = lrows_grid(s2.A - 1, G.n1, ZM_DF_MINGRID_CH);
        const size_t sbh = (size_t)phys_host(G.n1 << rbh) * sizeof(ulonglong2);
        const size_t sch = (size_t)phys_host((G.n2 / 2) << rch) * sizeof(ulonglong2);
        if (!rc) rc = with_log2(s1.A, [&](auto lc) {
            return FftLaunch<decltype(lc)::value>::b_h(G.n2, rbh, sbh, c->stream, iL1, iL2, U2(c->fa), U2(c->tw1),
                                                       U2(c->fb));
        });
        if (!rc) rc = with_log2(s2.A - 1, [&](auto lc) {
            return FftLaunch<decltype(lc)::value>::c_h(G.n1, rch, sch, c->stream, split(scale / 2), U2(c->fb),
                                                       U2(c->twh), U2(c->tw2), F2(c->nrm), F2(c->q), F2(c->u),
                                                       F2(c->phi));
        });
    } else {
        if (!rc) rc = with_log2(s1.A, [&](auto lc) {
            constexpr int A = decltype(lc)::value;
            return s1.R > 1 ? df_mix_pass_b(A, G.n2, s1.R, rb, sb, c->stream, 1.0 / G.L1, 1.0 / G.L2, U2(c->fa),
                                            U2(c->tw1), U2(c->twl1), U2(c->fb))
                            : FftLaunch<A>::b(G.n2, rb, sb, c->stream, iL1, iL2, U2(c->fa), U2(c->tw1), U2(c->fb));
        });
        if (!rc) rc = with_log2(s2.A, [&](auto lc) {
            constexpr int A = decltype(lc)::value;
            return s2.R > 1 ? df_mix_pass_c(A, G.n1, s2.R, ra, sa, c->stream, scale, U2(c->fb), U2(c->tw2),
                                            U2(c->twl2), F2(c->nrm), F2(c->q), F2(c->u), F2(c->phi))
                            : FftLaunch<A>::c(G.n1, ra, sa, c->stream, split(scale), U2(c->fb), U2(c->tw2),
                                              F2(c->nrm), F2(c->q), F2(c->u), F2(c->phi));
        });
    }
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
    const bool visc = (c->mu != 0.0), p2 = pow2_side(c->geom.n1) && pow2_side(c->geom.n2);
#define ZM_VDF(V, M, P)                                                                                      \
    vorticity_df<V, M, P><<<grid, kTpb, 0, c->stream>>>(g, F2(c->phi), F2(y), F2(c->u), split(dt), split(ca), \
                                                        split(cb), F2(y0), F2(yout), F2(wdot_out))
    if (p2) {
        if (mode == 0) {
            if (visc) ZM_VDF(true, 0, true); else ZM_VDF(false, 0, true);
        } else {
            if (visc) ZM_VDF(true, 1, true); else ZM_VDF(false, 1, true);
        }
    } else {
        if (mode == 0) {
            if (visc) ZM_VDF(true, 0, false); else ZM_VDF(false, 0, false);
        } else {
            if (visc) ZM_VDF(true, 1, false); else ZM_VDF(false, 1, false);
        }
    }
#undef ZM_VDF
    prof_end(c, ZM_K_VORT, ev);
    return cuda_check(cudaGetLastError(), "double-word vorticity launch");
}

int df_convert(zm_ctx *c, const double *src, double *dst, size_t count, int state, int to_df)
{
    if (!src || !dst) return set_error(ZM_ERR_INVALID, "double-word conversion: missing buffer");
    const Geom &G = c->geom;
    const int grid = (int)std::min<size_t>((count + kTpb - 1) / kTpb, 4 * 152);
    if (to_df)
        to_df_kernel<<<grid, kTpb, 0, c->stream>>>(G.n2, G.N, count, G.dx1, G.dx2, state, src, F2(dst));
    else
        from_df_kernel<<<grid, kTpb, 0, c->stream>>>(G.n2, G.N, count, G.dx1, G.dx2, state, F2(src), dst);
    return cuda_check(cudaGetLastError(), "double-word conversion launch");
}

int df_check_finite(zm_ctx *c, const double *y, size_t nvalues, int *dev_flag)
{
    int rc = cuda_check(cudaMemsetAsync(dev_flag, 0, sizeof(int), c->stream), "finite flag clear");
    if (rc) return rc;
    finite_f32_kernel<<<4 * 152, kTpb, 0, c->stream>>>(2 * nvalues, reinterpret_cast<const float *>(y), dev_flag);
    return cuda_check(cudaGetLastError(), "finite check launch");
}

ZM_BOUNDS_READER(bounds_lowdf)

}  // namespace zm
