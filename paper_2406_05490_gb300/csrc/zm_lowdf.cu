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

#include "zm_df64.cuh"
#include "zm_internal.cuh"

namespace zm {
namespace {

using namespace dw;

constexpr int kTpb = 256;
constexpr int kFftTpb = 256;

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
__device__ __forceinline__ df ldf(const float2 *__restrict__ f, size_t k) { return from_f2(f[k]); }

struct DfGeo {
    int n1, n2, l2;
    int N;
    Dc i12a, i12b;    // 1 / (12 dx1), 1 / (12 dx2)
    Dc i12a2, i12b2;  // 1 / (12 dx1^2), 1 / (12 dx2^2)
    Dc grav;          // g
    Dc m2a;           // -2 A
    Dc mu;
};

// Periodic 4th-order first difference along one axis at node p: the four neighbours are
// p + k * stride for k = -2, -1, 1, 2 after wrapping the axis index c0 + k into [0, n).
struct Nb {
    size_t m2, m1, p1, p2;
};

__device__ __forceinline__ Nb nb_axis0(int i, int j, const DfGeo &g)
{
    const int m = g.n1 - 1;
    return Nb{((size_t)((i - 2) & m) << g.l2) + j, ((size_t)((i - 1) & m) << g.l2) + j,
              ((size_t)((i + 1) & m) << g.l2) + j, ((size_t)((i + 2) & m) << g.l2) + j};
}

__device__ __forceinline__ Nb nb_axis1(int i, int j, const DfGeo &g)
{
    const int m = g.n2 - 1;
    const size_t r = (size_t)i << g.l2;
    return Nb{r + ((j - 2) & m), r + ((j - 1) & m), r + ((j + 1) & m), r + ((j + 2) & m)};
}

// ((f-2 - f+2) + 8 (f+1 - f-1)) / (12 dx)
__device__ __forceinline__ df diff1_df(const float2 *__restrict__ f, const Nb &n, df inv12)
{
    const df a = sub(ldf(f, n.m2), ldf(f, n.p2));
    const df b = sub(ldf(f, n.p1), ldf(f, n.m1));
    return mul(add(a, scale2(b, 8.0f)), inv12);
}

// (16 (f-1 + f+1) - (f-2 + f+2) - 30 f0) / (12 dx^2), accurate sums: the three groups cancel
// to O(dx^2) of their size.
__device__ __forceinline__ df diff2_df(const float2 *__restrict__ f, const Nb &n, size_t p0, df inv12sq)
{
    const df s1 = add_acc(ldf(f, n.m1), ldf(f, n.p1));
    const df s2 = add_acc(ldf(f, n.m2), ldf(f, n.p2));
    const df t = sub_acc(sub_acc(scale2(s1, 16.0f), s2), mul_f(ldf(f, p0), 30.0f));
    return mul(t, inv12sq);
}

// Geometry pass: unit normal N = a1 x a2 / |a1 x a2| and q = g z3 + 1/8 w^T h^-1 w, using
// |a1 x a2|^2 = h11 h22 - h12^2 = det (Lagrange's identity) and 1/det = rsqrt(det)^2.
__global__ void __launch_bounds__(kTpb)
    geometry_df(DfGeo g, const float2 *__restrict__ y, float2 *__restrict__ q, float2 *__restrict__ nrm)
{
    const int p = blockIdx.x * kTpb + threadIdx.x;
    if (p >= g.N) return;
    const int i = p >> g.l2, j = p & (g.n2 - 1);
    const size_t N = g.N;
    const Nb na = nb_axis0(i, j, g), nb = nb_axis1(i, j, g);
    const df ia = dc(g.i12a), ib = dc(g.i12b);
    df a1[3], a2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a1[c] = diff1_df(y + c * N, na, ia);
        a2[c] = diff1_df(y + c * N, nb, ib);
    }
    a1[0] = add(from_f(1.0f), a1[0]);
    a2[1] = add(from_f(1.0f), a2[1]);
    const df nx = sub(mul(a1[1], a2[2]), mul(a1[2], a2[1]));
    const df ny = sub(mul(a1[2], a2[0]), mul(a1[0], a2[2]));
    const df nz = sub(mul(a1[0], a2[1]), mul(a1[1], a2[0]));
    const df det = add(add(sqr(nx), sqr(ny)), sqr(nz));
    const df rs = rsqrt(det);
    nrm[p] = to_f2(mul(nx, rs));
    nrm[N + p] = to_f2(mul(ny, rs));
    nrm[2 * N + p] = to_f2(mul(nz, rs));

    const df h11 = add(add(sqr(a1[0]), sqr(a1[1])), sqr(a1[2]));
    const df h22 = add(add(sqr(a2[0]), sqr(a2[1])), sqr(a2[2]));
    const df h12 = add(add(mul(a1[0], a2[0]), mul(a1[1], a2[1])), mul(a1[2], a2[2]));
    const df w1 = ldf(y, 3 * N + p), w2 = ldf(y, 4 * N + p);
    // h22 w1^2 - 2 h12 w1 w2 + h11 w2^2
    const df t = add(sub(mul(h22, sqr(w1)), scale2(mul(h12, mul(w1, w2)), 2.0f)), mul(h11, sqr(w2)));
    const df jump = scale2(mul(t, sqr(rs)), 0.125f);
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
    const size_t N = g.N;
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
// epilogue), on complex double words (float4) in shared memory.  Butterflies are radix-2^2:
// two radix-2 stages fused into one radix-4 step with three twiddle products instead of
// four, which keeps the bit-reversed order of plain radix-2 (one radix-2 stage when log2 L is
// odd).  Twiddles W_L^k = exp(-2 pi i k / L) come from a half table (k < L/2), the upper
// range by W_L^(k + L/2) = -W_L^k, conjugated for the inverse.

__device__ __forceinline__ int bitrev(int j, int logL) { return (int)(__brev((unsigned)j) >> (32 - logL)); }

__device__ __forceinline__ cdf tw_get(const float4 *__restrict__ tw, int k, int half, int sgn)
{
    const bool up = k >= half;
    float4 v = __ldg(tw + (up ? k - half : k));
    if (up) v = make_float4(-v.x, -v.y, -v.z, -v.w);
    if (sgn > 0) {
        v.z = -v.z;
        v.w = -v.w;
    }
    return ld_c(v);
}

// Decimation in frequency on `rows` rows of length L = 2^logL: natural order in, bit-reversed
// order out.  sgn = -1 forward, +1 inverse (unnormalised).
__device__ void dif_df(float4 *x, int rows, int logL, const float4 *__restrict__ tw, int sgn)
{
    const int L = 1 << logL, half = L >> 1, quarter = L >> 2;
    if (logL & 1) {
        for (int b = threadIdx.x; b < rows * half; b += blockDim.x) {
            const int row = b >> (logL - 1), pos = b & (half - 1);
            float4 *xr = x + (row << logL);
            const cdf u = ld_c(xr[pos]), v = ld_c(xr[pos + half]);
            const cdf d = csub(u, v);
            xr[pos] = st_c(cadd(u, v));
            xr[pos + half] = st_c(pos ? cmul(d, tw_get(tw, pos, half, sgn)) : d);
        }
        __syncthreads();
    }
    for (int h = (logL & 1) ? (L >> 3) : (L >> 2); h >= 1; h >>= 2) {
        const int lh = __ffs(h) - 1;
        const int step = half / (2 * h);  // W_{4h}^m = W_L^(m * step)
        for (int b = threadIdx.x; b < rows * quarter; b += blockDim.x) {
            const int row = b >> (logL - 2), idx = b & (quarter - 1);
            const int pos = idx & (h - 1);
            float4 *xr = x + (row << logL) + ((idx >> lh) << (lh + 2)) + pos;
            const cdf a0 = ld_c(xr[0]), a1 = ld_c(xr[h]), a2 = ld_c(xr[2 * h]), a3 = ld_c(xr[3 * h]);
            const cdf s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3);
            const cdf d13 = cmul_pm_i(csub(a1, a3), sgn);  // times W_{4h}^h = -+i
            const cdf X0 = cadd(s02, s13), X2 = csub(s02, s13);
            const cdf X1 = cadd(d02, d13), X3 = csub(d02, d13);
            xr[0] = st_c(X0);
            if (pos == 0) {
                xr[h] = st_c(X2);
                xr[2 * h] = st_c(X1);
                xr[3 * h] = st_c(X3);
            } else {
                xr[h] = st_c(cmul(X2, tw_get(tw, 2 * pos * step, half, sgn)));
                xr[2 * h] = st_c(cmul(X1, tw_get(tw, pos * step, half, sgn)));
                xr[3 * h] = st_c(cmul(X3, tw_get(tw, 3 * pos * step, half, sgn)));
            }
        }
        __syncthreads();
    }
}

// Decimation in time: bit-reversed order in, natural order out.
__device__ void dit_df(float4 *x, int rows, int logL, const float4 *__restrict__ tw, int sgn)
{
    const int L = 1 << logL, half = L >> 1, quarter = L >> 2;
    for (int h = 1; 4 * h <= L; h <<= 2) {
        const int lh = __ffs(h) - 1;
        const int step = half / (2 * h);
        for (int b = threadIdx.x; b < rows * quarter; b += blockDim.x) {
            const int row = b >> (logL - 2), idx = b & (quarter - 1);
            const int pos = idx & (h - 1);
            float4 *xr = x + (row << logL) + ((idx >> lh) << (lh + 2)) + pos;
            const cdf a0 = ld_c(xr[0]);
            cdf c1 = ld_c(xr[h]), c2 = ld_c(xr[2 * h]), c3 = ld_c(xr[3 * h]);
            if (pos) {
                c1 = cmul(c1, tw_get(tw, 2 * pos * step, half, sgn));
                c2 = cmul(c2, tw_get(tw, pos * step, half, sgn));
                c3 = cmul(c3, tw_get(tw, 3 * pos * step, half, sgn));
            }
            const cdf s01 = cadd(a0, c1), d01 = csub(a0, c1), s23 = cadd(c2, c3);
            const cdf d23 = cmul_pm_i(csub(c2, c3), sgn);
            xr[0] = st_c(cadd(s01, s23));
            xr[2 * h] = st_c(csub(s01, s23));
            xr[h] = st_c(cadd(d01, d23));
            xr[3 * h] = st_c(csub(d01, d23));
        }
        __syncthreads();
    }
    if (logL & 1) {
        for (int b = threadIdx.x; b < rows * half; b += blockDim.x) {
            const int row = b >> (logL - 1), pos = b & (half - 1);
            float4 *xr = x + (row << logL);
            const cdf u = ld_c(xr[pos]);
            cdf v = ld_c(xr[pos + half]);
            if (pos) v = cmul(v, tw_get(tw, pos, half, sgn));
            xr[pos] = st_c(cadd(u, v));
            xr[pos + half] = st_c(csub(u, v));
        }
        __syncthreads();
    }
}

// pass A: rows i (length n2) of c = w1 + i w2; forward; write out[j][i] (transposed).
__global__ void __launch_bounds__(kFftTpb)
    pass_a_df(int n1, int n2, int l2, int lr, const float2 *__restrict__ w,
              const float4 *__restrict__ tw2, float4 *__restrict__ out)
{
    extern __shared__ float4 sx[];
    const int rows = 1 << lr;
    const int i0 = blockIdx.x * rows;
    const size_t N = (size_t)n1 * n2;
    const size_t o = (size_t)i0 * n2;
    for (int e = threadIdx.x; e < (rows << l2); e += blockDim.x) {
        const float2 a = w[o + e], b = w[N + o + e];
        sx[e] = make_float4(a.x, a.y, b.x, b.y);
    }
    __syncthreads();
    dif_df(sx, rows, l2, tw2, -1);
    for (int e = threadIdx.x; e < (rows << l2); e += blockDim.x) {
        const int j = e >> lr, r = e & (rows - 1);
        out[(size_t)j * n1 + i0 + r] = sx[(r << l2) + bitrev(j, l2)];
    }
}

// pass B: rows j (length n1) of the transpose; forward; multiply by -(k2 + i k1)/|k| (zero at
// k = 0 and on the Nyquist row and column); inverse; write out[i][j].  k_l / |k| is formed from
// t_l = m_l / L_l (the 2 pi cancels).
__global__ void __launch_bounds__(kFftTpb)
    pass_b_df(int n1, int n2, int l1, int lr, Dc invL1, Dc invL2, const float4 *__restrict__ in,
              const float4 *__restrict__ tw1, float4 *__restrict__ out)
{
    extern __shared__ float4 sx[];
    const int rows = 1 << lr;
    const int j0 = blockIdx.x * rows;
    const float4 *src = in + ((size_t)j0 << l1);
    for (int e = threadIdx.x; e < (rows << l1); e += blockDim.x) sx[e] = src[e];
    __syncthreads();
    dif_df(sx, rows, l1, tw1, -1);
    for (int e = threadIdx.x; e < (rows << l1); e += blockDim.x) {
        const int r = e >> l1, pos = e & (n1 - 1);
        const int i = bitrev(pos, l1), j = j0 + r;
        const int m1 = (i < n1 / 2) ? i : i - n1;
        const int m2 = (j < n2 / 2) ? j : j - n2;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!(m1 == 0 && m2 == 0) && 2 * i != n1 && 2 * j != n2) {
            const df t1 = mul_f(dc(invL1), (float)m1), t2 = mul_f(dc(invL2), (float)m2);
            const df rs = rsqrt(add(sqr(t1), sqr(t2)));
            const cdf mult{neg(mul(t2, rs)), neg(mul(t1, rs))};
            v = st_c(cmul(ld_c(sx[e]), mult));
        }
        sx[e] = v;
    }
    __syncthreads();
    dit_df(sx, rows, l1, tw1, +1);
    for (int e = threadIdx.x; e < (rows << l1); e += blockDim.x) {
        const int i = e >> lr, r = e & (rows - 1);
        out[(size_t)i * n2 + j0 + r] = sx[(r << l1) + i];
    }
}

// pass C: rows i (length n2); inverse; s = Re / (n1 n2); u = -s/2 N; Phi = q + |u|^2 / 2.
__global__ void __launch_bounds__(kFftTpb)
    pass_c_df(int n1, int n2, int l2, int lr, float scale, const float4 *__restrict__ in,
              const float4 *__restrict__ tw2, const float2 *__restrict__ nrm,
              const float2 *__restrict__ q, float2 *__restrict__ u, float2 *__restrict__ phi)
{
    extern __shared__ float4 sx[];
    const int rows = 1 << lr;
    const int i0 = blockIdx.x * rows;
    const size_t N = (size_t)n1 * n2;
    const size_t o = (size_t)i0 * n2;
    for (int e = threadIdx.x; e < (rows << l2); e += blockDim.x) sx[e] = in[o + e];
    __syncthreads();
    dif_df(sx, rows, l2, tw2, +1);
    for (int e = threadIdx.x; e < (rows << l2); e += blockDim.x) {
        const int r = e >> l2, j = e & (n2 - 1);
        const size_t p = o + e;
        const float4 v = sx[(r << l2) + bitrev(j, l2)];
        const df s = scale2(df{v.x, v.y}, scale);  // scale = -1 / (2 n1 n2), a power of two
        const df ux = mul(s, ldf(nrm, p)), uy = mul(s, ldf(nrm, N + p)), uz = mul(s, ldf(nrm, 2 * N + p));
        u[p] = to_f2(ux);
        u[N + p] = to_f2(uy);
        u[2 * N + p] = to_f2(uz);
        const df k2 = add(add(sqr(ux), sqr(uy)), sqr(uz));
        phi[p] = to_f2(add(ldf(q, p), scale2(k2, 0.5f)));
    }
}

__global__ void twiddle_df_kernel(int L, float4 *tw)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L / 2) return;
    double s, c;
    sincospi(-2.0 * (double)k / (double)L, &s, &c);
    const float ch = __double2float_rn(c), sh = __double2float_rn(s);
    tw[k] = make_float4(ch, __double2float_rn(c - (double)ch), sh, __double2float_rn(s - (double)sh));
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

int ilog2(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// rows per CTA of an FFT pass: rows * L * 16 bytes <= 64 KiB
int lrows_for(int L) { return ilog2(std::max(1, std::min(8, 4096 / L))); }

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
    g.grav = split(c->g);
    g.m2a = split(-2.0 * c->atwood);
    g.mu = split(c->mu);
    return g;
}

inline const float2 *F2(const double *p) { return reinterpret_cast<const float2 *>(p); }
inline float2 *F2(double *p) { return reinterpret_cast<float2 *>(p); }
inline const float4 *F4(const double2 *p) { return reinterpret_cast<const float4 *>(p); }
inline float4 *F4(double2 *p) { return reinterpret_cast<float4 *>(p); }

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
    twiddle_df_kernel<<<(g.n1 / 2 + 255) / 256, 256>>>(g.n1, F4(c->tw1));
    twiddle_df_kernel<<<(g.n2 / 2 + 255) / 256, 256>>>(g.n2, F4(c->tw2));
    const int smax = 64 * 1024;
    int rc = cuda_check(cudaFuncSetAttribute(pass_a_df, cudaFuncAttributeMaxDynamicSharedMemorySize, smax),
                        "df fft smem attribute");
    if (!rc) rc = cuda_check(cudaFuncSetAttribute(pass_b_df, cudaFuncAttributeMaxDynamicSharedMemorySize, smax),
                             "df fft smem attribute");
    if (!rc) rc = cuda_check(cudaFuncSetAttribute(pass_c_df, cudaFuncAttributeMaxDynamicSharedMemorySize, smax),
                             "df fft smem attribute");
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
    const int ra = lrows_for(G.n2), rb = lrows_for(G.n1);
    prof_begin(c, ZM_K_FFT, &ev);
    pass_a_df<<<G.n1 >> ra, kFftTpb, (G.n2 << ra) * sizeof(float4), c->stream>>>(
        G.n1, G.n2, l2, ra, F2(y) + 3 * (size_t)G.N, F4(c->tw2), F4(c->fa));
    pass_b_df<<<G.n2 >> rb, kFftTpb, (G.n1 << rb) * sizeof(float4), c->stream>>>(
        G.n1, G.n2, l1, rb, split(1.0 / G.L1), split(1.0 / G.L2), F4(c->fa), F4(c->tw1), F4(c->fb));
    const float scale = (float)(-0.5 / ((double)G.n1 * (double)G.n2));
    pass_c_df<<<G.n1 >> ra, kFftTpb, (G.n2 << ra) * sizeof(float4), c->stream>>>(
        G.n1, G.n2, l2, ra, scale, F4(c->fb), F4(c->tw2), F2(c->nrm), F2(c->q), F2(c->u), F2(c->phi));
    prof_end(c, ZM_K_FFT, ev);
    c->prof.acc.launches[ZM_K_FFT] += 2;  // three kernels per Riesz evaluation
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
