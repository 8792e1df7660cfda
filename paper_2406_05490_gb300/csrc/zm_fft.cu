// zm_fft.cu -- low-order velocity by FFT Riesz transforms (paper Sec. 2: the low-order Z-Model
// approximates the Birkhoff-Rott integral with FFTs; Sec. 3.1 ZModel Order::Low; periodic only):
//     s = R1 w1 + R2 w2,  R_l^(k) = -i k_l / |k|,  k_l = 2 pi m_l / L_l,
//     multiplier zero at k = 0 and on the Nyquist row and column;  u = -1/2 s N,
//     Phi = q + 1/2 |u|^2.
// Single-GPU design (no distributed FFT): the two real fields are packed as c = w1 + i w2 and
// one complex transform suffices, because s = Re IFFT[(m1 - i m2) FFT(c)] with m_l = -i k_l/|k|
// (the imaginary part of that inverse is R1 w2 - R2 w1 and is dropped).  Three passes, each
// reading and writing the n1 x n2 complex field once:
//   pass A: rows (along alpha2) forward, transposed write          [n1][n2] -> [n2][n1]
//   pass B: rows of the transpose (along alpha1) forward, multiply by -(k2 + i k1)/|k|,
//           inverse along alpha1, transposed write                  [n2][n1] -> [n1][n2]
//   pass C: rows inverse along alpha2, real part / (n1 n2), epilogue u = -s/2 N, Phi.
// Each CTA holds `rows` complete rows in shared memory and runs radix-2^2 butterflies there:
// decimation in frequency (natural order in, bit-reversed out) for the forward transforms and
// for pass C, decimation in time (bit-reversed in, natural out) for the inverse of pass B.
// Sides L = R M with M = 2^a (a >= 3) and R odd (3 .. 19; 4864 = 19 x 256 is the paper's
// low-order mesh, Sec. 5.1) add one radix-R stage: before the length-M transforms in decimation
// in frequency, after them in decimation in time.  Frequency R k1 + k2 then sits at position
// k2 M + bitrev(k1) of a row.
#include <algorithm>

#include "zm_internal.cuh"

namespace zm {
namespace {

constexpr int kFftTpb = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ int bitrev(int j, int logL) { return (int)(__brev((unsigned)j) >> (32 - logL)); }

// W_L^k = exp(-2 pi i k / L) for 0 <= k < 3L/4 from the half table tw[k] (k < L/2), using
// W_L^(k + L/2) = -W_L^k; conjugated for the inverse (sgn = +1).
__device__ __forceinline__ double2 twiddle(const double2 *__restrict__ tw, int k, int half, int sgn)
{
    double2 w = tw[k >= half ? k - half : k];
    if (k >= half) w = make_double2(-w.x, -w.y);
    if (sgn > 0) w.y = -w.y;
    return w;
}

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
// a * (+i) for s > 0, a * (-i) for s < 0 (exact)
__device__ __forceinline__ double2 cmul_pm_i(double2 a, int s)
{
    return s > 0 ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x);
}

// Decimation in frequency, in place on `rows` rows of length L = 2^l >= 8 in shared memory:
// natural order in, bit-reversed order out.  Pairs of radix-2 stages (spans 2h, h) are fused
// into radix-2^2 butterflies on x[p], x[p+h], x[p+2h], x[p+3h] of a block of 4h, which take three
// twiddle products per four values instead of four and keep the radix-2 output order; when
// log2 L is odd, one radix-2 stage (span L/2) comes first.  W^0 = 1 products are skipped.
__device__ void fft_dif(double2 *x, int rows, int L, const double2 *__restrict__ tw, int sgn)
{
    const int l = __ffs(L) - 1, half = L >> 1, quarter = L >> 2;
    if (l & 1) {
        for (int b = threadIdx.x; b < rows * half; b += blockDim.x) {
            const int row = b >> (l - 1), pos = b & (half - 1);
            double2 *xr = x + ((size_t)row << l);
            const double2 u = xr[pos], v = xr[pos + half];
            xr[pos] = cadd(u, v);
            const double2 d = csub(u, v);
            xr[pos + half] = pos ? cmul(d, twiddle(tw, pos, half, sgn)) : d;
        }
        __syncthreads();
    }
    for (int h = (l & 1) ? (L >> 3) : (L >> 2); h >= 1; h >>= 2) {
        const int lh = __ffs(h) - 1;
        const int step = half / (2 * h);  // W_{4h}^m = W_L^(m * step)
        for (int b = threadIdx.x; b < rows * quarter; b += blockDim.x) {
            const int row = b >> (l - 2), idx = b & (quarter - 1);
            const int pos = idx & (h - 1);
            double2 *xr = x + ((size_t)row << l) + ((idx >> lh) << (lh + 2)) + pos;
            const double2 a0 = xr[0], a1 = xr[h], a2 = xr[2 * h], a3 = xr[3 * h];
            const double2 s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3);
            const double2 d13 = cmul_pm_i(csub(a1, a3), sgn);  // times W_{4h}^h = -+i
            const double2 x2 = csub(s02, s13), x1 = cadd(d02, d13), x3 = csub(d02, d13);
            xr[0] = cadd(s02, s13);
            const int e1 = pos * step;
            if (e1 == 0) {
                xr[h] = x2;
                xr[2 * h] = x1;
                xr[3 * h] = x3;
            } else {
                xr[h] = cmul(x2, twiddle(tw, 2 * e1, half, sgn));
                xr[2 * h] = cmul(x1, twiddle(tw, e1, half, sgn));
                xr[3 * h] = cmul(x3, twiddle(tw, 3 * e1, half, sgn));
            }
        }
        __syncthreads();
    }
}

// Decimation in time, in place: bit-reversed order in, natural order out (the mirror of fft_dif:
// fused pairs of spans (h, 2h) from h = 1, then one radix-2 stage of span L/2 when log2 L is odd).
__device__ void fft_dit(double2 *x, int rows, int L, const double2 *__restrict__ tw, int sgn)
{
    const int l = __ffs(L) - 1, half = L >> 1, quarter = L >> 2;
    for (int h = 1; 4 * h <= L; h <<= 2) {
        const int lh = __ffs(h) - 1;
        const int step = half / (2 * h);
        for (int b = threadIdx.x; b < rows * quarter; b += blockDim.x) {
            const int row = b >> (l - 2), idx = b & (quarter - 1);
            const int pos = idx & (h - 1);
            double2 *xr = x + ((size_t)row << l) + ((idx >> lh) << (lh + 2)) + pos;
            const double2 a0 = xr[0];
            double2 c1 = xr[h], c2 = xr[2 * h], c3 = xr[3 * h];
            const int e1 = pos * step;
            if (e1) {
                c1 = cmul(c1, twiddle(tw, 2 * e1, half, sgn));
                c2 = cmul(c2, twiddle(tw, e1, half, sgn));
                c3 = cmul(c3, twiddle(tw, 3 * e1, half, sgn));
            }
            const double2 s01 = cadd(a0, c1), d01 = csub(a0, c1), s23 = cadd(c2, c3);
            const double2 d23 = cmul_pm_i(csub(c2, c3), sgn);
            xr[0] = cadd(s01, s23);
            xr[2 * h] = csub(s01, s23);
            xr[h] = cadd(d01, d23);
            xr[3 * h] = csub(d01, d23);
        }
        __syncthreads();
    }
    if (l & 1) {
        for (int b = threadIdx.x; b < rows * half; b += blockDim.x) {
            const int row = b >> (l - 1), pos = b & (half - 1);
            double2 *xr = x + ((size_t)row << l);
            const double2 u = xr[pos];
            const double2 v = pos ? cmul(xr[pos + half], twiddle(tw, pos, half, sgn)) : xr[pos + half];
            xr[pos] = cadd(u, v);
            xr[pos + half] = csub(u, v);
        }
        __syncthreads();
    }
}

// DFT of length R (odd) in registers, v[t] -> sum_t v[t] W_R^(t k), W_R = exp(sgn 2 pi i / R),
// from the half table of W_L (W_R^e = W_L^(e M)); output k goes to out(k, X_k).  v is
// overwritten by the sums s_n = v_n + v_{R-n} and differences d_n = v_n - v_{R-n}: outputs k
// and R - k share A_k = v0 + sum_n s_n Re W^(nk) and B_k = sum_n d_n Im W^(nk), as
// X_k = A_k + i B_k and X_{R-k} = A_k - i B_k (W^(n(R-k)) is the conjugate of W^(nk)).
template <int R, class Out>
__device__ __forceinline__ void dft_small(double2 (&v)[R], const double2 *__restrict__ twl, int M, int half,
                                          int sgn, Out out)
{
    constexpr int H = (R - 1) / 2;
    double2 x0 = v[0];
#pragma unroll
    for (int n = 1; n <= H; ++n) {
        const double2 a = v[n], b = v[R - n];
        v[n] = cadd(a, b);
        v[R - n] = csub(a, b);
        x0 = cadd(x0, v[n]);
    }
    out(0, x0);
#pragma unroll 1
    for (int k = 1; k <= H; ++k) {  // not unrolled: keeps the live registers to v and two sums
        double2 a = v[0], b = make_double2(0.0, 0.0);
#pragma unroll
        for (int n = 1; n <= H; ++n) {
            const double2 w = twiddle(twl, ((n * k) % R) * M, half, sgn);
            a.x = fma(v[n].x, w.x, a.x);
            a.y = fma(v[n].y, w.x, a.y);
            b.x = fma(v[R - n].x, w.y, b.x);
            b.y = fma(v[R - n].y, w.y, b.y);
        }
        out(k, make_double2(a.x - b.y, a.y + b.x));      // a + i b
        out(R - k, make_double2(a.x + b.y, a.y - b.x));  // a - i b
    }
}

// Radix-R stage of decimation in frequency on `rows` rows of length L = R M in shared memory:
// for each n1 < M the values x[n1 + M t] (t < R) become W_L^(n1 k) DFT_R(x)[k] at n1 + M k, so
// that sub-row k (positions k M .. k M + M - 1) transforms, with length M, to outputs R k1 + k.
// Not inlined: each radix is compiled once per pass kernel instead of once per call site.
template <int R>
__device__ __noinline__ void radix_dif_r(double2 *x, int rows, int M, int lM, const double2 *__restrict__ twl,
                                         int sgn)
{
    const int L = R * M, half = L >> 1;
    for (int b = threadIdx.x; b < rows * M; b += blockDim.x) {
        const int row = b >> lM, n1 = b & (M - 1);
        if (!ZM_IDX_OK(row, rows)) continue;
        double2 *xr = x + (size_t)row * L + n1;
        double2 v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = xr[t * M];
        dft_small<R>(v, twl, M, half, sgn, [&](int k, double2 val) {
            xr[k * M] = (n1 && k) ? cmul(val, twiddle(twl, n1 * k, half, sgn)) : val;
        });
    }
    __syncthreads();
}

// The mirror stage of decimation in time: sub-row k holds, in natural order n1, the length-M
// transform of the outputs R k1 + k; the values x[k M + n1] times W_L^(n1 k) go through DFT_R
// over k, and output t lands at n1 + M t (in place: each thread owns its column n1).
template <int R>
__device__ __noinline__ void radix_dit_r(double2 *x, int rows, int M, int lM, const double2 *__restrict__ twl,
                                         int sgn)
{
    const int L = R * M, half = L >> 1;
    for (int b = threadIdx.x; b < rows * M; b += blockDim.x) {
        const int row = b >> lM, n1 = b & (M - 1);
        if (!ZM_IDX_OK(row, rows)) continue;
        double2 *xr = x + (size_t)row * L + n1;
        double2 v[R];
        v[0] = xr[0];
#pragma unroll
        for (int k = 1; k < R; ++k) v[k] = n1 ? cmul(xr[k * M], twiddle(twl, n1 * k, half, sgn)) : xr[k * M];
        dft_small<R>(v, twl, M, half, sgn, [&](int t, double2 val) { xr[t * M] = val; });
    }
    __syncthreads();
}

#define ZM_FOR_RADICES(X) X(3) X(5) X(7) X(9) X(11) X(13) X(15) X(17) X(19)

__device__ void radix_dif(double2 *x, int rows, int R, int M, int lM, const double2 *__restrict__ twl, int sgn)
{
    switch (R) {
#define ZM_CASE(r) \
    case r: radix_dif_r<r>(x, rows, M, lM, twl, sgn); break;
        ZM_FOR_RADICES(ZM_CASE)
#undef ZM_CASE
    default: break;
    }
}

__device__ void radix_dit(double2 *x, int rows, int R, int M, int lM, const double2 *__restrict__ twl, int sgn)
{
    switch (R) {
#define ZM_CASE(r) \
    case r: radix_dit_r<r>(x, rows, M, lM, twl, sgn); break;
        ZM_FOR_RADICES(ZM_CASE)
#undef ZM_CASE
    default: break;
    }
}

// One side of the transform: L = R M, M = 2^lM; tw = half table of W_M, twl = half table of W_L
// (used only when R > 1).
struct Side {
    int L, R, M, lM;
    const double2 *tw, *twl;
};

// Forward (sgn -1) or inverse (sgn +1) transform of `rows` rows by decimation in frequency.
template <bool kMix>
__device__ __forceinline__ void side_dif(double2 *x, int rows, const Side &s, int sgn)
{
    if (kMix) {
        if (s.R > 1) radix_dif(x, rows, s.R, s.M, s.lM, s.twl, sgn);
        fft_dif(x, rows * s.R, s.M, s.tw, sgn);
    } else {
        fft_dif(x, rows, s.L, s.tw, sgn);
    }
}

template <bool kMix>
__device__ __forceinline__ void side_dit(double2 *x, int rows, const Side &s, int sgn)
{
    if (kMix) {
        fft_dit(x, rows * s.R, s.M, s.tw, sgn);
        if (s.R > 1) radix_dit(x, rows, s.R, s.M, s.lM, s.twl, sgn);
    } else {
        fft_dit(x, rows, s.L, s.tw, sgn);
    }
}

// Position in a row after decimation in frequency of the output with index f (natural order).
template <bool kMix>
__device__ __forceinline__ int dif_pos(int f, const Side &s)
{
    if (!kMix) return bitrev(f, s.lM);
    const int k1 = f / s.R, k2 = f - k1 * s.R;
    return k2 * s.M + bitrev(k1, s.lM);
}

// Output index f (natural order) held at position `pos` after decimation in frequency.
template <bool kMix>
__device__ __forceinline__ int dif_freq(int pos, const Side &s)
{
    if (!kMix) return bitrev(pos, s.lM);
    return s.R * bitrev(pos & (s.M - 1), s.lM) + (pos >> s.lM);
}

// pass A: rows i of length n2 from w1 + i w2; forward; write out[j][i] (transposed).
template <bool kMix>
__global__ void __launch_bounds__(kFftTpb, kMix ? 2 : 1)
    pass_a(int n1, int n2, Side s2, int rows, const double *__restrict__ w, double2 *__restrict__ out)
{
    extern __shared__ double2 sx[];
    const int i0 = blockIdx.x * rows;
    const size_t N = (size_t)n1 * n2;
    for (int e = threadIdx.x; e < rows * n2; e += blockDim.x) {
        const int r = e / n2, j = e - r * n2;
        const size_t p = (size_t)(i0 + r) * n2 + j;
        sx[e] = ZM_IDX_OK(p, N) ? make_double2(w[p], w[N + p]) : make_double2(0.0, 0.0);
    }
    __syncthreads();
    side_dif<kMix>(sx, rows, s2, -1);
    for (int e = threadIdx.x; e < rows * n2; e += blockDim.x) {
        const int j = e / rows, r = e - j * rows;
        const size_t o = (size_t)j * n1 + i0 + r;
        const int k = r * n2 + dif_pos<kMix>(j, s2);
        if (ZM_IDX_OK(o, N) && ZM_IDX_OK(k, rows * n2)) out[o] = sx[k];
    }
}

// pass B: rows j (length n1) of the transpose; forward; multiply; inverse; write out[i][j].
template <bool kMix>
__global__ void __launch_bounds__(kFftTpb, kMix ? 2 : 1)
    pass_b(int n1, int n2, Side s1, int rows, double invL1, double invL2, const double2 *__restrict__ in,
           double2 *__restrict__ out)
{
    extern __shared__ double2 sx[];
    const int j0 = blockIdx.x * rows;
    for (int e = threadIdx.x; e < rows * n1; e += blockDim.x)
        sx[e] = ZM_IDX_OK((size_t)j0 * n1 + e, (size_t)n1 * n2) ? in[(size_t)j0 * n1 + e] : make_double2(0.0, 0.0);
    __syncthreads();
    side_dif<kMix>(sx, rows, s1, -1);
    for (int e = threadIdx.x; e < rows * n1; e += blockDim.x) {
        const int r = e / n1, pos = e - r * n1;
        const int i = dif_freq<kMix>(pos, s1), j = j0 + r;  // frequency indices
        const int m1 = (2 * i < n1) ? i : i - n1;
        const int m2 = (2 * j < n2) ? j : j - n2;
        double2 v = make_double2(0.0, 0.0);
        if (!(m1 == 0 && m2 == 0) && 2 * i != n1 && 2 * j != n2) {
            // k_l / |k| with k_l = 2 pi m_l / L_l: the 2 pi cancels, t_l = m_l / L_l
            const double k1 = m1 * invL1, k2 = m2 * invL2;
            const double ik = dev::rsqrt_nr(k1 * k1 + k2 * k2);
            // multiplier -(k2 + i k1) / |k|
            v = cmul(sx[e], make_double2(-k2 * ik, -k1 * ik));
        }
        sx[e] = v;
    }
    __syncthreads();
    side_dit<kMix>(sx, rows, s1, +1);
    for (int e = threadIdx.x; e < rows * n1; e += blockDim.x) {
        const int i = e / rows, r = e - i * rows;
        if (ZM_IDX_OK((size_t)i * n2 + j0 + r, (size_t)n1 * n2)) out[(size_t)i * n2 + j0 + r] = sx[(size_t)r * n1 + i];
    }
}

// pass C: rows i (length n2); inverse; s = Re / (n1 n2); u = -s/2 N; Phi = q + |u|^2 / 2.
template <bool kMix>
__global__ void __launch_bounds__(kFftTpb, kMix ? 2 : 1)
    pass_c(int n1, int n2, Side s2, int rows, double inv, const double2 *__restrict__ in,
           const double *__restrict__ nrm, const double *__restrict__ q, double *__restrict__ u,
           double *__restrict__ phi)
{
    extern __shared__ double2 sx[];
    const int i0 = blockIdx.x * rows;
    const size_t N = (size_t)n1 * n2;
    for (int e = threadIdx.x; e < rows * n2; e += blockDim.x)
        sx[e] = ZM_IDX_OK((size_t)i0 * n2 + e, N) ? in[(size_t)i0 * n2 + e] : make_double2(0.0, 0.0);
    __syncthreads();
    side_dif<kMix>(sx, rows, s2, +1);
    for (int e = threadIdx.x; e < rows * n2; e += blockDim.x) {
        const int r = e / n2, j = e - r * n2;
        const size_t p = (size_t)(i0 + r) * n2 + j;
        const int k = r * n2 + dif_pos<kMix>(j, s2);
        if (!ZM_IDX_OK(p, N) || !ZM_IDX_OK(k, rows * n2)) continue;
        const double s = sx[k].x * inv;
        const double ux = -0.5 * s * nrm[p], uy = -0.5 * s * nrm[N + p], uz = -0.5 * s * nrm[2 * N + p];
        u[p] = ux;
        u[N + p] = uy;
        u[2 * N + p] = uz;
        phi[p] = q[p] + 0.5 * (ux * ux + uy * uy + uz * uz);
    }
}

__global__ void twiddle_kernel(int L, double2 *tw)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L / 2) return;
    double s, c;
    sincospi(-2.0 * (double)k / (double)L, &s, &c);
    tw[k] = make_double2(c, s);
}

int ilog2(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// Rows per CTA: a power of two (it must divide the other side, which has a factor 2^3), at most
// 8 and at most 4096 / L.
int rows_for(int L)
{
    int r = 8;
    while (r > 1 && r * L > 4096) r >>= 1;
    return r;
}

// Rows per CTA, halved (down to one) while the pass would launch fewer than ZM_FFT_MINGRID CTAs
// over its `avail` rows, so that small meshes spread over every SM.
#ifndef ZM_FFT_MINGRID
#define ZM_FFT_MINGRID 304  // two CTAs per SM of the 152
#endif
int rows_grid(int L, int avail)
{
    int r = rows_for(L);
    while (r > 1 && avail / r < ZM_FFT_MINGRID) r >>= 1;
    return r;
}

// Largest row held in shared memory by one CTA: 8192 complex doubles (128 KiB).
constexpr int kMaxSide = 8192;

Side make_side(int L, const double2 *tw, const double2 *twl)
{
    Side s;
    s.L = L;
    s.M = L & -L;
    s.R = L / s.M;
    s.lM = ilog2(s.M);
    s.tw = tw;
    s.twl = twl;
    return s;
}

template <bool kMix>
int set_smem_limits()
{
    const int smax = kMaxSide * (int)sizeof(double2);
    int rc = cuda_check(cudaFuncSetAttribute(pass_a<kMix>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax),
                        "fft smem attribute");
    if (!rc)
        rc = cuda_check(cudaFuncSetAttribute(pass_b<kMix>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax),
                        "fft smem attribute");
    if (!rc)
        rc = cuda_check(cudaFuncSetAttribute(pass_c<kMix>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax),
                        "fft smem attribute");
    return rc;
}

template <bool kMix>
int launch_passes(zm_ctx *c, const double *w)
{
    const Geom &g = c->geom;
    const Side s1 = make_side(g.n1, c->tw1, c->twl1), s2 = make_side(g.n2, c->tw2, c->twl2);
    const int ra = rows_grid(g.n2, g.n1), rb = rows_grid(g.n1, g.n2);
    if (g.n1 % ra || g.n2 % rb) return set_error(ZM_ERR_INVALID, "Riesz pass: rows per CTA do not divide the side");
    pass_a<kMix><<<g.n1 / ra, kFftTpb, ra * g.n2 * sizeof(double2), c->stream>>>(g.n1, g.n2, s2, ra, w, c->fa);
    pass_b<kMix><<<g.n2 / rb, kFftTpb, rb * g.n1 * sizeof(double2), c->stream>>>(
        g.n1, g.n2, s1, rb, 1.0 / g.L1, 1.0 / g.L2, c->fa, c->fb);
    pass_c<kMix><<<g.n1 / ra, kFftTpb, ra * g.n2 * sizeof(double2), c->stream>>>(
        g.n1, g.n2, s2, ra, 1.0 / ((double)g.n1 * (double)g.n2), c->fb, c->nrm, c->q, c->u, c->phi);
    return ZM_OK;
}

}  // namespace

bool fft_side_ok(int L)
{
    if (L < 8 || L > kMaxSide) return false;
    const int M = L & -L, R = L / M;
    if (M < 8) return false;
    switch (R) {
    case 1:
#define ZM_CASE(r) case r:
        ZM_FOR_RADICES(ZM_CASE)
#undef ZM_CASE
        return true;
    default: return false;
    }
}

int fft_setup(zm_ctx *c)
{
    const Geom &g = c->geom;
    const size_t N = g.N;
    const Side s1 = make_side(g.n1, nullptr, nullptr), s2 = make_side(g.n2, nullptr, nullptr);
    if (cudaMalloc(&c->fa, N * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&c->fb, N * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&c->tw1, (s1.M / 2) * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&c->tw2, (s2.M / 2) * sizeof(double2)) != cudaSuccess ||
        (s1.R > 1 && cudaMalloc(&c->twl1, (g.n1 / 2) * sizeof(double2)) != cudaSuccess) ||
        (s2.R > 1 && cudaMalloc(&c->twl2, (g.n2 / 2) * sizeof(double2)) != cudaSuccess)) {
        cudaGetLastError();
        return set_error(ZM_ERR_NOMEM, "fft_setup: device allocation failed");
    }
    twiddle_kernel<<<(s1.M / 2 + 255) / 256, 256>>>(s1.M, c->tw1);
    twiddle_kernel<<<(s2.M / 2 + 255) / 256, 256>>>(s2.M, c->tw2);
    if (c->twl1) twiddle_kernel<<<(g.n1 / 2 + 255) / 256, 256>>>(g.n1, c->twl1);
    if (c->twl2) twiddle_kernel<<<(g.n2 / 2 + 255) / 256, 256>>>(g.n2, c->twl2);
    int rc = set_smem_limits<false>();
    if (!rc) rc = set_smem_limits<true>();
    if (!rc) rc = cuda_check(cudaGetLastError(), "twiddle kernel");
    return rc;
}

int launch_riesz(zm_ctx *c, const double *y)
{
    if (!y || !c->fa || !c->fb || !c->tw1 || !c->tw2 || !c->nrm || !c->q || !c->u || !c->phi)
        return set_error(ZM_ERR_INVALID, "Riesz pass: missing buffer");
    const Geom &g = c->geom;
    const bool pow1 = (g.n1 & (g.n1 - 1)) == 0, pow2 = (g.n2 & (g.n2 - 1)) == 0;
    if ((!pow1 && !c->twl1) || (!pow2 && !c->twl2))
        return set_error(ZM_ERR_INVALID, "Riesz pass: missing twiddle table");
    const bool mix = !(pow1 && pow2);
    const double *w = y + 3 * (size_t)g.N;
    cudaEvent_t ev = nullptr;
    prof_begin(c, ZM_K_FFT, &ev);
    const int rc = mix ? launch_passes<true>(c, w) : launch_passes<false>(c, w);
    prof_end(c, ZM_K_FFT, ev);
    if (rc) return rc;
    c->prof.acc.launches[ZM_K_FFT] += 2;  // three kernels per Riesz evaluation
    return cuda_check(cudaGetLastError(), "Riesz FFT launch");
}

ZM_BOUNDS_READER(bounds_fft)

}  // namespace zm
