// zm_lowdf_mix.cu -- double-word FFT Riesz passes over sides L = R 2^A (R odd, 3 .. 19), among
// them the paper's 4864 = 19 x 2^8 low-order mesh (Sec. 5.1): one radix-R stage around the
// power-of-two chunk passes of zm_dffft.cuh.  Paper Sec. 2 (low-order model).
#include "zm_dffft.cuh"

namespace zm {
namespace {

// ---- sides L = R 2^A (R odd, 3 .. 19) -----------------------------------------------------------
// One radix-R stage in double words around the length-2^A transforms of the passes above: in
// decimation in frequency the R values x[n1 + M t] (M = 2^A, t < R) of column n1 become
// W_L^(n1 k) DFT_R(x)[k] at n1 + M k, so that sub-row k of the row transforms, with length M,
// to the outputs R k1 + k (at position k M + bitrev(k1)); decimation in time runs the mirror
// stage after the length-M transforms.  The length-R DFT pairs outputs k and R - k through the
// sums s_n = x_n + x_{R-n} and differences d_n = x_n - x_{R-n}: X_k = A_k + i B_k and
// X_{R-k} = A_k - i B_k with A_k = x_0 + sum_n s_n Re W^(nk), B_k = sum_n d_n Im W^(nk).

__device__ __forceinline__ u64 bcast(float x) { return pk(x, x); }

// acc += x c for a real double word c given as (c.hi, c.hi), (c.lo, c.lo): the leading product
// exact (two_prod), its error and the cross terms into the low part; acc stays unnormalised.
__device__ __forceinline__ void acc_real(C2 &acc, C2 x, u64 ch, u64 cl)
{
    const u64 p = mul2(x.h, ch);
    u64 t = fma2(x.h, ch, neg2(p));
    t = fma2(x.h, cl, t);
    t = fma2(x.l, ch, t);
    u64 s, e;
    two_sum2(acc.h, p, s, e);
    acc = C2{s, add2(acc.l, add2(t, e))};
}

// DFT of length R of v (overwritten by the sums and differences); output k goes to out(k, X_k).
// Roots W_R^e = W_L^(e M) from the half table of W_L.
template <int R, class Out>
__device__ __forceinline__ void dft_df(C2 (&v)[R], const ulonglong2 *__restrict__ twl, int M, int half, int sgn,
                                       Out out)
{
    constexpr int H = (R - 1) / 2;
    C2 x0 = v[0];
#pragma unroll
    for (int n = 1; n <= H; ++n) {
        const C2 a = v[n], b = v[R - n];
        v[n] = cadd2(a, b);
        v[R - n] = csub2(a, b);
        x0 = cadd2(x0, v[n]);
    }
    out(0, x0);
#pragma unroll 1
    for (int k = 1; k <= H; ++k) {  // not unrolled: the body is H double-word terms already
        C2 A = v[0], B = C2{0ull, 0ull};
#pragma unroll
        for (int n = 1; n <= H; ++n) {
            const C2 w = tw_get(twl, ((n * k) % R) * M, half, sgn);
            acc_real(A, v[n], bcast(lane0(w.h)), bcast(lane0(w.l)));
            acc_real(B, v[R - n], bcast(lane1(w.h)), bcast(lane1(w.l)));
        }
        A = fast_two_sum2(A.h, A.l);
        B = fast_two_sum2(B.h, B.l);
        const C2 iB = cmul_i2(B, +1);
        out(k, cadd2(A, iB));
        out(R - k, csub2(A, iB));
    }
}

// Decimation-in-frequency radix-R stage: column n1 of row `row` read from global memory (pass
// A: the pair (w1, w2) of node row * L + index packed as one complex value; passes B and C: the
// complex value src[row * L + index]), written to shared memory (rows of length L = R M,
// padded).  Not inlined: the nine radices are compiled once, not once per pass and row length.
template <int R>
__device__ __noinline__ void radix_dif_df(ulonglong2 *sx, int rows, int lM, const ulonglong2 *__restrict__ twl,
                                          int sgn, const float2 *__restrict__ w1, const float2 *__restrict__ w2,
                                          const ulonglong2 *__restrict__ src)
{
    const int M = 1 << lM, L = R * M, half = L >> 1;
    for (int b = threadIdx.x; b < rows * M; b += blockDim.x) {
        const int row = b >> lM, n1 = b & (M - 1);
        if (!ZM_IDX_OK(row, rows)) continue;
        const int base = row * L + n1;
        C2 v[R];
#pragma unroll
        for (int t = 0; t < R; ++t)
            v[t] = src ? ld2(src[base + M * t]) : ld2(c2_pack(w1[base + M * t], w2[base + M * t]));
        dft_df<R>(v, twl, M, half, sgn, [&](int k, C2 x) {
            sx[phys(base + M * k)] = st2((n1 && k) ? cmul2(x, tw_get(twl, n1 * k, half, sgn)) : x);
        });
    }
}

// Decimation-in-time radix-R stage, in place in shared memory (each thread owns its column).
template <int R>
__device__ __noinline__ void radix_dit_df(ulonglong2 *sx, int rows, int lM, const ulonglong2 *__restrict__ twl,
                                          int sgn)
{
    const int M = 1 << lM, L = R * M, half = L >> 1;
    for (int b = threadIdx.x; b < rows * M; b += blockDim.x) {
        const int row = b >> lM, n1 = b & (M - 1);
        if (!ZM_IDX_OK(row, rows)) continue;
        const int base = row * L + n1;
        C2 v[R];
        v[0] = ld2(sx[phys(base)]);
#pragma unroll
        for (int k = 1; k < R; ++k) {
            const C2 x = ld2(sx[phys(base + M * k)]);
            v[k] = n1 ? cmul2(x, tw_get(twl, n1 * k, half, sgn)) : x;
        }
        dft_df<R>(v, twl, M, half, sgn, [&](int t, C2 x) { sx[phys(base + M * t)] = st2(x); });
    }
}

__device__ __forceinline__ void radix_dif_any(ulonglong2 *sx, int rows, int R, int lM,
                                              const ulonglong2 *__restrict__ twl, int sgn, const float2 *w1,
                                              const float2 *w2, const ulonglong2 *src)
{
    switch (R) {
#define ZM_CASE(r) \
    case r: radix_dif_df<r>(sx, rows, lM, twl, sgn, w1, w2, src); break;
        ZM_DF_RADICES(ZM_CASE)
#undef ZM_CASE
    default: break;
    }
    __syncthreads();
}

__device__ __forceinline__ void radix_dit_any(ulonglong2 *sx, int rows, int R, int lM,
                                              const ulonglong2 *__restrict__ twl, int sgn)
{
    switch (R) {
#define ZM_CASE(r) \
    case r: radix_dit_df<r>(sx, rows, lM, twl, sgn); break;
        ZM_DF_RADICES(ZM_CASE)
#undef ZM_CASE
    default: break;
    }
    __syncthreads();
}

constexpr int kMixTpb = 256;

// Position, after decimation in frequency, of output f of a row of length R 2^A.
template <int A>
__device__ __forceinline__ int mix_pos(int f, int R)
{
    const int k1 = f / R;
    return (f - k1 * R) * (1 << A) + bitrev(k1, A);
}

// pass A on rows of length n2 = R 2^A.
template <int A>
__global__ void __launch_bounds__(kMixTpb, 2)
    pass_a_dfm(int n1, int R, int lr, const float2 *__restrict__ w, const ulonglong2 *__restrict__ tw2,
               const ulonglong2 *__restrict__ twl2, ulonglong2 *__restrict__ out)
{
    extern __shared__ ulonglong2 sx[];
    const int L = R << A, rows = 1 << lr;
    const int i0 = blockIdx.x * rows;
    if (!ZM_IDX_OK(i0 + rows - 1, n1)) return;  // checked build: the CTA's rows exist
    const size_t N = (size_t)n1 * L;
    const float2 *w1 = w + (size_t)i0 * L, *w2 = w1 + N;
    radix_dif_any(sx, rows, R, A, twl2, -1, w1, w2, nullptr);
    auto lds = [&](int row, int i) { return ld2(sx[phys((row << A) + i)]); };
    dif_seq<A, 0, nc_of(A) - 1>(sx, tw2, rows * R, -1, lds);
    for (int e = threadIdx.x; e < rows * L; e += blockDim.x) {
        const int j = e >> lr, r = e & (rows - 1);
        out[(size_t)j * n1 + i0 + r] = sx[phys(r * L + mix_pos<A>(j, R))];
    }
}

// pass B on columns of length n1 = R 2^A.
template <int A>
__global__ void __launch_bounds__(kMixTpb, 2)
    pass_b_dfm(int n2, int R, int lr, Dc invL1, Dc invL2, const ulonglong2 *__restrict__ in,
               const ulonglong2 *__restrict__ tw1, const ulonglong2 *__restrict__ twl1, ulonglong2 *__restrict__ out)
{
    extern __shared__ ulonglong2 sx[];
    constexpr int NC = nc_of(A);
    const int L = R << A, rows = 1 << lr;
    const int j0 = blockIdx.x * rows;
    if (!ZM_IDX_OK(j0 + rows - 1, n2)) return;  // checked build: the CTA's columns exist
    radix_dif_any(sx, rows, R, A, twl1, -1, nullptr, nullptr, in + (size_t)j0 * L);
    if constexpr (NC > 1) {
        auto lds = [&](int row, int i) { return ld2(sx[phys((row << A) + i)]); };
        dif_seq<A, 0, NC - 2>(sx, tw1, rows * R, -1, lds);
    }
    mid_b<A, true>(sx, rows * R, j0, n2, invL1, invL2, tw1, R);
    __syncthreads();
    dit_seq<A, NC - 2>(sx, tw1, rows * R, +1);
    radix_dit_any(sx, rows, R, A, twl1, +1);
    for (int e = threadIdx.x; e < rows * L; e += blockDim.x) {
        const int i = e >> lr, r = e & (rows - 1);
        out[(size_t)i * n2 + j0 + r] = sx[phys(r * L + i)];
    }
}

// pass C on rows of length n2 = R 2^A.
template <int A>
__global__ void __launch_bounds__(kMixTpb, 2)
    pass_c_dfm(int n1, int R, int lr, Dc scale, const ulonglong2 *__restrict__ in,
               const ulonglong2 *__restrict__ tw2, const ulonglong2 *__restrict__ twl2, const float2 *__restrict__ nrm,
               const float2 *__restrict__ q, float2 *__restrict__ u, float2 *__restrict__ phi)
{
    extern __shared__ ulonglong2 sx[];
    const int L = R << A, rows = 1 << lr;
    const int i0 = blockIdx.x * rows;
    if (!ZM_IDX_OK(i0 + rows - 1, n1)) return;  // checked build: the CTA's rows exist
    const size_t N = (size_t)n1 * L;
    const size_t o = (size_t)i0 * L;
    radix_dif_any(sx, rows, R, A, twl2, +1, nullptr, nullptr, in + o);
    auto lds = [&](int row, int i) { return ld2(sx[phys((row << A) + i)]); };
    dif_seq<A, 0, nc_of(A) - 1>(sx, tw2, rows * R, +1, lds);
    for (int e = threadIdx.x; e < rows * L; e += blockDim.x) {
        const int r = e / L, j = e - r * L;
        const size_t p = o + e;
        const df s = mul(c2_re(ld2(sx[phys(r * L + mix_pos<A>(j, R))])), dc(scale));  // -1/(2 n1 n2)
        const df ux = mul(s, ldf(nrm, p)), uy = mul(s, ldf(nrm, N + p)), uz = mul(s, ldf(nrm, 2 * N + p));
        u[p] = to_f2(ux);
        u[N + p] = to_f2(uy);
        u[2 * N + p] = to_f2(uz);
        const df k2 = add(add(sqr(ux), sqr(uy)), sqr(uz));
        phi[p] = to_f2(add(ldf(q, p), scale2(k2, 0.5f)));
    }
}

// Launches of the three passes for rows of length R 2^A (R odd, > 1).
template <int A>
struct FftLaunchMix {
    static int a(int n1, int R, int lr, size_t smem, cudaStream_t s, const float2 *w, const ulonglong2 *tw2,
                 const ulonglong2 *twl2, ulonglong2 *out)
    {
        int rc = smem_attr((const void *)pass_a_dfm<A>, smem);
        if (rc) return rc;
        pass_a_dfm<A><<<n1 >> lr, kMixTpb, smem, s>>>(n1, R, lr, w, tw2, twl2, out);
        return cuda_check(cudaGetLastError(), "double-word FFT pass A launch");
    }
    static int b(int n2, int R, int lr, size_t smem, cudaStream_t s, Dc invL1, Dc invL2, const ulonglong2 *in,
                 const ulonglong2 *tw1, const ulonglong2 *twl1, ulonglong2 *out)
    {
        int rc = smem_attr((const void *)pass_b_dfm<A>, smem);
        if (rc) return rc;
        pass_b_dfm<A><<<n2 >> lr, kMixTpb, smem, s>>>(n2, R, lr, invL1, invL2, in, tw1, twl1, out);
        return cuda_check(cudaGetLastError(), "double-word FFT pass B launch");
    }
    static int c(int n1, int R, int lr, size_t smem, cudaStream_t s, Dc scale, const ulonglong2 *in,
                 const ulonglong2 *tw2, const ulonglong2 *twl2, const float2 *nrm, const float2 *q, float2 *u,
                 float2 *phi)
    {
        int rc = smem_attr((const void *)pass_c_dfm<A>, smem);
        if (rc) return rc;
        pass_c_dfm<A><<<n1 >> lr, kMixTpb, smem, s>>>(n1, R, lr, scale, in, tw2, twl2, nrm, q, u, phi);
        return cuda_check(cudaGetLastError(), "double-word FFT pass C launch");
    }
};

}  // namespace

int df_mix_pass_a(int A, int n1, int R, int lr, size_t smem, cudaStream_t s, const float2 *w,
                  const ulonglong2 *tw2, const ulonglong2 *twl2, ulonglong2 *out)
{
    return with_log2(A, [&](auto lc) { return FftLaunchMix<decltype(lc)::value>::a(n1, R, lr, smem, s, w, tw2, twl2, out); });
}

int df_mix_pass_b(int A, int n2, int R, int lr, size_t smem, cudaStream_t s, double invL1, double invL2,
                  const ulonglong2 *in, const ulonglong2 *tw1, const ulonglong2 *twl1, ulonglong2 *out)
{
    return with_log2(A, [&](auto lc) {
        return FftLaunchMix<decltype(lc)::value>::b(n2, R, lr, smem, s, split(invL1), split(invL2), in, tw1, twl1, out);
    });
}

int df_mix_pass_c(int A, int n1, int R, int lr, size_t smem, cudaStream_t s, double scale, const ulonglong2 *in,
                  const ulonglong2 *tw2, const ulonglong2 *twl2, const float2 *nrm, const float2 *q, float2 *u,
                  float2 *phi)
{
    return with_log2(A, [&](auto lc) {
        return FftLaunchMix<decltype(lc)::value>::c(n1, R, lr, smem, s, split(scale), in, tw2, twl2, nrm, q, u, phi);
    });
}

ZM_BOUNDS_READER(bounds_lowdf_mix)

}  // namespace zm
