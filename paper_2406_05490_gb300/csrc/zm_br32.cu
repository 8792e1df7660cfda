// zm_br32.cu -- FP32-compensated all-pairs Birkhoff-Rott sum (paper Sec. 2 BRSolver, Sec. 3.2.1
// ExactBRSolver, the high-order model), with FP64 accumulation across source tiles:
//     u_i = sum_j (z_j - z_i) x gamma'_j / (|z_j - z_i|^2 + delta^2)^(3/2).
//
// Work decomposition.  Targets come in groups of one 16 x 16 mesh tile (256 targets, 64
// threads x 4 targets in registers); sources in 16 x 16 tiles.  The iteration space
// (target group x source tile) is cut into equal contiguous ranges, one per persistent CTA
// (a stream-K decomposition): every CTA does the same number of tile pairs, whatever the mesh
// size, and writes one partial sum per target group its range touches.  A second kernel adds
// the partials of each target in a fixed order and forms Phi, so results are deterministic.
//
// Two source paths, chosen per (target group, source tile) from bounding spheres:
//   near (spheres within 1.25 x the sum of radii): positions as FP32 hi/lo pairs,
//     r = (zh_j - zh_i) + (zl_j - zl_i), then the direct formula -- 23 FP32 + 1 MUFU per pair;
//   far: tile-local coordinates s_j = z_j - c_T and t_i = z_i - c_T (c_T the tile centre), the
//     distance in Gram form |r|^2 + delta^2 = (|s_j|^2 + delta^2) + |t_i|^2 - 2 s_j . t_i, and the
//     cross product split as sum K (s_j x gamma_j) - t_i x sum K gamma_j -- 12 FP32 + 1 MUFU per
//     pair.  With the spheres apart, |s|, |t| and |r| are of one order, so neither the Gram
//     form nor the split loses more than a few units of FP32 rounding.  Two adjacent sources
//     share one packed FP32x2 instruction (fma/mul/add .f32x2): the FP32 work is unchanged but
//     issue slots halve, so the loop is bound by the FP32 pipe rather than by issue.
// Source tiles of both kinds arrive by 1D bulk TMA (cp.async.bulk) into a double-buffered
// shared-memory stage; every thread reads the same source at once (broadcast).
#include <algorithm>

#include "zm_internal.cuh"

namespace zm {
namespace {

constexpr int kT = 64;     // threads per CTA
constexpr int kR = 4;      // targets per thread
constexpr int kTs = 256;   // sources per tile (16 x 16)
constexpr int kGroup = 1;  // tiles per target group
constexpr float kFarFactor = 1.25f;

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
__device__ __forceinline__ u64 pack2(float lo, float hi)
{
    u64 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ float sum2(u64 v)
{
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return lo + hi;
}
__device__ __forceinline__ u64 rsqrt2(u64 v)
{
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return pack2(dev::rsqrt_approx(lo), dev::rsqrt_approx(hi));
}

struct Args {
    int n1, n2, N;
    int nt2, ntiles, ng2, ngroups;
    long long units;
    int ctas, kseg;
    float d2;
    const float *near_rec;  // [tile][9][256]: zh, zl, gamma'
    const float *far_rec;   // [tile][10][256]: s, |s|^2 + delta^2, gamma', s x gamma'
    const float4 *tinfo;    // [tile]: centre (x, y, z), radius
    double *part;           // [ctas * kseg][3][512]
    int *err;
};

__device__ __forceinline__ int cta_of_unit(long long k, long long units, int ctas)
{
    return (int)(((k + 1) * ctas - 1) / units);
}

// bounding sphere of target group G (one or two tiles)
__device__ __forceinline__ void group_sphere(const Args &a, int G, float3 &c, float &rad)
{
    const int ti = G / a.ng2, gj = G - ti * a.ng2;
    const int t0 = ti * a.nt2 + kGroup * gj;
    const float4 s0 = a.tinfo[t0];
    if (kGroup > 1 && kGroup * gj + 1 < a.nt2) {
        const float4 s1 = a.tinfo[t0 + 1];
        c = make_float3(0.5f * (s0.x + s1.x), 0.5f * (s0.y + s1.y), 0.5f * (s0.z + s1.z));
        const float d0 = sqrtf((s0.x - c.x) * (s0.x - c.x) + (s0.y - c.y) * (s0.y - c.y) + (s0.z - c.z) * (s0.z - c.z));
        const float d1 = sqrtf((s1.x - c.x) * (s1.x - c.x) + (s1.y - c.y) * (s1.y - c.y) + (s1.z - c.z) * (s1.z - c.z));
        rad = fmaxf(d0 + s0.w, d1 + s1.w);
    } else {
        c = make_float3(s0.x, s0.y, s0.z);
        rad = s0.w;
    }
}

__device__ __forceinline__ bool is_far(const Args &a, int G, int S)
{
    float3 c;
    float rg;
    group_sphere(a, G, c, rg);
    const float4 t = a.tinfo[S];
    const float dx = c.x - t.x, dy = c.y - t.y, dz = c.z - t.z;
    return sqrtf(dx * dx + dy * dy + dz * dz) >= kFarFactor * (rg + t.w);
}

// thread 0: decide the path of unit k (flag kept in shared memory for the consumers) and start
// the bulk copy of its source tile into stage `buf`
__device__ __forceinline__ void issue_unit(const Args &a, long long u, float *stage, int *flag,
                                           uint64_t *bar)
{
    const int G = (int)(u / a.ntiles), S = (int)(u - (long long)G * a.ntiles);
    const bool far = is_far(a, G, S);
    *flag = far ? 1 : 0;
    if (far)
        dev::tma_load_1d(stage, a.far_rec + (size_t)S * kRec32F * kTs, kRec32F * kTs * sizeof(float), bar);
    else
        dev::tma_load_1d(stage, a.near_rec + (size_t)S * kRec32 * kTs, kRec32 * kTs * sizeof(float), bar);
}

__global__ void __launch_bounds__(kT, 8) br32_kernel(Args a)
{
    __shared__ __align__(128) float stage[2][kRec32F * kTs];
    // FP64 accumulators of this thread's targets, [component][target r][thread]
    __shared__ double acc[3][kR][kT];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int flag[2];

    const int tid = threadIdx.x;
    const int cta = blockIdx.x;
    const long long u0 = (long long)cta * a.units / a.ctas;
    const long long u1 = (long long)(cta + 1) * a.units / a.ctas;
    const int nu = (int)(u1 - u0);
    const int g_first = (int)(u0 / a.ntiles);

    if (tid == 0) {
        dev::mbar_init(&bar[0], 1);
        dev::mbar_init(&bar[1], 1);
        dev::fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < 2 && k < nu; ++k) issue_unit(a, u0 + k, stage[k], &flag[k], &bar[k]);
    }
    __syncthreads();

#pragma unroll
    for (int r = 0; r < kR; ++r) acc[0][r][tid] = acc[1][r][tid] = acc[2][r][tid] = 0.0;
    int cur_g = -1;
    int t_of[2];  // tiles of the current group (the second repeats the first for kGroup = 1)
    t_of[0] = t_of[1] = 0;
    int bad = 0, kb = 0;

    for (int k = 0; k < nu; ++k) {
        const long long u = u0 + k;
        const int G = (int)(u / a.ntiles), S = (int)(u - (long long)G * a.ntiles);
        if (G != cur_g) {
            if (cur_g >= 0) {
                double *o = a.part + (size_t)(cta * a.kseg + (cur_g - g_first)) * 3 * (kGroup * kTs);
#pragma unroll
                for (int r = 0; r < kR; ++r) {
                    const int idx = (r / (kR / kGroup)) * kTs + (r % (kR / kGroup)) * kT + tid;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        o[c * (kGroup * kTs) + idx] = acc[c][r][tid];
                        acc[c][r][tid] = 0.0;
                    }
                }
            }
            cur_g = G;
            const int ti = G / a.ng2, gj = G - ti * a.ng2;
            t_of[0] = ti * a.nt2 + kGroup * gj;
            t_of[1] = (kGroup > 1 && kGroup * gj + 1 < a.nt2) ? t_of[0] + 1 : t_of[0];
        }
        const int b = k & 1;
        const bool ok = dev::mbar_wait_bounded(&bar[b], (k >> 1) & 1);
        if (ok) {
            const float *s = stage[b];
            if (flag[b]) {
                // ---- far path ------------------------------------------------------------
                const float4 cs = a.tinfo[S];
                u64 m2x[kR], m2y[kR], m2z[kR], bb[kR];
                u64 ax[kR], ay[kR], az[kR], gxs[kR], gys[kR], gzs[kR];
#pragma unroll
                for (int r = 0; r < kR; ++r) {
                    const float *tr = a.near_rec + (size_t)t_of[r / (kR / kGroup)] * kRec32 * kTs +
                                      (r % (kR / kGroup)) * kT + tid;
                    const float tx = (__ldg(tr) - cs.x) + __ldg(tr + 3 * kTs);
                    const float ty = (__ldg(tr + kTs) - cs.y) + __ldg(tr + 4 * kTs);
                    const float tz = (__ldg(tr + 2 * kTs) - cs.z) + __ldg(tr + 5 * kTs);
                    m2x[r] = pack2(-2.0f * tx, -2.0f * tx);
                    m2y[r] = pack2(-2.0f * ty, -2.0f * ty);
                    m2z[r] = pack2(-2.0f * tz, -2.0f * tz);
                    const float b1 = fmaf(tx, tx, fmaf(ty, ty, tz * tz));
                    bb[r] = pack2(b1, b1);
                    ax[r] = ay[r] = az[r] = gxs[r] = gys[r] = gzs[r] = 0ull;
                }
                const u64 *s2 = reinterpret_cast<const u64 *>(s);  // row k, sources (2m, 2m+1)
#pragma unroll 1
                for (int m = 0; m < kTs / 2; ++m) {
                    const u64 sx = s2[m], sy = s2[kTs / 2 + m], sz = s2[kTs + m], sa = s2[3 * (kTs / 2) + m];
                    const u64 gx = s2[2 * kTs + m], gy = s2[5 * (kTs / 2) + m], gz = s2[3 * kTs + m];
                    const u64 mx = s2[7 * (kTs / 2) + m], my = s2[4 * kTs + m], mz = s2[9 * (kTs / 2) + m];
#pragma unroll
                    for (int r = 0; r < kR; ++r) {
                        const u64 q = ffma2(sx, m2x[r], ffma2(sy, m2y[r], ffma2(sz, m2z[r], fadd2(sa, bb[r]))));
                        const u64 iq = rsqrt2(q);
                        const u64 kk = fmul2(fmul2(iq, iq), iq);
                        ax[r] = ffma2(kk, mx, ax[r]);
                        ay[r] = ffma2(kk, my, ay[r]);
                        az[r] = ffma2(kk, mz, az[r]);
                        gxs[r] = ffma2(kk, gx, gxs[r]);
                        gys[r] = ffma2(kk, gy, gys[r]);
                        gzs[r] = ffma2(kk, gz, gzs[r]);
                    }
                }
#pragma unroll
                for (int r = 0; r < kR; ++r) {
                    // t = -m2 / 2 exactly (both lanes of m2 hold -2 t)
                    const float tx = -0.25f * sum2(m2x[r]), ty = -0.25f * sum2(m2y[r]), tz = -0.25f * sum2(m2z[r]);
                    const float bx = sum2(gxs[r]), by = sum2(gys[r]), bz = sum2(gzs[r]);
                    acc[0][r][tid] += (double)(sum2(ax[r]) - fmaf(ty, bz, -tz * by));
                    acc[1][r][tid] += (double)(sum2(ay[r]) - fmaf(tz, bx, -tx * bz));
                    acc[2][r][tid] += (double)(sum2(az[r]) - fmaf(tx, by, -ty * bx));
                }
            } else {
                // ---- near path -----------------------------------------------------------
                float hx[kR], hy[kR], hz[kR], lx[kR], ly[kR], lz[kR], px[kR], py[kR], pz[kR];
#pragma unroll
                for (int r = 0; r < kR; ++r) {
                    const float *tr = a.near_rec + (size_t)t_of[r / (kR / kGroup)] * kRec32 * kTs +
                                      (r % (kR / kGroup)) * kT + tid;
                    hx[r] = __ldg(tr);
                    hy[r] = __ldg(tr + kTs);
                    hz[r] = __ldg(tr + 2 * kTs);
                    lx[r] = __ldg(tr + 3 * kTs);
                    ly[r] = __ldg(tr + 4 * kTs);
                    lz[r] = __ldg(tr + 5 * kTs);
                    px[r] = py[r] = pz[r] = 0.0f;
                }
#pragma unroll 2
                for (int j = 0; j < kTs; ++j) {
                    const float shx = s[j], shy = s[kTs + j], shz = s[2 * kTs + j];
                    const float slx = s[3 * kTs + j], sly = s[4 * kTs + j], slz = s[5 * kTs + j];
                    const float gx = s[6 * kTs + j], gy = s[7 * kTs + j], gz = s[8 * kTs + j];
#pragma unroll
                    for (int r = 0; r < kR; ++r) {
                        const float rx = (shx - hx[r]) + (slx - lx[r]);
                        const float ry = (shy - hy[r]) + (sly - ly[r]);
                        const float rz = (shz - hz[r]) + (slz - lz[r]);
                        const float q = fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, a.d2)));
                        const float iq = dev::rsqrt_approx(q);
                        const float kk = iq * iq * iq;
                        px[r] = fmaf(kk, fmaf(ry, gz, -rz * gy), px[r]);
                        py[r] = fmaf(kk, fmaf(rz, gx, -rx * gz), py[r]);
                        pz[r] = fmaf(kk, fmaf(rx, gy, -ry * gx), pz[r]);
                    }
                }
#pragma unroll
                for (int r = 0; r < kR; ++r) {
                    acc[0][r][tid] += (double)px[r];
                    acc[1][r][tid] += (double)py[r];
                    acc[2][r][tid] += (double)pz[r];
                }
            }
        }
        bad = __syncthreads_or(!ok);
        if (bad) {
            kb = k;
            break;
        }
        if (tid == 0 && k + 2 < nu) {
            dev::fence_proxy_async();
            issue_unit(a, u0 + k + 2, stage[b], &flag[b], &bar[b]);
        }
    }
    if (bad) {
        if (tid == 0) {
            atomicOr(a.err, kErrTimeout);
            for (int k = kb; k < kb + 2 && k < nu; ++k)
                (void)dev::mbar_wait_bounded(&bar[k & 1], (k >> 1) & 1);
        }
        return;
    }
    if (cur_g >= 0) {
        double *o = a.part + (size_t)(cta * a.kseg + (cur_g - g_first)) * 3 * (kGroup * kTs);
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int idx = (r / (kR / kGroup)) * kTs + (r % (kR / kGroup)) * kT + tid;
#pragma unroll
            for (int c = 0; c < 3; ++c) o[c * (kGroup * kTs) + idx] = acc[c][r][tid];
        }
    }
}

// Sum the partials of every target in CTA order, write u in mesh order and Phi = q + |u|^2 / 2.
__global__ void __launch_bounds__(256)
    reduce32_kernel(Args a, const double *__restrict__ q, double *__restrict__ u, double *__restrict__ phi)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.N) return;
    const int i = p / a.n2, j = p - (p / a.n2) * a.n2;
    const int ti = i >> 4, tj = j >> 4;
    const int G = ti * a.ng2 + tj / kGroup;
    const int idx = (tj % kGroup) * kTs + ((i & 15) << 4) + (j & 15);
    const long long first = (long long)G * a.ntiles, last = first + a.ntiles - 1;
    const int c0 = cta_of_unit(first, a.units, a.ctas), c1 = cta_of_unit(last, a.units, a.ctas);
    double s[3] = {0.0, 0.0, 0.0};
    for (int c = c0; c <= c1; ++c) {
        const long long st = (long long)c * a.units / a.ctas;
        const int seg = G - (int)(st / a.ntiles);
        const double *o = a.part + (size_t)(c * a.kseg + seg) * 3 * (kGroup * kTs) + idx;
#pragma unroll
        for (int k = 0; k < 3; ++k) s[k] += o[k * (kGroup * kTs)];
    }
    const size_t N = a.N;
    u[p] = s[0];
    u[N + p] = s[1];
    u[2 * N + p] = s[2];
    phi[p] = q[p] + 0.5 * (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
}

// padding slots: zero strength and |s|^2 + delta^2 = delta^2, so they add exactly nothing
__global__ void init_far_kernel(float *far_rec, size_t nslots_tiles, float d2)
{
    const size_t total = nslots_tiles * kRec32F * kTs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int row = (int)((e / kTs) % kRec32F);
        far_rec[e] = (row == 3) ? d2 : 0.0f;
    }
}

Args make_args(zm_ctx *c)
{
    Args a;
    const Geom &g = c->geom;
    const Tiling &t = c->tiling;
    a.n1 = g.n1;
    a.n2 = g.n2;
    a.N = g.N;
    a.nt2 = t.nt2;
    a.ntiles = t.ntiles;
    a.ng2 = (t.nt2 + kGroup - 1) / kGroup;
    a.ngroups = t.nt1 * a.ng2;
    a.units = (long long)a.ngroups * t.ntiles;
    a.ctas = c->plan32.ctas;
    a.kseg = c->plan32.kseg;
    a.d2 = (float)(c->delta * c->delta);
    a.near_rec = static_cast<const float *>(c->src);
    a.far_rec = c->src_far;
    a.tinfo = c->tinfo;
    a.part = c->part;
    a.err = c->err;
    return a;
}

}  // namespace

Br32Plan plan_br32(const Geom &g, const Tiling &t, int sm_count)
{
    Br32Plan p;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, br32_kernel, kT, 0) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    const int ng2 = (t.nt2 + kGroup - 1) / kGroup;
    const long long units = (long long)t.nt1 * ng2 * t.ntiles;
    p.ctas = (int)std::min<long long>(units, (long long)occ * sm_count);
    const long long lmax = (units + p.ctas - 1) / p.ctas;
    p.kseg = (int)((lmax - 1) / t.ntiles) + 2;
    p.part_doubles = (size_t)p.ctas * p.kseg * 3 * kGroup * kTs;
    p.occupancy = occ;
    return p;
}

int init_far_records(zm_ctx *c)
{
    init_far_kernel<<<256, 256, 0, c->stream>>>(c->src_far, (size_t)c->tiling.ntiles,
                                               (float)(c->delta * c->delta));
    return cuda_check(cudaGetLastError(), "far-record init");
}

int launch_br32(zm_ctx *c)
{
    const Args a = make_args(c);
    cudaEvent_t ev = nullptr;
    prof_begin(c, ZM_K_BR, &ev);
    br32_kernel<<<a.ctas, kT, 0, c->stream>>>(a);
    prof_end(c, ZM_K_BR, ev);
    c->prof.pairs += (int64_t)a.N * (int64_t)a.N;
    int rc = cuda_check(cudaGetLastError(), "Birkhoff-Rott FP32C kernel launch");
    if (rc) return rc;
    prof_begin(c, ZM_K_REDUCE, &ev);
    reduce32_kernel<<<(a.N + 255) / 256, 256, 0, c->stream>>>(a, c->q, c->u, c->phi);
    prof_end(c, ZM_K_REDUCE, ev);
    return cuda_check(cudaGetLastError(), "Birkhoff-Rott FP32C reduction launch");
}

}  // namespace zm
