// zm_br.cu -- the exact all-pairs desingularised Birkhoff-Rott sum (paper Sec. 2 BRSolver,
// Sec. 3.2.1 ExactBRSolver, the high-order model):
//     u_i = sum_j (z_j - z_i) x gamma'_j / (|z_j - z_i|^2 + delta^2)^(3/2),
// with gamma'_j = (dx1 dx2 / 4 pi) (w1 a2 - w2 a1)_j prepared by the geometry pass; this equals
// -(dx1 dx2 / 4 pi) sum_j (z_i - z_j) x gamma_j / (...)^(3/2).
//
// GB300 design.  One CTA owns tpb * R targets (R per thread, held in registers) and sweeps a
// contiguous range of source tiles (grid.y splits the sources so that small meshes still fill
// 152 SMs).  Each tile's records are one contiguous block in HBM and arrive in shared memory by
// a single 1D bulk TMA copy (cp.async.bulk) completing on an mbarrier, double-buffered so the
// next tile lands while the current one is swept.  Every thread reads the same source at the
// same time (shared-memory broadcast), so the loop is bound by the FP32 (or FP64) pipe, not by
// memory.  Split partial sums go to a [nsplit][3][N] workspace reduced in a fixed order by the
// reduction kernel, which keeps results deterministic.
//
// Precision variants:
//   FP64:  every operation in FP64 (rsqrt from CUDA's double-precision math library).
//   FP32C: positions as FP32 hi/lo pairs, so r = (zh_j - zh_i) + (zl_j - zl_i) keeps near-pair
//          differences accurate to FP32 relative precision; pair terms in FP32 with one MUFU
//          rsqrt; per-tile FP32 partials; FP64 accumulation across tiles.
#include <algorithm>

#include "zm_internal.cuh"

namespace zm {
namespace {

constexpr int kTile1 = 16, kTile2 = 16;  // source tile: 16 x 16 mesh patch, 256 sources

template <int kTpb, int kR, int kTs>
__global__ void __launch_bounds__(kTpb)
    br64_kernel(int N, const double *__restrict__ z, const double *__restrict__ src, int ntiles,
                int tiles_per_split, double d2, double *__restrict__ part, int *err)
{
    constexpr uint32_t kBytes = kRec64 * kTs * sizeof(double);
    __shared__ __align__(128) double sh[2][kRec64 * kTs];
    __shared__ __align__(8) uint64_t bar[2];

    const int tid = threadIdx.x;
    const int t0 = blockIdx.y * tiles_per_split;
    const int nt = max(0, min(ntiles, t0 + tiles_per_split) - t0);

    double tx[kR], ty[kR], tz[kR], ax[kR], ay[kR], az[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int p = min(blockIdx.x * kTpb * kR + r * kTpb + tid, N - 1);
        tx[r] = z[p];
        ty[r] = z[(size_t)N + p];
        tz[r] = z[2 * (size_t)N + p];
        ax[r] = ay[r] = az[r] = 0.0;
    }

    if (tid == 0) {
        dev::mbar_init(&bar[0], 1);
        dev::mbar_init(&bar[1], 1);
        dev::fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < 2 && k < nt; ++k)
            dev::tma_load_1d(sh[k], src + (size_t)(t0 + k) * kRec64 * kTs, kBytes, &bar[k]);
    }

    int bad = 0, kb = 0;
    for (int k = 0; k < nt; ++k) {
        const int b = k & 1;
        const bool ok = dev::mbar_wait_bounded(&bar[b], (k >> 1) & 1);
        if (ok) {
            const double *s = sh[b];
#pragma unroll 2
            for (int jj = 0; jj < kTs; ++jj) {
                const double sx = s[jj], sy = s[kTs + jj], sz = s[2 * kTs + jj];
                const double gx = s[3 * kTs + jj], gy = s[4 * kTs + jj], gz = s[5 * kTs + jj];
#pragma unroll
                for (int r = 0; r < kR; ++r) {
                    const double rx = sx - tx[r], ry = sy - ty[r], rz = sz - tz[r];
                    const double q = fma(rx, rx, fma(ry, ry, fma(rz, rz, d2)));
                    const double iq = rsqrt(q);
                    const double kk = iq * iq * iq;
                    ax[r] = fma(kk, ry * gz - rz * gy, ax[r]);
                    ay[r] = fma(kk, rz * gx - rx * gz, ay[r]);
                    az[r] = fma(kk, rx * gy - ry * gx, az[r]);
                }
            }
        }
        bad = __syncthreads_or(!ok);
        if (bad) {
            kb = k;
            break;
        }
        if (tid == 0 && k + 2 < nt) {
            dev::fence_proxy_async();
            dev::tma_load_1d(sh[b], src + (size_t)(t0 + k + 2) * kRec64 * kTs, kBytes, &bar[b]);
        }
    }
    if (bad) {
        if (tid == 0) {
            atomicOr(err, kErrTimeout);
            // let the copies still in flight (tiles kb and kb + 1) land, again with a bounded
            // wait, before the CTA's shared memory is released
            for (int k = kb; k < kb + 2 && k < nt; ++k)
                (void)dev::mbar_wait_bounded(&bar[k & 1], (k >> 1) & 1);
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int p = blockIdx.x * kTpb * kR + r * kTpb + tid;
        if (p < N) {
            double *o = part + (size_t)blockIdx.y * 3 * N;
            o[p] = ax[r];
            o[(size_t)N + p] = ay[r];
            o[2 * (size_t)N + p] = az[r];
        }
    }
}

template <int kTpb, int kR, int kTs>
__global__ void __launch_bounds__(kTpb)
    br32c_kernel(int N, const double *__restrict__ z, const float *__restrict__ src, int ntiles,
                 int tiles_per_split, float d2, double *__restrict__ part, int *err)
{
    constexpr uint32_t kBytes = kRec32 * kTs * sizeof(float);
    __shared__ __align__(128) float sh[2][kRec32 * kTs];
    __shared__ __align__(8) uint64_t bar[2];

    const int tid = threadIdx.x;
    const int t0 = blockIdx.y * tiles_per_split;
    const int nt = max(0, min(ntiles, t0 + tiles_per_split) - t0);

    float hx[kR], hy[kR], hz[kR], lx[kR], ly[kR], lz[kR];
    double ax[kR], ay[kR], az[kR];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int p = min(blockIdx.x * kTpb * kR + r * kTpb + tid, N - 1);
        const double x = z[p], y = z[(size_t)N + p], w = z[2 * (size_t)N + p];
        hx[r] = __double2float_rn(x);
        hy[r] = __double2float_rn(y);
        hz[r] = __double2float_rn(w);
        lx[r] = __double2float_rn(x - (double)hx[r]);
        ly[r] = __double2float_rn(y - (double)hy[r]);
        lz[r] = __double2float_rn(w - (double)hz[r]);
        ax[r] = ay[r] = az[r] = 0.0;
    }

    if (tid == 0) {
        dev::mbar_init(&bar[0], 1);
        dev::mbar_init(&bar[1], 1);
        dev::fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < 2 && k < nt; ++k)
            dev::tma_load_1d(sh[k], src + (size_t)(t0 + k) * kRec32 * kTs, kBytes, &bar[k]);
    }

    int bad = 0, kb = 0;
    for (int k = 0; k < nt; ++k) {
        const int b = k & 1;
        const bool ok = dev::mbar_wait_bounded(&bar[b], (k >> 1) & 1);
        if (ok) {
            const float *s = sh[b];
            float px[kR], py[kR], pz[kR];
#pragma unroll
            for (int r = 0; r < kR; ++r) px[r] = py[r] = pz[r] = 0.0f;
#pragma unroll 2
            for (int jj = 0; jj < kTs; ++jj) {
                const float shx = s[jj], shy = s[kTs + jj], shz = s[2 * kTs + jj];
                const float slx = s[3 * kTs + jj], sly = s[4 * kTs + jj], slz = s[5 * kTs + jj];
                const float gx = s[6 * kTs + jj], gy = s[7 * kTs + jj], gz = s[8 * kTs + jj];
#pragma unroll
                for (int r = 0; r < kR; ++r) {
                    const float rx = (shx - hx[r]) + (slx - lx[r]);
                    const float ry = (shy - hy[r]) + (sly - ly[r]);
                    const float rz = (shz - hz[r]) + (slz - lz[r]);
                    const float q = fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, d2)));
                    const float iq = dev::rsqrt_approx(q);
                    const float kk = iq * iq * iq;
                    px[r] = fmaf(kk, fmaf(ry, gz, -rz * gy), px[r]);
                    py[r] = fmaf(kk, fmaf(rz, gx, -rx * gz), py[r]);
                    pz[r] = fmaf(kk, fmaf(rx, gy, -ry * gx), pz[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < kR; ++r) {
                ax[r] += (double)px[r];
                ay[r] += (double)py[r];
                az[r] += (double)pz[r];
            }
        }
        bad = __syncthreads_or(!ok);
        if (bad) {
            kb = k;
            break;
        }
        if (tid == 0 && k + 2 < nt) {
            dev::fence_proxy_async();
            dev::tma_load_1d(sh[b], src + (size_t)(t0 + k + 2) * kRec32 * kTs, kBytes, &bar[b]);
        }
    }
    if (bad) {
        if (tid == 0) {
            atomicOr(err, kErrTimeout);
            // let the copies still in flight (tiles kb and kb + 1) land, again with a bounded
            // wait, before the CTA's shared memory is released
            for (int k = kb; k < kb + 2 && k < nt; ++k)
                (void)dev::mbar_wait_bounded(&bar[k & 1], (k >> 1) & 1);
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int p = blockIdx.x * kTpb * kR + r * kTpb + tid;
        if (p < N) {
            double *o = part + (size_t)blockIdx.y * 3 * N;
            o[p] = ax[r];
            o[(size_t)N + p] = ay[r];
            o[2 * (size_t)N + p] = az[r];
        }
    }
}

constexpr int kTpb64 = 128, kR64 = 2;
constexpr int kTpb32 = 256, kR32 = 4;

}  // namespace

Tiling make_tiling(const Geom &g)
{
    Tiling t;
    t.tp1 = kTile1;
    t.tp2 = kTile2;
    t.ts = kTile1 * kTile2;
    t.nt1 = (g.n1 + kTile1 - 1) / kTile1;
    t.nt2 = (g.n2 + kTile2 - 1) / kTile2;
    t.ntiles = t.nt1 * t.nt2;
    return t;
}

BrPlan plan_br(const Geom &g, const Tiling &t, int fp32c, int sm_count)
{
    BrPlan p;
    p.tpb = fp32c ? kTpb32 : kTpb64;
    p.r = fp32c ? kR32 : kR64;
    const int per_cta = p.tpb * p.r;
    p.ntb = (g.N + per_cta - 1) / per_cta;
    // aim for about four resident CTAs per SM over the whole grid
    const int want = 4 * sm_count;
    int ns = (want + p.ntb - 1) / p.ntb;
    ns = std::max(1, std::min(ns, t.ntiles));
    p.tiles_per_split = (t.ntiles + ns - 1) / ns;
    p.nsplit = (t.ntiles + p.tiles_per_split - 1) / p.tiles_per_split;
    return p;
}

int launch_br(zm_ctx *c, const double *y)
{
    const Geom &g = c->geom;
    const BrPlan &p = c->plan;
    dim3 grid(p.ntb, p.nsplit);
    cudaEvent_t ev = nullptr;
    prof_begin(c, ZM_K_BR, &ev);
    const double d2 = c->delta * c->delta;
    if (c->fp32c) {
        br32c_kernel<kTpb32, kR32, kTile1 * kTile2><<<grid, kTpb32, 0, c->stream>>>(
            g.N, y, static_cast<const float *>(c->src), c->tiling.ntiles, p.tiles_per_split,
            (float)d2, c->part, c->err);
    } else {
        br64_kernel<kTpb64, kR64, kTile1 * kTile2><<<grid, kTpb64, 0, c->stream>>>(
            g.N, y, static_cast<const double *>(c->src), c->tiling.ntiles, p.tiles_per_split, d2,
            c->part, c->err);
    }
    prof_end(c, ZM_K_BR, ev);
    c->prof.pairs += (int64_t)g.N * (int64_t)g.N;
    return cuda_check(cudaGetLastError(), "Birkhoff-Rott kernel launch");
}

}  // namespace zm
