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
// This file holds the FP64 variant (every operation in FP64; the kernel (|r|^2 + delta^2)^(-3/2)
// from the hardware reciprocal-square-root estimate and one second-order correction, see
// dev::rsqrt_cube) -- the plain per-instance comparator -- and its allocation-free form; the
// FP32-compensated variant is in zm_br32.cu.  Per pair: 21 FP64 instructions (3 differences,
// 3 FMAs for |r|^2 + delta^2, 6 for the kernel, 6 for the cross product, 3 accumulations) and
// one MUFU operation, for 26 counted flops.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "zm_internal.cuh"

namespace zm {
namespace {

constexpr int kTile1 = 16, kTile2 = 16;  // source tile: 16 x 16 mesh patch, 256 sources

template <int kTpb, int kR, int kTs>
__global__ void __launch_bounds__(kTpb)
    br64_kernel(int N, const double *__restrict__ z, const double *__restrict__ src, int ntiles,
                int tiles_per_split, int qsplit, double d2, double *__restrict__ part, int *err)
{
    constexpr uint32_t kBytes = kRec64 * kTs * sizeof(double);
    __shared__ __align__(128) double sh[2][kRec64 * kTs];
    __shared__ __align__(8) uint64_t bar[2];

    const int tid = threadIdx.x;
    // split blockIdx.y: a range of whole tiles, or (qsplit > 1, small meshes) one
    // 1/qsplit part of one tile's sources
    int t0, nt, j0 = 0, j1 = kTs;
    if (qsplit > 1) {
        t0 = blockIdx.y / qsplit;
        nt = 1;
        j0 = (blockIdx.y - t0 * qsplit) * (kTs / qsplit);
        j1 = j0 + kTs / qsplit;
    } else {
        t0 = blockIdx.y * tiles_per_split;
        nt = max(0, min(ntiles, t0 + tiles_per_split) - t0);
    }
    // checked build: every tile this CTA copies must exist, and the source slice lie in a tile
    if (nt > 0 && (!ZM_IDX_OK(t0, ntiles) || !ZM_IDX_OK(t0 + nt - 1, ntiles) || !ZM_IDX_OK(j0, kTs) ||
                   !ZM_IDX_OK(j1 - 1, kTs)))
        nt = 0;

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
            for (int jj = j0; jj < j1; ++jj) {
                const double sx = s[jj], sy = s[kTs + jj], sz = s[2 * kTs + jj];
                const double gx = s[3 * kTs + jj], gy = s[4 * kTs + jj], gz = s[5 * kTs + jj];
#pragma unroll
                for (int r = 0; r < kR; ++r) {
                    const double rx = sx - tx[r], ry = sy - ty[r], rz = sz - tz[r];
                    const double q = fma(rx, rx, fma(ry, ry, fma(rz, rz, d2)));
                    const double kk = dev::rsqrt_cube(q);
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
            int flags = kErrTimeout;
            // let the copies still in flight (tiles kb and kb + 1) land, again with a bounded
            // wait, before the CTA's shared memory is released
            for (int k = kb; k < kb + 2 && k < nt; ++k)
                if (!dev::mbar_wait_bounded(&bar[k & 1], (k >> 1) & 1)) flags |= kErrDrain;
            atomicOr(err, flags);
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int p = blockIdx.x * kTpb * kR + r * kTpb + tid;
        if (p < N && ZM_IDX_OK(p, N)) {
            double *o = part + (size_t)blockIdx.y * 3 * N;
            o[p] = ax[r];
            o[(size_t)N + p] = ay[r];
            o[2 * (size_t)N + p] = az[r];
        }
    }
}

constexpr int kTpb64 = 128, kR64 = 2;
constexpr int kTpb64s = 32;  // small meshes: one warp per target block

}  // namespace

Tiling make_tiling_shape(const Geom &g, int tp1, int tp2)
{
    Tiling t;
    t.tp1 = tp1;
    t.tp2 = tp2;
    t.ts = tp1 * tp2;
    t.nt1 = (g.n1 + tp1 - 1) / tp1;
    t.nt2 = (g.n2 + tp2 - 1) / tp2;
    t.ntiles = t.nt1 * t.nt2;
    return t;
}

Tiling make_tiling(const Geom &g) { return make_tiling_shape(g, kTile1, kTile2); }

BrPlan plan_br(const Geom &g, const Tiling &t, int sm_count)
{
    BrPlan p;
    p.tpb = kTpb64;
    p.r = kR64;
    p.qsplit = 1;
    const int want = 4 * sm_count;  // about four resident CTAs per SM over the grid
    p.ntb = (g.N + p.tpb * p.r - 1) / (p.tpb * p.r);
    if ((long long)p.ntb * t.ntiles < want) {
        // small mesh: one-warp target blocks and sources split below a tile
        p.tpb = kTpb64s;
        p.ntb = (g.N + p.tpb * p.r - 1) / (p.tpb * p.r);
        p.qsplit = 1;
        // up to 16 slices of 16 sources: a 32^2 mesh then runs 1024 one-warp CTAs (~7 per SM)
        while (p.qsplit < 16 && (long long)p.ntb * t.ntiles * p.qsplit < want) p.qsplit *= 2;
        if (p.qsplit > 1) {
            p.tiles_per_split = 1;
            p.nsplit = t.ntiles * p.qsplit;
            return p;
        }
    }
    int ns = (want + p.ntb - 1) / p.ntb;
    ns = std::max(1, std::min(ns, t.ntiles));
    p.tiles_per_split = (t.ntiles + ns - 1) / ns;
    p.nsplit = (t.ntiles + p.tiles_per_split - 1) / p.tiles_per_split;
    return p;
}

int launch_br(zm_ctx *c, const double *y)
{
    if (!y || !c->src || !c->part) return set_error(ZM_ERR_INVALID, "Birkhoff-Rott pass: missing buffer");
    const Geom &g = c->geom;
    const BrPlan &p = c->plan;
    dim3 grid(p.ntb, p.nsplit);
    cudaEvent_t ev = nullptr;
    prof_begin(c, ZM_K_BR, &ev);
    if (p.tpb == kTpb64s)
        br64_kernel<kTpb64s, kR64, kTile1 * kTile2><<<grid, kTpb64s, 0, c->stream>>>(
            g.N, y, static_cast<const double *>(c->src), c->tiling.ntiles, p.tiles_per_split,
            p.qsplit, c->delta * c->delta, c->part, c->err);
    else
        br64_kernel<kTpb64, kR64, kTile1 * kTile2><<<grid, kTpb64, 0, c->stream>>>(
            g.N, y, static_cast<const double *>(c->src), c->tiling.ntiles, p.tiles_per_split,
            p.qsplit, c->delta * c->delta, c->part, c->err);
    prof_end(c, ZM_K_BR, ev);
    c->prof.acc.pairs += (int64_t)g.N * (int64_t)g.N;
    return cuda_check(cudaGetLastError(), "Birkhoff-Rott kernel launch");
}

}  // namespace zm

// ---- Birkhoff-Rott sum that allocates nothing ------------------------------------------------
// A variant of the FP64 all-pairs sum for callers that cannot allocate device memory (for
// example a host application that reserves all GPU memory up front and forbids allocation
// afterwards, or code that must not trigger the device-wide synchronisation cudaMalloc and
// cudaFree imply).  Its workspace -- the tile-major source records, the split partial sums and
// a status word -- lives in one file-scope device array that every GPU loading this library
// holds until the process exits.

namespace zm {
namespace {

constexpr int kNaMaxN = 65536;                        // largest supported point count
constexpr int kNaTs = kTile1 * kTile2;                // 256 sources per tile
constexpr int kNaMaxTiles = kNaMaxN / kNaTs;          // 256
constexpr int kNaSplits = 4;                          // source splits (partial sums)
constexpr size_t kNaHead = 32;                        // 256 bytes: status word, padding
constexpr size_t kNaRec = (size_t)kNaMaxTiles * kRec64 * kNaTs;   // 3 MiB of records
constexpr size_t kNaPart = (size_t)kNaSplits * 3 * kNaMaxN;       // 6 MiB of partials
constexpr size_t kNaDoubles = kNaHead + kNaRec + kNaPart;         // 9 MiB + 256 B in total

}  // namespace
}  // namespace zm

static __device__ __align__(256) double zm_noalloc_scratch[zm::kNaDoubles];

namespace zm {
namespace {

// Records for this call: every slot of every used tile is written (padding slots with zero
// strength), so nothing left by an earlier call is read.  Also clears the status word.
__global__ void na_pack_kernel(int n, int ntiles, const double *__restrict__ z,
                               const double *__restrict__ gamma, double *__restrict__ rec,
                               int *status)
{
    const size_t total = (size_t)ntiles * kRec64 * kNaTs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int slot = (int)(e % kNaTs);
        const int row = (int)((e / kNaTs) % kRec64);
        const int tile = (int)(e / ((size_t)kNaTs * kRec64));
        const int p = tile * kNaTs + slot;
        double v = 0.0;
        if (p < n) v = (row < 3) ? z[(size_t)row * n + p] : gamma[(size_t)(row - 3) * n + p];
        rec[e] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *status = 0;
}

// A CTA whose bounded wait gave up wrote no partial sums, so the workspace may hold an earlier
// call's: u is then filled with NaN, which shows the failure even to a caller without `status`.
__global__ void na_reduce_kernel(int n, int nsplit, const double *__restrict__ part,
                                 double *__restrict__ u, const int *status_in, int32_t *status_out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool failed = (*status_in & kErrTimeout) != 0;
    if (p < n) {
        double s[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < nsplit; ++k)
            for (int c = 0; c < 3; ++c) s[c] += part[((size_t)k * 3 + c) * n + p];
        for (int c = 0; c < 3; ++c) u[(size_t)c * n + p] = failed ? __longlong_as_double(0x7ff8000000000000LL) : s[c];
    }
    if (status_out && p == 0) *status_out = failed ? ZM_ERR_TIMEOUT : ZM_OK;
}

std::mutex g_na_mutex;
constexpr int kNaMaxDevices = 64;
double *g_na_base[kNaMaxDevices];  // device address of zm_noalloc_scratch, per device

// Once per device, with that device current: look up the array's device address.  In host
// code the symbol names a host-side shadow, never the device memory itself.
int na_scratch(double **out)
{
    int dev = -1;
    int rc = cuda_check(cudaGetDevice(&dev), "zm_br_velocity_noalloc: cudaGetDevice");
    if (rc) return rc;
    if (dev < 0 || dev >= kNaMaxDevices)
        return set_error(ZM_ERR_UNSUPPORTED, "zm_br_velocity_noalloc: device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_base[dev]) {
        void *p = nullptr;
        rc = cuda_check(cudaGetSymbolAddress(&p, zm_noalloc_scratch),
                        "zm_br_velocity_noalloc: cudaGetSymbolAddress");
        if (rc) return rc;
        g_na_base[dev] = static_cast<double *>(p);
    }
    *out = g_na_base[dev];
    return ZM_OK;
}

// Device memory of the current device, or managed memory.  Memory of another GPU is refused:
// without peer access the kernels would fault on it.
bool on_device(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace
ZM_BOUNDS_READER(bounds_br)

}  // namespace zm

extern "C" int zm_br_velocity_noalloc(int32_t n, const double *z, const double *gamma,
                                      double delta, double *u, int32_t *status,
                                      void *cuda_stream)
{
    using namespace zm;
    if (n < 1 || n > kNaMaxN)
        return set_error(ZM_ERR_INVALID,
                         "zm_br_velocity_noalloc: n must be in [1, 65536] (size of the static workspace)");
    if (!z || !gamma || !u || !(delta > 0) || !std::isfinite(delta))
        return set_error(ZM_ERR_INVALID, "zm_br_velocity_noalloc: null pointer or delta <= 0");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ZM_ERR_INVALID, "zm_br_velocity_noalloc: no current CUDA device");
    }
    if (!on_device(z, dev) || !on_device(gamma, dev) || !on_device(u, dev) ||
        (status && !on_device(status, dev)))
        return set_error(ZM_ERR_INVALID,
                         "zm_br_velocity_noalloc: z, gamma, u, status must be memory of the current device");
    double *base = nullptr;
    int rc = na_scratch(&base);
    if (rc) return rc;
    int *flag = reinterpret_cast<int *>(base);
    double *rec = base + kNaHead;
    double *part = rec + kNaRec;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    const int ntiles = (n + kNaTs - 1) / kNaTs;
    const int tps = (ntiles + kNaSplits - 1) / kNaSplits;
    const int nsplit = (ntiles + tps - 1) / tps;
    na_pack_kernel<<<std::min(1024, (ntiles * kRec64 * kNaTs + 255) / 256), 256, 0, s>>>(
        n, ntiles, z, gamma, rec, flag);
    const int per_cta = kTpb64 * kR64;
    dim3 grid((n + per_cta - 1) / per_cta, nsplit);
    br64_kernel<kTpb64, kR64, kNaTs><<<grid, kTpb64, 0, s>>>(n, z, rec, ntiles, tps, 1, delta * delta,
                                                             part, flag);
    na_reduce_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, nsplit, part, u, flag, status);
    return cuda_check(cudaGetLastError(), "zm_br_velocity_noalloc: launch");
}
