// zm_br32.cu -- FP32-compensated all-pairs Birkhoff-Rott sum over a batch of interfaces (paper
// Sec. 2 BRSolver, Sec. 3.2.1 ExactBRSolver, the high-order model):
//     u_i = sum_j (z_j - z_i) x gamma'_j / (|z_j - z_i|^2 + delta^2)^(3/2),   i, j in one interface.
//
// Work.  A work item is (interface, target tile, chunk of consecutive source tiles); tiles are
// 16 x 16 mesh patches (256 points).  Persistent CTAs of 64 threads (4 targets per thread, one
// target tile per CTA at a time) take items from a global atomic counter, so near and far tile
// pairs of unequal cost and interfaces of unequal size balance dynamically.  Source tiles
// arrive by 1D bulk TMA (cp.async.bulk) into a double-buffered shared-memory stage; thread 0
// runs ahead one tile, choosing each tile's path and copying the matching record.
//
// Two source paths, per (target tile, source tile), from bounding spheres:
//   near (centres closer than 1.25 x the sum of radii): positions as FP32 hi/lo pairs,
//     r = (zh_j - zh_i) + (zl_j - zl_i), the direct formula -- 23 FP32 + 1 MUFU per pair;
//   far: tile-local coordinates s_j = z_j - c_T and t_i = z_i - c_T (c_T the source tile's
//     centre), |r|^2 + delta^2 in Gram form (|s_j|^2 + delta^2) + |t_i|^2 - 2 s_j . t_i and the
//     cross product split as sum K (s_j x gamma_j) - t_i x sum K gamma_j: 12 FP32 + 1 MUFU per
//     pair.  With the spheres apart, |s|, |t| and |r| are of one order, so neither form loses
//     more than a few units of FP32 rounding.  Two adjacent sources share one packed FP32x2
//     instruction (fma/mul/add .f32x2), which halves issue slots for the same FP32 work.
//
// Cutoff (paper Sec. 3.2.2 CutoffBRSolver: only sources within a 3D distance of the target).
// With a cutoff c, the tile spheres classify each (target tile, source tile): entirely beyond c
// (skipped: no copy, no work), entirely within c (the paths above), or straddling c (the near
// path with a per-pair test |r|^2 <= c^2 on the FP32 hi/lo difference, exact to about 2^-22 in
// the distance; a pair that close to c may fall either way).  Compact tiles of the
// mesh act as the cell list.  A relative margin of 1e-4 on c keeps the sphere decisions on the
// safe side of every pair decision.
//
// Accumulation.  Each (target, source tile) partial is an FP32 sum over 256 sources.  Partials
// are added exactly in 64-bit fixed point, value * 2^S with S per interface chosen from the
// bound |u| <= N max|gamma'| (2 / (3 sqrt 3)) / delta^2 so that no sum can overflow.  Integer
// addition is associative: the result is bitwise the same whatever the scheduling or the
// other interfaces in the batch, and it carries more than FP64's precision across tiles.
// Partials collect in shared memory while a CTA stays on one target tile and reach the
// per-interface accumulators by integer atomics when it moves on.
#include <algorithm>

#include "zm_br32_common.cuh"

namespace zm {
namespace {

#ifndef ZM_BR32_R
#define ZM_BR32_R 4
#endif
constexpr int kR = ZM_BR32_R;   // targets per thread
constexpr int kT = kTs / kR;    // threads per CTA: one target tile per CTA
#ifndef ZM_BR32_FAR
#define ZM_BR32_FAR 1.25f  // far path when the sphere centres are this many times the radii apart
#endif
constexpr float kFarFactor = ZM_BR32_FAR;

// compile-time tuning: unroll of the far loop over source pairs, and the minimum resident CTAs
// per SM the register allocation must allow
#ifndef ZM_BR32_UNROLL
#define ZM_BR32_UNROLL 2
#endif
#ifndef ZM_BR32_MINB
#define ZM_BR32_MINB 7
#endif
constexpr int kFarUnroll = ZM_BR32_UNROLL;

struct Unit {
    int inst;  // -1: no more work
    int tile;  // target tile
    int src;   // source tile
    int far;
};

// kCut: some interface of the batch sums within a cutoff, so straddling tile pairs (masked
// near path) can occur; without it that path is compiled out.
template <bool kCut>
__global__ void __launch_bounds__(kT, ZM_BR32_MINB)
    br32_batch_kernel(const Inst *__restrict__ insts, int ninst, long long nitems,
                      unsigned long long *counter, int *err)
{
    // a stage holds a near record (9 rows) or a far record: s, |s|^2 + delta^2 (rows 0-3) and
    // strength, s x strength (rows kFarRowG .. + 5), as stage rows 0-9
    constexpr int kStageRows = 10;
    __shared__ __align__(128) float stage[2][kStageRows * kTs];
    __shared__ long long acc[3][kR][kT];  // fixed-point partial sums of this thread's targets
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ Unit unit[2];

    const int tid = threadIdx.x;

    // ---- producer state (thread 0) ----
    int p_inst = 0, p_tile = 0, p_next = 0, p_left = 0;
    bool p_done = false;
    auto produce = [&](int buf) {
        while (true) {
            while (p_left == 0 && !p_done) {
                const long long it = (long long)atomicAdd(counter, 1ull);
                if (it >= nitems) {
                    p_done = true;
                    break;
                }
                int lo = 0, hi = ninst - 1;  // last interface with item0 <= it
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (insts[mid].item0 <= it) lo = mid;
                    else hi = mid - 1;
                }
                if (!ZM_IDX_OK(lo, ninst)) continue;
                const Inst &I = insts[lo];
                const long long local = it - I.item0;
                p_inst = lo;
                p_tile = (int)(local / I.nchunks);
                const int ch = (int)(local - (long long)p_tile * I.nchunks);
                p_next = ch * I.chunk;
                p_left = min(I.chunk, I.tiling.ntiles - p_next);
            }
            if (p_done) {
                unit[buf].inst = -1;
                return;
            }
            const Inst &I = insts[p_inst];
            const int S = p_next++;
            --p_left;
            // checked build: a tile number outside the interface's records is skipped
            if (!ZM_IDX_OK(p_tile, I.tiling.ntiles) || !ZM_IDX_OK(S, I.tiling.ntiles)) continue;
            const float4 a = I.tinfo[p_tile], b = I.tinfo[S];
            const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
            const float D = sqrtf(dx * dx + dy * dy + dz * dz);
            int path = (D >= kFarFactor * (a.w + b.w)) ? 1 : 0;  // 1 far, 0 near
            if (I.cutoff > 0.0) {
                const float c = (float)I.cutoff;
                if (D - a.w - b.w > c * 1.0001f) continue;          // every pair beyond c
                if (D + a.w + b.w >= c * 0.9999f) path = 2;         // straddles c: masked near
            }
            unit[buf].inst = p_inst;
            unit[buf].tile = p_tile;
            unit[buf].src = S;
            unit[buf].far = path;
            if (path == 1) {
                const float *rec = I.far_rec + (size_t)S * kRec32F * kTs;
                dev::mbar_expect_tx(&bar[buf], kStageRows * kTs * sizeof(float));
                dev::tma_copy_1d(stage[buf], rec, 4 * kTs * sizeof(float), &bar[buf]);
                dev::tma_copy_1d(stage[buf] + 4 * kTs, rec + kFarRowG * kTs, 6 * kTs * sizeof(float), &bar[buf]);
            } else
                dev::tma_load_1d(stage[buf], I.near_rec + (size_t)S * kRec32 * kTs,
                                 kRec32 * kTs * sizeof(float), &bar[buf]);
            return;
        }
    };

    if (tid == 0) {
        dev::mbar_init(&bar[0], 1);
        dev::mbar_init(&bar[1], 1);
        dev::fence_mbar_init();
    }
#pragma unroll
    for (int r = 0; r < kR; ++r) acc[0][r][tid] = acc[1][r][tid] = acc[2][r][tid] = 0;
    __syncthreads();
    if (tid == 0) {
        produce(0);
        produce(1);
    }
    __syncthreads();

    // ---- consumer state (all threads) ----
    int c_inst = -1, c_tile = -1;
    float c_d2 = 0.0f, c_mult = 1.0f, c_c2 = 0.0f;
    const float *c_near = nullptr;

    auto flush = [&]() {
        if (c_inst < 0) return;
        const Inst &I = insts[c_inst];
        const int ti = c_tile / I.tiling.nt2, tj = c_tile - ti * I.tiling.nt2;
        const size_t N = I.geom.N;
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int slot = r * kT + tid;
            const int lg2 = __ffs(I.tiling.tp2) - 1;  // tp2 is a power of two
            const int i = ti * I.tiling.tp1 + (slot >> lg2), j = tj * I.tiling.tp2 + (slot & (I.tiling.tp2 - 1));
            if (i < I.geom.n1 && j < I.geom.n2 && ZM_IDX_OK((size_t)i * I.geom.n2 + j, N)) {
                const size_t p = (size_t)i * I.geom.n2 + j;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const long long v = acc[c][r][tid];
                    if (v) atomicAdd(&I.ufix[c * N + p], (unsigned long long)v);
                }
            }
            acc[0][r][tid] = acc[1][r][tid] = acc[2][r][tid] = 0;
        }
    };

    int bad = 0, kb = 0;
    for (int k = 0;; ++k) {
        const int b = k & 1;
        const Unit un = unit[b];
        if (un.inst < 0) break;
        const bool ok = dev::mbar_wait_bounded(&bar[b], (k >> 1) & 1);
        if (un.inst != c_inst || un.tile != c_tile) {
            flush();
            if (un.inst != c_inst) {
                const Inst &I = insts[un.inst];
                const int sc = fix_scale(I);
                c_mult = __int_as_float((127 + sc) << 23);  // 2^scale, exact
                c_d2 = (float)(I.delta * I.delta);
                c_c2 = (float)(I.cutoff * I.cutoff);
                c_near = I.near_rec;
                if (tid == 0) *I.scale = sc;
            }
            c_inst = un.inst;
            c_tile = un.tile;
        }
        if (ok) {
            const float *s = stage[b];
            if (un.far == 1) {
                // ---- far path ------------------------------------------------------------
                const float4 cs = insts[c_inst].tinfo[un.src];
                u64 m2x[kR], m2y[kR], m2z[kR], bb[kR];
                u64 ax[kR], ay[kR], az[kR], gxs[kR], gys[kR], gzs[kR];
#pragma unroll
                for (int r = 0; r < kR; ++r) {
                    const float *tr = c_near + (size_t)c_tile * kRec32 * kTs + r * kT + tid;
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
#pragma unroll kFarUnroll
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
                    const float vx = sum2(ax[r]) - fmaf(ty, bz, -tz * by);
                    const float vy = sum2(ay[r]) - fmaf(tz, bx, -tx * bz);
                    const float vz = sum2(az[r]) - fmaf(tx, by, -ty * bx);
                    acc[0][r][tid] += __float2ll_rn(vx * c_mult);
                    acc[1][r][tid] += __float2ll_rn(vy * c_mult);
                    acc[2][r][tid] += __float2ll_rn(vz * c_mult);
                }
            } else if (!kCut || un.far == 0) {
                near_tile<false, kR, kT>(s, c_near + (size_t)c_tile * kRec32 * kTs + tid, c_d2, 0.0f, c_mult, acc, tid);
            } else {
                // the tile pair straddles the cutoff: mask each pair by its FP32 distance
                near_tile<true, kR, kT>(s, c_near + (size_t)c_tile * kRec32 * kTs + tid, c_d2, c_c2, c_mult, acc, tid);
            }
        }
        bad = __syncthreads_or(!ok);
        if (bad) {
            kb = k;
            break;
        }
        if (tid == 0) {
            dev::fence_proxy_async();
            produce(b);  // unit k + 2 into the stage just consumed
        }
    }
    if (bad) {
        if (tid == 0) {
            int flags = kErrTimeout;
            // let copies still in flight (units kb and kb + 1) land before shared memory is
            // released, again with bounded waits
            for (int k = kb; k < kb + 2; ++k)
                if (unit[k & 1].inst >= 0 && !dev::mbar_wait_bounded(&bar[k & 1], (k >> 1) & 1))
                    flags |= kErrDrain;
            atomicOr(err, flags);
        }
        return;
    }
    flush();
}

// padding slots: zero strength and |s|^2 + delta^2 = delta^2, so they add exactly nothing
__global__ void init_far_kernel(float *far_rec, size_t ntiles, float d2)
{
    const size_t total = ntiles * kRec32F * kTs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int row = (int)((e / kTs) % kRec32F);
        far_rec[e] = (row == 3) ? d2 : 0.0f;
    }
}

}  // namespace

int br32_occupancy()
{
    int occ = 0;
    int occ_cut = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, br32_batch_kernel<false>, kT, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_cut, br32_batch_kernel<true>, kT, 0) != cudaSuccess ||
        occ < 1 || occ_cut < 1) {
        cudaGetLastError();
        return 1;
    }
    return std::min(occ, occ_cut);
}

void init_far_records(float *far_rec, int ntiles, float d2, cudaStream_t s)
{
    init_far_kernel<<<256, 256, 0, s>>>(far_rec, (size_t)ntiles, d2);
}

int launch_br32_batch(const Inst *d_insts, int ninst, long long nitems, int ctas,
                      unsigned long long *counter, int *err, cudaStream_t s, bool any_cutoff)
{
    if (any_cutoff)
        br32_batch_kernel<true><<<ctas, kT, 0, s>>>(d_insts, ninst, nitems, counter, err);
    else
        br32_batch_kernel<false><<<ctas, kT, 0, s>>>(d_insts, ninst, nitems, counter, err);
    return cuda_check(cudaGetLastError(), "Birkhoff-Rott FP32C kernel launch");
}

ZM_BOUNDS_READER(bounds_br32)

}  // namespace zm
