// zm_br32tc.cu -- FP32-compensated all-pairs Birkhoff-Rott sum over a batch of interfaces with
// the far-field accumulation on the tensor cores (paper Sec. 2 BRSolver, Sec. 3.2.1
// ExactBRSolver, the high-order model):
//     u_i = sum_j (z_j - z_i) x gamma'_j / (|z_j - z_i|^2 + delta^2)^(3/2),   i, j in one interface.
//
// Work units, near/far classification, cutoff handling and fixed-point accumulation are those of
// zm_br32.cu (same work items, same tile spheres, same 64-bit fixed point); what differs is how
// a far (target tile, source tile) pair is summed.  In tile-local coordinates (s_j = z_j - c_S,
// t_i = z_i - c_S) a far pair contributes K_ij (s_j x g_j) - t_i x K_ij g_j with
// K_ij = (|s_j - t_i|^2 + delta^2)^(-3/2), so the tile's contribution to target i is
//     v_i = sum_j K_ij m_j - t_i x sum_j K_ij g_j,   m_j = s_j x g_j,
// and the two sums are one matrix product: the 256 x 256 matrix K times the tile's 256 x 6 source
// matrix [g | m].  The CUDA cores form K (|s - t|^2 + delta^2 in Gram form, one MUFU rsqrt, its
// cube: 6 FP32 lane operations per pair, packed two per instruction); the tensor cores do the
// product (tcgen05.mma kind::tf32, accumulating in FP32 in tensor memory).  Each operand is split
// into a TF32 part and a TF32 rest (K = Kh + Kl, B = Bh + Bl), and with B's columns laid out as
// [Bh | Bl] (16 columns) two MMAs per 8 sources, Kh [Bh | Bl] + Kl [Bh | Bl], give all four
// partial products; their column pairs are added when tensor memory is read.  That keeps about
// 21 significant bits per product, the accuracy of the FP32 path (a float32 emulation at 256^2:
// 6.7e-8 against 6.4e-8 relative L2 for the CUDA-core far path).  Near pairs (spheres closer
// than 1.25 x the radii) stay on the CUDA cores with FP32 hi/lo differences.
//
// Measured on GB300 (256^2, one launch, three CTAs per SM): 3.22 ms against 1.89 ms for the
// CUDA-core far path of zm_br32.cu, so it is not the default (ZM_FAR_TENSOR selects it).  The
// hand-offs bound it, not arithmetic: without the MMAs it takes 3.00 ms, without the K
// arithmetic 2.48 ms.  The 6-column product gives MMAs of M = 128, N = 16, K = 8, four per
// 8-source block (two row groups x Kh, Kl); one thread issues a tcgen05.mma every ~46 cycles
// whatever N, so a block costs ~184 cycles of issue against ~128 cycles of MUFU work for its K
// values, and with two A slots (128 tensor-memory columns per CTA) the compute warps wait on MMA
// completion.  Polling waits and deeper A pipelines did not help.
//
// CTA: 6 warps.  Warps 0-3 compute (thread t owns targets t and t + 128 of the target tile, TMEM
// lanes t in two 128-row groups); warp 4 lane 0 produces work units (work items from a global
// atomic counter, tile records by 1D bulk TMA into a double-buffered stage); warp 5 lane 0 issues
// the MMAs.  Hand-offs are mbarriers: record full / free per stage, A slot full / empty per
// 8-source block (K values in tensor memory), D full / empty per accumulation segment (two
// accumulator buffers; the compute warps add segment q after submitting segment q + 1).  Every wait is bounded: a wait that gives up sets the status word, and the role
// leaves its loop; the others then give up in turn.
//
// Tensor memory (128 columns per CTA): D, two buffers x two row groups x 16 columns (columns
// 0-63); A, two slots x two row groups x (8 columns Kh + 8 columns Kl) (columns 64-127).
#include <algorithm>

#include "zm_br32_common.cuh"
#include "zm_tc.cuh"

namespace zm {
namespace {

constexpr int kCW = 4;            // compute warps
constexpr int kCT = kCW * 32;     // compute threads: 128 rows per group
constexpr int kThreads = kCT + 64;  // + producer warp + MMA warp
#ifndef ZM_BR32TC_NA
#define ZM_BR32TC_NA 2
#endif
constexpr int kNA = ZM_BR32TC_NA;  // A slots (8-source blocks in flight)
constexpr int kBlocks = kTs / 8;  // 8-source blocks per source tile
// Accumulation segments: the MMAs accumulate in tensor memory over kSeg blocks only, then start
// a fresh accumulator; the compute warps add the segments in FP32 registers (round to nearest).
// The tensor cores' FP32 accumulation truncates toward zero, so its error grows with the length
// of an accumulation chain and does not average out (a 64-MMA chain per tile gave 1.6e-6
// relative L2 at 256^2).
#ifndef ZM_BR32TC_SEG
#define ZM_BR32TC_SEG 2
#endif
constexpr int kSeg = ZM_BR32TC_SEG;
static_assert(kBlocks % kSeg == 0, "segments must tile the source blocks");
constexpr uint32_t kColD = 0, kColA = 64;
constexpr uint32_t kTmemNeed = kColA + 32 * kNA;
constexpr uint32_t kTmemCols = kTmemNeed <= 128 ? 128 : kTmemNeed <= 256 ? 256 : 512;
constexpr int kStageRows = 20;    // far: s, |s|^2 + delta^2, B (rows 0-19 of the record); near: 9 rows
constexpr float kFarFactor = 1.25f;
#ifndef ZM_BR32TC_MINB
#define ZM_BR32TC_MINB (ZM_BR32TC_NA <= 2 ? 3 : 2)
#endif
// K-major, no swizzle: which descriptor field holds the K-direction stride
#ifndef ZM_TC_LBO_IS_K
#define ZM_TC_LBO_IS_K 1
#endif
constexpr uint32_t kLbo = ZM_TC_LBO_IS_K ? kTcStrideK : kTcStrideN;
constexpr uint32_t kSbo = ZM_TC_LBO_IS_K ? kTcStrideN : kTcStrideK;
constexpr uint32_t kIdesc = tc::idesc_tf32(128, 16);

// Bounded wait on a phase; false (and the status word set) if it gave up.  (Polling first,
// mbarrier.test_wait in a loop, or a 64 ns suspend hint measured no faster.)
__device__ __forceinline__ bool wait_or_flag(uint64_t *bar, uint32_t parity, int *err)
{
    if (dev::mbar_wait_bounded(bar, parity)) return true;
    atomicOr(err, kErrTimeout);
    return false;
}

// The same for a whole warp: lane 0 waits, and the warp goes on only if it saw the phase
// complete (so that the warp-collective tensor-memory moves after it stay converged).
__device__ __forceinline__ bool warp_wait_or_flag(uint64_t *bar, uint32_t parity, int *err)
{
    bool ok = true;
    if ((threadIdx.x & 31) == 0) ok = wait_or_flag(bar, parity, err);
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    __syncwarp();  // the lanes see what lane 0 acquired
    return ok;
}

struct Unit {
    int inst;  // -1: no more work
    int tile;  // target tile
    int src;   // source tile
    int path;  // 0 near, 1 far, 2 near masked at the cutoff
};

template <bool kCut>
__global__ void __launch_bounds__(kThreads, ZM_BR32TC_MINB)
    br32tc_kernel(const Inst *__restrict__ insts, int ninst, long long nitems, unsigned long long *counter,
                  int *err)
{
    __shared__ __align__(1024) float stage[2][kStageRows * kTs];
    __shared__ long long acc[3][2][kCT];
    __shared__ __align__(8) uint64_t rec_full[2], rec_free[2], a_full[kNA], a_empty[kNA], d_full[2], d_empty[2];
    __shared__ __align__(8) uint64_t mma_drain;
    __shared__ Unit unit[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int k = 0; k < 2; ++k) {
            dev::mbar_init(&rec_full[k], 1);
            dev::mbar_init(&rec_free[k], kCW + 1);
            dev::mbar_init(&d_full[k], 1);
            dev::mbar_init(&d_empty[k], kCW);
        }
        for (int k = 0; k < kNA; ++k) {
            dev::mbar_init(&a_full[k], kCW);
            dev::mbar_init(&a_empty[k], 1);
        }
        dev::mbar_init(&mma_drain, 1);
        dev::fence_mbar_init();
        abort_flag = 0;
    }
    if (warp == 0) {
        tc::alloc(&tmem_base, kTmemCols);
        tc::relinquish();
    }
    if (tid < kCT) {
#pragma unroll
        for (int r = 0; r < 2; ++r) acc[0][r][tid] = acc[1][r][tid] = acc[2][r][tid] = 0;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = tmem_base;

    if (warp == kCW) {
        // ---------------- producer: work units and their records ----------------
        if (lane == 0) {
            int p_inst = 0, p_tile = 0, p_next = 0, p_left = 0;
            bool done = false, clean = false;
            int last_copy[2] = {-1, -1};  // unit whose record was last copied into each stage
            for (int u = 0;; ++u) {
                const int s = u & 1;
                if (u >= 2 && !wait_or_flag(&rec_free[s], ((u - 2) >> 1) & 1, err)) break;
                if (*(volatile int *)&abort_flag) break;
                Unit un;
                un.inst = -1;
                while (!done) {
                    while (p_left == 0 && !done) {
                        const long long it = (long long)atomicAdd(counter, 1ull);
                        if (it >= nitems) {
                            done = true;
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
                    if (done) break;
                    const Inst &I = insts[p_inst];
                    const int S = p_next++;
                    --p_left;
                    if (!ZM_IDX_OK(p_tile, I.tiling.ntiles) || !ZM_IDX_OK(S, I.tiling.ntiles)) continue;
                    const float4 a = I.tinfo[p_tile], b = I.tinfo[S];
                    const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
                    const float D = sqrtf(dx * dx + dy * dy + dz * dz);
                    int path = (D >= kFarFactor * (a.w + b.w)) ? 1 : 0;
                    if (kCut && I.cutoff > 0.0) {
                        const float c = (float)I.cutoff;
                        if (D - a.w - b.w > c * 1.0001f) continue;   // every pair beyond c
                        if (D + a.w + b.w >= c * 0.9999f) path = 2;  // straddles c: masked near
                    }
                    un.inst = p_inst;
                    un.tile = p_tile;
                    un.src = S;
                    un.path = path;
                    break;
                }
                unit[s] = un;
                if (un.inst < 0) {
                    dev::mbar_arrive(&rec_full[s]);  // the end marker
                    clean = true;
                    break;
                }
                last_copy[s] = u;
                const Inst &I = insts[un.inst];
                if (un.path == 1) {
                    dev::mbar_expect_tx(&rec_full[s], kStageRows * kTs * sizeof(float));
                    dev::tma_copy_1d(stage[s], I.far_rec + (size_t)un.src * kRec32F * kTs,
                                     kStageRows * kTs * sizeof(float), &rec_full[s]);
                } else {
                    dev::mbar_expect_tx(&rec_full[s], kRec32 * kTs * sizeof(float));
                    dev::tma_copy_1d(stage[s], I.near_rec + (size_t)un.src * kRec32 * kTs,
                                     kRec32 * kTs * sizeof(float), &rec_full[s]);
                }
            }
            // after an abnormal exit, let this thread's copies still in flight land before the
            // CTA's shared memory is released (bounded as well)
            if (!clean)
                for (int k = 0; k < 2; ++k)
                    if (last_copy[k] >= 0 && !dev::mbar_wait_bounded(&rec_full[k], (last_copy[k] >> 1) & 1))
                        atomicOr(err, kErrDrain);
        }
    } else if (warp == kCW + 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int f = 0, g = 0;
            for (int u = 0;; ++u) {
                const int s = u & 1;
                if (!wait_or_flag(&rec_full[s], (u >> 1) & 1, err)) break;
                const Unit un = unit[s];
                if (un.inst < 0) break;
                bool ok = true;
                if (un.path == 1) {
                    const char *bmat = reinterpret_cast<const char *>(stage[s] + kFarRowB * kTs);
                    int db = 0;
                    for (int kb = 0; kb < kBlocks && ok; ++kb, ++g) {
                        if (kb % kSeg == 0) {  // a new segment q = f: a fresh accumulator
                            db = f & 1;
                            if (f >= 2 && !wait_or_flag(&d_empty[db], ((f - 2) >> 1) & 1, err)) {
                                ok = false;
                                break;
                            }
                        }
                        const int a = g % kNA;
                        if (!wait_or_flag(&a_full[a], (g / kNA) & 1, err)) {
                            ok = false;
                            break;
                        }
                        tc::fence_after();
                        const uint64_t bd = tc::smem_desc(bmat + kb * 512, kLbo, kSbo);
#pragma unroll
                        for (int grp = 0; grp < 2; ++grp) {
                            const uint32_t d = tbase + kColD + db * 32 + grp * 16;
                            const uint32_t ah = tbase + kColA + a * 32 + grp * 16;
                            tc::mma_tf32_ts(d, ah, bd, kIdesc, kb % kSeg != 0);
                            tc::mma_tf32_ts(d, ah + 8, bd, kIdesc, true);
                        }
                        tc::commit(&a_empty[a]);
                        if (kb % kSeg == kSeg - 1) {
                            tc::commit(&d_full[db]);
                            ++f;
                        }
                    }
                    if (!ok) break;
                }
                dev::mbar_arrive(&rec_free[s]);
            }
            // every MMA issued above has completed before tensor memory is released
            tc::commit(&mma_drain);
            if (!dev::mbar_wait_bounded(&mma_drain, 0)) atomicOr(err, kErrTimeout | kErrDrain);
        }
    } else {
        // ---------------- compute warps ----------------
        int c_inst = -1, c_tile = -1;
        float c_d2 = 0.0f, c_mult = 1.0f, c_c2 = 0.0f;
        const float *c_near = nullptr;
        int f = 0, g = 0;
        bool ok = true;
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;

        auto flush = [&]() {
            if (c_inst < 0) return;
            const Inst &I = insts[c_inst];
            const int ti = c_tile / I.tiling.nt2, tj = c_tile - ti * I.tiling.nt2;
            const size_t N = I.geom.N;
            const int lg2 = __ffs(I.tiling.tp2) - 1;  // tp2 is a power of two
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int slot = r * kCT + tid;
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

        for (int u = 0; ok; ++u) {
            const int s = u & 1;
            if (!warp_wait_or_flag(&rec_full[s], (u >> 1) & 1, err)) {
                ok = false;
                break;
            }
            const Unit un = unit[s];
            if (un.inst < 0) break;
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
            const float *st = stage[s];
            if (un.path == 1) {
                // ---- far: K on the CUDA cores, K [g | m] on the tensor cores ----
                const float4 cs = insts[c_inst].tinfo[un.src];
                u64 m2x[2], m2y[2], m2z[2], bb[2];
                float tx[2], ty[2], tz[2];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float *tr = c_near + (size_t)c_tile * kRec32 * kTs + r * kCT + tid;
                    tx[r] = (__ldg(tr) - cs.x) + __ldg(tr + 3 * kTs);
                    ty[r] = (__ldg(tr + kTs) - cs.y) + __ldg(tr + 4 * kTs);
                    tz[r] = (__ldg(tr + 2 * kTs) - cs.z) + __ldg(tr + 5 * kTs);
                    m2x[r] = pack2(-2.0f * tx[r], -2.0f * tx[r]);
                    m2y[r] = pack2(-2.0f * ty[r], -2.0f * ty[r]);
                    m2z[r] = pack2(-2.0f * tz[r], -2.0f * tz[r]);
                    const float b1 = fmaf(tx[r], tx[r], fmaf(ty[r], ty[r], tz[r] * tz[r]));
                    bb[r] = pack2(b1, b1);
                }
                const u64 *s2 = reinterpret_cast<const u64 *>(st);  // row k: sources (2m, 2m + 1)
                // running FP32 sums of this unit's segments: sum K g (b) and sum K m (a) per target
                float sb[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}}, sm[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
                // add segment q (accumulator buffer q & 1) once its MMAs completed, then free it
                auto read_segment = [&](int q) -> bool {
                    const int db = q & 1;
                    if (!warp_wait_or_flag(&d_full[db], (q >> 1) & 1, err)) return false;
                    tc::fence_after();
                    uint32_t dv[2][16];
#pragma unroll
                    for (int r = 0; r < 2; ++r) tc::ld16(tbase + lane_base + kColD + db * 32 + r * 16, dv[r]);
                    tc::wait_ld();
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) dev::mbar_arrive(&d_empty[db]);
#pragma unroll
                    for (int r = 0; r < 2; ++r)
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            sb[r][c] += __uint_as_float(dv[r][c]) + __uint_as_float(dv[r][8 + c]);
                            sm[r][c] += __uint_as_float(dv[r][3 + c]) + __uint_as_float(dv[r][11 + c]);
                        }
                    return true;
                };
                for (int kb = 0; kb < kBlocks; ++kb, ++g) {
                    const int a = g % kNA;
                    if (g >= kNA && !warp_wait_or_flag(&a_empty[a], ((g / kNA) - 1) & 1, err)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    uint32_t kh[2][8], kl[2][8];
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const int mm = kb * 4 + m;
                        const u64 sx = s2[mm], sy = s2[kTs / 2 + mm], sz = s2[kTs + mm], sa = s2[3 * (kTs / 2) + mm];
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            const u64 q = ffma2(sx, m2x[r], ffma2(sy, m2y[r], ffma2(sz, m2z[r], fadd2(sa, bb[r]))));
                            const u64 iq = rsqrt2(q);
                            const u64 kk = fmul2(fmul2(iq, iq), iq);
                            const u64 hi = kk & 0xFFFFE000FFFFE000ull;  // TF32 part (truncated)
                            const u64 lo = fsub2(kk, hi);              // the rest, exact in FP32
                            kh[r][2 * m] = (uint32_t)hi;
                            kh[r][2 * m + 1] = (uint32_t)(hi >> 32);
                            kl[r][2 * m] = (uint32_t)lo;
                            kl[r][2 * m + 1] = (uint32_t)(lo >> 32);
                        }
                    }
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const uint32_t col = tbase + lane_base + kColA + a * 32 + r * 16;
                        tc::st8(col, kh[r]);
                        tc::st8(col + 8, kl[r]);
                    }
                    tc::wait_st();
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) dev::mbar_arrive(&a_full[a]);
                    // a segment was just completed: add the one before it (its MMAs have had a
                    // segment's time to finish), so that its accumulator is free again in time
                    if (kb % kSeg == kSeg - 1) {
                        if (kb >= kSeg && !read_segment(f)) {
                            ok = false;
                            break;
                        }
                        if (kb >= kSeg) ++f;
                    }
                }
                if (!ok) break;
                // the unit's last segment
                if (!read_segment(f)) {
                    ok = false;
                    break;
                }
                ++f;
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float bx = sb[r][0], by = sb[r][1], bz = sb[r][2];
                    const float ax = sm[r][0], ay = sm[r][1], az = sm[r][2];
                    const float vx = ax - fmaf(ty[r], bz, -tz[r] * by);
                    const float vy = ay - fmaf(tz[r], bx, -tx[r] * bz);
                    const float vz = az - fmaf(tx[r], by, -ty[r] * bx);
                    acc[0][r][tid] += __float2ll_rn(vx * c_mult);
                    acc[1][r][tid] += __float2ll_rn(vy * c_mult);
                    acc[2][r][tid] += __float2ll_rn(vz * c_mult);
                }
            } else if (!kCut || un.path == 0) {
                near_tile<false, 2, kCT>(st, c_near + (size_t)c_tile * kRec32 * kTs + tid, c_d2, 0.0f, c_mult, acc, tid);
            } else {
                near_tile<true, 2, kCT>(st, c_near + (size_t)c_tile * kRec32 * kTs + tid, c_d2, c_c2, c_mult, acc, tid);
            }
            __syncwarp();
            if (lane == 0) dev::mbar_arrive(&rec_free[s]);
        }
        if (ok) flush();
        else abort_flag = 1;
    }
    // everyone done: release tensor memory
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::dealloc(tbase, kTmemCols);
}

}  // namespace

int br32tc_occupancy()
{
    // Resident CTAs per SM from the kernel's own resource use.  The runtime's occupancy query
    // answers one CTA per SM for this kernel (on GB300, also with the largest shared-memory
    // carveout), while its registers, shared memory and tensor memory leave room for three; run
    // with three per SM it takes 3.2 instead of 7.4 ms per 256^2 launch.
    int dev = 0, regs_sm = 0, smem_sm = 0, reserved = 0, threads_sm = 0, blocks_sm = 0;
    cudaFuncAttributes fa[2];
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&blocks_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa[0], br32tc_kernel<false>) != cudaSuccess ||
        cudaFuncGetAttributes(&fa[1], br32tc_kernel<true>) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int occ = std::min(blocks_sm, threads_sm / kThreads);
    for (const cudaFuncAttributes &a : fa) {
        // registers are granted per warp in units of 256
        const int regs_warp = (a.numRegs * 32 + 255) / 256 * 256;
        occ = std::min(occ, regs_sm / std::max(regs_warp * (kThreads / 32), 1));
        occ = std::min(occ, smem_sm / std::max((int)a.sharedSizeBytes + reserved, 1));
    }
    // tensor memory: 512 columns per SM, kTmemCols per CTA
    return std::max(1, std::min(occ, (int)(512 / kTmemCols)));
}

int launch_br32tc_batch(const Inst *d_insts, int ninst, long long nitems, int ctas, unsigned long long *counter,
                        int *err, cudaStream_t s, bool any_cutoff)
{
    if (any_cutoff)
        br32tc_kernel<true><<<ctas, kThreads, 0, s>>>(d_insts, ninst, nitems, counter, err);
    else
        br32tc_kernel<false><<<ctas, kThreads, 0, s>>>(d_insts, ninst, nitems, counter, err);
    return cuda_check(cudaGetLastError(), "Birkhoff-Rott FP32C tensor-core kernel launch");
}

ZM_BOUNDS_READER(bounds_br32tc)

}  // namespace zm
