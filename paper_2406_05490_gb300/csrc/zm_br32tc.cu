// zm_br32tc.cu -- FP32-compensated all-pairs Birkhoff-Rott sum over a batch of interfaces with
// the far pairs' |z_j - z_i|^2 formed on the tensor cores (paper Sec. 2 BRSolver, Sec. 3.2.1
// ExactBRSolver, the high-order model):
//     u_i = sum_j (z_j - z_i) x gamma'_j / (|z_j - z_i|^2 + delta^2)^(3/2),   i, j in one interface.
//
// Work units, near/far classification, cutoff handling, records and fixed-point accumulation are
// those of zm_br32.cu; what differs is how a far (target tile, source tile) pair forms its
// kernel values.  In tile-local coordinates (t_i = z_i - c_S, s_j = z_j - c_S, c_S the source
// tile's centre)
//     q_ij = |t_i|^2 + Y_ij,   Y_ij = (|s_j|^2 + delta^2) - 2 t_i . s_j,
// and Y is a matrix product: A (row i: -2 t_i, 1) times B (column j: s_j, |s_j|^2 + delta^2),
// K = 4.  Both operands are split into a TF32 part and a TF32 rest; two MMAs (kind::tf32, K = 8,
// M = 128 targets, N = 32 sources) give (A_hi + A_lo)(B_hi + B_lo): the first reads
// [A_hi | A_hi] against [B_hi ; B_lo], the second [A_lo | A_lo] (the same 4-column core matrix
// read twice, descriptor stride 0 along K).  |t_i|^2, the term of q's own size, is added on the
// CUDA cores, so the tensor cores' FP32 accumulation, which truncates toward zero, only touches
// the smaller Y, over one product of 16 terms (a float32 emulation at 256^2: 7.0e-8 relative L2
// against 6.9e-8 for the CUDA-core Gram form; measured 1.37e-7 on u for both paths).  The CUDA
// cores then take the reciprocal square root, its cube and the six accumulations
// sum_j K (s_j x g_j), sum_j K g_j -- 9 FP32 lane operations per pair instead of 12.
//
// Measured on GB300 (256^2, one launch): 2.18 ms against 1.89 ms for zm_br32.cu, so it is not the
// default (ZM_FAR_TENSOR selects it).  ncu: issue 56 %, FMA pipe 54 %, 10.4 thread instructions
// per pair; the warps wait on fixed-latency dependencies and tensor-memory loads with three
// compute warps per scheduler.  Sweeps (chunks of 16 / 32 / 64 sources, one or two operand
// buffers, 2-4 CTAs per SM, one load of a whole chunk, scalar K or scalar q, 16-byte loads of the
// strengths) did not beat this layout.
//
// CTA: 6 warps.  Warps 0-3 compute (thread t owns targets t and t + 128 of the target tile, i.e.
// tensor-memory lane t in two row groups); warp 4 takes work items from a global atomic counter,
// copies the source records by 1D bulk TMA into a double-buffered stage and, for a far unit,
// writes the unit's operands A (256 targets) and B (256 sources) into shared memory (two
// buffers); warp 5 lane 0 issues the MMAs.  Hand-offs are mbarriers: record full / free per
// stage, operands full / empty per buffer, accumulator full / empty per row group and buffer
// (two 32-column accumulators per row group in tensor memory).  Every wait is bounded: a wait
// that gives up sets the status word and the role leaves its loop; the others then give up in
// turn.  Tensor memory: 128 columns per CTA.
#include <algorithm>

#include "zm_br32_common.cuh"
#include "zm_tc.cuh"

namespace zm {
namespace {

constexpr int kCW = 4;               // compute warps
constexpr int kCT = kCW * 32;        // compute threads: 128 rows per row group
constexpr int kThreads = kCT + 64;   // + producer warp + MMA warp
constexpr int kChunk = 32;           // sources per accumulator (the MMA's N)
constexpr int kNChunks = kTs / kChunk;
constexpr int kAB = 2;               // operand buffers
constexpr uint32_t kTmemCols = 4 * kChunk;  // two row groups x two accumulator buffers
__host__ __device__ constexpr uint32_t col_d(int g, int b) { return (uint32_t)(kChunk * (2 * b + g)); }
constexpr int kStageRows = 10;       // far: s (3), |s|^2 + delta^2, strength (3), s x strength (3)
constexpr float kFarFactor = 1.25f;
constexpr uint32_t kIdesc = tc::idesc_tf32(128, kChunk);
// Operand layout, K-major without swizzling (core matrices of 8 rows x 16 bytes): row r (a target
// of A, a source of B), part h (0: TF32 part, 1: rest), k < 4 at float op_off(r, h, k), i.e. byte
// (r / 8) 256 + h 128 + (r % 8) 16 + 4 k: the descriptors' stride along K is 128 bytes for B (part
// 0 then part 1) and 0 for A (one part read twice), along M / N 256 bytes.
constexpr int kOpFloatsA = 128 * 8;  // per row group
constexpr int kOpFloatsB = kTs * 8;
__device__ __forceinline__ int op_off(int r, int h, int k) { return (r >> 3) * 64 + h * 32 + (r & 7) * 4 + k; }

// Bounded wait on a phase; false (and the status word set) if it gave up.
__device__ __forceinline__ bool wait_or_flag(uint64_t *bar, uint32_t parity, int *err)
{
    if (dev::mbar_wait_bounded(bar, parity)) return true;
    atomicOr(err, kErrTimeout);
    return false;
}

// The same for a whole warp: lane 0 waits, and the warp goes on only if it saw the phase
// complete (so that the warp-collective tensor-memory loads after it stay converged).
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

// v = hi + lo with hi the TF32 value nearest v and lo the TF32 value nearest the rest
__device__ __forceinline__ void split4(const float v[4], float hi[4], float lo[4])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        hi[k] = dev::tf32_round(v[k]);
        lo[k] = dev::tf32_round(v[k] - hi[k]);
    }
}

__device__ __forceinline__ void st_part(float *base, int r, int h, const float v[4])
{
    *reinterpret_cast<float4 *>(base + op_off(r, h, 0)) = make_float4(v[0], v[1], v[2], v[3]);
}

template <bool kCut>
__global__ void __launch_bounds__(kThreads, 3)
    br32tc_kernel(const Inst *__restrict__ insts, int ninst, long long nitems, unsigned long long *counter,
                  int *err)
{
    __shared__ __align__(1024) float stage[2][kStageRows * kTs];
    __shared__ __align__(1024) float opA[kAB][2][kOpFloatsA];  // [buffer][row group]
    __shared__ __align__(1024) float opB[kAB][kOpFloatsB];
    __shared__ long long acc[3][2][kCT];
    __shared__ __align__(8) uint64_t rec_full[2], rec_free[2], ab_full[kAB], ab_empty[kAB];
    __shared__ __align__(8) uint64_t d_full[2][2], d_empty[2][2], mma_drain;
    __shared__ Unit unit[2];
    __shared__ uint32_t tmem_base;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int k = 0; k < 2; ++k) {
            dev::mbar_init(&rec_full[k], 1);
            dev::mbar_init(&rec_free[k], kCW + 1);
            if (k < kAB) {
                dev::mbar_init(&ab_full[k], 1);
                dev::mbar_init(&ab_empty[k], 1);
            }
            for (int g = 0; g < 2; ++g) {
                dev::mbar_init(&d_full[g][k], 1);
                dev::mbar_init(&d_empty[g][k], kCW);
            }
        }
        dev::mbar_init(&mma_drain, 1);
        dev::fence_mbar_init();
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
        // ------------- producer: work units, their records, and the far units' operands -------------
        int p_inst = 0, p_tile = 0, p_next = 0, p_left = 0;
        bool done = false, clean = false;
        int last_copy[2] = {-1, -1};
        int fcount = 0;
        for (int u = 0;; ++u) {
            const int s = u & 1;
            if (u >= 2 && !warp_wait_or_flag(&rec_free[s], ((u - 2) >> 1) & 1, err)) break;
            Unit un;
            un.inst = -1;
            un.tile = un.src = un.path = 0;
            if (lane == 0) {
                while (!done) {
                    while (p_left == 0 && !done) {
                        const long long it = (long long)atomicAdd(counter, 1ull);
                        if (it >= nitems) {
                            done = true;
                            break;
                        }
                        int lo = 0, hi = ninst - 1;
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
                        if (D - a.w - b.w > c * 1.0001f) continue;
                        if (D + a.w + b.w >= c * 0.9999f) path = 2;
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
                } else {
                    last_copy[s] = u;
                    const Inst &I = insts[un.inst];
                    if (un.path == 1) {
                        const float *rec = I.far_rec + (size_t)un.src * kRec32F * kTs;
                        dev::mbar_expect_tx(&rec_full[s], kStageRows * kTs * sizeof(float));
                        dev::tma_copy_1d(stage[s], rec, 4 * kTs * sizeof(float), &rec_full[s]);
                        dev::tma_copy_1d(stage[s] + 4 * kTs, rec + kFarRowG * kTs, 6 * kTs * sizeof(float),
                                         &rec_full[s]);
                    } else {
                        dev::mbar_expect_tx(&rec_full[s], kRec32 * kTs * sizeof(float));
                        dev::tma_copy_1d(stage[s], I.near_rec + (size_t)un.src * kRec32 * kTs,
                                         kRec32 * kTs * sizeof(float), &rec_full[s]);
                    }
                }
            }
            un.inst = __shfl_sync(0xffffffffu, un.inst, 0);
            un.tile = __shfl_sync(0xffffffffu, un.tile, 0);
            un.src = __shfl_sync(0xffffffffu, un.src, 0);
            un.path = __shfl_sync(0xffffffffu, un.path, 0);
            if (un.inst < 0) break;
            if (un.path != 1) continue;
            // far unit: its operands A (targets) and B (sources) into buffer fcount % kAB
            const int buf = fcount % kAB;
            if (fcount >= kAB && !warp_wait_or_flag(&ab_empty[buf], ((fcount - kAB) / kAB) & 1, err)) break;
            if (!warp_wait_or_flag(&rec_full[s], (u >> 1) & 1, err)) break;
            const Inst &I = insts[un.inst];
            const float4 cs = I.tinfo[un.src];
            const float *st = stage[s];
            const float *tgt = I.near_rec + (size_t)un.tile * kRec32 * kTs;
            for (int j = lane; j < kTs; j += 32) {
                // source j: (s, |s|^2 + delta^2)
                float v[4] = {st[j], st[kTs + j], st[2 * kTs + j], st[3 * kTs + j]}, hi[4], lo[4];
                split4(v, hi, lo);
                st_part(opB[buf], j, 0, hi);
                st_part(opB[buf], j, 1, lo);
                const float *tr = tgt + j;
                const float tx = (__ldg(tr) - cs.x) + __ldg(tr + 3 * kTs);
                const float ty = (__ldg(tr + kTs) - cs.y) + __ldg(tr + 4 * kTs);
                const float tz = (__ldg(tr + 2 * kTs) - cs.z) + __ldg(tr + 5 * kTs);
                // target slot j (row j % 128 of row group j / 128): (-2 t, 1), t as the compute
                // warps form it
                float a[4] = {-2.0f * tx, -2.0f * ty, -2.0f * tz, 1.0f};
                split4(a, hi, lo);
                st_part(opA[buf][j >> 7], j & 127, 0, hi);
                st_part(opA[buf][j >> 7], j & 127, 1, lo);
            }
            dev::fence_proxy_async();  // the tensor cores read what the threads wrote
            __syncwarp();
            if (lane == 0) dev::mbar_arrive(&ab_full[buf]);
            ++fcount;
        }
        // after an abnormal exit, let this warp's copies in flight land before shared memory is
        // released (bounded as well)
        if (lane == 0 && !clean)
            for (int k = 0; k < 2; ++k)
                if (last_copy[k] >= 0 && !dev::mbar_wait_bounded(&rec_full[k], (last_copy[k] >> 1) & 1))
                    atomicOr(err, kErrDrain);
    } else if (warp == kCW + 1) {
        // ---------------- MMA issuer: Y = A B per row group and 32-source chunk ----------------
        if (lane == 0) {
            int fcount = 0, dcnt = 0;
            for (int u = 0;; ++u) {
                const int s = u & 1;
                if (!wait_or_flag(&rec_full[s], (u >> 1) & 1, err)) break;
                const Unit un = unit[s];
                if (un.inst < 0) break;
                bool ok = true;
                if (un.path == 1) {
                    const int buf = fcount % kAB;
                    ok = wait_or_flag(&ab_full[buf], (fcount / kAB) & 1, err);
                    if (ok) {
                        tc::fence_after();
                        const char *pb = reinterpret_cast<const char *>(opB[buf]);
                        for (int c = 0; c < kNChunks && ok; ++c, ++dcnt) {
                            const int b = dcnt & 1;
                            const uint64_t bd = tc::smem_desc(pb + 32 * kChunk * c, 128, 256);
#pragma unroll
                            for (int g = 0; g < 2; ++g) {
                                if (dcnt >= 2 && !wait_or_flag(&d_empty[g][b], ((dcnt - 2) >> 1) & 1, err)) {
                                    ok = false;
                                    break;
                                }
                                tc::fence_after();
                                const char *pa = reinterpret_cast<const char *>(opA[buf][g]);
                                const uint32_t d = tbase + col_d(g, b);
                                // K-step 0: [A_hi | A_hi] x [B_hi; B_lo]; K-step 1: [A_lo | A_lo] x [B_hi; B_lo]
                                tc::mma_tf32_ss(d, tc::smem_desc(pa, 0, 256), bd, kIdesc, false);
                                tc::mma_tf32_ss(d, tc::smem_desc(pa + 128, 0, 256), bd, kIdesc, true);
                                tc::commit(&d_full[g][b]);
                            }
                        }
                        if (ok) tc::commit(&ab_empty[buf]);
                    }
                    ++fcount;
                }
                dev::mbar_arrive(&rec_free[s]);
                if (!ok) break;
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
        int dcnt = 0;
        bool ok = true;
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;

        auto flush = [&]() {
            if (c_inst < 0) return;
            const Inst &I = insts[c_inst];
            const int ti = c_tile / I.tiling.nt2, tj = c_tile - ti * I.tiling.nt2;
            const size_t N = I.geom.N;
            const int lg2 = __ffs(I.tiling.tp2) - 1;
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
                    c_mult = __int_as_float((127 + sc) << 23);
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
                // ---- far: q = |t|^2 + Y, Y from the tensor cores ----
                const float4 cs = insts[c_inst].tinfo[un.src];
                float tx[2], ty[2], tz[2];
                u64 bb[2], ax[2], ay[2], az[2], gxs[2], gys[2], gzs[2];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float *tr = c_near + (size_t)c_tile * kRec32 * kTs + r * kCT + tid;
                    tx[r] = (__ldg(tr) - cs.x) + __ldg(tr + 3 * kTs);
                    ty[r] = (__ldg(tr + kTs) - cs.y) + __ldg(tr + 4 * kTs);
                    tz[r] = (__ldg(tr + 2 * kTs) - cs.z) + __ldg(tr + 5 * kTs);
                    const float b1 = fmaf(tx[r], tx[r], fmaf(ty[r], ty[r], tz[r] * tz[r]));
                    bb[r] = pack2(b1, b1);
                    ax[r] = ay[r] = az[r] = gxs[r] = gys[r] = gzs[r] = 0ull;
                }
                const u64 *s2 = reinterpret_cast<const u64 *>(st);  // row k: sources (2m, 2m + 1)
                constexpr int H = kTs / 2;
                for (int c = 0; c < kNChunks; ++c, ++dcnt) {
                    const int b = dcnt & 1;
                    if (!warp_wait_or_flag(&d_full[0][b], (dcnt >> 1) & 1, err) ||
                        !warp_wait_or_flag(&d_full[1][b], (dcnt >> 1) & 1, err)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after();
#pragma unroll
                    for (int half = 0; half < kChunk / 16; ++half) {
                        uint32_t y[2][16];  // Y of this thread's two targets, 16 sources
                        tc::ld16(tbase + lane_base + col_d(0, b) + 16 * half, y[0]);
                        tc::ld16(tbase + lane_base + col_d(1, b) + 16 * half, y[1]);
                        tc::wait_ld();
                        if (half == kChunk / 16 - 1) {  // all read: the accumulators are free again
                            tc::fence_before();
                            __syncwarp();
                            if (lane == 0) {
                                dev::mbar_arrive(&d_empty[0][b]);
                                dev::mbar_arrive(&d_empty[1][b]);
                            }
                        }
#pragma unroll
                        for (int p = 0; p < 8; ++p) {
                            const int mm = c * (kChunk / 2) + half * 8 + p;  // source pair
                            const u64 gx = s2[4 * H + mm], gy = s2[5 * H + mm], gz = s2[6 * H + mm];
                            const u64 mx = s2[7 * H + mm], my = s2[8 * H + mm], mz = s2[9 * H + mm];
#pragma unroll
                            for (int r = 0; r < 2; ++r) {
                                const u64 yy = (u64)y[r][2 * p] | ((u64)y[r][2 * p + 1] << 32);
                                const u64 q = fadd2(bb[r], yy);
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
                    }
                }
                if (!ok) break;
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float bx = sum2(gxs[r]), by = sum2(gys[r]), bz = sum2(gzs[r]);
                    const float vx = sum2(ax[r]) - fmaf(ty[r], bz, -tz[r] * by);
                    const float vy = sum2(ay[r]) - fmaf(tz[r], bx, -tx[r] * bz);
                    const float vz = sum2(az[r]) - fmaf(tx[r], by, -ty[r] * bx);
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
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::dealloc(tbase, kTmemCols);
}

}  // namespace

int br32tc_occupancy()
{
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
        const int regs_warp = (a.numRegs * 32 + 255) / 256 * 256;
        occ = std::min(occ, regs_sm / std::max(regs_warp * (kThreads / 32), 1));
        occ = std::min(occ, smem_sm / std::max((int)a.sharedSizeBytes + reserved, 1));
    }
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
