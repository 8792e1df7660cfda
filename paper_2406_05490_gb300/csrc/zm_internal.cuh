// zm_internal.cuh -- internal declarations shared by the translation units of libzm.so.
// Not part of the public ABI (include/zm.h is).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "zm.h"

namespace zm {

// A named NVTX range over one host call (zm_step, zm_velocity, the batch and server steps), so
// that a profiler's timeline and ncu's --nvtx filters can attribute kernels to API calls.  NVTX3
// is header-only and costs a branch when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Mesh constants handed to every stencil kernel by value.
struct Geom {
    int n1, n2, N;
    double dx1, dx2, L1, L2;
    int periodic;
    double i12a, i12b;    // 1 / (12 dx1), 1 / (12 dx2): first-difference weights
    double i12a2, i12b2;  // 1 / (12 dx1^2), 1 / (12 dx2^2): second-difference weights
};

// Fill in the spacings and stencil weights of a Geom whose n1, n2, L1, L2 are set (on the host,
// so that no kernel divides per node).
inline void geom_finish(Geom &g)
{
    g.N = g.n1 * g.n2;
    g.dx1 = g.L1 / g.n1;
    g.dx2 = g.L2 / g.n2;
    g.i12a = 1.0 / (12.0 * g.dx1);
    g.i12b = 1.0 / (12.0 * g.dx2);
    g.i12a2 = 1.0 / (12.0 * g.dx1 * g.dx1);
    g.i12b2 = 1.0 / (12.0 * g.dx2 * g.dx2);
}

// Source records of the Birkhoff-Rott sum are stored tile-major: a tile is a tp1 x tp2 patch of
// the mesh (compact in space for a smooth interface), ts = tp1 * tp2 slots, padded with
// zero-strength sources where the patch runs past the mesh edge.
struct Tiling {
    int tp1, tp2, ts;
    int nt1, nt2, ntiles;
};

// FP64 record: rows 0-2 absolute position, rows 3-5 scaled sheet strength -> [tile][6][ts] double
// FP32C near record: rows 0-2 position hi, 3-5 position lo, 6-8 scaled strength -> [tile][9][ts]
// FP32C far record, [tile][10][ts] float (ts = 256):
//   rows 0-2 s = z - c_T (c_T the tile centre), row 3 |s|^2 + delta^2, rows 4-6 scaled strength,
//   rows 7-9 s x strength
constexpr int kRec64 = 6;
constexpr int kRec32 = 9;
constexpr int kRec32F = 10;
constexpr int kFarRowG = 4;

// Launch geometry of the all-pairs kernel.
struct BrPlan {
    int tpb;        // threads per CTA
    int r;          // targets per thread (register blocking)
    int nsplit;     // source splits (grid.y); partial sums reduced by a second kernel
    int tiles_per_split;
    int qsplit;     // > 1: each split is 1/qsplit of one tile's sources (small meshes)
    int ntb;        // target blocks (grid.x)
};

// Launch plan of the FP32C Birkhoff-Rott kernel (persistent, stream-K ranges).
struct Br32Plan {
    int ctas;           // persistent CTAs (grid size)
    int kseg;           // most target-group segments one CTA's range can touch
    int occupancy;      // resident CTAs per SM
    size_t part_doubles;
};

// Device-side status word bits.  kErrTimeout: a bounded wait gave up.  kErrDrain: after that,
// the wait for the CTA's own bulk copies still in flight gave up as well (the CTA then exits
// with a copy possibly landing in shared memory it has released; a copy that lands at all
// does so within microseconds, far inside the second that wait allows).
constexpr int kErrTimeout = 1;
constexpr int kErrDrain = 2;

// Optional CUDA-event timing of every launch, per kernel class (see zm_set_profiling).
struct Prof {
    int on = 0;
    zm_profile acc{};
    struct Ev {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<Ev> live;
    std::vector<cudaEvent_t> pool;
};

// One interface as the batched kernels see it (a plain struct mirrored into device memory).
struct Inst {
    Geom geom;
    Tiling tiling;
    double atwood, g, mu, delta;
    double dt;                  // RK3 step of this interface
    int keep_phi;               // medium order: Phi comes from the FFT velocity, not from u
    double cutoff;              // > 0: sum only over sources within this distance
    int block0;                 // first 256-thread block of this interface in the point kernels
    int chunk, nchunks;         // source tiles per Birkhoff-Rott work item; items per target tile
    long long item0;            // first Birkhoff-Rott work item of this interface
    double *y[3];               // state and two RK3 stage buffers, 5N doubles each
    double *u, *phi, *q;        // 3N, N, N
    float *near_rec, *far_rec;  // [tile][9][256], [tile][10][256]
    float4 *tinfo;              // [tile]: centre, radius
    unsigned long long *ufix;   // [3][N] fixed-point velocity accumulators (two's complement)
    unsigned int *gmax;         // float bits of max |gamma'| over the mesh
    int *scale;                 // fixed-point scale (power of two) used by the last sum
};

class Batch;

}  // namespace zm

struct zm_ctx {
    zm_mesh mesh;
    zm::Geom geom;
    double atwood, g, mu, delta;
    int order;  // ZM_ORDER_*
    int fp32c;  // reduced-precision Birkhoff-Rott pair terms
    int df64;   // low order in double-word arithmetic: every field below is float2 pairs
    int device;
    cudaStream_t stream;

    // state and stage buffers: 5N doubles each, (z1, z2, z3, w1, w2) component-major
    double *y0, *ya, *yb;
    double *u;    // 3N velocity of the last derivative evaluation
    double *phi;  // N
    double *q;    // N: g z3 + 1/8 w^T h^-1 w (the part of Phi that does not need u)
    double *nrm;  // 3N unit normals (low order)

    // Birkhoff-Rott source records and split partial sums
    zm::Tiling tiling;
    zm::BrPlan plan;
    void *src;
    size_t src_bytes;
    double *part;  // FP64: [nsplit][3][N]; FP32C: [ctas * kseg][3][512]
    float *src_far;   // FP32C far records
    float4 *tinfo;    // FP32C per-tile bounding sphere: centre, radius
    zm::Br32Plan plan32;

    // low order: FFT workspace (complex doubles) and twiddles: tw1, tw2 for the power-of-two
    // factor M of each side, twl1, twl2 for the whole side L = R M when R > 1 (else null)
    double2 *fa, *fb, *tw1, *tw2, *twl1, *twl2;
    double2 *twh;  // double word, both sides powers of two: half table of W_{n2/2} (else null)

    int *err;   // device status word (zm::kErr*)
    int *flag;  // device scratch flag (finite check)

    zm::Prof prof;
    zm::Batch *batch;  // FP32C high order: the interface lives in a batch of one

    // one RK3 step captured as a CUDA graph (FP64 and low order), replayed by zm_step
    cudaStream_t cap;
    cudaGraphExec_t gexec;
    double gdt;
    zm_profile step_launches;  // launches and pairs one replayed step adds to the counters
};

namespace zm {

// ---- error reporting (zm_api.cu) ------------------------------------------------------------
int set_error(int code, const std::string &msg);
int cuda_check(cudaError_t e, const char *what);

// ---- profiling helpers (zm_api.cu) -----------------------------------------------------------
void prof_begin(Prof &pr, cudaStream_t s, int cls, cudaEvent_t *a);
void prof_end(Prof &pr, cudaStream_t s, int cls, cudaEvent_t a);
void prof_fold(Prof &pr, cudaStream_t s);
void prof_release(Prof &pr);
inline void prof_begin(zm_ctx *c, int cls, cudaEvent_t *a) { prof_begin(c->prof, c->stream, cls, a); }
inline void prof_end(zm_ctx *c, int cls, cudaEvent_t a) { prof_end(c->prof, c->stream, cls, a); }

// ---- stencil kernels (zm_stencil.cu) -----------------------------------------------------------
// Geometry pass over state y (5N): writes source records (high order), q, and normals (low).
int launch_geometry(zm_ctx *c, const double *y);
// Vorticity pass.  mode 0: wdot_out = dw/dt (2N) from phi and y.  mode 1: RK3 stage combine
// yout = ca * y0 + cb * (y + dt * L(y)), L = (u, dw/dt).
int launch_vorticity(zm_ctx *c, const double *y, double *wdot_out, const double *y0, double *yout,
                     double dt, double ca, double cb, int mode);
// Reduce split partials into u and, if write_phi, Phi = q + |u|^2 / 2.
int launch_reduce(zm_ctx *c, bool write_phi);
// Set *dev_flag (device int) to 1 if any of y[0..n) is NaN/Inf.
int check_finite(zm_ctx *c, const double *y, size_t n, int *dev_flag);

// ---- Birkhoff-Rott kernels (zm_br.cu) ----------------------------------------------------------
BrPlan plan_br(const Geom &g, const Tiling &t, int sm_count);
Tiling make_tiling(const Geom &g);  // 16 x 16 patches
// tp1 x tp2 patches (tp1 * tp2 = 256 slots, both powers of two)
Tiling make_tiling_shape(const Geom &g, int tp1, int tp2);
int launch_br(zm_ctx *c, const double *y);  // FP64 path (then launch_reduce)

// ---- FP32C Birkhoff-Rott kernel over a batch of interfaces (zm_br32.cu) ----------------------------
int br32_occupancy();  // resident CTAs per SM of the batched kernel
int br32tc_occupancy();  // the same for the tensor-core far-path kernel
int launch_br32tc_batch(const Inst *d_insts, int ninst, long long nitems, int ctas, unsigned long long *counter,
                        int *err, cudaStream_t s, bool any_cutoff);
int launch_br32_batch(const Inst *d_insts, int ninst, long long nitems, int ctas,
                      unsigned long long *counter, int *err, cudaStream_t s, bool any_cutoff);
void init_far_records(float *far_rec, int ntiles, float d2, cudaStream_t s);

// ---- low order (zm_fft.cu) ---------------------------------------------------------------------
// Sides the FP64 FFT takes: L = R 2^a with a >= 3, R odd in 1 .. 19, L <= 8192.
bool fft_side_ok(int L);
// Sides the double-word FFT takes: powers of two 8 .. 4096, or R 2^a with a in 3 .. 12, R odd in
// 3 .. 19, L <= 8192.
bool df_side_ok(int L);
int fft_setup(zm_ctx *c);
int launch_riesz(zm_ctx *c, const double *y);

// ---- low order in double-word (FP32-pair) arithmetic (zm_lowdf.cu) -----------------------------
// Buffers keep their FP64 sizes; a double-word context stores float2 {hi, lo} per value, with z1
// and z2 as displacements from the mesh coordinates.
int df_setup(zm_ctx *c);
int df_derivative(zm_ctx *c, const double *y);
int df_vorticity(zm_ctx *c, const double *y, double *wdot_out, const double *y0, double *yout,
                 double dt, double ca, double cb, int mode);
// count values src -> dst, FP64 -> double word (to_df) or back; `state`: src/dst hold the 5N
// state and z1, z2 are taken relative to the mesh coordinates.  src may equal dst.
int df_convert(zm_ctx *c, const double *src, double *dst, size_t count, int state, int to_df);
int df_check_finite(zm_ctx *c, const double *y, size_t nvalues, int *dev_flag);

// ---- one full derivative evaluation (zm_api.cu) --------------------------------------------------
int derivative(zm_ctx *c, const double *y);

}  // namespace zm

// ---- device helpers ------------------------------------------------------------------------------
#ifdef __CUDACC__
namespace zm {
// ---- the checked build ------------------------------------------------------------------------
// Compiled with -DZM_CHECKS=1 (libzm_checked.so), the kernels test the indices they compute
// (gathers, wraps, tile and record numbers, transposed writes, shared-memory positions) before
// each access; an index outside its array is counted, the first one recorded, and the access
// skipped, so that the kernel neither faults nor traps.  zm_bounds_status() reads the counts.
// In the default build ZM_IDX_OK is the constant true and the tests compile away.
#ifndef ZM_CHECKS
#define ZM_CHECKS 0
#endif

#if ZM_CHECKS
namespace chk {
// one count per translation unit (device globals have internal linkage here), summed by the
// host readers below
static __device__ unsigned int g_hits;
static __device__ long long g_first;
static __device__ int g_site;

static __device__ __noinline__ bool fail(long long i, int site)
{
    if (atomicAdd(&g_hits, 1u) == 0) {
        g_first = i;
        g_site = site;
    }
    return false;
}
}  // namespace chk
#define ZM_IDX_OK(i, n) \
    ((long long)(i) >= 0 && (long long)(i) < (long long)(n) ? true : ::zm::chk::fail((long long)(i), __LINE__))
// Host side: adds this unit's counts to *hits (the first offending index and source line to
// *first, *site when none was recorded yet) and clears them when `clear`.
#define ZM_BOUNDS_READER(name)                                                                    \
    int name(unsigned int *hits, long long *first, int *site, int clear)                          \
    {                                                                                             \
        unsigned int h = 0;                                                                       \
        long long f = -1;                                                                         \
        int l = 0;                                                                                \
        if (cudaMemcpyFromSymbol(&h, chk::g_hits, sizeof(h)) != cudaSuccess ||                    \
            cudaMemcpyFromSymbol(&f, chk::g_first, sizeof(f)) != cudaSuccess ||                    \
            cudaMemcpyFromSymbol(&l, chk::g_site, sizeof(l)) != cudaSuccess)                       \
            return -1;                                                                            \
        if (h && *hits == 0) {                                                                    \
            *first = f;                                                                           \
            *site = l;                                                                            \
        }                                                                                         \
        *hits += h;                                                                               \
        if (clear) {                                                                              \
            const unsigned int z = 0;                                                             \
            if (cudaMemcpyToSymbol(chk::g_hits, &z, sizeof(z)) != cudaSuccess) return -1;         \
        }                                                                                         \
        return 0;                                                                                 \
    }
#else
#define ZM_IDX_OK(i, n) true
#define ZM_BOUNDS_READER(name) \
    int name(unsigned int *, long long *, int *, int) { return 0; }
#endif

// Readers of the translation units with kernels (zero work in the default build).
int bounds_api(unsigned int *, long long *, int *, int);
int bounds_batch(unsigned int *, long long *, int *, int);
int bounds_br(unsigned int *, long long *, int *, int);
int bounds_br32(unsigned int *, long long *, int *, int);
int bounds_br32tc(unsigned int *, long long *, int *, int);
int bounds_fft(unsigned int *, long long *, int *, int);
int bounds_lowdf(unsigned int *, long long *, int *, int);
int bounds_lowdf_mix(unsigned int *, long long *, int *, int);
int bounds_stencil(unsigned int *, long long *, int *, int);

namespace dev {

// Bounded waits: every spin on an mbarrier gives up after this many polls and reports
// kErrTimeout through the status word instead of hanging the GPU.
// Each mbarrier.try_wait poll that finds the phase incomplete suspends the thread for a few
// microseconds (measured on GB300: 2^26 polls took 252 s, 3.8 us each), so 2^18 polls bound a
// stuck wait to about one second; a bulk copy that does complete lands within microseconds.
constexpr uint32_t kSpinLimit = 1u << 18;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arm the barrier for `bytes` of asynchronous transactions and start one 1D bulk TMA copy
// global -> shared that completes them.  Both addresses 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void tma_load_1d(void *smem_dst, const void *gmem_src, uint32_t bytes,
                                            uint64_t *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(smem_dst)),
        "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Arm the barrier for `bytes` of asynchronous transactions (one arrival); the copies that
// complete them follow with tma_copy_1d.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// One 1D bulk copy global -> shared completing `bytes` transactions on the barrier (armed
// before).  Both addresses 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void tma_copy_1d(void *smem_dst, const void *gmem_src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(smem_dst)),
        "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Plain arrival (no transactions).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Round to TF32 (10 fraction bits), ties away from zero: the value a TF32 tensor-core operand
// holds exactly.
__host__ __device__ __forceinline__ float tf32_round(float x)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
#else
    uint32_t b;
    __builtin_memcpy(&b, &x, 4);
    b = (b + 0x1000u) & 0xFFFFE000u;
    float r;
    __builtin_memcpy(&r, &b, 4);
    return r;
#endif
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Returns false if the phase did not complete within kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    for (uint32_t it = 0; it < kSpinLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// 1 / sqrt(x) for a positive double inside the FP32 range: the FP32 estimate refined by two
// Newton-Raphson steps y <- y (3/2 - x/2 y^2) (relative error ~2^-22 -> ~2^-43 -> FP64 rounding),
// a few FP64 instructions instead of a correctly rounded square root and division.
__device__ __forceinline__ double rsqrt_nr(double x)
{
    const double hx = 0.5 * x;
    double y = (double)rsqrtf((float)x);
    y = y * fma(-hx * y, y, 1.5);
    y = y * fma(-hx * y, y, 1.5);
    return y;
}

// q^(-3/2) for a positive, normal double q: the hardware estimate y ~ q^(-1/2) (PTX
// rsqrt.approx.ftz.f64, relative error below 2^-20 as measured on GB300 over q in [1e-12, 10])
// corrected by the second-order binomial expansion of (1 - e)^(-3/2) = 1 + 3e/2 + 15e^2/8 + ...
// with the residual e = 1 - q y^2 formed by one FMA:  q^(-3/2) = y^3 (1 - e)^(-3/2).  The
// dropped third-order term is 35 e^3 / 16 with |e| < 2^-19, far below FP64 rounding: measured
// maximum relative error 4.4e-16 (about 2 ulp) over 6.7e7 samples.  Six FP64 instructions and
// one MUFU operation.
__device__ __forceinline__ double rsqrt_cube(double q)
{
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(q));
    const double y2 = y * y;
    const double e = fma(-q, y2, 1.0);
    const double y3 = y2 * y;
    const double p = fma(e, 1.875, 1.5);
    return fma(y3 * e, p, y3);
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

}  // namespace dev
}  // namespace zm
#endif
