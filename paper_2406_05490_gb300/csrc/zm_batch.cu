// zm_batch.cu -- many interfaces of uneven mesh sizes advanced together (high order, FP32C
// Birkhoff-Rott pair terms).  Each RK3 stage is four launches over the whole batch: the
// geometry pass, one persistent all-pairs launch over a shared work list (zm_br32.cu), the
// fixed-point finish (u, Phi) and the vorticity/RK3 pass; a whole step is captured once as a
// CUDA graph and replayed.  A single FP32C interface (zm_create with ZM_PREC_FP32C) is a batch
// of one.  Paper counterpart: the ZModel derivative and the TimeIntegrator of Sec. 3.1, per
// interface; batching many interfaces on one GPU has none.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "zm_batch.cuh"
#include "zm_stencil.cuh"

namespace zm {
namespace {

constexpr int kPtb = 256;  // threads per block of the point kernels

__global__ void __launch_bounds__(kPtb)
    batch_geometry_kernel(const Inst *__restrict__ insts, const int *__restrict__ block_inst, int yin)
{
    const Inst &I = insts[block_inst[blockIdx.x]];
    const int p = (blockIdx.x - I.block0) * kPtb + threadIdx.x;
    if (p >= I.geom.N || !ZM_IDX_OK(p, I.geom.N)) return;
    const double pref = I.geom.dx1 * I.geom.dx2 / (4.0 * 3.14159265358979323846);
    geometry_point<kGeoFp32c>(I.geom, I.tiling, p, I.y[yin], pref, I.g, (float)(I.delta * I.delta),
                              I.near_rec, I.far_rec, I.tinfo, I.gmax, I.q, nullptr);
}

// u = fixed-point sum * 2^-scale, Phi = q + |u|^2 / 2; clears the accumulators, the tile
// spheres, max |gamma'| and the work counter for the next evaluation.
__global__ void __launch_bounds__(kPtb)
    batch_finish_kernel(const Inst *__restrict__ insts, const int *__restrict__ block_inst,
                        unsigned long long *counter)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0ull;
    const Inst &I = insts[block_inst[blockIdx.x]];
    const int p = (blockIdx.x - I.block0) * kPtb + threadIdx.x;
    if (p >= I.geom.N || !ZM_IDX_OK(p, I.geom.N)) return;
    const size_t N = I.geom.N;
    const double inv = ldexp(1.0, -*I.scale);
    double s[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        s[c] = (double)(long long)I.ufix[c * N + p] * inv;
        I.ufix[c * N + p] = 0ull;
        I.u[c * N + p] = s[c];
    }
    if (!I.keep_phi) I.phi[p] = I.q[p] + 0.5 * (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    if (p < I.tiling.ntiles) I.tinfo[p] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (p == 0) *I.gmax = 0u;
}

// mode 0: dw/dt into the first 2N of stage buffer 2; mode 1: RK3 stage combine into y[yout].
template <int kMode>
__global__ void __launch_bounds__(kPtb)
    batch_vorticity_kernel(const Inst *__restrict__ insts, const int *__restrict__ block_inst, int yin,
                           int yout, double ca, double cb)
{
    const Inst &I = insts[block_inst[blockIdx.x]];
    const int p = (blockIdx.x - I.block0) * kPtb + threadIdx.x;
    if (p >= I.geom.N || !ZM_IDX_OK(p, I.geom.N)) return;
    if (I.mu != 0.0)
        vorticity_point<true, kMode>(I.geom, p, I.phi, I.y[yin], I.u, I.atwood, I.mu, I.dt, ca, cb,
                                     I.y[0], I.y[yout], I.y[2]);
    else
        vorticity_point<false, kMode>(I.geom, p, I.phi, I.y[yin], I.u, I.atwood, I.mu, I.dt, ca, cb,
                                      I.y[0], I.y[yout], I.y[2]);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// Candidate patch shapes of the tiles (256 mesh nodes each): square, and elongated ones that are
// more compact in space when the mesh spacing differs between the two directions.
const int kShapes[kNumShapes][2] = {{16, 16}, {8, 32}, {32, 8}, {4, 64}, {64, 4}};

// Tiles an interface's record buffers must hold for any candidate shape.
size_t tile_capacity(int n1, int n2)
{
    size_t m = 0;
    for (int k = 0; k < kNumShapes; ++k) {
        const size_t nt = (size_t)((n1 + kShapes[k][0] - 1) / kShapes[k][0]) * ((n2 + kShapes[k][1] - 1) / kShapes[k][1]);
        m = std::max(m, nt);
    }
    return m;
}

namespace {

// sizes of the pieces of one interface's slab, in order
void slab_layout(const zm_mesh &m, size_t sz[12])
{
    const size_t N = (size_t)m.n1 * m.n2;
    const size_t nt = tile_capacity(m.n1, m.n2);
    const size_t slots = nt * 256;
    const size_t s[12] = {5 * N * 8, 5 * N * 8, 5 * N * 8, 3 * N * 8, N * 8, N * 8, 3 * N * 8,
                          slots * kRec32 * 4, slots * kRec32F * 4, nt * 16, 4, 4};
    for (int k = 0; k < 12; ++k) sz[k] = s[k];
}

int default_chunk(int ntiles) { return std::max(1, std::min(8, ntiles / 16)); }

}  // namespace

void Batch::release()
{
    // the stream is borrowed (context's, caller's or server's): synchronise it once and forget
    // it, so that a second release never touches a stream its owner has destroyed
    if (stream) cudaStreamSynchronize(stream);
    stream = nullptr;
    drop_graph();
    if (cap) cudaStreamDestroy(cap);
    cap = nullptr;
    for (void *s : owned) cudaFree(s);
    owned.clear();
    if (d) cudaFree(d);
    if (block_inst) cudaFree(block_inst);
    if (counter) cudaFree(counter);
    if (err) cudaFree(err);
    d = nullptr;
    block_inst = nullptr;
    counter = nullptr;
    err = nullptr;
    d_cap = bi_cap = 0;
    prof_release(own);
}

size_t Batch::inst_bytes(const zm_mesh &m)
{
    size_t sz[12], total = 0;
    slab_layout(m, sz);
    for (int k = 0; k < 12; ++k) total += align256(sz[k]);
    return total;
}

int Batch::alloc_inst(Inst &I, const zm_mesh &m, double atwood, double g, double mu, double delta,
                      double dt, cudaStream_t s, bool async, void **slab_out)
{
    std::memset(&I, 0, sizeof(I));
    I.geom.n1 = m.n1;
    I.geom.n2 = m.n2;
    I.geom.N = m.n1 * m.n2;
    I.geom.L1 = m.L1;
    I.geom.L2 = m.L2;
    geom_finish(I.geom);
    I.geom.periodic = m.periodic ? 1 : 0;
    I.tiling = make_tiling(I.geom);
    I.atwood = atwood;
    I.g = g;
    I.mu = mu;
    I.delta = delta;
    I.dt = dt;
    size_t sz[12], off[12], total = 0;
    slab_layout(m, sz);
    for (int k = 0; k < 12; ++k) {
        off[k] = total;
        total += align256(sz[k]);
    }
    void *slab = nullptr;
    cudaError_t e = async ? cudaMallocAsync(&slab, total, s) : cudaMalloc(&slab, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(ZM_ERR_NOMEM, "interface state: device allocation failed");
    }
    e = async ? cudaMemsetAsync(slab, 0, total, s) : cudaMemset(slab, 0, total);
    if (e != cudaSuccess) return set_error(ZM_ERR_CUDA, "interface state: memset failed");
    char *b = static_cast<char *>(slab);
    for (int k = 0; k < 3; ++k) I.y[k] = reinterpret_cast<double *>(b + off[k]);
    I.u = reinterpret_cast<double *>(b + off[3]);
    I.phi = reinterpret_cast<double *>(b + off[4]);
    I.q = reinterpret_cast<double *>(b + off[5]);
    I.ufix = reinterpret_cast<unsigned long long *>(b + off[6]);
    I.near_rec = reinterpret_cast<float *>(b + off[7]);
    I.far_rec = reinterpret_cast<float *>(b + off[8]);
    I.tinfo = reinterpret_cast<float4 *>(b + off[9]);
    I.gmax = reinterpret_cast<unsigned int *>(b + off[10]);
    I.scale = reinterpret_cast<int *>(b + off[11]);
    init_far_records(I.far_rec, (int)tile_capacity(m.n1, m.n2), (float)(delta * delta), async ? s : nullptr);
    *slab_out = slab;
    return cuda_check(cudaGetLastError(), "interface state init");
}

int Batch::setup()
{
    cudaGetDevice(&device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    occ = tc ? br32tc_occupancy() : br32_occupancy();
    if (cudaMalloc(&counter, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ZM_ERR_NOMEM, "batch: device allocation failed");
    }
    cudaMemset(counter, 0, sizeof(unsigned long long));
    cudaMemset(err, 0, sizeof(int));
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
        return set_error(ZM_ERR_CUDA, "batch: stream creation failed");
    return cuda_check(cudaDeviceSynchronize(), "batch setup");
}

int Batch::init(int n, const zm_mesh *meshes, const double *atwood, double g, double mu,
                const double *delta)
{
    int rc = setup();
    if (rc) return rc;
    h.resize(n);
    for (int k = 0; k < n; ++k) {
        void *slab = nullptr;
        rc = alloc_inst(h[k], meshes[k], atwood[k], g, mu, delta[k], 0.0, nullptr, false, &slab);
        if (rc) return rc;
        owned.push_back(slab);
    }
    rc = plan();
    if (rc) return rc;
    return cuda_check(cudaDeviceSynchronize(), "batch init");
}

int Batch::plan()
{
    drop_graph();
    long long items = 0;
    int blocks = 0;
    for (auto &I : h) {
        I.block0 = blocks;
        blocks += (I.geom.N + kPtb - 1) / kPtb;
        I.chunk = chunk_override > 0 ? std::min(chunk_override, I.tiling.ntiles)
                                     : default_chunk(I.tiling.ntiles);
        I.nchunks = (I.tiling.ntiles + I.chunk - 1) / I.chunk;
        I.item0 = items;
        items += (long long)I.tiling.ntiles * I.nchunks;
    }
    nblocks = blocks;
    nitems = items;
    ctas = (int)std::max<long long>(1, std::min<long long>(nitems, (long long)occ * sms));
    const int n = (int)h.size();
    if (n == 0) return ZM_OK;
    bi_host.resize(nblocks);
    for (int k = 0; k < n; ++k) {
        const int nb = (h[k].geom.N + kPtb - 1) / kPtb;
        for (int q = 0; q < nb; ++q) bi_host[h[k].block0 + q] = k;
    }
    if (n > d_cap) {
        if (d) cudaFree(d);
        d_cap = std::max(n, 2 * d_cap);
        if (cudaMalloc(&d, d_cap * sizeof(Inst)) != cudaSuccess) {
            cudaGetLastError();
            d = nullptr;
            d_cap = 0;
            return set_error(ZM_ERR_NOMEM, "batch: descriptor allocation failed");
        }
    }
    if (nblocks > bi_cap) {
        if (block_inst) cudaFree(block_inst);
        bi_cap = std::max(nblocks, 2 * bi_cap);
        if (cudaMalloc(&block_inst, bi_cap * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            block_inst = nullptr;
            bi_cap = 0;
            return set_error(ZM_ERR_NOMEM, "batch: block table allocation failed");
        }
    }
    // stream-ordered after earlier work that read the old tables; the host vectors stay alive
    // until the next plan(), which first synchronises the stream
    cudaStreamSynchronize(stream);
    int rc = cuda_check(cudaMemcpyAsync(d, h.data(), n * sizeof(Inst), cudaMemcpyHostToDevice, stream),
                        "batch descriptor upload");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(block_inst, bi_host.data(), nblocks * sizeof(int),
                                             cudaMemcpyHostToDevice, stream),
                             "batch block table upload");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(stream), "batch plan");
    return rc;
}

int Batch::set_chunk(int chunk)
{
    chunk_override = chunk;
    return plan();
}

// ---- autotuner ------------------------------------------------------------------------------

namespace {
std::mutex g_tune_mutex;
std::map<std::string, int> g_tune_memo;  // key -> chosen work-item size, for this process

std::string tune_key(const Batch &b, bool shape_neutral = false)
{
    cudaDeviceProp prop;
    std::memset(&prop, 0, sizeof(prop));
    cudaGetDeviceProperties(&prop, b.device);
    std::string name = prop.name;
    for (auto &ch : name)
        if (ch == ' ' || ch == '|') ch = '_';
    long double pairs = 0;
    int maxtiles = 0;
    for (auto &I : b.h) {
        pairs += (long double)I.geom.N * I.geom.N;
        maxtiles = std::max(maxtiles, shape_neutral ? make_tiling(I.geom).ntiles : I.tiling.ntiles);
    }
    const int pb = (int)std::floor(std::log2((double)pairs + 1.0));
    const int ib = (int)std::floor(std::log2((double)b.h.size()));
    const int tb = (int)std::floor(std::log2((double)maxtiles + 1.0));
    return name + "|sm" + std::to_string(b.sms) + "|occ" + std::to_string(b.occ) + "|n2^" +
           std::to_string(ib) + "|pairs2^" + std::to_string(pb) + "|tiles2^" + std::to_string(tb);
}

bool cache_lookup(const char *path, const std::string &key, int *chunk)
{
    if (!path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char k[512];
    int c = 0;
    float ms = 0;
    bool found = false;
    while (std::fscanf(f, "%511s %d %f", k, &c, &ms) == 3)
        if (key == k) {  // the last entry for a key wins
            *chunk = c;
            found = true;
        }
    std::fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, int chunk, float ms)
{
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %.4f\n", key.c_str(), chunk, ms);
    std::fclose(f);
}
}  // namespace

int Batch::autotune(const char *cache_path, int *chosen, float *best_ms)
{
    if (h.empty()) return ZM_OK;
    const std::string key = tune_key(*this);
    int c = 0;
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tune_memo.find(key);
        if (it != g_tune_memo.end()) c = it->second;
    }
    if (c <= 0 && cache_lookup(cache_path, key, &c)) {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tune_memo[key] = c;
    }
    if (c > 0) {
        if (chosen) *chosen = c;
        if (best_ms) *best_ms = -1.0f;
        return set_chunk(c);
    }
    int maxtiles = 1;
    for (auto &I : h) maxtiles = std::max(maxtiles, I.tiling.ntiles);
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
        return set_error(ZM_ERR_CUDA, "autotune: event creation failed");
    Prof *saved = prof;
    Prof quiet;  // keep the tuning launches out of the caller's counters
    prof = &quiet;
    float best = 1e30f;
    int best_c = 1, rc = ZM_OK;
    for (int cand = 1; cand <= 32 && cand <= maxtiles; cand *= 2) {
        rc = set_chunk(cand);
        if (rc) break;
        rc = derivative(0, stream);  // warm-up
        float ms = 0.f, total = 0.f;
        for (int rep = 0; rep < 2 && !rc; ++rep) {
            cudaEventRecord(a, stream);
            rc = derivative(0, stream);
            cudaEventRecord(b, stream);
            cudaEventSynchronize(b);
            cudaEventElapsedTime(&ms, a, b);
            total += ms;
        }
        if (rc) break;
        if (total < best) {
            best = total;
            best_c = cand;
        }
    }
    prof = saved;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    prof_release(quiet);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tune_memo[key] = best_c;
    }
    cache_store(cache_path, key, best_c, best / 2);
    if (chosen) *chosen = best_c;
    if (best_ms) *best_ms = best / 2;
    return set_chunk(best_c);
}

float Batch::time_eval(int *rc)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        *rc = set_error(ZM_ERR_CUDA, "autotune: event creation failed");
        return 0.f;
    }
    float total = 0.f, ms = 0.f;
    *rc = derivative(0, stream);  // warm-up
    for (int rep = 0; rep < 2 && !*rc; ++rep) {
        cudaEventRecord(a, stream);
        *rc = derivative(0, stream);
        cudaEventRecord(b, stream);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
        total += ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return total;
}

int Batch::set_shape(int k)
{
    if (k < 0 || k >= kNumShapes) return set_error(ZM_ERR_INVALID, "tile shape: unknown candidate");
    shape = k;
    for (auto &I : h) {
        I.tiling = make_tiling_shape(I.geom, kShapes[k][0], kShapes[k][1]);
        // padding slots of the new tiling must hold zero-strength sources, not another shape's
        // nodes: clear the records of the whole capacity
        const size_t cap = tile_capacity(I.geom.n1, I.geom.n2);
        cudaMemsetAsync(I.near_rec, 0, cap * 256 * kRec32 * sizeof(float), stream);
        cudaMemsetAsync(I.tinfo, 0, cap * sizeof(float4), stream);
        init_far_records(I.far_rec, (int)cap, (float)(I.delta * I.delta), stream);
    }
    int rc = cuda_check(cudaGetLastError(), "tile shape change");
    return rc ? rc : plan();
}

int Batch::autotune_tiles(const char *cache_path, int *shape_out, int *chunk_out, float *best_ms)
{
    if (h.empty()) return ZM_OK;
    const std::string key = tune_key(*this, true) + "|tiles";
    int code = 0;  // shape * 1000 + chunk
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tune_memo.find(key);
        if (it != g_tune_memo.end()) code = it->second;
    }
    if (code <= 0 && cache_lookup(cache_path, key, &code)) {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tune_memo[key] = code;
    }
    int rc = ZM_OK;
    float best = -1.0f;
    if (code <= 0 || code / 1000 >= kNumShapes) {
        Prof *saved = prof;
        Prof quiet;  // keep the tuning launches out of the caller's counters
        prof = &quiet;
        // patch shapes at the default work-item size, then work-item sizes for the best shape
        int best_k = 0;
        float best_t = 1e30f;
        for (int k = 0; k < kNumShapes && !rc; ++k) {
            rc = set_shape(k);
            if (!rc) rc = set_chunk(0);
            const float t = rc ? 0.f : time_eval(&rc);
            if (!rc && t < best_t) {
                best_t = t;
                best_k = k;
            }
        }
        if (!rc) rc = set_shape(best_k);
        int maxtiles = 1;
        for (auto &I : h) maxtiles = std::max(maxtiles, I.tiling.ntiles);
        int best_c = 1;
        best_t = 1e30f;
        for (int cand = 1; cand <= 32 && cand <= maxtiles && !rc; cand *= 2) {
            rc = set_chunk(cand);
            const float t = rc ? 0.f : time_eval(&rc);
            if (!rc && t < best_t) {
                best_t = t;
                best_c = cand;
            }
        }
        prof = saved;
        prof_release(quiet);
        if (rc) return rc;
        code = best_k * 1000 + best_c;
        best = best_t / 2;
        {
            std::lock_guard<std::mutex> lk(g_tune_mutex);
            g_tune_memo[key] = code;
        }
        cache_store(cache_path, key, code, best);
    }
    rc = set_shape(code / 1000);
    if (!rc) rc = set_chunk(code % 1000);
    if (shape_out) *shape_out = code / 1000;
    if (chunk_out) *chunk_out = code % 1000;
    if (best_ms) *best_ms = best;
    return rc;
}

int Batch::set_dt(double dt)
{
    bool changed = false;
    for (auto &I : h)
        if (I.dt != dt) {
            I.dt = dt;
            changed = true;
        }
    return changed ? plan() : ZM_OK;
}

void Batch::drop_graph()
{
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
}

int Batch::derivative(int yin, cudaStream_t s)
{
    if (h.empty()) return ZM_OK;
    cudaEvent_t ev = nullptr;
    prof_begin(*prof, s, ZM_K_GEOMETRY, &ev);
    batch_geometry_kernel<<<nblocks, kPtb, 0, s>>>(d, block_inst, yin);
    prof_end(*prof, s, ZM_K_GEOMETRY, ev);
    int rc = cuda_check(cudaGetLastError(), "batch geometry launch");
    if (rc) return rc;
    prof_begin(*prof, s, ZM_K_BR, &ev);
    bool any_cutoff = false;
    for (const auto &I : h) any_cutoff = any_cutoff || I.cutoff > 0;
    rc = tc ? launch_br32tc_batch(d, (int)h.size(), nitems, ctas, counter, err, s, any_cutoff)
            : launch_br32_batch(d, (int)h.size(), nitems, ctas, counter, err, s, any_cutoff);
    prof_end(*prof, s, ZM_K_BR, ev);
    for (auto &I : h) prof->acc.pairs += (int64_t)I.geom.N * I.geom.N;
    if (rc) return rc;
    prof_begin(*prof, s, ZM_K_REDUCE, &ev);
    batch_finish_kernel<<<nblocks, kPtb, 0, s>>>(d, block_inst, counter);
    prof_end(*prof, s, ZM_K_REDUCE, ev);
    return cuda_check(cudaGetLastError(), "batch finish launch");
}

int Batch::vorticity(int yin, int mode, int yout, double ca, double cb, cudaStream_t s)
{
    if (h.empty()) return ZM_OK;
    cudaEvent_t ev = nullptr;
    prof_begin(*prof, s, ZM_K_VORT, &ev);
    if (mode == 0)
        batch_vorticity_kernel<0><<<nblocks, kPtb, 0, s>>>(d, block_inst, yin, yout, ca, cb);
    else
        batch_vorticity_kernel<1><<<nblocks, kPtb, 0, s>>>(d, block_inst, yin, yout, ca, cb);
    prof_end(*prof, s, ZM_K_VORT, ev);
    return cuda_check(cudaGetLastError(), "batch vorticity launch");
}

// SSP-RK3 (Shu-Osher): stage st writes ca y0 + cb (y_st + dt L(y_st)), dt per interface.
int Batch::rk3_step_launches(cudaStream_t s)
{
    static const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
    static const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
    static const int yin[3] = {0, 1, 2}, yout[3] = {1, 2, 0};
    for (int st = 0; st < 3; ++st) {
        int rc = derivative(yin[st], s);
        if (!rc) rc = vorticity(yin[st], 1, yout[st], ca[st], cb[st], s);
        if (rc) return rc;
    }
    return ZM_OK;
}

int Batch::step(int nsteps, bool use_graph)
{
    if (nsteps <= 0 || h.empty()) return ZM_OK;
    if (prof->on || !use_graph) {  // event timing needs plain launches
        for (int k = 0; k < nsteps; ++k) {
            int rc = rk3_step_launches(stream);
            if (rc) return rc;
        }
        return ZM_OK;
    }
    if (!gexec) {
        cudaGraph_t graph = nullptr;
        int rc = cuda_check(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal),
                            "step graph capture");
        if (rc) return rc;
        rc = rk3_step_launches(cap);
        cudaError_t e = cudaStreamEndCapture(cap, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        rc = cuda_check(e, "step graph capture end");
        if (!rc) rc = cuda_check(cudaGraphInstantiate(&gexec, graph, 0), "step graph instantiate");
        if (graph) cudaGraphDestroy(graph);
        if (rc) return rc;
        // the capture counted launches and pairs of one step; those launches never ran
        for (int k = 0; k < ZM_K_COUNT; ++k) prof->acc.launches[k] -= (k == ZM_K_FFT) ? 0 : 3;
        for (auto &I : h) prof->acc.pairs -= 3LL * I.geom.N * I.geom.N;
    }
    for (int k = 0; k < nsteps; ++k) {
        int rc = cuda_check(cudaGraphLaunch(gexec, stream), "step graph launch");
        if (rc) return rc;
    }
    for (int k = 0; k < ZM_K_COUNT; ++k) prof->acc.launches[k] += (k == ZM_K_FFT) ? 0 : 3LL * nsteps;
    for (auto &I : h) prof->acc.pairs += 3LL * nsteps * (int64_t)I.geom.N * I.geom.N;
    return ZM_OK;
}

int Batch::status()
{
    int hs = 0;
    int rc = cuda_check(cudaMemcpyAsync(&hs, err, sizeof(int), cudaMemcpyDeviceToHost, stream),
                        "batch status read");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(stream), "batch synchronize");
    if (!rc && (hs & kErrTimeout)) {
        cudaMemsetAsync(err, 0, sizeof(int), stream);
        rc = set_error(ZM_ERR_TIMEOUT, (hs & kErrDrain)
                                           ? "a bounded device-side wait gave up, and so did the wait for "
                                             "the copies in flight (status word set)"
                                           : "a bounded device-side wait gave up (status word set)");
    }
    return rc;
}

// ---- hooks used by zm_api.cu for an FP32C context (a batch of one) ---------------------------

Batch *batch_new_single(const zm_mesh *m, double atwood, double g, double mu, double delta, int *rc)
{
    Batch *b = new (std::nothrow) Batch();
    if (!b) {
        *rc = set_error(ZM_ERR_NOMEM, "batch: host allocation failed");
        return nullptr;
    }
    *rc = b->init(1, m, &atwood, g, mu, &delta);
    if (*rc) {
        delete b;
        return nullptr;
    }
    return b;
}
void batch_delete(Batch *b) { delete b; }
const Inst &batch_inst(Batch *b, int k) { return b->h[k]; }
void batch_bind(Batch *b, cudaStream_t s, Prof *p)
{
    if (b->stream != s) b->drop_graph();
    b->stream = s;
    b->prof = p;
}
int batch_derivative(Batch *b, int yin) { return b->derivative(yin, b->stream); }
int batch_vorticity_rate(Batch *b, int yin) { return b->vorticity(yin, 0, 0, 0, 0, b->stream); }
int batch_step(Batch *b, double dt, int nsteps)
{
    int rc = b->set_dt(dt);
    return rc ? rc : b->step(nsteps, true);
}
int batch_status(Batch *b) { return b->status(); }
int batch_set_cutoff(Batch *b, int index, double cutoff)
{
    for (int k = 0; k < (int)b->h.size(); ++k)
        if (index < 0 || index == k) b->h[k].cutoff = cutoff;
    return b->plan();
}
int batch_keep_phi(Batch *b, int on)
{
    for (auto &I : b->h) I.keep_phi = on;
    return b->plan();
}
int batch_autotune(Batch *b, const char *path, int *chosen, float *ms) { return b->autotune(path, chosen, ms); }
int batch_get_tile_shape(Batch *b, int *tp1, int *tp2)
{
    *tp1 = kShapes[b->shape][0];
    *tp2 = kShapes[b->shape][1];
    return ZM_OK;
}

int batch_set_far_path(Batch *b, int path)
{
    if (path != ZM_FAR_TENSOR && path != ZM_FAR_CUDA)
        return set_error(ZM_ERR_INVALID, "far path must be ZM_FAR_TENSOR or ZM_FAR_CUDA");
    b->tc = (path == ZM_FAR_TENSOR);
    b->occ = b->tc ? br32tc_occupancy() : br32_occupancy();
    return b->plan();
}

int batch_get_far_path(Batch *b) { return b->tc ? ZM_FAR_TENSOR : ZM_FAR_CUDA; }

int batch_set_tile_shape(Batch *b, int tp1, int tp2)
{
    for (int k = 0; k < kNumShapes; ++k)
        if (kShapes[k][0] == tp1 && kShapes[k][1] == tp2) return b->set_shape(k);
    return set_error(ZM_ERR_INVALID, "tile shape (tp1, tp2) must be (16,16), (8,32), (32,8), (4,64) or (64,4)");
}

int batch_autotune_tiles(Batch *b, const char *path, int *tp1, int *tp2, int *chunk, float *ms)
{
    int k = 0;
    const int rc = b->autotune_tiles(path, &k, chunk, ms);
    if (tp1) *tp1 = kShapes[k][0];
    if (tp2) *tp2 = kShapes[k][1];
    return rc;
}

ZM_BOUNDS_READER(bounds_batch)

}  // namespace zm

// ---- C ABI -------------------------------------------------------------------------------------

using namespace zm;

struct zm_batch {
    Batch b;
};

static bool batch_index_ok(zm_batch *bt, int32_t index)
{
    return bt && index >= 0 && index < (int32_t)bt->b.h.size();
}

static bool dev_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static int batch_copy(zm_batch *bt, void *dst, const void *src, size_t bytes, bool *host)
{
    const bool sd = dev_ptr(src), dd = dev_ptr(dst);
    if (!sd || !dd) *host = true;
    return cuda_check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, bt->b.stream), "batch copy");
}

extern "C" {

int zm_batch_create(int32_t count, const zm_mesh *meshes, const double *atwood, double g, double mu,
                    const double *delta, zm_batch **out)
{
    if (!out || !meshes || !atwood || !delta || count < 1 || count > (1 << 16))
        return set_error(ZM_ERR_INVALID, "zm_batch_create: bad arguments");
    *out = nullptr;
    if (!std::isfinite(g) || !(mu >= 0) || !std::isfinite(mu))
        return set_error(ZM_ERR_INVALID, "zm_batch_create: g must be finite and mu >= 0");
    for (int k = 0; k < count; ++k) {
        const zm_mesh &m = meshes[k];
        if (m.n1 < 5 || m.n2 < 5 || (int64_t)m.n1 * m.n2 > (1 << 24) || !(m.L1 > 0) || !(m.L2 > 0) ||
            !std::isfinite(m.L1) || !std::isfinite(m.L2) || !std::isfinite(atwood[k]) ||
            !(delta[k] > 0) || !std::isfinite(delta[k]))
            return set_error(ZM_ERR_INVALID, "zm_batch_create: bad mesh or parameter at index " +
                                                 std::to_string(k));
    }
    zm_batch *bt = new (std::nothrow) zm_batch();
    if (!bt) return set_error(ZM_ERR_NOMEM, "zm_batch_create: host allocation failed");
    int rc = bt->b.init(count, meshes, atwood, g, mu, delta);
    if (rc) {
        delete bt;
        return rc;
    }
    *out = bt;
    return ZM_OK;
}

int zm_batch_set_stream(zm_batch *bt, void *stream)
{
    if (!bt) return set_error(ZM_ERR_INVALID, "zm_batch_set_stream: null batch");
    batch_bind(&bt->b, static_cast<cudaStream_t>(stream), bt->b.prof);
    return ZM_OK;
}

int zm_batch_set_state(zm_batch *bt, int32_t index, const double *z, const double *w)
{
    if (!batch_index_ok(bt, index) || !z || !w)
        return set_error(ZM_ERR_INVALID, "zm_batch_set_state: bad arguments");
    const Inst &I = bt->b.h[index];
    const size_t N = I.geom.N;
    bool host = false;
    int rc = batch_copy(bt, I.y[0], z, 3 * N * sizeof(double), &host);
    if (!rc) rc = batch_copy(bt, I.y[0] + 3 * N, w, 2 * N * sizeof(double), &host);
    if (!rc && host) rc = cuda_check(cudaStreamSynchronize(bt->b.stream), "zm_batch_set_state");
    return rc;
}

int zm_batch_get_state(zm_batch *bt, int32_t index, double *z, double *w)
{
    if (!batch_index_ok(bt, index)) return set_error(ZM_ERR_INVALID, "zm_batch_get_state: bad arguments");
    const Inst &I = bt->b.h[index];
    const size_t N = I.geom.N;
    bool host = false;
    int rc = ZM_OK;
    if (z) rc = batch_copy(bt, z, I.y[0], 3 * N * sizeof(double), &host);
    if (!rc && w) rc = batch_copy(bt, w, I.y[0] + 3 * N, 2 * N * sizeof(double), &host);
    if (!rc && host) rc = bt->b.status();
    return rc;
}

int zm_batch_velocity(zm_batch *bt)
{
    if (!bt) return set_error(ZM_ERR_INVALID, "zm_batch_velocity: null batch");
    const NvtxRange range("zm_batch_velocity");
    int rc = bt->b.derivative(0, bt->b.stream);
    if (!rc) rc = bt->b.vorticity(0, 0, 0, 0, 0, bt->b.stream);
    return rc;
}

int zm_batch_get_velocity(zm_batch *bt, int32_t index, double *u, double *wdot)
{
    if (!batch_index_ok(bt, index)) return set_error(ZM_ERR_INVALID, "zm_batch_get_velocity: bad arguments");
    const Inst &I = bt->b.h[index];
    const size_t N = I.geom.N;
    bool host = false;
    int rc = ZM_OK;
    if (u) rc = batch_copy(bt, u, I.u, 3 * N * sizeof(double), &host);
    if (!rc && wdot) rc = batch_copy(bt, wdot, I.y[2], 2 * N * sizeof(double), &host);
    if (!rc && host) rc = bt->b.status();
    return rc;
}

int zm_batch_step(zm_batch *bt, double dt, int32_t nsteps)
{
    if (!bt || !std::isfinite(dt) || nsteps < 0) return set_error(ZM_ERR_INVALID, "zm_batch_step: bad arguments");
    const NvtxRange range("zm_batch_step");
    int rc = bt->b.set_dt(dt);
    return rc ? rc : bt->b.step(nsteps, true);
}

int zm_batch_sync(zm_batch *bt)
{
    if (!bt) return set_error(ZM_ERR_INVALID, "zm_batch_sync: null batch");
    return bt->b.status();
}

int zm_batch_set_chunk(zm_batch *bt, int32_t chunk)
{
    if (!bt || chunk < 0) return set_error(ZM_ERR_INVALID, "zm_batch_set_chunk: bad arguments");
    return bt->b.set_chunk(chunk);
}

int zm_batch_autotune(zm_batch *bt, const char *cache_path, int32_t *chosen, float *best_ms)
{
    if (!bt) return set_error(ZM_ERR_INVALID, "zm_batch_autotune: null batch");
    int c = 0;
    int rc = bt->b.autotune(cache_path, &c, best_ms);
    if (chosen) *chosen = c;
    return rc;
}

int zm_batch_set_tile_shape(zm_batch *bt, int32_t tp1, int32_t tp2)
{
    if (!bt) return set_error(ZM_ERR_INVALID, "zm_batch_set_tile_shape: null batch");
    return batch_set_tile_shape(&bt->b, tp1, tp2);
}

int zm_batch_set_far_path(zm_batch *bt, int32_t path)
{
    if (!bt) return set_error(ZM_ERR_INVALID, "zm_batch_set_far_path: null batch");
    return batch_set_far_path(&bt->b, path);
}

int zm_batch_get_far_path(zm_batch *bt, int32_t *path)
{
    if (!bt || !path) return set_error(ZM_ERR_INVALID, "zm_batch_get_far_path: null argument");
    *path = batch_get_far_path(&bt->b);
    return ZM_OK;
}

int zm_batch_get_tile_shape(zm_batch *bt, int32_t *tp1, int32_t *tp2)
{
    if (!bt || !tp1 || !tp2) return set_error(ZM_ERR_INVALID, "zm_batch_get_tile_shape: null argument");
    *tp1 = kShapes[bt->b.shape][0];
    *tp2 = kShapes[bt->b.shape][1];
    return ZM_OK;
}

int zm_batch_autotune_tiles(zm_batch *bt, const char *cache_path, int32_t *tp1, int32_t *tp2, int32_t *chunk,
                            float *best_ms)
{
    if (!bt) return set_error(ZM_ERR_INVALID, "zm_batch_autotune_tiles: null batch");
    int a = 0, b = 0, c = 0;
    const int rc = batch_autotune_tiles(&bt->b, cache_path, &a, &b, &c, best_ms);
    if (tp1) *tp1 = a;
    if (tp2) *tp2 = b;
    if (chunk) *chunk = c;
    return rc;
}

int zm_batch_set_cutoff(zm_batch *bt, int32_t index, double cutoff)
{
    if (!bt || index < -1 || index >= (int32_t)bt->b.h.size() || !(cutoff >= 0) || !std::isfinite(cutoff))
        return set_error(ZM_ERR_INVALID, "zm_batch_set_cutoff: bad arguments");
    return batch_set_cutoff(&bt->b, index, cutoff);
}

int zm_batch_info(zm_batch *bt, int64_t *points, int64_t *pairs_per_eval, int64_t *work_items,
                  int32_t *ctas)
{
    if (!bt) return set_error(ZM_ERR_INVALID, "zm_batch_info: null batch");
    int64_t pts = 0, prs = 0;
    for (auto &I : bt->b.h) {
        pts += I.geom.N;
        prs += (int64_t)I.geom.N * I.geom.N;
    }
    if (points) *points = pts;
    if (pairs_per_eval) *pairs_per_eval = prs;
    if (work_items) *work_items = bt->b.nitems;
    if (ctas) *ctas = bt->b.ctas;
    return ZM_OK;
}

int zm_batch_set_profiling(zm_batch *bt, int on)
{
    if (!bt) return set_error(ZM_ERR_INVALID, "zm_batch_set_profiling: null batch");
    prof_fold(*bt->b.prof, bt->b.stream);
    std::memset(&bt->b.prof->acc, 0, sizeof(zm_profile));
    bt->b.prof->on = on ? 1 : 0;
    return ZM_OK;
}

int zm_batch_get_profile(zm_batch *bt, zm_profile *out)
{
    if (!bt || !out) return set_error(ZM_ERR_INVALID, "zm_batch_get_profile: null argument");
    prof_fold(*bt->b.prof, bt->b.stream);
    int rc = cuda_check(cudaStreamSynchronize(bt->b.stream), "zm_batch_get_profile");
    *out = bt->b.prof->acc;
    return rc;
}

void zm_batch_destroy(zm_batch *bt) { delete bt; }

}  // extern "C"
