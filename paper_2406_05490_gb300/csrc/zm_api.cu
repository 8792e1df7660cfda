// zm_api.cu -- the C ABI of libzm.so (declared and documented in include/zm.h): context
// lifecycle, argument checks, host/device pointer handling, and the orchestration of one
// derivative evaluation (paper Sec. 3.1 ZModel) and of SSP-RK3 steps (Sec. 3.1 TimeIntegrator).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "zm_internal.cuh"

namespace zm {

static thread_local std::string g_last_error;

int set_error(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

int cuda_check(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return ZM_OK;
    return set_error(ZM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ---- profiling ------------------------------------------------------------------------------

void prof_fold(Prof &pr, cudaStream_t s)
{
    if (pr.live.empty()) return;
    cudaStreamSynchronize(s);
    for (auto &e : pr.live) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) pr.acc.ms[e.cls] += ms;
        pr.pool.push_back(e.a);
        pr.pool.push_back(e.b);
    }
    pr.live.clear();
}

void prof_release(Prof &pr)
{
    for (auto &e : pr.live) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    for (auto e : pr.pool) cudaEventDestroy(e);
    pr.live.clear();
    pr.pool.clear();
}

static cudaEvent_t prof_event(Prof &pr)
{
    if (pr.pool.empty()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
    cudaEvent_t e = pr.pool.back();
    pr.pool.pop_back();
    return e;
}

void prof_begin(Prof &pr, cudaStream_t s, int cls, cudaEvent_t *a)
{
    pr.acc.launches[cls] += 1;
    *a = nullptr;
    if (!pr.on) return;
    if (pr.live.size() >= 4096) prof_fold(pr, s);
    *a = prof_event(pr);
    if (*a) cudaEventRecord(*a, s);
}

void prof_end(Prof &pr, cudaStream_t s, int cls, cudaEvent_t a)
{
    if (!pr.on || !a) return;
    cudaEvent_t b = prof_event(pr);
    if (!b) return;
    cudaEventRecord(b, s);
    pr.live.push_back({cls, a, b});
}

// hooks into zm_batch.cu (an FP32C context is a batch of one interface)
Batch *batch_new_single(const zm_mesh *m, double atwood, double g, double mu, double delta, int *rc);
void batch_delete(Batch *b);
const Inst &batch_inst(Batch *b, int k);
void batch_bind(Batch *b, cudaStream_t s, Prof *p);
int batch_derivative(Batch *b, int yin);
int batch_vorticity_rate(Batch *b, int yin);
int batch_step(Batch *b, double dt, int nsteps);
int batch_status(Batch *b);
int batch_keep_phi(Batch *b, int on);
int batch_set_cutoff(Batch *b, int index, double cutoff);
int batch_autotune(Batch *b, const char *path, int *chosen, float *ms);
int batch_autotune_tiles(Batch *b, const char *path, int *tp1, int *tp2, int *chunk, float *ms);
int batch_set_tile_shape(Batch *b, int tp1, int tp2);
int batch_set_far_path(Batch *b, int path);
int batch_get_far_path(Batch *b);
int batch_get_tile_shape(Batch *b, int *tp1, int *tp2);

static int stage_index(zm_ctx *c, const double *y) { return y == c->y0 ? 0 : (y == c->ya ? 1 : 2); }

// ---- derivative ---------------------------------------------------------------------------------

// One evaluation of L(y): after it, c->u holds dz/dt and c->phi holds Phi.
int derivative(zm_ctx *c, const double *y)
{
    if (c->batch) {
        batch_bind(c->batch, c->stream, &c->prof);
        if (c->order == ZM_ORDER_MEDIUM) {
            // normals and q, then u and Phi from the FFT velocity; the batched sum then
            // replaces u and leaves Phi (keep_phi)
            int rc = launch_geometry(c, y);
            if (!rc) rc = launch_riesz(c, y);
            if (rc) return rc;
        }
        return batch_derivative(c->batch, stage_index(c, y));
    }
    if (c->df64) return df_derivative(c, y);
    int rc = launch_geometry(c, y);
    if (rc) return rc;
    if (c->order == ZM_ORDER_LOW) return launch_riesz(c, y);
    if (c->order == ZM_ORDER_MEDIUM) {
        // Phi from the FFT velocity (written with u, which the BR sum then replaces)
        rc = launch_riesz(c, y);
        if (rc) return rc;
        rc = launch_br(c, y);
        return rc ? rc : launch_reduce(c, false);
    }
    rc = launch_br(c, y);
    if (rc) return rc;
    return launch_reduce(c, true);
}

static bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static int copy_in(zm_ctx *c, double *dst, const double *src, size_t count)
{
    const cudaMemcpyKind k = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    return cuda_check(cudaMemcpyAsync(dst, src, count * sizeof(double), k, c->stream), "copy in");
}

static int copy_out(zm_ctx *c, double *dst, const double *src, size_t count, bool *to_host)
{
    const bool dev = is_device_ptr(dst);
    if (!dev) *to_host = true;
    const cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    return cuda_check(cudaMemcpyAsync(dst, src, count * sizeof(double), k, c->stream), "copy out");
}

static int read_status(zm_ctx *c)
{
    int h = 0;
    int rc = cuda_check(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
                        "status read");
    if (rc) return rc;
    rc = cuda_check(cudaStreamSynchronize(c->stream), "stream synchronize");
    if (rc) return rc;
    if (h & kErrTimeout) {
        cudaMemsetAsync(c->err, 0, sizeof(int), c->stream);
        return set_error(ZM_ERR_TIMEOUT, (h & kErrDrain)
                                             ? "a bounded device-side wait gave up, and so did the wait for "
                                               "the copies in flight (status word set)"
                                             : "a bounded device-side wait gave up (status word set)");
    }
    if (c->batch) {
        batch_bind(c->batch, c->stream, &c->prof);
        return batch_status(c->batch);
    }
    return ZM_OK;
}

ZM_BOUNDS_READER(bounds_api)

}  // namespace zm

using namespace zm;

extern "C" {

const char *zm_error_string(int code)
{
    switch (code) {
    case ZM_OK: return "ok";
    case ZM_ERR_INVALID: return "invalid argument";
    case ZM_ERR_NOMEM: return "out of memory";
    case ZM_ERR_CUDA: return "CUDA error";
    case ZM_ERR_TIMEOUT: return "device-side wait timed out";
    case ZM_ERR_UNSUPPORTED: return "unsupported configuration";
    case ZM_ERR_NONFINITE: return "state is not finite";
    case ZM_ERR_BUSY: return "resource budget exhausted";
    default: return "unknown status";
    }
}

const char *zm_last_error(void) { return g_last_error.c_str(); }


void zm_destroy(zm_ctx *c)
{
    if (!c) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    prof_release(c->prof);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->batch) {  // state buffers belong to the batch
        batch_delete(c->batch);
        c->batch = nullptr;
        c->y0 = c->ya = c->yb = c->u = c->phi = c->q = nullptr;
    }
    void *bufs[] = {c->y0, c->ya, c->yb, c->u, c->phi, c->q, c->nrm, c->src, c->part,
                    c->fa, c->fb, c->tw1, c->tw2, c->twl1, c->twl2, c->twh, c->err, c->flag};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (prev >= 0) cudaSetDevice(prev);
    delete c;
}

int zm_create(const zm_mesh *mesh, double atwood, double g, double mu, double delta, int order,
              zm_ctx **out)
{
    if (!mesh || !out) return set_error(ZM_ERR_INVALID, "zm_create: null mesh or out pointer");
    *out = nullptr;
    const int ord = order & 0xff;
    const int fp32c = (order & ZM_PREC_FP32C) ? 1 : 0;
    const int df64 = (order & ZM_PREC_DF64) ? 1 : 0;
    if ((order & ~(0xff | ZM_PREC_FP32C | ZM_PREC_DF64)) != 0 || ord > ZM_ORDER_HIGH || (fp32c && df64))
        return set_error(ZM_ERR_INVALID, "zm_create: unknown order/precision flags");
    if (df64 && ord != ZM_ORDER_LOW)
        return set_error(ZM_ERR_UNSUPPORTED, "zm_create: double-word precision is built for low order only");
    if (mesh->n1 < 5 || mesh->n2 < 5 || (int64_t)mesh->n1 * mesh->n2 > (1 << 26))
        return set_error(ZM_ERR_INVALID, "zm_create: mesh sides must be >= 5 and n1*n2 <= 2^26");
    if (!(mesh->L1 > 0) || !(mesh->L2 > 0) || !std::isfinite(mesh->L1) || !std::isfinite(mesh->L2))
        return set_error(ZM_ERR_INVALID, "zm_create: L1, L2 must be finite and > 0");
    if (!std::isfinite(atwood) || !std::isfinite(g) || !(mu >= 0) || !std::isfinite(mu))
        return set_error(ZM_ERR_INVALID, "zm_create: atwood, g must be finite and mu >= 0");
    if (ord == ZM_ORDER_HIGH && !(delta > 0 && std::isfinite(delta)))
        return set_error(ZM_ERR_INVALID, "zm_create: the Birkhoff-Rott core size delta must be > 0");
    const bool fft = (ord == ZM_ORDER_LOW || ord == ZM_ORDER_MEDIUM);
    if (ord == ZM_ORDER_MEDIUM && !(delta > 0 && std::isfinite(delta)))
        return set_error(ZM_ERR_INVALID, "zm_create: the Birkhoff-Rott core size delta must be > 0");
    if (fft && !mesh->periodic)
        return set_error(ZM_ERR_UNSUPPORTED,
                         "zm_create: low and medium order need a periodic mesh (periodic FFT solver)");
    if (fft && df64 && (!df_side_ok(mesh->n1) || !df_side_ok(mesh->n2)))
        return set_error(ZM_ERR_UNSUPPORTED,
                         "zm_create: double-word low order needs sides 2^a <= 4096 or R 2^a <= 8192 (3 <= a <= 12, R odd <= 19)");
    if (fft && !df64 && (!fft_side_ok(mesh->n1) || !fft_side_ok(mesh->n2)))
        return set_error(ZM_ERR_UNSUPPORTED,
                         "zm_create: low and medium order need sides R 2^a <= 8192 (a >= 3, R odd <= 19)");

    zm_ctx *c = new (std::nothrow) zm_ctx();
    if (!c) return set_error(ZM_ERR_NOMEM, "zm_create: host allocation failed");
    c->mesh = *mesh;
    c->atwood = atwood;
    c->g = g;
    c->mu = mu;
    c->delta = delta;
    c->order = ord;
    c->fp32c = fp32c;
    c->df64 = df64;
    c->stream = nullptr;
    cudaGetDevice(&c->device);
    Geom &G = c->geom;
    G.n1 = mesh->n1;
    G.n2 = mesh->n2;
    G.N = mesh->n1 * mesh->n2;
    G.L1 = mesh->L1;
    G.L2 = mesh->L2;
    geom_finish(G);
    G.periodic = mesh->periodic ? 1 : 0;
    const size_t N = G.N;

    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);

    auto alloc = [&](void **p, size_t bytes) -> bool {
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return true;
    };
    bool ok = alloc((void **)&c->err, sizeof(int)) && alloc((void **)&c->flag, sizeof(int));
    if (ok && (ord == ZM_ORDER_HIGH || ord == ZM_ORDER_MEDIUM) && fp32c) {
        int rc = ZM_OK;
        c->batch = batch_new_single(mesh, atwood, g, mu, delta, &rc);
        if (!c->batch) {
            zm_destroy(c);
            return rc;
        }
        if (ord == ZM_ORDER_MEDIUM && (rc = batch_keep_phi(c->batch, 1)) != ZM_OK) {
            zm_destroy(c);
            return rc;
        }
        const Inst &I = batch_inst(c->batch, 0);
        c->y0 = I.y[0];
        c->ya = I.y[1];
        c->yb = I.y[2];
        c->u = I.u;
        c->phi = I.phi;
        c->q = I.q;
        c->tiling = I.tiling;
    } else if (ok) {
        ok = alloc((void **)&c->y0, 5 * N * sizeof(double)) &&
             alloc((void **)&c->ya, 5 * N * sizeof(double)) &&
             alloc((void **)&c->yb, 5 * N * sizeof(double)) &&
             alloc((void **)&c->u, 3 * N * sizeof(double)) &&
             alloc((void **)&c->phi, N * sizeof(double)) && alloc((void **)&c->q, N * sizeof(double));
    }
    if (ok && (ord == ZM_ORDER_HIGH || ord == ZM_ORDER_MEDIUM) && !fp32c) {
        c->tiling = make_tiling(G);
        const size_t slots = (size_t)c->tiling.ntiles * c->tiling.ts;
        c->plan = plan_br(G, c->tiling, sms);
        c->src_bytes = slots * kRec64 * sizeof(double);
        ok = alloc(&c->src, c->src_bytes) &&
             alloc((void **)&c->part, (size_t)c->plan.nsplit * 3 * N * sizeof(double));
        // padding slots of edge tiles stay zero for good: zero strength, no contribution
        if (ok) ok = cudaMemset(c->src, 0, c->src_bytes) == cudaSuccess;
    }
    if (ok && fft) ok = alloc((void **)&c->nrm, 3 * N * sizeof(double));
    if (ok) ok = cudaMemset(c->err, 0, sizeof(int)) == cudaSuccess &&
                 cudaMemset(c->y0, 0, 5 * N * sizeof(double)) == cudaSuccess;
    if (!ok) {
        zm_destroy(c);
        return set_error(ZM_ERR_NOMEM, "zm_create: device allocation failed");
    }
    if (fft) {
        int rc = df64 ? df_setup(c) : fft_setup(c);
        if (rc) {
            zm_destroy(c);
            return rc;
        }
    }
    int rc = cuda_check(cudaDeviceSynchronize(), "zm_create");
    if (rc) {
        zm_destroy(c);
        return rc;
    }
    *out = c;
    return ZM_OK;
}

int zm_set_stream(zm_ctx *c, void *stream)
{
    if (!c) return set_error(ZM_ERR_INVALID, "zm_set_stream: null context");
    c->stream = static_cast<cudaStream_t>(stream);
    return ZM_OK;
}

int zm_set_state(zm_ctx *c, const double *z, const double *w)
{
    if (!c || !z || !w) return set_error(ZM_ERR_INVALID, "zm_set_state: null argument");
    const size_t N = c->geom.N;
    double *dst = c->df64 ? c->yb : c->y0;  // double word: stage FP64 in yb, convert into y0
    int rc = copy_in(c, dst, z, 3 * N);
    if (!rc) rc = copy_in(c, dst + 3 * N, w, 2 * N);
    if (!rc && c->df64) rc = df_convert(c, c->yb, c->y0, 5 * N, 1, 1);
    if (!rc && (!is_device_ptr(z) || !is_device_ptr(w)))
        rc = cuda_check(cudaStreamSynchronize(c->stream), "zm_set_state");
    return rc;
}

int zm_get_state(zm_ctx *c, double *z, double *w)
{
    if (!c) return set_error(ZM_ERR_INVALID, "zm_get_state: null context");
    const size_t N = c->geom.N;
    bool host = false;
    int rc = ZM_OK;
    const double *src = c->y0;
    if (c->df64) {  // FP64 copy of the state in yb (a stage buffer, free between calls)
        rc = df_convert(c, c->y0, c->yb, 5 * N, 1, 0);
        src = c->yb;
    }
    if (!rc && z) rc = copy_out(c, z, src, 3 * N, &host);
    if (!rc && w) rc = copy_out(c, w, src + 3 * N, 2 * N, &host);
    if (!rc && host) rc = read_status(c);
    return rc;
}

int zm_velocity(zm_ctx *c, const double *z, const double *w, double *u, double *wdot)
{
    if (!c || !u) return set_error(ZM_ERR_INVALID, "zm_velocity: null context or u");
    const NvtxRange range("zm_velocity");
    if ((z == nullptr) != (w == nullptr))
        return set_error(ZM_ERR_INVALID, "zm_velocity: give both z and w, or neither");
    const size_t N = c->geom.N;
    const double *y = c->y0;
    int rc = ZM_OK;
    if (z) {
        double *dst = c->df64 ? c->yb : c->ya;
        rc = copy_in(c, dst, z, 3 * N);
        if (!rc) rc = copy_in(c, dst + 3 * N, w, 2 * N);
        if (!rc && c->df64) rc = df_convert(c, c->yb, c->ya, 5 * N, 1, 1);
        y = c->ya;
    }
    if (!rc) rc = derivative(c, y);
    bool host = false;
    if (!rc && c->df64) {
        // dw/dt as double words into yb[3N, 5N), then both fields to FP64 in yb
        if (wdot) rc = df_vorticity(c, y, c->yb + 3 * N, nullptr, nullptr, 0, 0, 0, 0);
        if (!rc && wdot) rc = df_convert(c, c->yb + 3 * N, c->yb + 3 * N, 2 * N, 0, 0);
        if (!rc) rc = df_convert(c, c->u, c->yb, 3 * N, 0, 0);
        if (!rc && wdot) rc = copy_out(c, wdot, c->yb + 3 * N, 2 * N, &host);
        if (!rc) rc = copy_out(c, u, c->yb, 3 * N, &host);
        if (!rc && host) rc = read_status(c);
        return rc;
    }
    if (!rc && wdot && c->batch) {
        rc = batch_vorticity_rate(c->batch, stage_index(c, y));  // dw/dt into yb[0, 2N)
        if (!rc) rc = copy_out(c, wdot, c->yb, 2 * N, &host);
    } else if (!rc && wdot) {
        if (is_device_ptr(wdot)) {
            rc = launch_vorticity(c, y, wdot, nullptr, nullptr, 0, 0, 0, 0);
        } else {
            rc = launch_vorticity(c, y, c->yb, nullptr, nullptr, 0, 0, 0, 0);
            if (!rc) rc = copy_out(c, wdot, c->yb, 2 * N, &host);
        }
    }
    if (!rc) rc = copy_out(c, u, c->u, 3 * N, &host);
    if (!rc && host) rc = read_status(c);
    return rc;
}

// One SSP-RK3 step (Shu-Osher): stage s writes ca[s] * y0 + cb[s] * (y_s + dt L(y_s)).
static int rk3_step_launches(zm_ctx *c, double dt)
{
    static const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
    static const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
    const double *yin[3] = {c->y0, c->ya, c->yb};
    double *yout[3] = {c->ya, c->yb, c->y0};
    for (int st = 0; st < 3; ++st) {
        int rc = derivative(c, yin[st]);
        if (!rc && c->df64) rc = df_vorticity(c, yin[st], nullptr, c->y0, yout[st], dt, ca[st], cb[st], 1);
        else if (!rc) rc = launch_vorticity(c, yin[st], nullptr, c->y0, yout[st], dt, ca[st], cb[st], 1);
        if (rc) return rc;
    }
    return ZM_OK;
}

// Launch and pair counts of one captured step (what each replay adds to the counters).
static zm_profile step_counts(const zm_ctx *c)
{
    zm_profile d{};
    d.launches[ZM_K_GEOMETRY] = 3;
    d.launches[ZM_K_VORT] = 3;
    if (c->order == ZM_ORDER_LOW) {
        d.launches[ZM_K_FFT] = 9;
    } else if (c->order == ZM_ORDER_MEDIUM) {
        d.launches[ZM_K_GEOMETRY] = 6;
        d.launches[ZM_K_FFT] = 9;
        d.launches[ZM_K_BR] = 3;
        d.launches[ZM_K_REDUCE] = 3;
        d.pairs = 3LL * c->geom.N * c->geom.N;
    } else {
        d.launches[ZM_K_BR] = 3;
        d.launches[ZM_K_REDUCE] = 3;
        d.pairs = 3LL * c->geom.N * c->geom.N;
    }
    return d;
}

int zm_step(zm_ctx *c, double dt, int nsteps)
{
    if (!c) return set_error(ZM_ERR_INVALID, "zm_step: null context");
    const NvtxRange range("zm_step");
    if (!std::isfinite(dt) || nsteps < 0)
        return set_error(ZM_ERR_INVALID, "zm_step: dt must be finite and nsteps >= 0");
    if (c->batch && c->order == ZM_ORDER_HIGH) {
        batch_bind(c->batch, c->stream, &c->prof);
        return batch_step(c->batch, dt, nsteps);
    }
    if (nsteps == 0) return ZM_OK;
    if (c->prof.on) {  // event timing needs plain launches
        for (int s = 0; s < nsteps; ++s) {
            int rc = rk3_step_launches(c, dt);
            if (rc) return rc;
        }
        return ZM_OK;
    }
    if (!c->gexec || c->gdt != dt) {
        if (c->gexec) cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
        if (!c->cap && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess)
            return set_error(ZM_ERR_CUDA, "zm_step: stream creation failed");
        cudaStream_t user = c->stream;
        c->stream = c->cap;
        zm_profile before = c->prof.acc;
        cudaGraph_t graph = nullptr;
        int rc = cuda_check(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal), "zm_step capture");
        if (!rc) {
            rc = rk3_step_launches(c, dt);
            cudaError_t e = cudaStreamEndCapture(c->cap, &graph);
            if (!rc) rc = cuda_check(e, "zm_step capture end");
        }
        c->stream = user;
        c->prof.acc = before;  // the capture itself launched nothing
        if (!rc) rc = cuda_check(cudaGraphInstantiate(&c->gexec, graph, 0), "zm_step graph instantiate");
        if (graph) cudaGraphDestroy(graph);
        if (rc) return rc;
        c->gdt = dt;
        c->step_launches = step_counts(c);
    }
    for (int s = 0; s < nsteps; ++s) {
        int rc = cuda_check(cudaGraphLaunch(c->gexec, c->stream), "zm_step graph launch");
        if (rc) return rc;
    }
    for (int k = 0; k < ZM_K_COUNT; ++k) c->prof.acc.launches[k] += (int64_t)nsteps * c->step_launches.launches[k];
    c->prof.acc.pairs += (int64_t)nsteps * c->step_launches.pairs;
    return ZM_OK;
}

int zm_check_finite(zm_ctx *c)
{
    if (!c) return set_error(ZM_ERR_INVALID, "zm_check_finite: null context");
    int rc = c->df64 ? df_check_finite(c, c->y0, 5 * (size_t)c->geom.N, c->flag)
                     : check_finite(c, c->y0, 5 * (size_t)c->geom.N, c->flag);
    int h = 0;
    if (!rc) rc = cuda_check(cudaMemcpyAsync(&h, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
                             "finite flag read");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(c->stream), "zm_check_finite");
    if (!rc && h) rc = set_error(ZM_ERR_NONFINITE, "zm_check_finite: state holds NaN or Inf");
    return rc;
}

int zm_set_cutoff(zm_ctx *c, double cutoff)
{
    if (!c || !(cutoff >= 0) || !std::isfinite(cutoff))
        return set_error(ZM_ERR_INVALID, "zm_set_cutoff: bad arguments");
    if (!c->batch)
        return set_error(ZM_ERR_UNSUPPORTED, "zm_set_cutoff: the cutoff sum runs on FP32C contexts");
    batch_bind(c->batch, c->stream, &c->prof);
    return batch_set_cutoff(c->batch, 0, cutoff);
}

int zm_autotune(zm_ctx *c, const char *cache_path, int32_t *chosen)
{
    if (!c) return set_error(ZM_ERR_INVALID, "zm_autotune: null context");
    if (!c->batch) {  // only the FP32C all-pairs kernel has a tunable work decomposition
        if (chosen) *chosen = 0;
        return ZM_OK;
    }
    batch_bind(c->batch, c->stream, &c->prof);
    int ch = 0;
    int rc = batch_autotune(c->batch, cache_path, &ch, nullptr);
    if (chosen) *chosen = ch;
    return rc;
}

int zm_autotune_tiles(zm_ctx *c, const char *cache_path, int32_t *tp1, int32_t *tp2, int32_t *chunk)
{
    if (!c) return set_error(ZM_ERR_INVALID, "zm_autotune_tiles: null context");
    if (!c->batch) {  // only the FP32C all-pairs kernel is tiled this way
        if (tp1) *tp1 = 0;
        if (tp2) *tp2 = 0;
        if (chunk) *chunk = 0;
        return ZM_OK;
    }
    batch_bind(c->batch, c->stream, &c->prof);
    int a = 0, b = 0, k = 0;
    const int rc = batch_autotune_tiles(c->batch, cache_path, &a, &b, &k, nullptr);
    if (tp1) *tp1 = a;
    if (tp2) *tp2 = b;
    if (chunk) *chunk = k;
    return rc;
}

int zm_set_tile_shape(zm_ctx *c, int32_t tp1, int32_t tp2)
{
    if (!c) return set_error(ZM_ERR_INVALID, "zm_set_tile_shape: null context");
    if (!c->batch) return set_error(ZM_ERR_UNSUPPORTED, "zm_set_tile_shape: tiles belong to FP32C high/medium contexts");
    batch_bind(c->batch, c->stream, &c->prof);
    return batch_set_tile_shape(c->batch, tp1, tp2);
}

int zm_set_far_path(zm_ctx *c, int32_t path)
{
    if (!c) return set_error(ZM_ERR_INVALID, "zm_set_far_path: null context");
    if (!c->batch) return set_error(ZM_ERR_UNSUPPORTED, "zm_set_far_path: FP32C high/medium contexts only");
    batch_bind(c->batch, c->stream, &c->prof);
    return batch_set_far_path(c->batch, path);
}

int zm_get_far_path(zm_ctx *c, int32_t *path)
{
    if (!c || !path) return set_error(ZM_ERR_INVALID, "zm_get_far_path: null argument");
    if (!c->batch) return set_error(ZM_ERR_UNSUPPORTED, "zm_get_far_path: FP32C high/medium contexts only");
    *path = batch_get_far_path(c->batch);
    return ZM_OK;
}

int zm_get_tile_shape(zm_ctx *c, int32_t *tp1, int32_t *tp2)
{
    if (!c || !tp1 || !tp2) return set_error(ZM_ERR_INVALID, "zm_get_tile_shape: null argument");
    if (!c->batch) return set_error(ZM_ERR_UNSUPPORTED, "zm_get_tile_shape: tiles belong to FP32C high/medium contexts");
    int a = 0, b = 0;
    const int rc = batch_get_tile_shape(c->batch, &a, &b);
    *tp1 = a;
    *tp2 = b;
    return rc;
}

int zm_sync(zm_ctx *c)
{
    if (!c) return set_error(ZM_ERR_INVALID, "zm_sync: null context");
    return read_status(c);
}

int zm_set_profiling(zm_ctx *c, int on)
{
    if (!c) return set_error(ZM_ERR_INVALID, "zm_set_profiling: null context");
    if (on) zm_reset_profile(c);
    c->prof.on = on ? 1 : 0;
    return ZM_OK;
}

int zm_reset_profile(zm_ctx *c)
{
    if (!c) return set_error(ZM_ERR_INVALID, "zm_reset_profile: null context");
    prof_fold(c->prof, c->stream);
    std::memset(&c->prof.acc, 0, sizeof(c->prof.acc));
    return ZM_OK;
}

int zm_get_profile(zm_ctx *c, zm_profile *out)
{
    if (!c || !out) return set_error(ZM_ERR_INVALID, "zm_get_profile: null argument");
    prof_fold(c->prof, c->stream);
    int rc = cuda_check(cudaStreamSynchronize(c->stream), "zm_get_profile");
    *out = c->prof.acc;
    return rc;
}

}  // extern "C"
