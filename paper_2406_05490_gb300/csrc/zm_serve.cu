// zm_serve.cu -- a serving loop for interface solves with continuous batching.  Clients submit
// requests (mesh, parameters, initial state, step count); a worker thread admits them in
// arrival order as slots and device memory (a byte budget) free up, keeps every admitted
// interface's state resident, advances all resident interfaces together by one RK3 step per
// iteration (the batched FP32C path of zm_batch.cu), and retires finished ones (result copied
// to the host, memory returned) between iterations, so requests that arrive while others run
// join the next iteration.  Per-interface results do not depend on the mix (exact fixed-point
// accumulation).  The paper has no serving form: it runs one interface per job (Sec. 4-5).
//
// Scheduling policies (zm_server_set_policy):
//   ZM_SERVE_ALL   admission first come, first served; every resident interface advances one
//                  step per iteration.  Under overload every request then finishes near the
//                  makespan: each iteration costs as much as stepping the whole resident set.
//   ZM_SERVE_SRPT  shortest remaining work first: queued requests are admitted least total
//                  work first wherever they fit, and each iteration advances the resident
//                  interfaces with the least remaining work (pairs left) first, as many as fit
//                  a cap of pair interactions per iteration (always at least one).  Small
//                  requests overtake large ones at iteration granularity; with a finite trace
//                  every request finishes, but under endless overload the largest can starve.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "zm_batch.cuh"

namespace zm {
namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t id = 0;
    zm_mesh mesh{};
    double atwood = 0, delta = 0, dt = 0;
    int nsteps = 0, remaining = 0;
    std::vector<double> z, w;  // initial state in, final state out (host)
    size_t bytes = 0;
    void *slab = nullptr;
    Inst inst{};
    int state = ZM_REQ_QUEUED;
    int status = ZM_OK;
    bool cancel = false;
    double t_submit = 0, t_admit = 0, t_done = 0;
    // Birkhoff-Rott pair interactions still to evaluate (three evaluations per step)
    int64_t work() const { return 3LL * remaining * ((int64_t)mesh.n1 * mesh.n2) * ((int64_t)mesh.n1 * mesh.n2); }
};

}  // namespace

class Server {
public:
    size_t budget = 0, used = 0, peak_used = 0;
    int max_slots = 0, peak_slots = 0;
    int policy = ZM_SERVE_ALL;
    int64_t pairs_cap = 0;  // SRPT: pair interactions per iteration (<= 0: no cap)
    double g = 1.0, mu = 0.0;
    int device = 0;
    cudaStream_t stream = nullptr;
    Batch batch;
    std::mutex m;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::vector<Request *> running;
    std::unordered_map<int64_t, Request *> all;
    std::thread worker;
    bool stop = false;
    int64_t next_id = 1;
    int fatal = ZM_OK;
    // statistics
    int64_t iterations = 0, steps = 0, pairs = 0, completed = 0, failed = 0;
    double busy_s = 0;

    int start()
    {
        cudaGetDevice(&device);
        if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess)
            return set_error(ZM_ERR_CUDA, "server: stream creation failed");
        int rc = batch.setup();
        if (rc) return rc;
        batch.stream = stream;
        try {
            worker = std::thread([this] { loop(); });
        } catch (...) {
            return set_error(ZM_ERR_NOMEM, "server: worker thread creation failed");
        }
        return ZM_OK;
    }

    void shutdown()
    {
        {
            std::lock_guard<std::mutex> lk(m);
            stop = true;
        }
        cv_work.notify_all();
        if (worker.joinable()) worker.join();
        cudaSetDevice(device);
        if (stream) cudaStreamSynchronize(stream);
        for (auto &kv : all) {
            if (kv.second->slab) cudaFree(kv.second->slab);
            delete kv.second;
        }
        all.clear();
        batch.h.clear();
        batch.release();  // also forgets the stream before it is destroyed below
        if (stream) cudaStreamDestroy(stream);
        stream = nullptr;
    }

    // one iteration of the loop: admit, step every resident interface once, retire
    void loop()
    {
        cudaSetDevice(device);
        std::vector<Request *> admitted, finished, sel;
        std::vector<int64_t> sel_ids, prev_ids;  // the stepped set of this and the last iteration
        int stable = 0;  // iterations since the stepped set last changed
        while (true) {
            admitted.clear();
            {
                std::unique_lock<std::mutex> lk(m);
                cv_work.wait(lk, [&] { return stop || !queue.empty() || !running.empty(); });
                if (stop) break;
                // cancellations of queued requests
                for (auto it = queue.begin(); it != queue.end();) {
                    if ((*it)->cancel) {
                        (*it)->state = ZM_REQ_FAILED;
                        (*it)->status = ZM_ERR_INVALID;
                        (*it)->t_done = now_s();
                        ++failed;
                        it = queue.erase(it);
                        cv_done.notify_all();
                    } else {
                        ++it;
                    }
                }
                if (policy == ZM_SERVE_SRPT) {
                    // least total work first (arrival order among equals), wherever it fits
                    std::stable_sort(queue.begin(), queue.end(),
                                     [](const Request *a, const Request *b) { return a->work() < b->work(); });
                    for (auto it = queue.begin();
                         it != queue.end() && (int)(running.size() + admitted.size()) < max_slots;) {
                        if (used + (*it)->bytes <= budget) {
                            used += (*it)->bytes;
                            admitted.push_back(*it);
                            it = queue.erase(it);
                        } else {
                            ++it;
                        }
                    }
                } else {
                    // first come, first served: the head waits until it fits
                    while (!queue.empty() && (int)(running.size() + admitted.size()) < max_slots &&
                           used + queue.front()->bytes <= budget) {
                        Request *r = queue.front();
                        queue.pop_front();
                        used += r->bytes;
                        admitted.push_back(r);
                    }
                }
                peak_used = std::max(peak_used, used);
            }
            const double t0 = now_s();
            for (Request *r : admitted) {
                int rc = Batch::alloc_inst(r->inst, r->mesh, r->atwood, g, mu, r->delta, r->dt, stream,
                                           true, &r->slab);
                const size_t N = (size_t)r->mesh.n1 * r->mesh.n2;
                if (!rc) rc = cuda_check(cudaMemcpyAsync(r->inst.y[0], r->z.data(), 3 * N * sizeof(double),
                                                         cudaMemcpyHostToDevice, stream), "server upload");
                if (!rc) rc = cuda_check(cudaMemcpyAsync(r->inst.y[0] + 3 * N, r->w.data(), 2 * N * sizeof(double),
                                                         cudaMemcpyHostToDevice, stream), "server upload");
                std::lock_guard<std::mutex> lk(m);
                r->t_admit = now_s();
                if (rc) {
                    r->status = rc;
                    r->state = ZM_REQ_FAILED;
                    r->t_done = r->t_admit;
                    used -= r->bytes;
                    ++failed;
                    cv_done.notify_all();
                    continue;
                }
                r->state = ZM_REQ_RUNNING;
                running.push_back(r);
            }
            // running cancellations leave between iterations
            for (Request *r : running)
                if (r->cancel && r->remaining > 0) {
                    r->remaining = 0;
                    r->status = ZM_ERR_INVALID;
                }
            // the interfaces this iteration advances
            sel.clear();
            for (Request *r : running)
                if (r->remaining > 0) sel.push_back(r);
            if (policy == ZM_SERVE_SRPT) {
                std::stable_sort(sel.begin(), sel.end(),
                                 [](const Request *a, const Request *b) { return a->work() < b->work(); });
                if (pairs_cap > 0) {
                    int64_t acc = 0;
                    size_t k = 0;
                    for (; k < sel.size(); ++k) {
                        const int64_t nn = (int64_t)sel[k]->mesh.n1 * sel[k]->mesh.n2;
                        const int64_t step_pairs = 3 * nn * nn;
                        if (k > 0 && acc + step_pairs > pairs_cap) break;
                        acc += step_pairs;
                    }
                    sel.resize(k);
                }
            }
            sel_ids.clear();
            for (Request *r : sel) sel_ids.push_back(r->id);
            if (sel_ids != prev_ids) {
                batch.h.clear();
                for (Request *r : sel) batch.h.push_back(r->inst);
                int rc = batch.plan();  // drops the captured step graph
                if (rc) {
                    fail_all(rc);
                    continue;
                }
                prev_ids.swap(sel_ids);
                stable = 0;
            } else {
                ++stable;
            }
            peak_slots = std::max(peak_slots, (int)running.size());
            if (!sel.empty()) {
                // plain launches right after a membership change; once the same set has run an
                // iteration, the step is captured as a graph and replayed until the set changes
                int rc;
                {
                    const NvtxRange range("zm_server_iteration");
                    rc = batch.step(1, stable >= 1);
                }
                if (rc) {
                    fail_all(rc);
                    continue;
                }
                ++steps;
                for (Request *r : sel) {
                    r->remaining -= 1;
                    pairs += 3LL * r->inst.geom.N * r->inst.geom.N;
                }
            }
            finished.clear();
            for (Request *r : running)
                if (r->remaining == 0) {
                    const size_t N = (size_t)r->mesh.n1 * r->mesh.n2;
                    cudaMemcpyAsync(r->z.data(), r->inst.y[0], 3 * N * sizeof(double), cudaMemcpyDeviceToHost, stream);
                    cudaMemcpyAsync(r->w.data(), r->inst.y[0] + 3 * N, 2 * N * sizeof(double),
                                    cudaMemcpyDeviceToHost, stream);
                    finished.push_back(r);
                }
            int rc = batch.status();  // synchronises the stream; bounded device waits report here
            const double t1 = now_s();
            busy_s += t1 - t0;
            ++iterations;
            if (rc) {
                fail_all(rc);
                continue;
            }
            std::lock_guard<std::mutex> lk(m);
            for (Request *r : finished) {
                bool finite = true;
                for (double v : r->z) finite &= std::isfinite(v);
                for (double v : r->w) finite &= std::isfinite(v);
                if (r->status == ZM_OK && !finite) r->status = ZM_ERR_NONFINITE;
                r->state = (r->status == ZM_OK) ? ZM_REQ_DONE : ZM_REQ_FAILED;
                r->t_done = t1;
                cudaFreeAsync(r->slab, stream);
                r->slab = nullptr;
                used -= r->bytes;
                if (r->status == ZM_OK) ++completed;
                else ++failed;
            }
            if (!finished.empty()) {
                std::vector<Request *> keep;
                for (Request *r : running)
                    if (r->remaining > 0) keep.push_back(r);
                running.swap(keep);
                cv_done.notify_all();
            }
        }
    }

    void fail_all(int rc)
    {
        std::lock_guard<std::mutex> lk(m);
        fatal = rc;
        for (Request *r : running) {
            r->state = ZM_REQ_FAILED;
            r->status = rc;
            r->t_done = now_s();
            if (r->slab) cudaFreeAsync(r->slab, stream);
            r->slab = nullptr;
            used -= r->bytes;
            ++failed;
        }
        running.clear();
        batch.h.clear();
        cv_done.notify_all();
    }

    int set_policy(int p, int64_t cap)
    {
        std::lock_guard<std::mutex> lk(m);
        policy = p;
        pairs_cap = cap;
        return ZM_OK;
    }
};

}  // namespace zm

using namespace zm;

struct zm_server {
    Server s;
};

extern "C" {

int zm_server_create(size_t mem_budget_bytes, int32_t max_slots, double g, double mu, zm_server **out)
{
    if (!out || max_slots < 1 || mem_budget_bytes == 0 || !std::isfinite(g) || !(mu >= 0))
        return set_error(ZM_ERR_INVALID, "zm_server_create: bad arguments");
    *out = nullptr;
    zm_server *sv = new (std::nothrow) zm_server();
    if (!sv) return set_error(ZM_ERR_NOMEM, "zm_server_create: host allocation failed");
    sv->s.budget = mem_budget_bytes;
    sv->s.max_slots = max_slots;
    sv->s.g = g;
    sv->s.mu = mu;
    int rc = sv->s.start();
    if (rc) {
        sv->s.shutdown();
        delete sv;
        return rc;
    }
    *out = sv;
    return ZM_OK;
}

int zm_server_submit(zm_server *sv, const zm_mesh *mesh, double atwood, double delta, double dt,
                     int32_t nsteps, const double *z, const double *w, int64_t *id)
{
    if (!sv || !mesh || !z || !w || !id || nsteps < 0 || !std::isfinite(dt) || !(delta > 0) ||
        mesh->n1 < 5 || mesh->n2 < 5 || (int64_t)mesh->n1 * mesh->n2 > (1 << 24) || !(mesh->L1 > 0) ||
        !(mesh->L2 > 0) || !std::isfinite(atwood))
        return set_error(ZM_ERR_INVALID, "zm_server_submit: bad arguments");
    Request *r = new (std::nothrow) Request();
    if (!r) return set_error(ZM_ERR_NOMEM, "zm_server_submit: host allocation failed");
    const size_t N = (size_t)mesh->n1 * mesh->n2;
    r->mesh = *mesh;
    r->atwood = atwood;
    r->delta = delta;
    r->dt = dt;
    r->nsteps = r->remaining = nsteps;
    r->bytes = Batch::inst_bytes(*mesh);
    if (r->bytes > sv->s.budget) {
        delete r;
        return set_error(ZM_ERR_BUSY, "zm_server_submit: request larger than the memory budget");
    }
    try {
        r->z.assign(z, z + 3 * N);
        r->w.assign(w, w + 2 * N);
    } catch (...) {
        delete r;
        return set_error(ZM_ERR_NOMEM, "zm_server_submit: host allocation failed");
    }
    {
        std::lock_guard<std::mutex> lk(sv->s.m);
        if (sv->s.fatal) {
            delete r;
            return set_error(sv->s.fatal, "zm_server_submit: the server stopped after an error");
        }
        r->id = sv->s.next_id++;
        r->t_submit = now_s();
        sv->s.all[r->id] = r;
        sv->s.queue.push_back(r);
        *id = r->id;
    }
    sv->s.cv_work.notify_all();
    return ZM_OK;
}

int zm_server_request_bytes(const zm_mesh *mesh, size_t *bytes)
{
    if (!mesh || !bytes || mesh->n1 < 5 || mesh->n2 < 5)
        return set_error(ZM_ERR_INVALID, "zm_server_request_bytes: bad arguments");
    *bytes = Batch::inst_bytes(*mesh);
    return ZM_OK;
}

int zm_server_poll(zm_server *sv, int64_t id, int32_t *state)
{
    if (!sv || !state) return set_error(ZM_ERR_INVALID, "zm_server_poll: bad arguments");
    std::lock_guard<std::mutex> lk(sv->s.m);
    auto it = sv->s.all.find(id);
    if (it == sv->s.all.end()) return set_error(ZM_ERR_INVALID, "zm_server_poll: unknown request");
    *state = it->second->state;
    return ZM_OK;
}

int zm_server_wait(zm_server *sv, int64_t id, double timeout_s)
{
    if (!sv) return set_error(ZM_ERR_INVALID, "zm_server_wait: null server");
    std::unique_lock<std::mutex> lk(sv->s.m);
    auto it = sv->s.all.find(id);
    if (it == sv->s.all.end()) return set_error(ZM_ERR_INVALID, "zm_server_wait: unknown request");
    Request *r = it->second;
    const auto pred = [&] { return r->state == ZM_REQ_DONE || r->state == ZM_REQ_FAILED; };
    if (timeout_s < 0) sv->s.cv_done.wait(lk, pred);
    else if (!sv->s.cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
        return set_error(ZM_ERR_TIMEOUT, "zm_server_wait: not finished within the timeout");
    return r->status;
}

int zm_server_result(zm_server *sv, int64_t id, double *z, double *w, double *latency_s, double *queue_s)
{
    if (!sv) return set_error(ZM_ERR_INVALID, "zm_server_result: null server");
    std::lock_guard<std::mutex> lk(sv->s.m);
    auto it = sv->s.all.find(id);
    if (it == sv->s.all.end()) return set_error(ZM_ERR_INVALID, "zm_server_result: unknown request");
    Request *r = it->second;
    if (r->state != ZM_REQ_DONE && r->state != ZM_REQ_FAILED)
        return set_error(ZM_ERR_BUSY, "zm_server_result: request not finished");
    if (z && r->state == ZM_REQ_DONE) std::memcpy(z, r->z.data(), r->z.size() * sizeof(double));
    if (w && r->state == ZM_REQ_DONE) std::memcpy(w, r->w.data(), r->w.size() * sizeof(double));
    if (latency_s) *latency_s = r->t_done - r->t_submit;
    if (queue_s) *queue_s = r->t_admit - r->t_submit;
    const int status = r->status;
    sv->s.all.erase(it);
    delete r;
    return status;
}

int zm_server_cancel(zm_server *sv, int64_t id)
{
    if (!sv) return set_error(ZM_ERR_INVALID, "zm_server_cancel: null server");
    {
        std::lock_guard<std::mutex> lk(sv->s.m);
        auto it = sv->s.all.find(id);
        if (it == sv->s.all.end()) return set_error(ZM_ERR_INVALID, "zm_server_cancel: unknown request");
        it->second->cancel = true;
    }
    sv->s.cv_work.notify_all();
    return ZM_OK;
}

int zm_server_set_policy(zm_server *sv, int32_t policy, int64_t pairs_per_iteration)
{
    if (!sv || (policy != ZM_SERVE_ALL && policy != ZM_SERVE_SRPT))
        return set_error(ZM_ERR_INVALID, "zm_server_set_policy: bad arguments");
    return sv->s.set_policy(policy, policy == ZM_SERVE_SRPT ? pairs_per_iteration : 0);
}

int zm_server_get_stats(zm_server *sv, zm_server_stats *out)
{
    if (!sv || !out) return set_error(ZM_ERR_INVALID, "zm_server_get_stats: bad arguments");
    std::lock_guard<std::mutex> lk(sv->s.m);
    out->iterations = sv->s.iterations;
    out->steps = sv->s.steps;
    out->pairs = sv->s.pairs;
    out->completed = sv->s.completed;
    out->failed = sv->s.failed;
    out->queued = (int64_t)sv->s.queue.size();
    out->running = (int64_t)sv->s.running.size();
    out->peak_running = sv->s.peak_slots;
    out->bytes_in_use = (int64_t)sv->s.used;
    out->peak_bytes = (int64_t)sv->s.peak_used;
    out->busy_s = sv->s.busy_s;
    return ZM_OK;
}

void zm_server_destroy(zm_server *sv)
{
    if (!sv) return;
    sv->s.shutdown();
    delete sv;
}

}  // extern "C"
