// Serving runtime (C ABI in include/mpdata.h: mpdata_server_*, mpdata_submit,
// mpdata_poll, mpdata_wait, mpdata_cancel, mpdata_request_times).
//
// A scheduler thread owns one CUDA stream and runs continuous batching:
//   * admission: queued requests (FIFO) are admitted while their device
//     footprint (h, psi, scratch, u1, u2, u3) fits the HBM budget and a slot is
//     free; their fields are copied in on the stream;
//   * tick: every resident request is advanced by the same chunk of steps
//     (chunk = min(chunk_steps, fewest remaining)); each step is one batched
//     launch per kernel variant over the tiles of all resident requests, one
//     CTA per tile, largest tiles first (the same kernels and tiles as a
//     single-grid step, so each result is bit-identical to running that
//     request alone);
//   * completion: a finished request's psi is copied back to its host buffer,
//     its device memory is freed and its budget released once the copy is
//     done; requests that arrive meanwhile join at the next tick.
// Host-side waits are bounded (mpdata_wait takes a timeout); nothing on the
// device waits on anything.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mpdata_internal.cuh"

using mpdata::BatchGrid;

namespace {

using Clock = std::chrono::steady_clock;

int sfail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return mpdata::set_error(code, buf);
}

// Kernel variants of a tick: the two-column kernel with x and y periodic, or
// with a lid on x or y (every FP32 grid runs the two-column kernel).
enum Variant { kPairsPeriodic = 0, kPairsLid = 1, kNumVariants = 2 };

struct Request {
    uint64_t ticket = 0;
    mpdata_request req;
    int state = MPDATA_REQ_QUEUED;
    int error = MPDATA_OK;
    std::atomic<bool> cancel{false};
    size_t field_bytes = 0, bytes = 0;
    int remaining = 0;
    int variant = kPairsPeriodic, ntiles = 0;
    BatchGrid bg;  // buf[0] holds the current state, buf[1] its partner
    float *dev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t done_ev = nullptr;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

struct TickBuffers {
    BatchGrid *d_grids = nullptr;
    int2 *d_items = nullptr;
    int *d_begin = nullptr;
    size_t cap_grids = 0, cap_items = 0, cap_begin = 0;
    std::vector<BatchGrid> h_grids;
    std::vector<int2> h_items;
    std::vector<int> h_begin;
    cudaEvent_t ev = nullptr;
    bool in_flight = false;
};

double now_s(Clock::time_point t0) {
    return std::chrono::duration<double>(Clock::now() - t0).count();
}

}  // namespace

struct mpdata_server {
    mpdata_server_opts o;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::vector<Request *> active, copying;
    std::unordered_map<uint64_t, Request *> all;
    size_t admitted_bytes = 0, reserved_bytes = 0;
    uint64_t next_ticket = 1;
    unsigned admissions = 0;
    bool stop = false;
    std::thread thr;
    Clock::time_point t0 = Clock::now();
    TickBuffers tick[2];
    int tick_index = 0;
    double cell_steps = 0.0;
    uint64_t completed = 0;
};

namespace {

void free_request_device(mpdata_server *s, Request *r) {
    for (auto &p : r->dev) {
        if (p) cudaFreeAsync(p, s->stream);
        p = nullptr;
    }
}

// Make room for n elements of a device array (synchronises first: the old
// array may still be read by an earlier tick).
template <typename T>
cudaError_t ensure(T **ptr, size_t *cap, size_t n, cudaStream_t st) {
    if (n <= *cap) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    cudaFree(*ptr);
    *ptr = nullptr;
    size_t c = std::max<size_t>(n, 2 * *cap);
    e = cudaMalloc((void **)ptr, sizeof(T) * c);
    *cap = e == cudaSuccess ? c : 0;
    return e;
}

void fail_request(mpdata_server *s, Request *r, int code) {
    r->state = MPDATA_REQ_FAILED;
    r->error = code;
    r->t_done = now_s(s->t0);
    free_request_device(s, r);
}

// Allocate and copy in an admitted request (no lock held: only the
// scheduler thread touches a request between admission and completion).
int load_request(mpdata_server *s, Request *r, bool injected) {
    cudaError_t e = injected ? cudaErrorMemoryAllocation : cudaSuccess;
    for (int f = 0; f < 6 && e == cudaSuccess; ++f)
        e = cudaMallocAsync((void **)&r->dev[f], r->field_bytes, s->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MPDATA_ENOMEM;
    }
    const void *src[5] = {r->req.h, r->req.psi, r->req.u1, r->req.u2, r->req.u3};
    float *dst[5] = {r->dev[0], r->dev[1], r->dev[3], r->dev[4], r->dev[5]};
    for (int f = 0; f < 5 && e == cudaSuccess; ++f)
        e = cudaMemcpyAsync(dst[f], src[f], r->field_bytes, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return MPDATA_ECUDA;
    BatchGrid &g = r->bg;
    g.h = r->dev[0];
    g.buf[0] = r->dev[1];
    g.buf[1] = r->dev[2];
    g.u1 = r->dev[3];
    g.u2 = r->dev[4];
    g.u3 = r->dev[5];
    return MPDATA_OK;
}

// One tick over `act` (no lock held): upload the work list, launch `chunk`
// steps, and for requests that finish (or are cancelled) queue the copy-out,
// the frees and the completion event.  Returns a CUDA error or success.
cudaError_t run_tick(mpdata_server *s, const std::vector<Request *> &act, int chunk,
                     std::vector<char> &finished) {
    TickBuffers &T = s->tick[s->tick_index & 1];
    cudaError_t e = cudaSuccess;
    if (T.in_flight) {
        e = cudaEventSynchronize(T.ev);  // keep at most two ticks in flight
        if (e != cudaSuccess) return e;
        T.in_flight = false;
    }
    const int na = (int)act.size();
    T.h_grids.resize(na);
    T.h_items.clear();
    int voff[kNumVariants] = {0, 0};
    std::vector<double> cost[kNumVariants];
    std::vector<int2> items[kNumVariants];
    for (int a = 0; a < na; ++a) {
        Request *r = act[a];
        T.h_grids[a] = r->bg;
        const int ty = s->o.tile_y;
        for (int t = 0; t < r->ntiles; ++t) {
            items[r->variant].push_back(make_int2(a, t));
            cost[r->variant].push_back(32.0 * ty * (r->bg.g.nz + 3));
        }
    }
    int ncta[kNumVariants];
    std::vector<int> begin_all;
    int item_base = 0;
    for (int v = 0; v < kNumVariants; ++v) {
        voff[v] = (int)begin_all.size();
        const int n = (int)items[v].size();
        ncta[v] = n;  // one CTA per tile
        if (n) {
            std::vector<int> order(n);
            for (int k = 0; k < n; ++k) order[k] = k;
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[v][x] > cost[v][y]; });
            for (int k = 0; k < n; ++k) T.h_items.push_back(items[v][order[k]]);
            for (int k = 0; k <= n; ++k) begin_all.push_back(item_base + k);
        }
        item_base += n;
    }
    T.h_begin = begin_all;
    e = ensure(&T.d_grids, &T.cap_grids, (size_t)na, s->stream);
    if (e == cudaSuccess) e = ensure(&T.d_items, &T.cap_items, T.h_items.size(), s->stream);
    if (e == cudaSuccess) e = ensure(&T.d_begin, &T.cap_begin, T.h_begin.size(), s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(T.d_grids, T.h_grids.data(), sizeof(BatchGrid) * na, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess && !T.h_items.empty())
        e = cudaMemcpyAsync(T.d_items, T.h_items.data(), sizeof(int2) * T.h_items.size(), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess && !T.h_begin.empty())
        e = cudaMemcpyAsync(T.d_begin, T.h_begin.data(), sizeof(int) * T.h_begin.size(), cudaMemcpyHostToDevice, s->stream);
    for (int st = 0; st < chunk && e == cudaSuccess; ++st) {
        const int parity = st & 1;
        for (int v = 0; v < kNumVariants && e == cudaSuccess; ++v) {
            if (!ncta[v]) continue;
            const int *begin = T.d_begin + voff[v];
            e = mpdata::launch_fused_pairs_batch(32, s->o.tile_y, s->o.nonoscillatory, v == kPairsLid,
                                                     T.d_grids, T.d_items, begin, ncta[v], parity, s->stream);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(T.ev, s->stream);
    if (e != cudaSuccess) return e;
    T.in_flight = true;
    s->tick_index++;
    finished.assign(na, 0);
    for (int a = 0; a < na && e == cudaSuccess; ++a) {
        Request *r = act[a];
        r->remaining -= chunk;
        if (chunk & 1) std::swap(r->bg.buf[0], r->bg.buf[1]);
        const bool cancel = r->cancel.load();
        if (r->remaining > 0 && !cancel) continue;
        finished[a] = cancel ? 2 : 1;
        if (!cancel)
            e = cudaMemcpyAsync(r->req.psi, r->bg.buf[0], r->field_bytes, cudaMemcpyDeviceToHost, s->stream);
        free_request_device(s, r);
        if (e == cudaSuccess) e = cudaEventRecord(r->done_ev, s->stream);
    }
    return e;
}

void finish_copies(mpdata_server *s) {  // lock held
    std::vector<Request *> still;
    bool any = false;
    for (Request *r : s->copying) {
        cudaError_t q = cudaEventQuery(r->done_ev);
        if (q == cudaErrorNotReady) { still.push_back(r); continue; }
        s->admitted_bytes -= r->bytes;
        if (r->state != MPDATA_REQ_CANCELLED) {
            if (q == cudaSuccess) {
                r->state = MPDATA_REQ_DONE;
                ++s->completed;
            } else {
                r->state = MPDATA_REQ_FAILED;
                r->error = MPDATA_ECUDA;
            }
        }
        r->t_done = now_s(s->t0);
        any = true;
    }
    s->copying.swap(still);
    if (any) s->cv_done.notify_all();
}

void scheduler(mpdata_server *s) {
    cudaSetDevice(s->device);
    std::vector<Request *> act, admit;
    std::vector<char> admit_injected, finished;
    for (;;) {
        admit.clear();
        admit_injected.clear();
        {
            std::unique_lock<std::mutex> lk(s->mu);
            finish_copies(s);
            for (auto it = s->queue.begin(); it != s->queue.end();) {  // cancelled while queued
                Request *r = *it;
                if (r->cancel.load()) {
                    r->state = MPDATA_REQ_CANCELLED;
                    r->t_done = now_s(s->t0);
                    if (r->bytes <= s->reserved_bytes) s->reserved_bytes -= r->bytes;
                    it = s->queue.erase(it);
                    s->cv_done.notify_all();
                } else {
                    ++it;
                }
            }
            // admission: FIFO while the budget and the slots allow
            while (!s->stop && !s->queue.empty()) {
                Request *r = s->queue.front();
                if (s->active.size() + admit.size() >= (size_t)s->o.max_active) break;
                if (s->admitted_bytes + r->bytes > s->o.hbm_budget_bytes) break;
                s->queue.pop_front();
                s->admitted_bytes += r->bytes;
                if (r->bytes <= s->reserved_bytes) s->reserved_bytes -= r->bytes;
                ++s->admissions;
                admit.push_back(r);
                admit_injected.push_back(s->o.inject_alloc_failure > 0 &&
                                         s->admissions % (unsigned)s->o.inject_alloc_failure == 0);
            }
            if (s->active.empty() && admit.empty()) {
                if (s->stop && s->copying.empty()) break;
                if (!s->copying.empty()) {
                    lk.unlock();
                    std::this_thread::sleep_for(std::chrono::microseconds(50));
                } else {
                    s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
                }
                continue;
            }
            if (s->stop)
                for (Request *r : s->active) r->cancel.store(true);
        }
        // copy-in of the admitted requests (no lock)
        std::vector<int> load_rc(admit.size());
        for (size_t i = 0; i < admit.size(); ++i) load_rc[i] = load_request(s, admit[i], admit_injected[i]);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (size_t i = 0; i < admit.size(); ++i) {
                Request *r = admit[i];
                if (load_rc[i] != MPDATA_OK) {
                    fail_request(s, r, load_rc[i]);
                    s->admitted_bytes -= r->bytes;
                    s->cv_done.notify_all();
                    continue;
                }
                r->state = MPDATA_REQ_RUNNING;
                r->t_admit = now_s(s->t0);
                s->active.push_back(r);
            }
            act = s->active;
        }
        if (act.empty()) continue;
        int chunk = s->o.chunk_steps;
        for (Request *r : act) chunk = std::min(chunk, std::max(r->remaining, 1));
        cudaError_t e = run_tick(s, act, chunk, finished);  // no lock
        {
            std::lock_guard<std::mutex> lk(s->mu);
            std::vector<Request *> still;
            for (size_t a = 0; a < act.size(); ++a) {
                Request *r = act[a];
                if (e != cudaSuccess) {
                    fail_request(s, r, MPDATA_ECUDA);
                    s->admitted_bytes -= r->bytes;
                    continue;
                }
                s->cell_steps += (double)r->req.nx * r->req.ny * r->req.nz * chunk;
                if (finished[a]) {
                    if (finished[a] == 2) r->state = MPDATA_REQ_CANCELLED;
                    s->copying.push_back(r);
                } else {
                    still.push_back(r);
                }
            }
            s->active.swap(still);
            if (e != cudaSuccess) {
                cudaGetLastError();
                s->cv_done.notify_all();
            }
        }
    }
    cudaStreamSynchronize(s->stream);
}

}  // namespace

extern "C" {

void mpdata_server_opts_default(mpdata_server_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->size = sizeof *o;
    o->hbm_budget_bytes = (size_t)8 << 30;
    o->max_active = 256;
    o->max_queued = 1 << 20;
    o->chunk_steps = 8;
    o->tile_y = 24;
    o->nonoscillatory = 1;
    o->inject_alloc_failure = 0;
    o->eps = 1e-15;
}

int mpdata_server_create(const mpdata_server_opts *opts, mpdata_server_t **out) {
    if (!out) return sfail(MPDATA_EINVAL, "out is NULL");
    *out = nullptr;
    mpdata_server_opts o;
    if (opts) o = *opts; else mpdata_server_opts_default(&o);
    if (o.size < sizeof(mpdata_server_opts)) return sfail(MPDATA_EINVAL, "opts.size too small");
    if (o.hbm_budget_bytes == 0) return sfail(MPDATA_EINVAL, "hbm_budget_bytes must be > 0");
    if (o.max_active < 1 || o.max_queued < 0 || o.chunk_steps < 1) return sfail(MPDATA_EINVAL, "max_active >= 1, max_queued >= 0, chunk_steps >= 1");
    if (o.tile_y != 16 && o.tile_y != 24) return sfail(MPDATA_EINVAL, "tile_y must be 16 or 24");
    if (!(o.eps > 0.0)) return sfail(MPDATA_EINVAL, "eps must be > 0");
    mpdata_server *s = new (std::nothrow) mpdata_server();
    if (!s) return sfail(MPDATA_ENOMEM, "host allocation failed");
    s->o = o;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&s->tick[i].ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (s->stream) cudaStreamDestroy(s->stream);
        delete s;
        return sfail(MPDATA_ECUDA, "server setup: %s", cudaGetErrorString(e));
    }
    s->thr = std::thread(scheduler, s);
    *out = s;
    return MPDATA_OK;
}

int mpdata_submit(mpdata_server_t *s, const mpdata_request *req, uint64_t *ticket) {
    if (!s || !req || !ticket) return sfail(MPDATA_EINVAL, "NULL argument");
    if (req->size < sizeof(mpdata_request)) return sfail(MPDATA_EINVAL, "request.size too small");
    const int nx = req->nx, ny = req->ny, nz = req->nz;
    if (nx < 1 || ny < 1 || nz < 1 || ny > 65535 || nz > 65535 || (long long)nx * ny * nz >= (1LL << 31))
        return sfail(MPDATA_EINVAL, "bad dims %d x %d x %d", nx, ny, nz);
    if (req->nsteps < 0) return sfail(MPDATA_EINVAL, "nsteps must be >= 0");
    if (!req->h || !req->psi || !req->u1 || !req->u2 || !req->u3) return sfail(MPDATA_EINVAL, "NULL field pointer");
    for (int d = 0; d < 3; ++d)
        if (req->periodic[d] != 0 && req->periodic[d] != 1) return sfail(MPDATA_EINVAL, "periodic flags must be 0 or 1");
    Request *r = new (std::nothrow) Request();
    if (!r) return sfail(MPDATA_ENOMEM, "host allocation failed");
    r->req = *req;
    r->field_bytes = (size_t)nx * ny * nz * sizeof(float);
    r->bytes = 6 * r->field_bytes;
    r->remaining = req->nsteps;
    BatchGrid &g = r->bg;
    memset(&g, 0, sizeof g);
    g.g.nx = nx; g.g.ny = ny; g.g.nz = nz;
    for (int d = 0; d < 3; ++d) g.g.per[d] = req->periodic[d];
    g.eps = (float)s->o.eps;
    r->variant = (!g.g.per[0] || !g.g.per[1]) ? kPairsLid : kPairsPeriodic;
    const int tx = 32, ty = s->o.tile_y;
    g.ntx = (nx + tx - 1) / tx;
    r->ntiles = g.ntx * ((ny + ty - 1) / ty);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) { delete r; return sfail(MPDATA_EINVAL, "server is shutting down"); }
    if (r->bytes > s->o.hbm_budget_bytes) {
        delete r;
        return sfail(MPDATA_EINVAL, "request needs %zu bytes, more than the whole budget", (size_t)6 * (size_t)nx * ny * nz * 4);
    }
    const size_t committed = s->admitted_bytes + s->reserved_bytes;
    if ((int)s->queue.size() >= s->o.max_queued && committed + r->bytes > s->o.hbm_budget_bytes) {
        delete r;
        return sfail(MPDATA_EBUSY, "over the HBM budget and the admission queue is full");
    }
    if (cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete r;
        return sfail(MPDATA_ECUDA, "cudaEventCreate failed");
    }
    r->ticket = s->next_ticket++;
    r->t_submit = now_s(s->t0);
    s->reserved_bytes += r->bytes;
    if (req->nsteps == 0) {  // nothing to do: psi already holds the answer
        r->state = MPDATA_REQ_DONE;
        r->t_admit = r->t_done = r->t_submit;
        s->reserved_bytes -= r->bytes;
    } else {
        s->queue.push_back(r);
    }
    s->all[r->ticket] = r;
    *ticket = r->ticket;
    s->cv_work.notify_one();
    return MPDATA_OK;
}

int mpdata_poll(mpdata_server_t *s, uint64_t ticket, int *state) {
    if (!s || !state) return sfail(MPDATA_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return sfail(MPDATA_ENOENT, "unknown ticket %llu", (unsigned long long)ticket);
    *state = it->second->state;
    return MPDATA_OK;
}

int mpdata_wait(mpdata_server_t *s, uint64_t ticket, int timeout_ms) {
    if (!s) return sfail(MPDATA_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return sfail(MPDATA_ENOENT, "unknown ticket %llu", (unsigned long long)ticket);
    Request *r = it->second;
    auto finished = [r] { return r->state == MPDATA_REQ_DONE || r->state == MPDATA_REQ_FAILED || r->state == MPDATA_REQ_CANCELLED; };
    if (timeout_ms < 0) s->cv_done.wait(lk, finished);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished))
        return sfail(MPDATA_ETIMEDOUT, "ticket %llu not finished after %d ms", (unsigned long long)ticket, timeout_ms);
    if (r->state == MPDATA_REQ_DONE) return MPDATA_OK;
    if (r->state == MPDATA_REQ_CANCELLED) return sfail(MPDATA_ECANCELED, "ticket %llu was cancelled", (unsigned long long)ticket);
    return sfail(r->error ? r->error : MPDATA_ECUDA, "ticket %llu failed", (unsigned long long)ticket);
}

int mpdata_cancel(mpdata_server_t *s, uint64_t ticket) {
    if (!s) return sfail(MPDATA_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return sfail(MPDATA_ENOENT, "unknown ticket %llu", (unsigned long long)ticket);
    it->second->cancel.store(true);
    s->cv_work.notify_one();
    return MPDATA_OK;
}

int mpdata_request_times(mpdata_server_t *s, uint64_t ticket, double *t3) {
    if (!s || !t3) return sfail(MPDATA_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return sfail(MPDATA_ENOENT, "unknown ticket %llu", (unsigned long long)ticket);
    t3[0] = it->second->t_submit;
    t3[1] = it->second->t_admit;
    t3[2] = it->second->t_done;
    return MPDATA_OK;
}

int mpdata_server_stats(mpdata_server_t *s, double *stats) {
    if (!s || !stats) return sfail(MPDATA_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    stats[0] = (double)s->completed;
    stats[1] = s->cell_steps;
    stats[2] = (double)s->admitted_bytes;
    stats[3] = (double)s->queue.size();
    stats[4] = (double)s->active.size();
    stats[5] = now_s(s->t0);
    return MPDATA_OK;
}

int mpdata_server_destroy(mpdata_server_t *s) {
    if (!s) return MPDATA_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Request *r : s->queue) {
            r->state = MPDATA_REQ_CANCELLED;
        }
        s->queue.clear();
        s->cv_work.notify_all();
    }
    if (s->thr.joinable()) s->thr.join();
    s->cv_done.notify_all();
    for (auto &kv : s->all) {
        if (kv.second->done_ev) cudaEventDestroy(kv.second->done_ev);
        delete kv.second;
    }
    for (auto &T : s->tick) {
        cudaFree(T.d_grids);
        cudaFree(T.d_items);
        cudaFree(T.d_begin);
        if (T.ev) cudaEventDestroy(T.ev);
    }
    cudaStreamDestroy(s->stream);
    delete s;
    return MPDATA_OK;
}

}  // extern "C"
