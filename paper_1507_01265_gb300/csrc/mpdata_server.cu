// Serving runtime (C ABI in include/mpdata.h: mpdata_server_*, mpdata_submit,
// mpdata_poll, mpdata_wait, mpdata_cancel, mpdata_release,
// mpdata_request_times).
//
// A scheduler thread runs continuous batching on three CUDA streams:
//   * admission: queued requests (FIFO) are admitted while their device
//     footprint (h, psi, scratch, u1, u2, u3) fits the HBM budget and a slot is
//     free; their memory is allocated and their fields copied in on the
//     copy-in stream, and an event marks the end of the copy;
//   * a loading request joins the resident set once that event has
//     completed, so its copy runs on a copy engine under the ticks of the
//     requests already resident instead of in front of them;
//   * tick: every resident request is advanced by the same chunk of steps
//     (chunk = min(chunk_steps, fewest remaining)) on the tick stream; each
//     step is one batched launch per kernel variant over the tiles of all
//     resident requests, one CTA per tile, largest tiles first (the same
//     kernels and tiles as a single-grid step, so each result is
//     bit-identical to running that request alone);
//   * completion: the copy-out stream waits for the tick that finished a
//     request, copies its psi back to the host buffer and frees its device
//     memory; the budget is released once that copy is done.  Requests that
//     arrive meanwhile join at a later tick.
// Finished requests stay queryable until mpdata_release, or until more than
// retain_finished newer requests have finished (the oldest go first); a
// request that a thread is waiting on is never retired.  Host-side waits are
// bounded (mpdata_wait takes a timeout); nothing on the device waits on
// anything.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <memory>
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
    cudaEvent_t ready_ev = nullptr;  // copy-in done (copy-in stream)
    cudaEvent_t done_ev = nullptr;   // copy-out done (copy-out stream)
    int waiters = 0;                 // threads inside mpdata_wait on this request
    double t_submit = 0, t_admit = 0, t_done = 0;
};

bool terminal(const Request *r) {
    return r->state == MPDATA_REQ_DONE || r->state == MPDATA_REQ_FAILED ||
           r->state == MPDATA_REQ_CANCELLED;
}

void destroy_events(Request *r) {
    if (r->ready_ev) cudaEventDestroy(r->ready_ev);
    if (r->done_ev) cudaEventDestroy(r->done_ev);
    r->ready_ev = r->done_ev = nullptr;
}

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
    cudaStream_t stream = nullptr;                            // ticks
    cudaStream_t copy_in = nullptr, copy_out = nullptr;       // admissions, results
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::vector<Request *> loading, active, copying;
    std::unordered_map<uint64_t, Request *> all;
    std::deque<uint64_t> finished_order;  // tickets in the order they finished
    int waiters = 0;                      // threads inside mpdata_wait
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

void free_request_device(Request *r, cudaStream_t st) {
    for (auto &p : r->dev) {
        if (p) cudaFreeAsync(p, st);
        p = nullptr;
    }
}

// Retire finished requests beyond the retained count, oldest first, skipping
// any that a thread is waiting on (lock held).
void retire_excess(mpdata_server *s) {
    const size_t keep = (size_t)s->o.retain_finished;
    for (auto it = s->finished_order.begin(); s->finished_order.size() > keep && it != s->finished_order.end();) {
        auto f = s->all.find(*it);
        if (f == s->all.end()) {  // released already
            it = s->finished_order.erase(it);
            continue;
        }
        Request *r = f->second;
        if (r->waiters > 0) {
            ++it;
            continue;
        }
        destroy_events(r);
        delete r;
        s->all.erase(f);
        it = s->finished_order.erase(it);
    }
}

// A request reached DONE, FAILED or CANCELLED (lock held).
void mark_terminal(mpdata_server *s, Request *r) {
    s->finished_order.push_back(r->ticket);
    retire_excess(s);
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

// An admitted request failed: free its memory on stream st, release its
// budget, make it terminal (lock held; r may be retired on return).
void fail_request(mpdata_server *s, Request *r, int code, cudaStream_t st) {
    r->state = MPDATA_REQ_FAILED;
    r->error = code;
    r->t_done = now_s(s->t0);
    free_request_device(r, st);
    destroy_events(r);
    s->admitted_bytes -= r->bytes;
    mark_terminal(s, r);
}

// Allocate and start the copy-in of an admitted request on the copy-in
// stream; ready_ev marks its end (no lock held: only the scheduler thread
// touches a request between admission and completion).
int load_request(mpdata_server *s, Request *r, bool injected) {
    cudaError_t e = injected ? cudaErrorMemoryAllocation : cudaSuccess;
    for (int f = 0; f < 6 && e == cudaSuccess; ++f)
        e = cudaMallocAsync((void **)&r->dev[f], r->field_bytes, s->copy_in);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MPDATA_ENOMEM;
    }
    const void *src[5] = {r->req.h, r->req.psi, r->req.u1, r->req.u2, r->req.u3};
    float *dst[5] = {r->dev[0], r->dev[1], r->dev[3], r->dev[4], r->dev[5]};
    for (int f = 0; f < 5 && e == cudaSuccess; ++f)
        e = cudaMemcpyAsync(dst[f], src[f], r->field_bytes, cudaMemcpyHostToDevice, s->copy_in);
    if (e == cudaSuccess) e = cudaEventRecord(r->ready_ev, s->copy_in);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MPDATA_ECUDA;
    }
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
    int ncta[kNumVariants], ibase[kNumVariants];
    std::vector<int> begin_all;
    int item_base = 0;
    for (int v = 0; v < kNumVariants; ++v) {
        voff[v] = (int)begin_all.size();
        ibase[v] = item_base;
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
    // Direct launches: each variant's items are runs of consecutive tiles of
    // one request (all tiles of a request cost the same, so the stable sort
    // keeps them together); with at most kDirectMaxRuns runs per variant the
    // grid table travels in the kernel parameters and nothing is uploaded.
    std::unique_ptr<mpdata::DirectBatch> direct[kNumVariants];
    bool all_direct = true;
    for (int v = 0; v < kNumVariants && all_direct; ++v) {
        if (!ncta[v]) continue;
        direct[v].reset(new (std::nothrow) mpdata::DirectBatch);
        mpdata::DirectBatch *d = direct[v].get();
        if (!d) { all_direct = false; break; }
        d->nruns = 0;
        for (int k = 0; k < ncta[v]; ++k) {
            const int2 w = T.h_items[ibase[v] + k];
            if (k > 0) {
                const int2 prev = T.h_items[ibase[v] + k - 1];
                if (prev.x == w.x && prev.y + 1 == w.y) continue;
            }
            if (d->nruns == mpdata::kDirectMaxRuns) { all_direct = false; break; }
            d->start[d->nruns] = k;
            d->tile0[d->nruns] = w.y;
            d->g[d->nruns] = T.h_grids[w.x];
            ++d->nruns;
        }
        d->start[d->nruns] = ncta[v];
    }
    if (all_direct) {
        for (int st = 0; st < chunk && e == cudaSuccess; ++st)
            for (int v = 0; v < kNumVariants && e == cudaSuccess; ++v)
                if (ncta[v])
                    e = mpdata::launch_fused_pairs_direct(s->o.tile_y, 0, s->o.nonoscillatory, v == kPairsLid,
                                                          *direct[v], st & 1, s->stream);
    } else {
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
                e = mpdata::launch_fused_pairs_batch(32, s->o.tile_y, 0, s->o.nonoscillatory, v == kPairsLid,
                                                         T.d_grids, T.d_items, begin, ncta[v], parity, s->stream);
            }
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(T.ev, s->stream);
    if (e != cudaSuccess) return e;
    T.in_flight = true;
    s->tick_index++;
    finished.assign(na, 0);
    bool joined = false;  // copy-out stream ordered after this tick
    for (int a = 0; a < na && e == cudaSuccess; ++a) {
        Request *r = act[a];
        r->remaining -= chunk;
        if (chunk & 1) std::swap(r->bg.buf[0], r->bg.buf[1]);
        const bool cancel = r->cancel.load();
        if (r->remaining > 0 && !cancel) continue;
        finished[a] = cancel ? 2 : 1;
        if (!joined) {
            e = cudaStreamWaitEvent(s->copy_out, T.ev, 0);
            joined = true;
        }
        if (e == cudaSuccess && !cancel)
            e = cudaMemcpyAsync(r->req.psi, r->bg.buf[0], r->field_bytes, cudaMemcpyDeviceToHost, s->copy_out);
        free_request_device(r, s->copy_out);
        if (e == cudaSuccess) e = cudaEventRecord(r->done_ev, s->copy_out);
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
                cudaGetLastError();
                r->state = MPDATA_REQ_FAILED;
                r->error = MPDATA_ECUDA;
            }
        }
        r->t_done = now_s(s->t0);
        destroy_events(r);
        mark_terminal(s, r);
        any = true;
    }
    s->copying.swap(still);
    if (any) s->cv_done.notify_all();
}

// Loading requests whose copy-in has completed join the resident set (lock
// held).  Returns true if any request is still loading.
bool promote_loaded(mpdata_server *s) {
    std::vector<Request *> still;
    for (Request *r : s->loading) {
        cudaError_t q = cudaEventQuery(r->ready_ev);
        if (q == cudaErrorNotReady) { still.push_back(r); continue; }
        if (q != cudaSuccess) {
            cudaGetLastError();
            fail_request(s, r, MPDATA_ECUDA, s->copy_in);
            s->cv_done.notify_all();
        } else if (r->cancel.load() || s->stop) {
            r->state = MPDATA_REQ_CANCELLED;
            r->t_done = now_s(s->t0);
            free_request_device(r, s->copy_in);
            destroy_events(r);
            s->admitted_bytes -= r->bytes;
            mark_terminal(s, r);
            s->cv_done.notify_all();
        } else {
            s->active.push_back(r);
        }
    }
    s->loading.swap(still);
    return !s->loading.empty();
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
                    destroy_events(r);
                    mark_terminal(s, r);
                    s->cv_done.notify_all();
                } else {
                    ++it;
                }
            }
            promote_loaded(s);
            // admission: FIFO while the budget and the slots allow
            while (!s->stop && !s->queue.empty()) {
                Request *r = s->queue.front();
                if (s->active.size() + s->loading.size() + admit.size() >= (size_t)s->o.max_active) break;
                if (s->admitted_bytes + r->bytes > s->o.hbm_budget_bytes) break;
                s->queue.pop_front();
                s->admitted_bytes += r->bytes;
                if (r->bytes <= s->reserved_bytes) s->reserved_bytes -= r->bytes;
                ++s->admissions;
                r->state = MPDATA_REQ_RUNNING;
                r->t_admit = now_s(s->t0);
                admit.push_back(r);
                admit_injected.push_back(s->o.inject_alloc_failure > 0 &&
                                         s->admissions % (unsigned)s->o.inject_alloc_failure == 0);
            }
            if (s->stop)
                for (Request *r : s->active) r->cancel.store(true);
            if (s->active.empty() && admit.empty()) {
                if (s->stop && s->copying.empty() && s->loading.empty()) break;
                if (!s->copying.empty() || !s->loading.empty()) {
                    lk.unlock();
                    std::this_thread::sleep_for(std::chrono::microseconds(50));
                } else {
                    s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
                }
                continue;
            }
        }
        // copy-in of the admitted requests (no lock): enqueued on the copy-in
        // stream; they join the ticks once their copies have landed
        std::vector<int> load_rc(admit.size());
        for (size_t i = 0; i < admit.size(); ++i) load_rc[i] = load_request(s, admit[i], admit_injected[i]);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (size_t i = 0; i < admit.size(); ++i) {
                Request *r = admit[i];
                if (load_rc[i] != MPDATA_OK) {
                    fail_request(s, r, load_rc[i], s->copy_in);
                    s->cv_done.notify_all();
                    continue;
                }
                s->loading.push_back(r);
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
                    fail_request(s, r, MPDATA_ECUDA, s->stream);
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
    cudaStreamSynchronize(s->copy_in);
    cudaStreamSynchronize(s->copy_out);
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
    o->retain_finished = 1 << 16;
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
    if (o.retain_finished < 0) return sfail(MPDATA_EINVAL, "retain_finished must be >= 0");
    mpdata_server *s = new (std::nothrow) mpdata_server();
    if (!s) return sfail(MPDATA_ENOMEM, "host allocation failed");
    s->o = o;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy_out, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&s->tick[i].ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (auto &T : s->tick)
            if (T.ev) cudaEventDestroy(T.ev);
        for (cudaStream_t st : {s->stream, s->copy_in, s->copy_out})
            if (st) cudaStreamDestroy(st);
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
    if (req->nsteps > 0 && (cudaEventCreateWithFlags(&r->ready_ev, cudaEventDisableTiming) != cudaSuccess ||
                            cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming) != cudaSuccess)) {
        cudaGetLastError();
        destroy_events(r);
        delete r;
        return sfail(MPDATA_ECUDA, "cudaEventCreate failed");
    }
    r->ticket = s->next_ticket++;
    r->t_submit = now_s(s->t0);
    s->all[r->ticket] = r;
    if (req->nsteps == 0) {  // nothing to do: psi already holds the answer
        r->state = MPDATA_REQ_DONE;
        r->t_admit = r->t_done = r->t_submit;
        *ticket = r->ticket;
        mark_terminal(s, r);  // (may retire it at once when retain_finished is 0)
        return MPDATA_OK;
    }
    s->reserved_bytes += r->bytes;
    s->queue.push_back(r);
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
    // while counted as a waiter the request is neither retired nor freed by
    // mpdata_server_destroy
    ++r->waiters;
    ++s->waiters;
    auto finished = [r] { return terminal(r); };
    bool done = true;
    if (timeout_ms < 0) s->cv_done.wait(lk, finished);
    else done = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished);
    const int state = r->state, error = r->error;
    --r->waiters;
    if (--s->waiters == 0) s->cv_done.notify_all();  // mpdata_server_destroy may be waiting
    if (done) retire_excess(s);
    if (!done)
        return sfail(MPDATA_ETIMEDOUT, "ticket %llu not finished after %d ms", (unsigned long long)ticket, timeout_ms);
    if (state == MPDATA_REQ_DONE) return MPDATA_OK;
    if (state == MPDATA_REQ_CANCELLED) return sfail(MPDATA_ECANCELED, "ticket %llu was cancelled", (unsigned long long)ticket);
    return sfail(error ? error : MPDATA_ECUDA, "ticket %llu failed", (unsigned long long)ticket);
}

int mpdata_release(mpdata_server_t *s, uint64_t ticket) {
    if (!s) return sfail(MPDATA_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return sfail(MPDATA_ENOENT, "unknown ticket %llu", (unsigned long long)ticket);
    Request *r = it->second;
    if (!terminal(r)) return sfail(MPDATA_EBUSY, "ticket %llu has not finished", (unsigned long long)ticket);
    if (r->waiters > 0) return sfail(MPDATA_EBUSY, "ticket %llu is being waited on", (unsigned long long)ticket);
    destroy_events(r);
    delete r;
    s->all.erase(it);  // its entry in finished_order is skipped when reached
    return MPDATA_OK;
}

int mpdata_server_retained(mpdata_server_t *s, uint64_t *count) {
    if (!s || !count) return sfail(MPDATA_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *count = (uint64_t)s->all.size();
    return MPDATA_OK;
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
            r->t_done = now_s(s->t0);
        }
        s->queue.clear();
        s->cv_work.notify_all();
    }
    // the scheduler cancels resident and loading requests and drains the
    // copies before it returns: every request is then finished
    if (s->thr.joinable()) s->thr.join();
    {
        // release the threads blocked in mpdata_wait and let them read their
        // request before anything is freed
        std::unique_lock<std::mutex> lk(s->mu);
        for (auto &kv : s->all)
            if (!terminal(kv.second)) kv.second->state = MPDATA_REQ_CANCELLED;
        s->cv_done.notify_all();
        s->cv_done.wait(lk, [s] { return s->waiters == 0; });
    }
    for (auto &kv : s->all) {
        destroy_events(kv.second);
        delete kv.second;
    }
    for (auto &T : s->tick) {
        cudaFree(T.d_grids);
        cudaFree(T.d_items);
        cudaFree(T.d_begin);
        if (T.ev) cudaEventDestroy(T.ev);
    }
    cudaStreamDestroy(s->stream);
    cudaStreamDestroy(s->copy_in);
    cudaStreamDestroy(s->copy_out);
    delete s;
    return MPDATA_OK;
}

}  // extern "C"
