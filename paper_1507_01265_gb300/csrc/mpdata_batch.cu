// Batched launch of many independent grids (C ABI in include/mpdata.h:
// mpdata_batch_*).
//
// Every grid is cut into the same tiles as a single-grid launch with its
// tile shape (per grid: 32x24, 32x16 or 32x28).  Tiles of all grids that use
// the same kernel variant (tile shape, lid or not) form one work-item list
// (grid, tile), ordered by decreasing estimated cost (tile area x (nz + 3)
// planes); a launch runs the list with CTA c taking the contiguous items
// [begin[c], begin[c+1]).  The default split gives every item its own CTA,
// so the hardware hands the largest tiles out first and every free SM takes
// the next one; the balanced split (one CTA per SM, contiguous ranges of
// nearly equal cost) and any other split, including the uneven ones of the
// speed-function autotuner, can be installed instead.  A step of the batch is
// one launch per variant (with several variants, each variant's launches run
// on a stream of its own, concurrently with the others'); nsteps steps can be
// captured once into a CUDA graph and replayed.  32x24 and 32x28 tiles of
// grids with nx % 4 == 0 run the kernel with loader warps, as a single-grid
// launch with that tile does.  Each
// tile is computed by the same code whichever CTA runs it, so every grid's
// result is bit-identical to the single-grid launch.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "mpdata_internal.cuh"

using mpdata::BatchGrid;
using mpdata::Grid;

namespace {

enum Variant {
    kPairs24Periodic = 0,  // two columns per thread, tile 32x24, x and y periodic (nx % 4 != 0)
    kPairs24Lid = 1,       // same with a lid on x or y
    kLd24Periodic = 2,     // tile 32x24 with loader warps, x and y periodic (nx % 4 == 0)
    kPairs16Periodic = 3,  // two columns per thread, tile 32x16 (any nx)
    kPairs16Lid = 4,
    kPairs28Periodic = 5,  // two columns per thread, tile 32x28 (nx % 4 != 0)
    kPairs28Lid = 6,
    kLd24Lid = 7,          // tile 32x24 with loader warps, a lid on x or y (nx % 4 == 0)
    kLd28Periodic = 8,     // tile 32x28 with loader warps (nx % 4 == 0)
    kLd28Lid = 9,
    kNumVariants = 10
};

int variant_tile_y(int v) {
    if (v == kPairs24Periodic || v == kPairs24Lid || v == kLd24Periodic || v == kLd24Lid) return 24;
    if (v == kPairs28Periodic || v == kPairs28Lid || v == kLd28Periodic || v == kLd28Lid) return 28;
    return 16;
}
bool variant_lid(int v) {
    return v == kPairs24Lid || v == kPairs16Lid || v == kPairs28Lid || v == kLd24Lid || v == kLd28Lid;
}
bool variant_ld(int v) { return v == kLd24Periodic || v == kLd24Lid || v == kLd28Periodic || v == kLd28Lid; }

struct Group {
    std::vector<int2> items;  // (grid, tile), by decreasing cost
    std::vector<double> cost; // per item
    std::vector<int> begin;   // ncta + 1
    int2 *d_items = nullptr;
    int *d_begin = nullptr;
    int ncta = 0;
    bool dirty = true;
};

}  // namespace

struct mpdata_batch {
    int ngrids = 0;
    mpdata_opts opts;
    int nsm = 0;
    std::vector<BatchGrid> grids;    // host copy of the descriptors
    std::vector<int> variant;        // per grid
    std::vector<size_t> bytes;       // per grid psi size
    std::vector<bool> has_fields;
    BatchGrid *d_grids = nullptr;
    bool grids_dirty = true;
    Group group[kNumVariants];
    cudaStream_t capture_stream = nullptr;
    // with several non-empty variants, each variant's chain of steps runs on
    // a stream of its own, forked from and joined back into the caller's
    cudaStream_t vstream[kNumVariants] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kNumVariants] = {};
    int nvariants = 0;  // non-empty variants
    std::map<int, cudaGraphExec_t> graphs;  // by nsteps
    std::map<int, cudaGraph_t> graph_defs;
};

namespace {

int bfail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return mpdata::set_error(code, buf);
}

int bcuda(cudaError_t e, const char *what) {
    return bfail(MPDATA_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

void drop_graphs(mpdata_batch *b) {
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    for (auto &kv : b->graph_defs) cudaGraphDestroy(kv.second);
    b->graphs.clear();
    b->graph_defs.clear();
}

// Split items into ncta contiguous ranges of (nearly) equal total cost: the
// boundary of CTA c sits at the item boundary closest to c/ncta of the total.
void balanced_split(const std::vector<double> &cost, int ncta, std::vector<int> &begin) {
    const int n = (int)cost.size();
    std::vector<double> prefix(n + 1, 0.0);
    for (int i = 0; i < n; ++i) prefix[i + 1] = prefix[i] + cost[i];
    begin.assign(ncta + 1, 0);
    for (int c = 1; c < ncta; ++c) {
        const double target = prefix[n] * c / ncta;
        int i = (int)(std::lower_bound(prefix.begin(), prefix.end(), target) - prefix.begin());
        if (i > 0 && target - prefix[i - 1] < prefix[i] - target) --i;
        begin[c] = std::max(begin[c - 1], std::min(i, n));
    }
    begin[ncta] = n;
}

double item_cost(const BatchGrid &g, int tx, int ty) { return (double)tx * ty * (g.g.nz + 3); }

// One CTA per item (the default).
void per_item_split(Group &G) {
    const int n = (int)G.items.size();
    G.ncta = n;
    G.begin.resize(n + 1);
    for (int i = 0; i <= n; ++i) G.begin[i] = i;
}

int upload_group(mpdata_batch *b, int v) {
    Group &G = b->group[v];
    if (!G.dirty) return MPDATA_OK;
    cudaFree(G.d_items);
    cudaFree(G.d_begin);
    G.d_items = nullptr;
    G.d_begin = nullptr;
    if (G.items.empty()) { G.dirty = false; return MPDATA_OK; }
    cudaError_t e = cudaMalloc((void **)&G.d_items, sizeof(int2) * G.items.size());
    if (e == cudaSuccess) e = cudaMalloc((void **)&G.d_begin, sizeof(int) * G.begin.size());
    if (e == cudaSuccess) e = cudaMemcpy(G.d_items, G.items.data(), sizeof(int2) * G.items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(G.d_begin, G.begin.data(), sizeof(int) * G.begin.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bcuda(e, "batch work-list upload");
    G.dirty = false;
    return MPDATA_OK;
}

// The direct form of a variant's launch (grid table in the kernel
// parameters): only for the default split (one CTA per item, in order) and
// at most kDirectMaxRuns runs of consecutive tiles of one grid.  Returns
// false when the variant needs the general kernel.
bool build_direct(const mpdata_batch *b, const Group &G, mpdata::DirectBatch &d) {
    const int n = (int)G.items.size();
    if (G.ncta != n || (int)G.begin.size() != n + 1) return false;
    for (int i = 0; i <= n; ++i)
        if (G.begin[i] != i) return false;
    d.nruns = 0;
    for (int i = 0; i < n; ++i) {
        const int2 w = G.items[i];
        const bool extend = d.nruns > 0 && G.items[i - 1].x == w.x && G.items[i - 1].y + 1 == w.y;
        if (extend) continue;
        if (d.nruns == mpdata::kDirectMaxRuns) return false;
        d.start[d.nruns] = i;
        d.tile0[d.nruns] = w.y;
        d.g[d.nruns] = b->grids[w.x];
        ++d.nruns;
    }
    d.start[d.nruns] = n;
    return d.nruns > 0;
}

int enqueue_steps(mpdata_batch *b, int nsteps, cudaStream_t s) {
    // direct-launch tables of the variants that can use them (host memory;
    // a launch copies its parameters)
    std::vector<std::unique_ptr<mpdata::DirectBatch>> direct(kNumVariants);
    for (int v = 0; v < kNumVariants; ++v) {
        if (b->group[v].items.empty()) continue;
        direct[v].reset(new (std::nothrow) mpdata::DirectBatch);
        if (direct[v] && !build_direct(b, b->group[v], *direct[v])) direct[v].reset();
    }
    if (nsteps & 1) {
        for (int i = 0; i < b->ngrids; ++i) {
            cudaError_t e = cudaMemcpyAsync(b->grids[i].buf[1], b->grids[i].buf[0], b->bytes[i],
                                            cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return bcuda(e, "cudaMemcpyAsync");
        }
    }
    // The grids of different variants are disjoint, so with several variants
    // each one's steps run on its own stream: the launches of one variant
    // fill the SMs that another's last wave of tiles leaves idle.
    const bool fork = b->nvariants > 1;
    if (fork) {
        cudaError_t e = cudaEventRecord(b->fork_ev, s);
        if (e != cudaSuccess) return bcuda(e, "cudaEventRecord");
    }
    for (int v = 0; v < kNumVariants; ++v) {
        Group &G = b->group[v];
        if (G.items.empty()) continue;
        cudaStream_t vs = fork ? b->vstream[v] : s;
        if (fork) {
            cudaError_t e = cudaStreamWaitEvent(vs, b->fork_ev, 0);
            if (e != cudaSuccess) return bcuda(e, "cudaStreamWaitEvent");
        }
        const int nonosc = b->opts.nonoscillatory, lid = variant_lid(v);
        const int ty = variant_tile_y(v), ld = variant_ld(v);
        for (int st = 0; st < nsteps; ++st) {
            const int parity = (nsteps & 1) ? ((st + 1) & 1) : (st & 1);
            cudaError_t e;
            if (direct[v])
                e = mpdata::launch_fused_pairs_direct(ty, ld, nonosc, lid, *direct[v], parity, vs);
            else
                e = mpdata::launch_fused_pairs_batch(32, ty, ld, nonosc, lid, b->d_grids, G.d_items,
                                                     G.d_begin, G.ncta, parity, vs);
            if (e != cudaSuccess) return bcuda(e, "batched kernel launch");
        }
        if (fork) {
            cudaError_t e = cudaEventRecord(b->join_ev[v], vs);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->join_ev[v], 0);
            if (e != cudaSuccess) return bcuda(e, "joining a variant's stream");
        }
    }
    return MPDATA_OK;
}

}  // namespace

extern "C" {

int mpdata_batch_create(int ngrids, const int *dims, const int *periodic, const mpdata_opts *opts,
                        mpdata_batch_t **out) {
    return mpdata_batch_create_tiles(ngrids, dims, periodic, nullptr, opts, out);
}

int mpdata_batch_create_tiles(int ngrids, const int *dims, const int *periodic, const int *tile_y,
                              const mpdata_opts *opts, mpdata_batch_t **out) {
    if (!out) return bfail(MPDATA_EINVAL, "out is NULL");
    *out = nullptr;
    if (ngrids < 1 || !dims) return bfail(MPDATA_EINVAL, "need ngrids >= 1 and dims");
    mpdata_opts o;
    if (opts) o = *opts; else mpdata_opts_default(&o);
    if (o.size < sizeof(mpdata_opts)) return bfail(MPDATA_EINVAL, "opts.size too small");
    if (o.dtype != MPDATA_F32 || o.iterations != 2 || o.path != MPDATA_PATH_FUSED ||
        o.extrema != MPDATA_EXTREMA_BOTH || o.precision != MPDATA_PREC_PURE)
        return bfail(MPDATA_EINVAL, "batches run the FP32 fused step with 2 iterations, the default "
                                    "extrema set and pure precision");
    if (!(o.eps > 0.0)) return bfail(MPDATA_EINVAL, "eps must be > 0");
    const int tx = o.tile_x ? o.tile_x : 32, ty_default = o.tile_y ? o.tile_y : 24;
    if (!(tx == 32 && (ty_default == 16 || ty_default == 24 || ty_default == 28)))
        return bfail(MPDATA_EINVAL, "batch tile must be 32x16, 32x24 or 32x28");
    if (tile_y)
        for (int i = 0; i < ngrids; ++i)
            if (tile_y[i] != 0 && tile_y[i] != 16 && tile_y[i] != 24 && tile_y[i] != 28)
                return bfail(MPDATA_EINVAL, "tile_y[%d] = %d: must be 0 (the batch default), 16, 24 or 28", i, tile_y[i]);

    mpdata_batch *b = new (std::nothrow) mpdata_batch();
    if (!b) return bfail(MPDATA_ENOMEM, "host allocation failed");
    b->ngrids = ngrids;
    b->opts = o;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) { delete b; return bcuda(e, "cudaDeviceGetAttribute"); }
    b->grids.resize(ngrids);
    b->variant.resize(ngrids);
    b->bytes.resize(ngrids);
    b->has_fields.assign(ngrids, false);
    for (int i = 0; i < ngrids; ++i) {
        const int nx = dims[3 * i], ny = dims[3 * i + 1], nz = dims[3 * i + 2];
        if (nx < 1 || ny < 1 || nz < 1 || ny > 65535 || nz > 65535 || (long long)nx * ny * nz >= (1LL << 31)) {
            mpdata_batch_destroy(b);
            return bfail(MPDATA_EINVAL, "grid %d has bad dims %d x %d x %d", i, nx, ny, nz);
        }
        BatchGrid &g = b->grids[i];
        memset(&g, 0, sizeof g);
        g.g.nx = nx; g.g.ny = ny; g.g.nz = nz;
        for (int d = 0; d < 3; ++d) {
            int p = periodic ? periodic[3 * i + d] : o.periodic[d];
            if (p != 0 && p != 1) { mpdata_batch_destroy(b); return bfail(MPDATA_EINVAL, "periodic flags must be 0 or 1"); }
            g.g.per[d] = p;
        }
        g.eps = (float)o.eps;
        const int ty = (tile_y && tile_y[i]) ? tile_y[i] : ty_default;
        const bool lid = !g.g.per[0] || !g.g.per[1];
        const bool a16 = nx % 4 == 0;
        const int v = ty == 24 ? (a16 ? (lid ? kLd24Lid : kLd24Periodic) : (lid ? kPairs24Lid : kPairs24Periodic))
                      : ty == 28 ? (a16 ? (lid ? kLd28Lid : kLd28Periodic) : (lid ? kPairs28Lid : kPairs28Periodic))
                                 : (lid ? kPairs16Lid : kPairs16Periodic);
        g.ntx = (nx + tx - 1) / tx;
        const int ntiles = g.ntx * ((ny + ty - 1) / ty);
        b->variant[i] = v;
        b->bytes[i] = (size_t)nx * ny * nz * sizeof(float);
        for (int tl = 0; tl < ntiles; ++tl) {
            b->group[v].items.push_back(make_int2(i, tl));
            b->group[v].cost.push_back(item_cost(g, tx, ty));
        }
        e = cudaMalloc((void **)&g.buf[1], b->bytes[i]);  // scratch partner of psi
        if (e != cudaSuccess) { cudaGetLastError(); mpdata_batch_destroy(b); return bfail(MPDATA_ENOMEM, "scratch allocation for grid %d failed", i); }
    }
    for (int v = 0; v < kNumVariants; ++v) {
        Group &G = b->group[v];
        // largest items first (stable: a grid's tiles keep their order)
        std::vector<int> order(G.items.size());
        for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return G.cost[x] > G.cost[y]; });
        std::vector<int2> items(order.size());
        std::vector<double> cost(order.size());
        for (size_t k = 0; k < order.size(); ++k) { items[k] = G.items[order[k]]; cost[k] = G.cost[order[k]]; }
        G.items.swap(items);
        G.cost.swap(cost);
        per_item_split(G);
    }
    e = cudaMalloc((void **)&b->d_grids, sizeof(BatchGrid) * ngrids);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    for (int v = 0; v < kNumVariants; ++v)
        if (!b->group[v].items.empty()) ++b->nvariants;
    if (b->nvariants > 1) {
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
        for (int v = 0; v < kNumVariants && e == cudaSuccess; ++v) {
            if (b->group[v].items.empty()) continue;
            e = cudaStreamCreateWithFlags(&b->vstream[v], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev[v], cudaEventDisableTiming);
        }
    }
    if (e != cudaSuccess) { mpdata_batch_destroy(b); return bcuda(e, "batch allocation"); }
    *out = b;
    return MPDATA_OK;
}

int mpdata_batch_set_fields(mpdata_batch_t *b, int grid, const void *h, void *psi, const void *u1,
                            const void *u2, const void *u3) {
    if (!b) return bfail(MPDATA_EINVAL, "batch is NULL");
    if (grid < 0 || grid >= b->ngrids) return bfail(MPDATA_EINVAL, "grid index %d out of range", grid);
    const void *p[5] = {h, psi, u1, u2, u3};
    for (int f = 0; f < 5; ++f)
        if (!p[f] || ((uintptr_t)p[f] & 15u)) return bfail(MPDATA_EINVAL, "field pointers must be non-NULL and 16-byte aligned");
    BatchGrid &g = b->grids[grid];
    g.h = (const float *)h;
    g.u1 = (const float *)u1;
    g.u2 = (const float *)u2;
    g.u3 = (const float *)u3;
    g.buf[0] = (float *)psi;
    b->has_fields[grid] = true;
    b->grids_dirty = true;
    drop_graphs(b);
    return MPDATA_OK;
}

int mpdata_batch_grid_variant(mpdata_batch_t *b, int grid, int *variant) {
    if (!b || !variant || grid < 0 || grid >= b->ngrids) return bfail(MPDATA_EINVAL, "bad arguments");
    *variant = b->variant[grid];
    return MPDATA_OK;
}

int mpdata_batch_work(mpdata_batch_t *b, int variant, int *nitems, int *ncta) {
    if (!b || variant < 0 || variant >= kNumVariants) return bfail(MPDATA_EINVAL, "bad batch or variant");
    if (nitems) *nitems = (int)b->group[variant].items.size();
    if (ncta) *ncta = b->group[variant].ncta;
    return MPDATA_OK;
}

int mpdata_batch_get_split(mpdata_batch_t *b, int variant, int *begin) {
    if (!b || variant < 0 || variant >= kNumVariants || !begin) return bfail(MPDATA_EINVAL, "bad arguments");
    const Group &G = b->group[variant];
    for (size_t i = 0; i < G.begin.size(); ++i) begin[i] = G.begin[i];
    return MPDATA_OK;
}

int mpdata_batch_set_split(mpdata_batch_t *b, int variant, int ncta, const int *begin) {
    if (!b || variant < 0 || variant >= kNumVariants) return bfail(MPDATA_EINVAL, "bad arguments");
    Group &G = b->group[variant];
    const int n = (int)G.items.size();
    if (!begin) {  // the balanced split over ncta CTAs
        if (ncta < 1) return bfail(MPDATA_EINVAL, "ncta must be >= 1");
        if (n == 0) return MPDATA_OK;
        G.ncta = std::min(ncta, n);
        balanced_split(G.cost, G.ncta, G.begin);
        G.dirty = true;
        drop_graphs(b);
        return MPDATA_OK;
    }
    if (ncta < 1 || begin[0] != 0 || begin[ncta] != n)
        return bfail(MPDATA_EINVAL, "split must have ncta >= 1, begin[0] = 0, begin[ncta] = %d", n);
    for (int c = 0; c < ncta; ++c)
        if (begin[c + 1] < begin[c]) return bfail(MPDATA_EINVAL, "split offsets must be nondecreasing");
    G.begin.assign(begin, begin + ncta + 1);
    G.ncta = ncta;
    G.dirty = true;
    drop_graphs(b);
    return MPDATA_OK;
}

int mpdata_batch_step(mpdata_batch_t *b, int nsteps, int use_graph, void *stream) {
    if (!b) return bfail(MPDATA_EINVAL, "batch is NULL");
    if (nsteps < 0) return bfail(MPDATA_EINVAL, "nsteps must be >= 0");
    for (int i = 0; i < b->ngrids; ++i)
        if (!b->has_fields[i]) return bfail(MPDATA_EINVAL, "grid %d has no fields (mpdata_batch_set_fields)", i);
    if (nsteps == 0) return MPDATA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (b->grids_dirty) {
        cudaError_t e = cudaMemcpyAsync(b->d_grids, b->grids.data(), sizeof(BatchGrid) * b->ngrids,
                                        cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return bcuda(e, "descriptor upload");
        e = cudaStreamSynchronize(s);  // the host copy may change after return
        if (e != cudaSuccess) return bcuda(e, "descriptor upload");
        b->grids_dirty = false;
    }
    for (int v = 0; v < kNumVariants; ++v) {
        int rc = upload_group(b, v);
        if (rc) return rc;
    }
    if (!use_graph) return enqueue_steps(b, nsteps, s);
    auto it = b->graphs.find(nsteps);
    if (it == b->graphs.end()) {
        cudaStream_t cs = b->capture_stream;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return bcuda(e, "cudaStreamBeginCapture");
        int rc = enqueue_steps(b, nsteps, cs);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cs, &graph);
        if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
        if (e != cudaSuccess) return bcuda(e, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) { cudaGraphDestroy(graph); return bcuda(e, "cudaGraphInstantiate"); }
        b->graph_defs[nsteps] = graph;
        it = b->graphs.emplace(nsteps, exec).first;
    }
    cudaError_t e = cudaGraphLaunch(it->second, s);
    return e == cudaSuccess ? MPDATA_OK : bcuda(e, "cudaGraphLaunch");
}

int mpdata_batch_destroy(mpdata_batch_t *b) {
    if (!b) return MPDATA_OK;
    drop_graphs(b);
    for (auto &g : b->grids) cudaFree(g.buf[1]);
    for (auto &G : b->group) { cudaFree(G.d_items); cudaFree(G.d_begin); }
    cudaFree(b->d_grids);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    for (int v = 0; v < kNumVariants; ++v) {
        if (b->vstream[v]) cudaStreamDestroy(b->vstream[v]);
        if (b->join_ev[v]) cudaEventDestroy(b->join_ev[v]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    delete b;
    return MPDATA_OK;
}

}  // extern "C"
