// C ABI of libmpdata (declared in include/mpdata.h): argument checking,
// device-buffer ownership and the step loop.  All arithmetic of the step runs
// in the kernels of mpdata_fused.cu / mpdata_stages.cu / mpdata_reduce.cu.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <string>

#include "mpdata_internal.cuh"

using mpdata::Grid;

struct mpdata_handle {
    int nx, ny, nz;
    long long n;
    size_t esize;
    mpdata_opts opts;
    Grid grid;
    int tile_x, tile_y;
    bool banded;              // default tile: rows in 32x28 and 32x24 bands (launch_fused_bands)
    mpdata::BandPlan band;
    cudaStream_t band_stream;  // the 32x24 bands' launches
    cudaEvent_t band_fork, band_join;
    void *scratch;            // psi-sized ping-pong partner
    mpdata::StageBuffers st;  // stage-per-kernel intermediates (path STAGES only)
    double *partials;         // mass reduction partials (kReduceBlocks x 3)
    void *host_fields[5];     // device copies for mpdata_solve_host (lazy); slot 0 of the pipeline
    // mpdata_host_submit pipeline (created on the first submit)
    bool pipe_ready;
    void *pipe_fields[5];     // slot 1
    cudaStream_t pipe_in, pipe_out;
    cudaEvent_t loaded[2], stepped[2], freed[2];  // per slot
    cudaEvent_t done[16];                         // per ticket, ring of 16
    bool slot_used[2];
    unsigned long long issued, waited;
};

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

}  // namespace

int mpdata::set_error(int code, const char *message) {
    g_last_error = message;
    return code;
}

namespace {

int cuda_fail(cudaError_t e, const char *what) {
    return fail(MPDATA_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

bool aligned16(const void *p) { return p && ((uintptr_t)p & 15u) == 0; }

int check_opts(const mpdata_opts *o) {
    if (o->size < sizeof(mpdata_opts)) return fail(MPDATA_EINVAL, "opts.size too small (use mpdata_opts_default)");
    if (o->iterations < 1 || o->iterations > 3) return fail(MPDATA_EINVAL, "iterations must be 1, 2 or 3");
    if (o->nonoscillatory != 0 && o->nonoscillatory != 1) return fail(MPDATA_EINVAL, "nonoscillatory must be 0 or 1");
    for (int d = 0; d < 3; ++d)
        if (o->periodic[d] != 0 && o->periodic[d] != 1) return fail(MPDATA_EINVAL, "periodic[%d] must be 0 or 1", d);
    if (o->dtype != MPDATA_F32 && o->dtype != MPDATA_F64) return fail(MPDATA_EINVAL, "dtype must be MPDATA_F32 or MPDATA_F64");
    if (o->path != MPDATA_PATH_FUSED && o->path != MPDATA_PATH_STAGES) return fail(MPDATA_EINVAL, "unknown path");
    if (!(o->eps > 0.0)) return fail(MPDATA_EINVAL, "eps must be > 0");
    if (o->extrema != MPDATA_EXTREMA_BOTH && o->extrema != MPDATA_EXTREMA_CORRECTED)
        return fail(MPDATA_EINVAL, "extrema must be MPDATA_EXTREMA_BOTH or MPDATA_EXTREMA_CORRECTED");
    if (o->precision != MPDATA_PREC_PURE && o->precision != MPDATA_PREC_F64_BETA)
        return fail(MPDATA_EINVAL, "precision must be MPDATA_PREC_PURE or MPDATA_PREC_F64_BETA");
    if (o->path == MPDATA_PATH_FUSED && o->iterations > 1 &&
        (o->iterations == 3 || o->extrema != MPDATA_EXTREMA_BOTH ||
         (o->precision != MPDATA_PREC_PURE && o->dtype == MPDATA_F32)))
        return fail(MPDATA_EINVAL, "the fused kernel runs two passes with the default extrema set in "
                                   "pure precision; use path = MPDATA_PATH_STAGES for this option");
    return MPDATA_OK;
}

constexpr int kDoneRing = 16;

void free_handle(mpdata_t *m) {
    if (!m) return;
    if (m->banded) {
        if (m->band_join) cudaEventSynchronize(m->band_join);
        if (m->band_fork) cudaEventDestroy(m->band_fork);
        if (m->band_join) cudaEventDestroy(m->band_join);
        if (m->band_stream) cudaStreamDestroy(m->band_stream);
    }
    if (m->pipe_ready) {
        // the last copy out ends after every pipelined copy and step
        if (m->issued) cudaEventSynchronize(m->done[m->issued % kDoneRing]);
        for (int i = 0; i < 2; ++i) {
            cudaEventDestroy(m->loaded[i]);
            cudaEventDestroy(m->stepped[i]);
            cudaEventDestroy(m->freed[i]);
        }
        for (int i = 0; i < kDoneRing; ++i) cudaEventDestroy(m->done[i]);
        cudaStreamDestroy(m->pipe_in);
        cudaStreamDestroy(m->pipe_out);
        for (int f = 0; f < 5; ++f) cudaFree(m->pipe_fields[f]);
    }
    cudaFree(m->scratch);
    cudaFree(m->st.psi1);
    cudaFree(m->st.v1);
    cudaFree(m->st.v2);
    cudaFree(m->st.v3);
    cudaFree(m->st.bup);
    cudaFree(m->st.bdn);
    cudaFree(m->st.psi2);
    cudaFree(m->st.w1);
    cudaFree(m->st.w2);
    cudaFree(m->st.w3);
    cudaFree(m->partials);
    for (int f = 0; f < 5; ++f) cudaFree(m->host_fields[f]);
    delete m;
}

int launch_one(mpdata_t *m, const void *h, const void *src, const void *u1, const void *u2,
               const void *u3, void *dst, cudaStream_t s) {
    const mpdata_opts &o = m->opts;
    cudaError_t e;
    if (o.iterations == 1)
        e = mpdata::launch_donor(o.dtype, m->grid, h, src, u1, u2, u3, dst, s);
    else if (o.path == MPDATA_PATH_STAGES)
        e = mpdata::launch_stage_step(o.dtype, m->grid, o.iterations, o.nonoscillatory, o.extrema,
                                      o.precision, o.eps, h, src, u1, u2, u3, dst, m->st, s);
    else if (m->banded)
        e = mpdata::launch_fused_bands(m->grid, o.nonoscillatory, o.eps, m->band, h, src, u1, u2, u3, dst, s,
                                       m->band_stream, m->band_fork, m->band_join);
    else
        e = mpdata::launch_fused_step(o.dtype, m->grid, o.nonoscillatory, o.eps, m->tile_x,
                                      m->tile_y, h, src, u1, u2, u3, dst, s);
    return e == cudaSuccess ? MPDATA_OK : cuda_fail(e, "kernel launch");
}

}  // namespace

extern "C" {

void mpdata_opts_default(mpdata_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->size = sizeof *o;
    o->iterations = 2;
    o->nonoscillatory = 1;
    o->periodic[0] = o->periodic[1] = o->periodic[2] = 1;
    o->dtype = MPDATA_F32;
    o->path = MPDATA_PATH_FUSED;
    o->tile_x = o->tile_y = 0;
    o->eps = 1e-15;
    o->extrema = MPDATA_EXTREMA_BOTH;
    o->precision = MPDATA_PREC_PURE;
}

int mpdata_create(int nx, int ny, int nz, const mpdata_opts *opts, mpdata_t **out) {
    if (!out) return fail(MPDATA_EINVAL, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(MPDATA_EINVAL, "dims must be >= 1 (got %d x %d x %d)", nx, ny, nz);
    long long n = (long long)nx * ny * nz;
    // in-plane offsets are 32-bit, plane offsets 64-bit
    if ((long long)nx * ny >= (1LL << 31)) return fail(MPDATA_EINVAL, "nx * ny = %lld: one z-plane must hold fewer than 2^31 cells", (long long)nx * ny);
    if (n >= (1LL << 40)) return fail(MPDATA_EINVAL, "grid of %lld cells is too large (limit 2^40 - 1)", n);
    if (ny > 65535 || nz > 65535) return fail(MPDATA_EINVAL, "ny and nz must be <= 65535");
    mpdata_opts o;
    if (opts) o = *opts; else mpdata_opts_default(&o);
    int rc = check_opts(&o);
    if (rc) return rc;
    Grid grid;
    grid.nx = nx; grid.ny = ny; grid.nz = nz;
    for (int d = 0; d < 3; ++d) grid.per[d] = o.periodic[d];
    int tx = o.tile_x, ty = o.tile_y;
    mpdata::BandPlan band{0, 0};
    bool banded = false;
    if (tx == 0 && ty == 0) {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            nsm = 0;  // no device yet: the SM count only tunes the default tile
        }
        mpdata::fused_default_tile(o.dtype, grid, nsm, &tx, &ty);
        // a large FP32 grid may run as rows in 28- and 24-row bands instead
        banded = o.dtype == MPDATA_F32 && o.path == MPDATA_PATH_FUSED && o.iterations == 2 && tx == 32 &&
                 (ty == 24 || ty == 28) && mpdata::fused_band_plan(grid, nsm, &band);
    }
    if (o.path == MPDATA_PATH_FUSED && o.iterations == 2 && !mpdata::fused_tile_supported(o.dtype, grid, tx, ty))
        return fail(MPDATA_EINVAL, "no fused kernel for tile %d x %d on this grid", tx, ty);

    mpdata_t *m = new (std::nothrow) mpdata_handle();
    if (!m) return fail(MPDATA_ENOMEM, "host allocation failed");
    memset(m, 0, sizeof *m);
    m->nx = nx; m->ny = ny; m->nz = nz; m->n = n;
    m->opts = o;
    m->esize = o.dtype == MPDATA_F64 ? sizeof(double) : sizeof(float);
    m->grid = grid;
    m->tile_x = tx; m->tile_y = ty;
    const size_t bytes = (size_t)n * m->esize;
    cudaError_t e = cudaMalloc(&m->scratch, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->partials, sizeof(double) * 3 * mpdata::kReduceBlocks);
    if (e == cudaSuccess && o.path == MPDATA_PATH_STAGES) {
        void **b[6] = {&m->st.psi1, &m->st.v1, &m->st.v2, &m->st.v3, &m->st.bup, &m->st.bdn};
        for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaMalloc(b[i], bytes);
        if (o.iterations == 3) {
            void **b3[4] = {&m->st.psi2, &m->st.w1, &m->st.w2, &m->st.w3};
            for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaMalloc(b3[i], bytes);
        }
    }
    if (e == cudaSuccess && banded) {
        m->banded = true;
        m->band = band;
        e = cudaStreamCreateWithFlags(&m->band_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->band_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->band_join, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_handle(m);
        return e == cudaErrorMemoryAllocation ? fail(MPDATA_ENOMEM, "device allocation of %zu bytes failed", bytes)
                                              : cuda_fail(e, "cudaMalloc");
    }
    *out = m;
    return MPDATA_OK;
}

int mpdata_destroy(mpdata_t *m) {
    free_handle(m);
    return MPDATA_OK;
}

int mpdata_get_tile(const mpdata_t *m, int *tile_x, int *tile_y) {
    if (!m || !tile_x || !tile_y) return fail(MPDATA_EINVAL, "NULL argument");
    const bool fused = m->opts.path == MPDATA_PATH_FUSED && m->opts.iterations == 2;
    *tile_x = fused ? m->tile_x : 0;
    *tile_y = fused ? m->tile_y : 0;
    return MPDATA_OK;
}

int mpdata_plan_bands(int nx, int ny, int nz, const int *periodic, int nsm, int *n28, int *n24) {
    if (!periodic || !n28 || !n24) return fail(MPDATA_EINVAL, "NULL argument");
    if (nx < 1 || ny < 1 || nz < 1 || nsm < 0) return fail(MPDATA_EINVAL, "bad dims or nsm");
    Grid g;
    g.nx = nx; g.ny = ny; g.nz = nz;
    for (int d = 0; d < 3; ++d) g.per[d] = periodic[d] != 0;
    mpdata::BandPlan b{0, 0};
    const bool use = mpdata::fused_band_plan(g, nsm, &b);
    *n28 = use ? b.n28 : 0;
    *n24 = use ? b.n24 : 0;
    return MPDATA_OK;
}

int mpdata_default_tile(int nx, int ny, int nz, int dtype, int nsm, int *tile_x, int *tile_y) {
    if (!tile_x || !tile_y) return fail(MPDATA_EINVAL, "NULL argument");
    if (nx < 1 || ny < 1 || nz < 1 || nsm < 0) return fail(MPDATA_EINVAL, "bad dims or nsm");
    if (dtype != MPDATA_F32 && dtype != MPDATA_F64) return fail(MPDATA_EINVAL, "dtype must be MPDATA_F32 or MPDATA_F64");
    Grid g;
    g.nx = nx; g.ny = ny; g.nz = nz;
    for (int d = 0; d < 3; ++d) g.per[d] = 1;
    mpdata::fused_default_tile(dtype, g, nsm, tile_x, tile_y);
    return MPDATA_OK;
}

int mpdata_get_bands(const mpdata_t *m, int *n28, int *n24) {
    if (!m || !n28 || !n24) return fail(MPDATA_EINVAL, "NULL argument");
    *n28 = m->banded ? m->band.n28 : 0;
    *n24 = m->banded ? m->band.n24 : 0;
    return MPDATA_OK;
}

int mpdata_step(mpdata_t *m, const void *h, void *psi, const void *u1, const void *u2,
                const void *u3, int nsteps, void *stream) {
    if (!m) return fail(MPDATA_EINVAL, "handle is NULL");
    if (nsteps < 0) return fail(MPDATA_EINVAL, "nsteps must be >= 0");
    const void *ptrs[5] = {h, psi, u1, u2, u3};
    const char *names[5] = {"h", "psi", "u1", "u2", "u3"};
    for (int f = 0; f < 5; ++f)
        if (!aligned16(ptrs[f])) return fail(MPDATA_EINVAL, "%s is NULL or not 16-byte aligned", names[f]);
    if (psi == m->scratch) return fail(MPDATA_EINVAL, "psi aliases the handle's scratch buffer");
    if (nsteps == 0) return MPDATA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    void *cur = psi, *other = m->scratch;
    if (nsteps & 1) {
        cudaError_t e = cudaMemcpyAsync(m->scratch, psi, (size_t)m->n * m->esize, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
        cur = m->scratch;
        other = psi;
    }
    for (int st = 0; st < nsteps; ++st) {
        int rc = launch_one(m, h, cur, u1, u2, u3, other, s);
        if (rc) return rc;
        void *tmp = cur; cur = other; other = tmp;
    }
    return MPDATA_OK;
}

namespace {

// Device copies of the five fields for a host solve (allocated once).
int alloc_fields(mpdata_t *m, void **f) {
    const size_t bytes = (size_t)m->n * m->esize;
    for (int k = 0; k < 5; ++k) {
        if (f[k]) continue;
        cudaError_t e = cudaMalloc(&f[k], bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            f[k] = nullptr;
            return fail(MPDATA_ENOMEM, "device allocation of %zu bytes failed", bytes);
        }
    }
    return MPDATA_OK;
}

int check_host_args(const void *const src[5], int nsteps) {
    const char *names[5] = {"h", "psi", "u1", "u2", "u3"};
    for (int f = 0; f < 5; ++f)
        if (!src[f]) return fail(MPDATA_EINVAL, "%s is NULL", names[f]);
    if (nsteps < 0) return fail(MPDATA_EINVAL, "nsteps must be >= 0");
    return MPDATA_OK;
}

int pipe_init(mpdata_t *m) {
    cudaError_t e = cudaStreamCreateWithFlags(&m->pipe_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m->pipe_out, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&m->loaded[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->stepped[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->freed[i], cudaEventDisableTiming);
    }
    for (int i = 0; i < kDoneRing && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&m->done[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "creating the host pipeline's streams and events");
    m->pipe_ready = true;
    return MPDATA_OK;
}

}  // namespace

int mpdata_solve_host(mpdata_t *m, const void *h, void *psi, const void *u1, const void *u2,
                      const void *u3, int nsteps, void *stream) {
    if (!m) return fail(MPDATA_EINVAL, "handle is NULL");
    const void *src[5] = {h, psi, u1, u2, u3};
    int rc = check_host_args(src, nsteps);
    if (rc) return rc;
    if ((rc = alloc_fields(m, m->host_fields))) return rc;
    const size_t bytes = (size_t)m->n * m->esize;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    // pipelined solves share slot 0 and the scratch buffer: wait for the last
    // one to be copied out (every earlier one has been by then)
    if (m->pipe_ready && m->issued && (e = cudaStreamWaitEvent(s, m->done[m->issued % kDoneRing], 0)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamWaitEvent");
    for (int f = 0; f < 5; ++f) {
        e = cudaMemcpyAsync(m->host_fields[f], src[f], bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync host to device");
    }
    rc = mpdata_step(m, m->host_fields[0], m->host_fields[1], m->host_fields[2],
                     m->host_fields[3], m->host_fields[4], nsteps, stream);
    if (rc) return rc;
    e = cudaMemcpyAsync(psi, m->host_fields[1], bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync device to host");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return MPDATA_OK;
}

int mpdata_host_submit(mpdata_t *m, const void *h, const void *psi_in, const void *u1,
                       const void *u2, const void *u3, int nsteps, void *psi_out, void *stream,
                       unsigned long long *ticket) {
    if (!m) return fail(MPDATA_EINVAL, "handle is NULL");
    if (!psi_out || !ticket) return fail(MPDATA_EINVAL, "psi_out or ticket is NULL");
    const void *src[5] = {h, psi_in, u1, u2, u3};
    int rc = check_host_args(src, nsteps);
    if (rc) return rc;
    if (!m->pipe_ready && (rc = pipe_init(m))) return rc;
    const int sl = (int)(m->issued & 1);  // ticket issued + 1 takes slot issued % 2
    void **f = sl ? m->pipe_fields : m->host_fields;
    if ((rc = alloc_fields(m, f))) return rc;
    const size_t bytes = (size_t)m->n * m->esize;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned long long t = m->issued + 1;
    cudaError_t e = cudaSuccess;
    // copy in once the slot's previous solve has been copied out
    if (m->slot_used[sl]) e = cudaStreamWaitEvent(m->pipe_in, m->freed[sl], 0);
    for (int k = 0; k < 5 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(f[k], src[k], bytes, cudaMemcpyHostToDevice, m->pipe_in);
    if (e == cudaSuccess) e = cudaEventRecord(m->loaded[sl], m->pipe_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, m->loaded[sl], 0);
    if (e != cudaSuccess) return cuda_fail(e, "enqueueing the copy in");
    if ((rc = mpdata_step(m, f[0], f[1], f[2], f[3], f[4], nsteps, stream))) return rc;
    e = cudaEventRecord(m->stepped[sl], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(m->pipe_out, m->stepped[sl], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(psi_out, f[1], bytes, cudaMemcpyDeviceToHost, m->pipe_out);
    if (e == cudaSuccess) e = cudaEventRecord(m->freed[sl], m->pipe_out);
    if (e == cudaSuccess) e = cudaEventRecord(m->done[t % kDoneRing], m->pipe_out);
    if (e != cudaSuccess) return cuda_fail(e, "enqueueing the copy out");
    m->slot_used[sl] = true;
    m->issued = t;
    *ticket = t;
    return MPDATA_OK;
}

int mpdata_host_wait(mpdata_t *m, unsigned long long ticket) {
    if (!m) return fail(MPDATA_EINVAL, "handle is NULL");
    if (ticket == 0 || ticket > m->issued) return fail(MPDATA_ENOENT, "ticket %llu was not issued", ticket);
    if (ticket <= m->waited) return MPDATA_OK;
    // a ring entry re-recorded by a later ticket completes after this one
    // (the copies out run in submit order), so the wait is never early
    cudaError_t e = cudaEventSynchronize(m->done[ticket % kDoneRing]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    m->waited = ticket;
    return MPDATA_OK;
}

int mpdata_mass(mpdata_t *m, const void *h, const void *psi, void *out3, void *stream) {
    if (!m) return fail(MPDATA_EINVAL, "handle is NULL");
    if (!aligned16(h) || !aligned16(psi)) return fail(MPDATA_EINVAL, "h or psi is NULL or not 16-byte aligned");
    if (!out3 || ((uintptr_t)out3 & 7u)) return fail(MPDATA_EINVAL, "out3 is NULL or not 8-byte aligned");
    cudaError_t e = mpdata::launch_mass(m->opts.dtype, m->n, h, psi, m->partials, (double *)out3,
                                        (cudaStream_t)stream);
    return e == cudaSuccess ? MPDATA_OK : cuda_fail(e, "mass kernel launch");
}

int mpdata_courant_max(mpdata_t *m, const void *h, const void *u1, const void *u2, const void *u3,
                       void *out3, void *stream) {
    if (!m) return fail(MPDATA_EINVAL, "handle is NULL");
    const void *ptrs[4] = {h, u1, u2, u3};
    const char *names[4] = {"h", "u1", "u2", "u3"};
    for (int f = 0; f < 4; ++f)
        if (!aligned16(ptrs[f])) return fail(MPDATA_EINVAL, "%s is NULL or not 16-byte aligned", names[f]);
    if (!out3 || ((uintptr_t)out3 & 7u)) return fail(MPDATA_EINVAL, "out3 is NULL or not 8-byte aligned");
    cudaError_t e = mpdata::launch_courant_max(m->opts.dtype, m->grid, h, u1, u2, u3, m->partials,
                                               (double *)out3, (cudaStream_t)stream);
    return e == cudaSuccess ? MPDATA_OK : cuda_fail(e, "courant kernel launch");
}

int mpdata_mass_noalloc(const void *h, const void *psi, long long n, int dtype, void *out3,
                        void *stream) {
    if (n < 1 || n >= (1LL << 31))
        return fail(MPDATA_EINVAL, "n = %lld is outside [1, 2^31 - 1], the largest grid this entry point accepts", n);
    if (dtype != MPDATA_F32 && dtype != MPDATA_F64) return fail(MPDATA_EINVAL, "dtype must be MPDATA_F32 or MPDATA_F64");
    if (!aligned16(h) || !aligned16(psi)) return fail(MPDATA_EINVAL, "h or psi is NULL or not 16-byte aligned");
    if (!out3 || ((uintptr_t)out3 & 7u)) return fail(MPDATA_EINVAL, "out3 is NULL or not 8-byte aligned");
    double *partials = nullptr;
    cudaError_t e = mpdata::noalloc_partials(&partials);
    if (e != cudaSuccess) return cuda_fail(e, "static scratch lookup (cudaGetSymbolAddress)");
    e = mpdata::launch_mass(dtype, n, h, psi, partials, (double *)out3, (cudaStream_t)stream);
    return e == cudaSuccess ? MPDATA_OK : cuda_fail(e, "mass kernel launch");
}

const char *mpdata_strerror(int code) {
    switch (code) {
    case MPDATA_OK: return "ok";
    case MPDATA_EINVAL: return "invalid argument";
    case MPDATA_ENOMEM: return "out of memory";
    case MPDATA_ECUDA: return "CUDA error";
    case MPDATA_EBUSY: return "busy: over budget";
    case MPDATA_ETIMEDOUT: return "timed out";
    case MPDATA_ENOENT: return "no such ticket";
    case MPDATA_ECANCELED: return "cancelled";
    default: return "unknown error";
    }
}

const char *mpdata_last_error_message(void) { return g_last_error.c_str(); }

const char *mpdata_version(void) { return "mpdata-gb300 0.1 (sm_103a)"; }

}  // extern "C"
