/*
 * mpdata.h -- C ABI of the GB300 (sm_103a) MPDATA advection library.
 *
 * One MPDATA time step advances a scalar psi carried by a density h and
 * staggered Courant numbers u1, u2, u3: each step reads these five fields and
 * produces one (§5.2).
 * The step is the nonoscillatory forward-in-time scheme the paper refers to
 * in §5.2: a donor-cell (upstream) pass, antidiffusive pseudo-velocities with
 * cross terms, the nonoscillatory limiter (local extrema as in Listing 1,
 * stage 8, then limiter factors) and a corrective donor-cell pass.
 *
 * Layout of every field: contiguous [nz][ny][nx], x fastest, element index
 * (k*ny + j)*nx + i, in the handle's dtype (float for MPDATA_F32, double for
 * MPDATA_F64).  u1[k][j][i] is the Courant number on the x-face between
 * cells i-1 and i (the lower x-face of cell i); u2 and u3 likewise for y and
 * z.  On a periodic axis face 0 is the face between cells n-1 and 0.  On a
 * rigid-lid axis faces 0 and n carry zero velocity: the stored face-0 value
 * is never read, and ghost cells beyond the lid are zero-gradient copies of
 * the edge cell.  psi is expected to be >= 0 (the scheme is positive
 * definite), h > 0, and the caller keeps the Courant numbers stable
 * (sum_d |u_d| / h <= 1 per cell).
 *
 * Pointers: "device" arguments are CUDA device pointers (e.g. the data of
 * torch CUDA tensors), 16-byte aligned.  "host" arguments are ordinary host
 * pointers (pinned memory gives the fastest copies).  The caller owns every
 * field buffer; the library never frees them.
 *
 * Streams: `stream` is a cudaStream_t passed as void*; NULL is the legacy
 * default stream.  Entry points marked "async" only enqueue work.
 *
 * Errors: every entry point returns MPDATA_OK (0) or a negative MPDATA_E*
 * code; nothing aborts, traps or prints.  mpdata_strerror() names a code and
 * mpdata_last_error_message() gives the detail of the calling thread's last
 * failure.  A handle is used by one host thread at a time.  A handle's
 * device scratch is shared by its calls: mpdata_step uses its psi-sized
 * ping-pong buffer, mpdata_mass and mpdata_courant_max its reduction
 * partials, so the calls on one handle must run in order on one stream (or
 * be serialised by the caller); calls on different streams race on them.
 */
#ifndef MPDATA_H
#define MPDATA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPDATA_OK 0
#define MPDATA_EINVAL (-1)    /* bad argument: dims, null/misaligned pointer, option */
#define MPDATA_ENOMEM (-2)    /* device or host allocation failed */
#define MPDATA_ECUDA (-3)     /* a CUDA call or kernel launch failed */
#define MPDATA_EBUSY (-4)     /* admission refused: over the server's budget */
#define MPDATA_ETIMEDOUT (-5) /* a wait ran out of time */
#define MPDATA_ENOENT (-6)    /* unknown ticket */
#define MPDATA_ECANCELED (-7) /* request was cancelled */

#define MPDATA_F32 0
#define MPDATA_F64 1

#define MPDATA_PATH_FUSED 0  /* all stages of a step in one kernel */
#define MPDATA_PATH_STAGES 1 /* one kernel per stage, intermediates in HBM */

/* Bounding set of the limiter's local extrema (max/min over a cell and its
 * six face neighbours, Listing 1 "stage 8"; the set itself follows
 * Smolarkiewicz & Grabowski 1990). */
#define MPDATA_EXTREMA_BOTH 0      /* psi^n and the field being corrected (default) */
#define MPDATA_EXTREMA_CORRECTED 1 /* the field being corrected only */

/* Arithmetic of an FP32 step. */
#define MPDATA_PREC_PURE 0     /* every operation in the dtype (default) */
#define MPDATA_PREC_F64_BETA 1 /* FP32 fields; the limiter's in/out flux sums and
                                  beta factors in FP64 (stage path only) */

typedef struct mpdata_opts {
    uint32_t size;          /* sizeof(mpdata_opts); set by mpdata_opts_default */
    int32_t iterations;     /* 1: donor cell only; 2: one corrective pass (default);
                               3: two corrective passes, the second built from the
                               velocities the first transported with (stage path) */
    int32_t nonoscillatory; /* 1: limit the antidiffusive velocities (default) */
    int32_t periodic[3];    /* per axis x, y, z: 1 periodic (default), 0 rigid lid */
    int32_t dtype;          /* MPDATA_F32 (default) or MPDATA_F64 */
    int32_t path;           /* MPDATA_PATH_FUSED (default) or MPDATA_PATH_STAGES */
    int32_t tile_x, tile_y; /* fused-kernel output tile.  FP32: 32x28, 32x24, 32x16 or
                               32x12 (two CTAs per SM) run the two-column kernel
                               (any nx), 24x24, 24x16, 16x16 the one-column kernel;
                               FP64: 16x16.  0 x 0 picks the tile of least
                               predicted step time for the grid on this device
                               (waves of tiles x measured per-plane time) */
    double eps;             /* > 0, added to every A, B and limiter denominator; default 1e-15 */
    int32_t extrema;        /* MPDATA_EXTREMA_BOTH (default) or _CORRECTED (stage path) */
    int32_t precision;      /* MPDATA_PREC_PURE (default) or _F64_BETA (FP32, stage path) */
} mpdata_opts;

typedef struct mpdata_handle mpdata_t;

/* Fill *opts with the defaults listed above. */
void mpdata_opts_default(mpdata_opts *opts);

/* Create a solver for an nx x ny x nz grid on the current CUDA device: the
 * MPDATA step of §5.2, run (path FUSED) with all its stages in one kernel
 * pass over the grid, the GPU form of the paper's fused block-wise
 * execution (§5.3), or (path STAGES) one kernel per stage.
 * Limits: each dimension >= 1, ny and nz <= 65535, nx * ny < 2^31 (one
 * z-plane), nx * ny * nz < 2^40 (beyond 2^31 cells the grid is addressed
 * with 64-bit plane offsets; device memory is the practical limit: 6 fields
 * of 4 or 8 bytes per cell).  The handle owns one psi-sized device scratch buffer (the step's
 * ping-pong partner) and, for the stage-per-kernel path, the intermediate
 * arrays; they are allocated here and freed by mpdata_destroy.
 * With tile_x = tile_y = 0 a large FP32 grid may run in row bands of two
 * tile heights (mpdata_get_bands).
 * The fused path implements iterations 1 and 2 with the default extrema set
 * and pure precision; iterations = 3, MPDATA_EXTREMA_CORRECTED and
 * MPDATA_PREC_F64_BETA (with MPDATA_F32) need path = MPDATA_PATH_STAGES.
 * Errors: EINVAL (dims, opts, an option the chosen path lacks), ENOMEM, ECUDA. */
int mpdata_create(int nx, int ny, int nz, const mpdata_opts *opts, mpdata_t **out);

/* Free the handle and everything it owns (NULL is accepted). */
int mpdata_destroy(mpdata_t *handle);

/* The fused-kernel output tile the handle runs (the default one when
 * opts.tile_x = tile_y = 0), written to *tile_x and *tile_y; 0 x 0 for the
 * stage path.  Errors: EINVAL (NULL argument). */
int mpdata_get_tile(const mpdata_t *handle, int *tile_x, int *tile_y);

/* Row bands of a default-tile handle (FP32, fused, iterations 2, nx % 4 == 0,
 * when the tile model predicts them faster): each step
 * runs rows [0, 28 * n28) in 32x28 tiles and the rest in n24 bands of 32x24
 * tiles (the last may end past ny), as two launches that run concurrently
 * (a stream and two events owned by the handle fork from and join back into
 * the caller's stream), so the SMs take tiles of both heights and no band is
 * left mostly empty.  Results are bit-identical to a single tile shape.
 * *n28 = *n24 = 0 when the handle runs one tile shape (mpdata_get_tile).
 * Errors: EINVAL (NULL argument). */
int mpdata_get_bands(const mpdata_t *handle, int *n28, int *n24);

/* The row-band plan mpdata_create would take for an FP32 nx x ny x nz grid
 * with the default tile on a device of nsm SMs (host only, no device call):
 * *n28, *n24 as in mpdata_get_bands, 0 and 0 for one tile shape.  Plans are
 * considered for grids with nx % 4 == 0 and at most 48 waves of tiles.  Errors: EINVAL (NULL argument, dims < 1, nsm < 0). */
int mpdata_plan_bands(int nx, int ny, int nz, const int *periodic, int nsm, int *n28, int *n24);

/* The fused-kernel tile mpdata_create takes for an nx x ny x nz grid of dtype
 * with tile_x = tile_y = 0 on a device of nsm SMs (host only, no device
 * call; nsm = 0: a device of unknown size, every grid one wave): the tile of
 * least predicted step time, ceil(tiles / (nsm x CTAs per SM)) waves x the
 * tile's per-plane time measured on GB300 (one-wave time while the tiles do
 * not outnumber the SMs).  The boundaries do not enter the choice.  Errors:
 * EINVAL (NULL argument, dims < 1, nsm < 0, unknown dtype). */
int mpdata_default_tile(int nx, int ny, int nz, int dtype, int nsm, int *tile_x, int *tile_y);

/* Advance psi by nsteps MPDATA steps in place (async on `stream`): each
 * step reads the five fields and writes psi (§5.2); a run is a loop of such
 * steps (§6 times 40 of them).
 * h, u1, u2, u3, psi: device pointers to nx*ny*nz elements of the handle's
 * dtype; psi is read and overwritten, the others only read.  Step s reads
 * one buffer and writes the other of the pair (psi, handle scratch); when
 * nsteps is odd one extra device copy of psi is made first so that the
 * result lands in psi.  nsteps == 0 does nothing.
 * Errors: EINVAL (null/misaligned pointer, nsteps < 0), ECUDA (launch). */
int mpdata_step(mpdata_t *handle, const void *h, void *psi, const void *u1, const void *u2,
                const void *u3, int nsteps, void *stream);

/* Same as mpdata_step (§5.2) on HOST arrays: copies h, psi, u1, u2, u3 to device
 * buffers owned by the handle (allocated on first use), runs nsteps steps
 * and copies psi back, then waits for the stream.  Returns when psi holds
 * the result.  Errors: EINVAL, ENOMEM, ECUDA. */
int mpdata_solve_host(mpdata_t *handle, const void *h, void *psi, const void *u1,
                      const void *u2, const void *u3, int nsteps, void *stream);

/* Pipelined solves on HOST arrays: the §5.2 step loop of mpdata_solve_host
 * for a sequence of independent problems (one problem after another through
 * one device, each on its own fields), with the copies of one solve
 * overlapping the steps of its neighbours.  Enqueues without blocking the
 * host: the copy of h, psi_in, u1, u2, u3 into one of two device slots owned
 * by the handle (on a copy-in stream of the handle), nsteps steps of that slot
 * on `stream`, and the copy of the result to psi_out (on a copy-out stream of
 * the handle).  Consecutive submits alternate slots; the steps of all solves
 * run in submit order on `stream`; the copy into a slot waits until the solve
 * that used the slot two submits earlier has been copied out.
 * Host arrays: nx*ny*nz elements of the handle's dtype.  Page-locked memory
 * (cudaHostAlloc, cudaHostRegister, torch pin_memory) is needed for the
 * copies to overlap; pageable memory gives correct results but the copies
 * then block the host.  Ownership: the caller keeps all six arrays valid,
 * the five inputs unmodified and psi_out unread and unwritten, until
 * mpdata_host_wait on this solve's ticket (or a later one) has returned.
 * psi_out may be psi_in of the same submit.  Solves in flight may share
 * input arrays; psi_out must not overlap an input of another solve in
 * flight, and when several solves in flight write the same psi_out the
 * latest submit's result is what remains (the copies out run in submit
 * order).
 * *ticket receives the solve's id: 1 for the handle's first submit, then
 * increasing by one.
 * Errors: EINVAL (null argument, nsteps < 0), ENOMEM, ECUDA. */
int mpdata_host_submit(mpdata_t *handle, const void *h, const void *psi_in, const void *u1,
                       const void *u2, const void *u3, int nsteps, void *psi_out, void *stream,
                       unsigned long long *ticket);

/* Block the calling thread until solve `ticket` of this handle has written
 * psi_out; every earlier solve has then finished too (the copies out run in
 * submit order).  A ticket that has already been waited for returns at once.
 * Errors: ENOENT (ticket 0 or not yet issued), ECUDA (a copy or a step of
 * this or an earlier solve failed). */
int mpdata_host_wait(mpdata_t *handle, unsigned long long ticket);

/* Diagnostics (async; the paper defines none: sum h*psi is the quantity the
 * flux form of the §5.2 scheme conserves): out3[0] = sum of h*psi over all cells, out3[1] =
 * min psi, out3[2] = max psi, written as three doubles to the DEVICE
 * pointer out3.  The sum is taken in FP64 with a fixed reduction tree (no
 * atomics on values), so it is bit-reproducible run to run.
 * Errors: EINVAL, ECUDA. */
int mpdata_mass(mpdata_t *handle, const void *h, const void *psi, void *out3, void *stream);

/* Stability check (async): the largest outflow Courant number over all
 * cells, max_c sum_d ([U_d(c + e_d)]+ - [U_d(c)]-) / h_c, with the handle's
 * boundary conditions (lid faces carry no velocity).  The donor-cell pass
 * keeps psi >= 0 -- and the scheme is stable -- only while it is <= 1; the
 * library does not check it on every step, the caller does.  Written as
 * three doubles to the DEVICE pointer out3: out3[1] = out3[2] = the maximum
 * (out3[0] = 0), computed in FP64 with a fixed reduction tree.
 * h, u1, u2, u3: device pointers (16-byte aligned) of the handle's dtype.
 * Errors: EINVAL, ECUDA. */
int mpdata_courant_max(mpdata_t *handle, const void *h, const void *u1, const void *u2,
                       const void *u3, void *out3, void *stream);

/* mpdata_mass without a handle and without any device allocation, for
 * callers that cannot allocate device memory themselves: code embedded in a
 * host framework whose allocator owns all device memory and forbids raw
 * cudaMalloc, services that budget every allocation up front, and loops
 * that cannot afford the implicit synchronisation of cudaMalloc/cudaFree.
 * (The paper has no counterpart; this is a library-integration entry point.)
 *
 * Computes the same three doubles as mpdata_mass (sum h*psi in FP64 with the
 * same fixed reduction tree, min psi, max psi) over n elements of dtype
 * (MPDATA_F32 or MPDATA_F64) into the DEVICE pointer out3, async on stream.
 * h and psi are device pointers (16-byte aligned), out3 is 8-byte aligned;
 * the caller still provides all inputs and outputs.
 *
 * Scratch: the reduction partials live in a fixed static device array of
 * 3 x 1024 doubles (24 KiB) inside the library, held by every GPU that
 * loads it until the process exits; no cudaMalloc, cudaFree or other
 * allocating call is made.  Limit: n must be in [1, 2^31 - 1] (EINVAL
 * otherwise).  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  The address is cached per device ordinal
 * and belongs to that device's primary context (the one the CUDA runtime
 * uses): it does not survive cudaDeviceReset, and a caller that makes a
 * different driver context current on the same device must not use this
 * entry point from it.  All calls share the one array and every
 * call overwrites all partials it reads, so nothing has to start at zero --
 * but calls whose kernels overlap on the GPU (other streams, other threads)
 * race on it and must be serialised by the caller.
 * Errors: EINVAL, ECUDA. */
int mpdata_mass_noalloc(const void *h, const void *psi, long long n, int dtype, void *out3,
                        void *stream);

/* ---- batches: many independent grids advanced by batched launches ----
 *
 * The paper's team decomposition (§5.3) assigns sub-domains to groups of
 * cores; here every grid of the batch is cut into the same tiles as a
 * single-grid launch, the tiles of all grids form a work-item list ordered by
 * decreasing estimated cost (tile area x (nz + 3)), and a launch runs the
 * list with CTA c taking the contiguous items [begin[c], begin[c+1]).  The
 * default split gives every item its own CTA (the hardware starts the largest
 * tiles first and hands each free SM the next one).  mpdata_batch_set_split
 * installs any other: the balanced persistent split (one CTA per SM,
 * contiguous ranges of nearly equal cost) or the uneven splits of the
 * speed-function partitioner (Algorithm 1, §4), whose processors are
 * persistent CTAs.  Each grid has its own tile shape (32x24, 32x16 or
 * 32x28) and runs the kernel a single-grid launch with that tile runs:
 * variant 0 (tile 32x24, x and y periodic, nx % 4 != 0), 1 (32x24, a lid on
 * x or y, nx % 4 != 0), 2 (32x24 with loader warps, periodic, nx % 4 == 0),
 * 7 (32x24 with loader warps, lid, nx % 4 == 0), 3 (32x16, periodic), 4
 * (32x16, lid), 5 (32x28, periodic, nx % 4 != 0), 6 (32x28, lid,
 * nx % 4 != 0), 8 (32x28 with loader warps, periodic, nx % 4 == 0), 9 (32x28
 * with loader warps, lid, nx % 4 == 0).  One launch per
 * non-empty variant and step.  FP32, iterations = 2 only.  Each
 * grid's result is bit-identical to mpdata_step on that grid alone with the
 * same tile. */
typedef struct mpdata_batch mpdata_batch_t;

/* dims: 3*ngrids ints (nx, ny, nz of each grid); periodic: 3*ngrids flags or
 * NULL for opts->periodic on every grid; opts: NULL for defaults (dtype must
 * be MPDATA_F32; tile 32x24 (default), 32x16 or 32x28).  Allocates one psi-sized
 * scratch buffer per grid.  Errors: EINVAL, ENOMEM, ECUDA. */
int mpdata_batch_create(int ngrids, const int *dims, const int *periodic, const mpdata_opts *opts,
                        mpdata_batch_t **out);
/* mpdata_batch_create with a tile height per grid: tile_y[i] is 16, 24, 28, or 0
 * for the batch default (opts->tile_y); tile_y may be NULL (all default). */
int mpdata_batch_create_tiles(int ngrids, const int *dims, const int *periodic, const int *tile_y,
                              const mpdata_opts *opts, mpdata_batch_t **out);
/* The variant (0 .. 9, see above) that runs grid `grid`. */
int mpdata_batch_grid_variant(mpdata_batch_t *batch, int grid, int *variant);
/* Device pointers (16-byte aligned) of grid `grid`; psi is advanced in
 * place.  Must be set for every grid before the first step. */
int mpdata_batch_set_fields(mpdata_batch_t *batch, int grid, const void *h, void *psi,
                            const void *u1, const void *u2, const void *u3);
/* Number of work items and CTAs of a variant (0 .. 9). */
int mpdata_batch_work(mpdata_batch_t *batch, int variant, int *nitems, int *ncta);
/* Copy the current split of a variant (ncta + 1 ints) into begin. */
int mpdata_batch_get_split(mpdata_batch_t *batch, int variant, int *begin);
/* Install a split: ncta CTAs, begin[0] = 0, begin[ncta] = nitems,
 * nondecreasing (a CTA may get no item).  begin == NULL installs the balanced
 * split over min(ncta, nitems) CTAs: CTA c's last item is the one whose
 * cumulative cost is closest to (c+1)/ncta of the total. */
int mpdata_batch_set_split(mpdata_batch_t *batch, int variant, int ncta, const int *begin);
/* nsteps steps of every grid (async on stream; with several non-empty
 * variants each variant's launches run on a stream of the batch that forks
 * from and joins back into `stream`).  use_graph != 0 captures the
 * whole sequence once per nsteps into a CUDA graph and replays it (the graph
 * is rebuilt after set_fields or set_split).  Odd nsteps copies each psi to
 * its scratch first so that the result lands in psi. */
int mpdata_batch_step(mpdata_batch_t *batch, int nsteps, int use_graph, void *stream);
int mpdata_batch_destroy(mpdata_batch_t *batch);

/* ---- serving: continuous batching of advection solves ----
 * (No counterpart in the paper: a front end that runs many independent
 * solves of the §5.2 step on one GPU.)
 *
 * A server owns a scheduler thread and three CUDA streams on the device
 * current at creation: one for the ticks, one for copies in, one for copies
 * out.  Requests (host fields, FP32) are admitted first-in first-out while
 * their device footprint (6 fields: h, psi, psi scratch, u1, u2, u3) fits
 * the HBM budget and fewer than max_active are resident.  An admitted
 * request's fields are copied in on the copy-in stream while the ticks of the
 * requests already resident go on; it joins the ticks once its copy has
 * landed.  Every tick advances all resident requests by the same chunk of
 * steps in one batched launch per kernel variant (see mpdata_batch_*), so
 * requests that arrive while others run join a later tick and share the GPU.
 * A finished request's psi is copied back into its host buffer on the
 * copy-out stream (after the tick that finished it, without holding up the
 * next one), then its memory and budget are released.  Each result is
 * bit-identical to mpdata_step on that grid alone with tile 32 x tile_y.
 * Host buffers must stay valid until the request finishes; pinned memory
 * keeps the scheduler from blocking on copies.
 *
 * Tickets: a finished request (DONE, FAILED or CANCELLED) stays known to
 * mpdata_poll, mpdata_wait and mpdata_request_times until mpdata_release is
 * called on it, or until more than retain_finished requests that finished
 * later are still held, whichever comes first; after that its ticket gives
 * ENOENT.  A request that a thread is waiting on is not retired until that
 * wait returns.  So a server that runs indefinitely holds at most
 * retain_finished finished requests (plus those queued or resident).
 *
 * All entry points are thread-safe.  mpdata_server_destroy may be called
 * while other threads are blocked in mpdata_wait: they return (ECANCELED for
 * requests it cancelled) before it frees anything.  No thread may start a
 * call on the server once mpdata_server_destroy has been called. */
#define MPDATA_REQ_QUEUED 0    /* waiting for budget or a slot */
#define MPDATA_REQ_RUNNING 1   /* resident on the device */
#define MPDATA_REQ_DONE 2      /* psi holds the result */
#define MPDATA_REQ_FAILED 3    /* see mpdata_wait's return code */
#define MPDATA_REQ_CANCELLED 4

typedef struct mpdata_server_opts {
    uint32_t size;              /* sizeof(mpdata_server_opts) */
    size_t hbm_budget_bytes;    /* device memory the server may hold (default 8 GiB) */
    int32_t max_active;         /* resident requests at most (default 256) */
    int32_t max_queued;         /* requests waiting for memory; a submit beyond this that
                                   cannot be covered by the budget gets EBUSY (default 2^20;
                                   0 = reserve budget at submit, refuse when over) */
    int32_t chunk_steps;        /* steps per tick (default 8) */
    int32_t tile_y;             /* 24 (default) or 16 for the two-column kernel */
    int32_t nonoscillatory;     /* default 1 */
    int32_t inject_alloc_failure; /* test hook: every n-th admission fails as out of memory (0 = off) */
    double eps;                 /* default 1e-15 */
    int32_t retain_finished;    /* finished requests kept queryable before the oldest are
                                   retired (default 65536; 0 = retire each one as soon as it
                                   has finished and nobody waits on it) */
} mpdata_server_opts;

typedef struct mpdata_request {
    uint32_t size;              /* sizeof(mpdata_request) */
    int32_t nx, ny, nz;
    int32_t periodic[3];
    int32_t nsteps;             /* >= 0 */
    const void *h, *u1, *u2, *u3; /* host float32 [nz][ny][nx] */
    void *psi;                  /* host float32: initial state in, result out */
} mpdata_request;

typedef struct mpdata_server mpdata_server_t;

void mpdata_server_opts_default(mpdata_server_opts *opts);
/* Errors: EINVAL (options), ENOMEM, ECUDA. */
int mpdata_server_create(const mpdata_server_opts *opts, mpdata_server_t **out);
/* Queue a request; *ticket identifies it.  Errors: EINVAL (bad request, or
 * larger than the whole budget), EBUSY (queue full and over budget). */
int mpdata_submit(mpdata_server_t *server, const mpdata_request *req, uint64_t *ticket);
/* Non-blocking state (MPDATA_REQ_*).  ENOENT for an unknown ticket. */
int mpdata_poll(mpdata_server_t *server, uint64_t ticket, int *state);
/* Block until the request finishes or timeout_ms passes (< 0: no limit).
 * Returns OK (done), ETIMEDOUT, ECANCELED, ENOENT, or the failure code
 * (ENOMEM when admission could not allocate, ECUDA). */
int mpdata_wait(mpdata_server_t *server, uint64_t ticket, int timeout_ms);
/* Cancel a queued or running request (takes effect at the next tick). */
int mpdata_cancel(mpdata_server_t *server, uint64_t ticket);
/* Submit, admit and finish times of a request, seconds since server start. */
int mpdata_request_times(mpdata_server_t *server, uint64_t ticket, double *t3);
/* Forget a finished request: its ticket gives ENOENT from now on.  Errors:
 * ENOENT (unknown or already retired), EBUSY (not finished yet, or a thread
 * is waiting on it). */
int mpdata_release(mpdata_server_t *server, uint64_t ticket);
/* *count = requests the server holds: queued, resident, being copied out,
 * and finished ones not yet released or retired. */
int mpdata_server_retained(mpdata_server_t *server, uint64_t *count);
/* stats[0..5]: completed, cell-steps done, admitted bytes, queued, resident,
 * seconds since start. */
int mpdata_server_stats(mpdata_server_t *server, double *stats);
/* Cancel queued and resident work, stop the scheduler, release the threads
 * blocked in mpdata_wait, free everything. */
int mpdata_server_destroy(mpdata_server_t *server);

/* ---- functional-performance-model partitioning (§2-§4) ----
 * A speed function is a table of npts measured points (xs[i], ss[i]), sizes
 * increasing, speeds > 0 (work units per second of one processor running a
 * workload of size xs[i] while all processors run); it is linearly
 * interpolated and never extrapolated.  Execution time of x is x / s(x). */

/* Algorithm 1 (§4) as printed: n units over an even number p of identical
 * processors, each a multiple of dx (n/p must be one); p/2 processors take
 * *x_left and p/2 take *x_right, minimising the larger execution time
 * *t_min.  The loop bound is read as "while x_left - dx > 0".
 * Errors: EINVAL. */
int mpdata_fpm_algorithm1(double n, int p, double dx, const double *xs, const double *ss, int npts,
                          double *x_left, double *x_right, double *t_min);
/* Generalisation to any p: *k_right processors take *x_right >= n/p and the
 * other p - k_right take *x_left = (n - k x_right)/(p - k), both multiples of
 * dx; k_right = 0 means the balanced split n/p.  Errors: EINVAL (including
 * "no split fits the table"). */
int mpdata_fpm_partition(double n, int p, double dx, const double *xs, const double *ss, int npts,
                         int *k_right, double *x_left, double *x_right, double *t_min);
/* Condition (2) of §3 on a table: returns 1 (and the two sizes) if some
 * larger workload has a higher speed-to-size ratio -- load balancing is then
 * not guaranteed optimal -- 0 if condition (1) holds on the table, < 0 on
 * error. */
int mpdata_fpm_condition2(const double *xs, const double *ss, int npts, double *x_at, double *x_more);

/* Name of an error code. */
const char *mpdata_strerror(int code);

/* Detail of the calling thread's last failure ("" if none). */
const char *mpdata_last_error_message(void);

/* Library version string. */
const char *mpdata_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MPDATA_H */
