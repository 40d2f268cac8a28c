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
 * failure.  A handle is used by one host thread at a time.
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

typedef struct mpdata_opts {
    uint32_t size;          /* sizeof(mpdata_opts); set by mpdata_opts_default */
    int32_t iterations;     /* 1: donor cell only; 2: one corrective pass (default) */
    int32_t nonoscillatory; /* 1: limit the antidiffusive velocities (default) */
    int32_t periodic[3];    /* per axis x, y, z: 1 periodic (default), 0 rigid lid */
    int32_t dtype;          /* MPDATA_F32 (default) or MPDATA_F64 */
    int32_t path;           /* MPDATA_PATH_FUSED (default) or MPDATA_PATH_STAGES */
    int32_t tile_x, tile_y; /* fused-kernel output tile; 0 picks the default */
    double eps;             /* > 0, added to every A, B and limiter denominator; default 1e-15 */
} mpdata_opts;

typedef struct mpdata_handle mpdata_t;

/* Fill *opts with the defaults listed above. */
void mpdata_opts_default(mpdata_opts *opts);

/* Create a solver for an nx x ny x nz grid (each >= 1) on the current CUDA
 * device.  The handle owns one psi-sized device scratch buffer (the step's
 * ping-pong partner) and, for the stage-per-kernel path, the intermediate
 * arrays; they are allocated here and freed by mpdata_destroy.
 * Errors: EINVAL (dims, opts), ENOMEM, ECUDA. */
int mpdata_create(int nx, int ny, int nz, const mpdata_opts *opts, mpdata_t **out);

/* Free the handle and everything it owns (NULL is accepted). */
int mpdata_destroy(mpdata_t *handle);

/* Advance psi by nsteps MPDATA steps in place (async on `stream`).
 * h, u1, u2, u3, psi: device pointers to nx*ny*nz elements of the handle's
 * dtype; psi is read and overwritten, the others only read.  Step s reads
 * one buffer and writes the other of the pair (psi, handle scratch); when
 * nsteps is odd one extra device copy of psi is made first so that the
 * result lands in psi.  nsteps == 0 does nothing.
 * Errors: EINVAL (null/misaligned pointer, nsteps < 0), ECUDA (launch). */
int mpdata_step(mpdata_t *handle, const void *h, void *psi, const void *u1, const void *u2,
                const void *u3, int nsteps, void *stream);

/* Same as mpdata_step on HOST arrays: copies h, psi, u1, u2, u3 to device
 * buffers owned by the handle (allocated on first use), runs nsteps steps
 * and copies psi back, then waits for the stream.  Returns when psi holds
 * the result.  Errors: EINVAL, ENOMEM, ECUDA. */
int mpdata_solve_host(mpdata_t *handle, const void *h, void *psi, const void *u1,
                      const void *u2, const void *u3, int nsteps, void *stream);

/* Diagnostics (async): out3[0] = sum of h*psi over all cells, out3[1] =
 * min psi, out3[2] = max psi, written as three doubles to the DEVICE
 * pointer out3.  The sum is taken in FP64 with a fixed reduction tree (no
 * atomics on values), so it is bit-reproducible run to run.
 * Errors: EINVAL, ECUDA. */
int mpdata_mass(mpdata_t *handle, const void *h, const void *psi, void *out3, void *stream);

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
 * call before any stream capture.  All calls share the one array and every
 * call overwrites all partials it reads, so nothing has to start at zero --
 * but calls whose kernels overlap on the GPU (other streams, other threads)
 * race on it and must be serialised by the caller.
 * Errors: EINVAL, ECUDA. */
int mpdata_mass_noalloc(const void *h, const void *psi, long long n, int dtype, void *out3,
                        void *stream);

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
