/*
 * fish.h -- C ABI of libfish.so: FISH's operator-split ideal-MHD sweep on one
 * GB300 GPU (Kaeppeli et al., "FISH: A 3D parallel MHD code for astrophysical
 * applications", arXiv:0910.2854).
 *
 * Problem statement (Sec. 2): a box of nx*ny*nz Cartesian cells of widths
 * dx, dy, dz; ideal gas of ratio of specific heats gamma (eq0050); cell
 * averages u = (rho, rho v, E) (eq0070) and face averages of the magnetic
 * field b = B/sqrt(4 pi) (eq0080-eq0080b); optional fixed gravitational
 * potential phi (Sec. 2.3, "given and constant in time"); periodic or
 * zeroth-order-extrapolation boundaries (Sec. 4).
 *
 * State layout (host and device): 8 fields of nx*ny*nz values each, one
 * after the other, x fastest, index i + nx*(j + ny*k):
 *   rho, m_x, m_y, m_z, E, b_x, b_y, b_z
 * where b_x[i,j,k] is the average over the face at x_{i+1/2} (likewise b_y at
 * y_{j+1/2}, b_z at z_{k+1/2}).  With outflow boundaries the faces at
 * x_{-1/2}, y_{-1/2}, z_{-1/2} are ghosts (copies of the faces at +1/2).
 *
 * Conventions:
 *  - Every call returns FISH_OK (0) or a FISH_ERR_* code; no exception or
 *    exit crosses the ABI.  fish_last_error() gives a text for the last error.
 *  - Caller-owned buffers are only read from or written to during the call;
 *    the library owns all device memory it allocates and frees it in
 *    fish_destroy().
 *  - Work is queued asynchronously on the context's stream.  Device-side
 *    errors (rho <= 0, p <= 0, NaN: reading C-16 -- no floor is applied) are
 *    sticky per context and returned as FISH_ERR_NONPHYSICAL by the next
 *    synchronising call (fish_cfl_dt, fish_get_state*, fish_diagnostics,
 *    fish_sync, fish_last_dt).
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef FISH_H
#define FISH_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fish_ctx fish_ctx;

enum {
    FISH_OK = 0,
    FISH_ERR_ARG = 1,          /* invalid argument (sizes, keys, values, NULL) */
    FISH_ERR_CUDA = 2,         /* CUDA runtime error (text in fish_last_error) */
    FISH_ERR_OOM = 3,          /* device allocation failed */
    FISH_ERR_STATE = 4,        /* call out of order (e.g. step before set_state) */
    FISH_ERR_NONPHYSICAL = 5,  /* rho <= 0, p <= 0 or NaN met on the device */
    FISH_ERR_TIMEOUT = 6       /* a bounded device-side wait gave up */
};

enum { FISH_BC_PERIODIC = 0, FISH_BC_OUTFLOW = 1 };

/* option keys for fish_set_option */
enum {
    FISH_OPT_PRECISION = 0,  /* FISH_PREC_FP64 (default) or FISH_PREC_FP32 */
    FISH_OPT_LIMITER = 1,    /* FISH_LIM_VANLEER (default, eq0200), FISH_LIM_MINMOD (eq0190),
                                FISH_LIM_NONE (first order, eq0140), FISH_LIM_HYBRID (Sec. 2.2:
                                minmod at interfaces where either cell has |v_d| > c_S, Van
                                Leer elsewhere; the constrained transport keeps Van Leer) */
    FISH_OPT_HSE = 2,        /* 1: hydrostatic-gradient correction, eq0321-eq03261 */
    FISH_OPT_PRED_DISS = 3,  /* predictor freezing-speed factor in [0,1] (Sec. 2.2); default 1 */
    FISH_OPT_DX = 4,         /* cell widths; default 1/nx, 1/ny, 1/nz */
    FISH_OPT_DY = 5,
    FISH_OPT_DZ = 6,
    FISH_OPT_GRAVITY = 7,    /* FISH_GRAV_UNSPLIT (default): potential source terms inside L_d
                                (eq0253-eq0255); FISH_GRAV_SPLIT: L_d becomes G_d(dt/2) L_d G_d(dt/2)
                                with G_d: m_d -= (dt/2) rho dphi/dx_d (centred difference) and E
                                changed by the kinetic energy change (eq025111-eq02513).  Split
                                gravity and FISH_OPT_HSE = 1 exclude each other (FISH_ERR_ARG).
                                The kicks run inside the fluid sweep (separate passes on an
                                irregular mesh). */
    FISH_OPT_KERNELS = 8     /* kernel family of the FP32 fluid sweep (results are bitwise the
                                same): FISH_KERNELS_COLUMN (default) the register-prefetch column
                                march; FISH_KERNELS_RING the march fed through a shared-memory
                                ring of TMA bulk copies (boxes whose fast extents are multiples of
                                four, no potential, uniform mesh; elsewhere the column march).
                                The ring is measured slower on GB300 and kept as an option. */
};
enum { FISH_KERNELS_COLUMN = 0, FISH_KERNELS_RING = 1 };
enum { FISH_GRAV_UNSPLIT = 0, FISH_GRAV_SPLIT = 1 };
enum { FISH_PREC_FP64 = 0, FISH_PREC_FP32 = 1 };
enum { FISH_LIM_VANLEER = 0, FISH_LIM_MINMOD = 1, FISH_LIM_NONE = 2, FISH_LIM_HYBRID = 3 };

/* dtype codes of device buffers */
enum { FISH_F64 = 0, FISH_F32 = 1 };

/* operators for fish_apply */
enum { FISH_OP_FLUID = 0, FISH_OP_CT = 1 };

/* Create a context for an nx*ny*nz box (each >= 1) with ratio of specific
 * heats gamma > 1 and boundary condition bc.  No device memory is allocated
 * until the first fish_set_state*.  *out receives the handle. */
int fish_create(int nx, int ny, int nz, double gamma, int bc, fish_ctx **out);

/* Set an option (keys above).  PRECISION may only change before the first
 * fish_set_state*; the others may change between steps.  FISH_ERR_ARG for an
 * unknown key or a value out of range. */
int fish_set_option(fish_ctx *ctx, int key, double value);

/* Queue all further work on this CUDA stream (a cudaStream_t, e.g. PyTorch's
 * current stream); NULL selects the context's own non-blocking stream. */
int fish_set_stream(fish_ctx *ctx, void *cuda_stream);

/* Route the context's device allocations through a caller allocator (e.g.
 * PyTorch's caching allocator): alloc(size, user) returns a device pointer or
 * NULL, free(ptr, user) releases it.  Must be called before the first
 * fish_set_state*.  NULL alloc restores cudaMalloc/cudaFree. */
int fish_set_allocator(fish_ctx *ctx, void *(*alloc)(size_t size, void *user),
                       void (*free_fn)(void *ptr, void *user), void *user);

/* Upload the state from a host buffer of 8*nx*ny*nz doubles (layout above).
 * Allocates device memory on first use.  Synchronous with respect to the
 * host buffer (it may be reused on return). */
int fish_set_state(fish_ctx *ctx, const double *state);

/* Same from a device buffer of 8*nx*ny*nz values of dtype FISH_F64 or
 * FISH_F32 (converted to the context precision).  Queued on the stream. */
int fish_set_state_device(fish_ctx *ctx, const void *state, int dtype);

/* Same from a host buffer of dtype FISH_F64 or FISH_F32 (pinned host memory
 * gives full copy bandwidth).  Returns once the buffer has been read. */
int fish_set_state_host(fish_ctx *ctx, const void *state, int dtype);

/* Fixed cell-centred potential phi (nx*ny*nz doubles, host) for the unsplit
 * gravity source (eq0253-eq0255) or the split operator of FISH_OPT_GRAVITY;
 * NULL removes gravity. */
int fish_set_potential(fish_ctx *ctx, const double *phi);

/* Irregular Cartesian mesh (Sec. 2.5, eq037, eq0420): host arrays of nx, ny,
 * nz cell widths (each finite and > 0; copied, the caller keeps ownership).
 * A NULL axis keeps the width of FISH_OPT_DX/DY/DZ for all its cells; all
 * three NULL restores the uniform mesh.  With a mesh set, every update uses
 * the width of the cell it changes, the TVD slopes are per unit length over
 * the centre distances, potential differences are taken over the centre
 * span, CT face and edge velocities are linear interpolations, the CFL step
 * follows eq0420 and fish_diagnostics weights each cell by its own volume.
 * Ghost cells have the width of the cell they copy.  No CFL is fused into
 * the last sweep (a separate CFL pass reads the widths).
 * Widths are uploaded at the next stepping call.  FISH_ERR_ARG on a bad
 * width. */
int fish_set_mesh(fish_ctx *ctx, const double *dx, const double *dy, const double *dz);

/* CFL time step dt = k * min over cells and axes d of h_d / (|v_d| + c_F,d)
 * (eq0083-eq0084, reading C-15) for the current state.  Synchronises. */
int fish_cfl_dt(fish_ctx *ctx, double k, double *dt_out);

/* The same over the z-planes k0 .. k0+nk-1 only (a z-slab of a box split
 * over several GPUs, whose ghost planes stay out of the minimum; the slab's
 * time step is then the minimum over all slabs).  FISH_ERR_ARG for a range
 * outside [0, nz). */
int fish_cfl_dt_planes(fish_ctx *ctx, double k, int k0, int nk, double *dt_out);

/* One full double step u^{n+2} = L_fwd L_bwd u^n (eq0081-eq0082, reading
 * C-4): L_x B_x L_y B_y L_z B_z B_z L_z B_y L_y B_x L_x, every operator with
 * the full dt, so time advances by 2*dt.  Asynchronous. */
int fish_step(fish_ctx *ctx, double dt);

/* nsteps double steps, each with dt = k * CFL of the state at its start,
 * computed on the device (no host round trip); replayed as one CUDA graph
 * per call after the first.  Asynchronous; fish_last_dt reads the last dt. */
int fish_step_cfl(fish_ctx *ctx, double k, int nsteps);

/* dt used by the last step of fish_step / fish_step_cfl.  Synchronises. */
int fish_last_dt(fish_ctx *ctx, double *dt_out);

/* Apply one operator -- FISH_OP_FLUID (L_dir) or FISH_OP_CT (B_dir) -- along
 * axis dir (0 = x, 1 = y, 2 = z) with time step dt.  Asynchronous. */
int fish_apply(fish_ctx *ctx, int op, int dir, double dt);

/* Download the state to a host buffer of 8*nx*ny*nz doubles.  Synchronises. */
int fish_get_state(fish_ctx *ctx, double *state);

/* Download the state to a host buffer of dtype FISH_F64 or FISH_F32 (same
 * layout; pinned host memory gives full copy bandwidth), converting on the
 * device where the context precision differs.  Synchronises and returns
 * pending device errors, like fish_get_state. */
int fish_get_state_host(fish_ctx *ctx, void *state, int dtype);

/* Copy the state into a device buffer of dtype FISH_F64 / FISH_F32.  Queued
 * on the stream; returns pending device errors only after fish_sync. */
int fish_get_state_device(fish_ctx *ctx, void *state, int dtype);

/* Copy the z-planes k0 .. k0+nk-1 of all 8 fields to (get) or from (set) a
 * buffer of 8*nk*nx*ny values in the context's precision, field after field,
 * each field's nk planes contiguous, every plane in the context's current
 * memory layout (x fastest, or y fastest while an x sweep pair is active; a
 * z-plane is contiguous in both).  The buffer may be host or device memory
 * (pinned host memory for full bandwidth).  Queued on the stream; the
 * caller synchronises before reading or reusing the buffer.  Used to
 * exchange ghost slabs between the z-slabs of a box split over several
 * GPUs (the paper's cuboid decomposition, Sec. 3).  FISH_ERR_ARG for a range
 * outside [0, nz) or a NULL buffer. */
int fish_get_planes(fish_ctx *ctx, int k0, int nk, void *dst);
int fish_set_planes(fish_ctx *ctx, int k0, int nk, const void *src);

/* out[0..7] = volume-weighted totals of the 8 fields (FP64 accumulation in a
 * fixed order); out[8] = max |div b| (eq0341) over cells whose six faces are
 * stored.  Synchronises. */
int fish_diagnostics(fish_ctx *ctx, double out[9]);

/* Wait for queued work; returns sticky device errors. */
int fish_sync(fish_ctx *ctx);

/* Clear the sticky device error flags (after the caller has handled them). */
int fish_clear_error(fish_ctx *ctx);

/* Text of the last error of this context (never NULL; "" if none). */
const char *fish_last_error(fish_ctx *ctx);

/* Number of kernel launches queued by this context since creation. */
long long fish_launch_count(fish_ctx *ctx);

/* Measurement helper with no counterpart in the paper: the FP64 pipe
 * throughput of the current device in fused multiply-adds per second
 * (each thread of sms x 8 blocks of 256 runs eight independent FMA chains;
 * three timed launches after one warm-up).  It is the peak the FP64 sweeps
 * are compared against, since GB300's FP64 rate is far below its bandwidth.
 * Allocates and frees its own scratch; synchronous.  FISH_ERR_ARG on a NULL
 * output, FISH_ERR_CUDA if any CUDA call fails (*fma_per_s is then 0). */
int fish_probe_fp64_fma(double *fma_per_s);

/* ---- batches of independent boxes (FP32) ---------------------------------
 * Many boxes of uneven sizes advanced together: every sweep of every box is
 * one persistent launch over a device work queue, each box keeps its own CFL
 * time step on the device, and the double step of the whole batch is one
 * CUDA graph.  Each box follows exactly the single-box FP32 path (eq0081-
 * eq0084 with the operators of Sec. 2): its result equals that of a fish_ctx
 * of the same box stepped with fish_step_cfl.  The state layout of a box is
 * the one above.  Every box needs even nx and ny (the x and y columns are
 * advanced in pairs); all boxes together hold at most 2^31 - 2^20 cells
 * (FISH_ERR_ARG beyond). */
typedef struct fish_batch fish_batch;

/* batch option keys (fish_batch_set_option) */
enum {
    FISH_BATCH_OPT_LIMITER = 0, /* FISH_LIM_VANLEER (default) or FISH_LIM_MINMOD */
    FISH_BATCH_OPT_ORDER = 1,   /* work-item order: 0 box order, 1 longest first, 2 round robin */
    FISH_BATCH_OPT_GROUPS = 2,  /* column groups (128 threads) per work item: 1, 2, 4, 8 */
    FISH_BATCH_OPT_GRID = 3,    /* persistent grid = SMs x resident blocks x (1, 2 or 4) */
    FISH_BATCH_OPT_CTROWS = 4   /* tile height of the constrained-transport sweeps: rows (warps) of
                                   31 columns per work-item group, 4 (default) or 8 */
};

/* nbox boxes: dims[3k..3k+2] = nx, ny, nz of box k, gamma[k] > 1, bc[k]
 * FISH_BC_*, h[3k..3k+2] cell widths (NULL: 1/n per axis).  Allocates the
 * device memory of all boxes (two buffers of 8 FP32 fields). */
int fish_batch_create(int nbox, const int *dims, const double *gamma, const int *bc, const double *h,
                      fish_batch **out);
int fish_batch_set_option(fish_batch *b, int key, double value);
/* queue all further work on this CUDA stream (NULL: the batch's own) */
int fish_batch_set_stream(fish_batch *b, void *cuda_stream);
/* upload box `box` from a host buffer of 8*nx*ny*nz doubles; synchronous */
int fish_batch_set_state(fish_batch *b, int box, const double *state);
/* nsteps double steps of every box, each with dt = k * CFL of that box's
 * state at the start of the step, computed on the device.  Asynchronous. */
int fish_batch_step(fish_batch *b, double k, int nsteps);
/* download box `box` into a host buffer of 8*nx*ny*nz doubles; synchronises
 * and returns FISH_ERR_NONPHYSICAL if any box met rho <= 0, p <= 0 or NaN */
int fish_batch_get_state(fish_batch *b, int box, double *state);
/* dt of the last step of every box into dt[nbox]; synchronises */
int fish_batch_last_dt(fish_batch *b, double *dt);
int fish_batch_sync(fish_batch *b);
const char *fish_batch_last_error(fish_batch *b);
long long fish_batch_launch_count(fish_batch *b);
/* total cells of all boxes */
long long fish_batch_cells(fish_batch *b);
void fish_batch_destroy(fish_batch *b);

/* Allocation-free diagnostics of a device-resident state.  The paper has no
 * counterpart: this call serves callers that cannot let a library allocate
 * device memory -- host codes that own all device memory through their own
 * pool or budget, or time loops where a cudaMalloc (which may synchronise
 * the device) is not allowed.  It needs no fish_ctx.
 *   state : device buffer of 8*nx*ny*nz values of dtype FISH_F64/FISH_F32
 *           in the state layout above (read only);
 *   bc, dx, dy, dz : boundary condition and cell widths (> 0);
 *   out   : DEVICE buffer of 9 doubles, written asynchronously on `stream`
 *           (a cudaStream_t, NULL = legacy default stream): out[0..7] the
 *           volume-weighted totals of the 8 fields, out[8] max |div b| over
 *           cells whose six faces are stored -- the quantities of
 *           fish_diagnostics, summed plane by plane in a fixed order.
 * Scratch: a fixed device array of 4096 rows of 9 doubles (288 KiB) that
 * every GPU loading the library keeps until exit; nz > 4096 is rejected
 * with FISH_ERR_ARG.  All calls share it and each call rewrites the rows it
 * uses, so calls whose kernels overlap on the GPU (unordered streams) race:
 * order them.  Every call looks up the array's device address
 * (cudaGetSymbolAddress) with the caller's device current, so a device reset
 * between calls is followed; the first call on a device may load the
 * library's device code, so make that first call before any stream capture.  Allocates nothing (no cudaMalloc, no
 * allocator callback).  Returns FISH_ERR_ARG for bad arguments and
 * FISH_ERR_CUDA if a launch fails. */
int fish_diagnostics_noalloc(const void *state, int dtype, int nx, int ny, int nz, int bc, double dx,
                             double dy, double dz, double *out, void *stream);

/* Free all device memory and the handle.  NULL is ignored. */
void fish_destroy(fish_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* FISH_H */
