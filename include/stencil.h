/*
 * stencil.h -- C ABI of the GB300 (sm_103a) library for iterated explicit 2D
 * stencil sweeps.
 *
 * The operation (paper, Sec. II-C, the Jacobi update, and Sec. II-B for the
 * Star / Box shapes of radius r):
 *
 *     u^{t+1}[i][j] = sum_{dy,dx in [-r, r]} W[dy+r][dx+r] * u~^{t}[i+dy][j+dx],
 *     t = 0 .. T-1,
 *
 * on an ny x nx grid stored row-major (i = row, j = column, j contiguous).
 * u~ extends u outside the grid: by zeros for STENCIL_BOUNDARY_ZERO (the
 * paper's fixed zero padding, Sec. IV-A) or by wrapping for
 * STENCIL_BOUNDARY_PERIODIC.  Every one of the ny*nx points is updated at every
 * step; the zero halo is never updated.  W is a (2r+1)x(2r+1) row-major FP32
 * array; entries off the footprint are 0.  The sum is a cross-correlation
 * (no kernel flip).  All arithmetic is FP32 (FMA); the storage type of the
 * grid in device memory may be FP32, BF16 or FP16 (rounded to nearest even on
 * every store to device memory).
 *
 * Conventions for every entry point:
 *   - Grid pointers are DEVICE pointers unless the name says _host.  The
 *     caller owns them.  Rows are dense (row pitch = nx elements).
 *   - Weights are HOST pointers and are copied; the caller may free them on return.
 *   - Work is enqueued on `stream` (NULL = legacy default stream) and the call
 *     returns without synchronising, except where stated.
 *   - Errors: argument errors are reported synchronously and nothing is
 *     enqueued.  A CUDA error becomes STENCIL_ERR_CUDA.  Device-side checks
 *     (bounded waits that ran out, failed consistency checks) are recorded in
 *     a status word that stencil_plan_status() / stencil_batch_status() read.
 *     The library never traps and never aborts the process.
 *   - stencil_last_error() returns a message for the last failure on the
 *     calling thread.
 *   - A plan (or batch) may be used by one stream at a time.
 */
#ifndef GB300_STENCIL_H
#define GB300_STENCIL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t, declared here so callers need no CUDA header. */
typedef struct CUstream_st* stencil_stream_t;

typedef enum {
    STENCIL_OK = 0,
    STENCIL_ERR_INVALID_ARG = 1,   /* null pointer, bad size, bad enum value        */
    STENCIL_ERR_UNSUPPORTED = 2,   /* valid but not implemented (e.g. radius > 3)   */
    STENCIL_ERR_CUDA = 3,          /* a CUDA runtime call failed                    */
    STENCIL_ERR_OOM = 4,           /* device or host allocation failed              */
    STENCIL_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out            */
    STENCIL_ERR_DEVICE_CHECK = 6   /* a device-side consistency check failed        */
} stencil_status_t;

typedef enum { STENCIL_F32 = 0, STENCIL_BF16 = 1, STENCIL_F16 = 2 } stencil_dtype_t;

typedef enum { STENCIL_BOUNDARY_ZERO = 0, STENCIL_BOUNDARY_PERIODIC = 1 } stencil_boundary_t;

/* Arithmetic engine.  AUTO and FP32 use the CUDA cores.  The tensor-core
 * engines treat each weight row of a radius-3 (7x7) stencil as a banded
 * Toeplitz matrix and run the step as MMAs with FP32 accumulation (Sec.
 * II-D's stencil-as-matrix-product idea): TC_TF32 rounds inputs and weights
 * to TF32, TC_BF16 to BF16 (both round-to-nearest-even).  TC_3XTF32 recovers
 * accuracy: inputs and weights split into TF32 hi + lo parts and each
 * product is hi*hi + hi*lo + lo*hi (three MMAs, FP32-level error; warp-MMA
 * engine, FP32 storage only).  Storage FP32 or BF16.  Other radii or FP16
 * storage: STENCIL_ERR_UNSUPPORTED.
 * LOWRANK (any radius, FP32 storage, either boundary): the weights are factored
 * by an SVD into rho separable terms, W[dy][dx] = sum_k c_k[dy] v_k[dx] (rho =
 * the numerical rank, singular values above 1e-6 of the largest, or
 * options.rank), and each step runs as rho row passes and rho column passes
 * in FP32 on the CUDA cores: 2 rho (2r+1) FMAs per point instead of (2r+1)^2,
 * one step per launch.  Exact up to FP32 rounding of the factors when W has
 * rank rho; a truncation otherwise (the paper's related work on low-rank
 * tensor-core stencils, Sec. II-D). */
typedef enum {
    STENCIL_COMPUTE_AUTO = 0,
    STENCIL_COMPUTE_FP32 = 1,
    STENCIL_COMPUTE_TC_TF32 = 2,
    STENCIL_COMPUTE_TC_BF16 = 3,
    STENCIL_COMPUTE_TC_3XTF32 = 4,
    STENCIL_COMPUTE_LOWRANK = 5
} stencil_compute_t;

/* Kernel family.  The tensor-core contraction (7x7 box, one step per launch)
 * has two engines: warp-level MMAs (any storage/engine pair, both boundaries)
 * and tcgen05 MMAs with tensor-memory accumulators and TMA-staged operands,
 * which take zero-boundary grids stored in the MMA operand type (BF16 storage
 * with TC_BF16, FP32 with TC_TF32), rows of a multiple of 16 bytes,
 * ny >= 134 and nx >= 128.  With TC_TF32 the first launch of a run (which rounds the
 * caller's FP32 input to TF32) always runs on the warp-MMA engine.  kernel = TC
 * or AUTO picks tcgen05 where it applies (the faster engine as measured); with
 * autotune the first run times both. */
typedef enum {
    STENCIL_KERNEL_AUTO = 0,
    STENCIL_KERNEL_NAIVE = 1,      /* one thread per point, one step per launch      */
    STENCIL_KERNEL_STREAM = 2,     /* row-streaming tiles, k steps per launch        */
    STENCIL_KERNEL_TC = 3,         /* tensor cores: tcgen05 where it applies, else warp MMA */
    STENCIL_KERNEL_TC_WARP = 4,    /* tensor cores, warp-MMA engine only             */
    STENCIL_KERNEL_TC_UMMA = 5,    /* tensor cores, tcgen05 engine (UNSUPPORTED where it does not apply) */
    STENCIL_KERNEL_RESIDENT = 6,   /* small grids: the whole grid in one thread-block cluster's shared
                                      memory, every step of a run in one launch                        */
    STENCIL_KERNEL_LOWRANK = 7     /* chosen by compute = LOWRANK (reported by stencil_plan_info only) */
} stencil_kernel_t;

/* Optional plan settings; pass NULL for defaults.  0 means "choose".
 * kernel = AUTO with FP32 arithmetic picks RESIDENT when the grid fits one
 * cluster (two FP32 copies in the shared memory of at most 16 CTAs; roughly up
 * to 700 x 700 for radius 1) and no streaming-kernel option (tb_depth,
 * threads, tile_rows) is set; otherwise STREAM.  With autotune the first run
 * times both (and, for RESIDENT, every cluster size and blocking depth).  With
 * kernel = RESIDENT, tb_depth sets its steps per halo exchange (default 1).
 * stencil_plan_info reports tb_depth = 0 for RESIDENT (one launch per run),
 * ctas = the cluster size and tile_rows = the slab height. */
typedef struct {
    int compute;      /* stencil_compute_t                                          */
    int kernel;       /* stencil_kernel_t                                           */
    int tb_depth;     /* time steps per launch (temporal blocking depth k)          */
    int threads;      /* threads per CTA of the streaming kernel (multiple of 32)   */
    int tile_rows;    /* output rows per CTA tile of the streaming kernel           */
    int autotune;     /* 1: time candidate configurations on first run              */
    int mma_n;        /* tcgen05 engine: N of the widest MMA.  16, 32, 64 (BF16) or
                         16, 32 (TF32): one weight row per MMA, 128 x 128 output
                         tiles; 96 or 128: three or four weight rows stacked in one
                         MMA over 32-column N-tiles, 126- or 125-row output tiles   */
    int timeout_ms;   /* tcgen05 engine and TMA-fed streaming kernel: limit of each
                         device-side wait in ms (0 = 2000)                             */
    int debug_withhold; /* test hook, 0 in normal use: 1 makes CTA 0 of the tcgen05
                           engine withhold its first accumulator-ready signal, and CTA 0
                           of the TMA-fed streaming kernel wait for 16 bytes more than
                           its first row brings, so a wait runs out and the run
                           reports TIMEOUT                                             */
    int load;         /* streaming kernel's input rows: stencil_load_t                */
    int rank;         /* compute = LOWRANK: separable terms kept (0 = numerical rank,
                         else 1..2r+1)                                                 */
} stencil_options_t;

/* How the streaming kernel brings input rows into shared memory.  AUTO: the
 * library default (and, with autotune, both timed).  CP_ASYNC: each thread
 * copies its 16 bytes of every row (cp.async).  TMA: one thread issues 2D
 * tensor copies of each row (cp.async.bulk.tensor, completion on an mbarrier;
 * the copy engine's zero fill is the zero halo); FP32 storage, the zero rule
 * and nx a multiple of 4 only (else STENCIL_ERR_UNSUPPORTED at create).  Each
 * wait for a row is bounded by timeout_ms (an expired wait is reported as
 * STENCIL_ERR_TIMEOUT by stencil_plan_status).  Same arithmetic and bits
 * either way. */
typedef enum { STENCIL_LOAD_AUTO = 0, STENCIL_LOAD_CP_ASYNC = 1, STENCIL_LOAD_TMA = 2 } stencil_load_t;

/* What a plan decided.  Filled by stencil_plan_info(). */
typedef struct {
    int64_t ny, nx;
    int radius;
    int shape;             /* 0 = general box, 1 = star (off-axis weights are 0)   */
    int dtype, boundary, compute, kernel;
    int tb_depth;          /* k                                                     */
    int threads;           /* CTA size                                              */
    int halo_cols;         /* halo columns loaded on each side of a strip          */
    int tile_cols;         /* output columns per CTA                                */
    int tile_rows;         /* output rows per CTA                                   */
    int ctas;              /* CTAs per launch                                       */
    int smem_bytes;        /* dynamic shared memory per CTA                         */
    int64_t workspace_bytes;  /* device workspace the plan owns                    */
    int mma_n;             /* tcgen05 engine in use: N of one MMA; 0 = not in use   */
    int load;              /* streaming kernel's row loads (stencil_load_t); 0 = other kernel */
    int rank;              /* LOWRANK: separable terms in use; 0 = other kernel      */
} stencil_plan_info_t;

typedef struct stencil_plan stencil_plan_t;

/*
 * Create a plan for T-step sweeps of one grid shape and weight set.
 *   plan      out: the new plan (NULL on failure).
 *   ny, nx    grid rows and columns, each >= 1.
 *   radius    r in 1..3 (larger: STENCIL_ERR_UNSUPPORTED).
 *   weights   HOST, (2r+1)^2 FP32, row-major, weights[(dy+r)*(2r+1)+(dx+r)]; copied.
 *   dtype     stencil_dtype_t: storage type of grids in device memory.
 *   boundary  stencil_boundary_t.
 *   opt       NULL or settings.
 * Allocates one grid-sized device workspace (ping-pong buffer) on the current device.
 */
stencil_status_t stencil_plan_create(stencil_plan_t** plan, int64_t ny, int64_t nx, int radius,
                                     const float* weights, int dtype, int boundary,
                                     const stencil_options_t* opt);

/* Release a plan and its device workspace.  NULL is accepted. */
void stencil_plan_destroy(stencil_plan_t* plan);

/* Replace the plan's weights (HOST, (2r+1)^2 FP32, copied) without creating a
 * new plan: the workspace, the tuned configuration and any adjoint scratch are
 * kept, so a training loop can update the weights every iteration.  Work
 * already enqueued keeps the weights it was enqueued with.  The new weights
 * must keep the footprint class (star or box) a streaming or cluster-resident
 * plan was chosen for (else STENCIL_ERR_UNSUPPORTED, nothing changed); a
 * LOWRANK plan refactors them. */
stencil_status_t stencil_plan_set_weights(stencil_plan_t* plan, const float* weights);

/* Report the plan's choices (after stencil_plan_create; tuning may refine them on first run). */
stencil_status_t stencil_plan_info(const stencil_plan_t* plan, stencil_plan_info_t* info);

/*
 * out = A^T in: T Jacobi steps (the paper's Sec. II-C update repeated, Sec. VI-A).
 *   in, out   DEVICE grids of ny*nx elements of the plan's dtype.  `in` is only
 *             read.  in == out is allowed.  Other partial overlap is an error
 *             the library cannot detect.
 *   T         >= 0.  T == 0 copies in to out.
 * Launches ceil(T/k) kernels (k = tb_depth, +1 if in == out and that count is odd).
 */
stencil_status_t stencil_run(stencil_plan_t* plan, const void* in, void* out, int64_t T,
                             stencil_stream_t stream);

/*
 * As stencil_run, with HOST input and output: copies in_host to a device buffer
 * the plan owns, runs T steps, copies the result to out_host, and synchronises
 * `stream` before returning.  Pinned host memory gives full copy bandwidth.
 */
stencil_status_t stencil_run_host(stencil_plan_t* plan, const void* in_host, void* out_host,
                                  int64_t T, stencil_stream_t stream);

/*
 * As stencil_run_host without the final synchronisation: the copy in, the T
 * steps and the copy out are enqueued on `stream`, and out_host holds the
 * result once the stream has reached the end of that work.  Both host buffers
 * must stay valid until then; with pinned host memory the copies overlap work
 * on other streams (runs of two plans on two streams pipeline each other's
 * copies with their sweeps), pageable memory may make them synchronous.
 */
stencil_status_t stencil_run_host_async(stencil_plan_t* plan, const void* in_host, void* out_host,
                                        int64_t T, stencil_stream_t stream);

/* Number of kernel launches stencil_run(plan, in, out, T) makes (in != out). */
int64_t stencil_run_launches(const stencil_plan_t* plan, int64_t T);

/*
 * Synchronise the plan's last stream and read its device status word:
 * STENCIL_OK, STENCIL_ERR_TIMEOUT or STENCIL_ERR_DEVICE_CHECK.  Clears the word.
 */
stencil_status_t stencil_plan_status(stencil_plan_t* plan);

/*
 * T steps with a convergence check every m steps (the paper's periodic
 * convergence checks, Sec. IV).  After every m-th step t (t = m, 2m, ... <= T)
 * residuals[t/m - 1] = || u_t - u_{t-1} ||_2 over the whole grid (FP64,
 * deterministic).  Same operation, arguments and result bits as stencil_run
 * (periodic grids with nx % 4 != 0: the same values up to rounding, since
 * their results depend on the launch depths at the rounding level).
 *   residuals  DEVICE, floor(T/m) doubles, written.
 *   m          >= 1.
 * Each checked interval runs m-1 steps temporally blocked and its last step
 * as a single launch into a second buffer (the plan keeps two extra grids).
 */
stencil_status_t stencil_run_residual(stencil_plan_t* plan, const void* in, void* out, int64_t T,
                                      int64_t m, double* residuals, stencil_stream_t stream);

/* Message for the last failure of stencil_run_residual on the calling thread. */
const char* stencil_residual_last_error(void);

/*
 * Reverse-mode gradient of T steps (the adjoint of the Sec. II-C update).
 * For a loss L(u_T) whose gradient at u_T is grad_uT:
 *     lambda_T = grad_uT,  lambda_t = A^T lambda_{t+1}  (correlation with the
 *     flipped weights W[-dy][-dx], same boundary rule),
 *     grad_u0 = lambda_0,
 *     grad_w[(dy+r)*(2r+1)+(dx+r)] = sum_{t<T} sum_{i,j} lambda_{t+1}[i][j] u~_t[i+dy][j+dx].
 *   plan           an FP32 plan (other dtypes: STENCIL_ERR_UNSUPPORTED).
 *   u0, grad_uT    DEVICE, ny*nx FP32, only read.
 *   grad_u0        DEVICE, ny*nx FP32, written (may equal grad_uT).
 *   grad_w         (2r+1)^2 FP64, written; NULL to skip.  DEVICE memory (asynchronous
 *                  like the rest), or HOST memory (pageable or pinned: the call then
 *                  synchronises `stream` before it returns).  Every entry of the
 *                  square is returned, off-footprint ones included.
 *   ckpt_interval  steps between checkpoints; 0 = ceil(sqrt(T)).  The result does
 *                  not depend on it (same bits).
 * States are recomputed from checkpoints, not stored: the plan allocates and
 * keeps (ceil(T/s) + s + 2) grids of scratch, s = ckpt_interval.  The weight
 * gradient is reduced deterministically (fixed order, FP64 partials).
 * Asynchronous on `stream` like stencil_run.
 */
stencil_status_t stencil_adjoint(stencil_plan_t* plan, const void* u0, const void* grad_uT, int64_t T,
                                 void* grad_u0, double* grad_w, int64_t ckpt_interval,
                                 stencil_stream_t stream);

/* Kernel launches stencil_adjoint makes for T and ckpt_interval (grad_w != NULL). */
int64_t stencil_adjoint_launches(const stencil_plan_t* plan, int64_t T, int64_t ckpt_interval);

/* Message for the last failure of stencil_adjoint on the calling thread. */
const char* stencil_adjoint_last_error(void);

/*
 * ---- Batches: many independent grids in one persistent launch ----------------
 *
 * Each grid of a batch is its own Jacobi problem (Sec. II-C): its own size,
 * radius, weights, boundary and number of steps T.  stencil_run_batched runs
 * them all in one persistent kernel per radius (plus one launch per leftover
 * depth when k does not divide some T), replayed from a CUDA graph that the
 * first call captures.  The result of every grid is bit-identical to
 * stencil_run on a plan of the same grid (same arithmetic per point).
 */
typedef struct {
    int64_t ny, nx;         /* grid rows and columns, each >= 1                        */
    int radius;             /* 1..3                                                   */
    const float* weights;   /* HOST, (2r+1)^2 FP32, as for stencil_plan_create; copied */
    int boundary;           /* stencil_boundary_t (periodic needs nx % 4 == 0)        */
    int64_t T;              /* steps for this grid, >= 0                              */
    const void* in;         /* DEVICE, ny*nx dense row-major; only read               */
    void* out;              /* DEVICE, ny*nx dense row-major; may equal in            */
} stencil_grid_desc_t;

typedef struct {
    int tb_depth;           /* steps per work item k; 0 = 4, capped per radius (8 / 2 / 2) */
    int threads;            /* CTA size, multiple of 32 in 32..256; 0 = 128            */
    int tile_rows;          /* rows per tile; 0 = 256 (at least R*k + 2R + 2)          */
    int autotune;           /* 1: time each depth and CTA size on the whole batch at create */
    int timeout_ms;         /* bound of every device-side wait; 0 = 2000 ms             */
    int debug_withhold_item;/* test hook: 1 + index of a work item whose completion is never
                               published, so dependent waits run out (0 = off)          */
} stencil_batch_options_t;

typedef struct {
    int n;                  /* grids                                                   */
    int tb_depth, threads;
    int tiles;              /* tiles over all grids                                     */
    int64_t items;          /* work items (tile x time block) per run                  */
    int launches;           /* kernel launches per run                                 */
    int ctas;               /* CTAs of the first (persistent) launch                   */
    int64_t point_steps;    /* sum over grids of ny*nx*T                                */
} stencil_batch_info_t;

typedef struct stencil_batch stencil_batch_t;

/*
 * Create a batch of n grids.  Copies the descriptors and weights; the device
 * pointers must stay valid while the batch is used.  Allocates two padded
 * work grids per grid (row pitch rounded up to 4 elements), the item queue
 * and the counters.  With opt->autotune the batch is run several times here.
 */
stencil_status_t stencil_batch_create(stencil_batch_t** batch, int n, const stencil_grid_desc_t* grids,
                                      int dtype, const stencil_batch_options_t* opt);

/* Run every grid of the batch on `stream` (graph captured on the first call;
 * that first call must not be inside a stream capture of the caller). */
stencil_status_t stencil_run_batched(stencil_batch_t* batch, stencil_stream_t stream);

/* Synchronise the device and read the batch's status word (STENCIL_ERR_TIMEOUT
 * if a dependency wait ran out).  Clears the word. */
stencil_status_t stencil_batch_status(stencil_batch_t* batch);

stencil_status_t stencil_batch_info(const stencil_batch_t* batch, stencil_batch_info_t* info);

void stencil_batch_destroy(stencil_batch_t* batch);

/* Message for the last failure of a stencil_batch_* call on the calling thread. */
const char* stencil_batch_last_error(void);

/*
 * ---- Row slabs: one grid split across ranks ------------------------------------
 *
 * The paper splits the grid into tiles with a halo each (Sec. IV-A) and swaps
 * halos between neighbouring tiles before every step (Sec. IV-B to IV-D).
 * Here rank p of P owns the rows [y0, y1) of an ny x nx grid (full width) and
 * keeps G = radius * steps_per_exchange ghost rows above and below them, so
 * that it can advance steps_per_exchange steps between two exchanges.  Full
 * rows carry the corner values, so no two-stage corner forwarding is needed.
 *
 * The slab buffer (DEVICE, caller-owned, dense row-major) holds buffer_rows x
 * nx elements: buffer row b is global row y0 - ghost_above + b (mod ny for the
 * periodic rule).  Under the zero rule a slab at the top (bottom) edge of the
 * grid has no ghost rows there (ghost_above or ghost_below = 0).
 *
 * One temporal block:
 *   1. exchange: send buffer rows [send_above_row, +G) to the rank above (they
 *      become its rows [recv_below_row, +G)) and rows [send_below_row, +G) to
 *      the rank below (its rows [recv_above_row, +G)); receive likewise.  The
 *      rank above rank p is p-1, the one below p+1, wrapping for periodic.
 *   2. stencil_slab_step(slab, buf, s, stream), s <= steps_per_exchange:
 *      afterwards the owned rows hold u_{t+s} exactly (bit-identical to a
 *      single-domain stencil_run for FP32 storage); ghost rows are stale.
 * The library does steps 2 only; the exchange is the caller's (NCCL or any
 * other transport: the rows are contiguous).
 *
 * Requirements: every slab with a ghost region owns at least G rows, and
 * under the zero rule has G rows of neighbours on each side that has ghosts
 * (otherwise STENCIL_ERR_UNSUPPORTED).
 */
typedef struct {
    int64_t ny, nx;              /* the whole grid                                         */
    int64_t y0, y1;              /* owned global rows [y0, y1)                             */
    int radius, boundary;
    int64_t steps_per_exchange;  /* S                                                      */
    int64_t ghost_depth;         /* G = radius * S                                         */
    int64_t ghost_above, ghost_below;  /* G or 0 (zero rule at the grid's top/bottom edge) */
    int64_t buffer_rows;         /* ghost_above + (y1 - y0) + ghost_below                  */
    int64_t send_above_row, send_below_row;  /* first buffer row of the G rows sent up / down */
    int64_t recv_above_row, recv_below_row;  /* first buffer row of the ghost rows received   */
} stencil_slab_info_t;

typedef struct stencil_slab stencil_slab_t;

/* Geometry of a slab (host only: needs no GPU, allocates nothing). */
stencil_status_t stencil_slab_geometry(int64_t ny, int64_t nx, int64_t y0, int64_t y1, int radius,
                                       int boundary, int64_t steps_per_exchange,
                                       stencil_slab_info_t* info);

/* Create a slab: its geometry and a streaming-kernel plan (FP32 arithmetic,
 * `dtype` storage) for its buffer, which owns a buffer-sized workspace.
 * Arguments as for stencil_plan_create; opt may be NULL, opt->kernel must be
 * AUTO or STREAM and opt->compute AUTO or FP32 (else STENCIL_ERR_UNSUPPORTED). */
stencil_status_t stencil_slab_create(stencil_slab_t** slab, int64_t ny, int64_t nx, int64_t y0, int64_t y1,
                                     int radius, const float* weights, int dtype, int boundary,
                                     int64_t steps_per_exchange, const stencil_options_t* opt);

void stencil_slab_destroy(stencil_slab_t* slab);

stencil_status_t stencil_slab_info(const stencil_slab_t* slab, stencil_slab_info_t* info);

/* The slab's plan (owned by the slab): for stencil_plan_info / stencil_plan_status. */
stencil_plan_t* stencil_slab_plan(stencil_slab_t* slab);

/* Advance the owned rows of `buf` (DEVICE, buffer_rows x nx, in place) by
 * `steps` in 0..steps_per_exchange Jacobi steps; the ghost rows must hold the
 * neighbours' current rows on entry and are stale on return. */
stencil_status_t stencil_slab_step(stencil_slab_t* slab, void* buf, int64_t steps, stencil_stream_t stream);

/* Message for the last failure of a stencil_slab_* call on the calling thread. */
const char* stencil_slab_last_error(void);

/*
 * ---- Allocation-free sweep (no counterpart in the paper) ----------------------
 *
 * For callers that must not allocate device memory when they run a sweep: an
 * inference-engine plugin whose enqueue step may not allocate, code running
 * while a framework's caching allocator already holds the free memory, or a
 * latency-critical loop that cannot afford cudaMalloc's implicit device-wide
 * synchronisation.  It needs no plan (stencil_plan_create allocates a
 * workspace) and calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * Same operation and argument meaning as stencil_plan_create + stencil_run,
 * with the library's default configuration (no autotuning).  The ping-pong
 * buffer is a fixed device array of STENCIL_NOALLOC_MAX_BYTES inside the
 * library, kept on every GPU where it was set up until the process exits.
 * Grids with ny*nx*element_size above that limit are rejected with
 * STENCIL_ERR_UNSUPPORTED (see stencil_noalloc_last_error()).
 *   - The first call on each device (after its arguments pass the checks; a
 *     call with T == 0 will do) sets the array up: it looks up the array's
 *     device address and, under CUDA's default lazy module loading, loads the
 *     module that holds it, which reserves STENCIL_NOALLOC_MAX_BYTES of device
 *     memory at that moment (STENCIL_ERR_CUDA if that memory is not free).
 *     Make that first call before any region that must not allocate and
 *     before any stream capture.  Later calls allocate nothing.
 *   - All calls share the array and it keeps the last call's contents; nothing
 *     in it needs to start at zero.  Calls whose work overlaps on the GPU (two
 *     streams at once, or two threads) race on the array and give wrong results.
 *   - in == out is allowed; T == 0 copies in to out.
 */
#define STENCIL_NOALLOC_MAX_BYTES (64ull << 20)

stencil_status_t stencil_run_noalloc(int64_t ny, int64_t nx, int radius, const float* weights,
                                     int dtype, int boundary, const void* in, void* out, int64_t T,
                                     stencil_stream_t stream);

/* Message for the last failure of stencil_run_noalloc on the calling thread. */
const char* stencil_noalloc_last_error(void);

/* Human-readable name of a status code (static string). */
const char* stencil_status_string(stencil_status_t status);

/* Message describing the last failure on the calling thread ("" if none). */
const char* stencil_last_error(void);

/* Library version: major*10000 + minor*100 + patch. */
int stencil_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GB300_STENCIL_H */
