/*
 * sd.h -- C ABI of the GB300-native leading-order Stokesian-dynamics library.
 *
 * Method: Kopp & Hoefling, "GPU-accelerated simulation of colloidal suspensions
 * with direct hydrodynamic interactions" (arXiv:1205.6333).
 *
 *   v_i = sum_j mu_ij F_j = mu0 F_i + sum_{j != i} T(r_i - r_j) F_j        (Sec. 2.2, Eq. rotneMobility)
 *   mu0 = 1/(6 pi eta a)                                                  (Sec. 2.2)
 *   T(r) = mu0 3a/(4r) (I + rr) + mu0 a^3/(2 r^3) (I - 3 rr)  Rotne-Prager  (Sec. 2.2, Eq. rotneMobility)
 *   G(r) = (I + rr) / (8 pi eta r)                            Oseen        (Sec. 2.2, Eq. oseenTensor)
 *   r_i <- r_i + dt v_i                                       Euler        (Sec. 3.1, step 1)
 *
 * The mobility matrix is never stored (Sec. 3.1): every apply is a matrix-free
 * all-pairs sum on the GPU.
 *
 * Conventions for every entry point:
 *   - Arrays of vectors are n x 3 row-major (x0 y0 z0 x1 y1 z1 ...).
 *   - `on_device` = 1: the pointer is CUDA device memory of the handle's device;
 *     the call is asynchronous on the handle's stream and device-side errors
 *     (non-finite input, coincident particles, watchdog) surface at the next
 *     synchronising call (sd_synchronize or any host-pointer call).
 *     `on_device` = 0: the pointer is host memory; the call copies, runs, and
 *     synchronises the stream before returning.
 *     `on_device` = 2 (sd_set_positions, sd_get_positions, sd_set_forces only):
 *     host memory, copied asynchronously on the handle's stream (a DMA when the
 *     memory is page-locked).  The caller keeps it alive and unchanged (or unread,
 *     for sd_get_positions) until the stream has passed the copy; errors are
 *     deferred as for device pointers.
 *   - Caller pointers are borrowed for the duration of the call only.
 *   - The handle owns its device buffers, allocated through cfg.alloc/cfg.free
 *     when given (e.g. bound to a framework's caching allocator), else cudaMalloc.
 *   - Every call returns an sd_status; nothing aborts and no C++ exception
 *     crosses this boundary.  sd_last_error() gives a thread-local message.
 *   - A handle must not be used from two host threads at once.
 */
#ifndef SD_H
#define SD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SD_OK = 0,
    SD_ERR_ARG = 1,          /* invalid argument (null pointer, n < 0, a <= 0, ...)            */
    SD_ERR_CUDA = 2,         /* a CUDA runtime call failed                                       */
    SD_ERR_OOM = 3,          /* device allocation failed (cudaMalloc or cfg.alloc returned NULL) */
    SD_ERR_COINCIDENT = 4,   /* two distinct particles at r = 0 in RP or Oseen mode              */
    SD_ERR_NONFINITE = 5,    /* NaN or Inf in positions or forces                                */
    SD_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up (results of that call invalid) */
    SD_ERR_STATE = 7,        /* call out of order (e.g. step before positions were set)          */
    SD_ERR_UNSUPPORTED = 8,  /* valid request this build does not implement                      */
    SD_ERR_INTERNAL = 9      /* a device-side index check failed (debug builds, -DSD_DEBUG)      */
} sd_status;

/* Pair tensor.  RPY = Rotne-Prager for r >= 2a continued inside r < 2a by the
 * Yamakawa form mu0[(1 - 9r/(32a)) I + (3r/(32a)) rr] (not in the paper; the
 * textbook regularisation of overlapping spheres, finite at r = 0).
 * RP = the paper's Rotne-Prager form for every r > 0.  OSEEN = Eq. oseenTensor. */
typedef enum { SD_TENSOR_RPY = 0, SD_TENSOR_RP = 1, SD_TENSOR_OSEEN = 2 } sd_tensor;

/* Arithmetic of the all-pairs sum (Sec. 3.2, last paragraph: pair terms in single
 * precision, accumulation in higher precision).
 *   FP32C: FP32 pair terms, compensated (two-float) accumulation, FP64 near/self
 *          terms and FP64 position state.
 *   FP64 : everything in FP64 (reference path).
 *   FP32 : FP32 pair terms and plain FP32 accumulation (ablation only).        */
typedef enum { SD_PREC_FP32C = 0, SD_PREC_FP64 = 1, SD_PREC_FP32 = 2 } sd_precision;

typedef enum { SD_DTYPE_F32 = 0, SD_DTYPE_F64 = 1 } sd_dtype;

/* How the all-pairs kernel visits the pairs.
 *   DIRECTED : every ordered pair (i, j) separately, as in Sec. 3.2.
 *   SYMMETRIC: every unordered pair once, its term used for both particles
 *              (mu_ij = mu_ji, Sec. 2.2).  Each direction's term is the same as
 *              DIRECTED's, bit for bit; only the order of the sums differs.  The
 *              particles are cut into nb = npad / B blocks (npad = n rounded up
 *              to a multiple of 1024; FP32 modes: B = 512 from npad = 32768 on,
 *              else 256; FP64: B = 128), and the source-side partial sums take
 *              nb (nb + 1) / 2 * 3 B words (FP32 modes: 4-byte, FP64: 8-byte) of
 *              device memory.
 *   AUTO     : SYMMETRIC once there is at least one block pair per two SMs
 *              (nb (nb + 1) / 2 >= SMs / 2; on a 152-SM GB300: n > 2048 in the FP32
 *              modes, n > 1024 in FP64), else DIRECTED. */
typedef enum { SD_DENSE_AUTO = 0, SD_DENSE_DIRECTED = 1, SD_DENSE_SYMMETRIC = 2 } sd_dense_kernel;

typedef struct sd_config {
    int32_t n;               /* particles; 0 <= n <= 2^24                                  */
    double a;                /* sphere radius, > 0                                          */
    double eta;              /* viscosity, > 0                                              */
    int32_t tensor;          /* sd_tensor                                                   */
    int32_t prec;            /* sd_precision                                                */
    double box[3];           /* per dimension: 0 = unbounded (default); L > 0 = periodic with
                                side L, each pair interacting through its nearest image only
                                (Sec. 3.1 footnote).  L must be >= 3 max(r_near, rep_rc when
                                rep_eps != 0, 3a with lubrication) (SD_ERR_ARG).  Positions
                                are integrated unwrapped; sd_get_positions returns them so.
                                Batches return SD_ERR_UNSUPPORTED for a periodic box.        */
    double r_near;           /* pairs closer than r_near get their term in FP64; 0 = 2.5a;
                                must be >= 2.2a                                             */
    double rep_eps;          /* soft repulsion U = rep_eps (2a/r)^12 for r < rep_rc; 0 = off */
    double rep_rc;           /* repulsion cutoff (0 = 2.5a)                                 */
    double gravity[3];       /* uniform force added to every particle                       */
    int32_t device;          /* CUDA device ordinal                                         */
    void *stream;            /* cudaStream_t to run on; NULL = the legacy default stream    */
    void *(*alloc)(size_t bytes, void *ctx);   /* optional device allocator; it must return
                                                  memory aligned to 256 bytes, as cudaMalloc
                                                  does (the kernels use 16-byte vector loads
                                                  and bulk copies)                          */
    void (*free)(void *ptr, void *ctx);        /* its matching free                      */
    void *alloc_ctx;
    int32_t dense_kernel;    /* sd_dense_kernel                                             */
    int32_t lubrication;     /* 1: sd_step adds to each particle's force the singular lubrication
                                friction of the pairs with 2a < r < 3a (Sec. 2.3 Eq. lubrication,
                                truncated at s = r/a - 2 = 1), -sum_j zeta_ij (v_i - v_j), with the
                                velocities of the previous step (Sec. 3.1 step 2; zero before the
                                first step and after sd_set_positions).  Overlapping pairs (s <= 0)
                                get no term.  FP64.  Not with sd_adjoint or sd_batch_create
                                (SD_ERR_UNSUPPORTED). */
    double verlet_skin;      /* neighbour-list skin of sd_step (Sec. 3.1 step 2, Verlet lists): 0 = default
                                0.5a, < 0 = off.  The steps keep an FP64 near-pair list of the pairs
                                within its cutoff + skin, built by sd_set_positions and rebuilt once some
                                particle has moved skin / 4 relative to particle 0 since the last
                                build (a uniform translation never forces one; up to skin / 2 the
                                list still holds every pair within its cutoff, the largest of r_near,
                                rep_rc with repulsion and 3a with lubrication).  With constant forces
                                the rebuild and the near terms run beside the all-pairs kernel; with
                                repulsion or lubrication their pairs come from the same list, and the
                                near terms alone run beside it.  Each particle's list is in ascending
                                partner order, so a step gives the same result bit for bit from a
                                fresh or a reused list.  Off automatically when a periodic side is
                                below 3 (max cutoff + skin). */
} sd_config;

typedef struct sd_handle sd_handle;
typedef struct sd_batch sd_batch;

/* Fill *cfg with defaults: a = eta = 1, RPY, FP32C, unbounded, r_near = 2.5a,
 * no repulsion (rep_rc = 2.5a), no gravity, device 0, default stream, cudaMalloc,
 * Verlet skin 0.5a. */
void sd_config_init(sd_config *cfg);

/* Create a system of cfg->n particles.  Positions must be set before use; forces
 * default to zero.  *out receives the handle (NULL on failure). */
sd_status sd_create(const sd_config *cfg, sd_handle **out);
void sd_destroy(sd_handle *h);

/* Positions r_i (n x 3 doubles), copied into the handle's FP64 state; also
 * refreshes the FP32 mirror the all-pairs kernel reads; with Verlet lists it also
 * builds the steps' near-pair list around the new positions, so a trajectory
 * resumed from positions read back continues bit for bit.  Non-finite values give
 * SD_ERR_NONFINITE (host pointers: from this call; device pointers: deferred). */
sd_status sd_set_positions(sd_handle *h, const double *xyz, int on_device);
sd_status sd_get_positions(sd_handle *h, double *xyz, int on_device);

/* Per-particle external forces F_ext,i (n x 3 doubles), held constant by sd_step.
 * The force used in a step is F_ext,i + gravity + repulsion (Sec. 3.1, step 2). */
sd_status sd_set_forces(sd_handle *h, const double *f, int on_device);

/* Velocities V = mu(x) F at the current positions for the given forces F
 * (n x 3, dtype sd_dtype for both F and V) -- Sec. 2.2, Eq. rotneMobility;
 * Sec. 3.1, step 3.  Does not change the handle's state. */
sd_status sd_mobility_apply(sd_handle *h, const void *F, void *V, int dtype, int on_device);

/* nsteps explicit Euler steps (Sec. 3.1): F = F(x_n), v = mu(x_n) F, x_{n+1} = x_n + dt v.
 * Position state is FP64.  Steps run as a replayed CUDA graph on the handle's stream
 * (asynchronous; errors surface at the next synchronising call).  nsteps >= 0. */
sd_status sd_step(sd_handle *h, double dt, int64_t nsteps);

/* Row shards of the two calls above, for splitting one system over devices by
 * target rows (each device holds all n positions and forces and computes the
 * velocities of its own rows; the sum over j stays whole, Sec. 3.1 step 3).
 *   sd_mobility_apply_rows: rows row0 .. row1-1 of V = mu(x) F; F holds all n
 *     forces, V holds (row1 - row0) x 3 values.
 *   sd_step_rows: one Euler step in which only rows row0 .. row1-1 advance; the
 *     other rows keep their positions (the caller replaces them with the other
 *     shards' results, e.g. by an all-gather and sd_set_positions).  Eager, no graph.
 * Each row is bit-identical to the same row of sd_mobility_apply / sd_step(h, dt, 1):
 * the shard runs exactly the CTAs of the full launch that cover its rows, with the
 * same tiles.  Needs the directed all-pairs kernel (cfg.dense_kernel =
 * SD_DENSE_DIRECTED, or FP64): SD_ERR_UNSUPPORTED with the symmetric one, whose
 * source-side sums cross rows; sd_step_rows also with lubrication (the previous
 * velocities of other shards' rows are not known).  0 <= row0 <= row1 <= n, else
 * SD_ERR_ARG. */
sd_status sd_mobility_apply_rows(sd_handle *h, const void *F, void *V, int dtype, int on_device, int32_t row0,
                                 int32_t row1);
sd_status sd_step_rows(sd_handle *h, double dt, int32_t row0, int32_t row1);

/* Tile shards: one system split over nshards ranks by pairs, with either all-pairs
 * kernel (directed or symmetric) and every precision (Sec. 3.1 step 3: the N^2 sum
 * is divided, not the rows).  Every rank holds the whole state (all n positions and
 * forces).  Shard s runs the all-pairs kernel's persistent CTAs
 * [s G / nshards, (s + 1) G / nshards) of the full launch of G CTAs, which hold
 * equal runs of tiles, so the shards do equal pair work; for the symmetric kernel a
 * tile serves both particles of every pair in it, so a shard's share reaches rows
 * outside any one block of rows.
 *   *_part    : writes to P (device, n x 3 doubles) the shard's raw share of
 *               sum_{j != i} T(r_i - r_j) F_j / mu0 for every row i (no self term,
 *               no FP64 near-pair correction).  The near pass runs in every shard
 *               (the kernel's clamping follows it).
 *   *_combine : Pall (device, nparts x n x 3 doubles) holds the shards' P in shard
 *               order (e.g. from an all-gather); the call adds them in that order,
 *               then the self term and the near-pair corrections, and gives
 *               V = mu(x) F (sd_mobility_apply_combine) or the Euler update
 *               x <- x + dt V (sd_step_combine).
 * A combine must follow its part on the same handle with no other computing call
 * in between (SD_ERR_STATE otherwise); sd_mobility_apply_combine uses the forces
 * staged by sd_mobility_apply_part.  Every rank that combines the same Pall gets the
 * same result bit for bit, so replicated states stay identical.  The result equals
 * the unsharded call up to the order of the FP64 sums.  Asynchronous on the
 * handle's stream except for host F / V (on_device = 0), which synchronise.
 * 0 <= shard < nshards, nparts >= 1, else SD_ERR_ARG. */
sd_status sd_mobility_apply_part(sd_handle *h, const void *F, int dtype, int on_device, int32_t shard,
                                 int32_t nshards, double *P);
sd_status sd_mobility_apply_combine(sd_handle *h, const double *Pall, int32_t nparts, void *V, int dtype,
                                    int on_device);
sd_status sd_step_part(sd_handle *h, int32_t shard, int32_t nshards, double *P);
sd_status sd_step_combine(sd_handle *h, double dt, const double *Pall, int32_t nparts);

/* Synchronise the handle's stream and report deferred device-side errors. */
sd_status sd_synchronize(sd_handle *h);

/* Vector-Jacobian products of v(x, F) = mu(x) F at the current positions:
 *   gX = (dv/dx)^T W,   gF = mu(x)^T W = mu(x) W     (derivative of Eq. rotneMobility)
 * F, W inputs; gX, gF outputs (n x 3, dtype). */
sd_status sd_mobility_vjp(sd_handle *h, const void *F, const void *W, void *gX, void *gF, int dtype,
                          int on_device);

/* Gradient through nsteps Euler steps from the current positions x0 with the
 * handle's forces (F_ext + gravity; repulsion unsupported -> SD_ERR_UNSUPPORTED):
 *   lambda_T = gxT;  lambda_n = lambda_{n+1} + dt (dv/dx(x_n))^T lambda_{n+1};
 *   gx0 = lambda_0;  gF = dL/dF_ext = sum_n dt mu(x_n) lambda_{n+1}.
 * The forward pass is re-run with FP64 checkpoints every ckpt_every steps
 * (ckpt_every >= 1) and each segment is recomputed once.  The handle's positions
 * are restored to x0 on return.  gxT input, gx0 and gF outputs (n x 3 doubles). */
sd_status sd_adjoint(sd_handle *h, double dt, int64_t nsteps, int32_t ckpt_every, const double *gxT, double *gx0,
                     double *gF, int on_device);

/* Many independent clusters in one launch per step.  Cluster c holds particles
 * offsets[c] .. offsets[c+1]-1 (offsets: nclusters+1 int32, host memory,
 * non-decreasing, offsets[0] = 0, cluster sizes 0..256).  cfg->n is ignored; the
 * tensor, a, eta, gravity and prec (FP32C or FP64) of cfg apply.  Particles of
 * different clusters do not interact. */
sd_status sd_batch_create(const sd_config *cfg, const int32_t *offsets, int32_t nclusters, sd_batch **out);
void sd_batch_destroy(sd_batch *b);
sd_status sd_batch_set_positions(sd_batch *b, const double *xyz, int on_device);
sd_status sd_batch_get_positions(sd_batch *b, double *xyz, int on_device);
sd_status sd_batch_set_forces(sd_batch *b, const double *f, int on_device);
/* nsteps Euler steps of every cluster: one persistent kernel launch per step,
 * replayed from a CUDA graph.  The launch shape is picked by the built-in
 * autotuner on first use (or by sd_batch_autotune). */
sd_status sd_step_batched(sd_batch *b, double dt, int64_t nsteps);
/* Time the candidate launch shapes on the current state (state unchanged) and keep
 * the fastest.  *choice (may be NULL) receives the index of the chosen shape. */
sd_status sd_batch_autotune(sd_batch *b, int32_t *choice);
/* The candidate launch shapes, fixed at sd_batch_create: their number, and for shape
 * k in [0, count) the threads per CTA, the resident CTAs per SM and the targets per
 * thread (FP32C: 1 or 2 for the block kernel, which evaluates every ordered pair; 0
 * for the symmetric kernel, in which each warp takes two clusters and evaluates each
 * unordered pair once, mu_ij = mu_ji; FP64: 1).  Any output pointer may be NULL.
 * SD_ERR_ARG for a NULL batch or k out of range. */
int32_t sd_batch_shape_count(const sd_batch *b);
sd_status sd_batch_shape_info(const sd_batch *b, int32_t k, int32_t *threads, int32_t *ctas_per_sm,
                              int32_t *targets_per_thread);
/* Run the following steps with shape k instead of the autotuner's choice (SD_ERR_ARG
 * for k out of range). */
sd_status sd_batch_set_shape(sd_batch *b, int32_t k);
sd_status sd_batch_synchronize(sd_batch *b);

/* Velocities V = mu(x) F for n particles, computed without allocating any GPU
 * memory and without a handle.  The paper has no counterpart to this entry
 * point; it exists for callers that must not allocate: code running while a
 * stream is captured into a CUDA graph (cudaMalloc cannot be captured), plug-ins
 * whose host gives them a fixed device-memory budget, and loops that cannot
 * afford cudaMalloc's device synchronisation.
 *   x, F, V : device pointers, n x 3 doubles (positions, forces, velocities out).
 *   n       : 0 <= n <= 65536; larger n gives SD_ERR_ARG (the limit of the
 *             fixed scratch array below).
 *   a, eta  : radius and viscosity; tensor: sd_tensor.  Arithmetic: FP32 pair
 *             terms with compensated accumulation, self term and overlapping
 *             pairs exact, FP64 final sum (no FP64 near-pair pass).
 *   stream  : cudaStream_t the kernels are queued on (asynchronous; no sync).
 * Working memory is one static device array of about 14 MB, held by every GPU
 * that loads the library until the process exits; its device address is looked
 * up on the first call on each device, so make that first call before any stream
 * capture begins.  All calls share the array, so calls whose kernels overlap on
 * the GPU (different streams, or different host threads) race and give wrong
 * results: order them on one stream.  Coincident distinct particles in RP or
 * Oseen mode give NaN velocities (no error word is kept).  If a CUDA error from
 * the caller's earlier work is already pending when the call starts, it returns
 * SD_ERR_CUDA, queues nothing and leaves that error in place (it is not cleared). */
sd_status sd_mobility_apply_noalloc(const double *x, const double *F, double *V, int32_t n, double a, double eta,
                                    int32_t tensor, void *stream);

/* ---- memory-access study (App. A, Algorithms 3 and 4) -------------------- */

/* Kernels of the study: every thread j < n starts from in[j] and adds the n
 * elements in[map(k)], k = 0 .. n-1, storing the sum in out[j].
 *   SD_ACCESS_NAIVE        each thread loads its own map(k) from global memory;
 *   SD_ACCESS_TILING       the block stages tiles of `block` elements in shared
 *                          memory, thread t of the block loading map(m + t) with
 *                          its own j (App. A, Algorithm 4 with warpSize replaced
 *                          by the block size);
 *   SD_ACCESS_SMALLTILING  tiles of 32 elements loaded by the first warp (Algorithm 4);
 *   SD_ACCESS_BULK         linear map only: the tiling kernel with tiles of `block`
 *                          elements copied by cp.async.bulk into a double buffer.
 * Tile positions m + t >= n contribute zero (n need not be a multiple of the tile). */
typedef enum { SD_ACCESS_NAIVE = 0, SD_ACCESS_TILING = 1, SD_ACCESS_SMALLTILING = 2, SD_ACCESS_BULK = 3 } sd_access_algo;
/* Maps of App. A with p = 131 and M = 32 (j: the global index of the loading thread):
 * linear k -> k; strided k -> k p mod n; unordered k -> (k p + j M) mod n. */
typedef enum { SD_ACCESS_LINEAR = 0, SD_ACCESS_STRIDED = 1, SD_ACCESS_UNORDERED = 2 } sd_access_map;

/* Launch one study kernel on `stream` (asynchronous).  in, out: device arrays of n
 * elements, float (vec4 = 0) or float4 (vec4 = 1, componentwise sums, 16-byte
 * aligned), owned by the caller, not aliased.  block: threads per block, a multiple
 * of 32 in [32, 1024]; grid ceil(n / block).  Sums are formed in FP32 round-to-
 * nearest in the order k = 0 .. n-1 after in[j].  Errors: SD_ERR_ARG for an unknown
 * algorithm or map, the bulk kernel with a non-linear map or an input not 16-byte
 * aligned, a bad block size, n < 0 or NULL arrays with n > 0; SD_ERR_CUDA for a
 * failed launch.  n = 0 launches nothing. */
sd_status sd_access_run(int32_t algo, int32_t map, int32_t vec4, int32_t n, int32_t block, const void *in, void *out,
                        void *stream);
/* SD_ERR_TIMEOUT (and clears the flag) if a bulk kernel launched since the last call
 * gave up a bounded wait for a copy (its output is then invalid); otherwise SD_OK. */
sd_status sd_access_status(void);

/* ---- instrumentation (used by benchmarks and tests) ---------------------- */

/* Kernel families that can be timed with CUDA events on the handle's stream. */
typedef enum {
    SD_KERNEL_DENSE = 0,     /* all-pairs sum (the hot loop, Sec. 3.1 step 3)  */
    SD_KERNEL_EPILOGUE = 1,  /* split reduction + self term + Euler update     */
    SD_KERNEL_CELLS = 2,     /* cell-list build                                */
    SD_KERNEL_FORCES = 3,    /* force assembly (Sec. 3.1 step 2)               */
    SD_KERNEL_BATCHED = 4,   /* batched persistent kernel                      */
    SD_KERNEL_VJP = 5,       /* adjoint all-pairs kernel                       */
    SD_KERNEL_NEAR = 6,      /* FP64 near-pair pass before the all-pairs sum   */
    SD_KERNEL_COUNT = 7
} sd_kernel;

/* on = 1: record a CUDA event pair around every launch of each kernel family (steps
 * then run without graph replay).  Enabling clears the accumulated times. */
sd_status sd_profile(sd_handle *h, int on);
sd_status sd_batch_profile(sd_batch *b, int on);
/* Synchronise and return the summed event time (ms) and launch count of a family. */
sd_status sd_profile_read(sd_handle *h, int kernel, double *ms, int64_t *launches);
sd_status sd_batch_profile_read(sd_batch *b, int kernel, double *ms, int64_t *launches);
/* Number of kernel launches this handle has issued so far (graph replays count
 * every kernel node). */
int64_t sd_launch_count(const sd_handle *h);
/* The all-pairs kernel the handle runs: SD_DENSE_DIRECTED or SD_DENSE_SYMMETRIC
 * (AUTO resolved at sd_create); SD_DENSE_AUTO for a NULL handle or n = 0. */
int32_t sd_dense_kernel_used(const sd_handle *h);
int64_t sd_batch_launch_count(const sd_batch *b);
/* Iteration limit of every bounded device-side wait (default 1 << 22). */
sd_status sd_set_watchdog(sd_handle *h, int64_t iterations);
/* Failure injection for tests of the time-out path (no GPU fault, no unbounded
 * wait).  While on != 0, the first CTA of every all-pairs kernel launch of this
 * handle (sd_mobility_apply, sd_step, the row shards) never issues the bulk copy of
 * its first tile: its waits for that tile give up after the watchdog limit, the
 * kernel records the time-out, drains the copies it did issue and exits, and the
 * next synchronising call returns SD_ERR_TIMEOUT.  Results of such calls are
 * invalid (a step's positions too: set them again after switching it off).
 * Cached step graphs are dropped on every change. */
sd_status sd_inject_stall(sd_handle *h, int32_t on);

/* Thread-local message describing the last non-OK status ("" if none). */
const char *sd_last_error(void);
/* Library version string. */
const char *sd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SD_H */
