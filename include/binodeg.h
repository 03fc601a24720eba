/*
 * binodeg -- exact degree of the C*-solution set of a binomial system on GB300 (sm_103a).
 *
 * C ABI of libbinodeg.so.  Plain pointers and sizes only.  Unless stated otherwise every
 * pointer is a HOST pointer owned by the caller; the library copies what it needs and
 * never keeps a caller pointer after a call returns.  Integer matrices are row-major.
 * Every function returns a status code (BD_OK on success) and never throws; the message
 * of the last failure on the calling thread is available from bd_last_error().
 *
 * Method (Chen & Mehta, "Parallel degree computation for solution space of binomial
 * systems ...", arXiv 1501.02237):
 *   x^A = b with A in Z^{n x m} (Sec. 2, Eq. standard-form);  Smith form P A Q = D
 *   (Sec. 2, Eq. smith; Sec. 3);  the solution set has |prod d_j| components of dimension
 *   d = n - rank A (Prop. 1), each of degree d! Vol_d(conv{columns of P_0, 0}) (Prop. 4,
 *   Eq. deg-vol), computed as the sum of |det| over the cells of a regular triangulation
 *   obtained from generic lift heights (Sec. 4.1, Eq. lower-face, strict form of Sec. 5).
 */
#ifndef BINODEG_H
#define BINODEG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define BD_OK 0
#define BD_ERR_ARG 1       /* invalid argument (sizes, null pointers, limits) */
#define BD_ERR_OVERFLOW 2  /* an exact value would not fit: Smith form entries above 2^100,
                              or the Hadamard bound of the lifted minors above 2^126 */
#define BD_ERR_TIES 3      /* every one of the allowed liftings produced a tie */
#define BD_ERR_CUDA 4      /* a CUDA runtime call failed (message in bd_last_error) */
#define BD_ERR_TIMEOUT 5   /* a bounded device-side wait ran out */
#define BD_ERR_NOMEM 6     /* host or device allocation failed */
#define BD_ERR_STATE 7     /* call not valid in the object's current state */

/* flags reported in outputs */
#define BD_FLAG_DEGENERATE 1   /* points not full-dimensional: volume 0 */
#define BD_FLAG_INT128 2       /* the 128-bit kernel path was used */
#define BD_FLAG_INCONSISTENT 4 /* b^{Q_0} != 1: empty solution set, degree 0 */
#define BD_FLAG_PIVOT 8        /* the volume came from the pivoting walk (dimension above BD_KMAX) */

/* limits: K <= BD_KMAX lattice dimension, N <= BD_NMAX points (the origin included) */
#define BD_KMAX 14
#define BD_NMAX 64

typedef struct {
  uint64_t nvol_lo, nvol_hi; /* NVol_k(conv points) = k! Vol_k, exact unsigned 128-bit */
  uint64_t cells;            /* accepted cells (lower facets) of the final lifting */
  uint64_t singular;         /* (k+1)-subsets with zero simplex determinant */
  uint64_t ties;             /* tie subsets of the final lifting (0 whenever BD_OK) */
  uint64_t subsets;          /* C(npts, k+1): subsets tested per lifting */
  int32_t relifts;           /* liftings discarded because of ties */
  int32_t flags;             /* BD_FLAG_* */
  int32_t max_abs_coord;     /* largest |coordinate| of the input points */
  int32_t bound_bits;        /* ceil(log2) of the Hadamard bound that chose the int path */
} bd_volume_out;

typedef struct {
  uint64_t degree_lo, degree_hi; /* degree of the solution set = torsion * nvol (Props. 1, 4) */
  uint64_t nvol_lo, nvol_hi;     /* degree of one component, NVol_d(conv{P_0 columns, 0}) */
  uint64_t torsion;              /* number of components |prod d_j| (Prop. 1) */
  int32_t rank, dim;             /* rank A and d = n - rank A */
  int32_t consistent;            /* 1 unless coefficients were given and b^{Q_0} != 1 */
  int32_t relifts;
  uint64_t subsets, cells;
  int32_t flags;
  int32_t max_abs_coord;         /* largest |coordinate| of the reduced kernel points */
} bd_degree_out;

/* Fault injection for tests of the out-of-memory paths (host side: nothing fails on the GPU).
 * Arms the library's device-allocation wrapper so that the after-th device allocation from now
 * (0: the next one) fails as cudaMalloc does when the device is out of memory, once; the call
 * that makes it returns BD_ERR_NOMEM, as every call does on a real out-of-memory error, and
 * frees what it had allocated.  after < 0 disarms.  The environment variable
 * BD_INJECT_ALLOC_FAILURE, read when the library loads, arms it the same way.  Always BD_OK. */
int bd_inject_alloc_failure(int32_t after);

/* Message of the last failed call on this thread ("" if none). Owned by the library. */
const char* bd_last_error(void);

/* CUDA stream (a cudaStream_t, or NULL for the legacy default stream) used by the
 * synchronous calls below on this thread.  The library does not take ownership. */
int bd_set_stream(void* stream);

/*
 * Degree of V(x^A - b) (Props. 1, 2, 4).
 *   A    : n x m integers, column i = alpha_i - beta_i (Eq. standard-form); 1 <= n <= 126,
 *          0 <= m <= 256.
 *   coef : NULL (generic coefficients: the system is taken as consistent) or 4*m integers,
 *          binomial i -> (num1, den1, num2, den2) = c_{i,1}, c_{i,2} as fractions,
 *          b_i = -c_{i,2}/c_{i,1}; the consistency condition b^{Q_0} = 1 (Eq. consistency)
 *          is decided exactly.  Denominators and numerators must be nonzero.
 *   seed : lift seed; the result does not depend on it.
 * Host reduction (Smith form, LLL-reduced kernel basis, torsion) runs on the CPU; the
 * volume on the GPU: the subset enumeration up to dimension BD_KMAX and BD_NMAX points (n + 1,
 * the origin included), the pivoting walk of bd_volume_pivot beyond either (dimension up to 30;
 * BD_FLAG_PIVOT, subsets = ridges examined).
 * dim = 0 gives degree = torsion; dim = 1 is a segment, whose normalized
 * length max - min of the kernel points (and 0) is taken directly (kernel points of any size
 * below 2^62; the enumeration takes coordinates below 2^40).  Errors: BD_ERR_ARG,
 * BD_ERR_OVERFLOW, BD_ERR_TIES, BD_ERR_CUDA, BD_ERR_NOMEM.
 */
int bd_degree(const int64_t* A, int32_t n, int32_t m, const int64_t* coef, uint64_t seed,
              bd_degree_out* out);

/*
 * Host front end of bd_degree only (no GPU): Smith form, torsion, consistency and the
 * LLL-reduced kernel points; A as for bd_degree (1 <= n <= 126).  points receives (n + 1) x d integers (row i = point i, the
 * last row the origin) and must hold (n + 1) * n entries.  info receives 8 int64:
 * {rank, dim, torsion, consistent, max_abs_coord, 0, 0, 0}.
 */
int bd_reduce(const int64_t* A, int32_t n, int32_t m, const int64_t* coef, int64_t* points,
              int64_t* info);

/*
 * NVol_k(conv points) = k! Vol_k (Sec. 4, Eq. deg-nvol), exact.
 *   points : npts x k integers (row = point), k+1 <= npts <= BD_NMAX, 1 <= k <= BD_KMAX.
 *            The origin is NOT added.  Not full-dimensional -> volume 0, BD_FLAG_DEGENERATE.
 *   seed   : lift seed; ties are re-lifted (up to 8 liftings, then BD_ERR_TIES).
 */
int bd_volume(const int64_t* points, int32_t npts, int32_t k, uint64_t seed, bd_volume_out* out);

/* As bd_volume with caller-given lift heights (npts values, |lift| < 2^40) and no re-lift:
 * a tie is reported in out->ties and the call returns BD_ERR_TIES. */
int bd_volume_lifted(const int64_t* points, const int64_t* lifts, int32_t npts, int32_t k,
                     bd_volume_out* out);

/*
 * Lower-facet status of `count` given (k+1)-subsets (each k+1 strictly increasing uint8
 * indices, back to back) under the given lifts, on the GPU (Eq. lower-face, strict form).
 *   status[i] : 0 singular (zero determinant), 1 rejected (a point strictly below),
 *               2 accepted (every other point strictly above), 3 tie (none below, one on).
 *   absdet[i] : |det(a_{s_1} - a_{s_0}, .., a_{s_k} - a_{s_0})| as int64 (0 if singular,
 *               -1 if it needs more than 63 bits).
 */
int bd_classify(const int64_t* points, const int64_t* lifts, int32_t npts, int32_t k,
                const uint8_t* subsets, int32_t count, int32_t* status, int64_t* absdet);

/* ---- device-resident plans (the timed path of the benchmark) ------------------------- */

typedef struct bd_plan bd_plan;

typedef struct {
  int32_t warps_per_block;  /* 0: choose from shared-memory capacity */
  int32_t blocks_per_sm;    /* 0: occupancy calculator */
  int64_t item_subsets;     /* split prefixes until each holds at most this many subsets; 0: auto */
  int32_t force_int128;     /* 1: use the 128-bit path even when 64 bits suffice */
  int32_t bottom_stage;     /* the walk's last levels on the 32-bit coordinate path (k >= 4):
                               5 = the 5-D test (a det4 per quadruple after the Bareiss level
                               k-4), 4 = the 4-D test (a det3 per triple after level k-3),
                               0 = chosen from the point set: the 5-D test when k >= 6 and at
                               most half of a fixed sample of (k+1)-subsets is full-dimensional
                               (mostly singular systems; the 4-D test's finer work list wins
                               otherwise); other paths and k < 4 ignore it; any other value:
                               BD_ERR_ARG */
  int32_t reserved[2];
} bd_plan_opts;

/* Copies the points to device memory and builds the work list.  opts may be NULL. */
int bd_plan_create(const int64_t* points, int32_t npts, int32_t k, const bd_plan_opts* opts,
                   bd_plan** plan);
/* Enqueue one pass over all subsets with lifting (seed, attempt) on `stream` (NULL: the
 * thread's stream).  Asynchronous: nothing is copied to or from the host. */
int bd_plan_launch(bd_plan* plan, uint64_t seed, int32_t attempt, void* stream);
/* One shard of such a pass (multi-GPU sharding, one process per GPU): the work list's ranges
 * u with u % shards == shard, 0 <= shard < shards.  The shards of one (seed, attempt) together
 * cover every subset exactly once, so the exact volume is the sum of the shards' nvol, cells,
 * singular and ties (an all-reduce of a few words); a tie in any shard means a re-lift for all.
 * Every shard must use the same plan options on the same GPU model (the work list depends on
 * the resident warp count; bd_plan_info reports it for a cross-check).  bd_plan_read then
 * returns this shard's partial sums. */
int bd_plan_launch_shard(bd_plan* plan, uint64_t seed, int32_t attempt, int32_t shard, int32_t shards,
                         void* stream);
/* Wait for the last launch on its stream and read its result. */
int bd_plan_read(bd_plan* plan, bd_volume_out* out);
/* The full volume (launch, read, re-lift on ties) with inputs already on the device. */
int bd_plan_volume(bd_plan* plan, uint64_t seed, bd_volume_out* out);
/* Number of work items, kernel launch geometry and integer path: {items, blocks, warps_per_block,
 * shared_bytes_per_block, path (0: int32 coordinate / int64 lift minors, 1: int64, 2: int128),
 * slots_per_warp, ranges (work units: runs of consecutive items a warp takes at once), bottom
 * stage (the dimension of the walk's last test: 5, 4, 3 or 2)}. */
int bd_plan_info(const bd_plan* plan, int64_t* info);
int bd_plan_destroy(bd_plan* plan);

/* ---- batches (many systems in one persistent launch) ----------------------------------------
 *
 * A batch collects systems (bd_batch_add: an exponent matrix as for bd_degree; or
 * bd_batch_add_points: a point set as for bd_volume, dimension <= 12), reduces them on host
 * threads (bd_batch_prepare), then bd_batch_run enumerates all of them.  In the batched mode one
 * persistent kernel per integer path (int32/int64/int128 minors) pulls (system, prefix) work
 * items, largest predicted cost first, from one global list; each warp reloads the points of the
 * system it is working on.  Item sizes follow the per-system predicted cost (`cost`, e.g. from a
 * learned model; NULL: the closed-form bound C(N,k+1) (k^3/3 + (N-k)(k+1))).  The launches can
 * be captured in a CUDA graph and replayed; an autotuner can pick warps per block and items per
 * warp by timing candidates on a sample of the batch.  Systems with ties are re-lifted and rerun.
 * mode 1 instead calls bd_volume once per system (the plain form, for comparison).
 * Results are exact and identical in every mode.  The batch owns its device buffers (freed by
 * bd_batch_destroy).
 */
#define BD_FEATURES 16  /* per-system cost-model features written by bd_batch_features */

typedef struct bd_batch bd_batch;

typedef struct {
  int32_t mode;            /* 0: batched persistent launches, 1: one bd_volume per system */
  int32_t warps_per_block; /* 0: 4 (or the autotuned value) */
  int32_t item_factor;     /* work items per resident warp; 0: 4 (or the autotuned value) */
  int32_t use_graph;       /* 1: capture the batched launches in a CUDA graph and replay it */
  int32_t autotune;        /* 1: choose warps_per_block and item_factor by timing candidates */
  int32_t bottom_stage;    /* as in bd_plan_opts, per system; 0: the 5-D test for every system with
                              k >= 4 on the 32-bit path (in a shared launch it took fewer SM
                              cycles on every class of system); mode 0 */
  const float* cost;       /* NULL or one predicted cost per system (any positive unit) */
  int32_t reserved[4];
} bd_batch_opts;

typedef struct {
  double host_ms;          /* bd_batch_prepare wall time */
  double gpu_ms;           /* device time of the batched launches (CUDA events) */
  double wall_ms;          /* wall time of bd_batch_run (without autotuning) */
  double tune_ms;          /* device time spent by the autotuner */
  int64_t subsets;         /* (k+1)-subsets resolved per lifting, all systems */
  int64_t items;           /* work items launched */
  int32_t launches;        /* kernel launches (mode 1: one per system and lifting) */
  int32_t warps_per_block, item_factor;
  int32_t relifted;        /* systems re-lifted because of ties */
} bd_batch_stats;

int bd_batch_create(bd_batch** batch);
int bd_batch_add(bd_batch* batch, const int64_t* A, int32_t n, int32_t m, const int64_t* coef, uint64_t seed,
                 int32_t* index);
int bd_batch_add_points(bd_batch* batch, const int64_t* points, int32_t npts, int32_t k, uint64_t seed,
                        int32_t* index);
int bd_batch_size(const bd_batch* batch, int32_t* count);
/* Host reductions of every system on `threads` threads (0: all hardware threads). */
int bd_batch_prepare(bd_batch* batch, int32_t threads);
/* count x BD_FEATURES floats: N, k, log2 C(N,k+1), log2 closed-form cost, integer path, Hadamard
 * bits (all, coordinates), log2(1 + max |coordinate|), fraction of zero and of +-1 coordinates,
 * mean coordinate range, N - k, n, m, rank, log2 torsion.  Needs bd_batch_prepare. */
int bd_batch_features(const bd_batch* batch, float* features);
int bd_batch_run(bd_batch* batch, const bd_batch_opts* opts, bd_batch_stats* stats);
/* Result of system `index` after bd_batch_run; cycles (may be NULL) receives the SM cycles its
 * work items took in the batched mode (0 in mode 1). */
int bd_batch_result(const bd_batch* batch, int32_t index, bd_degree_out* out, uint64_t* cycles);
int bd_batch_destroy(bd_batch* batch);

/* ---- serving (continuous batching) ---------------------------------------------------------
 *
 * bd_server_start launches a host pump thread; one persistent kernel (launched on demand, gone
 * after ~40 ms without work) claims (slot, prefix) work items from a device ring, one ticket per
 * warp by fetch-and-add, while the pump keeps appending to it.  bd_server_submit reduces a system on the caller's thread
 * and queues it; the pump admits queued systems into free slots whenever the device budget
 * allows (a slot, ring room, and at most max_inflight_items items in flight), in arrival order
 * (order 0) or by smallest predicted cost (order 1; predicted_cost from the cost model, or <= 0
 * for the closed-form bound).  Admitted systems' items interleave on the device with those of
 * systems already running.  Finished degrees are returned by bd_server_poll with their latency
 * from submission.  Results are identical to bd_degree's.  The persistent kernel carries systems
 * of at most 32 points (31 variables) and dimension 10 whose minors fit 64 bits (its per-warp
 * shared memory is sized for them: 8 warps per SM, leaving room for other kernels); the others
 * (128-bit minors, dimension above 10, more points: up to 126 variables are accepted, as by
 * bd_degree) are served by a side worker thread that runs bd_degree's volume path, in arrival
 * order, on a stream of its own beside the persistent kernel.
 *
 * Every work item is published with a stamp (its ticket) written after it; a warp that claims
 * a ticket waits for the stamp, at most publish_wait_ms.  When that bound runs out the kernel
 * records the ticket and every warp exits (no GPU fault); the pump then fails the request that
 * owns the ticket with BD_ERR_TIMEOUT (bd_server_poll returns it with the ticket), puts the
 * other admitted requests back at the front of the queue (they run again from the start, so
 * their results stay exact), resets the ring and relaunches the kernel.  bd_server_stats counts
 * these faults.
 */
typedef struct bd_server bd_server;
typedef struct {
  int32_t slots;             /* systems resident at once (0: 256) */
  int32_t ring_items;        /* work-item ring capacity (0: 2^20) */
  int64_t memory_budget;     /* device bytes for slots and ring (0: as sized above) */
  int32_t warps_per_block;   /* 0: 4 */
  int32_t blocks_per_sm;     /* 0: occupancy minus one (room for other kernels) */
  int64_t item_subsets;      /* smallest work item in subsets (0: 256) */
  int64_t max_inflight_items;/* admitted but unfinished items (0: the ring capacity) */
  int32_t order;             /* 0 FIFO, 1 smallest predicted cost first */
  int32_t publish_wait_ms;   /* bound of the kernel's wait for a work item's publication (0: 1000) */
  int32_t test_withhold;     /* test hook, 0 in normal use: the n-th admission's publication stamps
                                are never written, so the bounded wait for them runs out */
  int32_t bottom_stage;      /* as in bd_plan_opts, per request; 0: chosen from its points when it
                                is admitted, for a request alone on the GPU (latency) or for one
                                sharing it with requests in flight or waiting (throughput) */
} bd_server_opts;
typedef struct {
  int64_t submitted, completed, relifted, launches;
  int64_t ring_items;
  int32_t slots, blocks, warps_per_block, waiting;
  int64_t routed;            /* requests served by the side route */
  int32_t peak_resident;     /* most requests holding a slot (items on the device) at once */
  int32_t faults;            /* publication waits that ran out (each reset the ring) */
} bd_server_stats;
int bd_server_start(const bd_server_opts* opts, bd_server** server);
int bd_server_submit(bd_server* server, const int64_t* A, int32_t n, int32_t m, const int64_t* coef, uint64_t seed,
                     double predicted_cost, int64_t* ticket);
/* One finished request, waiting up to wait_ms for one; BD_ERR_STATE when none is ready. */
int bd_server_poll(bd_server* server, int32_t wait_ms, int64_t* ticket, bd_degree_out* out, double* latency_ms);
int bd_server_stats_get(bd_server* server, bd_server_stats* stats);
/* Finishes every submitted request, then stops the kernel and frees the server. */
int bd_server_stop(bd_server* server);

/* ---- learned cost model ------------------------------------------------------------------
 *
 * A 16 -> 64 -> 64 -> 1 fully connected ReLU network in FP32 that predicts log2 of a system's
 * enumeration cost (SM cycles of its work items) from the BD_FEATURES features of
 * bd_batch_features.  Forward, backward and Adam run in this library's CUDA kernels.  The
 * prediction only sizes and orders work (bd_batch_opts.cost); it never touches a result.
 * Parameters: BD_MLP_PARAMS floats, W1[64][16], b1[64], W2[64][64], b2[64], W3[64], b3;
 * normalization: mean[16] then std[16] applied to the features before the first layer.
 */
#define BD_MLP_PARAMS 5313
typedef struct bd_mlp bd_mlp;
/* He-uniform initialisation from a counter-based generator seeded by `seed`. */
int bd_mlp_create(uint64_t seed, bd_mlp** mlp);
int bd_mlp_destroy(bd_mlp* mlp);
int bd_mlp_get_params(const bd_mlp* mlp, float* params, float* norm /* NULL or 32 floats */);
int bd_mlp_set_params(bd_mlp* mlp, const float* params, const float* norm /* NULL or 32 floats */);
/* y[i] = network(features of row i), X: count x 16 host floats. */
int bd_mlp_predict(bd_mlp* mlp, const float* X, int32_t count, float* y);
/* Gradient of the mean squared error (1/count) sum (f(x_i) - y_i)^2 with respect to every
 * parameter (BD_MLP_PARAMS floats) and the loss itself, at the current parameters. */
int bd_mlp_gradient(bd_mlp* mlp, const float* X, const float* y, int32_t count, float* grad, float* loss);
/* Adam (lr, beta 0.9/0.999) on the mean squared error, minibatches of `batch`, `epochs` passes
 * over a seeded permutation; sets the normalization from X first.  final_loss: the mean
 * squared error over the last epoch. */
int bd_mlp_train(bd_mlp* mlp, const float* X, const float* y, int32_t count, int32_t epochs, int32_t batch, float lr,
                 uint64_t seed, float* final_loss);

/* ---- allocation-free variant ------------------------------------------------------------
 *
 * bd_volume_noalloc: the same exact volume as bd_volume (same kernel, same liftings, same
 * result fields), for callers that cannot allocate device memory: for instance a process whose
 * device memory is entirely reserved by another allocator, or a latency-critical loop in which
 * cudaMalloc / cudaFree are not acceptable because they can block and synchronize the device.
 * The paper has no counterpart: this is a deployment convenience of this library.
 *
 * Inputs and outputs are the caller's HOST buffers, as for bd_volume.  All device scratch (the
 * staged points, the work list, the work counter and the accumulators) lives in one static
 * device array of BD_NOALLOC_SCRATCH_BYTES bytes inside the library image, which every GPU that
 * loads the library keeps until the process exits; the call itself never allocates.  The work
 * list is capped at BD_NOALLOC_MAX_ITEMS prefixes (the split is coarsened to fit); point sets
 * beyond BD_NMAX points or BD_KMAX dimensions are rejected with BD_ERR_ARG.
 *
 * The first call on each device looks up the device address of the array (a one-time set-up
 * with that device current) and keeps it for the life of the process.  Every call synchronizes
 * the thread's stream, so none may be made while that stream is being captured.  A device reset (cudaDeviceReset) unloads the array with the
 * library image and makes later calls on that device invalid.  Every call shares the array and
 * the array keeps the last call's contents; the call clears what must start at zero.  Calls
 * from this process are serialized, and every call synchronizes the thread's stream before it
 * returns (on success and on every error after its first copy), so the array is idle between
 * calls; two calls whose work overlapped on the GPU (for instance from two processes sharing
 * the library image through another loader) would race on the shared array.
 */
#define BD_NOALLOC_MAX_ITEMS 65536
#define BD_NOALLOC_SCRATCH_BYTES (8192 + 16 * BD_NOALLOC_MAX_ITEMS)
int bd_volume_noalloc(const int64_t* points, int32_t npts, int32_t k, uint64_t seed, bd_volume_out* out);

/* ---- integer issue peak (the denominator of the roofline; measurement only) ---------------
 *
 * The lower-facet test is bound by instruction issue on the integer and single-precision pipes
 * (Sec. 4's test runs on exact integer minors, no memory stream and no dense contraction), so
 * its roofline is the rate at which this GPU issues 32-bit lane operations.  bd_issue_peak
 * measures it: every thread of a full-occupancy grid (blocks_per_sm x SMs blocks of 256
 * threads; 0 = the resident maximum) runs iters x 16 rounds of eight coupled recurrences of one
 * instruction kind, each step one instruction (see the kinds below), on the stream of
 * bd_set_stream.  out receives the lane operations, the CUDA-event time, lane operations per
 * second, the largest block's SM cycle count (clock64) and the SM clock it implies, and the
 * lane operations per SM per cycle.  Allocates and frees two small device buffers.
 *   kind 0: LOP3 (logic, ALU pipe)    1: IMAD (32-bit multiply-add)   2: LOP3 and IMAD alternating
 *   kind 3: FFMA (single precision)   4: LOP3 and FFMA alternating
 * Errors: BD_ERR_ARG (kind, iters outside [1, 2^20], blocks_per_sm above the resident limit),
 * BD_ERR_CUDA. */
typedef struct {
  double lane_ops;            /* lane operations executed */
  double ms;                  /* kernel time (CUDA events) */
  double lane_ops_per_s;
  double sm_cycles;           /* cycles of the slowest block's timed loop */
  double sm_mhz;              /* sm_cycles / ms: the SM clock during the run */
  double lane_ops_per_sm_clk; /* per SM per cycle over the run (the slowest block's cycles) */
  int32_t sms, blocks, threads_per_block, kind;
} bd_peak_out;
int bd_issue_peak(int32_t kind, int32_t blocks_per_sm, int32_t iters, bd_peak_out* out);

/* ---- host emulation (CPU tests and the native CPU baseline; never used by the calls above) */

typedef struct bd_host_opts {
  int32_t threads;       /* CPU threads, each emulating one single-lane team (<= 0: 1) */
  int32_t force_int128;  /* nonzero: run the 128-bit walker whatever the bound */
  uint64_t item_subsets; /* work-item split threshold in subsets (0: 4096; 1: deepest items) */
  int32_t team_width;    /* > 1: one team of this many lanes, run as threads in lockstep */
  int32_t shard;         /* with shards > 1: only the work ranges u with u % shards == shard */
  int32_t shards;        /* <= 1: the whole enumeration */
  int32_t bottom_stage;  /* as in bd_plan_opts (0: chosen from the point set) */
} bd_host_opts;

/* Runs the same lower-facet enumeration as the GPU kernel on CPU threads, with the given
 * lifts (no re-lift); opts may be NULL (one thread, default split).  Returns BD_ERR_TIES
 * when the lifting has a tie. */
int bd_host_volume_lifted(const int64_t* points, const int64_t* lifts, int32_t npts, int32_t k,
                          const bd_host_opts* opts, bd_volume_out* out);

/* ---- cells of the triangulation and their inner normals (Sec. 6, witness-set start systems) */

/* The cells of the regular triangulation of conv(points) that the volume's lifting induces
 * (bd_volume's lifting for this seed, re-lifted on ties), in lexicographic order, each with its
 * inner normal (Eq. lower-d-face-again): alpha^ = (alpha, 1) with <a_j, alpha> + omega_j = beta
 * on the cell's points and > beta on every other point; (alpha, beta) give the change of
 * variables t_i = y_i s^alpha_i and the factor s^-beta of the cell's homotopy.
 *   cells : capacity x (k+1) point indices, increasing within a cell
 *   den   : capacity positive denominators: alpha = alpha_num / den, beta = beta_num / den
 *   alpha : capacity x k numerators
 *   beta  : capacity x 2 words, the 128-bit numerator: low 64 bits, then high 64 bits
 *   count : the number of cells; when it exceeds capacity nothing is written and the call
 *           returns BD_ERR_ARG (capacity 0 just counts)
 *   out   : the volume result (the sum of the cells' normalized volumes)
 * Errors: BD_ERR_ARG, BD_ERR_OVERFLOW (a normal outside the output range), BD_ERR_TIES,
 * BD_ERR_CUDA, BD_ERR_NOMEM. */
int bd_cells(const int64_t* points, int32_t npts, int32_t k, uint64_t seed, int64_t capacity, uint8_t* cells,
             int64_t* den, int64_t* alpha, int64_t* beta, int64_t* count, bd_volume_out* out);
/* The same with the given lifts on one host core (CPU tests); BD_ERR_TIES when the lifting has
 * a tie. */
int bd_host_cells(const int64_t* points, const int64_t* lifts, int32_t npts, int32_t k, int64_t capacity,
                  uint8_t* cells, int64_t* den, int64_t* alpha, int64_t* beta, int64_t* count);

/* The start solutions of the witness-set homotopy, cell by cell (Sec. 6): for every cell of
 * bd_cells (same seed, lexicographic order) and generic coefficients c_{i,q} = exp(2 pi i u),
 * u from SplitMix64 on the stream mix(coef_seed XOR 0xC2B2AE3D27D4EB4F) at counter
 * i*npts + q + 1, the solutions of the cell's start system (Eq. affine-cut-starting, reduced
 * to the binomial system of Eq. affine-cut-eliminated), |det| of them per cell and the volume
 * in all.
 *   sols          : capacity x k complex numbers (re, im interleaved); solution s, coordinate
 *                   i at sols[2 (s k + i)]; a device pointer when sols_on_device is nonzero
 *   count         : the number of solutions (when above capacity: BD_ERR_ARG, nothing written)
 *   max_residual  : NULL, or receives the largest |y^{E_j} / b_j - 1| over all solutions and
 *                   equations (checked on the device)
 * Errors: BD_ERR_ARG, BD_ERR_OVERFLOW, BD_ERR_TIES, BD_ERR_CUDA, BD_ERR_NOMEM. */
int bd_start_solutions(const int64_t* points, int32_t npts, int32_t k, uint64_t seed, uint64_t coef_seed,
                       int64_t capacity, double* sols, int32_t sols_on_device, int64_t* count, double* max_residual);
/* The same on one host core with the given lifts (CPU tests). */
int bd_host_start_solutions(const int64_t* points, const int64_t* lifts, int32_t npts, int32_t k, uint64_t coef_seed,
                            int64_t capacity, double* sols, int64_t* count, double* max_residual);

/* ---- mixed volume: the BKK generalisation of the degree (Appendix A) ------------------- */

typedef struct {
  uint64_t mv_lo, mv_hi;  /* MV(conv A_1, .., conv A_k), exact unsigned 128-bit; MV(P, .., P) = NVol(P) */
  uint64_t cells;         /* fine mixed cells of the final lifting */
  uint64_t singular;      /* tuples of pairs with det M = 0 */
  uint64_t ties;          /* tie tuples of the final lifting (0 whenever BD_OK) */
  uint64_t tuples;        /* prod_i C(|A_i|, 2): tuples of pairs resolved per lifting */
  int32_t relifts;        /* liftings discarded because of ties */
  int32_t flags;          /* BD_FLAG_INT128, BD_FLAG_DEGENERATE (a component without two distinct
                             points: MV = 0, nothing launched) */
  int32_t bound_bits;     /* ceil(log2) of the Hadamard bound that chose the integer path */
  int32_t reserved;
  double device_ms;       /* the final lifting's enumeration kernel, CUDA events on the library's
                             stream; 0 for the host emulation */
} bd_mixed_out;

/*
 * Mixed volume of k lattice point sets in Z^k (Bernstein's count of the isolated C*-solutions
 * of a generic system with these supports), by enumerating the fine mixed cells of a random
 * lifting on the GPU: every tuple of one pair {p_i, q_i} per set with M = [a_{q_i} - a_{p_i}]
 * nonsingular, whose inner normal puts every other point of every set strictly above its
 * pair; MV = sum |det M| over them.
 *   points : the sets back to back, sum(counts) x k integers (row = point), |x| < 2^40
 *   counts : k set sizes, each >= 1, sum <= BD_NMAX; 1 <= k <= BD_KMAX
 *   seed   : lift seed (heights as bd_volume's for the flat point list); ties are re-lifted
 *            (up to 8 liftings, then BD_ERR_TIES).  The result does not depend on it.
 * Errors: BD_ERR_ARG (sizes, limits, more than 2^62 tuples, walk state above shared memory),
 * BD_ERR_OVERFLOW (exact minors beyond 128 bits), BD_ERR_TIES, BD_ERR_CUDA, BD_ERR_NOMEM.
 */
int bd_mixed_volume(const int64_t* points, const int32_t* counts, int32_t k, uint64_t seed, bd_mixed_out* out);

/* As bd_mixed_volume with caller-given heights (sum(counts) values, |lift| < 2^40) and no
 * re-lift (a tie returns BD_ERR_TIES), optionally listing the fine mixed cells:
 *   cells    : NULL, or capacity x 2k indices: cell c, set i -> (p, q), p < q, local indices
 *              into set i, at cells[c * 2k + 2i]; cells in lexicographic order of these rows
 *   absdet   : NULL, or capacity values |det M| (-1 when above 63 bits)
 *   capacity : cells the buffers hold; fewer than out->cells -> BD_ERR_ARG (out->cells counts)
 *   force_int128 : nonzero takes the 128-bit path even when 64 bits suffice. */
int bd_mixed_volume_lifted(const int64_t* points, const int32_t* counts, int32_t k, const int64_t* lifts,
                           int32_t force_int128, bd_mixed_out* out, int32_t* cells, int64_t capacity,
                           int64_t* absdet);
/* The same walker on CPU threads (team_width 1: one lane per thread, items taken in turn) or as
 * one lockstep team of team_width lanes run as threads (1..32), for CPU tests.  prefix_levels > 0
 * fixes that many levels per work item (at most k-1, k-2 with the 3-D leaf stage; 0: the
 * library's choice); leaf3 1 / 0 forces the 3-D leaf stage on / off where the 64-bit path and
 * k >= 3 allow it (-1: the library's choice). */
int bd_host_mixed_volume_lifted(const int64_t* points, const int32_t* counts, int32_t k, const int64_t* lifts,
                                int32_t team_width, int32_t force_int128, int32_t prefix_levels, int32_t leaf3,
                                bd_mixed_out* out, int32_t* cells, int64_t capacity, int64_t* absdet);

/* ---- output-sensitive volume by simplicial pivoting (Sec. 4.2, Eq. pivot) -------------- */

/*
 * NVol_k(conv points) by walking the cells of the lifting's triangulation from one to the next
 * across their ridges (breadth first, on the GPU) instead of testing every (k+1)-subset: the
 * work grows with the number of cells, not with C(npts, k+1).  The start cell is found by
 * extension from the lowest lifted point; the neighbour across a ridge is the point beyond it
 * of least height / (-barycentric coordinate), decided exactly.
 *   points : npts x k integers, |x| < 2^20, k+1 <= npts <= 127, 1 <= k <= 30 (a cell is a mask
 *            of its points: one 64-bit word up to 64 points, two words above)
 *   seed   : lift seed: heights 1 + (top 40 bits of bd_volume's SplitMix64 stream), in [1, 2^40],
 *            wider than bd_volume's because up to ~1e8 cells are walked; a tie re-lifts (8 liftings)
 *   out    : nvol, cells, ties, relifts, flags (BD_FLAG_DEGENERATE when not full-dimensional;
 *            BD_FLAG_INT128 when the tableau took 128-bit entries), bound_bits; subsets holds the
 *            ridges examined, (k+1) * cells
 *   device_ms : NULL, or the traversal's time on the GPU (CUDA events; all levels)
 * The tableau's entries are minors of the cells' difference matrices: 64-bit while Hadamard's
 * bound on them (bound_bits) stays below 2^62, 128-bit above (fewer warps per SM, slower pivots).
 * Errors: BD_ERR_ARG, BD_ERR_OVERFLOW (heights D h(p), a minor times a 41-bit lift difference
 * summed over k+1 terms, may leave 127 bits: bound_bits above about 84; or the start cell's
 * support function, reduced by the gcd of its coefficients, left 128 bits), BD_ERR_TIES,
 * BD_ERR_CUDA, BD_ERR_NOMEM (more than 2^30 cells).
 */
int bd_volume_pivot(const int64_t* points, int32_t npts, int32_t k, uint64_t seed, bd_volume_out* out,
                    double* device_ms);

/* The same traversal on the host with the given heights (|lift| <= 2^40, no re-lift: a tie
 * returns BD_ERR_TIES), one team of team_width lanes (1..32; more than 1 runs them as threads in
 * lockstep), for CPU tests.  walk_budget: cells entered in place (by one tableau pivot each)
 * below every eliminated cell (the GPU path uses 64; 0 eliminates every cell).  cells: NULL, or
 * capacity bitmasks of the cells' points (bit p for point p; npts <= 64), increasing; fewer than
 * out->cells -> BD_ERR_ARG. */
int bd_host_volume_pivot(const int64_t* points, const int64_t* lifts, int32_t npts, int32_t k, int32_t team_width,
                         int32_t walk_budget, bd_volume_out* out, uint64_t* cells, int64_t capacity);

/* Test hook of the pivoting walk (process-wide; the paper has no counterpart): while on != 0,
 * bd_volume_pivot, bd_host_volume_pivot and bd_degree_pivot take 128-bit tableau entries
 * whatever the bound, so that the wide path runs on small inputs too.  Returns the previous
 * setting. */
int bd_pivot_force_wide(int32_t on);

/* bd_degree with the volume always by pivoting: up to 126 variables and solution sets of
 * dimension up to 30, e.g. the master spaces of Table mspace-deg. */
int bd_degree_pivot(const int64_t* A, int32_t n, int32_t m, const int64_t* coef, uint64_t seed, bd_degree_out* out);

#ifdef __cplusplus
}
#endif

#endif /* BINODEG_H */
