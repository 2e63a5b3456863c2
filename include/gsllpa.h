/*
 * gsllpa.h -- C ABI of the GB300 (sm_103a) GSL-LPA library.
 *
 * GSL-LPA (arXiv 2403.01261) is label-propagation community detection
 * followed by a split-last step that relabels every community into its
 * internally connected pieces.  This library runs both phases, and the
 * modularity score, as CUDA kernels on one GPU.
 *
 * Graph.  An undirected graph G(V, E, w) (Section 3, "Preliminaries") is
 * passed as symmetric CSR: every edge {i, j} is stored twice, as (i, j) in
 * row i and (j, i) in row j, with equal weights.  Symmetry is required but
 * not checked.  Rows need not be sorted; a repeated entry adds its weight
 * once per occurrence.
 *
 * Memory.  Unless a name ends in _host, every pointer argument that refers
 * to graph or label data is a DEVICE pointer on the context's device, owned
 * by the caller, and must stay valid until the call has completed on its
 * stream.  Scratch memory (label double buffers, frontier flags, worklists,
 * hash tables, union-find parents) is owned by the context, grown on demand
 * and reused across calls.  A context is not thread safe: use one per host
 * thread.
 *
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL: the legacy
 * default stream).  Work is queued on that stream and every entry point
 * synchronises it before returning: the sweep loop reads the change count
 * back after every sweep (the stop test of Algorithm 3 needs it) and all
 * calls report device-detected input errors through their return code.
 *
 * Errors.  Every entry point returns GSL_OK (0) or one of the GSL_ERR_*
 * codes below; gsl_strerror() names them and gsl_ctx_last_error() returns a
 * one-line detail for the last failing call on a context.  On error the
 * contents of output buffers are unspecified.
 */
#ifndef GSLLPA_H
#define GSLLPA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GSL_OK 0
#define GSL_ERR_INVALID 1   /* bad argument or malformed graph / labels          */
#define GSL_ERR_OVERFLOW 2  /* a weighted degree (sum of a row's weights) >= 2^31 */
#define GSL_ERR_NOMEM 3     /* device or pinned host allocation failed            */
#define GSL_ERR_CUDA 4      /* a CUDA runtime call failed                         */
#define GSL_ERR_TIMEOUT 5   /* a device-side retry loop hit its iteration cap     */

#define GSL_MODE_SYNC 0     /* Jacobi sweeps: every vertex reads the previous labels */
#define GSL_MODE_ASYNC 1    /* in-place sweeps, as Algorithm 3 updates C             */

#define GSL_STATS_SWEEPS 64

typedef struct gsl_ctx gsl_ctx;

/* Symmetric CSR on the device.  0 <= n < 2^31; offsets has n+1 entries with
 * offsets[0] = 0, offsets[i] <= offsets[i+1], offsets[n] = nnz; cols has nnz
 * entries, each in [0, n). */
typedef struct gsl_csr {
  int64_t n;
  int64_t nnz;
  const int64_t* offsets;
  const int32_t* cols;
} gsl_csr;

/* Per-call statistics (host struct, optional). */
typedef struct gsl_stats {
  int32_t iterations;                 /* sweeps performed (l_i of Algorithm 3)          */
  int32_t converged;                  /* 1: stopped by dN/N <= tolerance; 0: max_iters  */
  int64_t changed[GSL_STATS_SWEEPS];  /* dN of sweep t (t < 64)                          */
  int64_t active[GSL_STATS_SWEEPS];   /* vertices processed in sweep t (pruned frontier) */
  int64_t edges_scanned;              /* CSR entries read by all sweeps                  */
  int64_t communities;                /* after a split: number of pieces, else 0         */
  float ms_lpa;                       /* device time of the sweep phase                  */
  float ms_split;                     /* device time of the split phase (gsl_gsllpa)     */
} gsl_stats;

/* Creates a context on CUDA device `device`.  *ctx receives the handle. */
int gsl_ctx_create(gsl_ctx** ctx, int device);

/* Frees the context and all scratch memory it owns.  NULL is accepted. */
int gsl_ctx_destroy(gsl_ctx* ctx);

/* Degree-class thresholds of the sweep kernels: vertices of degree
 * 33..warp_max are handled by one warp each, degree warp_max+1..blk_max by
 * one block each, larger degrees (hubs) by one 8-CTA thread-block cluster
 * each (or in 8192-entry pieces spread over blocks: see
 * gsl_ctx_set_hub_cluster).  Label sums use shared-memory hash tables
 * (8 KB per warp, 96 KB per block, 8 x 96 KB per cluster) and spill to
 * context-owned global tables when a vertex has more distinct neighbour
 * labels than fit.  Defaults 1024 and 32768.  Requires 32 <= warp_max <=
 * 2^20 and warp_max <= blk_max.  Results do not depend on these values. */
int gsl_ctx_set_tuning(gsl_ctx* ctx, int32_t warp_max, int32_t blk_max);

/* Shape of the block kernel (degree warp_max+1..blk_max and hub pieces):
 * threads per block (128, 256 or 512) and shared-memory table slots per
 * block (8 bytes each; at least 16 * threads, so that the slots warps may
 * still claim after a table is declared full -- up to 128 per warp -- fit
 * in its last quarter, and the table must fit one block's shared memory).  Defaults 512 and 12288.  Hub rows are split into pieces only
 * while a piece always fits the table (at least ~11,600 slots); below that
 * hubs take one block each.  Results do not depend on these values. */
int gsl_ctx_set_block_config(gsl_ctx* ctx, int32_t threads, int32_t table_slots);

/* Own-label majority filter for rows of the two longest table classes
 * (degree above 256 up to blk_max; the paper has no counterpart), and also
 * for the rows of 33..256 entries from sweep 4 on in single-graph calls and
 * from sweep 6 on in the batched loop.  Before their hash tables are built,
 * one lean warp-per-row pass sums the weight of a row's entries carrying
 * the vertex's own label; when it is more than half of the row's weight
 * (the vertex itself excluded) the own label is Eq. 2's strict argmax and
 * the row is done.  mode 0: never; 1 (default): from sweep 3 on (sweep 2
 * reads the nearly all-distinct labels of sweep 1); 2: every sweep after
 * the first.  Labels and statistics do not depend on the mode. */
int gsl_ctx_set_majority(gsl_ctx* ctx, int32_t mode);

/* Two-phase synchronous sweeps (the paper has no counterpart: it is a GPU
 * scheduling choice).  In a two-phase sweep one edge-parallel pass first
 * gathers the label of every CSR entry's neighbour into a context-owned
 * int32[nnz] array, and the per-vertex kernels then read those labels
 * sequentially instead of gathering them.  mode 0: never; 1:
 * when the graph has at least 2^22 entries and the sweep runs on all
 * vertices or the previous sweep changed more than a quarter of them;
 * 2: every synchronous sweep that reads labels (not sweep 1 from the
 * identity labelling).  Default 0; gsl_autotune may choose 1.  Labels and
 * statistics do not depend on the mode. */
int gsl_ctx_set_pregather(gsl_ctx* ctx, int32_t mode);

/* Float-weight sweeps (gsl_lpa_f32, gsl_gsllpa_f32): 1 (default) runs them
 * on the integer path when the weights have the exact fixed-point form
 * described at gsl_lpa_f32, 0 always sums in float64.  Other values:
 * GSL_ERR_INVALID.  Labels do not depend on it. */
int gsl_ctx_set_f32_fixed(gsl_ctx* ctx, int32_t mode);

/* Hub rows (synchronous or asynchronous sweeps, integer weights) whose
 * degree is at most max_degree are aggregated by one thread-block cluster
 * of 8 CTAs each: the row's label table is spread over the 8 CTAs' shared
 * memories and filled with distributed-shared-memory atomics.  A row with
 * more distinct labels than those tables hold is redone in a global-memory
 * table.  Longer hubs are cut into pieces of 8192 entries.  0 turns the
 * clusters off; by default every hub row goes to a cluster.  max_degree
 * < 0: GSL_ERR_INVALID.  Labels and statistics do not depend on it. */
int gsl_ctx_set_hub_cluster(gsl_ctx* ctx, int64_t max_degree);

/* Bounds of the device-side retry loops (the paper has no counterpart).
 * Every open-addressing insert of the sweep tables stops after probe_bound
 * probes, and every union-find find or union of the split after
 * unionfind_bound steps; a loop that reaches its bound raises an error bit,
 * the kernel finishes without waiting on anything, and the call returns
 * GSL_ERR_TIMEOUT (labels unspecified).  The defaults (2^24 probes, 2^26
 * steps) cannot be reached on valid input: tables always keep free slots
 * and union-find paths are shorter than n.  Lower values exist so that
 * tests can drive that error path without a fault or a hang.  0 restores a
 * default; negative values: GSL_ERR_INVALID. */
int gsl_ctx_set_retry_bounds(gsl_ctx* ctx, int32_t probe_bound, int32_t unionfind_bound);

/* Result of gsl_autotune and gsl_autotune_batch: the chosen setting (now
 * set on the context) and the timings. */
typedef struct {
  int32_t warp_max;     /* degree-class thresholds (gsl_ctx_set_tuning) */
  int32_t blk_max;
  int32_t pregather;    /* two-phase mode (gsl_ctx_set_pregather) */
  int32_t candidates;   /* settings timed */
  int32_t sweeps;       /* sweeps timed per setting (gsl_autotune), max_iters (gsl_autotune_batch) */
  float best_ms;        /* device time with the chosen setting */
  float entry_ms;       /* and with the setting the context had on entry */
  int32_t majority;     /* own-label majority mode (gsl_ctx_set_majority) */
  int32_t blk_threads;  /* block shape (gsl_ctx_set_block_config) */
  int32_t blk_slots;
} gsl_tune_result;

/* Autotuner of the sweep kernels' settings (the paper has no counterpart:
 * its CPU design has no degree classes).  Runs the first `sweeps` sweeps
 * of synchronous or asynchronous LPA (mode) from the identity labels on
 * graph g (device CSR, weights as in gsl_lpa) once per candidate setting
 * and times each run with CUDA events on `stream`.  Candidates: warp_max
 * in {128, 256, 512, 1024} x blk_max in {4096, 12288, 32768, 131072} with
 * blk_max >= warp_max, x block shape (threads, table slots) in {(512,
 * 12288), (256, 6144)}, x majority mode in {0, 1, 2}, x two-phase mode in
 * {0, 1}; settings that run the same kernels on g (the same binning of
 * g's degrees, and a block shape or majority mode only where g has rows
 * that use it) are timed once.  The fastest setting is set on the context
 * (the setting the context had on entry wins ties).  1 <= sweeps <= 64.
 * Labels do not depend on any of these settings, so tuning changes only
 * speed.  The context's scratch is used; the graph is only read.
 * Synchronises `stream`.  Errors as gsl_lpa; on error the entry setting
 * is restored. */
int gsl_autotune(gsl_ctx* ctx, const gsl_csr* g, const int32_t* weights, int32_t mode, int32_t sweeps,
                 gsl_tune_result* out, void* stream);

/* The same search for the batched path: each candidate setting (as for
 * gsl_autotune, without two-phase sweeps, which the batched loop does not
 * use) runs gsl_gsllpa_batch on the packed graphs (arguments as there; a
 * sample of the graphs a caller will batch), once to capture its CUDA
 * graph and once timed (gsl_batch_stats.ms).  labels_out receives the
 * batch's labels (the same for every setting); the fastest setting stays
 * on the context.  Synchronises `stream`. */
int gsl_autotune_batch(gsl_ctx* ctx, const gsl_csr* g, int32_t num_graphs, const int64_t* vptr_host,
                       const int32_t* weights, double tolerance, int32_t max_iters, int32_t mode,
                       int32_t* labels_out, gsl_tune_result* out, void* stream);

/* Label propagation: lpa() of Algorithm 3 without its final split (the
 * "GVE-LPA" phase).  Labels start as labels_init (device int32[n], values
 * in [0, n)) or, when labels_init is NULL, as C = [0 .. n).  Each sweep
 * moves every vertex i of the frontier to
 *     argmax_c  sum_{j in J_i, j != i, C_j = c} w_ij         (Eq. 2)
 * with ties to the smallest label, and keeps the label of a vertex with no
 * neighbour other than itself.  The frontier is every vertex in sweep 1
 * and afterwards the changed vertices and their neighbours (the pruning of
 * lpaMove()).  After sweep t the call stops if dN_t / n <= tolerance or
 * t = max_iters.
 *   weights     device int32[nnz], every entry >= 1, or NULL for unit weights
 *               (Section 3).  Sums are exact int32: every weighted degree
 *               must be < 2^31 (else GSL_ERR_OVERFLOW).
 *   tolerance   tau >= 0 of Algorithm 3.
 *   max_iters   MAX_ITERATIONS >= 0; 0 returns the initial labels.
 *   mode        GSL_MODE_SYNC: Jacobi sweeps, deterministic, equal to the
 *               unpruned synchronous definition label for label.
 *               GSL_MODE_ASYNC: labels updated in place, so a vertex may
 *               see neighbours already moved in the same sweep; the result
 *               depends on scheduling.
 *   labels_out  device int32[n]; may equal labels_init.
 *   stats       optional host struct.
 */
int gsl_lpa(gsl_ctx* ctx, const gsl_csr* g, const int32_t* weights, const int32_t* labels_init,
            double tolerance, int32_t max_iters, int32_t mode, int32_t* labels_out,
            gsl_stats* stats, void* stream);

/* Float weights at the paper's precision (Section 4.1: 32-bit float edge
 * weights, 64-bit float label sums).  Same arguments and behaviour as
 * gsl_lpa / gsl_gsllpa / gsl_modularity except that `weights` is a device
 * float[nnz] (required when nnz > 0) whose every value must be finite and
 * > 0 (else GSL_ERR_INVALID).  The label with the largest float64 sum
 * wins, ties to the smallest label.  Sums of non-integer weights depend on
 * the order of the additions, which is not fixed on the GPU, so labels are
 * not guaranteed bit-identical to a sequential evaluation where two sums
 * agree to rounding; they are whenever every partial sum is exact in
 * float64 (for instance small integers or multiples of 1/8).  Modularity is
 * formed from float64 sums.  When every weight is a multiple of 2^-S and
 * every row's total times 2^S stays below 2^31 (checked through the largest
 * weight and the largest degree), every float64 sum is exact and the
 * sweeps run on the integer path with weights w * 2^S, which compares the
 * same sums scaled by 2^S: the labels are the float path's
 * (gsl_ctx_set_f32_fixed turns this off). */
int gsl_lpa_f32(gsl_ctx* ctx, const gsl_csr* g, const float* weights, const int32_t* labels_init,
                double tolerance, int32_t max_iters, int32_t mode, int32_t* labels_out, gsl_stats* stats,
                void* stream);
int gsl_gsllpa_f32(gsl_ctx* ctx, const gsl_csr* g, const float* weights, double tolerance, int32_t max_iters,
                   int32_t mode, int32_t* labels_out, gsl_stats* stats, void* stream);
int gsl_modularity_f32(gsl_ctx* ctx, const gsl_csr* g, const float* weights, const int32_t* labels,
                       double* q_out, void* stream);

/* Split last: splitDisconnectedBfs() of Algorithm 2.  labels_out[v] becomes
 * the smallest vertex id of the connected piece of v's community that holds
 * v, where the pieces are the connected components of the subgraph of edges
 * (u, v) with labels_in[u] == labels_in[v].  This is the labelling Algorithm
 * 2 produces when each BFS starts from the first unvisited vertex in
 * ascending order (and the fixed point of Algorithm 1).
 *   labels_in   device int32[n], any values (only compared for equality).
 *   labels_out  device int32[n]; may equal labels_in.
 *   renumber    0: pieces keep their smallest-vertex-id labels;
 *               1: pieces are numbered 0..k-1 in increasing order of their
 *                  smallest vertex id.
 *   k_out       optional HOST pointer receiving k, the number of pieces.
 */
int gsl_split(gsl_ctx* ctx, const gsl_csr* g, const int32_t* labels_in, int32_t* labels_out,
              int32_t renumber, int64_t* k_out, void* stream);

/* Split by label propagation: splitDisconnectedLp() of Algorithm 1 (SL-LP,
 * or SL-LPP with pruning).  labels_out starts as the vertex ids; every sweep
 * each vertex (with pruning: each vertex of the frontier, initially all)
 * takes the smallest labels_out value over itself and its neighbours with
 * the same labels_in value, in place; with pruning a vertex that changed
 * puts those neighbours in the next frontier.  Sweeps repeat until one
 * changes nothing.  The fixed point is the labelling gsl_split returns with
 * renumber = 0 (the smallest vertex id of every piece); the number of sweeps
 * depends on the update order and is not deterministic.
 *   labels_in   device int32[n], any values (only compared for equality).
 *   labels_out  device int32[n]; must not overlap labels_in.
 *   pruning     0: SL-LP, 1: SL-LPP.
 *   sweeps_out  optional HOST pointer receiving the sweeps run (the last one
 *               changes nothing).
 * Synchronises `stream` after every sweep (the stop test reads the change
 * count).  Errors: GSL_ERR_INVALID for bad arguments or columns;
 * GSL_ERR_TIMEOUT if more than n + 1 sweeps would be needed (cannot happen
 * on valid input). */
int gsl_split_lp(gsl_ctx* ctx, const gsl_csr* g, const int32_t* labels_in, int32_t* labels_out, int32_t pruning,
                 int32_t* sweeps_out, void* stream);

/* Disconnected communities: disconnectedCommunities() of Algorithm 4.  A
 * community (a labels value) is disconnected when the subgraph of edges
 * inside it has more than one connected piece.
 *   labels      device int32[n], values in [0, n) (else GSL_ERR_INVALID).
 *   flags_out   optional device uint8[n]: flags_out[c] = 1 for every
 *               disconnected community c, else 0.
 *   count_out   HOST pointer receiving the number of disconnected
 *               communities.
 * Uses the union-find of gsl_split; synchronises `stream`. */
int gsl_disconnected(gsl_ctx* ctx, const gsl_csr* g, const int32_t* labels, uint8_t* flags_out, int64_t* count_out,
                     void* stream);

/* Modularity, Eq. 1:  Q = sum_c [ sigma_c / 2m - (Sigma_c / 2m)^2 ], with
 * 2m the sum of all entry weights, sigma_c the weight of entries inside c
 * and Sigma_c the summed weighted degree of c's vertices.  The three sums
 * are exact integers (Sigma_c^2 summed in 128 bits) and Q is formed once in
 * double; an empty graph gives 0.
 *   labels   device int32[n], values in [0, n) (else GSL_ERR_INVALID).
 *   q_out    HOST double.
 */
int gsl_modularity(gsl_ctx* ctx, const gsl_csr* g, const int32_t* weights, const int32_t* labels,
                   double* q_out, void* stream);

/* Modularity without any allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory -- a
 * request loop that must not pay the device-wide synchronisation that
 * cudaMalloc / cudaFree can cause, or a process whose GPU memory is already
 * reserved in full by another allocator.  It needs no context and computes
 * the same value as gsl_modularity (same exact integer sums, same double
 * combine), with all scratch in one fixed device array that the library
 * reserves on every GPU that loads it (about 32 MB, until the process
 * exits).  It calls no cudaMalloc, cudaFree or other allocating routine.
 *   g, weights, labels, q_out, stream   as for gsl_modularity; the graph is
 *              on the current CUDA device.
 *   n          at most GSL_NOALLOC_MAX_N vertices; larger graphs return
 *              GSL_ERR_INVALID without touching the device.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * The call reads its sums back and waits for `stream` to finish before it
 * returns.  Every call uses the same array and clears what it needs at its
 * start, so calls whose work overlaps on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  Returns
 * GSL_ERR_INVALID for malformed input detected on the device (offsets not
 * starting at 0, decreasing or not ending at nnz; a column or label outside
 * [0, n); a weight <= 0) -- the next call starts from cleared sums -- and
 * GSL_ERR_CUDA for a runtime error of this call's own launches or copies (a
 * launch error left pending by earlier work on the thread is cleared at
 * entry). */
#define GSL_NOALLOC_MAX_N 4194304
int gsl_modularity_noalloc(const gsl_csr* g, const int32_t* weights, const int32_t* labels,
                           double* q_out, void* stream);

/* GSL-LPA: lpa() of Algorithm 3 including its final split, i.e. gsl_lpa
 * from C = [0 .. n) followed by gsl_split with renumber = 0.  labels_out
 * receives connected-community labels (smallest vertex id of each piece). */
int gsl_gsllpa(gsl_ctx* ctx, const gsl_csr* g, const int32_t* weights, double tolerance,
               int32_t max_iters, int32_t mode, int32_t* labels_out, gsl_stats* stats,
               void* stream);

/* Batched GSL-LPA: many independent graphs in one call.  The graphs are
 * packed into one CSR `g` (their disjoint union): graph k owns vertices
 * [vptr[k], vptr[k+1]) and its rows may only hold those vertices
 * (GSL_ERR_INVALID otherwise).  Every graph gets exactly what gsl_gsllpa
 * would give it alone -- its own change count, its own stop test
 * dN_k / N_k <= tolerance, its own number of sweeps -- and labels_out holds,
 * for every vertex, the smallest LOCAL vertex id (id - vptr[k]) of its
 * connected community piece.  The whole sweep loop runs as one CUDA graph
 * launch (captured on first use, replayed while the arguments are the same);
 * sweeps after every graph has stopped return at once.
 *   vptr_host       HOST int64[num_graphs+1], vptr[0] = 0, vptr[num_graphs] = n.
 *   iterations_out  optional HOST int32[num_graphs]: sweeps per graph.
 *   stats           optional. */
typedef struct gsl_batch_stats {
  int32_t num_graphs;
  int32_t pad;
  int64_t graph_launches;   /* CUDA graph launches used by the sweep loop (1) */
  float ms;                 /* device time of the call                        */
} gsl_batch_stats;
int gsl_gsllpa_batch(gsl_ctx* ctx, const gsl_csr* g, int32_t num_graphs, const int64_t* vptr_host,
                     const int32_t* weights, double tolerance, int32_t max_iters, int32_t mode,
                     int32_t* labels_out, int32_t* iterations_out, gsl_batch_stats* stats, void* stream);

/* How gsl_gsllpa_batch runs its sweep loop: 1 (default) as one CUDA graph,
 * captured on first use and replayed while the arguments repeat; 0 as
 * direct kernel launches (better when every call has a new shape, as in the
 * request server).  Results are the same. */
int gsl_ctx_set_batch_mode(gsl_ctx* ctx, int32_t use_cuda_graph);

/* ---------------------------------------------------------------------
 * Request server with continuous batching.
 *
 * Each request is one graph (HOST CSR).  The server runs `slots` workers,
 * each with its own context, CUDA stream and device buffers that stay
 * resident for the server's life.  A free worker admits the oldest waiting
 * requests that fit its buffers (admission by device memory), packs them
 * into one batch CSR on the device and runs gsl_gsllpa_batch on it; a
 * request of 2^22 entries or more keeps the GPU busy on its own and is run
 * alone through gsl_gsllpa.  Requests that arrive while batches are running
 * are admitted by the next worker to free up, so the work of different
 * requests overlaps on the GPU.  Every request gets exactly its solo
 * gsl_gsllpa result.
 * --------------------------------------------------------------------- */
typedef struct gsl_server gsl_server;

typedef struct gsl_server_config {
  int32_t device;
  int32_t slots;              /* concurrent batches (workers), 1..64                       */
  int64_t slot_vertices;      /* vertex capacity of one batch; 0: derived from free memory */
  int64_t slot_entries;       /* CSR entry capacity of one batch; 0: derived               */
  double memory_fraction;     /* share of free device memory used when deriving (0: 0.5)   */
  int32_t max_batch_graphs;   /* graphs per batch (0: 1024; at most 65535)                 */
  int32_t mode;               /* GSL_MODE_SYNC or GSL_MODE_ASYNC                           */
  double tolerance;
  int32_t max_iters;
  int32_t pad;
} gsl_server_config;

typedef struct gsl_request_info {
  int32_t status;             /* GSL_OK or an error code                                   */
  int32_t sweeps;             /* sweeps performed for this graph                           */
  int64_t batch_graphs;       /* graphs in the batch that served it                        */
  double queue_ms;            /* submit -> admitted                                        */
  double service_ms;          /* admitted -> labels on the host                            */
  double latency_ms;          /* submit -> labels on the host                              */
  /* Device time (CUDA events on the worker's stream) of the batch that
   * served the request, split into the host-to-device copies, the kernels
   * (GSL-LPA with its per-sweep host reads) and the label copy back.       */
  double h2d_ms;
  double compute_ms;
  double d2h_ms;
} gsl_request_info;

typedef struct gsl_server_stats {
  int64_t completed;
  int64_t batches;
  int64_t queued;
  int64_t max_concurrent_batches;
} gsl_server_stats;

int gsl_server_create(gsl_server** server, const gsl_server_config* config);
/* Largest graph (vertices, entries) a batch can hold. */
int gsl_server_capacity(gsl_server* server, int64_t* max_vertices, int64_t* max_entries);
/* Queues one graph.  offsets (n+1) and cols (nnz) are HOST buffers owned by
 * the caller and must stay valid until gsl_server_wait returns for it.
 * Thread safe.  GSL_ERR_NOMEM if the graph can never fit a batch. */
int gsl_server_submit(gsl_server* server, int64_t n, int64_t nnz, const int64_t* offsets, const int32_t* cols,
                      int64_t* request_id);
/* Blocks until the request is done; labels_out (HOST int32[n], nullable)
 * receives its connected-community labels.  Each id can be waited once. */
int gsl_server_wait(gsl_server* server, int64_t request_id, int32_t* labels_out, gsl_request_info* info);
int gsl_server_get_stats(gsl_server* server, gsl_server_stats* stats);
/* Finishes every queued request, stops the workers and frees all memory. */
int gsl_server_destroy(gsl_server* server);

/* gsl_gsllpa on HOST buffers: copies offsets, cols and weights (nullable) to
 * the device, runs GSL-LPA and copies the labels back to labels_out_host
 * (host int32[n]).  Device copies of the graph are context scratch.  Host
 * buffers may be pageable or pinned (pinned is faster).  Labels and
 * statistics are those of gsl_gsllpa.
 *
 * With pinned cols (cudaHostAlloc / cudaHostRegister), unit weights,
 * synchronous mode and at least gsl_ctx_set_host_overlap entries, the
 * column copy overlaps the first two sweeps.  The columns travel in
 * row-aligned chunks on a context-owned copy stream.  Sweep 1 is evaluated
 * first from each row's first entries, read by the device straight from the
 * pinned buffer, assuming every row is strictly increasing.  Each chunk is
 * then checked, and its rows swept a second time, as soon as it lands.  If a
 * row turns out not to be strictly increasing, the call redoes GSL-LPA on
 * the copied graph, so the result is the same either way.  The call returns
 * only after every copy has finished. */
int gsl_gsllpa_host(gsl_ctx* ctx, int64_t n, int64_t nnz, const int64_t* offsets_host,
                    const int32_t* cols_host, const int32_t* weights_host, double tolerance,
                    int32_t max_iters, int32_t mode, int32_t* labels_out_host, gsl_stats* stats,
                    void* stream);

/* Smallest number of CSR entries from which gsl_gsllpa_host overlaps its
 * column copy with the first two sweeps (default 2^24; 0 never; the paper
 * has no counterpart).  Results do not depend on it.  min_entries < 0:
 * GSL_ERR_INVALID. */
int gsl_ctx_set_host_overlap(gsl_ctx* ctx, int64_t min_entries);

/* Profiling.  When enabled on a context, every launch sequence of the
 * context is bracketed by CUDA events on the call's stream and its device
 * time, vertex and entry counts and algorithmic bytes are accumulated per
 * slot (frontier binning, each degree class of the sweep, union-find split,
 * piece count / renumbering, modularity, ...).  Algorithmic bytes count each
 * array element the definition has to touch once (a CSR column, a gathered
 * label, a written label), not the sectors the hardware moves.
 * gsl_ctx_set_profiling(ctx, 1) enables and zeroes the accumulators; 0
 * disables.  Enabling adds two event records per launch sequence. */
#define GSL_PROFILE_SLOTS 24
typedef struct gsl_profile_slot {
  char name[32];
  int64_t launches;   /* launch sequences timed          */
  int64_t kernels;    /* kernels in those sequences       */
  double ms;          /* summed CUDA-event device time    */
  int64_t vertices;   /* vertices processed               */
  int64_t entries;    /* CSR entries read                 */
  double bytes;       /* algorithmic bytes                */
} gsl_profile_slot;
typedef struct gsl_profile {
  int32_t nslots;
  gsl_profile_slot slot[GSL_PROFILE_SLOTS];
} gsl_profile;
int gsl_ctx_set_profiling(gsl_ctx* ctx, int32_t enable);
int gsl_ctx_get_profile(gsl_ctx* ctx, gsl_profile* out);

/* Number of CUDA kernels this library has launched in this process. */
int64_t gsl_kernel_launches(void);

/* Static message for an error code. */
const char* gsl_strerror(int code);

/* Detail of the last error on ctx ("" if none).  Valid until the next call. */
const char* gsl_ctx_last_error(gsl_ctx* ctx);

/* Library version as major*10000 + minor*100 + patch. */
int gsl_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GSLLPA_H */
