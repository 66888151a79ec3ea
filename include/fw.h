/*
 * fw.h -- C ABI of the GB300 blocked Floyd-Warshall library (libfw.so).
 *
 * Problem (Sec. 2.3 of Calderon, Rucci, Chichizola, "Enhanced OpenMP Algorithm
 * to Compute All-Pairs Shortest Path on x86 Architectures"): given a dense
 * n x n distance matrix D whose entry D[i][j] is the weight of the edge i -> j
 * (INF when there is no edge, 0 on the diagonal), compute in place the length
 * of the shortest i -> j path for every pair, and a matrix P that records the
 * paths.  The blocked schedule (Sec. 2.3, Fig. 2: R = ceil(n/BS) rounds of pivot
 * block, pivot row/column blocks, remaining blocks) and the intra-round
 * concurrency of Opt-9 (Sec. 3.2) are realised on the GPU by the kernels
 * behind these calls; the library form itself is the reusable library the paper
 * lists as future work (Sec. 5).
 *
 * Conventions shared by every entry point
 *   - Matrices are row-major with leading dimension ld >= n (elements).  Rows
 *     must start on 16-byte boundaries: the base pointer is 16-byte aligned and
 *     ld is a multiple of 4.  Entries in columns [n, ld) are never read or
 *     written.
 *   - int32 path: a missing edge is FW_INF_I32 = 2^29; weights are in
 *     [0, FW_INF_I32) and every simple path is shorter than FW_INF_I32, i.e.
 *     (n-1) * max_weight < 2^29.  Results for unreachable pairs are exactly
 *     FW_INF_I32.  int64 path: the same with FW_INF_I64 = 2^61.  fp32 and
 *     fp64 paths: a missing edge is +inf; no NaN.
 *   - D[i][i] must be 0 on entry and weights must be >= 0; results for
 *     negative weights are undefined, except that a negative diagonal entry
 *     seen during the solve is reported as FW_ERR_NEG_CYCLE.
 *   - Predecessors: pred[i][j] is the LAST HOP of the chosen shortest i -> j
 *     path (the vertex just before j), -1 on the diagonal and for unreachable
 *     pairs.  The paper's P stores the intermediate vertex k and compares with
 *     ">="; this library relaxes only on a strict improvement and stores the
 *     last hop, which makes pred independent of the blocked visiting order on
 *     every pair whose shortest path is unique.  Where several shortest paths
 *     exist, pred is the last hop of one of them.  While an int32 solve runs,
 *     pred also holds intermediate entries (values <= -2); the final values
 *     are in place once the stream has passed the call's last kernel.
 *   - Device calls are asynchronous and stream-ordered on `stream` (a
 *     cudaStream_t; NULL is the legacy default stream).  Argument errors are
 *     detected on the host and returned before anything is launched.  Errors
 *     found on the device (a dependency wait that timed out, a negative cycle)
 *     are recorded in the status word of the stream's workspace, which
 *     fw_sync_status reads.
 *   - The library owns a workspace per (device, stream): tile flags, panel
 *     snapshots and the status word.  It is allocated on first use with
 *     cudaMalloc, grows when a larger problem arrives, and is freed by
 *     fw_release_workspace.  Two solves in flight on the same stream share it
 *     safely (stream order); solves on different streams use different
 *     workspaces.  Allocation cannot happen during CUDA-graph capture: run one
 *     solve of the largest size on the stream before capturing.
 *   - Thread safety: every entry point may be called from several host threads
 *     on different streams.
 */
#ifndef FW_GB300_H
#define FW_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FW_INF_I32 (1 << 29)
#define FW_INF_I64 (1LL << 61)

/* Element type of dist.  FW_I32 / FW_F32: the hot path (DPX packed keys for
 * int32).  FW_I64 / FW_F64: the paper's double-precision runs (Sec. 4, float
 * and double) and 64-bit integer weights; fw_solve, fw_solve_ex and
 * fw_solve_host take them, with BS 32 or 64 (three 128 x 128 tiles of 8-byte
 * elements do not fit in one SM's shared memory); the batched, backward,
 * allocation-free and certificate entry points return FW_ERR_UNSUPPORTED. */
typedef enum { FW_I32 = 0, FW_F32 = 1, FW_I64 = 2, FW_F64 = 3 } fw_dtype;

typedef enum {
  FW_OK = 0,
  FW_ERR_ARG = 1,          /* invalid argument (NULL, n <= 0, ld < n, misaligned, bad option) */
  FW_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  FW_ERR_TIMEOUT = 3,      /* a device-side dependency wait exceeded its bound */
  FW_ERR_NEG_CYCLE = 4,    /* some D[i][i] < 0 after the solve */
  FW_ERR_NOMEM = 5,        /* device or pinned-host allocation failed */
  FW_ERR_UNSUPPORTED = 6   /* dtype or size not supported by this entry point */
} fw_status;

typedef enum {
  FW_DRIVER_AUTO = 0,       /* persistent driver */
  FW_DRIVER_PERSISTENT = 1, /* one cooperative launch; tiles scheduled by ready flags */
  FW_DRIVER_PHASED = 2      /* one launch per phase per round (pivot, panels, remaining) */
} fw_driver;

typedef struct fw_options {
  int32_t bs;                 /* block size BS (Sec. 2.3): 0 = automatic (32 up to n = 512,
                                 64 up to 3072, else 128), else 32, 64 or 128 */
  int32_t driver;             /* fw_driver */
  int32_t lookahead;          /* persistent driver: remaining-block tasks of round r queued
                                 between the pivot and the panels of round r+1; -1 = automatic
                                 (six per CTA, fewer when a round has few tasks) */
  int32_t grid;               /* persistent driver: CTAs; 0 = every co-resident CTA */
  int64_t timeout_ns;         /* bound on one device-side dependency wait; 0 = 2 s */
  int32_t packed_keys;        /* int32 only: 1 (default) relaxes packed (distance, pivot) keys
                                 when the tile bounds allow it, 0 = always the generic kernel */
  int32_t debug_skip_release; /* >= 0: the persistent driver never publishes the completion of
                                 this task index, so that its dependents time out; -1 = off */
  void* ev_start;             /* optional cudaEvent_t recorded just before the solver kernels */
  void* ev_stop;              /* optional cudaEvent_t recorded just after them (before the
                                 int32 solve's final predecessor-resolution pass) */
  uint64_t* trace;            /* optional device buffer of trace_cap x 10 uint64: a %globaltimer
                                 timeline of every trace_stride-th task of the persistent driver
                                 (claim, inputs ready, operands issued, published; compute start
                                 and end), the GPU view of the idle time Opt-9 targets (Sec. 4.3).
                                 Min-plus tasks add SM-cycle counts: column 7 = tile-load wait |
                                 operand-chunk waits << 20 | predecessor-tile wait << 40 (20 bits
                                 each, saturating), column 8 = cycles from task start to the end
                                 of the relaxation | whole task << 32.  Pivot and panel tasks:
                                 column 7 = operands loaded | relaxed << 32, column 8 = results
                                 stored | whole task << 32 (SM cycles from the task's start).
                                 Column 0 = task | type << 32 | graph << 40, type 0-3 as in
                                 fw_queue_tasks and 4 for remaining tile (r+1, r+1) of round r
                                 run together with the pivot of round r+1 (that pivot's own
                                 entry is then skipped and not traced) */
  int64_t trace_cap;
  int32_t trace_stride;
  int32_t tile_tma;           /* persistent driver: 1 (default) loads each remaining or panel
                                 tile with one 2-D TMA tensor copy, 0 = one bulk copy per row */
  uint64_t debug_shuffle;     /* batched plans: nonzero = a seed; the plan's claim order is
                                 permuted at random inside each wave segment (one phase of one
                                 round of every graph: tasks none of which depends on another),
                                 a stress of the dependency protocol under other orders of the
                                 same tasks; 0 = off (the planned order).  Single solves ignore
                                 it (their queue order is computed on the device) */
} fw_options;

/* Fills *opt with the defaults used by fw_solve. */
void fw_options_default(fw_options* opt);

/* Human-readable name of a status code (static storage). */
const char* fw_status_string(fw_status s);

/*
 * fw_solve: all-pairs shortest paths of one graph, in place (Sec. 2.3, the
 * blocked algorithm of Sec. 2.3, Fig. 2).
 *   dist  device pointer, n x ld, dtype elements; holds the weights on entry
 *         and the distances on exit.
 *   pred  device pointer, n x ld int32, output only (may not alias dist); NULL
 *         for a distance-only solve (no predecessor work at all; fp32 then
 *         relaxes with an add and a min per step and keeps no argmin).
 *   n     vertices, 1 <= n <= 131072.   ld  leading dimension, ld >= n, ld % 4 == 0.
 *   dtype FW_I32, FW_F32, FW_I64 or FW_F64.
 * Returns FW_OK once the work is enqueued; FW_ERR_UNSUPPORTED for BS = 128
 * with a 64-bit dtype (automatic BS for them: 32 up to n = 512, else 64).
 */
fw_status fw_solve(void* dist, int32_t* pred, int64_t n, int64_t ld, fw_dtype dtype, void* stream);

/* fw_solve with explicit options (opt may be NULL for the defaults). */
fw_status fw_solve_ex(void* dist, int32_t* pred, int64_t n, int64_t ld, fw_dtype dtype,
                      const fw_options* opt, void* stream);

/*
 * fw_solve_host: the same solve on HOST buffers.  dist_host (n x ld, dtype)
 * is copied to the device, solved, and dist_host / pred_host (n x ld int32)
 * receive the results (pred_host NULL: distances only); the columns n..ld-1
 * of the host buffers are neither read nor written.  Pinned host memory
 * gives full copy bandwidth; pageable
 * memory works too.  Synchronous: returns after the results are on the host,
 * with any device-side error (as fw_sync_status would report it).  Device
 * buffers are cached per (device, stream) like the workspace.  The distances
 * are copied back on an internal stream as soon as they are final, while the
 * int32 solve's predecessor pass still runs; opt->ev_stop, when given, is the
 * event that marks that point.
 */
fw_status fw_solve_host(void* dist_host, int32_t* pred_host, int64_t n, int64_t ld,
                        fw_dtype dtype, const fw_options* opt, void* stream);

/*
 * fw_solve_host_io: fw_solve_host with the weights in their own host buffer:
 * w_host (n x ld, dtype) is copied to the device and left unchanged, and the
 * distances go to dist_host (n x ld, dtype), the predecessors to pred_host
 * (NULL: distances only).  dist_host == w_host is the in-place fw_solve_host;
 * any other overlap of the buffers is not allowed.  A caller that solves
 * the same or new weights again needs no copy of them to restore the input,
 * and the results land in buffers that the host has not just rewritten
 * (copies into host memory the CPU has just written ran up to 5x slower on
 * GB300).  FW_ERR_ARG for a null w_host or dist_host, and as fw_solve_host.
 */
fw_status fw_solve_host_io(const void* w_host, void* dist_host, int32_t* pred_host, int64_t n,
                           int64_t ld, fw_dtype dtype, const fw_options* opt, void* stream);

/*
 * Batched solve of many independent graphs of different sizes in one
 * persistent launch (graphs interleave in one task queue; BS is chosen per
 * size class).  The plan fixes the sizes and leading dimensions; its device
 * tables and workspace are allocated at creation, so fw_solve_batched itself
 * allocates nothing and can be captured into a CUDA graph.
 *   n[b], ld[b]  vertex count and leading dimension of graph b (same rules as
 *                fw_solve), 0 <= b < batch, 1 <= batch <= 65536.
 *   opt->bs      0 = per-size-class choice (autotuned table), else a fixed BS.
 *   opt->trace   optional task trace of every solve with this plan (as for
 *                fw_solve_ex; the global task index is the position in the
 *                plan's interleaved list, and word 0 also carries the graph
 *                index in bits 40-63).
 */
typedef struct fw_batched_plan fw_batched_plan;

fw_status fw_batched_plan_create(fw_batched_plan** plan, const int64_t* n, const int64_t* ld,
                                 int64_t batch, fw_dtype dtype, const fw_options* opt);

/* dist[b], pred[b]: HOST arrays of device pointers (batch entries each); pred
 * NULL (or a NULL entry) solves for distances only.  A plan has one workspace
 * and one recorded launch sequence, so its solves must not overlap on the
 * GPU: issue them on one stream (stream order keeps them apart), or let the
 * previous solve finish (e.g. synchronize its stream) before solving with the
 * same plan on another stream.  Solves with different plans are independent. */
fw_status fw_solve_batched(fw_batched_plan* plan, void* const* dist, int32_t* const* pred,
                           void* stream);

/* Block size chosen for graph b, and the total number of tasks in the queue. */
fw_status fw_batched_plan_info(const fw_batched_plan* plan, int32_t* bs_per_graph,
                               int64_t* total_tasks);

fw_status fw_batched_plan_destroy(fw_batched_plan* plan);

/*
 * fw_batched_task_list: diagnostic view of the claim order a batched plan
 * uses for `batch` graphs of n[b] vertices and block sizes bs[b] (32, 64 or
 * 128) on a GPU with `sms` CTAs, with opt->debug_shuffle applied (opt NULL:
 * defaults, no shuffle).  Writes two int32 per task -- the graph, and the
 * task's index in that graph's queue as fw_queue_tasks numbers it -- for all
 * sum_b ceil(n[b] / bs[b])^3 tasks; *count gets that total.  Host only.
 * FW_ERR_ARG for a NULL pointer, batch outside [1, 65536], sms < 1, an n
 * outside [1, 131072], another block size, or cap (rows of out) below the
 * total; FW_ERR_UNSUPPORTED when a graph would have over 1024 rounds.
 */
fw_status fw_batched_task_list(const int64_t* n, const int32_t* bs, int64_t batch, int32_t sms,
                               const fw_options* opt, int32_t* out, int64_t cap, int64_t* count);

/*
 * Block-size table of the batched planner for element type dtype (FW_I32 or
 * FW_F32; used when opt->bs == 0): one entry per size class n <= 128, 256,
 * 512, 1024, 2048, 4096, larger (7 entries), each 32, 64 or 128.  set != 0
 * writes `table`, set == 0 reads it into `table`.  The paper's BS sweep
 * (Sec. 4, Tables 2-3) is the motivation: the best block size depends on the
 * problem size (and here on the element type).  The defaults are
 * fw_autotune_bs's choices on a GB300.  FW_ERR_ARG for a null table, another
 * dtype or an entry outside {32, 64, 128}; FW_ERR_UNSUPPORTED for the 64-bit
 * types (no batched path).
 */
fw_status fw_bs_table(fw_dtype dtype, int32_t* table, int32_t set);

/*
 * fw_autotune_bs: measures, for every size class up to max_n, a batched solve
 * of graphs_per_class synthetic graphs of the class's largest size with BS =
 * 32, 64 and 128, stores the fastest BS of each class in dtype's table and copies
 * the table to table_out (7 entries) and the best times in ms to ms_out (may
 * be NULL).  Classes above max_n keep their entries.  Synchronous; allocates
 * its own inputs.
 */
fw_status fw_autotune_bs(fw_dtype dtype, int64_t graphs_per_class, int64_t max_n, void* stream,
                         int32_t* table_out, double* ms_out);

/*
 * fw_backward: gradient of a scalar loss L through the fp32 distances.  Given
 * grad_dist = dL/dD, the forward result dist and its predecessors pred, writes
 * grad_w = dL/dW, where W is the weight matrix the forward solve received:
 *   dL/dW[u][v] = sum over pairs (i, j) whose recorded path i -> j uses the
 *                 edge u -> v of dL/dD[i][j].
 * The path of (i, j) is the one recorded by pred (a subgradient where shortest
 * paths are not unique).  grad_w is 0 on non-edges, non-tree edges and the
 * diagonal; dL/dD on the diagonal and on unreachable pairs is ignored.  Not
 * part of the paper; it makes the solve usable inside a training graph.
 * All pointers are device memory, n x ld (grad_w fully overwritten on [0,n)^2).
 */
fw_status fw_backward(const float* grad_dist, const float* dist, const int32_t* pred,
                      float* grad_w, int64_t n, int64_t ld, void* stream);

/* fw_backward over `batch` graphs of the same n stored `stride` elements apart. */
fw_status fw_backward_strided(const float* grad_dist, const float* dist, const int32_t* pred,
                              float* grad_w, int64_t n, int64_t ld, int64_t batch,
                              int64_t stride, void* stream);

/*
 * fw_sync_status: waits for `stream`, then returns and clears the sticky
 * device-side status recorded by solves on this (device, stream) pair
 * (FW_ERR_TIMEOUT, FW_ERR_NEG_CYCLE), or FW_ERR_CUDA when the stream reports a
 * CUDA error.
 */
fw_status fw_sync_status(void* stream);

/* Frees every cached workspace of the calling thread's current device. */
fw_status fw_release_workspace(void);

/*
 * fw_peak_probe: measures the min-plus relaxation peak of this GPU at its
 * current clocks with register-resident relaxation chains on every SM (the
 * same instruction the solver's inner loop issues: __viaddmin for int32,
 * add + min for fp32, fp64 and int64).  Outputs relaxations per second, relaxations per SM
 * clock cycle (clock-independent) and the average SM clock in MHz seen by the
 * probe.  Synchronous.  Not part of the paper: it provides the roofline.
 */
fw_status fw_peak_probe(fw_dtype dtype, double* relax_per_s, double* relax_per_sm_clk,
                        double* sm_mhz, void* stream);

/*
 * fw_verify_certificate: GPU check of the LP-duality certificate of exact
 * int32 shortest distances (the checks a correct solve must pass at any size):
 *   bad[0] D[i][i] != 0;  bad[1] a reachable (i, j) whose pred is not a tight
 *   last hop (D[i][p] + W[p][j] != D[i][j] or no edge p -> j);  bad[2] an edge
 *   u -> v with D[i][v] > D[i][u] + W[u][v];  bad[3] pred set on the diagonal
 *   or an unreachable pair, or missing on a reachable one.
 * W, dist, pred: device, n x ld.  bad: HOST array of 4 int64.  Synchronous.
 * It shares no code with the solver kernels.
 */
fw_status fw_verify_certificate(const int32_t* W, const int32_t* dist, const int32_t* pred,
                                int64_t n, int64_t ld, int64_t* bad, void* stream);

/*
 * fw_solve_noalloc: fw_solve for callers that cannot allocate device memory.
 * There is no counterpart in the paper; it exists for integrators.
 *
 * fw_solve obtains its workspace with cudaMalloc.  Callers that run under a
 * device-memory budget owned by another allocator (a framework's caching pool,
 * a server that reserved all free memory up front), or that cannot afford the
 * device-wide synchronisation cudaMalloc may imply, use this entry point: it
 * calls no cudaMalloc, cudaFree or other allocating routine.  Its workspace is
 * one static device array of 12 MiB inside the library, which every GPU that
 * loads the library's kernels holds until the process exits.
 *
 *   dist, pred, ld, dtype  as for fw_solve (device pointers, caller-owned).
 *   n                      1 <= n <= 4096; larger n returns FW_ERR_UNSUPPORTED
 *                          (use fw_solve).  BS is 32 for n <= 512, else 64.
 *   stream                 the solve is enqueued on it and waited for.
 * Synchronous: returns after the solve has finished, with FW_OK or the
 * device-side error (FW_ERR_TIMEOUT, FW_ERR_NEG_CYCLE) of this call.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress with that device current) and caches it; make that
 * first call before any stream capture on the device.  The cached address
 * does not survive cudaDeviceReset: calls after a reset of the device are not
 * supported.  Every call, from any
 * thread or stream, uses the same array and clears the parts that must start
 * at zero; calls whose executions overlap on the GPU race on it and produce
 * wrong results, so serialise them (one at a time per device).
 */
fw_status fw_solve_noalloc(void* dist, int32_t* pred, int64_t n, int64_t ld, fw_dtype dtype,
                           void* stream);

/*
 * fw_paths: the shortest paths that a solved predecessor matrix records
 * (Sec. 2.3: P lets the paths be rebuilt), for a batch of (source, target)
 * pairs, on the GPU.  pred: device, n x ld int32, as a solve with
 * predecessors leaves it (last hops, -1 where there is none).  src, dst:
 * device arrays of npairs vertex ids.  out: device, npairs x max_len int32;
 * row q receives the vertices of the path from src[q] to dst[q] in order
 * (src[q] first, dst[q] last).  len: device, npairs int32: the vertex count
 * of each path (1 when src == dst), 0 when dst is unreachable from src, -1
 * when an id is outside [0, n), the path has more than max_len vertices, or
 * pred is not a tree of last hops (a walk would leave [0, n) or take more
 * than n vertices); out row q is then unspecified.  Every walk is bounded by
 * n hops.  Asynchronous on stream; FW_ERR_ARG for null pointers, n outside
 * [1, 131072], ld < n, npairs < 0 or max_len < 1.
 */
fw_status fw_paths(const int32_t* pred, int64_t n, int64_t ld, const int32_t* src,
                   const int32_t* dst, int64_t npairs, int32_t* out, int64_t max_len,
                   int32_t* len, void* stream);

/*
 * fw_intermediate: the path matrix in the bookkeeping of the paper's Fig. 1
 * (Sec. 2.3), where P_ij is the intermediate vertex k through which (i, j)
 * last improved.  For every pair, out[i][j] = the largest vertex strictly
 * between i and j on the path that the last-hop matrix pred records; -1 on
 * the diagonal, for a path that is a single edge, for an unreachable pair
 * (pred -1) and where pred does not lead back to the source.  On a pair with
 * a unique shortest path this is exactly the k of Fig. 1's last improvement
 * (strict "<"); with several shortest paths it is the largest intermediate
 * of the recorded one, and a path rebuilds recursively from it: the paths
 * i -> k and k -> j joined at k.
 * pred: device, batch matrices of n x ld int32 (a solve's last hops), matrix
 * b at pred + b * stride.  out: device, same layout; out == pred (in place)
 * is allowed, a partial overlap is not.  Asynchronous on stream.  FW_ERR_ARG
 * for null pointers, n < 1, ld < n, batch < 0, stride < n * ld when
 * batch > 1, or batch * n >= 2^31; FW_ERR_UNSUPPORTED for n > 57344 (the
 * kernel keeps 4 bytes per vertex of a row in shared memory); batch = 0 is a
 * no-op.
 */
fw_status fw_intermediate(const int32_t* pred, int32_t* out, int64_t n, int64_t ld,
                          int64_t batch, int64_t stride, void* stream);

/*
 * fw_solve_plan: what fw_solve_ex would choose for n vertices of element type
 * dtype and *opt (NULL: defaults) on a GPU with `sms` co-resident CTAs (one
 * per SM): the block size
 * BS, the number of rounds R = ceil(n / BS) (Sec. 2.3), the lookahead of the
 * persistent queue, and the bytes of device workspace it keeps per (device,
 * stream) besides the caller's matrices (tile versions, queue offsets, pivot
 * and panel snapshots).  Any output pointer may be NULL.  Host only: no CUDA
 * call.  FW_ERR_ARG for n outside [1, 131072], sms < 1, an invalid dtype or
 * invalid options; FW_ERR_UNSUPPORTED when R would exceed 1024 or a 64-bit
 * dtype is given BS = 128 (as fw_solve_ex).
 */
fw_status fw_solve_plan(int64_t n, fw_dtype dtype, const fw_options* opt, int32_t sms,
                        int32_t* bs, int32_t* rounds, int64_t* lookahead,
                        int64_t* workspace_bytes);

/*
 * fw_queue_tasks: diagnostic view of the persistent driver's task queue for R
 * tile rows (R = ceil(n / BS)) and a given lookahead (the value fw_options
 * .lookahead resolves to).  Writes 4 int32 per task -- type (0 pivot, 1 row
 * panel, 2 column panel, 3 remaining tile), round, tile row, tile column --
 * for the tasks [first, first + count) of the R^3 in the queue.  Host only.
 */
fw_status fw_queue_tasks(int32_t R, int64_t lookahead, int64_t first, int64_t count, int32_t* out);

/*
 * Tile-level calls of the blocked algorithm (Sec. 2.3, Fig. 2), for callers
 * that keep a matrix in pieces -- the single-graph solve spread over several
 * GPUs (2-D block-cyclic tiles, one exchange of pivot and panels per round;
 * the exchange is the caller's).  All matrices are tile-PADDED: whole
 * bs x bs tiles, padding vertices isolated (INF off the diagonal, 0 on it);
 * pointers 16-byte aligned, leading dimensions multiples of 4, dtype as for
 * fw_solve, bs 32, 64 or 128 (64-bit dtypes: 32 or 64).  Predecessors are
 * last hops in global vertex ids; pred pointers may be NULL together (a
 * distance-only solve).  Asynchronous on stream.
 *
 * fw_tile_closure: phase 1 -- the in-place strict-< FW closure of the
 * bs x bs tile at `tile` (leading dimension ld) and its predecessors `pred`
 * (same ld).  A negative diagonal entry is recorded in the stream's status
 * word (fw_sync_status returns FW_ERR_NEG_CYCLE).
 */
fw_status fw_tile_closure(void* tile, int32_t* pred, int64_t ld, int32_t bs, fw_dtype dtype,
                          void* stream);

/*
 * fw_tile_minplus: phases 2 to 4 -- for every output tile (i, j), 0 <= i <
 * tiles_m, 0 <= j < tiles_n, of C (leading dimension ldc):
 *     C_ij = min(C_ij, A_i (x) B_j),   (x) the min-plus product over bs steps,
 * with A_i the bs x bs block (i, 0) of A (lda) and B_j the block (0, j) of B
 * (ldb).  Where the entry strictly improves through step kk, Pc (leading
 * dimension ldc) takes Pb[kk][column] (Pb: bs rows, leading dimension ldpb),
 * the last hop of B's row kk.  With a closed pivot tile as A (row panel, B =
 * C, Pb = Pc) or as B (column panel, A = C, Pb = the pivot's predecessors)
 * this is the in-place panel update; with the column panel as A and the row
 * panel as B it is the update of the remaining tiles.  C may be the same
 * memory as A only when tiles_n == 1 and as B only when tiles_m == 1 (each
 * output tile then reads exactly itself); any other overlap returns
 * FW_ERR_ARG.  Tiles in tile row skip_tile_row or tile column skip_tile_col
 * (-1: none) are not touched.  tiles_m <= 65535.
 */
fw_status fw_tile_minplus(void* C, int32_t* Pc, int64_t ldc, const void* A, int64_t lda,
                          const void* B, int64_t ldb, const int32_t* Pb, int64_t ldpb,
                          int64_t tiles_m, int64_t tiles_n, int32_t bs, int64_t skip_tile_row,
                          int64_t skip_tile_col, fw_dtype dtype, void* stream);

/*
 * fw_block_init_pred: the initial predecessors (Sec. 2.3 leaves them open:
 * the row's vertex on an edge, -1 elsewhere) of a rows x cols local block of
 * a block-cyclic layout.  Local row a is global vertex (row_tile0 + (a / bs) *
 * row_tile_step) * bs + a % bs, columns likewise; entries whose global row or
 * column is >= n (padding) get -1.  dist and pred: leading dimension ld.
 */
fw_status fw_block_init_pred(const void* dist, int32_t* pred, int64_t ld, int64_t rows,
                             int64_t cols, int32_t bs, int64_t n, int64_t row_tile0,
                             int64_t row_tile_step, int64_t col_tile0, int64_t col_tile_step,
                             fw_dtype dtype, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FW_GB300_H */
