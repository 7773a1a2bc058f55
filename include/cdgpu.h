/*
 * cdgpu — community detection (Label Propagation and Louvain) on one GPU.
 *
 * C ABI of libcdgpu.so. Every call takes plain pointers and sizes; a flag
 * says whether a caller buffer lives in host or device memory. All device
 * work of a graph runs on the CUDA stream given at upload, in the order the
 * calls are made; every call returns after its results are valid in the
 * caller's buffers.
 *
 * Method (arXiv 2507.06471, "Designing Parallel Algorithms for Community
 * Detection using Arachne"):
 *   - graph model, weighted degree, volume, cut: Sec. II-A
 *   - modularity and the move gain (Eq. deltaQ): Sec. II-C
 *   - Label Propagation: Algorithm 1 (PLP / PLPMove), Sec. III-A
 *   - Louvain local moving: Algorithm 2, Sec. III-B-1
 *   - Louvain aggregation and driver: Algorithm 3, Sec. III-B-2
 *
 * Schedule (fixed so that results are reproducible bit for bit; the paper's
 * Chapel loops are asynchronous): rounds are synchronous — every decision
 * reads the labels and community volumes of the start of the round, then all
 * moves apply at once. A vertex whose decision differs from its label commits
 * the move in round r of level l only if bit 63 of SplitMix64 draw number
 * (l << 48 | r << 32 | v) from state `sched_seed` is set, else it defers to
 * the next round (it stays active). Louvain moves need a strictly positive
 * gain, ties go to the smallest community id, and a singleton joins another
 * singleton only if that one has the smaller id. LPA keeps the current label
 * when it attains the maximum weight, else takes the smallest maximal label.
 * The next round examines the moved vertices, their neighbours and the
 * deferred vertices.
 *
 * Graph input convention: a symmetric CSR. A non-loop edge {u,v} of weight w
 * is the two arcs u->v and v->u, each carrying w; a loop of weight L on v is
 * the single arc v->v carrying L (deg_w counts it twice, Sec. II-A). Vertex
 * ids are int32 in [0, n); weights are int32 >= 1, or NULL for unit weights.
 */
#ifndef CDGPU_H
#define CDGPU_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* Status codes: 0 on success, a negative code otherwise. */
#define CD_OK 0
#define CD_EINVAL (-1)    /* null pointer, bad size, weight < 1, bad label   */
#define CD_EBOUNDS (-2)   /* a column id outside [0, n)                      */
#define CD_ENOMEM (-3)    /* device allocation failed                        */
#define CD_ECUDA (-4)     /* a CUDA runtime error (see cd_last_cuda_error)   */
#define CD_EOVERFLOW (-5) /* vol(V) >= 2^62 or n >= 2^31                     */
#define CD_ETIMEOUT (-6)  /* a bounded device wait ran out                   */
#define CD_ENOTSYM (-7)   /* offsets not monotone / arcs not paired          */

typedef struct cd_graph cd_graph; /* opaque; owns a device copy of the CSR */

typedef struct cd_params {
  int32_t max_iter;         /* rounds at most: per call (LPA) or per level (Louvain); default 100 */
  int32_t max_levels;       /* Louvain levels at most; default 64 */
  int64_t threshold;        /* LPA stops after a round with moved + deferred <= threshold; default 0 */
  int32_t tie_keep_current; /* LPA tie rule: 1 keep the current label on a tie (default), 0 smallest */
  int32_t singleton_rule;   /* Louvain: 1 (default) singleton joins only a smaller-id singleton */
  int32_t use_frontier;     /* 1 (default): examine only flagged vertices; 0: all, every round */
  int32_t timing;           /* 0: none; 2: CUDA-event times per round (trace scan_ms/round_ms),
                               kernels of different degree bins still run concurrently;
                               1: per round and per kernel (trace and profile), the bins'
                               kernels then run one after another so each event pair
                               brackets one kernel alone */
  uint64_t sched_seed;      /* state of the deferral coin's SplitMix64 stream; default 0x5EED5EED */
  int32_t aggregation;      /* Louvain aggregation: 0 hash-combine per community (default), 1 radix sort
                               of all arcs; the coarse graphs have the same rows either way */
  int32_t asynchronous;     /* 1: the asynchronous variant (Sec. III-A-2, Sec. III-B-1): a committed move
                               takes effect at once and later decisions of the same round may see it
                               (the deferral coin still applies: without it adjacent vertices swap
                               labels in lockstep); results vary from run to run. 0 (default):
                               synchronous rounds, reproducible */
  int32_t device_loop;      /* Where the round loop runs. 1 (default): in batched runs (cd_batch_*) the
                               rounds after the first of a run or Louvain level run as one captured CUDA
                               graph (a conditional WHILE node whose body is one round; the round number,
                               the stop tests and the trace stay on the device), so a level costs one
                               graph launch and no per-round host synchronisation; other runs keep the
                               host loop (building a graph per level costs more than the few round trips
                               of a small graph saves). 2: every run uses the device loop. 0: the host
                               loop everywhere (one read-back per round). Results are identical in every
                               mode; timing != 0 always uses the host loop (it records per-round events) */
} cd_params;

/* Per-round record of the last run on a graph (cd_trace_get). */
typedef struct cd_round_trace {
  int32_t level;    /* Louvain level (0 for LPA) */
  int32_t round;    /* round within the level */
  int64_t active;   /* vertices examined */
  int64_t arcs;     /* arcs scanned = sum of row lengths of examined vertices */
  int64_t moved;    /* vertices that changed label */
  int64_t deferred; /* vertices whose move was deferred by the coin */
  float scan_ms;    /* device time of the scan kernels (timing != 0) */
  float round_ms;   /* device time of the whole round (timing != 0) */
  int64_t cands;    /* candidate pairs: distinct neighbour labels (own one included) summed over examined vertices */
  int64_t moved_arcs; /* arcs of the vertices that moved (their neighbours are flagged) */
} cd_round_trace;

/* Per-kernel totals of the last run (cd_profile_get; timing = 1). One entry per
 * launch group: ingest, scan_tile4/8/16/32, scan_warp, scan_blk128, scan_blk512
 * (the degree bins' scans; round 0 of a run is counted under its bin),
 * hub_prepare (hub-table compactions, clears and routing), hub_build (hub-table
 * builds), hub_eval, hub_mark (flags and logged hub-histogram updates of
 * committed moves), apply_moves, frontier, renumber, agg_emit, radix_sort,
 * agg_reduce, modularity. */
typedef struct cd_kernel_profile {
  char name[32];
  int64_t launches;
  double total_ms;  /* sum of CUDA-event durations of its launches */
  double alg_bytes; /* algorithmic bytes moved by all its launches */
} cd_kernel_profile;

/* Fill *p with the defaults listed above. */
int cd_params_default(cd_params* p);

/* Sec. II-A: copy a symmetric CSR into library-owned device memory,
 * validate it (columns in range, offsets monotone, weights >= 1) and compute
 * deg_w(v) (loops counted twice) and vol(V). offsets has n+1 entries (int64
 * if offsets_is_i64, else int32) with offsets[0] = 0 and offsets[n] = nnz;
 * cols has nnz int32 entries; w has nnz int32 entries or is NULL (unit
 * weights). ptrs_on_device says whether the three arrays are device (1) or
 * host (0) pointers; the caller keeps ownership of them. stream is a
 * cudaStream_t (NULL = the legacy default stream). *out receives the handle.
 * Errors: CD_EINVAL, CD_EBOUNDS, CD_ENOTSYM, CD_EOVERFLOW, CD_ENOMEM, CD_ECUDA. */
int cd_csr_upload(const void* offsets, int offsets_is_i64, const int32_t* cols,
                  const int32_t* w, int64_t n, int64_t nnz, int ptrs_on_device,
                  void* stream, cd_graph** out);

/* Release a handle and all device memory it owns. NULL is accepted. */
int cd_graph_free(cd_graph* g);

/* Sizes of a handle: vertices, arcs, vol(V). Any output may be NULL. */
int cd_graph_info(const cd_graph* g, int64_t* n, int64_t* nnz, int64_t* vol);

/* Copy the CSR of a handle out in the input convention (a loop arc carries
 * L). off: n+1 int64, cols: nnz int32, w: nnz int64 (may be NULL).
 * Coarse graphs from cd_louvain_aggregate have rows grouped by vertex but
 * columns in no particular order. */
int cd_graph_download(const cd_graph* g, int64_t* off, int32_t* cols, int64_t* w,
                      int ptrs_on_device);

/* Algorithm 1 (PLP): labels start as vertex ids; rounds run until
 * moved + deferred <= threshold or max_iter rounds. labels_out: n int32
 * (host or device per on_device). *rounds_out (may be NULL) = rounds run. */
int cd_lpa_run(cd_graph* g, const cd_params* p, int32_t* labels_out, int on_device,
               int32_t* rounds_out);

/* Algorithm 2 (local moving) on g. If init_given is 0 the partition starts as
 * singletons (comID = vertex id), else from labels_io (n int32 in [0, n)).
 * Runs until a round in which no vertex moves or defers, or max_iter rounds;
 * uses coin level 0. labels_io receives comID. *moves_out (may be NULL) =
 * total moves; *rounds_out (may be NULL) = rounds run. */
int cd_louvain_local_move(cd_graph* g, const cd_params* p, int32_t* labels_io, int init_given,
                          int on_device, int64_t* moves_out, int32_t* rounds_out);

/* Algorithm 3, Aggregation: remap the communities of `labels` (n int32 in
 * [0, n)) to 0..k-1 in ascending id order and build the coarse graph in which
 * edge {A,B} carries the summed weight of the edges between A and B (a loop
 * {A,A} carries A's internal weight). *coarse_out receives a new handle on
 * the same stream; newid_out (n int32, may be NULL) receives the new id of
 * every community id (-1 if unused); *k_out = k. */
int cd_louvain_aggregate(cd_graph* g, const int32_t* labels, int on_device, cd_graph** coarse_out,
                         int32_t* newid_out, int64_t* k_out);

/* Sec. II-C: modularity of `labels` (n int32 in [0, n)) on g, exact in
 * integers: Q = (I vol - sum_c vol(c)^2) / vol^2 with I = sum of the arc
 * weights inside communities (loops twice); the quotient is taken in FP64.
 * Q = 0 when vol(V) = 0. */
int cd_modularity(cd_graph* g, const int32_t* labels, int on_device, double* q_out);

/* Algorithm 3 (Louvain): local moving (coin level = level index) and
 * aggregation until a level ends with every vertex in its own community, or
 * max_levels levels. labels_out: n int32, the final community of every input
 * vertex, contiguous ids. *levels_out and *q_out (modularity on g) may be
 * NULL. */
int cd_louvain_run(cd_graph* g, const cd_params* p, int32_t* labels_out, int on_device,
                   int32_t* levels_out, double* q_out);

/* Batched mode (Algorithms 1-3 applied to many graphs at once). Declare that
 * g is n_graphs independent graphs packed block-diagonally: graph b owns the
 * vertices [vstart[b], vstart[b+1]) (vstart: n_graphs+1 int64, vstart[0] = 0,
 * vstart[n_graphs] = n, host or device per on_device) and no arc may leave
 * its block (CD_EINVAL otherwise). The cd_batch_* calls then solve every
 * graph exactly as a solo run of that graph would (same labels): gains use
 * the graph's own vol(V), the deferral coin uses ids local to the graph, and
 * stop tests are per graph. Other calls on g still treat it as one graph. */
int cd_graph_set_batches(cd_graph* g, const int64_t* vstart, int64_t n_graphs, int on_device);

/* Algorithm 1 on every graph of a batched g. labels_out: n int32, labels as
 * graph-local vertex ids; rounds_out (host, n_graphs int32, may be NULL):
 * each graph's round count (it stops after its own round with
 * moved + deferred <= threshold). */
int cd_batch_lpa_run(cd_graph* g, const cd_params* p, int32_t* labels_out, int on_device,
                     int32_t* rounds_out);

/* Algorithm 3 on every graph of a batched g, levels in lockstep (a graph that
 * is done stays frozen). labels_out: n int32, each graph's communities
 * numbered 0..k_b-1; levels_out and q_out (host, n_graphs, may be NULL): each
 * graph's level count and modularity (Sec. II-C) on its own graph. */
int cd_batch_louvain_run(cd_graph* g, const cd_params* p, int32_t* labels_out, int on_device,
                         int32_t* levels_out, double* q_out);

/* Serving engine: one GPU answering a stream of requests, each LPA
 * (Algorithm 1) or Louvain (Algorithm 3) on one graph. The paper runs one
 * graph per call; this adds continuous batching around the same solvers.
 * Requests are admitted in arrival order onto `slots` worker threads, each
 * with its own CUDA stream, as soon as a slot is free and the estimated
 * device memory of the request fits in what is left of the budget (a
 * request that does not fit reserves its share, so it is not starved).
 * Waiting requests with n <= small_n of the same algorithm are packed
 * block-diagonally, up to batch_arcs arcs, into one cd_batch_* call. Every
 * request gets the labels a solo run on its graph gives. */
typedef struct cd_server cd_server; /* opaque */

enum { CD_REQ_LPA = 1, CD_REQ_LOUVAIN = 2 };

typedef struct cd_request_result {
  int32_t status;       /* CD_OK or the error of the solve */
  int32_t iters;        /* LPA rounds or Louvain levels */
  int64_t n;            /* vertices (length of the labels) */
  double q;             /* Louvain: modularity (Sec. II-C); LPA: 0 */
  double queue_ms;      /* submit -> start of the solve */
  double latency_ms;    /* submit -> result ready */
  int32_t batched_with; /* requests solved in the same call (1 = alone) */
  int32_t reserved;
} cd_request_result;

/* Start a server on the current device with parameters p (copied; timing is
 * ignored; device_loop = 1 keeps the host loop in the workers' packed calls,
 * where concurrent graph instantiation costs more than it saves, and 2 still
 * uses the device loop everywhere), 1 <= slots <= 64 workers, a device-memory budget in bytes (<= 0:
 * 80% of the free memory now), the packing limits small_n and batch_arcs
 * (0 turns packing off). Errors: CD_EINVAL, CD_ECUDA. */
int cd_server_create(const cd_params* p, int32_t slots, int64_t mem_budget_bytes, int64_t small_n,
                     int64_t batch_arcs, cd_server** out);

/* Queue a request; the graph (HOST arrays in the cd_csr_upload convention,
 * copied before return) is validated when it runs. *id_out receives its id.
 * Errors: CD_EINVAL (bad kind or pointers, server stopping), CD_ENOMEM
 * (larger than the whole budget). */
int cd_server_submit(cd_server* s, int32_t kind, const void* offsets, int offsets_is_i64,
                     const int32_t* cols, const int32_t* w, int64_t n, int64_t nnz, int64_t* id_out);

/* Wait up to timeout_ms (< 0: without limit) for request id; on completion
 * fill *res (may be NULL) and labels_out (host, n int32, may be NULL; written
 * only on success), forget the request and return its status. CD_ETIMEOUT
 * if it is not done in time (it stays queued), CD_EINVAL for an unknown id. */
int cd_server_wait(cd_server* s, int64_t id, int64_t timeout_ms, cd_request_result* res,
                   int32_t* labels_out);

/* Counters: requests admitted and completed, packed calls made, bytes of the
 * budget in use. Outputs may be NULL. */
int cd_server_stats(cd_server* s, int64_t* admitted, int64_t* completed, int64_t* packed_calls,
                    int64_t* in_use);

/* Finish every queued request, stop the workers and free the server. No
 * other call on s may run concurrently or follow. */
int cd_server_destroy(cd_server* s);

/* Degree bins (performance only; results never depend on them): vertices of
 * degree 33..t_warp are scanned by one warp, t_warp+1..t_hub by 128 threads
 * (degree <= 1024) or 512 threads (<= 4096) with a shared-memory table, and
 * vertices above t_hub keep persistent label histograms updated by their
 * neighbours' moves. 32 <= t_warp <= 256, t_warp <= t_hub <= 4096; defaults
 * 256 and 1024, except that a Louvain coarse graph of at least 2^27 arcs takes
 * t_hub = 512 (its levels run many rounds that move few vertices). Thresholds
 * set here (or by cd_autotune) are kept by every coarse graph made from g. */
int cd_graph_set_bins(cd_graph* g, int32_t t_warp, int32_t t_hub);

/* Autotuner: time `rounds` rounds of LPA plus `rounds` rounds of local moving
 * for every candidate (t_warp in {64,128,256}) x (t_hub in {512,1024,2048,4096}),
 * keep the fastest bins on g (coarse Louvain levels inherit them) and report
 * them (outputs may be NULL). */
int cd_autotune(cd_graph* g, const cd_params* p, int32_t rounds, int32_t* t_warp_out, int32_t* t_hub_out);

/* Copy up to cap per-round records of the last run on g into out; *count
 * receives the number of records available. */
int cd_trace_get(const cd_graph* g, cd_round_trace* out, int32_t cap, int32_t* count);

/* Copy up to cap per-kernel profiles of the last run on g (timing = 1). */
int cd_profile_get(const cd_graph* g, cd_kernel_profile* out, int32_t cap, int32_t* count);

/* Human-readable text of a status code. */
const char* cd_status_string(int status);

/* The last CUDA runtime error seen by the library (cudaError_t as int). */
int cd_last_cuda_error(void);

/* Number of CUDA kernels the library has launched in this process so far. */
int64_t cd_launch_count(void);

/* Modularity without any device allocation. The paper has no counterpart to
 * this entry point: it serves callers that cannot call cudaMalloc, such as a
 * process whose device memory is wholly owned and budgeted by another
 * allocator, where one more driver allocation may fail or is not allowed.
 * Same result as cd_csr_upload + cd_modularity: Q of `labels` on the graph
 * (off: n+1 int64, cols: nnz int32, w: nnz int32 or NULL for unit weights, a
 * loop arc v->v carrying L; labels: n int32 in [0, n)), all DEVICE pointers
 * owned by the caller; the work runs on `stream` and the call returns after
 * *q_out is written. Scratch is a static device array inside the library
 * (16 MiB, held by every GPU that loads the library until exit), so n may be
 * at most 2,097,152; larger n gives CD_EINVAL. The first call on each device
 * looks the array's device address up and loads this entry point's kernels
 * (with that device current), so make it before any stream capture; the kept
 * address belongs to the device's primary context, so the library must not
 * be used after cudaDeviceReset. All calls share the array: calls that
 * overlap on the GPU race and must not be issued. Errors: CD_EINVAL (null pointer, n
 * too large, label outside [0, n), weight < 1), CD_EBOUNDS (column outside
 * [0, n)), CD_ENOTSYM (offsets outside [0, nnz] or decreasing), CD_ECUDA. */
int cd_modularity_noalloc(const int64_t* off, const int32_t* cols, const int32_t* w,
                          const int32_t* labels, int64_t n, int64_t nnz, void* stream,
                          double* q_out);

#ifdef __cplusplus
}
#endif
#endif
