/*
 * fastged.h -- C ABI of the GB300 (sm_103a) K-Best graph edit distance library.
 *
 * The library computes, for every (g1, g2) pair of a batch, the K-Best upper bound on the
 * graph edit distance of Dabah & Herten, "Efficient Accelerated Graph Edit Distance
 * Computation on GPU":
 *   - GED is the minimum total cost over edit paths transforming g1 into g2 (Sec. 2.2);
 *   - edit operations are vertex-centric: substitution v -> u, deletion v -> eps,
 *     insertion eps -> u, with edge operations implied by the vertex map (Sec. 2.3, 2.3.1);
 *   - the search (Algorithm 1) branches the g1 vertices in index order; each kept node
 *     spawns one substitution child per g2 vertex still free (R_V2) and one deletion
 *     child (Sec. 4.1.1); a child's partial edit distance PED is its parent's plus the new
 *     vertex operation and the edge operations it implies against vertices already mapped
 *     (Sec. 4.1.2, Algorithm 2); only the best K children survive each level (Sec. 4.2);
 *     once every g1 vertex is processed the free g2 vertices and their edges are inserted
 *     (Sec. 4.4) and the cheapest completed leaf is returned with its vertex map.
 *
 * Ties are broken deterministically: the kept list of a level is the first K entries of
 * the order (PED, parent slot, child index j), with j = 0..n2-1 the substitution by u_j
 * and j = n2 the deletion; kept nodes are stored in that order (slot = rank). The final
 * argmin takes the lowest slot among equal costs. Every result is bit-exact with the
 * serial CPU oracle that restates Algorithm 1.
 *
 * Graphs are simple, undirected, labelled, without loops (Sec. 2.1). Costs are the six
 * non-negative integers of the paper's experimental setup (Sec. 5); substitution costs
 * are charged only when the two labels differ (Sec. 2.4).
 *
 * Threading: a handle may be used by one host thread at a time. Distinct handles are
 * independent. Error messages are kept per calling thread.
 *
 * Memory: every pointer argument of fastged_batch / fastged_batch_ex / fastged_plan_* is
 * a HOST pointer owned by the caller; the library never keeps a caller pointer after a
 * call returns. Device memory, streams, CUDA graphs and pinned staging buffers belong to
 * the handle (or plan / server) and are released by the matching destroy / stop call.
 * Outputs are written only when the call returns FASTGED_OK.
 */
#ifndef FASTGED_H
#define FASTGED_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FASTGED_VERSION 10000

/* status codes (0 = success, negative = failure; see fastged_last_error for details) */
#define FASTGED_OK               0
#define FASTGED_ERR_INVALID_ARG -1   /* a size, label, index, edge or cost is out of range */
#define FASTGED_ERR_OOM         -2   /* device or pinned host memory could not be obtained */
#define FASTGED_ERR_CUDA        -3   /* a CUDA runtime call or kernel failed               */
#define FASTGED_ERR_TIMEOUT     -4   /* a bounded wait ran out (serving / fault injection)  */
#define FASTGED_ERR_BUSY        -5   /* serving: admission refused, request queue is full  */
#define FASTGED_ERR_STOPPED     -6   /* serving: the server is stopped                      */
#define FASTGED_ERR_CANCELLED   -7   /* serving: the query was cancelled before it ran      */

/* limits of the library */
#define FASTGED_MAX_N      1024      /* vertices per graph                                  */
#define FASTGED_MAX_K      1048576   /* beam width (2^20)                                   */
#define FASTGED_MAX_ELABEL 255       /* edge labels are 0..255                              */

/* Cost model (Sec. 2.4; the six explicit costs of Sec. 5). All entries must be >= 0.
 * v_sub / e_sub are charged only when the two vertex / edge labels differ. */
typedef struct {
    int32_t v_sub, v_del, v_ins;
    int32_t e_sub, e_del, e_ins;
} fastged_cost_model;

/* One graph (Sec. 2.1). n vertices 0..n-1 with labels vlabel[n] (any int32; only equality
 * matters). m undirected edges as edges[2*k], edges[2*k+1] (endpoints in 0..n-1, distinct;
 * either order; no duplicates). elabel[m] holds the edge labels (0..FASTGED_MAX_ELABEL) or
 * is NULL for unlabelled edges (every edge then has label 0). */
typedef struct {
    int32_t n;
    const int32_t *vlabel;
    int32_t m;
    const int32_t *edges;
    const int32_t *elabel;
} fastged_graph;

/* A batch: n_graphs graphs and n_pairs pairs; pairs[2*p] is the source g1 and
 * pairs[2*p+1] the target g2 of pair p (the paper's direction, Sec. 5). A graph may
 * appear in many pairs. */
typedef struct {
    int32_t n_graphs;
    const fastged_graph *graphs;
    int32_t n_pairs;
    const int32_t *pairs;
} fastged_pair_list;

#define FASTGED_FORM_BATCHED 0   /* one persistent launch per size class over a work queue */
#define FASTGED_FORM_PLAIN   1   /* one launch per pair, in pair order, on one stream       */

typedef struct {
    int32_t form;            /* FASTGED_FORM_BATCHED (default) or FASTGED_FORM_PLAIN          */
    int32_t variant;         /* 0 (default): complete the K kept leaves;                      */
                             /* 1: complete every successor of the last level (never worse)   */
    const int32_t *k_per_pair; /* optional host array [n_pairs] of per-pair K (1..K); NULL =  */
                             /* the K argument for every pair                                 */
    int32_t hist_window;     /* 0 = default. Width (2..32) of the PED histogram window of     */
                             /* the selection step; small values force its exact fallback     */
                             /* path (a testing knob; results do not depend on it)            */
    int32_t block_threads;   /* 0 = autotuned; else 128, 256 or 512 threads per team          */
    int32_t use_cuda_graph;  /* plans only: 1 = capture the run once and replay it as a CUDA  */
                             /* graph, 0 = launch directly (a NULL options pointer means 1)   */
    int32_t autotune;        /* plans only: 1 = before the plan is built, time every size     */
                             /* class that the tuning table does not know yet with each team  */
                             /* shape (threads per CTA, or CTAs per cluster for large pairs)  */
                             /* on a sample of its pairs, and record the fastest; 0 = use the */
                             /* table's entries where present, built-in rules elsewhere       */
    int32_t vertex_order;    /* order in which the levels branch the source vertices:        */
                             /* FASTGED_ORDER_INDEX (0, the paper's v_0..v_{n1-1}) or         */
                             /* FASTGED_ORDER_DEGREE (1: descending degree, ties by index;    */
                             /* an extension, not part of the paper). Maps are returned in   */
                             /* source index order either way                                 */
    int32_t team;            /* FASTGED_TEAM_AUTO (0): pairs with at most 64 vertices in g1,  */
                             /* at most 63 in g2 and K <= 128 are solved by one warp each,    */
                             /* the others by a CTA (or a cluster of CTAs) each;              */
                             /* FASTGED_TEAM_CTA (1): every pair by a CTA or cluster.         */
                             /* Results do not depend on it                                   */
    int32_t max_sms;         /* 0 = no cap; else the resident teams of each size class are   */
                             /* capped to what fits this many SMs (whole clusters, at least   */
                             /* one team), so that other work keeps the remaining SMs; pairs  */
                             /* then queue for the capped teams. Results do not depend on it  */
    int32_t cluster;         /* 0 = built-in rule or tuning table; 1, 2, 4, 8 or 16: CTAs per */
                             /* team for the classes that may use cluster teams (fewer pairs  */
                             /* than SMs, wide bitsets or very wide beams). Small clusters do */
                             /* the most work per SM, large ones finish a single pair soonest */
} fastged_options;

#define FASTGED_TEAM_AUTO 0
#define FASTGED_TEAM_CTA  1

#define FASTGED_ORDER_INDEX 0
#define FASTGED_ORDER_DEGREE 1

typedef struct fastged_handle fastged_handle;
typedef struct fastged_plan fastged_plan;
typedef struct fastged_server fastged_server;

/* Library version (FASTGED_VERSION). */
int fastged_version(void);

/* Last error message of the calling thread ("" when none). The handle argument may be
 * NULL; messages are per thread, not per handle. The string stays valid until the next
 * fastged call on the same thread. */
const char *fastged_last_error(const fastged_handle *h);

/* Creates a handle on the current CUDA device with the given cost model (Sec. 2.4).
 * Returns FASTGED_ERR_INVALID_ARG for a NULL argument or a negative cost,
 * FASTGED_ERR_CUDA when no device is usable. *out receives the handle on success. */
int fastged_create(const fastged_cost_model *cost, fastged_handle **out);

/* Releases the handle and everything it owns. NULL is ignored. */
void fastged_destroy(fastged_handle *h);

/* K-Best GED of every pair (Algorithm 1) with host inputs and outputs.
 *   K            beam width, 1..FASTGED_MAX_K
 *   out_cost     [n_pairs] GED upper bound of each pair
 *   out_mapping  [sum over pairs of n1] concatenated in pair order: for pair p, entry k is
 *                the g2 vertex that v_k of g1 is substituted by, or -1 when v_k is deleted
 * The call blocks until results are on the host. */
int fastged_batch(fastged_handle *h, const fastged_pair_list *pairs, int32_t K,
                  int32_t *out_cost, int32_t *out_mapping);

/* As fastged_batch, with options (NULL = defaults) and an optional out_nevals[n_pairs]
 * (may be NULL): the number of successors scored at every level plus leaves completed. */
int fastged_batch_ex(fastged_handle *h, const fastged_pair_list *pairs, int32_t K,
                     const fastged_options *opt, int32_t *out_cost, int32_t *out_mapping,
                     int64_t *out_nevals);

/* Device-resident plan: the batch is validated, flattened and copied to the device once;
 * fastged_plan_run then re-runs the whole device path (bitset packing, the K-Best levels,
 * completion) from the resident inputs. Outputs stay on the device until fastged_plan_read. */
int fastged_plan_create(fastged_handle *h, const fastged_pair_list *pairs, int32_t K,
                        const fastged_options *opt, fastged_plan **out);

/* Enqueues one run of the plan on `stream` (a cudaStream_t; NULL = the plan's own stream)
 * and returns without waiting. */
int fastged_plan_run(fastged_plan *p, void *stream);

/* Waits for the plan's last run and copies its results to host memory (any of the three
 * pointers may be NULL). Checks the device-side error flag first. */
int fastged_plan_read(fastged_plan *p, int32_t *out_cost, int32_t *out_mapping,
                      int64_t *out_nevals);

typedef struct {
    int32_t n_pairs;
    int32_t n_classes;        /* size classes (one persistent launch each)                 */
    int32_t launches_per_run; /* kernels launched by one fastged_plan_run                  */
    int32_t graph_replay;     /* 1 if runs replay a captured CUDA graph                    */
    int64_t input_bytes;      /* resident input bytes (flattened graphs, tables)           */
    int64_t device_bytes;     /* all device bytes the plan holds                           */
    int64_t output_bytes;     /* bytes fastged_plan_read copies back (cost, map, evals)    */
    int32_t block_threads[8]; /* per class (the first 8 classes)                           */
    int32_t grid[8];          /* per class (the first 8 classes)                           */
    int32_t words[8];         /* per class: 64-bit words per bitset                        */
    int32_t smem_bytes[8];    /* per class: dynamic shared memory per team                 */
} fastged_plan_stats;

int fastged_plan_info(const fastged_plan *p, fastged_plan_stats *out);

/* Device time (ms) of the K-Best launches of the plan's last run: from the end of the
 * bitset packing to the end of the last size class, measured with CUDA events recorded on
 * the run's stream (inside the replayed graph when the plan replays one). Waits for the run. */
int fastged_plan_kernel_ms(fastged_plan *p, float *ms);

/* Releases the plan (waits for its last run). NULL is ignored. */
void fastged_plan_destroy(fastged_plan *p);

/* ---------------------------------------------------------------------------------------
 * Serving: continuous batching of GED queries on one GPU.
 *
 * fastged_serve_submit copies a query (g1, g2, K) into the server and returns. A dispatcher
 * thread keeps up to `lanes` batches in flight, each lane owning its own streams and
 * grow-only device buffers (graph bit-sets, beams and outputs stay resident between
 * batches). While batches run, newly arrived queries are grouped by size bucket (the size
 * classes: one-warp pairs by word width, the others by the bitset words of the target
 * graph) and launched as the
 * next batch as soon as a lane is free and one of these holds: min_batch_pairs of the oldest
 * query's bucket are pending, the oldest query has waited max_wait_us, or nothing else is
 * running. Batches of pairs with more than 256 target vertices run on two-CTA clusters
 * (the most work per SM), hold at most three lanes in eight and together at most half of
 * the SMs; every other batch keeps its teams on at most a third of the SMs, so that small
 * queries arriving meanwhile find free SMs. Before
 * launching, free device memory must exceed the batch's footprint plus hbm_reserve_bytes
 * (otherwise the batch waits for a running one to finish). Results are identical to
 * fastged_batch_ex on the same query.
 * --------------------------------------------------------------------------------------- */
/* A server's lanes run concurrently only on distinct hardware queues: start the process with
 * CUDA_DEVICE_MAX_CONNECTIONS=32 (read when the CUDA context is created), or small queries
 * may wait behind large batches that share their queue. */
typedef struct {
    int32_t lanes;             /* batches in flight at most, 1..16 (default 16)            */
    int32_t max_batch_pairs;   /* queries per batch at most (default 4096)                 */
    int32_t min_batch_pairs;   /* launch once this many queries of a bucket wait (64)      */
    int32_t max_pending;       /* queued queries at most; beyond: FASTGED_ERR_BUSY (2^20)  */
    int32_t max_wait_us;       /* longest wait of the oldest query before launch (200)     */
    int32_t max_retries;       /* times a query of a failed batch is queued again (0)      */
    int64_t hbm_reserve_bytes; /* device memory kept free by admission (1 GiB)             */
} fastged_serve_config;

typedef struct {
    uint64_t tag;              /* the caller's tag from fastged_serve_submit                */
    int32_t status;            /* FASTGED_OK or the error of the batch the query was in     */
    int32_t cost;              /* GED upper bound                                           */
    int32_t n1;                /* entries of the vertex map (0 if status is not FASTGED_OK) */
    int32_t pad;
    int64_t map_offset;        /* first entry of the map in the poll's map buffer           */
    int64_t n_evals;           /* successors scored plus leaves completed                   */
    double latency_ms;         /* submit -> result ready                                    */
    double queue_ms;           /* submit -> batch launch                                    */
} fastged_serve_result;

typedef struct {
    int64_t submitted, completed, failed, batches, batched_pairs, rejected_busy,
        admission_waits, pending, lanes_busy;
} fastged_serve_stats;

/* Starts a server on the current device (cfg NULL = the defaults above). */
int fastged_serve_start(const fastged_cost_model *cost, const fastged_serve_config *cfg,
                        fastged_server **out);

/* Queues one query; the graphs are copied, so the caller may reuse them at once. Returns
 * FASTGED_ERR_INVALID_ARG for invalid graphs or K (same rules as fastged_batch, duplicate
 * edges included), FASTGED_ERR_BUSY when max_pending queries are queued, and
 * FASTGED_ERR_STOPPED after fastged_serve_stop. Thread-safe. */
int fastged_serve_submit(fastged_server *s, const fastged_graph *g1, const fastged_graph *g2,
                         int32_t K, uint64_t tag);

/* Moves up to max_results finished queries into out[], their vertex maps into map_buf
 * (capacity map_cap entries; each result's map_offset points into it, n1 entries long; a
 * failed query has n1 = 0 and no map), waiting up to timeout_ms for the first one. Returns
 * the number of results (0 on timeout) or a negative status (FASTGED_ERR_INVALID_ARG if even
 * the first map does not fit). */
int fastged_serve_poll(fastged_server *s, fastged_serve_result *out, int32_t max_results,
                       int32_t *map_buf, int64_t map_cap, int32_t timeout_ms);

/* Cancels every query with this tag that is still queued (not yet in a batch): each comes
 * back through fastged_serve_poll with status FASTGED_ERR_CANCELLED and no map, so every
 * submitted query still yields exactly one result. Queries already in a batch run to the end.
 * Returns how many queries were cancelled (0 if none was queued), or FASTGED_ERR_INVALID_ARG
 * for a null server. Thread-safe. */
int fastged_serve_cancel(fastged_server *s, uint64_t tag);

/* Counters of the server so far (completed counts every result handed to the completion
 * queue: succeeded, failed or cancelled). */
int fastged_serve_get_stats(fastged_server *s, fastged_serve_stats *out);

/* Stops accepting queries, runs every queued one and waits for all batches; results stay
 * available to fastged_serve_poll. */
void fastged_serve_stop(fastged_server *s);

/* Stops the server if needed and releases it (unpolled results are discarded). */
void fastged_serve_destroy(fastged_server *s);

/* Host threads: batches are validated and staged on a process-wide thread pool whose size
 * the environment variable FASTGED_HOST_THREADS sets when the pool is first used (threads
 * of one batch, the calling thread included; 1 = the caller alone; default: up to 16). The
 * staged bytes and every result are the same for any size. */

/* Tuning table of the process (size-class shape -> team shape). If the environment variable
 * FASTGED_AUTOTUNE_FILE names a file, the table is read from it on first use and every new
 * entry is appended to it. fastged_autotune_entries returns the number of entries;
 * fastged_autotune_clear forgets them all (the file is left alone). FASTGED_CLUSTER = 1, 2,
 * 4, 8 or 16 forces the CTAs per team of the classes that may use thread-block clusters (few
 * pairs of four or more words, or two-word pairs with very wide beams), over the table. */
int fastged_autotune_entries(void);
void fastged_autotune_clear(void);

/* ---------------------------------------------------------------------------------------
 * Edit paths and GED matrices (Sec. 6 of the paper uses both: the edit path between two
 * architectures, half of whose operations are applied to cross them over, and the GED of
 * every test graph to every training graph for nearest-neighbour classification).
 * --------------------------------------------------------------------------------------- */
#define FASTGED_OP_VINS 0   /* insert g2 vertex g2_u                                       */
#define FASTGED_OP_VSUB 1   /* relabel g1 vertex g1_u to the label of g2 vertex g2_u        */
#define FASTGED_OP_EDEL 2   /* delete g1 edge (g1_u, g1_v)                                 */
#define FASTGED_OP_ESUB 3   /* relabel g1 edge (g1_u, g1_v) to the label of g2 edge        */
                            /* (g2_u, g2_v)                                                */
#define FASTGED_OP_EINS 4   /* insert g2 edge (g2_u, g2_v)                                 */
#define FASTGED_OP_VDEL 5   /* delete g1 vertex g1_u                                       */

typedef struct {
    int32_t kind;   /* FASTGED_OP_*                                                        */
    int32_t cost;   /* the operation's cost under the cost model                           */
    int32_t g1_u;   /* source-side vertex, or first edge endpoint; -1 if none              */
    int32_t g1_v;   /* source-side second edge endpoint; -1 if none                        */
    int32_t g2_u;   /* target-side vertex, or first edge endpoint (the image of g1_u for   */
                    /* an edge substitution); -1 if none                                  */
    int32_t g2_v;   /* target-side second edge endpoint; -1 if none                        */
} fastged_edit_op;

/* The edit path that the vertex map `mapping` (n1 entries: the g2 image of each g1 vertex,
 * -1 = deleted; as fastged_batch returns it) induces from g1 to g2 (Sec. 2.2-2.4): only
 * operations that change something are listed (a substitution keeping the label is not an
 * edit), in this order, each group by increasing index (edges in input order):
 *   vertex insertions (g2 vertices outside the image), vertex substitutions (label
 *   changes), edge deletions (g1 edges whose image is not a g2 edge), edge substitutions
 *   (label changes), edge insertions (g2 edges that are no image), vertex deletions.
 * Every prefix of the list is a valid sequence: inserted vertices exist before edges use
 * them, and a vertex is deleted only after its edges.
 *   ops        array of capacity `cap`, or NULL to only count
 *   n_ops      receives the number of operations (at most n1 + n2 + m1 + m2)
 *   total_cost receives their summed cost (= the cost of the map); may be NULL
 * Errors: FASTGED_ERR_INVALID_ARG for an invalid graph, a map that is not an injective
 * partial map into g2, or ops != NULL with cap < the number of operations (nothing is
 * written then except n_ops). Host function; no GPU work. */
int fastged_edit_path(const fastged_cost_model *cost, const fastged_graph *g1,
                      const fastged_graph *g2, const int32_t *mapping, fastged_edit_op *ops,
                      int32_t cap, int32_t *n_ops, int64_t *total_cost);

/* Applies the first n_apply operations of the edit path that `mapping` induces from g1 to
 * g2 (as fastged_edit_path lists them) to g1 and writes the resulting graph (the map tells
 * which g1 vertex an inserted edge's endpoint is): its vertices are the g1 vertices not
 * deleted (in g1 order) followed by the inserted g2 vertices (in operation order); edges
 * refer to those new ids. With every operation applied the result equals g2 up to the
 * vertex renaming the map gives. Output capacities: out_vlabel n1 + n2 entries, out_edges
 * 2 (m1 + m2), out_elabel m1 + m2 (NULL when neither graph has edge labels).
 * Errors: FASTGED_ERR_INVALID_ARG for invalid graphs or operations. Host function. */
int fastged_apply_edit_ops(const fastged_graph *g1, const fastged_graph *g2,
                           const int32_t *mapping, const fastged_edit_op *ops,
                           int32_t n_apply, int32_t *out_n,
                           int32_t *out_vlabel, int32_t *out_m, int32_t *out_edges,
                           int32_t *out_elabel);

/* GED matrix: out[r * n_cols + c] = K-Best GED (upper bound) from graphs[rows[r]] to
 * graphs[cols[c]], every entry computed as one pair of a single batch (with rows == cols it
 * is the all-pairs matrix of a set; the diagonal is computed too). opt as in
 * fastged_batch_ex (NULL = defaults; k_per_pair must be NULL). Errors as fastged_batch_ex. */
int fastged_cross(fastged_handle *h, const fastged_graph *graphs, int32_t n_graphs,
                  const int32_t *rows, int32_t n_rows, const int32_t *cols, int32_t n_cols,
                  int32_t K, const fastged_options *opt, int32_t *out);

/* ---------------------------------------------------------------------------------------
 * Failure handling (no counterpart in the paper).
 *
 * fastged_set_timeout bounds how long fastged_batch / fastged_batch_ex on this handle wait for
 * the device: past `ms` milliseconds (0 = no bound, the default) they return
 * FASTGED_ERR_TIMEOUT without results while the batch finishes in the background; the next
 * call on the handle first waits for it, so the handle stays usable. The wait polls an event;
 * no kernel ever spins, traps or is cut short.
 *
 * fastged_inject_fault arms a one-shot host-side fault for tests: the `countdown`-th event of
 * `kind` from now fails (countdown 0 disarms). Kinds: FASTGED_INJECT_ALLOC (a device or
 * pinned allocation reports FASTGED_ERR_OOM; the buffer it would replace is kept),
 * FASTGED_INJECT_LAUNCH (a K-Best launch is skipped and the call reports FASTGED_ERR_CUDA),
 * FASTGED_INJECT_ADMISSION (the server's admission check refuses a batch once, as if device
 * memory were short; the batch waits and is retried). Faults are process-wide and touch no
 * GPU state: the calls that fail leave their handle or server usable.
 * --------------------------------------------------------------------------------------- */
#define FASTGED_INJECT_ALLOC 0
#define FASTGED_INJECT_LAUNCH 1
#define FASTGED_INJECT_ADMISSION 2

int fastged_set_timeout(fastged_handle *h, int32_t ms);
int fastged_inject_fault(int32_t kind, int32_t countdown);

/* Integer-pipe throughput of the current device (no counterpart in the paper; it is the
 * measured peak the benchmark compares the successor evaluation against). Runs three
 * short probe kernels issuing independent 32-bit LOP3, IADD and POPC chains on every SM
 * and writes the device-wide rate of each (instructions x lanes per second); any output
 * pointer may be NULL. Allocates and frees a 16 KB device buffer. */
int fastged_measure_int_peak(double *lop3_per_s, double *iadd_per_s, double *popc_per_s);

/* ---------------------------------------------------------------------------------------
 * Allocation-free batch (the paper has no counterpart; this is a deployment aid).
 *
 * For callers that cannot allocate device memory themselves or let a library do it: code
 * embedded in an application that owns every device allocation through its own pool, a
 * plugin handed a fixed device budget, or a runtime where cudaMalloc at an arbitrary point
 * is forbidden. The caller passes device inputs and device outputs; all scratch the path
 * needs (graph table, work queue, status word, adjacency bit-set pools, per-team working
 * sets) comes from one file-scope device array of FASTGED_NOALLOC_SCRATCH_BYTES that the
 * library module carries, so every GPU that loads the library holds that memory until the
 * process exits. The call performs no cudaMalloc / cudaFree and no other allocation.
 *
 * All graph arrays are DEVICE pointers in the flattened form below; max_n, max_m,
 * max_elabel and total_vertices are host values that bound the device data (they size the
 * kernels' working sets). The results are identical to fastged_batch_ex with the same
 * graphs, pairs, cost model and K.
 * --------------------------------------------------------------------------------------- */
#define FASTGED_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

typedef struct {
    int32_t n_graphs;
    int32_t n_pairs;
    int32_t max_n;            /* host: >= every graph's vertex count; 1..FASTGED_MAX_N     */
    int32_t max_m;            /* host: >= every graph's edge count                          */
    int32_t max_elabel;       /* host: >= every edge label (0 for unlabelled graphs)        */
    int32_t pad;
    int64_t total_vertices;   /* host: entries of vlabel, >= sum of graph_n                 */
    int64_t total_edges;      /* host: edges in edges (and entries of elabel)               */
    int64_t map_len;          /* host: entries of out_mapping                               */
    const int32_t *graph_n;   /* device [n_graphs] vertices per graph                       */
    const int32_t *graph_m;   /* device [n_graphs] edges per graph                          */
    const int64_t *vlabel_off;/* device [n_graphs] first label of graph g in vlabel (ranges */
                              /* may overlap: graphs may share label rows)                  */
    const int64_t *edge_off;  /* device [n_graphs] first edge of graph g in edges / elabel  */
    const int32_t *vlabel;    /* device [total_vertices] vertex labels                      */
    const int32_t *edges;     /* device [2 * total edges] endpoint pairs, as fastged_graph  */
    const int32_t *elabel;    /* device [total edges] edge labels, or NULL                  */
    const int32_t *pairs;     /* device [2 * n_pairs] (source g1, target g2) graph indices  */
    const int64_t *map_off;   /* device [n_pairs] first entry of pair p's map in out_mapping*/
                              /* (map_off[p] + n of the source graph <= map_len)            */
} fastged_device_batch;

/* K-Best GED of every pair of a device-resident batch without allocating memory.
 *   cost         host cost model (all entries >= 0)
 *   batch        host struct of device arrays and host bounds (above)
 *   K            beam width, 1..FASTGED_MAX_K
 *   out_cost     device [n_pairs]; out_mapping device [sum of n1], laid out by map_off;
 *   out_nevals   device [n_pairs] or NULL
 *   stream       cudaStream_t the work is enqueued on (NULL = the legacy default stream)
 * Blocks until the results are on the device (it reads back a status word twice).
 * Errors: FASTGED_ERR_INVALID_ARG for out-of-range host bounds, for device data that breaks
 * them (vertex / edge counts above max_n / max_m, label or edge ranges past total_vertices /
 * total_edges, more vertices in all than total_vertices, endpoints, self-loops, duplicate
 * edges, labels, pair indices, maps past map_len; these are checked on the device before any
 * kernel reads an edge or writes a map, and the outputs are then unspecified), and for a
 * batch whose tables, bit-set pools and one team's working set do not fit
 * FASTGED_NOALLOC_SCRATCH_BYTES; FASTGED_ERR_CUDA otherwise.
 * The scratch array is shared by every call in the process: calls whose device work
 * overlaps (on different streams, or from several host threads) race and corrupt each
 * other's results, so issue them one after another. It keeps the last call's contents;
 * each call clears what must start at zero itself. The first call on a device resolves the
 * array's device address (with that device current), and so does the first call after the
 * device's context was replaced (e.g. by cudaDeviceReset); the call waits for its stream, so
 * it cannot be captured into a CUDA graph. */
int fastged_batch_noalloc(const fastged_cost_model *cost, const fastged_device_batch *batch,
                          int32_t K, int32_t *out_cost, int32_t *out_mapping,
                          int64_t *out_nevals, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FASTGED_H */
