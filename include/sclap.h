/*
 * sclap.h -- C ABI of the GB300 (sm_103a) multilevel size-constrained label
 * propagation (SCLaP) graph partitioner.
 *
 * Method: Meyerhenke, Sanders, Schulz, "Partitioning Complex Networks via
 * Size-constrained Clustering".  The problem (Sec. 2.1): given an undirected
 * graph G = (V, E, c, w) with node weights c and edge weights w, find blocks
 * V_0..V_{k-1} partitioning V with c(V_i) <= Lmax for every i that minimise
 * the cut sum_{i<j} w(E_ij).  Here Lmax = floor((1+eps) * ceil(c(V)/k)), the
 * paper's unweighted form of the balance constraint applied to c(V).
 * The multilevel scheme (Sec. 1 Fig. 1, Sec. 3) coarsens by size-constrained
 * LP clustering (cluster bound U = max(max_v c(v), floor(Lmax/f)), Sec. 3.1)
 * and cluster contraction, partitions the coarsest graph, then projects and
 * refines each level with LP local search under Lmax (Sec. 3.1) using active
 * nodes (Sec. 4).  Every step runs in CUDA kernels on the current device.
 *
 * Determinism: the result is a pure function of (graph, k, eps, seed, cfg).
 * It equals the round-synchronous variant of the CPU oracle bit for bit and
 * does not depend on which other graphs share a batch.
 *
 * Graph format (all entry points):
 *   n        number of nodes, 1 <= n < 2^31
 *   row_ptr  int64[n+1], row_ptr[0] = 0, non-decreasing; m = row_ptr[n] arcs
 *   col      int32[m], neighbour ids in [0, n); the graph must be symmetric
 *            (every arc (u,v) has its twin (v,u) with the same weight) and
 *            contain no self-loops.  Row order is free.
 *   node_w   int32[n], positive, sum < 2^31; NULL means unit weights
 *   edge_w   int32[m], positive; NULL means unit weights
 * Symmetry is the caller's contract and is not checked; everything else is,
 * before any kernel reads the graph.
 *
 * Ownership: the caller owns every buffer passed in; the library copies what
 * it needs and keeps no pointer after a call returns.  Working memory comes
 * from the CUDA stream-ordered allocator of the current device.
 *
 * Errors: every function returns SCLAP_OK (0) or a negative SCLAP_E* code;
 * sclap_error_string() describes it.  No exception crosses the ABI.  The only
 * device-side waits are the grid barriers of the cooperative admission kernel
 * (tuning field fused_admission); they are bounded, and one that runs out
 * ends the call with SCLAP_ETIMEOUT.  Every other device loop is bounded by
 * its data size.
 */
#ifndef SCLAP_H
#define SCLAP_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SCLAP_OK = 0,
  SCLAP_EINVAL = -1,      /* bad argument (k < 1, k > n, eps < 0, NULL pointer, ...) */
  SCLAP_ECSR = -2,        /* malformed CSR: row_ptr, col range, self-loop, weights   */
  SCLAP_ENOMEM = -3,      /* device allocation failed                                */
  SCLAP_ECUDA = -4,       /* a CUDA call failed                                      */
  SCLAP_EOVERFLOW = -5,   /* a coarse edge weight or c(V) does not fit in int32      */
  SCLAP_EINFEASIBLE = -6, /* blocks stay above Lmax after repair (outputs written)   */
  SCLAP_ETIMEOUT = -7,    /* a bounded device-side wait ran out                      */
  SCLAP_EINTERNAL = -8,   /* internal consistency check failed                       */
  SCLAP_PENDING = 1       /* sclap_server_poll: the request has not finished yet     */
};

/* Tunables.  Defaults (sclap_default_config): the paper's parameters (Sec. 5):
 * l = 10 LP rounds per level in coarsening and uncoarsening, f = 18; plus
 * coarsening down to max(1000, 60k) nodes, 16 initial-partitioning trials,
 * 8 colour classes per synchronous round, 64 repair rounds, 64 levels, and
 * clustering without active nodes.
 * graph_rounds = 1 runs each level's LP rounds as one CUDA graph: a
 * conditional WHILE node around one round, whose condition the device sets
 * at the end of the round, so the host neither waits nor decides between
 * rounds (it then launches every bucket's kernel; empty ones exit at once).
 * 0 (default) drives the rounds from the host, which reads the bucket sizes
 * once per round and skips empty launches.  Results are identical.
 * ensemble = 1 turns on ensemble clusterings during coarsening (Sec. 4
 * "Ensemble Clusterings", configuration E): every level computes l
 * clusterings (the first with the run's seed, clustering j >= 1 with the key
 * hkey(seed, 7, level, j)) and contracts their overlay, in which two nodes
 * share a cluster iff every clustering puts them together.  l =
 * ensemble_size if > 0, else the paper's rule (Sec. 5): 18 for k < 16, 7 for
 * k = 16..32, 3 above.
 * vcycles = number of multilevel cycles (Sec. 4 "Iterated Multilevel
 * Algorithms", App. A; configuration V uses 3, Sec. 5); default 1.  Every
 * cycle after the first coarsens with clusterings that stay inside the
 * blocks of the current partition (so no cut edge is contracted), starts
 * from that partition on its coarsest graph, refines every level on the way
 * back and repairs balance; cycle c uses hkey(seed, 8, c, 0) as its seed.
 * cluster_active = 1 turns on active nodes during coarsening (Sec. 4 "Active
 * Nodes", configuration A of Table 2): after the first round a clustering
 * round visits only nodes with a neighbour that changed its cluster in the
 * round before.  (Configuration R, a random node order, is what the
 * synchronous rounds do already: nodes are split into colour classes by a
 * per-round hash.) */
typedef struct sclap_config {
  int32_t lp_rounds_coarse;
  int32_t lp_rounds_refine;
  int32_t f;
  int32_t coarse_min_nodes;
  int32_t ip_trials;
  int32_t sub_rounds;
  int32_t repair_rounds;
  int32_t max_levels;
  int32_t cluster_active;
  int32_t graph_rounds;
  int32_t ensemble;
  int32_t ensemble_size;
  int32_t vcycles;
} sclap_config;

/* Per-call statistics (optional output). */
typedef struct sclap_stats {
  int32_t levels;              /* graphs in the hierarchy, input included   */
  int64_t level_n[64];
  int64_t level_m[64];         /* arcs per level                            */
  int32_t cluster_rounds[64];  /* LP rounds run clustering level l          */
  int32_t refine_rounds[64];   /* LP rounds run refining level l            */
  int32_t ip_best_trial;
  int64_t ip_cut;
  int64_t Lmax, U;
  int64_t lp_arcs;             /* arcs scanned by LP sweeps (all levels)    */
} sclap_stats;

void sclap_default_config(sclap_config* cfg);
const char* sclap_error_string(int code);
/* Message of the last error raised on the calling thread ("" after success). */
const char* sclap_last_error(void);

/* Partition one graph held in HOST memory (Sec. 2.1 problem statement).
 * block_out: caller-owned int32[n], receives block ids in [0, k).
 * cut_out: receives the edge cut.  max_block_weight_out, stats: nullable.
 * cfg: nullable (defaults).  Synchronous: returns when results are written.
 * Returns SCLAP_EINFEASIBLE (with outputs written) if balance could not be
 * reached, which needs node weights above the eps slack. */
int sclap_partition(int64_t n, const int64_t* row_ptr, const int32_t* col,
                    const int32_t* node_w, const int32_t* edge_w, int32_t k, double eps,
                    uint64_t seed, const sclap_config* cfg, int32_t* block_out,
                    int64_t* cut_out, int64_t* max_block_weight_out, sclap_stats* stats);

/* Same, with every array in DEVICE memory (block_out too) and the work
 * ordered on `stream` (a cudaStream_t; NULL = legacy default stream).  The
 * call synchronises the stream before returning (level sizes are read back
 * between levels). */
int sclap_partition_device(int64_t n, const int64_t* row_ptr, const int32_t* col,
                           const int32_t* node_w, const int32_t* edge_w, int32_t k,
                           double eps, uint64_t seed, const sclap_config* cfg,
                           int32_t* block_out, int64_t* cut_out,
                           int64_t* max_block_weight_out, sclap_stats* stats, void* stream);

/* One graph of a batch.  Inputs as above; block_out caller-owned int32[n];
 * cut, max_block_weight and status are written by the call. */
typedef struct sclap_graph {
  int64_t n;
  const int64_t* row_ptr;
  const int32_t* col;
  const int32_t* node_w;
  const int32_t* edge_w;
  int32_t k;
  double eps;
  uint64_t seed;
  int32_t* block_out;
  int64_t cut;
  int64_t max_block_weight;
  int32_t status;
} sclap_graph;

/* Partition `count` independent graphs together: every kernel launch covers
 * all graphs still active at that level, so small graphs share the GPU.
 * Each graph's result equals what sclap_partition returns for it alone.
 * device_ptrs = 0: arrays are in host memory; 1: in device memory.
 * Returns SCLAP_OK if every graph succeeded, else the first graph error
 * (per-graph codes in graphs[i].status). */
int sclap_partition_batch(int32_t count, sclap_graph* graphs, const sclap_config* cfg,
                          int32_t device_ptrs, void* stream);

/* ---- Step-level entry points (device pointers, stream-ordered, synchronous
 * on return).  They run exactly the kernels the partitioner uses, on one
 * graph, so each step can be checked on its own. ---- */

/* One synchronous LP round (Sec. 3.1) over all colour classes.
 * mode 0 = clustering (labels are node ids, W has n entries),
 * mode 1 = local search (labels are blocks 0..nlabels-1, W has nlabels).
 * label (int32[n]) and W (int64[nlabels]) are updated in place.
 * active_cur: uint8[n] or NULL (all active); active_next: uint8[n] or NULL,
 * receives 1 for each neighbour of a moved node.  moved_out: host int64. */
int sclap_lp_round(int32_t mode, int64_t n, const int64_t* row_ptr, const int32_t* col,
                   const int32_t* node_w, const int32_t* edge_w, int32_t* label, int64_t* W,
                   int64_t nlabels, int64_t bound, uint64_t rkey, int32_t sub_rounds,
                   const uint8_t* active_cur, uint8_t* active_next, int64_t* moved_out,
                   void* stream);

/* Size-constrained clustering of one level (Sec. 3.1): label_out int32[n]
 * (node id of each cluster's original representative); rounds_out: host. */
int sclap_cluster(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* node_w,
                  const int32_t* edge_w, int64_t U, uint64_t seed, int32_t level,
                  const sclap_config* cfg, int32_t* label_out, int32_t* rounds_out,
                  void* stream);

/* Cluster contraction (Sec. 3.1).  Coarse id = rank of the cluster label.
 * Outputs sized by the fine graph: cmap int32[n], cnode_w int32[n],
 * crow_ptr int64[n+1], ccol int32[m], cedge_w int32[m]; nc_out, mc_out on
 * the host.  Coarse rows are in no particular order. */
int sclap_contract(int64_t n, const int64_t* row_ptr, const int32_t* col,
                   const int32_t* node_w, const int32_t* edge_w, const int32_t* label,
                   int32_t* cmap, int64_t* nc_out, int32_t* cnode_w, int64_t* crow_ptr,
                   int32_t* ccol, int32_t* cedge_w, int64_t* mc_out, void* stream);

/* Clustering hierarchy without a partitioning target (Sec. 3.1 clustering
 * and contraction, repeated as in the coarsening phase; usable on its own
 * for size-constrained community-style coarsening).  Clusters the graph
 * with bound U (cluster weight <= U; nodes heavier than U stay alone), level
 * l hashing with level l; contracts; repeats while the current graph has
 * more than stop_nodes nodes, the hierarchy has fewer than cfg->max_levels
 * graphs, and the contraction removes at least 5% of the nodes (a
 * contraction that removes less is discarded).  Device: comm_out int32[n]
 * receives, for every input node, its node in the last graph (the
 * community id, in [0, level_n_out[levels])).  Host: *levels_out the number
 * of contractions kept; level_n_out (cap entries, may be NULL) the node
 * counts, input first.  Uses cfg->lp_rounds_coarse, sub_rounds,
 * cluster_active and max_levels. */
int sclap_cluster_hierarchy(int64_t n, const int64_t* row_ptr, const int32_t* col,
                            const int32_t* node_w, const int32_t* edge_w, int64_t U,
                            int64_t stop_nodes, uint64_t seed, const sclap_config* cfg,
                            int32_t* comm_out, int32_t* levels_out, int64_t* level_n_out,
                            int32_t cap, void* stream);

/* Initial partitioning of a (coarsest) graph: cfg->ip_trials trials of
 * greedy growing plus LP local search, best by (overload, cut, trial).
 * block_out int32[n]; cut_out, best_trial_out on the host. */
int sclap_initial_partition(int64_t n, const int64_t* row_ptr, const int32_t* col,
                            const int32_t* node_w, const int32_t* edge_w, int32_t k,
                            int64_t Lmax, int64_t avg, uint64_t seed, int32_t level,
                            const sclap_config* cfg, int32_t* block_out, int64_t* cut_out,
                            int32_t* best_trial_out, void* stream);

/* LP local search on one level (Sec. 3.1 last paragraph; active nodes,
 * Sec. 4).  block int32[n] in/out; phase selects the hash domain
 * (2 = refinement, 5 = initial-partitioning refinement). */
int sclap_refine(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* node_w,
                 const int32_t* edge_w, int32_t k, int64_t Lmax, uint64_t seed, int32_t phase,
                 int32_t level, const sclap_config* cfg, int32_t* block, int32_t* rounds_out,
                 void* stream);

/* Edge cut sum_{i<j} w(E_ij) (Sec. 2.1) of block (int32[n]); cut_out host. */
int sclap_cut(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* edge_w,
              const int32_t* block, int64_t* cut_out, void* stream);

/* ---- Serving (no counterpart in the paper, which partitions one graph per
 * run).  A server owns worker threads, each with its own CUDA stream on the
 * device that was current at creation.  Requests are copied in by
 * sclap_server_submit and queued in arrival order; a free worker takes the
 * longest run of queued requests from the front whose estimated device
 * memory fits in what the budget has left (a request alone is always
 * admitted when nothing else runs) and partitions them as one batch, as
 * sclap_partition_batch does.  Requests that arrive while a batch is on the
 * GPU go into the next batch a worker starts, which overlaps on the device
 * with those still running.  Each result is bit-identical to what
 * sclap_partition returns for the same request alone.
 *
 * Threads: submit and poll may be called from any threads at once; each
 * request id must be polled by one thread at a time; no other call may be in
 * progress on the server when sclap_server_destroy is called. ---- */
typedef struct sclap_server sclap_server;

typedef struct sclap_server_options {
  int64_t device_budget_bytes; /* admission budget; 0 = 120 GiB                   */
  int32_t workers;             /* batches in flight at once (0 = 2, at most 16)   */
  int32_t max_batch;           /* requests per batch (0 = 512)                    */
  int64_t linger_us;           /* wait for a partial batch to fill (0 = none)     */
} sclap_server_options;

/* cfg NULL = defaults; opts NULL = all defaults.  *out receives the server. */
int sclap_server_create(const sclap_config* cfg, const sclap_server_options* opts,
                        sclap_server** out);

/* Queue one partition request.  Arrays in HOST memory, format as above; the
 * server copies them before returning.  *request_id receives the request's
 * id.  Argument errors (and a request whose estimated device memory exceeds
 * the whole budget, SCLAP_ENOMEM) are returned here; errors found on the
 * device (malformed CSR, weight overflow, ...) are returned by the poll. */
int sclap_server_submit(sclap_server* srv, int64_t n, const int64_t* row_ptr, const int32_t* col,
                        const int32_t* node_w, const int32_t* edge_w, int32_t k, double eps,
                        uint64_t seed, int64_t* request_id);

/* Result of a request.  timeout_ms: 0 = do not wait, < 0 = wait until done,
 * > 0 = wait at most that long.  Returns SCLAP_PENDING if the request has
 * not finished; otherwise its status (SCLAP_OK, or an error code), writes
 * the outputs (block_out host int32[n]; cut, max block weight; each may be
 * NULL) when the status is SCLAP_OK or SCLAP_EINFEASIBLE, writes the time
 * from submit to completion in milliseconds, and releases the request (its
 * id is then unknown: SCLAP_EINVAL). */
int sclap_server_poll(sclap_server* srv, int64_t request_id, int32_t timeout_ms,
                      int32_t* block_out, int64_t* cut_out, int64_t* max_block_weight_out,
                      double* latency_ms_out);

/* Stops the workers after their current batches, drops queued requests and
 * frees the server. */
int sclap_server_destroy(sclap_server* srv);

/* ---- Cut and block weights without device allocation.  The paper has no
 * counterpart: this is a deployment variant of sclap_cut that also returns
 * the weight of every block.
 *
 * Every other entry point takes working memory from the CUDA allocator.
 * This one does not: its working memory is one fixed array in device global
 * memory, compiled into the library (2 + SCLAP_CUT_STATIC_MAX_K 64-bit words,
 * about 32 KB per device).  It is meant for callers that cannot allocate
 * device memory when they ask for the measure, e.g. a process that has
 * handed nearly all device memory to another allocator and keeps it, or a
 * latency-sensitive loop that must not enter the allocator, where an
 * allocation can block or fail.
 *
 * Arguments: the graph (device pointers, format as above; col may be NULL
 * only when row_ptr[n] == 0; node_w / edge_w NULL = unit), block int32[n]
 * on the device with every id in [0, k), 1 <= k <= min(n,
 * SCLAP_CUT_STATIC_MAX_K).  Outputs on the HOST: cut_out (int64, may be
 * NULL) and block_w_out (int64[k], c(V_i) per block, may be NULL).  The
 * work is ordered on `stream` and the call synchronises it before
 * returning.  Results equal sclap_cut's cut on the same input.
 *
 * Errors: k above SCLAP_CUT_STATIC_MAX_K, k > n, n out of range, NULL
 * row_ptr or block, or a block id outside [0, k) -> SCLAP_EINVAL; row_ptr
 * not starting at 0 or decreasing, a neighbour id outside [0, n), a
 * self-loop or a non-positive weight -> SCLAP_ECSR.  Symmetry is not
 * checked.
 *
 * Synchronisation: every call reads row_ptr[n] back to the host and waits
 * for `stream` twice (before its kernels and before returning), so it
 * cannot be called while `stream` is being captured into a CUDA graph.
 *
 * Set-up: the first call on a device looks up the array's device address
 * (once per device, with that device current), so that first call must come
 * before any stream capture starts.  The array is shared by all callers on
 * a device and keeps the last call's contents (each call clears the words
 * it uses first): calls that overlap in time (from two host threads, or on
 * two streams) race on it and must be serialised by the caller. */
#define SCLAP_CUT_STATIC_MAX_K 4096
int sclap_cut_static(int64_t n, const int64_t* row_ptr, const int32_t* col,
                     const int32_t* node_w, const int32_t* edge_w, const int32_t* block,
                     int32_t k, int64_t* cut_out, int64_t* block_w_out, void* stream);

/* ---- Host-side fault injection for tests (no counterpart in the paper).
 * Makes the library's own failure paths run without faulting the GPU:
 *   wait_limit   iteration limit of every bounded device-side wait (the grid
 *                barriers of the admission kernel, ~0.5 us per iteration);
 *                0 restores the default (2^22, about two seconds).  A small
 *                value makes the waits run out: the call returns
 *                SCLAP_ETIMEOUT, and the library stays usable.
 *   probe_limit  probes allowed per insertion into the LP sweep's open-
 *                addressing tables; 0 restores the default (the table size,
 *                which never runs out).  A small value makes insertions
 *                fail: the call returns SCLAP_EINTERNAL.
 *   fail_allocs  the fail_allocs-th device allocation of the library from
 *                now on fails once, as if the device were out of memory (the
 *                call making it returns SCLAP_ENOMEM); 0 clears.
 * The setting is process-wide and stays until changed.  SCLAP_EINVAL for a
 * negative value or a limit above 2^32 - 1. ---- */
int sclap_debug_inject(int64_t wait_limit, int64_t probe_limit, int32_t fail_allocs);

/* ---- Bounds-check build (no counterpart in the paper).  The library
 * compiled with -DSCLAP_CHECK=1 (python -m paper_1402_3281_gb300.build
 * --check writes libsclap_check.so) checks the data-dependent indices of its
 * kernels (neighbours, labels, coarse ids, table slots) against their
 * arrays' lengths; an index out of range is not used, and the call returns
 * SCLAP_EINTERNAL ("bounds check failed").  It stands in for a memory
 * checker where none can be run.
 *   sclap_check_build()     1 in the bounds-check build, 0 otherwise.
 *   sclap_check_selftest()  bounds-check build only: a kernel checks one
 *                           index inside and one just past a 4-element device
 *                           array (the second access is intercepted, never
 *                           made); SCLAP_OK when exactly the second was
 *                           caught.  SCLAP_EINVAL in the normal build. ---- */
int sclap_check_build(void);
int sclap_check_selftest(void* stream);

/* ---- Launch tuning and autotuning (no counterpart in the paper).  Choices
 * of the LP sweep that change scheduling, never results:
 *   small_max_deg      rows of degree <= 8 or <= 16 get one thread per node
 *                      (longer rows up to 128 get one warp per node)
 *   small_ctas_per_sm  grid cap of the thread-per-node launch (1..32)
 *   warp_ctas_per_sm   grid cap of the warp-per-node launch (1..32)
 *   admit_ctas_per_sm  grid cap of the admission kernels (1..64)
 *   concurrent         1: the propose launches of a colour class run
 *                      concurrently on side streams; 0: one after another
 *   pdl                1: kernels that follow a kernel of the same stream in
 *                      the host-driven round loop are launched as
 *                      programmatic dependent launches; 0: plain launches
 *   fused_admission    1: the admission and application of a colour class
 *                      run as one cooperative launch whose phases are
 *                      separated by bounded grid-wide barriers (a barrier
 *                      that waits too long ends the call with
 *                      SCLAP_ETIMEOUT); 0: a chain of six launches
 *   contract_table_slots  slots of the contraction table per pass: a level
 *                      whose table is larger is contracted in passes over
 *                      ranges of coarse nodes (same result); 0: automatic,
 *                      half of the device memory still obtainable
 *   ip_trial_group     initial-partitioning trials whose graph copies exist
 *                      at once (the trials run group after group; same
 *                      result); 0: automatic, as many as fit in half of the
 *                      device memory still obtainable
 *   contract_merge     1: contraction sorts the fine nodes by coarse node
 *                      and merges each coarse node's arcs in shared memory
 *                      (a level whose merge regions do not fit in the
 *                      memory of one contraction pass falls back to the
 *                      hash tables); 0: hash tables (same result up to the
 *                      order of each coarse row's arcs)
 * The setting is process-wide; defaults 16, 8, 8, 16, 1, 1, 0, 0, 0, 0. ---- */
typedef struct sclap_tuning {
  int32_t small_max_deg;
  int32_t small_ctas_per_sm;
  int32_t warp_ctas_per_sm;
  int32_t admit_ctas_per_sm;
  int32_t concurrent;
  int32_t pdl;
  int32_t fused_admission;
  int32_t contract_table_slots;
  int32_t ip_trial_group;
  int32_t contract_merge;
} sclap_tuning;
void sclap_get_tuning(sclap_tuning* out);
/* SCLAP_EINVAL for a value out of range (the setting is then unchanged). */
int sclap_set_tuning(const sclap_tuning* t);
/* Picks the tuning for a workload by coordinate descent: the batch (as for
 * sclap_partition_batch) is partitioned `reps` times per candidate setting
 * (each parameter in turn over a few values, the others fixed), the median
 * wall time is compared, and a candidate replaces the current choice only if
 * at least 2% faster.  Every run must give the same cut for every graph as
 * the first (SCLAP_EINTERNAL otherwise).  The best setting is installed and
 * written to *out (may be NULL).  The graphs' outputs hold the last run's
 * (identical) results. */
int sclap_autotune(int32_t count, sclap_graph* graphs, const sclap_config* cfg,
                   int32_t device_ptrs, int32_t reps, sclap_tuning* out, void* stream);

/* ---- Instrumentation (no counterpart in the paper).  Process-wide
 * counters read by the benchmark: every kernel launch is counted; with
 * profiling enabled, each launch of the LP propose sweep is bracketed by CUDA
 * events on its stream and its nodes/arcs are tallied per kernel family
 * (0: one thread per node, degree <= 16; 1: one warp per node, degree
 * 17..128, and CTAs of 128 threads per node, degree <= 512; 2: CTAs of
 * 256/512 threads, degree <= 8192; 3: one CTA per node with a global table).
 * Times are device milliseconds. ---- */
typedef struct sclap_profile {
  int64_t kernel_launches;
  int64_t propose_launches[4];
  double propose_ms[4];        /* per launch, events on its own stream      */
  int64_t propose_nodes[4];
  int64_t propose_arcs[4];
  double sweep_ms;             /* propose phases: the families of a sub-round
                                  run concurrently; first launch to last     */
  int64_t sweeps;
  int64_t propose_arcs_unit;   /* of all propose arcs, those on levels with
                                  unit edge weights (no weight array read)   */
} sclap_profile;
void sclap_profile_enable(int on);
void sclap_profile_reset(void);
void sclap_profile_read(sclap_profile* out);
/* One record per LP sub-round run while profiling was enabled, 7 doubles
 * each: run kind (1 clustering, 2 refinement, 3 initial-partitioning trial,
 * 5 trial refinement, 6 repair), round, colour class, listed nodes, their
 * arcs, propose-phase milliseconds (fork to join), admission milliseconds
 * (join to the end of apply).  Writes at most `cap` records to `out` (may be
 * NULL) and returns the number recorded since the last reset. */
int64_t sclap_profile_phases(double* out, int64_t cap);
/* Timeline mode: an event after every kernel launch and after every host
 * wait; sclap_profile_dump writes "name launches total_ms" lines (time since
 * the previous mark of the same call: device time plus any idle gap) into
 * buf (cap bytes, NUL-terminated), clears the timeline and returns the length
 * the full text needs. */
void sclap_profile_timeline(int on);
int64_t sclap_profile_dump(char* buf, int64_t cap);

#ifdef __cplusplus
}
#endif
#endif
