/*
 * sclap_oracle.h -- CPU oracle for multilevel size-constrained label
 * propagation (SCLaP) graph partitioning.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that
 * the CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product path never does.
 * It shares no code, header or constant table with the CUDA library.
 *
 * Two variants of the paper's method are implemented, single-threaded:
 *
 *  ORC_SEQ  -- the sequential algorithm as the paper states it: nodes visited
 *              in increasing degree order (Sec. 4, "Node Ordering"), every
 *              move applied immediately (Sec. 3.1), refinement driven by the
 *              two FIFO active-node queues (Sec. 4 "Active Nodes", App. B.2).
 *  ORC_SYNC -- a deterministic round-synchronous reading of the same method:
 *              each round is split into colour classes (sub-rounds); in a
 *              sub-round every node decides against the state at the
 *              sub-round start and the size bound is enforced by a
 *              deterministic admission rule.  The CUDA path reproduces this
 *              variant bit for bit.
 *
 * Conventions: graphs are undirected CSR (xadj int64[n+1], adj int32[m]),
 * symmetric, no self-loops, positive int32 node and edge weights.  All
 * weights and sums are integers; the only floating-point step is the
 * (1+eps) product in the balance bound.
 */
#ifndef SCLAP_ORACLE_H
#define SCLAP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_SYNC = 0, ORC_SEQ = 1 };
enum { ORC_MODE_CLUSTER = 0, ORC_MODE_REFINE = 1 };
/* Hash-domain tags for the counter-based generator (one per phase). */
enum {
  ORC_PH_CLUSTER = 1, ORC_PH_REFINE = 2, ORC_PH_TRIAL = 3,
  ORC_PH_GGG = 4, ORC_PH_IPREF = 5, ORC_PH_REPAIR = 6, ORC_PH_ENSEMBLE = 7, ORC_PH_VCYCLE = 8
};
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_EOVERFLOW = -2, ORC_EINFEASIBLE = -3 };

typedef struct orc_config {
  int32_t lp_rounds_coarse; /* max LP rounds per level when clustering (Sec. 5: 10) */
  int32_t lp_rounds_refine; /* max LP rounds per level when refining (10)           */
  int32_t f;                /* cluster bound factor, W = Lmax / f (Sec. 5: 18)     */
  int32_t coarse_min_nodes; /* coarsen while n > max(coarse_min_nodes, 60k)        */
  int32_t ip_trials;        /* initial-partitioning trials, best kept              */
  int32_t sub_rounds;       /* colour classes per synchronous round                */
  int32_t repair_rounds;    /* cap on final balance-repair rounds                  */
  int32_t max_levels;       /* cap on hierarchy depth                              */
  int32_t cluster_active;   /* 1: active nodes during coarsening (Sec. 4 "Active
                               Nodes", configuration A of Table 2): after the first
                               round, only nodes next to a node that changed its
                               cluster in the previous round are visited            */
  int32_t random_order;     /* sequential variant only, 1: visit nodes in hashed
                               random order instead of increasing degree
                               (configuration R of Table 2)                         */
  int32_t ensemble;         /* 1: ensemble clusterings during coarsening (Sec. 4
                               "Ensemble Clusterings", configuration E): each level
                               contracts the overlay of l clusterings             */
  int32_t ensemble_size;    /* l; 0 = the paper's rule (Sec. 5): 18 if k < 16, 7 if
                               k is 16 or 32, 3 if k > 32                           */
  int32_t vcycles;          /* multilevel cycles (Sec. 4 "Iterated Multilevel
                               Algorithms", App. A; configuration V, Sec. 5: 3);
                               1 = one plain multilevel run                         */
} orc_config;

typedef struct orc_stats {
  int32_t levels;               /* graphs in the hierarchy (input included)   */
  int64_t level_n[64];
  int64_t level_m[64];          /* arcs (2 x undirected edges)                */
  int32_t cluster_rounds[64];   /* LP rounds run while clustering level l     */
  int32_t refine_rounds[64];    /* LP rounds run while refining level l       */
  int32_t ip_best_trial;
  int64_t ip_cut;
  int64_t Lmax, U;
  int32_t repair_rounds;
} orc_stats;

void orc_default_config(orc_config* cfg);

/* SplitMix64 output function (Steele, Lea, Flood 2014) and the keyed chain
 * built from it; exposed so tests can pin the generator. */
uint64_t orc_mix64(uint64_t x);
uint64_t orc_hkey(uint64_t seed, uint64_t phase, uint64_t level, uint64_t round);

/* Balance bound Lmax = floor((1+eps) * ceil(cV/k)) (Sec. 2.1, unweighted form
 * applied to c(V)), cluster bound U = max(max_v c(v), floor(Lmax/f))
 * (Sec. 3.1). */
int orc_bounds(int64_t cV, int32_t max_c, int32_t k, double eps, int32_t f,
               int64_t* Lmax, int64_t* U);

/* One synchronous LP round (all colour classes) in CLUSTER or REFINE mode.
 * label/W are updated in place; W has nlabels entries.  active_cur==NULL
 * means every node is active; active_next (nullable, n bytes) receives the
 * neighbours of moved nodes.  Returns ORC_OK. */
int orc_lp_round(int32_t mode, int64_t n, const int64_t* xadj, const int32_t* adj,
                 const int32_t* nw, const int32_t* ew, int32_t* label, int64_t* W,
                 int64_t nlabels, int64_t bound, uint64_t rkey, int32_t sub_rounds,
                 const uint8_t* active_cur, uint8_t* active_next, int64_t* moved);

/* Size-constrained clustering of one level (Sec. 3.1), up to
 * cfg->lp_rounds_coarse rounds, stopping after a round that moved fewer than
 * 5% of the nodes.  label_out[v] is a node id (the cluster's original
 * representative). */
int orc_cluster(int32_t variant, int64_t n, const int64_t* xadj, const int32_t* adj,
                const int32_t* nw, const int32_t* ew, int64_t U, uint64_t seed,
                int32_t level, const orc_config* cfg, int32_t* label_out,
                int32_t* rounds_out);

/* Clustering hierarchy without a partitioning target (Sec. 3.1 clustering
 * and contraction, repeated as in the coarsening phase of Sec. 3): cluster
 * the current graph with bound U (level l uses hash level l), contract, and
 * repeat while the current graph has more than stop_nodes nodes, the
 * hierarchy has fewer than cfg->max_levels graphs, and the contraction
 * removes at least 5% of the nodes (a contraction removing less is
 * discarded).  comm_out[v] (n entries) receives the node of the last graph
 * that input node v belongs to; *levels_out the number of contractions
 * kept; level_n_out[0..min(levels, cap-1)] the node counts, input first. */
/* Size-constrained clustering that respects a partition (App. A): as
 * orc_cluster, but a node may only join clusters inside its own block blk[v]
 * (blk: n entries), so every cluster lies inside one block. */
int orc_cluster_in_blocks(int32_t variant, int64_t n, const int64_t* xadj, const int32_t* adj,
                          const int32_t* nw, const int32_t* ew, int64_t U, uint64_t seed,
                          int32_t level, const orc_config* cfg, const int32_t* blk,
                          int32_t* label_out, int32_t* rounds_out);

/* Overlay of two clusterings (Sec. 4 "Ensemble Clusterings"): two nodes
 * share an overlay cluster iff they share a cluster in a and in b.  Overlay
 * ids are numbered 0, 1, ... in the order the (a[v], b[v]) pairs first occur
 * for v = 0..n-1 (the paper's hash-map construction). */
int orc_overlay(int64_t n, const int32_t* a, const int32_t* b, int32_t* out);

int orc_cluster_hierarchy(int32_t variant, int64_t n, const int64_t* xadj, const int32_t* adj,
                          const int32_t* nw, const int32_t* ew, int64_t U, int64_t stop_nodes,
                          uint64_t seed, const orc_config* cfg, int32_t* comm_out,
                          int32_t* levels_out, int64_t* level_n_out, int32_t cap);

/* Cluster contraction (Sec. 3.1): coarse id = rank of the cluster label;
 * outputs sized by the fine graph (n, n+1, m entries). */
int orc_contract(int64_t n, const int64_t* xadj, const int32_t* adj, const int32_t* nw,
                 const int32_t* ew, const int32_t* label, int32_t* cmap_out,
                 int64_t* nc_out, int32_t* cnw_out, int64_t* cxadj_out,
                 int32_t* cadj_out, int32_t* cew_out, int64_t* mc_out);

/* One greedy-graph-growing trial followed by water-filling of leftovers;
 * block_out in [0,k), W_out has k entries. */
int orc_ggg(int64_t n, const int64_t* xadj, const int32_t* adj, const int32_t* nw,
            const int32_t* ew, int32_t k, int64_t avg, uint64_t tkey, int32_t level,
            int32_t* block_out, int64_t* W_out);

/* Initial partitioning: cfg->ip_trials trials (growing + LP refinement),
 * best by (overload, cut, trial). */
int orc_initial_partition(int32_t variant, int64_t n, const int64_t* xadj,
                          const int32_t* adj, const int32_t* nw, const int32_t* ew,
                          int32_t k, int64_t Lmax, int64_t avg, uint64_t seed,
                          int32_t level, const orc_config* cfg, int32_t* block_out,
                          int64_t* cut_out, int32_t* best_trial_out);

/* LP as local search (Sec. 3.1, last paragraph) on one level with active
 * nodes (Sec. 4), bound Lmax.  block is in/out. */
int orc_refine(int32_t variant, int64_t n, const int64_t* xadj, const int32_t* adj,
               const int32_t* nw, const int32_t* ew, int32_t k, int64_t Lmax,
               uint64_t seed, int32_t phase, int32_t level, const orc_config* cfg,
               int32_t* block, int32_t* rounds_out);

/* Final balance repair; returns ORC_EINFEASIBLE if blocks stay overloaded. */
int orc_repair(int64_t n, const int64_t* xadj, const int32_t* adj, const int32_t* nw,
               const int32_t* ew, int32_t k, int64_t Lmax, uint64_t seed,
               const orc_config* cfg, int32_t* block, int32_t* rounds_out);

/* Edge cut sum_{i<j} w(E_ij) (Sec. 2.1). */
int64_t orc_cut(int64_t n, const int64_t* xadj, const int32_t* adj, const int32_t* ew,
                const int32_t* block);

/* Whole multilevel partitioner.  nw/ew may be NULL (unit weights).  Returns
 * ORC_OK, or ORC_EINFEASIBLE with a best-effort partition. */
int orc_partition(int32_t variant, int64_t n, const int64_t* xadj, const int32_t* adj,
                  const int32_t* nw, const int32_t* ew, int32_t k, double eps,
                  uint64_t seed, const orc_config* cfg, int32_t* block_out,
                  int64_t* cut_out, int64_t* maxbw_out, orc_stats* stats);

#ifdef __cplusplus
}
#endif
#endif
