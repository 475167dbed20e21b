// lp.cu -- one synchronous round of size-constrained label propagation
// (Sec. 3.1), as clustering (bound U) or local search (bound Lmax, active
// nodes, Sec. 4), over every slot of a batched level at once.
//
// A round splits the participating nodes into S colour classes by a per-node
// hash; each class is a sub-round:
//   propose  every node computes its connection to each neighbouring label
//            (degree-bucketed: one thread per node with its row sorted in
//            registers up to degree 16, one warp per node with a shared-
//            memory table up to 128, one CTA per node with a shared-memory
//            table up to 8192, a global-memory table for hubs) and proposes
//            the strongest eligible label;
//   resolve  a target whose proposals all fit admits them all; otherwise the
//            proposals into it form a segment, and the longest prefix in
//            (gain desc, priority asc, node asc) order that fits is admitted
//            (one warp ranks all pairs of a segment of <= 64 entries, one CTA
//            locates the boundary of a larger one by radix select);
//   source   (local search) forced moves out of an overloaded block are capped
//            at the block's excess the same way;
//   apply    labels and label weights are updated with integer atomics
//            (order-free, hence deterministic) and moved nodes activate their
//            neighbours.
#include "common.cuh"

namespace sclap {
namespace {

struct LPArgs {
  // level
  const int64_t* row_ptr;
  const int32_t* col;
  const int32_t* ew;
  const int32_t* nw;
  const int32_t* gid;
  int32_t narrow;          // 1: every connection sum is below 2^32
  int32_t arcs32;          // 1: the level has fewer than 2^32 arcs
  int64_t M;               // arcs of the level (length of col / ew)
  int64_t N;               // nodes of the level (length of label, col's range)
  int64_t nlabels;         // length of W and in_w
  // slots
  const int64_t* noff;
  const int64_t* loff;
  const int64_t* bound;
  uint64_t* rkey;
  const int32_t* nlab;
  int32_t* done;
  int64_t* moved;
  int32_t* rounds;
  // state
  int32_t* label;
  wgt_t* W;
  int64_t* in_w;
  int32_t mode;
  int32_t S;
  // sub-round lists: for each listed node {v, own label, weight, slot} and
  // {row start, degree}, written by the bucketing pass
  int4* rec;
  longlong2* rec2;
  int32_t* prop_t;
  uint64_t* prop_key;
  int8_t* adm;
  int8_t* stage;
  int32_t* grp;
  // overflow segments
  int32_t* ovf_cnt;
  int32_t* ovf_fill;
  int64_t* ovf_base;
  int64_t* ctr;          // admission segment counters (8 words, see adm_ctr)
  int32_t* seg_g;
  int64_t* seg_base;
  int32_t* seg_cnt;
  int64_t* seg_thr;
  uint64_t* ent_key;
  int32_t* ent_v;
  int32_t* ent_w;
  int32_t* ent_i;
  uint64_t* sel_key[2];  // radix-select survivors (two copies used in turn)
  int32_t* sel_v[2];
  int32_t* sel_w[2];
  // bucketing
  int32_t* bcnt;
  int32_t* bfill;
  int64_t* boff;
  int64_t* arcs;         // arcs scanned (statistics)
  int64_t* karcs;        // arcs per (colour, bucket) key
  int32_t* flags;        // [0]: a listed node sits in an overloaded block
  int16_t* nkey;         // bucket key of each node this round (-1: not listed)
  // active nodes: act[r & 1] holds round r's flags, act[(r + 1) & 1] the
  // next round's (both NULL when all nodes are always active)
  uint8_t* act[2];
  // moved rows longer than mark_big arcs (0: none on the level) activate
  // their neighbours through a queue of arc chunks, per colour class
  // mqn[sub] entries, read by a launch of their own
  int64_t mark_big;
  longlong2* mq;
  int32_t* mqn;
  // round state on the device, so that a level's rounds need no host
  // decision: the round index, slots still running after k_round_end, and
  // the limits of the run
  int32_t* rnd;
  int32_t* live;
  int32_t rounds_max;
  int32_t stop_rule;
  // V-cycles: block of every node in a partition the clustering must respect
  // (a node joins only clusters of its own block), or NULL
  const int32_t* rblk;
  int32_t* err;
  uint32_t wait_limit;    // iterations of a bounded grid-barrier wait
  uint32_t probe_limit;   // probes of an open-addressing table (sclap_debug_inject)
};

__device__ __forceinline__ const uint8_t* act_cur(const LPArgs& a) {
  return a.act[0] ? a.act[a.rnd[0] & 1] : nullptr;
}
__device__ __forceinline__ uint8_t* act_next(const LPArgs& a) {
  return a.act[0] ? a.act[(a.rnd[0] + 1) & 1] : nullptr;
}
// Node range [beg, beg + cnt) of buckets [b0, b1) of colour class `sub`,
// read on the device from the bucketing offsets.
__device__ __forceinline__ void sub_range(const LPArgs& a, int sub, int b0, int b1,
                                          int64_t* beg, int64_t* cnt) {
  *beg = a.boff[sub * NB + b0];
  *cnt = a.boff[sub * NB + b1] - *beg;
}

struct NodeCtx {
  int32_t v, slot, own, cv, vb;
  int64_t bound, loff, rs, re;
  uint64_t hv;
};

__device__ __forceinline__ NodeCtx load_node(const LPArgs& a, int64_t i) {
  const int4 r = a.rec[i];
  const longlong2 r2 = a.rec2[i];
  NodeCtx c;
  c.v = r.x;
  c.own = r.y;
  c.cv = r.z;
  c.slot = r.w;
  c.rs = r2.x;
  c.re = r2.x + r2.y;
  c.bound = a.bound[c.slot];
  c.loff = a.loff[c.slot];
  c.hv = mix64(a.rkey[c.slot] ^ (uint64_t)(c.v - a.noff[c.slot]));
  c.vb = a.rblk ? a.rblk[c.v] : 0;
  return c;
}

// Block of cluster C when clustering must respect a partition (labels are
// node ids while clustering, so it is the block of node C); vb otherwise, so
// the comparison passes.  Loaded only for candidates still in question.
__device__ __forceinline__ int32_t cand_block(const LPArgs& a, const NodeCtx& c, bool need,
                                              int32_t C) {
  return a.rblk && need ? a.rblk[C] : c.vb;
}

__device__ __forceinline__ Cand make_cand(const NodeCtx& c, int32_t C, int64_t conn) {
  const int32_t Cl = (int32_t)(C - c.loff);
  return Cand{conn, mix64(c.hv ^ (uint64_t)(uint32_t)Cl), Cl};
}

__device__ __forceinline__ void write_prop(const LPArgs& a, int64_t i, const NodeCtx& c,
                                           const Cand& best, int64_t own_conn, bool overloaded) {
  const bool move = best.conn >= 0 && (overloaded || best.conn > own_conn);
  if (move) {
    const int32_t t = (int32_t)(c.loff + best.C);
    a.prop_t[i] = t;
    a.prop_key[i] = admission_key(best.conn - own_conn, (uint32_t)c.hv);
    if (SCLAP_OK(t, a.nlabels, a.err)) atomicAdd(ull(&a.in_w[t]), (unsigned long long)c.cv);
  } else {
    a.prop_t[i] = -1;
  }
}

// ------------------------------------------------------------- round control
__global__ void k_round_begin(LPArgs a, int32_t nslots, int32_t phase,
                              const uint64_t* seed, const int32_t* level, int32_t raw_key) {
  griddep_wait();
  const int32_t r = a.rnd[0];
  if (blockIdx.x == 0) {                 // per-round counters of the bucketing
    for (int j = threadIdx.x; j < a.S * NB; j += blockDim.x) {
      a.bcnt[j] = 0;
      a.karcs[j] = 0;
    }
    if (threadIdx.x == 0) {
      a.live[0] = 0;
      a.flags[0] = 0;
    }
    if (threadIdx.x < 8) a.ctr[threadIdx.x] = 0;   // admission segment counters
    if (a.mqn)
      for (int j = threadIdx.x; j < a.S; j += blockDim.x) a.mqn[j] = 0;
  }
  for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < nslots;
       s += gridDim.x * blockDim.x) {
    if (a.done[s]) continue;
    if (a.mode == MODE_REPAIR) {
      int64_t mx = 0;
      const int64_t lo = a.loff[s];
      for (int32_t b = 0; b < a.nlab[s]; ++b) mx = max64(mx, (int64_t)a.W[lo + b]);
      if (mx <= a.bound[s]) { a.done[s] = 1; continue; }
    }
    a.rkey[s] = raw_key ? seed[s] : hkey(seed[s], (uint64_t)phase, (uint64_t)level[s], (uint64_t)r);
    a.moved[s] = 0;
  }
}

__global__ void k_round_end(LPArgs a, int32_t nslots) {
  griddep_wait();
  int live = 0;
  for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < nslots;
       s += gridDim.x * blockDim.x) {
    if (a.done[s]) continue;
    a.rounds[s] += 1;
    const int64_t n = a.noff[s + 1] - a.noff[s];
    if (a.stop_rule && 20 * a.moved[s] < n) a.done[s] = 1;
    else ++live;
  }
  if (live) atomicAdd(a.live, live);
}

// Decides whether the run goes on: another round is allowed, the round just
// finished listed some node, and some slot is still running.  Advances the
// round index and, inside a graph, sets the loop's condition.
__global__ void k_round_cond(LPArgs a, int32_t nkeys, cudaGraphConditionalHandle h,
                             int32_t use_handle, int32_t* cont) {
  griddep_wait();
  const int32_t r = a.rnd[0];
  const bool more = r + 1 < a.rounds_max && a.boff[nkeys] > 0 && a.live[0] > 0;
  a.rnd[0] = r + 1;
  cont[0] = more ? 1 : 0;
  if (use_handle) cudaGraphSetConditional(h, more ? 1u : 0u);
}

// ------------------------------------------------------------- bucketing
// Pass 0 decides each node's (colour, bucket) key, stores it and counts per
// key; pass 1 scatters the listed nodes into their key's range.  Both passes
// aggregate per key in shared memory and touch the global counters once per
// key per block (same-address global atomics serialise in L2).
constexpr int BK_NT = 256;
constexpr int BK_PER = 8;                    // nodes per thread
constexpr int BK_TILE = BK_NT * BK_PER;      // nodes per block
constexpr int MAX_KEYS = 64 * NB;

__device__ __forceinline__ int node_key(const LPArgs& a, const uint8_t* ac, int64_t v,
                                        int64_t* deg_out, bool* ov_out) {
  const int32_t s = slot_at(a.gid, v);
  if (a.done[s]) return -1;
  const int64_t deg = a.row_ptr[v + 1] - a.row_ptr[v];
  bool take, ov = false;
  if (a.mode == MODE_CLUSTER) {
    take = deg > 0 && (ac == nullptr || ac[v]);
  } else {
    ov = a.W[a.label[v]] > a.bound[s];
    if (a.mode == MODE_REPAIR) take = ov;
    else take = (ac == nullptr || ac[v]) && (deg > 0 || ov);
  }
  if (!take) return -1;
  const uint64_t hv = mix64(a.rkey[s] ^ (uint64_t)(v - a.noff[s]));
  const int sub = (int)((uint32_t)(hv >> 32) % (uint32_t)a.S);
  *deg_out = deg;
  *ov_out = ov;
  return sub * NB + bucket_of(deg, ov);
}

// Per-key node counts and arc sums, first per CTA in shared memory.  The arc
// sums are 64-bit words, added with 32-bit atomics on the low word when the
// level has fewer than 2^32 arcs (a CTA's sum is then below 2^32 too): the
// lanes of a warp meet only a few keys, and contended 64-bit shared atomics
// serialise.
__global__ void __launch_bounds__(BK_NT) k_bucket_count(LPArgs a, int64_t N) {
  griddep_wait();
  __shared__ int sh_cnt[MAX_KEYS];
  __shared__ unsigned long long sh_arcs[MAX_KEYS];
  __shared__ int sh_ov;
  const int nkeys = a.S * NB;
  for (int j = threadIdx.x; j < nkeys; j += BK_NT) { sh_cnt[j] = 0; sh_arcs[j] = 0; }
  if (threadIdx.x == 0) sh_ov = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * BK_TILE;
  bool any_ov = false;
  const uint8_t* ac = act_cur(a);
  uint8_t* an = act_next(a);
#pragma unroll
  for (int j = 0; j < BK_PER; ++j) {
    const int64_t v = base + (int64_t)j * BK_NT + threadIdx.x;
    if (v >= N) break;
    if (an) an[v] = 0;                 // next round's flags start cleared
    int64_t deg = 0;
    bool ov = false;
    const int key = node_key(a, ac, v, &deg, &ov);
    a.nkey[v] = (int16_t)key;
    if (key >= 0) {
      atomicAdd(&sh_cnt[key], 1);
      if (a.arcs32) atomicAdd(reinterpret_cast<unsigned int*>(&sh_arcs[key]), (unsigned int)deg);
      else atomicAdd(&sh_arcs[key], (unsigned long long)deg);
      any_ov = any_ov || ov;
    }
  }
  if (any_ov) sh_ov = 1;
  __syncthreads();
  for (int j = threadIdx.x; j < nkeys; j += BK_NT) {
    if (sh_cnt[j]) {
      atomicAdd(&a.bcnt[j], sh_cnt[j]);
      atomicAdd(ull(&a.karcs[j]), sh_arcs[j]);
    }
  }
  if (threadIdx.x == 0 && sh_ov) atomicOr(&a.flags[0], 1);
}

__global__ void __launch_bounds__(BK_NT) k_bucket_scatter(LPArgs a, int64_t N) {
  griddep_wait();
  __shared__ int sh_cnt[MAX_KEYS];
  __shared__ int sh_base[MAX_KEYS];
  const int nkeys = a.S * NB;
  for (int j = threadIdx.x; j < nkeys; j += BK_NT) sh_cnt[j] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * BK_TILE;
  int key[BK_PER], rank[BK_PER];
#pragma unroll
  for (int j = 0; j < BK_PER; ++j) {
    const int64_t v = base + (int64_t)j * BK_NT + threadIdx.x;
    key[j] = v < N ? a.nkey[v] : -1;
    rank[j] = key[j] >= 0 ? atomicAdd(&sh_cnt[key[j]], 1) : 0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nkeys; j += BK_NT)
    sh_base[j] = sh_cnt[j] ? (int)atomicAdd(&a.bfill[j], sh_cnt[j]) : 0;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < BK_PER; ++j) {
    if (key[j] < 0) continue;
    const int64_t v = base + (int64_t)j * BK_NT + threadIdx.x;
    const int64_t pos = a.boff[key[j]] + sh_base[key[j]] + rank[j];
    const int64_t rs = a.row_ptr[v];
    a.rec[pos] = make_int4((int32_t)v, a.label[v], wat(a.nw, v), slot_at(a.gid, v));
    a.rec2[pos] = make_longlong2(rs, a.row_ptr[v + 1] - rs);
  }
}

__global__ void k_bucket_offsets(LPArgs a, int nkeys) {
  griddep_wait();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t s = 0, arcs = 0;
    for (int j = 0; j < nkeys; ++j) {
      a.boff[j] = s;
      s += a.bcnt[j];
      a.bfill[j] = 0;
      arcs += a.karcs[j];
    }
    a.boff[nkeys] = s;
    a.arcs[0] += arcs;
  }
}

// ------------------------------------------------------------- propose
// Degrees <= MAXD (4, 8 or 16): one thread per node, the whole row in
// registers.  The row's (label, weight) pairs are sorted by label with a
// bitonic network (compile-time indices, so the arrays stay in registers);
// equal labels then form runs, the run sums are the connections, and the
// last entry of each run is that label's candidate.  No cross-lane
// operation is involved, and apart from the loop every step is predicated
// loads, compares and selects.  Unused entries carry label INT32_MAX and
// sort to the end.  When the row's total weight exceeds int32 (heavy coarse
// edges) the run sums are kept in 64 bits.
template <int MAXD, typename SumT>
__device__ __forceinline__ void sorted_row_best(const LPArgs& a, const NodeCtx& c, int32_t (&C)[MAXD],
                                                int32_t (&w)[MAXD], long long& oc, Cand& best) {
#pragma unroll
  for (int k = 2; k <= MAXD; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int i = 0; i < MAXD; ++i) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const bool sw = up ? (C[i] > C[l]) : (C[i] < C[l]);
          const int32_t c0 = sw ? C[l] : C[i], c1 = sw ? C[i] : C[l];
          const int32_t w0 = sw ? w[l] : w[i], w1 = sw ? w[i] : w[l];
          C[i] = c0; C[l] = c1; w[i] = w0; w[l] = w1;
        }
      }
    }
  }
  SumT run[MAXD];
  bool end[MAXD];
#pragma unroll
  for (int j = 0; j < MAXD; ++j) {
    const SumT prev = j > 0 ? run[j - 1] : (SumT)0;
    run[j] = (j > 0 && C[j] == C[j - 1]) ? prev + (SumT)w[j] : (SumT)w[j];
    end[j] = C[j] != INT32_MAX && (j == MAXD - 1 || C[j] != C[j + 1]);
  }
  int32_t Wl[MAXD], Bl[MAXD];
#pragma unroll
  for (int j = 0; j < MAXD; ++j) {
    const bool q = end[j] & (C[j] != c.own);
    Wl[j] = q ? SCLAP_LD(a.W, C[j], a.nlabels, a.err) : 0;
    Bl[j] = cand_block(a, c, q, C[j]);
  }
#pragma unroll
  for (int j = 0; j < MAXD; ++j) {
    const bool own = end[j] & (C[j] == c.own);
    oc = own ? (long long)run[j] : oc;
    const bool elig = end[j] & (C[j] != c.own) & ((int64_t)Wl[j] + c.cv <= c.bound) &
                      (Bl[j] == c.vb);
    const int32_t Cl = (int32_t)(C[j] - c.loff);
    const Cand x{(int64_t)run[j], mix64(c.hv ^ (uint64_t)(uint32_t)Cl), Cl};
    best = cand_pick(elig & cand_better(x, best), x, best);
  }
}

template <int MAXD>
__device__ __forceinline__ void propose_thread(const LPArgs& a, int64_t lbeg, int64_t cnt,
                                               int64_t blk, int64_t nblk) {
  for (int64_t li = blk * blockDim.x + threadIdx.x; li < cnt; li += nblk * blockDim.x) {
    const int64_t i = lbeg + li;
    const NodeCtx c = load_node(a, i);
    const int deg = (int)(c.re - c.rs);
    int32_t C[MAXD], w[MAXD];
    int64_t total = 0;
#pragma unroll
    for (int j = 0; j < MAXD; ++j) {
      const bool in = j < deg;
      w[j] = in ? wat(a.ew, c.rs + j) : 0;
      C[j] = in ? a.col[c.rs + j] : -1;
      total += w[j];
    }
#pragma unroll
    for (int j = 0; j < MAXD; ++j) C[j] = C[j] >= 0 ? SCLAP_LD(a.label, C[j], a.N, a.err) : INT32_MAX;
    long long oc = 0;
    Cand best{-1, 0, 0};
    if (total <= INT32_MAX) sorted_row_best<MAXD, int32_t>(a, c, C, w, oc, best);
    else sorted_row_best<MAXD, int64_t>(a, c, C, w, oc, best);
    write_prop(a, i, c, best, oc, false);
  }
}

// The small-degree buckets of one sub-round in one launch: block ranges
// [bs[j], bs[j+1]) serve bucket j (degree <= 4, <= 8, <= 16), one thread per
// node.
// The grid is split among the three buckets in proportion to the blocks each
// needs (256 nodes per block), every non-empty bucket getting at least one;
// every block computes the same split from the device offsets.
// Split of a grid of G blocks among three buckets needing need[j] blocks
// (tot = sum > G): floor of the proportional share, raised to one for every
// non-empty bucket, and the difference to G (at most two blocks too many,
// or some too few) settled on the bucket with the largest share, which
// holds at least G / 3 blocks, so every non-empty bucket keeps >= 1 when
// G >= 3 (the host never launches fewer than the SM count).
__host__ __device__ __forceinline__ void split_small_grid(int64_t G, const int64_t (&need)[3],
                                                          int64_t tot, int64_t (&g)[3]) {
  int64_t used = 0;
  int big = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    g[j] = need[j] ? max64(1, G * need[j] / tot) : 0;
    used += g[j];
    if (g[j] > g[big]) big = j;
  }
  g[big] += G - used;
}

__global__ void __launch_bounds__(256, 4) k_propose_small(LPArgs a, int32_t sub, int32_t nb) {
  griddep_wait();
  const int64_t* bo = a.boff + sub * NB;
  int64_t c[3], need[3], tot = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    c[j] = j < nb ? bo[j + 1] - bo[j] : 0;
    need[j] = (c[j] + 255) / 256;
    tot += need[j];
  }
  if (tot == 0) return;
  const int64_t G = gridDim.x;
  int64_t g[3];
  if (tot <= G) {
#pragma unroll
    for (int j = 0; j < 3; ++j) g[j] = need[j];
  } else {
    split_small_grid(G, need, tot, g);
    // a non-empty bucket without a block would leave its nodes unproposed
    if (blockIdx.x == 0 && threadIdx.x == 0 &&
        ((need[0] && g[0] < 1) || (need[1] && g[1] < 1) || (need[2] && g[2] < 1)))
      atomicOr(a.err, DERR_INTERNAL);
  }
  const int64_t b = blockIdx.x;
  if (b < g[0]) propose_thread<4>(a, bo[0], c[0], b, g[0]);
  else if (b < g[0] + g[1]) propose_thread<8>(a, bo[1], c[1], b - g[0], g[1]);
  else if (b < g[0] + g[1] + g[2]) propose_thread<16>(a, bo[2], c[2], b - g[0] - g[1], g[2]);
}

__device__ __forceinline__ int64_t table_get(const int32_t* keys, const unsigned long long* vals,
                                             int logcap, int32_t C) {
  const uint32_t mask = (1u << logcap) - 1;
  uint32_t s = table_slot(C, logcap);
  for (uint32_t p = 0; p <= mask; ++p) {
    const int32_t k = keys[s];
    if (k == C) return (int64_t)vals[s];
    if (k == -1) return 0;
    s = (s + 1) & mask;
  }
  return 0;
}

template <int NT>
__device__ void block_reduce(long long& oc, Cand& cd, long long* sh_oc, Cand* sh_cd) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  oc = warp_max_ll(oc);
  cd = warp_best(cd);
  if (lane == 0) { sh_oc[wib] = oc; sh_cd[wib] = cd; }
  __syncthreads();
  if (wib == 0) {
    oc = lane < NT / 32 ? sh_oc[lane] : 0;
    cd = lane < NT / 32 ? sh_cd[lane] : Cand{-1, 0, 0};
    oc = warp_max_ll(oc);
    cd = warp_best(cd);
  }
}


// Adds an arc weight to a connection sum held in 64 bits.  When every sum of
// the level stays below 2^32 the add is a 32-bit atomic on the low word (the
// high word stays zero): on sm_103a a 64-bit shared-memory atomic add costs
// 6.7x a 32-bit one on distinct addresses and about 90x (16 addresses) to
// 800x (2 addresses) under the contention of a high-degree row that meets
// few labels (measured, 512 threads).
__device__ __forceinline__ void conn_add(unsigned long long* p, int32_t w, int32_t narrow) {
  if (narrow) atomicAdd(reinterpret_cast<unsigned int*>(p), (unsigned int)w);
  else atomicAdd(p, (unsigned long long)w);
}

// Degrees 17..128 (and nodes of overloaded blocks up to that degree): one
// warp per node, eight warps per CTA, each with a private WCAP-slot table in
// shared memory, so no CTA barrier is needed between nodes.  The row (at most
// four arcs per lane) is loaded up front and its labels gathered together;
// every arc is then added to its label's slot by shared-memory atomics (no
// warp-level pre-merge: reductions over per-label lane masks serialise per
// distinct label).  The lane that created a key evaluates it and later
// clears its slot, so the work per node follows the degree, not the table
// size.
constexpr int WARP_MAXDEG = B4_MAXDEG;
constexpr int WCAP = 2 * WARP_MAXDEG;        // at most half full
constexpr int WLOG = 8;                      // log2(WCAP)
constexpr int WPC = 8;                       // warps per CTA
static_assert((1 << WLOG) == WCAP, "WCAP must be 2^WLOG");

__global__ void __launch_bounds__(WPC * 32) k_propose_warp(LPArgs a, int32_t sub, int32_t b0) {
  griddep_wait();
  int64_t lbeg, cnt;
  sub_range(a, sub, b0, 5, &lbeg, &cnt);    // buckets b0..4 are adjacent
  if (cnt == 0) return;
  __shared__ unsigned long long sh_vals[WPC][WCAP];
  __shared__ int32_t sh_keys[WPC][WCAP];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  unsigned long long* vals = sh_vals[wib];
  int32_t* keys = sh_keys[wib];
  for (int j = lane; j < WCAP; j += 32) { keys[j] = -1; vals[j] = 0; }
  __syncwarp();
  const int64_t nwarps = (int64_t)gridDim.x * WPC;
  for (int64_t li = (int64_t)blockIdx.x * WPC + wib; li < cnt; li += nwarps) {
    const int64_t i = lbeg + li;
    const NodeCtx c = load_node(a, i);
    const bool ov = a.mode != MODE_CLUSTER && a.W[c.own] > c.bound;
    const int32_t nl = a.mode != MODE_CLUSTER ? a.nlab[c.slot] : 0;
    const bool direct = a.mode != MODE_CLUSTER && nl <= WCAP;
    const int deg = (int)(c.re - c.rs);
    int32_t C[4], w[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const bool in = t * 32 + lane < deg;
      const int64_t e = c.rs + t * 32 + lane;
      w[t] = in ? wat(a.ew, e) : 0;
      C[t] = in ? a.col[e] : -1;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (C[t] >= 0) C[t] = SCLAP_LD(a.label, C[t], a.N, a.err);
    // keys: local block id (direct) or label (hashed)
    int slot[4] = {0, 0, 0, 0};
    unsigned created = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (t * 32 >= deg) break;
      const int32_t key = C[t] < 0 ? -1 : (direct ? (int32_t)(C[t] - c.loff) : C[t]);
      if (key < 0) continue;
      if (direct) {
        conn_add(&vals[key], w[t], a.narrow);
      } else {
        uint32_t s = table_slot(key, WLOG);
        const uint32_t pmax = a.probe_limit < (uint32_t)WCAP ? a.probe_limit : (uint32_t)WCAP;
        bool placed = false;
        for (uint32_t p = 0; p < pmax; ++p) {
          const int32_t prev = atomicCAS(&keys[s], -1, key);
          if (prev == -1 || prev == key) {
            if (prev == -1) { created |= 1u << t; slot[t] = (int)s; }
            conn_add(&vals[s], w[t], a.narrow);
            placed = true;
            break;
          }
          s = (s + 1) & (WCAP - 1);
        }
        if (!placed) atomicOr(a.err, DERR_HASH_FULL);
      }
    }
    __syncwarp();
    long long oc = 0;
    bool has_oc = false;
    Cand cd{-1, 0, 0};
    if (direct) {
      const int32_t own_l = (int32_t)(c.own - c.loff);
      for (int32_t b = lane; b < nl; b += 32) {
        const int64_t conn = (int64_t)vals[b];
        if (b == own_l) { oc = conn; has_oc = true; continue; }
        if (conn == 0 && !ov) continue;
        const int32_t Cb = (int32_t)(c.loff + b);
        if ((int64_t)a.W[Cb] + c.cv > c.bound) continue;
        const Cand x = make_cand(c, Cb, conn);
        if (cd.conn < 0 || cand_better(x, cd)) cd = x;
      }
      __syncwarp();
      for (int32_t b = lane; b < nl; b += 32) vals[b] = 0;
    } else {
      int32_t Wk[4], Bk[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const bool q = ((created >> t) & 1u) && C[t] != c.own && !ov;
        Wk[t] = q ? SCLAP_LD(a.W, C[t], a.nlabels, a.err) : 0;
        Bk[t] = cand_block(a, c, q, C[t]);
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (!((created >> t) & 1u)) continue;
        const int64_t conn = (int64_t)vals[slot[t]];
        if (C[t] == c.own) { oc = conn; has_oc = true; continue; }
        if (ov || (int64_t)Wk[t] + c.cv > c.bound || Bk[t] != c.vb) continue;
        const Cand x = make_cand(c, C[t], conn);
        if (cd.conn < 0 || cand_better(x, cd)) cd = x;
      }
      if (ov) {
        // an overloaded node may move to any block that fits, connected or not
        for (int32_t b = lane; b < nl; b += 32) {
          const int32_t Cb = (int32_t)(c.loff + b);
          if (Cb == c.own || (int64_t)a.W[Cb] + c.cv > c.bound) continue;
          const Cand x = make_cand(c, Cb, table_get(keys, vals, WLOG, Cb));
          if (cd.conn < 0 || cand_better(x, cd)) cd = x;
        }
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if ((created >> t) & 1u) { keys[slot[t]] = -1; vals[slot[t]] = 0; }
    }
    const unsigned om = __ballot_sync(0xffffffffu, has_oc);
    oc = om ? __shfl_sync(0xffffffffu, oc, __ffs(om) - 1) : 0;
    cd = warp_best(cd);
    if (lane == 0) write_prop(a, i, c, cd, oc, ov);
    __syncwarp();
  }
}

// ---------------------------------------------------------------- bulk copies
// Hub rows are staged in shared memory by the bulk-copy engine: one thread
// issues a cp.async.bulk of a chunk of the row (col, and the weights when
// the level has them) completing on an mbarrier with the byte count, and
// every thread waits on the barrier's phase (bounded) before reading the
// chunk.  Source addresses and sizes are multiples of 16 bytes: the chunk
// is widened to 16-byte boundaries, and entries past the last full 16-byte
// word of the array are read from global memory directly.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
  return ok != 0;
}
// Waits until phase `parity` of the barrier completes, at most `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t it = 0; it <= limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

constexpr int HUB_NT = 512;
constexpr int HUB_CH = 4 * HUB_NT;           // arcs per staged chunk
constexpr int HUB_BUF = HUB_CH + 8;          // entries per buffer (16-byte widening)
constexpr size_t hub_smem_bytes() { return (size_t)2 * 2 * HUB_BUF * sizeof(int32_t); }

// The 16-byte-aligned window [a0, a1) of the chunk [e0, end) that is copied
// (a1 <= M rounded down to 16 bytes; entries at or past a1 are read from
// global memory), and the bulk copies of it into buffer b.
__device__ __forceinline__ void hub_window(int64_t e0, int64_t end, int64_t M, int64_t* a0,
                                           int64_t* a1) {
  *a0 = e0 & ~(int64_t)3;
  int64_t x = (end + 3) & ~(int64_t)3;
  const int64_t mlim = M & ~(int64_t)3;
  *a1 = x < mlim ? x : mlim;
  if (*a1 < *a0) *a1 = *a0;
}
__device__ __forceinline__ void hub_issue(const LPArgs& a, int64_t e0, int64_t end, int32_t* scol,
                                          int32_t* sew, uint64_t* bar) {
  int64_t a0, a1;
  hub_window(e0, end, a.M, &a0, &a1);
  const uint32_t bytes = (uint32_t)((a1 - a0) * 4);
  mbar_expect_tx(bar, a.ew ? 2 * bytes : bytes);
  if (bytes) {
    bulk_g2s(scol, a.col + a0, bytes, bar);
    if (a.ew) bulk_g2s(sew, a.ew + a0, bytes, bar);
  }
}

template <int SLOTS>
constexpr size_t blk_smem_bytes() {
  return (size_t)SLOTS * (sizeof(unsigned long long) + sizeof(int32_t)) +
         (size_t)(SLOTS / 2) * sizeof(int32_t);
}

// Degrees 129..8192 (buckets 5-7): one CTA of NT threads per node, a
// SLOTS-slot table in dynamic shared memory (keys, sums) plus a list of the
// slots created for the current node.  The row is read four strides at a
// time (loads first, then label gathers, then inserts), candidates are the
// created slots only, and only those slots are cleared afterwards.
template <int NT, int SLOTS>
__global__ void __launch_bounds__(NT) k_propose_blk(LPArgs a, int32_t sub, int32_t bucket) {
  griddep_wait();
  int64_t lbeg, cnt;
  sub_range(a, sub, bucket, bucket + 1, &lbeg, &cnt);
  if (cnt == 0) return;
  extern __shared__ unsigned long long smem_u64[];
  __shared__ long long sh_oc[NT / 32];
  __shared__ Cand sh_cd[NT / 32];
  __shared__ int sh_nc;
  unsigned long long* vals = smem_u64;
  int32_t* keys = reinterpret_cast<int32_t*>(smem_u64 + SLOTS);
  int32_t* clist = keys + SLOTS;
  constexpr int64_t tcap = SLOTS;
  const int tid = threadIdx.x, lane = tid & 31;
  for (int j = tid; j < SLOTS; j += NT) { keys[j] = -1; vals[j] = 0; }
  if (tid == 0) sh_nc = 0;
  __syncthreads();
  for (int64_t li = blockIdx.x; li < cnt; li += gridDim.x) {
    const int64_t i = lbeg + li;
    const NodeCtx c = load_node(a, i);
    const bool ov = a.mode != MODE_CLUSTER && a.W[c.own] > c.bound;
    const int32_t nl = a.mode != MODE_CLUSTER ? a.nlab[c.slot] : 0;
    const bool direct = a.mode != MODE_CLUSTER && nl <= tcap;
    const int64_t deg = c.re - c.rs;
    const int logcap = ceil_log2(max64(2 * deg, 32));
    const uint32_t mask = (1u << logcap) - 1;
    if (!direct && ((int64_t)1 << logcap) > tcap) {
      // a launch with a smaller table than this node's hashing needs (the
      // host only does this when every node indexes its block directly)
      if (tid == 0) {
        atomicOr(a.err, DERR_INTERNAL);
        a.prop_t[i] = -1;
      }
      continue;
    }
    for (int64_t e0 = c.rs; e0 < c.re; e0 += 4 * NT) {
      int32_t C[4], w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t e = e0 + (int64_t)u * NT + tid;
        const bool in = e < c.re;
        w[u] = in ? wat(a.ew, e) : 0;
        C[u] = in ? a.col[e] : -1;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (C[u] >= 0) C[u] = SCLAP_LD(a.label, C[u], a.N, a.err);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (e0 + (int64_t)u * NT >= c.re) break;
        const int32_t key = C[u] < 0 ? -1 : (direct ? (int32_t)(C[u] - c.loff) : C[u]);
        bool cr = false;
        uint32_t s = 0;
        if (key >= 0) {
          if (direct) {
            conn_add(&vals[key], w[u], a.narrow);
          } else {
            s = table_slot(key, logcap);
            const uint32_t pmax = a.probe_limit <= mask ? a.probe_limit : mask + 1;
            bool placed = false;
            for (uint32_t p = 0; p < pmax; ++p) {
              const int32_t prev = atomicCAS(&keys[s], -1, key);
              if (prev == -1 || prev == key) {
                cr = prev == -1;
                conn_add(&vals[s], w[u], a.narrow);
                placed = true;
                break;
              }
              s = (s + 1) & mask;
            }
            if (!placed) atomicOr(a.err, DERR_HASH_FULL);
          }
        }
        // one list reservation per warp for the slots it created
        const unsigned cm = __ballot_sync(0xffffffffu, cr);
        if (cm) {
          const int first = __ffs(cm) - 1;
          int base = 0;
          if (lane == first) base = atomicAdd(&sh_nc, __popc(cm));
          base = __shfl_sync(0xffffffffu, base, first);
          if (cr) clist[base + __popc(cm & ((1u << lane) - 1))] = (int32_t)s;
        }
      }
    }
    __syncthreads();
    long long oc = 0;
    Cand cd{-1, 0, 0};
    if (direct) {
      const int32_t own_l = (int32_t)(c.own - c.loff);
      for (int32_t b = tid; b < nl; b += NT) {
        const int64_t conn = (int64_t)vals[b];
        if (b == own_l) { oc = conn; continue; }
        if (conn == 0 && !ov) continue;
        const int32_t Cb = (int32_t)(c.loff + b);
        if ((int64_t)a.W[Cb] + c.cv > c.bound) continue;
        Cand x = make_cand(c, Cb, conn);
        if (cd.conn < 0 || cand_better(x, cd)) cd = x;
      }
      __syncthreads();
      for (int32_t b = tid; b < nl; b += NT) vals[b] = 0;
    } else {
      const int nc = sh_nc;
      for (int j = tid; j < nc; j += NT) {
        const int32_t s = clist[j];
        const int32_t K = keys[s];
        const int64_t conn = (int64_t)vals[s];
        if (K == c.own) { oc = conn; continue; }
        if (ov || (int64_t)a.W[K] + c.cv > c.bound) continue;
        if (cand_block(a, c, true, K) != c.vb) continue;
        Cand x = make_cand(c, K, conn);
        if (cd.conn < 0 || cand_better(x, cd)) cd = x;
      }
      if (ov) {
        for (int32_t b = tid; b < nl; b += NT) {
          const int32_t Cb = (int32_t)(c.loff + b);
          if (Cb == c.own || (int64_t)a.W[Cb] + c.cv > c.bound) continue;
          Cand x = make_cand(c, Cb, table_get(keys, vals, logcap, Cb));
          if (cd.conn < 0 || cand_better(x, cd)) cd = x;
        }
      }
      __syncthreads();
      for (int j = tid; j < nc; j += NT) {
        const int32_t s = clist[j];
        keys[s] = -1;
        vals[s] = 0;
      }
    }
    block_reduce<NT>(oc, cd, sh_oc, sh_cd);
    if (tid == 0) {
      write_prop(a, i, c, cd, oc, ov);
      sh_nc = 0;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ hubs
// Hubs (degree above 8192) are split over the grid in two launches.
//   k_hub_accum   the row of each hub is cut into parts of HUB_PART arcs;
//                 CTAs take parts in turn and add every arc's weight into
//                 the hub's table in global memory (its own region of
//                 hub_table_slots(degree) entries; in local search with few
//                 labels, direct-indexed by label and pre-summed per part in
//                 shared memory);
//   k_hub_select  the table (or the nl label entries) is cut into chunks of
//                 HUB_SC entries; CTAs take chunks in turn, evaluate the
//                 candidates of their chunk, reset the entries they read,
//                 and leave the chunk's best; the CTA that completes a
//                 hub's last chunk (a per-hub counter, no waiting) reduces
//                 the chunks' bests and writes the hub's proposal.
// The table pool is clean (keys -1, sums 0) before the first launch and
// after every selection.  Results equal the per-node procedure's: the same
// sums, the same candidates, the same order-free best.
constexpr int64_t HUB_PART = 16384;
constexpr int HUB_SC = 8192;
constexpr int HUB_DACC = 1024;

struct HubSel {
  int64_t* hoff;      // [cnt + 1] table regions (exclusive scan of table slots)
  int64_t* hpa;       // [cnt + 1] accumulation parts
  int64_t* hpb;       // [cnt + 1] selection chunks
  int32_t* hdone;     // [cnt] chunks selected so far
  Cand* pcd;          // best candidate of each selection chunk
  long long* poc;     // the node's own connection seen by each chunk
};

__device__ __forceinline__ bool hub_direct(const LPArgs& a, int32_t nl, int64_t tcap) {
  return a.mode != MODE_CLUSTER && nl <= tcap;
}

// Offsets of colour class `sub`'s hubs (one CTA, chunks of its size with a
// running carry): hoff / hpa / hpb = exclusive prefixes of table slots,
// parts and selection chunks over the class's hub list, with the totals at
// [cnt]; the done counters are cleared.
constexpr int HO_NT = 1024;
__global__ void __launch_bounds__(HO_NT) k_hub_offsets(LPArgs a, int32_t sub, HubSel h) {
  griddep_wait();
  __shared__ int64_t sh[3][HO_NT / 32];
  __shared__ int64_t carry[3];
  int64_t lbeg, cnt;
  sub_range(a, sub, NB - 1, NB, &lbeg, &cnt);
  if (threadIdx.x < 3) carry[threadIdx.x] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int64_t* const out[3] = {h.hoff, h.hpa, h.hpb};
  for (int64_t b0 = 0; b0 < cnt; b0 += HO_NT) {
    const int64_t li = b0 + threadIdx.x;
    int64_t x[3] = {0, 0, 0};
    if (li < cnt) {
      const int64_t deg = a.rec2[lbeg + li].y;
      const int32_t slot = a.rec[lbeg + li].w;
      const int64_t tcap = hub_table_slots(deg);
      const int32_t nl = a.mode != MODE_CLUSTER ? a.nlab[slot] : 0;
      const int64_t range = hub_direct(a, nl, tcap) ? nl : tcap;
      x[0] = tcap;
      x[1] = (deg + HUB_PART - 1) / HUB_PART;
      x[2] = max64((range + HUB_SC - 1) / HUB_SC, 1);
      h.hdone[li] = 0;
    }
    int64_t incl[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      incl[k] = x[k];
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, incl[k], o);
        if (lane >= o) incl[k] += y;
      }
      if (lane == 31) sh[k][wib] = incl[k];
    }
    __syncthreads();
    if (wib == 0) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        int64_t t = sh[k][lane];
        for (int o = 1; o < 32; o <<= 1) {
          const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
          if (lane >= o) t += y;
        }
        sh[k][lane] = t;                  // inclusive over warps
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int64_t before = carry[k] + (wib ? sh[k][wib - 1] : 0);
      if (li < cnt) out[k][li] = before + incl[k] - x[k];
    }
    __syncthreads();
    if (threadIdx.x < 3) carry[threadIdx.x] += sh[threadIdx.x][HO_NT / 32 - 1];
    __syncthreads();
  }
  if (threadIdx.x < 3) out[threadIdx.x][cnt] = carry[threadIdx.x];
}

// Last hub position li with off[li] <= q (off nondecreasing, off[0] = 0).
__device__ __forceinline__ int64_t hub_owner(const int64_t* off, int64_t cnt, int64_t q) {
  int64_t lo = 0, hi = cnt - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= q) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

constexpr size_t hub_accum_smem() {
  return hub_smem_bytes() + (size_t)HUB_DACC * sizeof(unsigned long long);
}

__global__ void __launch_bounds__(HUB_NT) k_hub_accum(LPArgs a, int32_t sub, int32_t* gkeys,
                                                      unsigned long long* gvals, HubSel h) {
  griddep_wait();
  int64_t lbeg, cnt;
  sub_range(a, sub, NB - 1, NB, &lbeg, &cnt);
  if (cnt == 0) return;
  extern __shared__ unsigned long long smem_u64[];
  __shared__ uint64_t hub_bar[2];
  const int tid = threadIdx.x;
  // rows staged chunk by chunk in two shared-memory buffers by bulk copies
  // (when col and the weights start on 16-byte boundaries); the next chunk
  // is copied while the CTA works on the current one
  int32_t* sb = reinterpret_cast<int32_t*>(smem_u64);
  int32_t* scol[2] = {sb, sb + HUB_BUF};
  int32_t* sew[2] = {sb + 2 * HUB_BUF, sb + 3 * HUB_BUF};
  unsigned long long* sacc = smem_u64 + (2 * 2 * HUB_BUF) / 2;   // after the staging buffers
  const bool staged =
      ((reinterpret_cast<uintptr_t>(a.col) | reinterpret_cast<uintptr_t>(a.ew)) & 15) == 0;
  uint32_t kchunk = 0, phs[2] = {0, 0};
  if (tid == 0) {
    mbar_init(&hub_bar[0], 1);
    mbar_init(&hub_bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int j = tid; j < HUB_DACC; j += HUB_NT) sacc[j] = 0;
  __syncthreads();
  const int64_t total = h.hpa[cnt];
  for (int64_t q = blockIdx.x; q < total; q += gridDim.x) {
    const int64_t li = hub_owner(h.hpa, cnt, q);
    const NodeCtx c = load_node(a, lbeg + li);
    const int64_t p0 = c.rs + (q - h.hpa[li]) * HUB_PART;
    const int64_t p1 = min64(p0 + HUB_PART, c.re);
    const int64_t deg = c.re - c.rs;
    const int64_t tcap = hub_table_slots(deg);
    int32_t* keys = gkeys + h.hoff[li];
    unsigned long long* vals = gvals + h.hoff[li];
    const int32_t nl = a.mode != MODE_CLUSTER ? a.nlab[c.slot] : 0;
    const bool direct = hub_direct(a, nl, tcap);
    const bool pre = direct && nl <= HUB_DACC;
    const int logcap = ceil_log2(tcap);
    const uint32_t mask = (1u << logcap) - 1;
    if (staged && tid == 0) {
      // the buffer was last read two chunks ago, before a CTA barrier
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      hub_issue(a, p0, min64(p0 + HUB_CH, p1), scol[kchunk & 1], sew[kchunk & 1],
                &hub_bar[kchunk & 1]);
    }
    for (int64_t e0 = p0; e0 < p1; e0 += HUB_CH) {
      int32_t C[4], w[4];
      if (staged) {
        const int b = (int)(kchunk & 1);
        const int64_t nx = e0 + HUB_CH;
        if (tid == 0 && nx < p1) {
          // buffer b ^ 1 was last read before the barrier that ended the
          // previous chunk; order those reads before the copy's writes
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          hub_issue(a, nx, min64(nx + HUB_CH, p1), scol[b ^ 1], sew[b ^ 1], &hub_bar[b ^ 1]);
        }
        const bool ok = mbar_wait(&hub_bar[b], phs[b], a.wait_limit);
        if (__syncthreads_or(!ok)) {
          // the copy did not complete in time: report, let the copies in
          // flight land (bounded), leave
          if (tid == 0) atomicOr(a.err, DERR_TIMEOUT);
          mbar_wait(&hub_bar[b], phs[b], a.wait_limit);
          if (nx < p1) mbar_wait(&hub_bar[b ^ 1], phs[b ^ 1], a.wait_limit);
          return;
        }
        phs[b] ^= 1u;
        int64_t w0, w1;
        hub_window(e0, min64(e0 + HUB_CH, p1), a.M, &w0, &w1);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t e = e0 + (int64_t)u * HUB_NT + tid;
          C[u] = -1;
          w[u] = 0;
          if (e < p1) {
            if (e < w1) {
              C[u] = scol[b][e - w0];
              w[u] = a.ew ? sew[b][e - w0] : 1;
            } else {
              C[u] = a.col[e];
              w[u] = wat(a.ew, e);
            }
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t e = e0 + (int64_t)u * HUB_NT + tid;
          const bool in = e < p1;
          w[u] = in ? wat(a.ew, e) : 0;
          C[u] = in ? a.col[e] : -1;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (C[u] >= 0) C[u] = SCLAP_LD(a.label, C[u], a.N, a.err);
      if (direct) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (C[u] < 0) continue;
          const int32_t key = (int32_t)(C[u] - c.loff);
          if (SCLAP_OK(key, pre ? (int64_t)HUB_DACC : tcap, a.err))
            conn_add(pre ? &sacc[key] : &vals[key], w[u], a.narrow);
        }
      } else {
        // the four arcs' first probes are independent: issue them together
        const uint32_t pmax = a.probe_limit <= mask ? a.probe_limit : mask + 1;
        uint32_t sl[4];
        int32_t prev[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          sl[u] = C[u] >= 0 ? table_slot(C[u], logcap) : 0;
          prev[u] = C[u] >= 0 && pmax > 0 ? atomicCAS(&keys[sl[u]], -1, C[u]) : -2;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (C[u] < 0) continue;
          const int32_t key = C[u];
          uint32_t s = sl[u];
          bool placed = prev[u] == -1 || prev[u] == key;
          for (uint32_t p = 1; !placed && p < pmax; ++p) {
            s = (s + 1) & mask;
            const int32_t pv = atomicCAS(&keys[s], -1, key);
            placed = pv == -1 || pv == key;
          }
          if (placed) conn_add(&vals[s], w[u], a.narrow);
          else atomicOr(a.err, DERR_HASH_FULL);
        }
      }
      if (staged) {          // every thread is done with this chunk's buffer
        ++kchunk;
        __syncthreads();
      }
    }
    if (pre) {
      // the part's per-label sums into the hub's entries (a part's sum of a
      // label is at most its row's, so the narrow rule still holds)
      __syncthreads();
      for (int32_t b = tid; b < nl; b += HUB_NT) {
        const unsigned long long x = sacc[b];
        if (!x) continue;
        sacc[b] = 0;
        if (a.narrow) atomicAdd(reinterpret_cast<unsigned int*>(&vals[b]), (unsigned int)x);
        else atomicAdd(&vals[b], x);
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ Cand ld_cand_cg(const Cand* p) {
  Cand c;
  c.conn = __ldcg(&p->conn);
  c.h = __ldcg(reinterpret_cast<const unsigned long long*>(&p->h));
  c.C = __ldcg(&p->C);
  return c;
}

__global__ void __launch_bounds__(HUB_NT) k_hub_select(LPArgs a, int32_t sub, int32_t* gkeys,
                                                       unsigned long long* gvals, HubSel h) {
  griddep_wait();
  int64_t lbeg, cnt;
  sub_range(a, sub, NB - 1, NB, &lbeg, &cnt);
  if (cnt == 0) return;
  __shared__ long long sh_oc[HUB_NT / 32];
  __shared__ Cand sh_cd[HUB_NT / 32];
  __shared__ int sh_last;
  const int tid = threadIdx.x;
  const int64_t total = h.hpb[cnt];
  for (int64_t q = blockIdx.x; q < total; q += gridDim.x) {
    const int64_t li = hub_owner(h.hpb, cnt, q);
    const int64_t i = lbeg + li;
    const NodeCtx c = load_node(a, i);
    const int64_t q0 = h.hpb[li], nchunks = h.hpb[li + 1] - q0;
    const int64_t tcap = hub_table_slots(c.re - c.rs);
    int32_t* keys = gkeys + h.hoff[li];
    unsigned long long* vals = gvals + h.hoff[li];
    const int32_t nl = a.mode != MODE_CLUSTER ? a.nlab[c.slot] : 0;
    const bool direct = hub_direct(a, nl, tcap);
    const bool ov = a.mode != MODE_CLUSTER && a.W[c.own] > c.bound;
    long long oc = 0;
    Cand cd{-1, 0, 0};
    const int64_t j0 = (q - q0) * HUB_SC;
    if (direct) {
      const int32_t own_l = (int32_t)(c.own - c.loff);
      const int64_t j1 = min64(j0 + HUB_SC, (int64_t)nl);
      for (int64_t b = j0 + tid; b < j1; b += HUB_NT) {
        const int64_t conn = (int64_t)vals[b];
        if (conn) vals[b] = 0;
        if (b == own_l) { oc = conn; continue; }
        if (conn == 0 && !ov) continue;
        const int32_t Cb = (int32_t)(c.loff + b);
        if ((int64_t)a.W[Cb] + c.cv > c.bound) continue;
        Cand x = make_cand(c, Cb, conn);
        if (cd.conn < 0 || cand_better(x, cd)) cd = x;
      }
    } else if (!ov) {
      // four entries per thread at a time: their loads, then their label
      // weight gathers, are in flight together
      const int64_t j1 = min64(j0 + HUB_SC, tcap);
      for (int64_t s0 = j0; s0 < j1; s0 += 4 * HUB_NT) {
        int32_t K[4];
        int64_t conn[4];
        wgt_t WK[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t sx = s0 + (int64_t)u * HUB_NT + tid;
          K[u] = sx < j1 ? keys[sx] : -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t sx = s0 + (int64_t)u * HUB_NT + tid;
          conn[u] = K[u] >= 0 ? (int64_t)vals[sx] : 0;
          WK[u] = K[u] >= 0 && K[u] != c.own ? SCLAP_LD(a.W, K[u], a.nlabels, a.err) : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (K[u] < 0) continue;
          const int64_t sx = s0 + (int64_t)u * HUB_NT + tid;
          keys[sx] = -1;
          vals[sx] = 0;
          if (K[u] == c.own) { oc = conn[u]; continue; }
          if ((int64_t)WK[u] + c.cv > c.bound) continue;
          if (cand_block(a, c, true, K[u]) != c.vb) continue;
          Cand x = make_cand(c, K[u], conn[u]);
          if (cd.conn < 0 || cand_better(x, cd)) cd = x;
        }
      }
    }
    block_reduce<HUB_NT>(oc, cd, sh_oc, sh_cd);
    if (tid == 0) {
      h.pcd[q] = cd;
      h.poc[q] = oc;
      __threadfence();
      sh_last = atomicAdd(&h.hdone[li], 1) == (int32_t)(nchunks - 1);
    }
    __syncthreads();
    if (sh_last) {
      __threadfence();
      oc = 0;
      cd = Cand{-1, 0, 0};
      if (!direct && ov) {
        // an overloaded node whose labels outnumber its table (local search
        // with more blocks than table entries): every label is a candidate,
        // its connection looked up; the chunks left the table to this CTA
        const int logcap = ceil_log2(tcap);
        oc = table_get(keys, vals, logcap, c.own);
        for (int32_t b = tid; b < nl; b += HUB_NT) {
          const int32_t Cb = (int32_t)(c.loff + b);
          if (Cb == c.own || (int64_t)a.W[Cb] + c.cv > c.bound) continue;
          Cand x = make_cand(c, Cb, table_get(keys, vals, logcap, Cb));
          if (cd.conn < 0 || cand_better(x, cd)) cd = x;
        }
        __syncthreads();
        for (int64_t s = tid; s < tcap; s += HUB_NT) {
          keys[s] = -1;
          vals[s] = 0;
        }
      } else {
        for (int64_t k = tid; k < nchunks; k += HUB_NT) {
          const long long o = __ldcg(&h.poc[q0 + k]);
          if (o > oc) oc = o;
          const Cand x = ld_cand_cg(&h.pcd[q0 + k]);
          if (x.conn >= 0 && (cd.conn < 0 || cand_better(x, cd))) cd = x;
        }
      }
      __syncthreads();                   // sh_oc / sh_cd reused
      block_reduce<HUB_NT>(oc, cd, sh_oc, sh_cd);
      if (tid == 0) {
        write_prop(a, i, c, cd, oc, ov);
        h.hdone[li] = 0;
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------- admission
// Admission and application of one colour class run as ONE cooperative
// launch (k_admit below), its phases separated by bounded grid barriers:
//   resolve   every proposal into a target whose proposals all fit is
//             admitted; the others are counted per target, and the first
//             proposal into an overflowing target registers the target as a
//             segment (with its admission threshold);
//   alloc     each segment takes its range of the entry arrays;
//   scatter   the overflowing proposals are written into their segments;
//   select    each segment admits its longest fitting prefix;
//   (source side, local search with overloaded blocks: forced moves out of
//   an overloaded block are grouped by source the same way)
//   apply     labels and label weights are updated.
// When no target overflows (known to every CTA after the first barrier) the
// kernel goes from resolve straight to apply: one barrier per colour class.
//
// Segment counters: ctr[set * 4 + side * 2 + {0: entry cursor, 1: segments}],
// set = colour class & 1; a launch clears the other set for the next class
// (k_round_begin clears both at the start of a round).
__device__ __forceinline__ int64_t* adm_ctr(const LPArgs& a, int sub, int side) {
  return a.ctr + (sub & 1) * 4 + side * 2;
}

__device__ void adm_resolve(const LPArgs& a, int64_t lbeg, int64_t cnt, int64_t* ct) {
  for (int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; li < cnt;
       li += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = lbeg + li;
    const int32_t t = a.prop_t[i];
    a.stage[i] = 0;
    if (t < 0) { a.adm[i] = 0; continue; }
    const int64_t bound = a.bound[a.rec[i].w];
    const int64_t Wt = SCLAP_LD(a.W, t, a.nlabels, a.err);
    if (Wt + SCLAP_LD(a.in_w, t, a.nlabels, a.err) <= bound) {
      a.adm[i] = 1;
    } else {
      a.adm[i] = 0;
      a.grp[i] = t;
      const int c = atomicAdd(&a.ovf_cnt[t], 1);
      a.stage[i] = c == 0 ? 2 : 1;
      if (c == 0) {                     // admit while the inclusive prefix <= bound - W[t]
        const int64_t seg = (int64_t)atomicAdd(ull(&ct[1]), 1ull);
        a.seg_g[seg] = t;
        a.seg_thr[seg] = bound - Wt;
      }
    }
  }
}

// Forced moves out of overloaded blocks (local search), grouped by source;
// admit while the exclusive prefix <= W[src] - bound - 1.
__device__ void adm_forced(const LPArgs& a, int64_t lbeg, int64_t cnt, int64_t* ct) {
  for (int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; li < cnt;
       li += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = lbeg + li;
    a.stage[i] = 0;
    if (a.adm[i] != 1) continue;
    const int4 r = a.rec[i];
    const int32_t own = r.y;
    const int64_t bound = a.bound[r.w];
    const int64_t Wo = SCLAP_LD(a.W, own, a.nlabels, a.err);
    if (Wo > bound) {
      a.grp[i] = own;
      const int c = atomicAdd(&a.ovf_cnt[own], 1);
      a.stage[i] = c == 0 ? 2 : 1;
      if (c == 0) {
        const int64_t seg = (int64_t)atomicAdd(ull(&ct[1]), 1ull);
        a.seg_g[seg] = own;
        a.seg_thr[seg] = Wo - bound - 1;
      }
    }
  }
}

// Each segment takes the range of its entries (order of segments is free).
__device__ void adm_alloc(const LPArgs& a, int64_t nseg, int64_t* ct) {
  for (int64_t sg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; sg < nseg;
       sg += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = a.seg_g[sg];
    const int32_t n = a.ovf_cnt[g];
    const int64_t base = (int64_t)atomicAdd(ull(&ct[0]), (unsigned long long)n);
    a.ovf_base[g] = base;
    a.seg_base[sg] = base;
    a.seg_cnt[sg] = n;
  }
}

__device__ void adm_scatter(const LPArgs& a, int64_t lbeg, int64_t cnt) {
  for (int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; li < cnt;
       li += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = lbeg + li;
    if (a.stage[i] == 0) continue;
    const int32_t g = a.grp[i];
    const int64_t pos = a.ovf_base[g] + atomicAdd(&a.ovf_fill[g], 1);
    const int4 r = a.rec[i];
    a.ent_key[pos] = a.prop_key[i];
    a.ent_v[pos] = r.x;
    a.ent_w[pos] = r.z;
    a.ent_i[pos] = (int32_t)(i);
  }
}

constexpr int SEL_NT = 256;
constexpr int SEL_SMALL = 64;     // all-pairs ranking up to this many entries

__device__ __forceinline__ bool key_less(uint64_t k1, int32_t v1, uint64_t k2, int32_t v2) {
  return k1 < k2 || (k1 == k2 && v1 < v2);
}
__device__ __forceinline__ uint32_t digit_of(uint64_t k, int32_t v, int p) {
  return p < 8 ? (uint32_t)(k >> (56 - 8 * p)) & 0xffu
               : ((uint32_t)v >> (24 - 8 * (p - 8))) & 0xffu;
}

// Admission inside one overflowing group: entries ordered by (key, node);
// target side admits while the inclusive prefix weight <= thr, source side
// while the exclusive prefix weight <= thr.  Groups of <= 64 entries rank
// all pairs in shared memory.  Larger ones locate the boundary entry (the
// first whose inclusive prefix exceeds thr) by an MSD radix select over the
// 96-bit (key, node) order: the bytes shared by the smallest and largest
// entry are skipped, each pass histograms the weights of the entries still
// matching the chosen prefix, and once <= 64 candidates remain they are
// ranked in shared memory.
__device__ __forceinline__ void select_rank_small(const LPArgs& a, int n, int64_t thr,
                                                  int64_t acc, uint64_t* sk, int32_t* sv,
                                                  int32_t* sw, int32_t* si, bool write_adm,
                                                  int32_t source, uint64_t* bk, int32_t* bv,
                                                  int* bfound) {
  // excl/incl prefix of every staged entry; write admissions directly, or
  // report the boundary entry (smallest with acc + incl > thr).
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    int64_t excl = acc;
    const uint64_t kj = sk[j];
    const int32_t vj = sv[j];
    for (int l = 0; l < n; ++l)
      if (key_less(sk[l], sv[l], kj, vj)) excl += sw[l];
    if (write_adm) {
      const bool ok = source ? (excl <= thr) : (excl + sw[j] <= thr);
      a.adm[si[j]] = ok ? 1 : 0;
    } else if (excl + sw[j] > thr && excl <= thr) {
      *bk = kj;      // the unique entry whose inclusive prefix first exceeds thr
      *bv = vj;
      *bfound = 1;
    }
  }
}

__device__ void adm_select(const LPArgs& a, int64_t nseg, int32_t source) {
  __shared__ uint64_t sk[SEL_SMALL];
  __shared__ int32_t sv[SEL_SMALL];
  __shared__ int32_t sw[SEL_SMALL];
  __shared__ int32_t si[SEL_SMALL];
  __shared__ unsigned long long hist[256];
  __shared__ unsigned int hcnt[256];
  __shared__ uint64_t PK, kmin_sh, kmax_sh, BK;
  __shared__ uint32_t PV;
  __shared__ int32_t vmin_sh, vmax_sh, BV;
  __shared__ long long acc_sh;
  __shared__ int found_sh, ncand_sh, bfound_sh, done_sh, x_sh, ncomp_sh;
  const int tid = threadIdx.x, lane = tid & 31;
  // Phase 1: groups of <= 64 entries, one warp each (entries lane and
  // lane + 32 in registers, every pair ranked through shuffles).
  {
    const int64_t nw = (int64_t)gridDim.x * (SEL_NT / 32);
    for (int64_t sg = (int64_t)blockIdx.x * (SEL_NT / 32) + (tid >> 5); sg < nseg; sg += nw) {
      const int32_t n = a.seg_cnt[sg];
      if (n > SEL_SMALL) continue;
      const int64_t base = a.seg_base[sg];
      const int64_t thr = a.seg_thr[sg];
      const bool h0 = lane < n, h1 = lane + 32 < n;
      const uint64_t k0 = h0 ? a.ent_key[base + lane] : ~0ull;
      const int32_t v0 = h0 ? a.ent_v[base + lane] : INT32_MAX;
      const int32_t w0 = h0 ? a.ent_w[base + lane] : 0;
      const uint64_t k1 = h1 ? a.ent_key[base + lane + 32] : ~0ull;
      const int32_t v1 = h1 ? a.ent_v[base + lane + 32] : INT32_MAX;
      const int32_t w1 = h1 ? a.ent_w[base + lane + 32] : 0;
      int64_t e0 = 0, e1 = 0;
      const int n0 = n < 32 ? n : 32;
      for (int l = 0; l < n0; ++l) {
        const uint64_t kl = __shfl_sync(0xffffffffu, k0, l);
        const int32_t vl = __shfl_sync(0xffffffffu, v0, l);
        const int32_t wl = __shfl_sync(0xffffffffu, w0, l);
        e0 += key_less(kl, vl, k0, v0) ? wl : 0;
        e1 += key_less(kl, vl, k1, v1) ? wl : 0;
      }
      for (int l = 32; l < n; ++l) {
        const uint64_t kl = __shfl_sync(0xffffffffu, k1, l - 32);
        const int32_t vl = __shfl_sync(0xffffffffu, v1, l - 32);
        const int32_t wl = __shfl_sync(0xffffffffu, w1, l - 32);
        e0 += key_less(kl, vl, k0, v0) ? wl : 0;
        e1 += key_less(kl, vl, k1, v1) ? wl : 0;
      }
      if (h0) a.adm[a.ent_i[base + lane]] = (source ? e0 <= thr : e0 + w0 <= thr) ? 1 : 0;
      if (h1) a.adm[a.ent_i[base + lane + 32]] = (source ? e1 <= thr : e1 + w1 <= thr) ? 1 : 0;
      if (lane == 0) {
        const int32_t g = a.seg_g[sg];
        a.ovf_cnt[g] = 0;
        a.ovf_fill[g] = 0;
      }
    }
  }
  // Phase 2: larger groups, one CTA each.
  for (int64_t sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
    const int64_t base = a.seg_base[sg];
    const int32_t n = a.seg_cnt[sg];
    const int64_t thr = a.seg_thr[sg];
    if (n <= SEL_SMALL) continue;
    {
      // smallest and largest (key, node): their shared leading bytes are skipped
      if (tid == 0) { kmin_sh = ~0ull; kmax_sh = 0; vmin_sh = INT32_MAX; vmax_sh = -1; }
      __syncthreads();
      uint64_t lmin = ~0ull, lmax = 0;
      for (int64_t j = tid; j < n; j += SEL_NT) {
        const uint64_t k = a.ent_key[base + j];
        lmin = k < lmin ? k : lmin;
        lmax = k > lmax ? k : lmax;
      }
      atomicMin(reinterpret_cast<unsigned long long*>(&kmin_sh), lmin);
      atomicMax(reinterpret_cast<unsigned long long*>(&kmax_sh), lmax);
      __syncthreads();
      const uint64_t kmin = kmin_sh, kmax = kmax_sh;
      int p0 = 0;
      while (p0 < 8 && digit_of(kmin, 0, p0) == digit_of(kmax, 0, p0)) ++p0;
      if (p0 == 8) {
        int32_t l1 = INT32_MAX, l2 = -1;
        for (int64_t j = tid; j < n; j += SEL_NT) {
          const int32_t v = a.ent_v[base + j];
          l1 = v < l1 ? v : l1;
          l2 = v > l2 ? v : l2;
        }
        atomicMin(&vmin_sh, l1);
        atomicMax(&vmax_sh, l2);
        __syncthreads();
        while (p0 < 12 && digit_of(0, vmin_sh, p0) == digit_of(0, vmax_sh, p0)) ++p0;
      }
      if (tid == 0) {
        PK = p0 >= 8 ? kmin : (p0 == 0 ? 0ull : (kmin >> (64 - 8 * p0)) << (64 - 8 * p0));
        const int pv = p0 > 8 ? p0 - 8 : 0;
        PV = pv == 0 ? 0u : (((uint32_t)vmin_sh >> (32 - 8 * pv)) << (32 - 8 * pv));
        acc_sh = 0;
        found_sh = 1;
        done_sh = 0;
        ncand_sh = 0;
        bfound_sh = 0;
      }
      __syncthreads();
      // Each pass histograms only the entries still sharing the chosen
      // prefix: after the digit is picked, the entries of its bin are
      // compacted into a scratch copy (two copies used in turn), so later
      // passes read the survivors, not the whole group.
      const uint64_t* ck = a.ent_key + base;
      const int32_t* cv = a.ent_v + base;
      const int32_t* cw = a.ent_w + base;
      int64_t cn = n;
      int buf = 0;
      int p = p0;
      for (; p < 12; ++p) {
        for (int j = tid; j < 256; j += SEL_NT) { hist[j] = 0; hcnt[j] = 0; }
        __syncthreads();
        {
          // runs of equal digits are summed in registers and added once: in
          // a large group most entries share the leading digits, and one
          // shared atomic per entry on the same bin would serialise
          uint32_t dc = 0xffffffffu;
          unsigned long long wacc = 0;
          unsigned int cacc = 0;
          for (int64_t j = tid; j < cn; j += SEL_NT) {
            const uint32_t d = digit_of(ck[j], cv[j], p);
            if (d != dc) {
              if (cacc) {
                atomicAdd(&hist[dc], wacc);
                atomicAdd(&hcnt[dc], cacc);
              }
              dc = d;
              wacc = 0;
              cacc = 0;
            }
            wacc += (unsigned long long)cw[j];
            cacc += 1;
          }
          if (cacc) {
            atomicAdd(&hist[dc], wacc);
            atomicAdd(&hcnt[dc], cacc);
          }
        }
        __syncthreads();
        if (tid < 32) {
          // first digit whose bin takes the running weight past thr: each
          // lane owns 8 consecutive bins, a warp scan gives its offset
          long long loc[8], sum = 0;
#pragma unroll
          for (int q = 0; q < 8; ++q) { loc[q] = (long long)hist[tid * 8 + q]; sum += loc[q]; }
          long long incl = sum;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o) incl += y;
          }
          long long run = acc_sh + incl - sum;
          int xq = -1;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (xq < 0) {
              if (run + loc[q] > thr) xq = q;
              else run += loc[q];
            }
          }
          const unsigned fm = __ballot_sync(0xffffffffu, xq >= 0);
          if (fm == 0) {
            if (tid == 0) found_sh = 0;   // every remaining entry fits
          } else if (tid == __ffs(fm) - 1) {
            const int x = tid * 8 + xq;
            acc_sh = run;
            if (p < 8) PK |= (uint64_t)x << (56 - 8 * p);
            else PV |= (uint32_t)x << (24 - 8 * (p - 8));
            if (hcnt[x] <= SEL_SMALL) done_sh = 1;
            x_sh = x;
            ncomp_sh = 0;
          }
        }
        __syncthreads();
        if (!found_sh) break;
        {
          const uint32_t x = (uint32_t)x_sh;
          uint64_t* dk = a.sel_key[buf] + base;
          int32_t* dv = a.sel_v[buf] + base;
          int32_t* dw = a.sel_w[buf] + base;
          for (int64_t j = tid; j < cn; j += SEL_NT) {
            const uint64_t k = ck[j];
            const int32_t v = cv[j];
            if (digit_of(k, v, p) == x) {
              const int q = atomicAdd(&ncomp_sh, 1);
              dk[q] = k;
              dv[q] = v;
              dw[q] = cw[j];
            }
          }
          __syncthreads();
          ck = dk;
          cv = dv;
          cw = dw;
          cn = ncomp_sh;
          buf ^= 1;
        }
        if (done_sh) break;
      }
      if (found_sh && done_sh && p < 11) {
        // the few survivors are the candidates sharing the chosen prefix
        for (int64_t j = tid; j < cn; j += SEL_NT) {
          sk[j] = ck[j];
          sv[j] = cv[j];
          sw[j] = cw[j];
        }
        if (tid == 0) ncand_sh = (int)cn;
        __syncthreads();
        select_rank_small(a, ncand_sh, thr, acc_sh, sk, sv, sw, si, false, source, &BK, &BV,
                          &bfound_sh);
        __syncthreads();
        if (tid == 0 && bfound_sh) { PK = BK; PV = (uint32_t)BV; }
        __syncthreads();
      }
      const int found = found_sh;
      const uint64_t pk = PK;
      const int32_t pv = (int32_t)PV;
      for (int64_t j = tid; j < n; j += SEL_NT) {
        const uint64_t k = a.ent_key[base + j];
        const int32_t v = a.ent_v[base + j];
        bool ok;
        if (!found) ok = true;
        else if (source) ok = key_less(k, v, pk, pv) || (k == pk && v == pv);
        else ok = key_less(k, v, pk, pv);
        a.adm[a.ent_i[base + j]] = ok ? 1 : 0;
      }
      __syncthreads();
    }
    if (tid == 0) {
      const int32_t g = a.seg_g[sg];
      a.ovf_cnt[g] = 0;
      a.ovf_fill[g] = 0;
    }
  }
}

// ------------------------------------------------------------- apply
// Admitted moves update labels and weights; moved nodes activate their
// neighbours (small rows by their own lane, larger rows by the whole warp).
// Label-weight changes are first summed per CTA in a small shared hash
// (label -> delta; a label that finds no slot within a few probes goes to
// global memory directly), then flushed with one atomic per label: in local
// search moves concentrate on a handful of blocks, and in clustering many
// nodes can join one cluster in a colour class (the leaves of a hub), whose
// global counters would otherwise take one atomic per moved node each.  The
// clusters that clustering moves leave are spread out and are updated
// directly.
constexpr int APPLY_SLOTS = 1024;
__device__ __forceinline__ void apply_delta(int32_t* hk, int32_t* hv, wgt_t* W, int32_t L,
                                            int32_t d, int64_t nW, int32_t* err) {
  uint32_t s = table_slot(L, 10);
#pragma unroll 1
  for (int p = 0; p < 8; ++p) {
    const int32_t prev = atomicCAS(&hk[s], -1, L);
    if (prev == -1 || prev == L) {
      atomicAdd(&hv[s], d);
      return;
    }
    s = (s + 1) & (APPLY_SLOTS - 1);
  }
  if (SCLAP_OK(L, nW, err)) atomicAdd(&W[L], (wgt_t)d);
}

constexpr int64_t MARK_CH = 4096;     // arcs per queued chunk of a moved long row

__device__ void adm_apply(const LPArgs& a, int64_t lbeg, int64_t cnt, int32_t sub) {
  uint8_t* const an = act_next(a);
  __shared__ int32_t hk[APPLY_SLOTS];
  __shared__ int32_t hv[APPLY_SLOTS];
  const bool agg_src = a.mode != MODE_CLUSTER;
  for (int j = threadIdx.x; j < APPLY_SLOTS; j += blockDim.x) { hk[j] = -1; hv[j] = 0; }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t run_slot = -1;           // moves counted in registers per slot run
  unsigned long long run_cnt = 0;
  for (int64_t b0 = w0 * 32; b0 < cnt; b0 += nw * 32) {
    const int64_t li = b0 + lane;
    int32_t slot = -1;
    int64_t rs = 0, re = 0;
    if (li < cnt) {
      const int64_t i = lbeg + li;
      const int32_t t = a.prop_t[i];
      const int8_t ad = a.adm[i];
      if (t >= 0 && SCLAP_OK(t, a.nlabels, a.err)) {
        a.in_w[t] = 0;
        if (ad) {
          const int4 r = a.rec[i];
          const int32_t v = r.x, own = r.y, cv = r.z;
          slot = r.w;
          if (an) {
            const longlong2 r2 = a.rec2[i];
            rs = r2.x;
            re = r2.x + r2.y;
          }
          if (SCLAP_OK(v, a.N, a.err)) a.label[v] = t;
          apply_delta(hk, hv, a.W, t, cv, a.nlabels, a.err);
          if (agg_src) apply_delta(hk, hv, a.W, own, -cv, a.nlabels, a.err);
          else if (SCLAP_OK(own, a.nlabels, a.err)) atomicSub(&a.W[own], (wgt_t)cv);
          if (re - rs <= 8) {
            for (int64_t e = rs; e < re; ++e)
              if (SCLAP_OK(a.col[e], a.N, a.err)) an[a.col[e]] = 1;
            re = rs;
          } else if (a.mark_big > 0 && re - rs > a.mark_big) {
            const int32_t nch = (int32_t)((re - rs + MARK_CH - 1) / MARK_CH);
            const int32_t q0 = atomicAdd(&a.mqn[sub], nch);
            for (int32_t c = 0; c < nch; ++c)
              a.mq[q0 + c] = make_longlong2(rs + c * MARK_CH, min64(rs + (c + 1) * MARK_CH, re));
            re = rs;
          }
        }
      }
    }
    unsigned big = __ballot_sync(0xffffffffu, re > rs);
    while (big) {
      const int src = __ffs(big) - 1;
      big &= big - 1;
      const int64_t s0 = __shfl_sync(0xffffffffu, (long long)rs, src);
      const int64_t s1 = __shfl_sync(0xffffffffu, (long long)re, src);
      for (int64_t e = s0 + lane; e < s1; e += 32)
        if (SCLAP_OK(a.col[e], a.N, a.err)) an[a.col[e]] = 1;
    }
    const unsigned mm = __match_any_sync(0xffffffffu, slot);
    if (slot >= 0 && lane == __ffs(mm) - 1) {
      if (slot == run_slot) {
        run_cnt += __popc(mm);
      } else {
        if (run_cnt) atomicAdd(ull(&a.moved[run_slot]), run_cnt);
        run_slot = slot;
        run_cnt = __popc(mm);
      }
    }
  }
  if (run_cnt) atomicAdd(ull(&a.moved[run_slot]), run_cnt);
  __syncthreads();
  for (int j = threadIdx.x; j < APPLY_SLOTS; j += blockDim.x)
    if (hk[j] >= 0 && hv[j] != 0 && SCLAP_OK(hk[j], a.nlabels, a.err))
      atomicAdd(&a.W[hk[j]], (wgt_t)hv[j]);
}

constexpr int ADM_NT = 256;

// The admission and application of colour class `sub` (see "admission"
// above).  source_chain: local search, forced moves out of overloaded
// blocks are possible this round.
__global__ void __launch_bounds__(ADM_NT) k_admit(LPArgs a, int32_t sub, int32_t source_chain,
                                                  GridSync* gs) {
  if (blockIdx.x == 0 && threadIdx.x < 4) a.ctr[((sub + 1) & 1) * 4 + threadIdx.x] = 0;
  // a bounded wait of an earlier launch ran out: the run is abandoned
  if (*(volatile int32_t*)a.err & DERR_TIMEOUT) return;
  int64_t lbeg, cnt;
  sub_range(a, sub, 0, NB, &lbeg, &cnt);
  const uint32_t lim = a.wait_limit;
  int64_t* ct = adm_ctr(a, sub, 0);
  adm_resolve(a, lbeg, cnt, ct);
  if (!grid_sync(gs, a.err, lim)) return;
  const int64_t nseg = *(volatile int64_t*)&ct[1];
  if (nseg > 0) {
    adm_alloc(a, nseg, ct);
    if (!grid_sync(gs, a.err, lim)) return;
    adm_scatter(a, lbeg, cnt);
    if (!grid_sync(gs, a.err, lim)) return;
    adm_select(a, nseg, 0);
    if (!grid_sync(gs, a.err, lim)) return;
  }
  if (source_chain && *(volatile int32_t*)a.flags != 0) {
    int64_t* cs = adm_ctr(a, sub, 1);
    adm_forced(a, lbeg, cnt, cs);
    if (!grid_sync(gs, a.err, lim)) return;
    const int64_t nsrc = *(volatile int64_t*)&cs[1];
    if (nsrc > 0) {
      adm_alloc(a, nsrc, cs);
      if (!grid_sync(gs, a.err, lim)) return;
      adm_scatter(a, lbeg, cnt);
      if (!grid_sync(gs, a.err, lim)) return;
      adm_select(a, nsrc, 1);
      if (!grid_sync(gs, a.err, lim)) return;
    }
  }
  adm_apply(a, lbeg, cnt, sub);
}

// The same phases as separate launches, chained on one stream with
// programmatic dependent launches (the default: on the 512-graph batch the
// chain measured faster than the cooperative kernel, whose launches also
// slowed the propose launches that follow them).  Every kernel waits for
// its predecessor first; the later phases read the segment counters on the
// device and return at once when there is nothing to do.
__global__ void __launch_bounds__(ADM_NT) k_resolve(LPArgs a, int32_t sub) {
  griddep_wait();
  if (blockIdx.x == 0 && threadIdx.x < 4) a.ctr[((sub + 1) & 1) * 4 + threadIdx.x] = 0;
  int64_t lbeg, cnt;
  sub_range(a, sub, 0, NB, &lbeg, &cnt);
  adm_resolve(a, lbeg, cnt, adm_ctr(a, sub, 0));
}
__global__ void __launch_bounds__(ADM_NT) k_forced(LPArgs a, int32_t sub) {
  griddep_wait();
  if (*(volatile int32_t*)a.flags == 0) return;   // no listed node in an overloaded block
  int64_t lbeg, cnt;
  sub_range(a, sub, 0, NB, &lbeg, &cnt);
  adm_forced(a, lbeg, cnt, adm_ctr(a, sub, 1));
}
__global__ void __launch_bounds__(ADM_NT) k_ovf_alloc(LPArgs a, int32_t sub, int32_t side) {
  griddep_wait();
  int64_t* ct = adm_ctr(a, sub, side);
  const int64_t nseg = *(volatile int64_t*)&ct[1];
  if (nseg > 0) adm_alloc(a, nseg, ct);
}
__global__ void __launch_bounds__(ADM_NT) k_ovf_scatter(LPArgs a, int32_t sub, int32_t side) {
  griddep_wait();
  if (*(volatile int64_t*)&adm_ctr(a, sub, side)[1] == 0) return;
  int64_t lbeg, cnt;
  sub_range(a, sub, 0, NB, &lbeg, &cnt);
  adm_scatter(a, lbeg, cnt);
}
__global__ void __launch_bounds__(SEL_NT) k_ovf_select(LPArgs a, int32_t sub, int32_t side) {
  griddep_wait();
  const int64_t nseg = *(volatile int64_t*)&adm_ctr(a, sub, side)[1];
  if (nseg > 0) adm_select(a, nseg, side);
}
__global__ void __launch_bounds__(ADM_NT) k_apply(LPArgs a, int32_t sub) {
  griddep_wait();
  int64_t lbeg, cnt;
  sub_range(a, sub, 0, NB, &lbeg, &cnt);
  adm_apply(a, lbeg, cnt, sub);
}

// Largest label count over the slots (local search: the largest k).
__global__ void k_max_labels(const int32_t* __restrict__ nlab, int32_t nslots, int64_t* out) {
  int32_t m = 0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nslots; i += gridDim.x * blockDim.x)
    m = max(m, nlab[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(reinterpret_cast<unsigned long long*>(out),
                                             (unsigned long long)m);
}

// The queued chunks of moved long rows of colour class `sub`: one CTA per
// chunk marks its heads active for the next round.
__global__ void __launch_bounds__(256) k_mark_rows(LPArgs a, int32_t sub) {
  griddep_wait();
  uint8_t* const an = act_next(a);
  const int32_t n = a.mqn[sub];
  for (int32_t q = blockIdx.x; q < n; q += gridDim.x) {
    const longlong2 c = a.mq[q];
    for (int64_t e = c.x + threadIdx.x; e < c.y; e += blockDim.x)
      if (SCLAP_OK(a.col[e], a.N, a.err)) an[a.col[e]] = 1;
  }
}

}  // namespace

// Limits of the bounded device-side loops, process-wide; changed only by the
// host-side fault injection of sclap_debug_inject (tests).
std::atomic<uint32_t> g_wait_limit{1u << 22};
std::atomic<uint32_t> g_probe_limit{0xffffffffu};
std::atomic<int32_t> g_fail_allocs{0};
uint32_t wait_limit() { return g_wait_limit.load(); }
uint32_t probe_limit() { return g_probe_limit.load(); }
void debug_inject(uint32_t wait, uint32_t probe, int32_t fail_allocs) {
  g_wait_limit.store(wait);
  g_probe_limit.store(probe);
  g_fail_allocs.store(fail_allocs);
}
// Counts down the allocations to the injected failure; true for the one
// that fails (the count then stays at zero).
bool take_injected_alloc_failure() {
  int32_t n = g_fail_allocs.load();
  while (n > 0) {
    if (g_fail_allocs.compare_exchange_weak(n, n - 1)) return n == 1;
  }
  return false;
}

// Launch tuning, process-wide (see sclap_tuning in sclap.h).
std::mutex g_tune_mu;
Tuning g_tune;
Tuning tuning_get() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_tune;
}
void tuning_set(const Tuning& t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune = t;
}

std::string alloc_failure_message(size_t bytes, cudaError_t e) {
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaMemPool_t pool;
  uint64_t reserved = 0, used = 0;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
  }
  cudaGetLastError();
  char buf[320];
  snprintf(buf, sizeof(buf),
           "device allocation of %.3f GB failed (%s); device free %.3f of %.3f GB, "
           "pool reserved %.3f GB, in use %.3f GB",
           bytes / 1e9, cudaGetErrorString(e), fr / 1e9, tot / 1e9, reserved / 1e9, used / 1e9);
  return buf;
}

int64_t table_pass_slots() {
  const Tuning t = tuning_get();
  if (t.contract_table_slots > 0) return t.contract_table_slots;
  return std::max<int64_t>((int64_t)1 << 20, obtainable_device_bytes() / 2 / 12);
}

int64_t obtainable_device_bytes() {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return (int64_t)1 << 32;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaMemPool_t pool;
  uint64_t reserved = 0, used = 0;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
    cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
  }
  cudaGetLastError();
  return (int64_t)fr + (int64_t)(reserved > used ? reserved - used : 0);
}

// Stream on which this thread captures graphs (non-blocking, created once).
cudaStream_t capture_stream() {
  thread_local cudaStream_t cs = nullptr;
  if (!cs) SCLAP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  return cs;
}

// Side streams for concurrent launches (non-blocking, created on first use
// and kept).  Each host thread has its own, so callers running partitions
// from several threads at once (the server's workers) do not serialise on
// one another's side streams.
cudaStream_t side_stream(int i) {
  thread_local std::vector<cudaStream_t> pool;
  while ((int)pool.size() <= i) {
    cudaStream_t st;
    SCLAP_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    pool.push_back(st);
  }
  return pool[i];
}

// Reused events without timing, for stream fork/join only.
std::mutex g_sync_ev_mu;
std::vector<cudaEvent_t> g_sync_events;
cudaEvent_t sync_event_get() {
  std::lock_guard<std::mutex> lk(g_sync_ev_mu);
  if (!g_sync_events.empty()) {
    cudaEvent_t e = g_sync_events.back();
    g_sync_events.pop_back();
    return e;
  }
  cudaEvent_t e;
  SCLAP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return e;
}
void sync_event_put(cudaEvent_t e) {
  std::lock_guard<std::mutex> lk(g_sync_ev_mu);
  g_sync_events.push_back(e);
}

// Reused CUDA events for the profiling brackets.
std::mutex g_event_mu;
std::vector<cudaEvent_t> g_events;
cudaEvent_t event_from_pool() {
  std::lock_guard<std::mutex> lk(g_event_mu);
  if (!g_events.empty()) {
    cudaEvent_t e = g_events.back();
    g_events.pop_back();
    return e;
  }
  cudaEvent_t e;
  SCLAP_CUDA(cudaEventCreate(&e));
  return e;
}
void event_to_pool(cudaEvent_t e) {
  std::lock_guard<std::mutex> lk(g_event_mu);
  g_events.push_back(e);
}

ProfileState& profile() {
  static ProfileState p;
  return p;
}

void timeline_mark(const char* name, cudaStream_t s) {
  cudaEvent_t e = event_from_pool();
  cudaEventRecord(e, s);
  ProfileState& P = profile();
  std::lock_guard<std::mutex> lk(P.mu);
  P.marks.emplace_back(name, e);
}

// Aggregates the timeline into "name count total_ms" lines (marks named
// "<call>" open a new segment and are not charged).
std::string timeline_dump() {
  ProfileState& P = profile();
  std::lock_guard<std::mutex> lk(P.mu);
  std::vector<std::string> names;
  std::vector<double> tot;
  std::vector<int64_t> cnt;
  cudaEvent_t prev = nullptr;
  for (auto& m : P.marks) {
    cudaEventSynchronize(m.second);
    if (prev && std::string(m.first) != "<call>") {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, prev, m.second);
      size_t j = 0;
      while (j < names.size() && names[j] != m.first) ++j;
      if (j == names.size()) { names.push_back(m.first); tot.push_back(0); cnt.push_back(0); }
      tot[j] += ms;
      cnt[j] += 1;
    }
    prev = m.second;
  }
  std::string out;
  char buf[256];
  for (size_t j = 0; j < names.size(); ++j) {
    snprintf(buf, sizeof(buf), "%s %lld %.6f\n", names[j].c_str(), (long long)cnt[j], tot[j]);
    out += buf;
  }
  for (auto& m : P.marks) event_to_pool(m.second);
  P.marks.clear();
  return out;
}

// ---------------------------------------------------------------------------
// Host driver of the rounds.
// ---------------------------------------------------------------------------
int64_t lp_run(const LevelView& lv, const SlotParams& sp, int32_t* label, wgt_t* W,
               int64_t Wsize, const LPRun& run, int32_t* d_err, cudaStream_t s,
               const uint8_t* active_init, uint8_t* active_next_out) {
  const int64_t N = lv.N;
  if (N == 0 || run.rounds <= 0) return 0;
  const int S = run.sub_rounds;
  const int nkeys = S * NB;
  const int sms = num_sms();

  DevBuf<int64_t> in_w((size_t)Wsize, s), ovf_base((size_t)Wsize, s);
  DevBuf<int32_t> ovf_cnt((size_t)Wsize, s), ovf_fill((size_t)Wsize, s);
  in_w.zero(); ovf_cnt.zero(); ovf_fill.zero();
  DevBuf<int4> rec(N, s);
  DevBuf<longlong2> rec2(N, s);
  DevBuf<int32_t> prop_t(N, s), grp(N, s), seg_g(N, s), seg_cnt(N, s);
  DevBuf<uint64_t> prop_key(N, s), ent_key(N, s);
  DevBuf<int8_t> adm(N, s), stage(N, s);
  DevBuf<int64_t> seg_base(N, s), seg_thr(N, s);
  DevBuf<int32_t> ent_v(N, s), ent_w(N, s), ent_i(N, s);
  DevBuf<uint64_t> sel_k0(N, s), sel_k1(N, s);
  DevBuf<int32_t> sel_v0(N, s), sel_v1(N, s), sel_w0(N, s), sel_w1(N, s);
  DevBuf<int64_t> ctr(8, s);
  ctr.zero();
  DevBuf<GridSync> gsync(1, s);
  gsync.zero();
  DevBuf<int32_t> bcnt(nkeys, s), bfill(nkeys, s);
  DevBuf<int64_t> boff(nkeys + 1, s), arcs(1, s), karcs(nkeys, s);
  DevBuf<int32_t> flags(1, s);
  DevBuf<int16_t> nkey(N, s);
  bfill.zero(); arcs.zero();

  const bool track_active = run.use_active || active_init != nullptr || active_next_out != nullptr;
  DevBuf<uint8_t> act_a, act_b;
  if (track_active) {
    act_a.alloc(N, s);
    act_b.alloc(N, s);
    if (active_init) SCLAP_CUDA(cudaMemcpyAsync(act_a.p, active_init, N, cudaMemcpyDeviceToDevice, s));
    else act_a.fill_bytes(1);
    act_b.zero();
  }

  // Global hash tables of hub nodes: a region per hub of a colour class,
  // sized to its degree (hub_table_slots), in a pool sized for the class's
  // hubs (host-driven rounds: 4 slots per arc + 32 per hub of the class, a
  // bound of the sum; CUDA-graph rounds: the sum over all hubs of the
  // level).
  int64_t pool_slots = 0;
  DevBuf<int32_t> gkeys, hub_done;
  DevBuf<unsigned long long> gvals;
  DevBuf<int64_t> hub_off;
  DevBuf<Cand> hub_pcd;
  DevBuf<long long> hub_poc;
  HubSel hs{};
  int gblocks = 0;
  // the pool starts clean (keys -1, sums 0); every selection leaves it so
  auto ensure_pool = [&](int64_t slots) {
    if (slots <= pool_slots) return;
    slots = std::max<int64_t>(slots, 1024);
    gkeys.alloc((size_t)slots, s);
    gvals.alloc((size_t)slots, s);
    gkeys.fill_bytes(0xff);
    gvals.zero();
    pool_slots = slots;
  };

  LPArgs a{};
  a.row_ptr = lv.row_ptr; a.col = lv.col; a.ew = lv.ew; a.nw = lv.nw; a.gid = lv.gid;
  a.narrow = lv.narrow ? 1 : 0;
  a.arcs32 = lv.M < ((int64_t)1 << 32) ? 1 : 0;
  a.M = lv.M;
  a.N = lv.N;
  a.nlabels = Wsize;
  a.noff = sp.noff; a.loff = sp.loff; a.bound = sp.bound; a.rkey = sp.rkey; a.nlab = sp.nlab;
  a.done = sp.done; a.moved = sp.moved; a.rounds = sp.rounds;
  a.label = label; a.W = W; a.in_w = in_w.p; a.mode = run.mode; a.S = S;
  a.rec = rec.p; a.rec2 = rec2.p; a.prop_t = prop_t.p; a.prop_key = prop_key.p; a.adm = adm.p; a.stage = stage.p;
  a.grp = grp.p; a.ovf_cnt = ovf_cnt.p; a.ovf_fill = ovf_fill.p; a.ovf_base = ovf_base.p;
  a.ctr = ctr.p; a.seg_g = seg_g.p; a.seg_base = seg_base.p; a.seg_cnt = seg_cnt.p;
  a.seg_thr = seg_thr.p; a.ent_key = ent_key.p; a.ent_v = ent_v.p; a.ent_w = ent_w.p;
  a.ent_i = ent_i.p; a.bcnt = bcnt.p;
  a.sel_key[0] = sel_k0.p; a.sel_key[1] = sel_k1.p;
  a.sel_v[0] = sel_v0.p; a.sel_v[1] = sel_v1.p;
  a.sel_w[0] = sel_w0.p; a.sel_w[1] = sel_w1.p; a.bfill = bfill.p; a.boff = boff.p; a.arcs = arcs.p;
  a.karcs = karcs.p;
  a.flags = flags.p;
  a.nkey = nkey.p;
  a.err = d_err;
  a.wait_limit = wait_limit();
  a.probe_limit = probe_limit();

  // ---- round-invariant setup ---------------------------------------------
  DevBuf<int32_t> rstate(3, s);        // round index, live slots, continue flag
  rstate.zero();
  a.rnd = rstate.p;
  a.live = rstate.p + 1;
  int32_t* const d_cont = rstate.p + 2;
  a.rounds_max = run.rounds;
  a.stop_rule = run.stop_rule ? 1 : 0;
  a.rblk = run.mode == MODE_CLUSTER ? run.rblk : nullptr;
  a.act[0] = track_active ? act_a.p : nullptr;
  a.act[1] = track_active ? act_b.p : nullptr;

  // The level's degrees decide which propose launches can ever have work
  // (and size the hub tables): one read-back per run, none per round.
  DevBuf<int64_t> dstat(4, s);
  dstat.zero();
  level_degree_stats(lv.row_ptr, N, B7_MAXDEG, dstat.p, s);
  if (run.mode != MODE_CLUSTER && sp.nslots > 0) {
    k_max_labels<<<grid_for(sp.nslots, 256, 64), 256, 0, s>>>(sp.nlab, sp.nslots, dstat.p + 3); SCLAP_NOTE_LAUNCH("k_max_labels");
  }
  int64_t hstat[4] = {0, 0, 0, 0};
  SCLAP_CUDA(cudaMemcpyAsync(hstat, dstat.p, sizeof(hstat), cudaMemcpyDeviceToHost, s));
  stream_sync(s);
  const int64_t maxdeg = hstat[0], nhubs = hstat[1], hub_slots = hstat[2];
  // local search where every slot has at most B5_SLOTS labels: every node of
  // the CTA buckets indexes its block directly, so buckets 6 and 7 need only
  // a B5_SLOTS-entry shared table (more CTAs per SM) instead of one sized
  // for hashing 2 x degree labels
  const bool compact_blk = run.mode != MODE_CLUSTER && hstat[3] > 0 && hstat[3] <= B5_SLOTS;
  const bool refine = run.mode != MODE_CLUSTER;
  const Tuning tu = tuning_get();
  const int nsb = tu.small_max_deg >= 16 ? 3 : 2;   // buckets of the thread-per-node launch
  const bool need[NB] = {true, true, true, refine || maxdeg > (nsb == 3 ? 16 : 8), false,
                         maxdeg > B4_MAXDEG, maxdeg > B5_MAXDEG, maxdeg > B6_MAXDEG,
                         maxdeg > B7_MAXDEG};
  if (need[8]) {
    gblocks = sms * 2;
    // per hub of a class: offsets of its table, parts and selection chunks
    // (three arrays), its done counter; per selection chunk (at most one per
    // HUB_SC table slots of the level's hubs, plus one per hub): its best
    hub_off.alloc((size_t)(3 * (nhubs + 1)), s);
    hub_done.alloc((size_t)nhubs, s);
    const int64_t nchunk = hub_slots / HUB_SC + nhubs + 1;
    hub_pcd.alloc((size_t)nchunk, s);
    hub_poc.alloc((size_t)nchunk, s);
    hs.hoff = hub_off.p;
    hs.hpa = hub_off.p + (nhubs + 1);
    hs.hpb = hub_off.p + 2 * (nhubs + 1);
    hs.hdone = hub_done.p;
    hs.pcd = hub_pcd.p;
    hs.poc = hub_poc.p;
    if (run.graph) ensure_pool(hub_slots);
  }
  // moved rows above 4096 arcs activate their neighbours through the chunk
  // queue (at most arcs / 4096 chunks plus one per such row, per class)
  DevBuf<longlong2> mark_q;
  DevBuf<int32_t> mark_n;
  if (track_active && maxdeg > MARK_CH) {
    mark_q.alloc((size_t)(2 * (lv.M / MARK_CH) + 2), s);
    mark_n.alloc((size_t)S, s);
    mark_n.zero();
    a.mark_big = MARK_CH;
    a.mq = mark_q.p;
    a.mqn = mark_n.p;
  }
  const unsigned grid_mark = (unsigned)(sms * 8);
  constexpr size_t smem5 = blk_smem_bytes<B5_SLOTS>();
  constexpr size_t smem6 = blk_smem_bytes<B6_SLOTS>();
  constexpr size_t smem7 = blk_smem_bytes<B7_SLOTS>();
  static std::once_flag attrs_once;
  std::call_once(attrs_once, [&] {
    SCLAP_CUDA(cudaFuncSetAttribute(k_propose_blk<256, B6_SLOTS>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem6));
    SCLAP_CUDA(cudaFuncSetAttribute(k_propose_blk<512, B7_SLOTS>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem7));
  });
  // fixed launch shapes: kernels read their node ranges on the device and
  // grid-stride over them
  const unsigned nsl_grid = grid_for(sp.nslots, 128, 1024);
  const unsigned bgrid = (unsigned)((N + BK_TILE - 1) / BK_TILE);
  const unsigned grid_small = (unsigned)(sms * tu.small_ctas_per_sm);
  const unsigned grid_warp = (unsigned)(sms * tu.warp_ctas_per_sm);
  const unsigned grid_b5 = (unsigned)(sms * 16), grid_b6 = (unsigned)(sms * 4);
  const unsigned grid_b7 = (unsigned)sms;
  const int32_t raw = run.raw_key ? 1 : 0;

  // ---- one round, as launches on s (shared by both drivers) ----------------
  // (every operation of a round goes to the stream passed in: the caller's
  // stream when driven directly, the capture stream when building the graph)
  // pdl: programmatic launches for kernels that follow a kernel of the same
  // stream (never for the first kernel after an event, a copy or a wait)
  auto head = [&](cudaStream_t s, bool pdl) {
    launch_k(false, k_round_begin, nsl_grid, 128, 0, s, a, sp.nslots, run.phase, sp.seed,
             sp.level, raw); SCLAP_NOTE_LAUNCH("k_round_begin");
    launch_k(pdl, k_bucket_count, bgrid, BK_NT, 0, s, a, N); SCLAP_NOTE_LAUNCH("k_bucket_count");
    launch_k(pdl, k_bucket_offsets, 1, 32, 0, s, a, nkeys); SCLAP_NOTE_LAUNCH("k_bucket_offsets");
    launch_k(pdl, k_bucket_scatter, bgrid, BK_NT, 0, s, a, N); SCLAP_NOTE_LAUNCH("k_bucket_scatter");
    SCLAP_LAUNCH_CHECK();
  };
  // Per-launch profiling of the direct driver (host offsets known).
  struct Timed { int family; cudaEvent_t a, b; };
  std::vector<Timed> timed;
  int64_t pn[4] = {}, pa[4] = {};
  std::vector<int64_t> hoff(nkeys + 1), hkarcs(nkeys);
  const bool prof = profile().enabled.load();
  const bool timeline = profile().timeline.load(std::memory_order_relaxed);
  // The propose launches of a colour class are independent of one another:
  // they run on side streams joined back by events, so latency-bound
  // launches overlap (serial when the timeline profiler is on).  With host
  // offsets (direct driver) empty launches are skipped and, when profiling,
  // each launch is timed and its nodes and arcs tallied by family.
  auto propose = [&](cudaStream_t s, int sub, bool fork, const int64_t* ho, bool pdl) {
    // the hub pool grows on the round's stream before the fork, so the side
    // streams see the allocation
    if (need[8] && ho) {
      const int64_t nh = ho[sub * NB + 9] - ho[sub * NB + 8];
      if (nh > 0) ensure_pool(4 * hkarcs[sub * NB + 8] + 32 * nh);
    }
    cudaEvent_t ev_fork = nullptr;
    if (fork) {
      ev_fork = sync_event_get();
      SCLAP_CUDA(cudaEventRecord(ev_fork, s));
    }
    int nside = 0;
    cudaStream_t joined[NB];
    auto lane = [&]() -> cudaStream_t {
      if (!fork) return s;
      cudaStream_t ss = side_stream(nside);
      SCLAP_CUDA(cudaStreamWaitEvent(ss, ev_fork, 0));
      joined[nside++] = ss;
      return ss;
    };
    // buckets [b0, b1) of this colour class in one launch of family fam; a
    // launch follows a kernel of its stream only when the launches are
    // serial, it is not the first, and no per-launch events are recorded
    int nlaunched = 0;
    auto launch = [&](int b0, int b1, int fam, auto&& fn) {
      if (ho && ho[sub * NB + b1] == ho[sub * NB + b0]) return;
      cudaStream_t ls = lane();
      Timed tm{fam, nullptr, nullptr};
      const bool timed_launch = prof && ho;
      if (timed_launch) {
        tm.a = event_from_pool();
        tm.b = event_from_pool();
        SCLAP_CUDA(cudaEventRecord(tm.a, ls));
        pn[fam] += ho[sub * NB + b1] - ho[sub * NB + b0];
        for (int q = b0; q < b1; ++q) pa[fam] += hkarcs[sub * NB + q];
      }
      fn(ls, pdl && !fork && !timed_launch && nlaunched > 0);
      ++nlaunched;
      if (prof && ho) {
        SCLAP_CUDA(cudaEventRecord(tm.b, ls));
        timed.push_back(tm);
      }
    };
    // grid of a launch over buckets [b0, b1): sized from the host counts
    // when known, else the fixed maximum (kernels grid-stride either way)
    auto grid = [&](int b0, int b1, int per, unsigned cap) -> unsigned {
      if (!ho) return cap;
      if (b0 == 0) {                  // one block per 256 nodes of each bucket
        int64_t nb = 0;
        for (int q = 0; q < b1; ++q) nb += (ho[sub * NB + q + 1] - ho[sub * NB + q] + 255) / 256;
        return (unsigned)std::max<int64_t>(1, std::min<int64_t>(nb, cap));
      }
      return grid_for(ho[sub * NB + b1] - ho[sub * NB + b0], per, cap);
    };
    // family 0 first: it holds most nodes, and the first launch gets the SMs
    launch(0, nsb, 0, [&](cudaStream_t ls, bool p) {
      launch_k(p, k_propose_small, grid(0, nsb, 256, grid_small), 256, 0, ls, a, sub, nsb); SCLAP_NOTE_LAUNCH("k_propose_small");
    });
    if (need[3]) launch(nsb, 5, 1, [&](cudaStream_t ls, bool p) {
      launch_k(p, k_propose_warp, grid(nsb, 5, WPC, grid_warp), WPC * 32, 0, ls, a, sub, nsb); SCLAP_NOTE_LAUNCH("k_propose_warp");
    });
    if (need[5]) launch(5, 6, 1, [&](cudaStream_t ls, bool p) {
      launch_k(p, k_propose_blk<128, B5_SLOTS>, grid(5, 6, 1, grid_b5), 128, smem5, ls, a, sub, 5); SCLAP_NOTE_LAUNCH("k_propose_blk128");
    });
    if (need[6]) launch(6, 7, 2, [&](cudaStream_t ls, bool p) {
      if (compact_blk)
        launch_k(p, k_propose_blk<256, B5_SLOTS>, grid(6, 7, 1, grid_b5), 256, smem5, ls, a, sub, 6);
      else
        launch_k(p, k_propose_blk<256, B6_SLOTS>, grid(6, 7, 1, grid_b6), 256, smem6, ls, a, sub, 6);
      SCLAP_NOTE_LAUNCH("k_propose_blk256");
    });
    if (need[7]) launch(7, 8, 2, [&](cudaStream_t ls, bool p) {
      if (compact_blk)
        launch_k(p, k_propose_blk<512, B5_SLOTS>, grid(7, 8, 1, grid_b6), 512, smem5, ls, a, sub, 7);
      else
        launch_k(p, k_propose_blk<512, B7_SLOTS>, grid(7, 8, 1, grid_b7), 512, smem7, ls, a, sub, 7);
      SCLAP_NOTE_LAUNCH("k_propose_blk512");
    });
    if (need[8]) launch(8, 9, 3, [&](cudaStream_t ls, bool p) {
      launch_k(p, k_hub_offsets, 1, HO_NT, 0, ls, a, sub, hs); SCLAP_NOTE_LAUNCH("k_hub_offsets");
      launch_k(tu.pdl != 0, k_hub_accum, (unsigned)gblocks, HUB_NT, hub_accum_smem(), ls, a, sub, gkeys.p, gvals.p, hs); SCLAP_NOTE_LAUNCH("k_hub_accum");
      launch_k(tu.pdl != 0, k_hub_select, (unsigned)gblocks, HUB_NT, 0, ls, a, sub, gkeys.p, gvals.p, hs); SCLAP_NOTE_LAUNCH("k_hub_select");
    });
    if (fork) {
      for (int j = 0; j < nside; ++j) {
        cudaEvent_t ej = sync_event_get();
        SCLAP_CUDA(cudaEventRecord(ej, joined[j]));
        SCLAP_CUDA(cudaStreamWaitEvent(s, ej, 0));
        sync_event_put(ej);
      }
      sync_event_put(ev_fork);
    }
    SCLAP_LAUNCH_CHECK();
  };
  // Admission and application of colour class `sub`: one cooperative launch
  // (k_admit).  The source-side phases (local search) are skipped by the
  // host when it knows no listed node sits in an overloaded block, else the
  // kernel checks that on the device.  The grid is sized from the host's
  // proposal count when known (fewer CTAs make the barriers cheaper), else
  // the largest co-resident grid.
  static int adm_occ = 0;
  static std::once_flag adm_once;
  std::call_once(adm_once, [&] {
    SCLAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&adm_occ, k_admit, ADM_NT, 0));
    if (adm_occ < 1) adm_occ = 1;
  });
  const unsigned grid_adm_coop =
      (unsigned)std::max(1, sms * std::min<int>(adm_occ, tu.admit_ctas_per_sm));
  const unsigned grid_adm_max = (unsigned)(sms * tu.admit_ctas_per_sm);
  const unsigned grid_sel = (unsigned)(sms * 4);
  auto admit = [&](cudaStream_t s, int sub, bool source_chain, int64_t cnt, bool pdl) {
    if (tu.fused_admission) {
      // one cooperative launch; it follows the propose join: plain launch
      const unsigned grid = cnt < 0 ? grid_adm_coop : grid_for(cnt, ADM_NT, grid_adm_coop);
      launch_coop(k_admit, grid, ADM_NT, 0, s, a, sub, source_chain ? 1 : 0, gsync.p);
      SCLAP_NOTE_LAUNCH("k_admit");
      if (a.mark_big) { launch_k(false, k_mark_rows, grid_mark, 256, 0, s, a, sub); SCLAP_NOTE_LAUNCH("k_mark_rows"); }
      SCLAP_LAUNCH_CHECK();
      return;
    }
    const unsigned grid_adm = cnt < 0 ? grid_adm_max : grid_for(cnt, ADM_NT, grid_adm_max);
    launch_k(false, k_resolve, grid_adm, ADM_NT, 0, s, a, sub); SCLAP_NOTE_LAUNCH("k_resolve");
    launch_k(pdl, k_ovf_alloc, grid_sel, ADM_NT, 0, s, a, sub, 0); SCLAP_NOTE_LAUNCH("k_ovf_alloc");
    launch_k(pdl, k_ovf_scatter, grid_adm, ADM_NT, 0, s, a, sub, 0); SCLAP_NOTE_LAUNCH("k_ovf_scatter");
    launch_k(pdl, k_ovf_select, grid_sel, SEL_NT, 0, s, a, sub, 0); SCLAP_NOTE_LAUNCH("k_ovf_select");
    if (source_chain) {
      launch_k(pdl, k_forced, grid_adm, ADM_NT, 0, s, a, sub); SCLAP_NOTE_LAUNCH("k_forced");
      launch_k(pdl, k_ovf_alloc, grid_sel, ADM_NT, 0, s, a, sub, 1); SCLAP_NOTE_LAUNCH("k_ovf_alloc");
      launch_k(pdl, k_ovf_scatter, grid_adm, ADM_NT, 0, s, a, sub, 1); SCLAP_NOTE_LAUNCH("k_ovf_scatter");
      launch_k(pdl, k_ovf_select, grid_sel, SEL_NT, 0, s, a, sub, 1); SCLAP_NOTE_LAUNCH("k_ovf_select");
    }
    launch_k(pdl, k_apply, grid_adm, ADM_NT, 0, s, a, sub); SCLAP_NOTE_LAUNCH("k_apply");
    if (a.mark_big) { launch_k(pdl, k_mark_rows, grid_mark, 256, 0, s, a, sub); SCLAP_NOTE_LAUNCH("k_mark_rows"); }
    SCLAP_LAUNCH_CHECK();
  };
  auto tail = [&](cudaStream_t s, cudaGraphConditionalHandle h, bool in_graph, bool pdl) {
    launch_k(false, k_round_end, nsl_grid, 128, 0, s, a, sp.nslots); SCLAP_NOTE_LAUNCH("k_round_end");
    launch_k(pdl, k_round_cond, 1, 1, 0, s, a, nkeys, h, in_graph ? 1 : 0, d_cont); SCLAP_NOTE_LAUNCH("k_round_cond");
    SCLAP_LAUNCH_CHECK();
  };

  // per sub-round record (direct driver, profiling): kind of run, round,
  // colour class, nodes, arcs and events at fork, join (end of the propose
  // phase) and after apply
  struct PhaseRec { int32_t ph, r, sub; int64_t nodes, arcs; cudaEvent_t a, b, c; };
  std::vector<PhaseRec> precs;

  if (run.graph && !prof && !timeline) {
    // ---- graph driver: the whole round loop is one CUDA graph, a WHILE
    // node around one round whose condition k_round_cond sets on the device
    // streams and events the capture will use are created beforehand (no
    // object creation while the stream is capturing)
    for (int j = 0; j < NB; ++j) (void)side_stream(j);
    (void)capture_stream();
    {
      cudaEvent_t warm[NB + 1];
      for (int j = 0; j <= NB; ++j) warm[j] = sync_event_get();
      for (int j = 0; j <= NB; ++j) sync_event_put(warm[j]);
    }
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    SCLAP_CUDA(cudaGraphCreate(&g, 0));
    const int64_t launches0 = profile().launches.load();
    try {
      cudaGraphConditionalHandle h;
      SCLAP_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t wnode;
      SCLAP_CUDA(cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &cp));
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      // the caller's stream may be the legacy default stream, which cannot
      // capture: the body is captured on a stream of this thread
      cudaStream_t cs = capture_stream();
      SCLAP_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
      try {
        // programmatic launches are captured as programmatic edges
        const bool pdl = tu.pdl != 0;
        head(cs, pdl);
        for (int sub = 0; sub < S; ++sub) {
          propose(cs, sub, tu.concurrent != 0, nullptr, pdl);
          admit(cs, sub, refine, -1, pdl);
        }
        tail(cs, h, true, pdl);
      } catch (...) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(cs, &junk);
        throw;
      }
      cudaGraph_t captured = nullptr;
      SCLAP_CUDA(cudaStreamEndCapture(cs, &captured));
      SCLAP_CUDA(cudaGraphInstantiate(&ex, g, 0));
      SCLAP_CUDA(cudaGraphLaunch(ex, s));
    } catch (...) {
      if (ex) cudaGraphExecDestroy(ex);
      cudaGraphDestroy(g);
      throw;
    }
    // the capture counted one round's launches; the graph ran them per round
    int32_t hr = 0;
    SCLAP_CUDA(cudaMemcpyAsync(&hr, a.rnd, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    stream_sync(s);
    cudaGraphExecDestroy(ex);
    cudaGraphDestroy(g);
    const int64_t per_round = profile().launches.load() - launches0;
    if (hr > 1) profile().launches.fetch_add(per_round * (hr - 1));
  } else {
    // ---- direct driver: one round at a time; the host reads the bucket
    // offsets after bucketing (one wait per round), skips empty launches and
    // colour classes, and stops at the first round that lists no node
    // the per-kernel timeline records an event after every launch
    const bool pdl = tu.pdl != 0 && !timeline;
    for (int r = 0; r < run.rounds; ++r) {
      head(s, pdl);
      int32_t hflags = 0;
      SCLAP_CUDA(cudaMemcpyAsync(hoff.data(), boff.p, (nkeys + 1) * sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, s));
      SCLAP_CUDA(cudaMemcpyAsync(hkarcs.data(), karcs.p, nkeys * sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, s));
      SCLAP_CUDA(cudaMemcpyAsync(&hflags, flags.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      stream_sync(s);
      if (hoff[nkeys] == 0) {
        tail(s, 0, false, pdl);
        break;
      }
      for (int sub = 0; sub < S; ++sub) {
        const int64_t cnt = hoff[(sub + 1) * NB] - hoff[sub * NB];
        if (cnt == 0) continue;
        Timed phase{-1, nullptr, nullptr};
        if (prof) {
          phase.a = event_from_pool();
          phase.b = event_from_pool();
          SCLAP_CUDA(cudaEventRecord(phase.a, s));
        }
        propose(s, sub, !timeline && tu.concurrent, hoff.data(), pdl);
        if (prof) {
          SCLAP_CUDA(cudaEventRecord(phase.b, s));
          timed.push_back(phase);
          int64_t sub_arcs = 0;
          for (int q = 0; q < NB; ++q) sub_arcs += hkarcs[sub * NB + q];
          precs.push_back(PhaseRec{run.phase, r, sub, cnt, sub_arcs, phase.a, phase.b,
                                   event_from_pool()});
        }
        admit(s, sub, refine && hflags != 0, cnt, pdl);
        if (prof) SCLAP_CUDA(cudaEventRecord(precs.back().c, s));
      }
      tail(s, 0, false, pdl);
    }
  }
  int32_t hr = 0;
  int64_t h_arcs = 0;
  SCLAP_CUDA(cudaMemcpyAsync(&hr, a.rnd, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SCLAP_CUDA(cudaMemcpyAsync(&h_arcs, arcs.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  stream_sync(s);
  if (active_next_out && track_active)
    SCLAP_CUDA(cudaMemcpyAsync(active_next_out, a.act[hr & 1], N, cudaMemcpyDeviceToDevice, s));
  if (prof) {
    ProfileState& P = profile();
    std::lock_guard<std::mutex> lk(P.mu);
    for (const Timed& t : timed) {
      float ms = 0.f;
      SCLAP_CUDA(cudaEventElapsedTime(&ms, t.a, t.b));
      if (t.family < 0) {
        P.sweep_ms += ms;
        P.sweeps += 1;
        continue;
      }
      P.ms[t.family] += ms;
      P.nlaunch[t.family] += 1;
    }
    for (int b = 0; b < 4; ++b) { P.nodes[b] += pn[b]; P.arcs[b] += pa[b]; }
    if (!lv.ew) for (int b = 0; b < 4; ++b) P.arcs_unit += pa[b];
    for (const PhaseRec& q : precs) {
      float sw = 0.f, ad = 0.f;
      SCLAP_CUDA(cudaEventElapsedTime(&sw, q.a, q.b));
      SCLAP_CUDA(cudaEventElapsedTime(&ad, q.b, q.c));
      const double rec[7] = {(double)q.ph, (double)q.r, (double)q.sub, (double)q.nodes,
                             (double)q.arcs, (double)sw, (double)ad};
      P.phases.insert(P.phases.end(), rec, rec + 7);
      event_to_pool(q.c);
    }
    for (const Timed& t : timed) { event_to_pool(t.a); event_to_pool(t.b); }
  }
  return h_arcs;
}

}  // namespace sclap
