// sclap_oracle.cpp -- plain single-threaded CPU oracle for multilevel
// size-constrained label propagation (SCLaP) partitioning.
//
// TEST INFRASTRUCTURE ONLY: checked against the CUDA path by the tests; never
// linked into the product.  Written for a reader holding the paper
// (Meyerhenke, Sanders, Schulz, "Partitioning Complex Networks via
// Size-constrained Clustering"): every function names the section it
// follows.  No blocking, fusion or reordering beyond what the definitions
// state; speed is not a goal.
#include "sclap_oracle.h"

#include <algorithm>
#include <map>
#include <climits>
#include <cmath>
#include <cstring>
#include <tuple>
#include <utility>
#include <vector>

namespace {

using std::vector;

// ---------------------------------------------------------------------------
// Counter-based generator.  SplitMix64's output function (Steele, Lea, Flood,
// "Fast splittable pseudorandom number generators", OOPSLA 2014): add the
// golden-gamma constant, then two xor-shift-multiply rounds and a final
// xor-shift.  Every random choice of the method ("ties are broken randomly",
// Sec. 3.1; random orders, seeds) is a pure function of such hashes, which
// makes every run reproducible.
// ---------------------------------------------------------------------------
uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t hkey(uint64_t seed, uint64_t phase, uint64_t level, uint64_t round) {
  return mix64(mix64(mix64(mix64(seed) ^ phase) ^ level) ^ round);
}

// Per-node hash of a round: high 32 bits pick the colour class, low 32 bits
// are the admission priority.
inline uint64_t node_hash(uint64_t rkey, int64_t v) { return mix64(rkey ^ (uint64_t)v); }
// Tie-break hash of candidate label C for the node with hash hv.
inline uint64_t cand_hash(uint64_t hv, int64_t C) { return mix64(hv ^ (uint64_t)C); }

struct G {
  int64_t n;
  const int64_t* xadj;
  const int32_t* adj;
  const int32_t* nw;
  const int32_t* ew;
  // V-cycles (App. A): block of every node in the partition a clustering
  // must respect (a cluster may only gather nodes of one block), or null
  const int32_t* rblk = nullptr;
  int64_t deg(int64_t v) const { return xadj[v + 1] - xadj[v]; }
};

// Owned graph (coarse levels).
struct OG {
  int64_t n = 0;
  vector<int64_t> xadj;
  vector<int32_t> adj, nw, ew;
  G view() const { return G{n, xadj.data(), adj.data(), nw.data(), ew.data()}; }
};

// Edge cut (Sec. 2.1): sum over undirected edges whose ends lie in different
// blocks; every edge is seen twice in CSR, hence the halving.
int64_t cut_of(const G& g, const int32_t* block) {
  int64_t twice = 0;
  for (int64_t v = 0; v < g.n; ++v)
    for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e)
      if (block[v] != block[g.adj[e]]) twice += g.ew[e];
  return twice / 2;
}

// ---------------------------------------------------------------------------
// Connection of a node to each neighbouring label: w({(v,u) : u in N(v),
// label(u) = C}) (Sec. 3.1).  A dense accumulator with a touched list; the
// decision below is independent of the order in which labels are visited.
// ---------------------------------------------------------------------------
struct Conn {
  vector<int64_t> acc;
  vector<int32_t> touched;
  explicit Conn(int64_t nlabels) : acc((size_t)nlabels, 0) {}
  void build(const G& g, const int32_t* label, int64_t v) {
    clear();
    for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
      int32_t C = label[g.adj[e]];
      if (C < 0) continue;
      if (acc[C] == 0) touched.push_back(C);
      acc[C] += g.ew[e];
    }
  }
  int64_t get(int32_t C) const { return C >= 0 ? acc[C] : 0; }
  void clear() {
    for (int32_t C : touched) acc[C] = 0;
    touched.clear();
  }
};

// ---------------------------------------------------------------------------
// Move rule of size-constrained LP (Sec. 3.1).
//  * A neighbouring label C != own is eligible if W[C] + c(v) <= bound (the
//    block "will not become overloaded once v is moved").
//  * v moves to the eligible label with the strongest connection; ties are
//    broken by the hash of (v, C), then by the smaller C; v stays if the best
//    connection does not exceed its connection to its own label (a tie keeps
//    the current label).
//  * Local-search mode with an overloaded own block (W[own] > bound): own is
//    not considered and v moves to the strongest eligible block, every block
//    being a candidate (connection 0 when not adjacent).
// Returns true with (t, gain) when v should move.
// ---------------------------------------------------------------------------
bool choose(int mode, const Conn& conn, int32_t own, int64_t cv, const int64_t* W,
            int64_t nlabels, int64_t bound, uint64_t hv, int32_t* t_out, int64_t* gain_out,
            const int32_t* rblk = nullptr, int32_t v = 0) {
  const int64_t own_conn = conn.get(own);
  const bool overloaded = (mode == ORC_MODE_REFINE) && W[own] > bound;
  bool have = false;
  int64_t bc = 0;
  uint64_t bh = 0;
  int32_t bC = -1;
  auto consider = [&](int32_t C, int64_t c) {
    if (C == own) return;
    if (W[C] + cv > bound) return;
    // a clustering that respects a partition joins only clusters of v's block
    // (labels are node ids while clustering, so rblk[C] is the cluster's block)
    if (rblk && rblk[C] != rblk[v]) return;
    uint64_t h = cand_hash(hv, C);
    if (!have || c > bc || (c == bc && (h < bh || (h == bh && C < bC)))) {
      have = true; bc = c; bh = h; bC = C;
    }
  };
  if (overloaded) {
    for (int32_t b = 0; b < (int32_t)nlabels; ++b) consider(b, conn.get(b));
  } else {
    for (int32_t C : conn.touched) consider(C, conn.get(C));
  }
  if (!have) return false;
  if (!overloaded && bc <= own_conn) return false;
  *t_out = bC;
  *gain_out = bc - own_conn;
  return true;
}

struct Prop {
  int32_t v, t, own;
  int64_t cv, gain;
  uint32_t prio;
};

inline int32_t gain_key(int64_t g) {
  return (int32_t)std::max<int64_t>(INT32_MIN, std::min<int64_t>(INT32_MAX, g));
}
// Admission order of competing proposals: larger gain first, then smaller
// priority hash, then smaller node id.
inline bool before(const Prop& a, const Prop& b) {
  int32_t ga = gain_key(a.gain), gb = gain_key(b.gain);
  if (ga != gb) return ga > gb;
  if (a.prio != b.prio) return a.prio < b.prio;
  return a.v < b.v;
}

// ---------------------------------------------------------------------------
// One synchronous sub-round.  Every node of the colour class decides with
// the labels and weights as they were at the sub-round start.  Admission
// keeps the size constraint exact without ordering the moves:
//  * target side: if all proposals into t fit (W[t] + sum c <= bound) they
//    are all admitted, otherwise the longest prefix in admission order whose
//    cumulative weight fits is admitted (departures from t in the same
//    sub-round are not credited, so the bound always holds);
//  * source side (local search only): moves out of an overloaded block are
//    admitted in admission order only while the weight already leaving is
//    below the block's excess, so an overloaded block is not emptied.
// Admitted moves are then applied; moved nodes activate their neighbours.
// ---------------------------------------------------------------------------
int64_t sync_subround(int mode, const G& g, int32_t* label, int64_t* W, int64_t nlabels,
                      int64_t bound, uint64_t rkey, const vector<int32_t>& nodes,
                      uint8_t* active_next, Conn& conn) {
  vector<Prop> props;
  for (int32_t v : nodes) {
    uint64_t hv = node_hash(rkey, v);
    conn.build(g, label, v);
    int32_t t;
    int64_t gain;
    if (choose(mode, conn, label[v], g.nw[v], W, nlabels, bound, hv, &t, &gain,
               mode == ORC_MODE_CLUSTER ? g.rblk : nullptr, v))
      props.push_back(Prop{v, t, label[v], (int64_t)g.nw[v], gain, (uint32_t)hv});
  }
  conn.clear();
  if (props.empty()) return 0;

  // Target side.
  vector<char> admitted(props.size(), 0);
  vector<size_t> idx(props.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
    if (props[a].t != props[b].t) return props[a].t < props[b].t;
    return before(props[a], props[b]);
  });
  for (size_t s = 0; s < idx.size();) {
    size_t e = s;
    int64_t sum = 0;
    const int32_t t = props[idx[s]].t;
    while (e < idx.size() && props[idx[e]].t == t) sum += props[idx[e++]].cv;
    const int64_t cap = bound - W[t];
    int64_t acc = 0;
    for (size_t i = s; i < e; ++i) {
      if (sum <= cap) { admitted[idx[i]] = 1; continue; }
      if (acc + props[idx[i]].cv > cap) break;
      acc += props[idx[i]].cv;
      admitted[idx[i]] = 1;
    }
    s = e;
  }

  // Source side (local search with overloaded blocks).
  if (mode == ORC_MODE_REFINE) {
    vector<size_t> forced;
    for (size_t i = 0; i < props.size(); ++i)
      if (admitted[i] && W[props[i].own] > bound) forced.push_back(i);
    std::sort(forced.begin(), forced.end(), [&](size_t a, size_t b) {
      if (props[a].own != props[b].own) return props[a].own < props[b].own;
      return before(props[a], props[b]);
    });
    for (size_t s = 0; s < forced.size();) {
      size_t e = s;
      const int32_t src = props[forced[s]].own;
      while (e < forced.size() && props[forced[e]].own == src) ++e;
      const int64_t excess = W[src] - bound;
      int64_t leaving = 0;
      for (size_t i = s; i < e; ++i) {
        if (leaving < excess) leaving += props[forced[i]].cv;
        else admitted[forced[i]] = 0;
      }
      s = e;
    }
  }

  // Apply.
  int64_t moved = 0;
  for (size_t i = 0; i < props.size(); ++i) {
    if (!admitted[i]) continue;
    const Prop& p = props[i];
    label[p.v] = p.t;
    W[p.t] += p.cv;
    W[p.own] -= p.cv;
    ++moved;
    if (active_next)
      for (int64_t e = g.xadj[p.v]; e < g.xadj[p.v + 1]; ++e) active_next[g.adj[e]] = 1;
  }
  return moved;
}

// One synchronous round: the active nodes (all when active_cur is NULL) are
// split by the colour hash into `S` classes processed one after another.
int64_t sync_round(int mode, const G& g, int32_t* label, int64_t* W, int64_t nlabels,
                   int64_t bound, uint64_t rkey, int S, const uint8_t* active_cur,
                   uint8_t* active_next) {
  vector<vector<int32_t>> cls((size_t)S);
  for (int64_t v = 0; v < g.n; ++v) {
    if (active_cur && !active_cur[v]) continue;
    uint64_t hv = node_hash(rkey, v);
    cls[(uint32_t)(hv >> 32) % (uint32_t)S].push_back((int32_t)v);
  }
  Conn conn(nlabels);
  int64_t moved = 0;
  for (int s = 0; s < S; ++s)
    moved += sync_subround(mode, g, label, W, nlabels, bound, rkey, cls[s], active_next, conn);
  return moved;
}

// Node order of the sequential algorithm: increasing degree (Sec. 4, "Node
// Ordering for Label Propagation"), equal degrees in hash order.
vector<int32_t> degree_order(const G& g, uint64_t rkey) {
  vector<std::tuple<int64_t, uint64_t, int32_t>> keyed((size_t)g.n);
  for (int64_t v = 0; v < g.n; ++v)
    keyed[v] = std::make_tuple(g.deg(v), node_hash(rkey, v), (int32_t)v);
  std::sort(keyed.begin(), keyed.end());
  vector<int32_t> order((size_t)g.n);
  for (int64_t i = 0; i < g.n; ++i) order[i] = std::get<2>(keyed[i]);
  return order;
}

// Random node order (configuration R of Table 2): the hash order alone.
vector<int32_t> hashed_order(const G& g, uint64_t rkey) {
  vector<std::pair<uint64_t, int32_t>> keyed((size_t)g.n);
  for (int64_t v = 0; v < g.n; ++v) keyed[v] = std::make_pair(node_hash(rkey, v), (int32_t)v);
  std::sort(keyed.begin(), keyed.end());
  vector<int32_t> order((size_t)g.n);
  for (int64_t i = 0; i < g.n; ++i) order[i] = keyed[i].second;
  return order;
}

// One sequential clustering round (Sec. 3.1): visit every node once, move it
// immediately to its strongest eligible cluster.  With active flags (Sec. 4,
// "Active Nodes"), nodes not flagged in active_cur are skipped and the
// neighbours of every moved node are flagged in active_next.
int64_t seq_cluster_round(const G& g, int32_t* label, int64_t* W, int64_t bound, uint64_t rkey,
                          Conn& conn, bool random_order, const uint8_t* active_cur,
                          uint8_t* active_next) {
  int64_t moved = 0;
  const vector<int32_t> order = random_order ? hashed_order(g, rkey) : degree_order(g, rkey);
  for (int32_t v : order) {
    if (active_cur && !active_cur[v]) continue;
    uint64_t hv = node_hash(rkey, v);
    conn.build(g, label, v);
    int32_t t;
    int64_t gain;
    if (choose(ORC_MODE_CLUSTER, conn, label[v], g.nw[v], W, g.n, bound, hv, &t, &gain,
               g.rblk, v)) {
      W[t] += g.nw[v];
      W[label[v]] -= g.nw[v];
      label[v] = t;
      ++moved;
      if (active_next)
        for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) active_next[g.adj[e]] = 1;
    }
  }
  conn.clear();
  return moved;
}

// Size-constrained clustering of one level (Sec. 3.1): every node starts in
// its own cluster; at most l rounds; stop after a round in which fewer than
// five percent of the nodes changed their cluster.
int cluster_level(int variant, const G& g, int64_t U, uint64_t seed, int32_t level,
                  const orc_config& cfg, int32_t* label, int32_t* rounds_out) {
  vector<int64_t> W((size_t)g.n);
  for (int64_t v = 0; v < g.n; ++v) { label[v] = (int32_t)v; W[v] = g.nw[v]; }
  Conn conn(g.n);
  int32_t rounds = 0;
  // active nodes (Sec. 4): every node is active in the first round; a node
  // is active in a later round iff a neighbour changed its cluster in the
  // round before
  const bool act = cfg.cluster_active != 0;
  vector<uint8_t> cur(act ? (size_t)g.n : 0, 1), nxt(act ? (size_t)g.n : 0, 0);
  for (int32_t r = 0; r < cfg.lp_rounds_coarse; ++r) {
    uint64_t rkey = hkey(seed, ORC_PH_CLUSTER, (uint64_t)level, (uint64_t)r);
    int64_t moved = variant == ORC_SYNC
        ? sync_round(ORC_MODE_CLUSTER, g, label, W.data(), g.n, U, rkey, cfg.sub_rounds,
                     act ? cur.data() : nullptr, act ? nxt.data() : nullptr)
        : seq_cluster_round(g, label, W.data(), U, rkey, conn, cfg.random_order != 0,
                            act ? cur.data() : nullptr, act ? nxt.data() : nullptr);
    ++rounds;
    if (act) {
      cur.swap(nxt);
      std::fill(nxt.begin(), nxt.end(), 0);
    }
    if (20 * moved < g.n) break;
  }
  if (rounds_out) *rounds_out = rounds;
  return ORC_OK;
}

// Overlay of two clusterings (Sec. 4, "Ensemble Clusterings"): the pair
// (a[v], b[v]) names v's overlay cluster; pairs are numbered by their first
// occurrence in node order.
void overlay(int64_t n, const int32_t* a, const int32_t* b, int32_t* out) {
  std::map<std::pair<int32_t, int32_t>, int32_t> H;
  int32_t c = 0;
  for (int64_t v = 0; v < n; ++v) {
    const auto key = std::make_pair(a[v], b[v]);
    auto it = H.find(key);
    if (it == H.end()) it = H.emplace(key, c++).first;
    out[v] = it->second;
  }
}

// Number of clusterings of an ensemble (Sec. 5).
int32_t ensemble_size_for(int32_t k, const orc_config& cfg) {
  if (cfg.ensemble_size > 0) return cfg.ensemble_size;
  return k < 16 ? 18 : (k <= 32 ? 7 : 3);
}

// Clustering of one coarsening level: plain, or the overlay of an ensemble
// of clusterings (clustering 0 uses the run's seed, clustering j >= 1 the
// key hkey(seed, ENSEMBLE, level, j)).  rounds_out: clustering 0's rounds.
void coarsen_clustering(int variant, const G& g, int64_t U, uint64_t seed, int32_t level,
                        int32_t k, const orc_config& cfg, int32_t* label, int32_t* rounds_out) {
  cluster_level(variant, g, U, seed, level, cfg, label, rounds_out);
  if (!cfg.ensemble) return;
  const int32_t ell = ensemble_size_for(k, cfg);
  vector<int32_t> C((size_t)g.n), O((size_t)g.n);
  for (int32_t j = 1; j < ell; ++j) {
    const uint64_t sj = hkey(seed, ORC_PH_ENSEMBLE, (uint64_t)level, (uint64_t)j);
    cluster_level(variant, g, U, sj, level, cfg, C.data(), nullptr);
    overlay(g.n, label, C.data(), O.data());
    std::copy(O.begin(), O.end(), label);
  }
}

// Cluster contraction (Sec. 3.1): each cluster becomes one node whose weight
// is the sum of its members; two coarse nodes are adjacent iff their clusters
// are, with the summed weight of the edges between them.  Coarse ids follow
// the order of the cluster labels; rows are sorted by neighbour id.
int contract(const G& g, const int32_t* label, vector<int32_t>& cmap, OG& c) {
  vector<int32_t> cid((size_t)g.n, -1);
  for (int64_t v = 0; v < g.n; ++v) cid[label[v]] = 0;
  int64_t nc = 0;
  for (int64_t C = 0; C < g.n; ++C)
    if (cid[C] == 0) cid[C] = (int32_t)nc++;
  cmap.assign((size_t)g.n, 0);
  c.n = nc;
  c.nw.assign((size_t)nc, 0);
  vector<std::tuple<int32_t, int32_t, int64_t>> arcs;
  for (int64_t v = 0; v < g.n; ++v) {
    cmap[v] = cid[label[v]];
    c.nw[cmap[v]] += g.nw[v];
  }
  for (int64_t v = 0; v < g.n; ++v)
    for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
      int32_t a = cmap[v], b = cmap[g.adj[e]];
      if (a != b) arcs.emplace_back(a, b, (int64_t)g.ew[e]);
    }
  std::sort(arcs.begin(), arcs.end());
  c.xadj.assign((size_t)nc + 1, 0);
  c.adj.clear();
  c.ew.clear();
  for (size_t i = 0; i < arcs.size();) {
    size_t j = i;
    int64_t w = 0;
    while (j < arcs.size() && std::get<0>(arcs[j]) == std::get<0>(arcs[i]) &&
           std::get<1>(arcs[j]) == std::get<1>(arcs[i]))
      w += std::get<2>(arcs[j++]);
    if (w > INT32_MAX) return ORC_EOVERFLOW;
    c.adj.push_back(std::get<1>(arcs[i]));
    c.ew.push_back((int32_t)w);
    c.xadj[std::get<0>(arcs[i]) + 1]++;
    i = j;
  }
  for (int64_t a = 0; a < nc; ++a) c.xadj[a + 1] += c.xadj[a];
  return ORC_OK;
}

// Leftover nodes (never reached by growing) go, in increasing id order, to
// the lightest blocks by water-filling: find the smallest level L with
// sum_b max(0, L - W[b]) >= R (R = leftover weight), lay the blocks' free
// capacities below L end to end in (weight, id) order and give each leftover
// node the block whose stretch contains its exclusive prefix weight.
void waterfill(const G& g, int32_t k, int32_t* label, int64_t* W) {
  int64_t R = 0;
  for (int64_t v = 0; v < g.n; ++v)
    if (label[v] < 0) R += g.nw[v];
  if (R == 0) return;
  int64_t lo = W[0], hi = W[0];
  for (int32_t b = 1; b < k; ++b) { lo = std::min(lo, W[b]); hi = std::max(hi, W[b]); }
  hi += R;
  auto fill = [&](int64_t L) {
    int64_t s = 0;
    for (int32_t b = 0; b < k; ++b) s += std::max<int64_t>(0, L - W[b]);
    return s;
  };
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (fill(mid) >= R) hi = mid; else lo = mid + 1;
  }
  const int64_t L = lo;
  vector<int32_t> order((size_t)k);
  for (int32_t b = 0; b < k; ++b) order[b] = b;
  std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return W[a] != W[b] ? W[a] < W[b] : a < b;
  });
  vector<int64_t> A((size_t)k);
  int64_t s = 0;
  for (int32_t j = 0; j < k; ++j) { A[j] = s; s += std::max<int64_t>(0, L - W[order[j]]); }
  int64_t p = 0;
  vector<int32_t> assigned;
  for (int64_t v = 0; v < g.n; ++v) {
    if (label[v] >= 0) continue;
    int32_t j = (int32_t)(std::upper_bound(A.begin(), A.end(), p) - A.begin()) - 1;
    label[v] = order[j];
    assigned.push_back((int32_t)v);
    p += g.nw[v];
  }
  for (int32_t v : assigned) W[label[v]] += g.nw[v];
}

// Greedy graph growing (initial partitioning of the coarsest graph; the paper
// uses KaHIP's, which it does not specify).  Blocks 0..k-1 are grown one
// after another: block j starts at the unassigned non-isolated node with the
// smallest hash and, step by step, absorbs the unassigned nodes connected to
// it in increasing id order, as long as its weight stays <= avg.  Nodes left
// over are water-filled.
void ggg(const G& g, int32_t k, int64_t avg, uint64_t tkey, int32_t level, int32_t* label,
         int64_t* W) {
  for (int64_t v = 0; v < g.n; ++v) label[v] = -1;
  for (int32_t b = 0; b < k; ++b) W[b] = 0;
  vector<int64_t> conn((size_t)g.n, 0);
  vector<int32_t> step;
  for (int32_t j = 0; j < k; ++j) {
    uint64_t skey = hkey(tkey, ORC_PH_GGG, (uint64_t)level, (uint64_t)j);
    int64_t seed = -1;
    uint64_t best = 0;
    for (int64_t v = 0; v < g.n; ++v) {
      if (label[v] >= 0 || g.deg(v) == 0) continue;
      uint64_t h = mix64(skey ^ (uint64_t)v);
      if (seed < 0 || h < best) { seed = v; best = h; }
    }
    if (seed < 0) break;
    std::fill(conn.begin(), conn.end(), 0);
    step.assign(1, (int32_t)seed);
    label[seed] = j;
    W[j] = g.nw[seed];
    while (true) {
      for (int32_t u : step)
        for (int64_t e = g.xadj[u]; e < g.xadj[u + 1]; ++e)
          if (label[g.adj[e]] < 0) conn[g.adj[e]] += g.ew[e];
      if (W[j] >= avg) break;
      step.clear();
      int64_t acc = W[j];
      for (int64_t u = 0; u < g.n; ++u) {
        if (label[u] >= 0 || conn[u] == 0) continue;
        if (acc + g.nw[u] > avg) break;
        acc += g.nw[u];
        step.push_back((int32_t)u);
      }
      if (step.empty()) break;
      for (int32_t u : step) label[u] = j;
      W[j] = acc;
    }
  }
  waterfill(g, k, label, W);
}

// LP as local search on one level (Sec. 3.1 last paragraph) with the active
// nodes approach (Sec. 4; always used in refinement).  SYNC: the active set
// of round r+1 is the set of neighbours of nodes moved in round r.  SEQ: two
// FIFO queues with membership bits (App. B.2); round 0 visits every node in
// degree order.  Stops after l rounds or a round moving < 5% of the nodes.
int refine_level(int variant, const G& g, int32_t k, int64_t Lmax, uint64_t seed,
                 int32_t phase, int32_t level, const orc_config& cfg, int32_t* block,
                 int64_t* W, int32_t* rounds_out) {
  int32_t rounds = 0;
  if (variant == ORC_SYNC) {
    vector<uint8_t> cur((size_t)g.n, 1), nxt((size_t)g.n, 0);
    for (int32_t r = 0; r < cfg.lp_rounds_refine; ++r) {
      uint64_t rkey = hkey(seed, (uint64_t)phase, (uint64_t)level, (uint64_t)r);
      int64_t moved = sync_round(ORC_MODE_REFINE, g, block, W, k, Lmax, rkey, cfg.sub_rounds,
                                 cur.data(), nxt.data());
      cur.swap(nxt);
      std::fill(nxt.begin(), nxt.end(), 0);
      ++rounds;
      if (20 * moved < g.n) break;
    }
  } else {
    Conn conn(k);
    vector<int32_t> queue = degree_order(g, hkey(seed, (uint64_t)phase, (uint64_t)level, 0));
    vector<uint8_t> in_cur((size_t)g.n, 1), in_next((size_t)g.n, 0);
    for (int32_t r = 0; r < cfg.lp_rounds_refine; ++r) {
      uint64_t rkey = hkey(seed, (uint64_t)phase, (uint64_t)level, (uint64_t)r);
      vector<int32_t> next;
      int64_t moved = 0;
      for (int32_t v : queue) {
        in_cur[v] = 0;
        uint64_t hv = node_hash(rkey, v);
        conn.build(g, block, v);
        int32_t t;
        int64_t gain;
        if (!choose(ORC_MODE_REFINE, conn, block[v], g.nw[v], W, k, Lmax, hv, &t, &gain))
          continue;
        W[t] += g.nw[v];
        W[block[v]] -= g.nw[v];
        block[v] = t;
        ++moved;
        for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
          int32_t u = g.adj[e];
          if (!in_next[u]) { in_next[u] = 1; next.push_back(u); }
        }
      }
      conn.clear();
      queue.swap(next);
      in_cur.swap(in_next);
      ++rounds;
      if (20 * moved < g.n) break;
    }
  }
  if (rounds_out) *rounds_out = rounds;
  return ORC_OK;
}

int64_t max_weight(const int64_t* W, int32_t k) {
  int64_t m = 0;
  for (int32_t b = 0; b < k; ++b) m = std::max(m, W[b]);
  return m;
}

void block_weights(const G& g, int32_t k, const int32_t* block, int64_t* W) {
  for (int32_t b = 0; b < k; ++b) W[b] = 0;
  for (int64_t v = 0; v < g.n; ++v) W[block[v]] += g.nw[v];
}

// Initial partitioning: `ip_trials` seeded trials of growing + LP local
// search; the trial with the smallest (overload, cut, trial index) is kept.
// Nodes without neighbours cannot affect a cut and never move in LP, so the
// trials run on the induced subgraph of the other nodes (ids renumbered in
// order); the isolated nodes are water-filled into the best trial's blocks.
int initial_partition(int variant, const G& g, int32_t k, int64_t Lmax, int64_t avg,
                      uint64_t seed, int32_t level, const orc_config& cfg, int32_t* block_out,
                      int64_t* cut_out, int32_t* best_out) {
  vector<int32_t> rank((size_t)g.n, -1);
  OG ga;
  for (int64_t v = 0; v < g.n; ++v)
    if (g.deg(v) > 0) rank[v] = (int32_t)ga.n++;
  ga.xadj.assign((size_t)ga.n + 1, 0);
  ga.nw.resize((size_t)ga.n);
  for (int64_t v = 0; v < g.n; ++v) {
    if (rank[v] < 0) continue;
    ga.nw[rank[v]] = g.nw[v];
    for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
      ga.adj.push_back(rank[g.adj[e]]);
      ga.ew.push_back(g.ew[e]);
    }
    ga.xadj[rank[v] + 1] = (int64_t)ga.adj.size();
  }
  const G gA = ga.view();
  vector<int32_t> lab((size_t)gA.n), best_lab((size_t)gA.n);
  vector<int64_t> W((size_t)k), best_W((size_t)k, 0);
  int64_t bo = -1, bc = 0;
  int32_t bt = 0;
  if (gA.n > 0) {
    bt = -1;
    for (int32_t t = 0; t < cfg.ip_trials; ++t) {
      uint64_t tkey = hkey(seed, ORC_PH_TRIAL, (uint64_t)level, (uint64_t)t);
      ggg(gA, k, avg, tkey, level, lab.data(), W.data());
      refine_level(variant, gA, k, Lmax, tkey, ORC_PH_IPREF, level, cfg, lab.data(), W.data(),
                   nullptr);
      int64_t ov = std::max<int64_t>(0, max_weight(W.data(), k) - Lmax);
      int64_t c = cut_of(gA, lab.data());
      if (bt < 0 || ov < bo || (ov == bo && c < bc)) {
        bo = ov; bc = c; bt = t;
        best_lab = lab;
        best_W = W;
      }
    }
  }
  for (int64_t v = 0; v < g.n; ++v) block_out[v] = rank[v] >= 0 ? best_lab[rank[v]] : -1;
  waterfill(g, k, block_out, best_W.data());
  if (cut_out) *cut_out = bc;
  if (best_out) *best_out = bt;
  return ORC_OK;
}

// Final balance repair on the input graph: synchronous local-search rounds
// restricted to the nodes of overloaded blocks (which must leave their block,
// Sec. 3.1), until every block is <= Lmax.
int repair(const G& g, int32_t k, int64_t Lmax, uint64_t seed, const orc_config& cfg,
           int32_t* block, int64_t* W, int32_t* rounds_out) {
  int32_t rounds = 0;
  vector<uint8_t> act((size_t)g.n);
  for (int32_t r = 0; r < cfg.repair_rounds; ++r) {
    if (max_weight(W, k) <= Lmax) break;
    for (int64_t v = 0; v < g.n; ++v) act[v] = W[block[v]] > Lmax;
    sync_round(ORC_MODE_REFINE, g, block, W, k, Lmax, hkey(seed, ORC_PH_REPAIR, 0, (uint64_t)r),
               cfg.sub_rounds, act.data(), nullptr);
    ++rounds;
  }
  if (rounds_out) *rounds_out = rounds;
  return max_weight(W, k) <= Lmax ? ORC_OK : ORC_EINFEASIBLE;
}

int bounds(int64_t cV, int32_t max_c, int32_t k, double eps, int32_t f, int64_t* Lmax,
           int64_t* U) {
  if (k < 1 || f < 1 || !(eps >= 0.0) || cV < 0) return ORC_EINVAL;
  const int64_t avg = (cV + k - 1) / k;
  const int64_t L = (int64_t)std::floor((1.0 + eps) * (double)avg);
  *Lmax = L;
  *U = std::max<int64_t>((int64_t)max_c, L / f);
  return ORC_OK;
}

}  // namespace

extern "C" {

void orc_default_config(orc_config* cfg) {
  cfg->lp_rounds_coarse = 10;
  cfg->lp_rounds_refine = 10;
  cfg->f = 18;
  cfg->coarse_min_nodes = 1000;
  cfg->ip_trials = 16;
  cfg->sub_rounds = 8;
  cfg->repair_rounds = 64;
  cfg->max_levels = 64;
  cfg->cluster_active = 0;
  cfg->random_order = 0;
  cfg->ensemble = 0;
  cfg->ensemble_size = 0;
  cfg->vcycles = 1;
}

uint64_t orc_mix64(uint64_t x) { return mix64(x); }
uint64_t orc_hkey(uint64_t s, uint64_t p, uint64_t l, uint64_t r) { return hkey(s, p, l, r); }

int orc_bounds(int64_t cV, int32_t max_c, int32_t k, double eps, int32_t f, int64_t* Lmax,
               int64_t* U) {
  return bounds(cV, max_c, k, eps, f, Lmax, U);
}

int orc_lp_round(int32_t mode, int64_t n, const int64_t* xadj, const int32_t* adj,
                 const int32_t* nw, const int32_t* ew, int32_t* label, int64_t* W,
                 int64_t nlabels, int64_t bound, uint64_t rkey, int32_t sub_rounds,
                 const uint8_t* active_cur, uint8_t* active_next, int64_t* moved) {
  if (sub_rounds < 1) return ORC_EINVAL;
  G g{n, xadj, adj, nw, ew};
  int64_t m = sync_round(mode, g, label, W, nlabels, bound, rkey, sub_rounds, active_cur,
                         active_next);
  if (moved) *moved = m;
  return ORC_OK;
}

int orc_cluster(int32_t variant, int64_t n, const int64_t* xadj, const int32_t* adj,
                const int32_t* nw, const int32_t* ew, int64_t U, uint64_t seed, int32_t level,
                const orc_config* cfg, int32_t* label_out, int32_t* rounds_out) {
  orc_config c;
  if (cfg) c = *cfg; else orc_default_config(&c);
  G g{n, xadj, adj, nw, ew};
  return cluster_level(variant, g, U, seed, level, c, label_out, rounds_out);
}

int orc_cluster_in_blocks(int32_t variant, int64_t n, const int64_t* xadj, const int32_t* adj,
                          const int32_t* nw, const int32_t* ew, int64_t U, uint64_t seed,
                          int32_t level, const orc_config* cfg, const int32_t* blk,
                          int32_t* label_out, int32_t* rounds_out) {
  if (n < 1 || !blk || !label_out) return ORC_EINVAL;
  orc_config c;
  if (cfg) c = *cfg; else orc_default_config(&c);
  G g{n, xadj, adj, nw, ew};
  g.rblk = blk;
  return cluster_level(variant, g, U, seed, level, c, label_out, rounds_out);
}

int orc_overlay(int64_t n, const int32_t* a, const int32_t* b, int32_t* out) {
  if (n < 0 || (n > 0 && (!a || !b || !out))) return ORC_EINVAL;
  overlay(n, a, b, out);
  return ORC_OK;
}

int orc_cluster_hierarchy(int32_t variant, int64_t n, const int64_t* xadj, const int32_t* adj,
                          const int32_t* nw, const int32_t* ew, int64_t U, int64_t stop_nodes,
                          uint64_t seed, const orc_config* cfg, int32_t* comm_out,
                          int32_t* levels_out, int64_t* level_n_out, int32_t cap) {
  if (n < 1 || U < 1 || !comm_out) return ORC_EINVAL;
  orc_config c;
  if (cfg) c = *cfg; else orc_default_config(&c);
  for (int64_t v = 0; v < n; ++v) comm_out[v] = (int32_t)v;
  OG cur;
  cur.n = n;
  cur.xadj.assign(xadj, xadj + n + 1);
  cur.adj.assign(adj, adj + xadj[n]);
  cur.nw.assign(nw, nw + n);
  cur.ew.assign(ew, ew + xadj[n]);
  int32_t levels = 0;
  if (level_n_out && cap > 0) level_n_out[0] = n;
  while (cur.n > stop_nodes && levels + 1 < c.max_levels) {
    const G g = cur.view();
    vector<int32_t> label((size_t)g.n);
    cluster_level(variant, g, U, seed, levels, c, label.data(), nullptr);
    vector<int32_t> cmap;
    OG coarse;
    const int rc = contract(g, label.data(), cmap, coarse);
    if (rc != ORC_OK) return rc;
    if (20 * (g.n - coarse.n) < g.n) break;      // shrink below 5%: discarded
    for (int64_t v = 0; v < n; ++v) comm_out[v] = cmap[comm_out[v]];
    cur = std::move(coarse);
    ++levels;
    if (level_n_out && levels < cap) level_n_out[levels] = cur.n;
  }
  if (levels_out) *levels_out = levels;
  return ORC_OK;
}

int orc_contract(int64_t n, const int64_t* xadj, const int32_t* adj, const int32_t* nw,
                 const int32_t* ew, const int32_t* label, int32_t* cmap_out, int64_t* nc_out,
                 int32_t* cnw_out, int64_t* cxadj_out, int32_t* cadj_out, int32_t* cew_out,
                 int64_t* mc_out) {
  G g{n, xadj, adj, nw, ew};
  vector<int32_t> cmap;
  OG c;
  int rc = contract(g, label, cmap, c);
  if (rc != ORC_OK) return rc;
  std::copy(cmap.begin(), cmap.end(), cmap_out);
  std::copy(c.nw.begin(), c.nw.end(), cnw_out);
  std::copy(c.xadj.begin(), c.xadj.end(), cxadj_out);
  std::copy(c.adj.begin(), c.adj.end(), cadj_out);
  std::copy(c.ew.begin(), c.ew.end(), cew_out);
  *nc_out = c.n;
  *mc_out = (int64_t)c.adj.size();
  return ORC_OK;
}

int orc_ggg(int64_t n, const int64_t* xadj, const int32_t* adj, const int32_t* nw,
            const int32_t* ew, int32_t k, int64_t avg, uint64_t tkey, int32_t level,
            int32_t* block_out, int64_t* W_out) {
  G g{n, xadj, adj, nw, ew};
  ggg(g, k, avg, tkey, level, block_out, W_out);
  return ORC_OK;
}

int orc_initial_partition(int32_t variant, int64_t n, const int64_t* xadj, const int32_t* adj,
                          const int32_t* nw, const int32_t* ew, int32_t k, int64_t Lmax,
                          int64_t avg, uint64_t seed, int32_t level, const orc_config* cfg,
                          int32_t* block_out, int64_t* cut_out, int32_t* best_trial_out) {
  orc_config c;
  if (cfg) c = *cfg; else orc_default_config(&c);
  G g{n, xadj, adj, nw, ew};
  return initial_partition(variant, g, k, Lmax, avg, seed, level, c, block_out, cut_out,
                           best_trial_out);
}

int orc_refine(int32_t variant, int64_t n, const int64_t* xadj, const int32_t* adj,
               const int32_t* nw, const int32_t* ew, int32_t k, int64_t Lmax, uint64_t seed,
               int32_t phase, int32_t level, const orc_config* cfg, int32_t* block,
               int32_t* rounds_out) {
  orc_config c;
  if (cfg) c = *cfg; else orc_default_config(&c);
  G g{n, xadj, adj, nw, ew};
  vector<int64_t> W((size_t)k);
  block_weights(g, k, block, W.data());
  return refine_level(variant, g, k, Lmax, seed, phase, level, c, block, W.data(), rounds_out);
}

int orc_repair(int64_t n, const int64_t* xadj, const int32_t* adj, const int32_t* nw,
               const int32_t* ew, int32_t k, int64_t Lmax, uint64_t seed,
               const orc_config* cfg, int32_t* block, int32_t* rounds_out) {
  orc_config c;
  if (cfg) c = *cfg; else orc_default_config(&c);
  G g{n, xadj, adj, nw, ew};
  vector<int64_t> W((size_t)k);
  block_weights(g, k, block, W.data());
  return repair(g, k, Lmax, seed, c, block, W.data(), rounds_out);
}

int64_t orc_cut(int64_t n, const int64_t* xadj, const int32_t* adj, const int32_t* ew,
                const int32_t* block) {
  G g{n, xadj, adj, nullptr, ew};
  return cut_of(g, block);
}

// The multilevel scheme (Sec. 1 Fig. 1, Sec. 3): cluster and contract while
// the graph is larger than max(coarse_min_nodes, 60k) and a contraction
// still removes at least 5% of the nodes; partition the coarsest graph;
// project back level by level (a fine node takes its coarse representative's
// block) and refine each level with LP local search; repair balance at the
// end if the coarsest graph could not be balanced.
int orc_partition(int32_t variant, int64_t n, const int64_t* xadj, const int32_t* adj,
                  const int32_t* nw_in, const int32_t* ew_in, int32_t k, double eps,
                  uint64_t seed, const orc_config* cfg_in, int32_t* block_out,
                  int64_t* cut_out, int64_t* maxbw_out, orc_stats* st) {
  orc_config cfg;
  if (cfg_in) cfg = *cfg_in; else orc_default_config(&cfg);
  if (n < 1 || k < 1 || k > n || !(eps >= 0.0) || cfg.sub_rounds < 1 || cfg.ip_trials < 1)
    return ORC_EINVAL;
  const int64_t m = xadj[n];
  vector<int32_t> nw_unit, ew_unit;
  const int32_t* nw = nw_in;
  const int32_t* ew = ew_in;
  if (!nw) { nw_unit.assign((size_t)n, 1); nw = nw_unit.data(); }
  if (!ew) { ew_unit.assign((size_t)m, 1); ew = ew_unit.data(); }
  int64_t cV = 0;
  int32_t maxc = 0;
  for (int64_t v = 0; v < n; ++v) { cV += nw[v]; maxc = std::max(maxc, nw[v]); }
  int64_t Lmax, U;
  int rc = bounds(cV, maxc, k, eps, cfg.f, &Lmax, &U);
  if (rc != ORC_OK) return rc;
  const int64_t avg = (cV + k - 1) / k;
  const int64_t T = std::max<int64_t>(cfg.coarse_min_nodes, 60 * (int64_t)k);

  G g0{n, xadj, adj, nw, ew};
  vector<OG> coarse;                 // coarse[l-1] is level l
  vector<vector<int32_t>> cmaps;     // cmaps[l]: level l -> level l+1
  vector<int32_t> crounds;
  auto level_graph = [&](size_t l) { return l == 0 ? g0 : coarse[l - 1].view(); };
  while (true) {
    G g = level_graph(coarse.size());
    if (g.n <= T || (int64_t)coarse.size() + 1 >= cfg.max_levels) break;
    vector<int32_t> label((size_t)g.n);
    int32_t r = 0;
    coarsen_clustering(variant, g, U, seed, (int32_t)coarse.size(), k, cfg, label.data(), &r);
    vector<int32_t> cmap;
    OG c;
    rc = contract(g, label.data(), cmap, c);
    if (rc != ORC_OK) return rc;
    crounds.push_back(r);
    if (20 * (g.n - c.n) < g.n) break;
    cmaps.push_back(std::move(cmap));
    coarse.push_back(std::move(c));
  }
  const int32_t q = (int32_t)coarse.size();
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->levels = q + 1;
    for (int32_t l = 0; l <= q && l < 64; ++l) {
      G g = level_graph(l);
      st->level_n[l] = g.n;
      st->level_m[l] = g.xadj[g.n];
    }
    for (size_t l = 0; l < crounds.size() && l < 64; ++l) st->cluster_rounds[l] = crounds[l];
    st->Lmax = Lmax;
    st->U = U;
  }

  vector<int32_t> blk((size_t)level_graph(q).n);
  int64_t ipcut = 0;
  int32_t best = 0;
  initial_partition(variant, level_graph(q), k, Lmax, avg, seed, q, cfg, blk.data(), &ipcut,
                    &best);
  vector<int64_t> W((size_t)k);
  block_weights(level_graph(q), k, blk.data(), W.data());
  for (int32_t l = q - 1; l >= 0; --l) {
    G g = level_graph(l);
    vector<int32_t> fine((size_t)g.n);
    for (int64_t v = 0; v < g.n; ++v) fine[v] = blk[cmaps[l][v]];
    blk.swap(fine);
    int32_t r = 0;
    refine_level(variant, g, k, Lmax, seed, ORC_PH_REFINE, l, cfg, blk.data(), W.data(), &r);
    if (st && l < 64) st->refine_rounds[l] = r;
  }
  int32_t rr = 0;
  rc = repair(g0, k, Lmax, seed, cfg, blk.data(), W.data(), &rr);
  // Iterated V-cycles (Sec. 4 "Iterated Multilevel Algorithms", App. A):
  // coarsen again with clusterings that respect the current partition (cut
  // edges are never contracted), start from that partition on the coarsest
  // graph, refine every level on the way back, repair.  Cycle c uses the key
  // hkey(seed, VCYCLE, c, 0) in place of the seed.
  for (int32_t cyc = 1; cyc < std::max(1, cfg.vcycles) && rc != ORC_EINVAL; ++cyc) {
    const uint64_t sc = hkey(seed, ORC_PH_VCYCLE, (uint64_t)cyc, 0);
    vector<OG> vco;                        // vco[l-1] is level l of this cycle
    vector<vector<int32_t>> vmaps, vblk;   // vblk[l]: the partition on level l
    vblk.push_back(blk);
    auto vgraph = [&](size_t l) {
      G g = l == 0 ? g0 : vco[l - 1].view();
      g.rblk = vblk[l].data();
      return g;
    };
    while (true) {
      G g = vgraph(vco.size());
      if (g.n <= T || (int64_t)vco.size() + 1 >= cfg.max_levels) break;
      vector<int32_t> label((size_t)g.n);
      coarsen_clustering(variant, g, U, sc, (int32_t)vco.size(), k, cfg, label.data(), nullptr);
      vector<int32_t> cmap;
      OG c;
      rc = contract(g, label.data(), cmap, c);
      if (rc != ORC_OK) return rc;
      if (20 * (g.n - c.n) < g.n) break;
      vector<int32_t> cb((size_t)c.n, 0);
      for (int64_t v = 0; v < g.n; ++v) cb[cmap[v]] = vblk.back()[v];
      vmaps.push_back(std::move(cmap));
      vco.push_back(std::move(c));
      vblk.push_back(std::move(cb));
    }
    const int32_t q2 = (int32_t)vco.size();
    vector<int32_t> cur = vblk[q2];
    for (int32_t l = q2; l >= 0; --l) {
      G g = vgraph(l);
      g.rblk = nullptr;
      if (l < q2) {
        vector<int32_t> fine((size_t)g.n);
        for (int64_t v = 0; v < g.n; ++v) fine[v] = cur[vmaps[l][v]];
        cur.swap(fine);
      }
      refine_level(variant, g, k, Lmax, sc, ORC_PH_REFINE, l, cfg, cur.data(), W.data(), nullptr);
    }
    blk.swap(cur);
    rc = repair(g0, k, Lmax, sc, cfg, blk.data(), W.data(), &rr);
  }
  std::copy(blk.begin(), blk.end(), block_out);
  if (cut_out) *cut_out = cut_of(g0, block_out);
  if (maxbw_out) *maxbw_out = max_weight(W.data(), k);
  if (st) { st->ip_best_trial = best; st->ip_cut = ipcut; st->repair_rounds = rr; }
  return rc;
}

}  // extern "C"
