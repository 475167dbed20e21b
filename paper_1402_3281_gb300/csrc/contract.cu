// contract.cu -- cluster contraction (Sec. 3.1) for every slot of a level.
//
// Each cluster becomes one coarse node (id = rank of its label, contiguous
// per slot); its weight is the sum of its members; two coarse nodes are
// adjacent iff their clusters are, with the summed weight of the fine edges
// between them.  GPU plan: rank the labels by a scan; stream the fine arcs in
// node order (warp per 32 nodes, arcs flattened across lanes) once to count
// each coarse node's inter-cluster arcs, size one open-addressing region per
// coarse node from that count (next_pow2 of it: the distinct coarse
// neighbours never outnumber the arcs, and are usually far fewer), stream the arcs again inserting (coarse
// neighbour, weight) with one 64-bit CAS or atomic add each (a claim also
// records the slot's owner and counts its degree), scan the degrees into row
// offsets, and place every occupied slot in its owner's row.  The order of a
// row's arcs is not fixed, which no later step depends on; all sums are
// integer, hence deterministic.
#include <algorithm>

#include "common.cuh"

namespace sclap {
namespace {

__global__ void k_mark(const int32_t* __restrict__ label, int64_t N, int32_t* __restrict__ flag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x)
    flag[label[v]] = 1;
}

__global__ void k_gather(const int64_t* __restrict__ src, const int64_t* __restrict__ idx, int n,
                         int64_t* __restrict__ dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}

struct CArgs {
  const int64_t* row_ptr;
  const int32_t* col;
  const int32_t* ew;
  const int32_t* nw;
  const int32_t* gid;
  const int32_t* label;
  const int64_t* cid;
  const int64_t* delta;
  const uint8_t* keep;
  int32_t* cmap;
  int32_t* cnw;
  int32_t* inter;          // inter-cluster arcs per coarse node
  const int64_t* tbase;    // table region of each coarse node
  unsigned long long* tslot;   // (coarse neighbour << 32) | summed weight; ~0 = empty
  int32_t* cdeg;           // distinct coarse neighbours per coarse node (slots claimed)
  int32_t* towner;         // coarse node owning each claimed slot
  int32_t* err;
  // pass of the table build: only sources with coarse id in [c_lo, c_hi)
  // insert, into the table regions of that range, which start at toff
  int32_t c_lo, c_hi;
  int64_t toff;
};

__global__ void k_map(CArgs a, int64_t N) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = slot_at(a.gid, v);
    if (!a.keep[s]) { a.cmap[v] = -1; continue; }
    const int32_t c = (int32_t)(a.cid[a.label[v]] + a.delta[s]);
    a.cmap[v] = c;
    atomicAdd(&a.cnw[c], wat(a.nw, v));
  }
}

// Visits every arc (v, u) of the level with cmap[v] >= 0, 32 source nodes per
// warp, the arcs of those nodes spread over the lanes; calls f(cv, cu, w) on
// every lane (cu = -1 on lanes without an inter-cluster arc) so the warp can
// cooperate.
template <class F>
__device__ __forceinline__ void for_inter_arcs(const CArgs& a, int64_t N, F f) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = w0 * 32; base < N; base += nwarps * 32) {
    const int64_t v = base + lane;
    int64_t rs = 0, d = 0;
    int32_t cv = -1;
    if (v < N) {
      cv = a.cmap[v];
      if (cv >= a.c_lo && cv < a.c_hi) {
        rs = a.row_ptr[v];
        d = a.row_ptr[v + 1] - rs;
      }
    }
    long long incl = d;
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const long long excl = incl - d;
    const long long total = __shfl_sync(0xffffffffu, incl, 31);
    for (long long x0 = 0; x0 < total; x0 += 32) {
      const long long x = x0 + lane;
      int L = 0;
      for (int step = 16; step > 0; step >>= 1) {
        long long y = __shfl_sync(0xffffffffu, incl, L + step - 1);
        if (y <= x) L += step;
      }
      const long long rsL = __shfl_sync(0xffffffffu, (long long)rs, L);
      const long long exL = __shfl_sync(0xffffffffu, excl, L);
      const int32_t cvL = __shfl_sync(0xffffffffu, cv, L);
      int32_t cu = -1, w = 0;
      if (x < total) {
        const int64_t e = rsL + (x - exL);
        cu = a.cmap[a.col[e]];
        if (cu == cvL) cu = -1;
        else w = wat(a.ew, e);
      }
      f(cvL, cu, w);
    }
  }
}

// Inter-cluster arcs per coarse node.  The lanes' arcs are in source order,
// so lanes with the same coarse source form runs of consecutive lanes; two
// ballots give each run's count and its last lane adds it (runs with equal
// sources that are not adjacent simply add separately).
__global__ void __launch_bounds__(256) k_count_inter(CArgs a, int64_t N) {
  const int lane = threadIdx.x & 31;
  for_inter_arcs(a, N, [&](int32_t cv, int32_t cu, int32_t) {
    const unsigned inter = __ballot_sync(0xffffffffu, cu >= 0);
    const int32_t prev = __shfl_up_sync(0xffffffffu, cv, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != cv);
    const bool last = lane == 31 || ((heads >> (lane + 1)) & 1u);
    if (last) {
      const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);   // lanes 0..lane
      const int first = 31 - __clz(heads & upto);                               // run start
      const int c = __popc(inter & upto & ~((1u << first) - 1u));
      if (c) atomicAdd(&a.inter[cv], c);
    }
  });
}

__global__ void k_table_caps(const int32_t* __restrict__ inter, int64_t Nc, int64_t* __restrict__ cap) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < Nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = inter[c];
    cap[c] = x > 0 ? ((int64_t)1 << ceil_log2((int64_t)x)) : 0;
  }
}

// A slot packs (coarse neighbour, summed weight) in one 64-bit word: the
// first arc claims an empty slot with one CAS carrying its weight, later arcs
// add to the low half with one atomicAdd.  A coarse edge weight must fit in
// int32, so a sum reaching 2^31 is reported (and cannot carry into the key).
__global__ void __launch_bounds__(256) k_insert(CArgs a, int64_t N) {
  for_inter_arcs(a, N, [&](int32_t cv, int32_t cu, int32_t w) {
    if (cu < 0) return;
    const int64_t sum = w;
    const int64_t base = a.tbase[cv] - a.toff;
    const int logcap = ceil_log2(a.tbase[cv + 1] - a.tbase[cv]);
    const uint32_t mask = (1u << logcap) - 1;
    uint32_t sl = table_slot(cu, logcap);
    const unsigned long long mine = ((unsigned long long)(uint32_t)cu << 32) | (uint64_t)sum;
    for (uint32_t p = 0; p <= mask; ++p) {
      unsigned long long* slot = &a.tslot[base + sl];
      unsigned long long cur = *slot;
      if (cur == ~0ull) {
        cur = atomicCAS(slot, ~0ull, mine);
        if (cur == ~0ull) {            // claimed: one more coarse arc of cv
          a.towner[base + sl] = cv;
          atomicAdd(&a.cdeg[cv], 1);
          return;
        }
      }
      if ((uint32_t)(cur >> 32) == (uint32_t)cu) {
        const unsigned long long old = atomicAdd(slot, (unsigned long long)sum);
        if ((old & 0xffffffffull) + (unsigned long long)sum > (unsigned long long)INT32_MAX)
          atomicOr(a.err, DERR_W_OVERFLOW);
        return;
      }
      sl = (sl + 1) & mask;
    }
    atomicOr(a.err, DERR_HASH_FULL);
  });
}

// Coarse rows: one thread per table slot; an occupied slot goes to its
// owner's row (offsets from a scan of the claimed-slot counts) at a position
// taken from a per-row counter.  The order of a row's arcs is therefore not
// fixed, as the slot order already was not (concurrent claims in one region
// race); nothing computed from a coarse graph depends on that order.
__global__ void k_emit(const unsigned long long* __restrict__ tslot,
                       const int32_t* __restrict__ towner, const int64_t* __restrict__ crow,
                       int32_t* __restrict__ fill, int64_t T, int32_t* __restrict__ ccol,
                       int32_t* __restrict__ cew) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < T;
       j += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long x = tslot[j];
    if (x == ~0ull) continue;
    const int32_t c = towner[j];
    const int64_t p = crow[c] + atomicAdd(&fill[c], 1);
    ccol[p] = (int32_t)(x >> 32);
    cew[p] = (int32_t)(x & 0xffffffffull);
  }
}

// row_ptr[c_lo + j] = base + part[j] for j in [0, n]: the row offsets of
// one pass's coarse nodes, placed after the rows of the earlier passes.
__global__ void k_rows_from_part(const int64_t* __restrict__ part, int64_t n, int64_t base,
                                 int64_t* __restrict__ row_ptr) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= n;
       j += (int64_t)gridDim.x * blockDim.x)
    row_ptr[j] = base + part[j];
}

// Overlay (ensemble clusterings): the pair (O[v], C[v]) keys an open-
// addressing table whose entry keeps the smallest node id with that pair.
// Labels are node ids < 2^31, so a key never equals the empty marker ~0.
__device__ __forceinline__ uint64_t pair_key(int32_t o, int32_t c) {
  return ((uint64_t)(uint32_t)o << 32) | (uint32_t)c;
}

__global__ void k_overlay_insert(const int32_t* __restrict__ gid, const int32_t* __restrict__ part,
                                 const int32_t* __restrict__ O, const int32_t* __restrict__ C,
                                 int64_t N, unsigned long long* keys, int32_t* rep, int logcap,
                                 int32_t* err) {
  const uint64_t mask = ((uint64_t)1 << logcap) - 1;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (!part[slot_at(gid, v)]) continue;
    const unsigned long long key = pair_key(O[v], C[v]);
    uint64_t s = mix64(key) & mask;
    bool placed = false;
    for (uint64_t p = 0; p <= mask; ++p) {
      unsigned long long cur = keys[s];
      if (cur == ~0ull) cur = atomicCAS(&keys[s], ~0ull, key);
      if (cur == ~0ull || cur == key) {
        atomicMin(&rep[s], (int32_t)v);
        placed = true;
        break;
      }
      s = (s + 1) & mask;
    }
    if (!placed) atomicOr(err, DERR_HASH_FULL);
  }
}

__global__ void k_overlay_apply(const int32_t* __restrict__ gid, const int32_t* __restrict__ part,
                                int32_t* O, const int32_t* __restrict__ C, int64_t N,
                                const unsigned long long* __restrict__ keys,
                                const int32_t* __restrict__ rep, int logcap) {
  const uint64_t mask = ((uint64_t)1 << logcap) - 1;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (!part[slot_at(gid, v)]) continue;
    const unsigned long long key = pair_key(O[v], C[v]);
    uint64_t s = mix64(key) & mask;
    for (uint64_t p = 0; p <= mask; ++p) {
      const unsigned long long cur = keys[s];
      if (cur == key) { O[v] = rep[s]; break; }
      if (cur == ~0ull) break;          // cannot happen after the insert pass
      s = (s + 1) & mask;
    }
  }
}

}  // namespace

void contract_rank(const LevelView& lv, const std::vector<int64_t>& noff, const int32_t* label,
                   ContractWork& w, std::vector<int64_t>& nc_slot, cudaStream_t s) {
  const int64_t N = lv.N;
  const int ns = (int)noff.size() - 1;
  w.flag.alloc(N, s);
  w.flag.zero();
  w.cid.alloc(N + 1, s);
  const int sms = num_sms();
  if (N > 0) { k_mark<<<grid_for(N, 256, (int64_t)sms * 16), 256, 0, s>>>(label, N, w.flag.p); SCLAP_NOTE_LAUNCH("k_mark"); }
  scan_excl_i32_to_i64(w.flag.p, w.cid.p, N, s);
  DevBuf<int64_t> idx(ns + 1, s), got(ns + 1, s);
  idx.upload(noff);
  k_gather<<<grid_for(ns + 1, 128, 64), 128, 0, s>>>(w.cid.p, idx.p, ns + 1, got.p); SCLAP_NOTE_LAUNCH("k_gather");
  SCLAP_LAUNCH_CHECK();
  w.cid_at.assign(ns + 1, 0);
  SCLAP_CUDA(cudaMemcpyAsync(w.cid_at.data(), got.p, (ns + 1) * sizeof(int64_t),
                             cudaMemcpyDeviceToHost, s));
  stream_sync(s);
  nc_slot.assign(ns, 0);
  for (int i = 0; i < ns; ++i) nc_slot[i] = w.cid_at[i + 1] - w.cid_at[i];
}

void contract_build(const LevelView& lv, const std::vector<int64_t>& noff, const int32_t* label,
                    const ContractWork& w, const std::vector<uint8_t>& keep, int32_t* cmap,
                    CoarseLevel& out, int32_t* d_err, cudaStream_t s) {
  const int64_t N = lv.N;
  const int ns = (int)noff.size() - 1;
  const int sms = num_sms();
  std::vector<int64_t> cno(ns + 1, 0), delta(ns, 0);
  for (int i = 0; i < ns; ++i) {
    const int64_t nc = keep[i] ? w.cid_at[i + 1] - w.cid_at[i] : 0;
    cno[i + 1] = cno[i] + nc;
    delta[i] = cno[i] - w.cid_at[i];
  }
  const int64_t Nc = cno[ns];
  DevBuf<int64_t> d_delta(ns, s);
  d_delta.upload(delta);
  DevBuf<uint8_t> d_keep(ns, s);
  d_keep.upload(keep);

  out.N = Nc;
  out.noff = cno;
  out.noff_d.alloc(ns + 1, s);
  out.noff_d.upload(cno);
  out.nw.alloc(std::max<int64_t>(Nc, 1), s);
  out.nw.zero();
  DevBuf<int32_t> inter(std::max<int64_t>(Nc, 1), s);
  DevBuf<int64_t> cap(std::max<int64_t>(Nc, 1), s), tbase(Nc + 1, s);
  inter.zero();

  CArgs a{};
  a.row_ptr = lv.row_ptr; a.col = lv.col; a.ew = lv.ew; a.nw = lv.nw; a.gid = lv.gid;
  a.label = label; a.cid = w.cid.p; a.delta = d_delta.p; a.keep = d_keep.p; a.cmap = cmap;
  a.cnw = out.nw.p; a.inter = inter.p; a.tbase = tbase.p; a.err = d_err;
  a.c_lo = 0; a.c_hi = INT32_MAX; a.toff = 0;

  const unsigned ng = grid_for(N, 256, (int64_t)sms * 16);
  const unsigned wg = grid_for(N, 256, (int64_t)sms * 16);   // 8 warps x 32 nodes per block
  if (N > 0) {
    k_map<<<ng, 256, 0, s>>>(a, N); SCLAP_NOTE_LAUNCH("k_map");
    k_count_inter<<<wg, 256, 0, s>>>(a, N); SCLAP_NOTE_LAUNCH("k_count_inter");
  }
  if (Nc > 0) {
    k_table_caps<<<grid_for(Nc, 256, (int64_t)sms * 16), 256, 0, s>>>(inter.p, Nc, cap.p); SCLAP_NOTE_LAUNCH("k_table_caps");
  }
  scan_excl_i64(cap.p, tbase.p, Nc, s);
  int64_t T = 0;
  SCLAP_CUDA(cudaMemcpyAsync(&T, tbase.p + Nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  stream_sync(s);
  // the inter-arc counts have served (table sizes); the array now counts
  // claimed slots, i.e. the coarse degrees
  a.cdeg = inter.p;
  SCLAP_CUDA(cudaMemsetAsync(inter.p, 0, (size_t)std::max<int64_t>(Nc, 1) * sizeof(int32_t), s));
  out.row_ptr.alloc(Nc + 1, s);
  const int64_t Tcap = table_pass_slots();
  if (T <= Tcap) {
    // one pass: the whole table at once
    DevBuf<unsigned long long> tslot(std::max<int64_t>(T, 1), s);
    DevBuf<int32_t> towner(std::max<int64_t>(T, 1), s);
    tslot.fill_bytes(0xff);
    a.tslot = tslot.p;
    a.towner = towner.p;
    if (N > 0 && T > 0) { k_insert<<<wg, 256, 0, s>>>(a, N); SCLAP_NOTE_LAUNCH("k_insert"); }
    scan_excl_i32_to_i64(inter.p, out.row_ptr.p, Nc, s);
    int64_t Mc = 0;
    SCLAP_CUDA(cudaMemcpyAsync(&Mc, out.row_ptr.p + Nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    stream_sync(s);
    out.M = Mc;
    out.col.alloc(std::max<int64_t>(Mc, 1), s);
    out.ew.alloc(std::max<int64_t>(Mc, 1), s);
    if (Nc > 0 && T > 0) {
      SCLAP_CUDA(cudaMemsetAsync(inter.p, 0, (size_t)Nc * sizeof(int32_t), s));   // row fill
      k_emit<<<grid_for(T, 256, (int64_t)sms * 32), 256, 0, s>>>(tslot.p, towner.p, out.row_ptr.p,
                                                                 inter.p, T, out.col.p, out.ew.p); SCLAP_NOTE_LAUNCH("k_emit");
    }
  } else {
    // Passes over ranges of coarse nodes whose table regions fit in Tcap
    // slots (a region larger than that gets a pass of its own).  Each pass
    // streams every fine node but inserts only the arcs of sources in its
    // range.  Sweep 1 counts the coarse degrees, which give the row offsets
    // and the exact size of the coarse arrays; sweep 2 inserts again and
    // emits every pass's rows in place.  Identical result to one pass.
    std::vector<int64_t> htb(Nc + 1);
    SCLAP_CUDA(cudaMemcpyAsync(htb.data(), tbase.p, (Nc + 1) * sizeof(int64_t),
                               cudaMemcpyDeviceToHost, s));
    stream_sync(s);
    std::vector<int32_t> cut_at{0};
    while (cut_at.back() < Nc) {
      const int64_t lo = cut_at.back();
      int64_t hi = std::upper_bound(htb.begin() + lo + 1, htb.end(), htb[lo] + Tcap) -
                   htb.begin() - 1;
      if (hi <= lo) hi = lo + 1;
      cut_at.push_back((int32_t)hi);
    }
    int64_t Tmax = 1;
    for (size_t q = 0; q + 1 < cut_at.size(); ++q)
      Tmax = std::max<int64_t>(Tmax, htb[cut_at[q + 1]] - htb[cut_at[q]]);
    DevBuf<unsigned long long> tslot(Tmax, s);
    DevBuf<int32_t> towner(Tmax, s), claims(std::max<int64_t>(Nc, 1), s);
    a.tslot = tslot.p;
    a.towner = towner.p;
    auto pass = [&](size_t q) {
      a.c_lo = cut_at[q];
      a.c_hi = cut_at[q + 1];
      a.toff = htb[a.c_lo];
      SCLAP_CUDA(cudaMemsetAsync(tslot.p, 0xff, (size_t)(htb[a.c_hi] - a.toff) * 8, s));
      if (N > 0) { k_insert<<<wg, 256, 0, s>>>(a, N); SCLAP_NOTE_LAUNCH("k_insert"); }
      return htb[a.c_hi] - a.toff;
    };
    for (size_t q = 0; q + 1 < cut_at.size(); ++q) pass(q);            // sweep 1: degrees
    scan_excl_i32_to_i64(inter.p, out.row_ptr.p, Nc, s);
    int64_t Mc = 0;
    SCLAP_CUDA(cudaMemcpyAsync(&Mc, out.row_ptr.p + Nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    stream_sync(s);
    out.M = Mc;
    out.col.alloc(std::max<int64_t>(Mc, 1), s);
    out.ew.alloc(std::max<int64_t>(Mc, 1), s);
    a.cdeg = claims.p;                   // sweep 2 counts claims apart from the row fill
    SCLAP_CUDA(cudaMemsetAsync(inter.p, 0, (size_t)Nc * sizeof(int32_t), s));   // row fill
    for (size_t q = 0; q + 1 < cut_at.size(); ++q) {                    // sweep 2: emit
      const int64_t Tp = pass(q);
      k_emit<<<grid_for(Tp, 256, (int64_t)sms * 32), 256, 0, s>>>(tslot.p, towner.p,
                                                                  out.row_ptr.p, inter.p, Tp,
                                                                  out.col.p, out.ew.p); SCLAP_NOTE_LAUNCH("k_emit");
    }
  }
  SCLAP_LAUNCH_CHECK();
  out.gid.alloc(std::max<int64_t>(Nc, 1), s);
  fill_gid(out.noff_d.p, ns, out.gid.p, Nc, s);
  DevBuf<int64_t> ga(ns + 1, s);
  k_gather<<<grid_for(ns + 1, 128, 64), 128, 0, s>>>(out.row_ptr.p, out.noff_d.p, ns + 1, ga.p); SCLAP_NOTE_LAUNCH("k_gather");
  SCLAP_LAUNCH_CHECK();
  out.aoff.assign(ns + 1, 0);
  SCLAP_CUDA(cudaMemcpyAsync(out.aoff.data(), ga.p, (ns + 1) * sizeof(int64_t),
                             cudaMemcpyDeviceToHost, s));
  stream_sync(s);
}

void overlay_labels(const LevelView& lv, const int32_t* part, int32_t* O, const int32_t* C,
                    int32_t* err, cudaStream_t s) {
  if (lv.N == 0) return;
  const int logcap = ceil_log2(std::max<int64_t>(2 * lv.N, 64));
  const int64_t cap = (int64_t)1 << logcap;
  DevBuf<unsigned long long> keys(cap, s);
  DevBuf<int32_t> rep(cap, s);
  keys.fill_bytes(0xff);
  rep.fill_bytes(0x7f);                    // 0x7f7f7f7f: above every node id
  const unsigned g = grid_for(lv.N, 256, (int64_t)num_sms() * 16);
  k_overlay_insert<<<g, 256, 0, s>>>(lv.gid, part, O, C, lv.N, keys.p, rep.p, logcap, err); SCLAP_NOTE_LAUNCH("k_overlay_insert");
  k_overlay_apply<<<g, 256, 0, s>>>(lv.gid, part, O, C, lv.N, keys.p, rep.p, logcap); SCLAP_NOTE_LAUNCH("k_overlay_apply");
  SCLAP_LAUNCH_CHECK();
}

}  // namespace sclap
