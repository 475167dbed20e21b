// scan.cu -- device-wide exclusive prefix sums (reduce / scan partials /
// scan-and-add, three launches, coalesced tiles) and the node -> slot map.
#include "common.cuh"

namespace sclap {
namespace {

constexpr int SB = 512;     // threads per block
constexpr int SI = 8;       // items per thread
constexpr int TILE = SB * SI;

template <class T>
__device__ T block_excl_scan(T x, T* sh, T* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T inc = x;
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) sh[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T v = lane < (int)(blockDim.x >> 5) ? sh[lane] : T(0);
    T vi = v;
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, vi, o);
      if (lane >= o) vi += y;
    }
    if (lane < (int)(blockDim.x >> 5)) sh[lane] = vi - v;
    if (lane == 31) sh[32] = vi;
  }
  __syncthreads();
  T res = sh[wid] + inc - x;
  *total = sh[32];
  __syncthreads();
  return res;
}

// Input transforms: plain value, or 1 for a non-negative int32 (an occupied
// hash slot), else 0.
struct Plain {
  template <class T>
  __device__ __forceinline__ T operator()(T x) const { return x; }
};
struct Occupied {
  __device__ __forceinline__ int64_t operator()(int32_t x) const { return x >= 0 ? 1 : 0; }
};

template <class Tin, class Tout, class F = Plain>
__global__ void __launch_bounds__(SB) k_reduce(const Tin* __restrict__ in, int64_t n,
                                               Tout* __restrict__ part) {
  __shared__ Tout sh[33];
  const int64_t base = (int64_t)blockIdx.x * TILE;
  Tout s = 0;
#pragma unroll
  for (int j = 0; j < SI; ++j) {
    int64_t i = base + (int64_t)j * SB + threadIdx.x;
    if (i < n) s += (Tout)F()(in[i]);
  }
  Tout tot;
  block_excl_scan<Tout>(s, sh, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

template <class Tout>
__global__ void __launch_bounds__(SB) k_scan_part(Tout* part, int64_t nb, Tout* total_out) {
  __shared__ Tout sh[33];
  Tout carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += SB) {
    int64_t i = b0 + threadIdx.x;
    Tout x = i < nb ? part[i] : Tout(0);
    Tout tot;
    Tout ex = block_excl_scan<Tout>(x, sh, &tot);
    if (i < nb) part[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

template <class Tin, class Tout, class F = Plain>
__global__ void __launch_bounds__(SB) k_scan_add(const Tin* __restrict__ in, int64_t n,
                                                 const Tout* __restrict__ part,
                                                 Tout* __restrict__ out) {
  __shared__ Tout sh[33];
  const int64_t base = (int64_t)blockIdx.x * TILE + (int64_t)threadIdx.x * SI;
  Tout v[SI];
  Tout s = 0;
#pragma unroll
  for (int j = 0; j < SI; ++j) {
    int64_t i = base + j;
    v[j] = i < n ? (Tout)F()(in[i]) : Tout(0);
    s += v[j];
  }
  Tout tot;
  Tout ex = block_excl_scan<Tout>(s, sh, &tot) + part[blockIdx.x];
#pragma unroll
  for (int j = 0; j < SI; ++j) {
    int64_t i = base + j;
    if (i < n) out[i] = ex;
    ex += v[j];
  }
}

template <class Tin, class Tout, class F = Plain>
void scan_excl(const Tin* in, Tout* out, int64_t n, cudaStream_t s) {
  if (n <= 0) {
    SCLAP_CUDA(cudaMemsetAsync(out, 0, sizeof(Tout), s));
    return;
  }
  const int64_t nb = (n + TILE - 1) / TILE;
  DevBuf<Tout> part((size_t)nb, s);
  k_reduce<Tin, Tout, F><<<(unsigned)nb, SB, 0, s>>>(in, n, part.p); SCLAP_NOTE_LAUNCH("k_scan_reduce");
  k_scan_part<Tout><<<1, SB, 0, s>>>(part.p, nb, out + n); SCLAP_NOTE_LAUNCH("k_scan_part");
  k_scan_add<Tin, Tout, F><<<(unsigned)nb, SB, 0, s>>>(in, n, part.p, out); SCLAP_NOTE_LAUNCH("k_scan_add");
  SCLAP_LAUNCH_CHECK();
}

__global__ void k_fill_gid(const int64_t* __restrict__ noff, int32_t nslots,
                           int32_t* __restrict__ gid, int64_t N) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    int32_t lo = 0, hi = nslots - 1;   // last slot with noff[s] <= v
    while (lo < hi) {
      int32_t mid = (lo + hi + 1) >> 1;
      if (noff[mid] <= v) lo = mid; else hi = mid - 1;
    }
    gid[v] = lo;
  }
}

// Largest degree of a level (out[0]), the number of nodes whose degree
// exceeds thr (out[1]), and the table slots those nodes need together
// (out[2]: the sum of hub_table_slots over them).
__global__ void k_degree_stats(const int64_t* __restrict__ row_ptr, int64_t N, int64_t thr,
                               unsigned long long* out) {
  unsigned long long m = 0, c = 0, t = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = row_ptr[v + 1] - row_ptr[v];
    m = (unsigned long long)d > m ? (unsigned long long)d : m;
    if (d > thr) {
      c += 1;
      t += (unsigned long long)hub_table_slots(d);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
    c += __shfl_xor_sync(0xffffffffu, c, o);
    t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (m) atomicMax(&out[0], m);
    if (c) atomicAdd(&out[1], c);
    if (t) atomicAdd(&out[2], t);
  }
}

}  // namespace

void level_degree_stats(const int64_t* row_ptr, int64_t N, int64_t thr, int64_t* out,
                        cudaStream_t s) {
  if (N <= 0) return;
  k_degree_stats<<<grid_for(N, 256, (int64_t)num_sms() * 8), 256, 0, s>>>(
      row_ptr, N, thr, reinterpret_cast<unsigned long long*>(out)); SCLAP_NOTE_LAUNCH("k_degree_stats");
  SCLAP_LAUNCH_CHECK();
}

void scan_excl_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  scan_excl<int32_t, int64_t>(in, out, n, s);
}
void scan_excl_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  scan_excl<int64_t, int64_t>(in, out, n, s);
}
void scan_excl_u8_to_i64(const uint8_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  scan_excl<uint8_t, int64_t>(in, out, n, s);
}
void scan_excl_occupied(const int32_t* keys, int64_t* out, int64_t n, cudaStream_t s) {
  scan_excl<int32_t, int64_t, Occupied>(keys, out, n, s);
}

void fill_gid(const int64_t* noff, int32_t nslots, int32_t* gid, int64_t N, cudaStream_t s) {
  if (N <= 0) return;
  k_fill_gid<<<grid_for(N, 256, (int64_t)num_sms() * 32), 256, 0, s>>>(noff, nslots, gid, N); SCLAP_NOTE_LAUNCH("k_fill_gid");
  SCLAP_LAUNCH_CHECK();
}

}  // namespace sclap
