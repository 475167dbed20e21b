// noalloc.cu -- the cut and the block weights of a partition computed with
// working memory taken from one fixed array in device global memory instead
// of the allocator.
//
// Meant for callers that cannot allocate device memory at the moment they
// ask for the measure: a host that has handed (nearly) all device memory to
// another allocator and keeps it, or a latency-sensitive loop that must not
// enter the CUDA allocator, where an allocation can block or fail.  The
// price is a hard bound on k and one shared array per device, so calls that
// overlap in time (two host threads, or two streams in flight at once) race
// on it and must be serialised by the caller.
#include "common.cuh"

namespace sclap {
void record_last_error(const char* msg);   // driver.cu

namespace {

// Layout (64-bit words): [0] twice the cut, [1] violation flags,
// [2 .. 2+k) block weights.  Only the first 2+k words are used by a call,
// and the call clears exactly those before its kernels run.
constexpr int64_t kStaticMaxK = SCLAP_CUT_STATIC_MAX_K;
static __device__ __align__(256) unsigned long long g_cut_scratch[2 + kStaticMaxK];

enum : unsigned long long {
  SF_ROWPTR = 1,   // row_ptr[0] != 0 or row_ptr decreasing
  SF_COL = 2,      // neighbour id outside [0, n) or self-loop
  SF_EDGE_W = 4,   // edge weight <= 0
  SF_NODE_W = 8,   // node weight <= 0
  SF_LABEL = 16,   // block id outside [0, k)
};

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
unsigned long long* g_scratch_ptr[kMaxDevices] = {};

// Address of the scratch array on the current device, looked up once per
// device with that device current.
unsigned long long* scratch_for_current_device() {
  int dev = 0;
  SCLAP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw Error(SCLAP_EINVAL, "device ordinal beyond 63");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_cut_scratch);
    if (e != cudaSuccess || !p)
      throw Error(SCLAP_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") +
                                   cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<unsigned long long*>(p);
  }
  return g_scratch_ptr[dev];
}

// Pass 1, one thread per node: the CSR row bounds, node weights and block ids
// are checked, and c(V_b) is summed per block, first in shared memory (k
// words of dynamic shared memory) and then once per CTA and block into the
// scratch.
__global__ void __launch_bounds__(256) k_static_nodes(const int64_t* __restrict__ row_ptr,
                                                      const int32_t* __restrict__ nw,
                                                      const int32_t* __restrict__ block,
                                                      int64_t n, int32_t k,
                                                      unsigned long long* __restrict__ scr) {
  extern __shared__ unsigned long long sh_w[];
  for (int b = threadIdx.x; b < k; b += blockDim.x) sh_w[b] = 0;
  __syncthreads();
  unsigned long long flags = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rs = row_ptr[v], re = row_ptr[v + 1];
    if ((v == 0 && rs != 0) || re < rs) flags |= SF_ROWPTR;
    const int32_t c = nw ? nw[v] : 1;
    if (c <= 0) flags |= SF_NODE_W;
    const int32_t b = block[v];
    if (b < 0 || b >= k) flags |= SF_LABEL;
    else if (c > 0) atomicAdd(&sh_w[b], (unsigned long long)c);
  }
  if (flags) atomicOr(&scr[1], flags);
  __syncthreads();
  for (int b = threadIdx.x; b < k; b += blockDim.x)
    if (sh_w[b]) atomicAdd(&scr[2 + b], sh_w[b]);
}

// Pass 2, 32 nodes per warp with their arcs spread over the lanes: twice the
// cut, sum over arcs (u, v) with block[u] != block[v] of w(u, v).  Runs only
// when pass 1 found the rows and labels sound, so every arc index stays in
// [0, row_ptr[n]) and every block lookup in [0, n).
__global__ void __launch_bounds__(256) k_static_cut(const int64_t* __restrict__ row_ptr,
                                                    const int32_t* __restrict__ col,
                                                    const int32_t* __restrict__ ew,
                                                    const int32_t* __restrict__ block,
                                                    int64_t n,
                                                    unsigned long long* __restrict__ scr) {
  if (*(volatile unsigned long long*)&scr[1] & (SF_ROWPTR | SF_LABEL)) return;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long flags = 0, sum = 0;
  for (int64_t base = w0 * 32; base < n; base += nwarps * 32) {
    const int64_t v = base + lane;
    int64_t rs = 0, d = 0;
    int32_t bv = 0;
    if (v < n) {
      rs = row_ptr[v];
      d = row_ptr[v + 1] - rs;
      bv = block[v];
    }
    long long incl = d;
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const long long excl = incl - d;
    const long long total = __shfl_sync(0xffffffffu, incl, 31);
    for (long long x0 = 0; x0 < total; x0 += 32) {
      const long long x = x0 + lane;
      // owner lane L: the first lane whose inclusive prefix exceeds x
      int L = 0;
      for (int step = 16; step > 0; step >>= 1) {
        const long long y = __shfl_sync(0xffffffffu, incl, L + step - 1);
        if (y <= x) L += step;
      }
      const long long rsL = __shfl_sync(0xffffffffu, (long long)rs, L);
      const long long exL = __shfl_sync(0xffffffffu, excl, L);
      const int32_t bL = __shfl_sync(0xffffffffu, bv, L);
      if (x < total) {
        const int64_t e = rsL + (x - exL);
        const int32_t u = col[e];
        const int32_t w = ew ? ew[e] : 1;
        if (w <= 0) flags |= SF_EDGE_W;
        if (u < 0 || u >= n || (int64_t)u == base + L) {
          flags |= SF_COL;
        } else if (block[u] != bL && w > 0) {
          sum += (unsigned long long)w;
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    flags |= __shfl_xor_sync(0xffffffffu, flags, o);
  }
  if (lane == 0) {
    if (sum) atomicAdd(&scr[0], sum);
    if (flags) atomicOr(&scr[1], flags);
  }
}

}  // namespace
}  // namespace sclap

extern "C" int sclap_cut_static(int64_t n, const int64_t* row_ptr, const int32_t* col,
                                const int32_t* node_w, const int32_t* edge_w,
                                const int32_t* block, int32_t k, int64_t* cut_out,
                                int64_t* block_w_out, void* stream) {
  using namespace sclap;
  try {
    if (n < 1 || n >= ((int64_t)1 << 31)) throw Error(SCLAP_EINVAL, "n must be in [1, 2^31)");
    if (!row_ptr || !block) throw Error(SCLAP_EINVAL, "NULL array");
    if (k < 1 || (int64_t)k > n) throw Error(SCLAP_EINVAL, "k must be in [1, n]");
    if ((int64_t)k > kStaticMaxK)
      throw Error(SCLAP_EINVAL, "k above SCLAP_CUT_STATIC_MAX_K (4096); use sclap_cut");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* scr = scratch_for_current_device();
    int64_t m = 0;
    SCLAP_CUDA(cudaMemcpyAsync(&m, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SCLAP_CUDA(cudaStreamSynchronize(s));
    if (m < 0) throw Error(SCLAP_ECSR, "row_ptr[n] < 0");
    if (m > 0 && !col) throw Error(SCLAP_EINVAL, "NULL col with arcs present");
    SCLAP_CUDA(cudaMemsetAsync(scr, 0, (size_t)(2 + k) * sizeof(unsigned long long), s));
    const unsigned g = grid_for(n, 256, (int64_t)num_sms() * 4);
    k_static_nodes<<<g, 256, (size_t)k * sizeof(unsigned long long), s>>>(row_ptr, node_w, block,
                                                                          n, k, scr);
    SCLAP_NOTE_LAUNCH("k_static_nodes");
    SCLAP_LAUNCH_CHECK();
    if (m > 0) {
      k_static_cut<<<grid_for(n, 256, (int64_t)num_sms() * 16), 256, 0, s>>>(row_ptr, col, edge_w,
                                                                             block, n, scr);
      SCLAP_NOTE_LAUNCH("k_static_cut");
      SCLAP_LAUNCH_CHECK();
    }
    unsigned long long hdr[2] = {0, 0};
    SCLAP_CUDA(cudaMemcpyAsync(hdr, scr, sizeof(hdr), cudaMemcpyDeviceToHost, s));
    if (block_w_out)
      SCLAP_CUDA(cudaMemcpyAsync(block_w_out, scr + 2, (size_t)k * sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, s));
    SCLAP_CUDA(cudaStreamSynchronize(s));
    if (hdr[1] & SF_LABEL) throw Error(SCLAP_EINVAL, "block id outside [0, k)");
    if (hdr[1]) throw Error(SCLAP_ECSR, "malformed CSR input");
    if (cut_out) *cut_out = (int64_t)(hdr[0] / 2);
    record_last_error("");
    return SCLAP_OK;
  } catch (const Error& e) {
    record_last_error(e.what());
    return e.code;
  } catch (...) {
    record_last_error("unknown exception");
    return SCLAP_EINTERNAL;
  }
}
