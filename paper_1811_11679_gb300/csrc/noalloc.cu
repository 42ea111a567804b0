// noalloc.cu -- hande_estimate_noalloc: the projected-energy sums of a walker
// list without any device allocation.
//
// Some callers may not allocate device memory at the moment they need this
// reduction: applications that reserve their whole device-memory budget at
// start-up and give plug-in code none of it (an allocation there either fails
// or pushes the process over its budget), code whose memory pool owns every
// free byte of the device (a foreign cudaMalloc then runs out of memory even
// though the pool has room), and latency-critical loops that must not call
// cudaMalloc/cudaFree because those calls can synchronise the whole device and
// stall the other streams.  For them the per-block partial sums live in one
// file-scope device array of fixed size instead of context scratch memory.
//
// The array is shared by every call in the process on a given device and
// keeps the previous call's contents; each call overwrites exactly the slots
// it reads, so nothing has to be cleared first.  Calls that overlap on the GPU
// (in flight at the same time on different streams) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "engine.h"

namespace hande {
namespace {

constexpr int kNoAllocChunk = 4096;       // determinants reduced by one block
constexpr int kNoAllocMaxBlocks = 4096;   // slots in the scratch array
constexpr int kNoAllocThreads = 256;

struct Partial {
  int64_t nw;
  int64_t n0;
  unsigned long long num_lo;
  long long num_hi;
};

// file-scope scratch: 4096 x 32 bytes = 128 KiB on every device that loads the library
static __device__ __align__(256) Partial g_noalloc_partials[kNoAllocMaxBlocks];

// per-device address of the scratch array, looked up once (host code cannot
// use the symbol itself as a device address)
std::mutex g_mutex;
void* g_scratch[256] = {};

template <int W, int SYS>
__global__ void __launch_bounds__(kNoAllocThreads) k_est_partials(SysDev sys, Key<W> d0, const uint64_t* keys,
                                                                  const int64_t* pops, int64_t n, Partial* part) {
  __shared__ int64_t sh64[32];
  __shared__ I128 sh128[32];
  const int64_t beg = (int64_t)blockIdx.x * kNoAllocChunk;
  const int64_t end = beg + kNoAllocChunk < n ? beg + kNoAllocChunk : n;
  int64_t nw = 0, n0 = 0;
  I128 num{0, 0};
  for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
    Key<W> k;
#pragma unroll
    for (int j = 0; j < W; ++j) k.w[j] = keys[i * W + j];
    const int64_t p = pops[i];
    nw += iabs64(p);
    if (key_eq<W>(k, d0)) {
      n0 += p;
    } else if (p != 0 && key_popc_xor<W>(k, d0) <= 4) {
      i128_add(num, fixed_term(p, h_elem<W, SYS>(sys, k, d0)));
    }
  }
  int64_t a = block_sum<int64_t>(nw, sh64);
  int64_t b = block_sum<int64_t>(n0, sh64);
  I128 c = block_sum_i128(num, sh128);
  if (threadIdx.x == 0) part[blockIdx.x] = Partial{a, b, c.lo, (long long)c.hi};
}

__global__ void k_est_final(const Partial* part, int nblocks, int64_t* out) {
  __shared__ int64_t sh64[32];
  __shared__ I128 sh128[32];
  int64_t nw = 0, n0 = 0;
  I128 num{0, 0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    nw += part[b].nw;
    n0 += part[b].n0;
    i128_add(num, I128{part[b].num_lo, (int64_t)part[b].num_hi});
  }
  int64_t a = block_sum<int64_t>(nw, sh64);
  int64_t z = block_sum<int64_t>(n0, sh64);
  I128 c = block_sum_i128(num, sh128);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = z;
    out[2] = (int64_t)c.lo;
    out[3] = c.hi;
  }
}

template <int W, int SYS>
void launch(const Engine& E, const uint64_t* keys, const int64_t* pops, int64_t n, int64_t* out, Partial* scratch) {
  Key<W> d0;
  for (int j = 0; j < W; ++j) d0.w[j] = E.P.d0[j];
  const int nblocks = (int)((n + kNoAllocChunk - 1) / kNoAllocChunk);
  if (nblocks > 0)
    k_est_partials<W, SYS><<<nblocks, kNoAllocThreads, 0, E.stream>>>(E.P.sys, d0, keys, pops, n, scratch);
  k_est_final<<<1, kNoAllocThreads, 0, E.stream>>>(scratch, nblocks, out);
}

template <int W>
void dispatch(const Engine& E, const uint64_t* keys, const int64_t* pops, int64_t n, int64_t* out, Partial* scratch) {
  if (E.kind == SYS_HUBBARD) launch<W, SYS_HUBBARD>(E, keys, pops, n, out, scratch);
  else if (E.kind == SYS_UEG) launch<W, SYS_UEG>(E, keys, pops, n, out, scratch);
  else launch<W, SYS_MOLECULE>(E, keys, pops, n, out, scratch);
}

}  // namespace
}  // namespace hande

using namespace hande;

extern "C" hande_status hande_estimate_noalloc(hande_ctx* ctx, const uint64_t* d_keys, const int64_t* d_pops,
                                               int64_t n, int64_t* d_out) {
  if (!ctx || !d_out || n < 0 || (n > 0 && (!d_keys || !d_pops))) return HANDE_ERR_INVALID;
  Engine& E = ctx->E;
  if (E.failed) return HANDE_ERR_STATE;
  if (n > (int64_t)kNoAllocChunk * kNoAllocMaxBlocks) {
    E.err = "hande_estimate_noalloc: more than 16777216 determinants (4096 blocks x 4096) do not fit "
            "its fixed scratch array";
    return HANDE_ERR_CAPACITY;
  }
  // The context's kernels and stream belong to the device it was created on;
  // that device is made current for the set-up and the launches, and the
  // caller's current device is restored afterwards.
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    cudaGetLastError();
    E.err = "hande_estimate_noalloc: no current CUDA device";
    return HANDE_ERR_CUDA;
  }
  const int dev = E.device;
  if (dev < 0 || dev >= 256) {
    E.err = "hande_estimate_noalloc: device index out of range";
    return HANDE_ERR_INVALID;
  }
  struct DeviceGuard {
    int prev;
    bool switched;
    ~DeviceGuard() {
      if (switched) cudaSetDevice(prev);
    }
  } guard{prev, prev != dev};
  if (guard.switched && cudaSetDevice(dev) != cudaSuccess) {
    cudaGetLastError();
    guard.switched = false;
    E.err = "hande_estimate_noalloc: cannot make the context's device current";
    return HANDE_ERR_CUDA;
  }
  Partial* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch[dev]) {
      // host code sees only a host-side stand-in for the array: its device
      // address is looked up here, once per device, with that device current
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        E.err = std::string("hande_estimate_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
        return HANDE_ERR_CUDA;
      }
      g_scratch[dev] = ptr;
    }
    scratch = static_cast<Partial*>(g_scratch[dev]);
  }
  if (E.W == 1) dispatch<1>(E, d_keys, d_pops, n, d_out, scratch);
  else if (E.W == 2) dispatch<2>(E, d_keys, d_pops, n, d_out, scratch);
  else dispatch<8>(E, d_keys, d_pops, n, d_out, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    E.err = std::string("hande_estimate_noalloc: launch failed: ") + cudaGetErrorString(e);
    return HANDE_ERR_CUDA;
  }
  return HANDE_OK;
}
