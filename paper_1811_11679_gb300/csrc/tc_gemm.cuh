// tc_gemm.cuh -- BF16 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
//   D[m][n] = sum_k A[m][k] B[n][k]        (A: M x K, B: N x K, both K-major
//                                           BF16 row-major; D: FP32)
//
// Output tiles of 128 x BN (BN = 128, or 256 when N > 128, so that A is read
// once for N <= 256), walked by one persistent CTA per SM (see
// k_gemm_bf16_tn_p below).  The K dimension is taken in chunks of 64 elements
// (128 bytes): a TMA tile load brings the A and B chunk of a stage into shared
// memory in the 128-byte-swizzled K-major layout the tensor core reads, four
// stages deep; one thread issues the MMAs (four 128 x BN x 16 tcgen05.mma per
// chunk, FP32 accumulators in tensor memory) and commits each stage to an
// mbarrier that frees it for the next TMA load.  Four warps read the
// accumulator rows they own (tcgen05.ld, 32 lanes x 32 columns at a time) and
// store them as FP32, or as BF16 after adding a bias and a ReLU (with a
// transposed copy if asked: the learned proposal's hidden layers and their
// backward operands).  Rows, columns and K beyond the matrix are zero-filled by
// the TMA and masked in the store, so any M, N, K >= 1 work (leading
// dimensions: multiples of 8 elements).
//
// Every wait is bounded: a wait that gives up sets bit ERR_MMA_TIMEOUT of *err,
// the kernel skips its remaining work, waits (bounded) for its own loads and
// MMAs and frees its tensor memory.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace hande {
namespace tc {

constexpr int kBM = 128;        // tile rows (MMA M)
constexpr int kBK = 64;         // K per stage: 64 BF16 = 128 bytes = one swizzle row
constexpr int kMmaK = 16;       // K of one tcgen05.mma kind::f16
constexpr int kStages = 4;
constexpr uint32_t kTileABytes = kBM * kBK * 2;
constexpr unsigned ERR_MMA_TIMEOUT = 1u;
// tile columns BN (MMA N, 128 or 256): the bytes of a B chunk
template <int BN>
struct Tile {
  static constexpr uint32_t kTileBBytes = BN * kBK * 2;
};
// epilogues: FP32 D, or BF16 act(D + bias) (ReLU or none) with an optional
// transposed BF16 copy
enum { EPI_F32 = 0, EPI_BF16_BIAS = 1 };
struct Epilogue {
  float* D;                 // EPI_F32: D[row * ldd + col]
  int64_t ldd;
  uint16_t* H;              // EPI_BF16_BIAS: H[row * ldh + col] = bf16(act(D + bias[col]))
  int64_t ldh;
  uint16_t* HT;             //   and, if not null, HT[col * ldt + row]
  int64_t ldt;
  const float* bias;
  int relu;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// ------------------------------------------------------------------ mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait for the phase with the given parity to complete: gives up after
// about one second of the global timer
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 15) == 15 && global_ns() - t0 > 1000000000ull) return false;
  }
}

// ------------------------------------------------------------------ TMA
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// ------------------------------------------------------------------ tcgen05
// shared-memory matrix descriptor: K-major operand in the 128-byte swizzle
// layout written by a TMA load with CU_TENSOR_MAP_SWIZZLE_128B (rows of 128
// bytes, groups of 8 rows 1024 bytes apart); the stage base is 1024-aligned
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);   // bits  0-13: start address / 16
                                             // bits 16-29: leading byte offset (unused: the
                                             // 32-byte K step stays inside one swizzle row)
  d |= (uint64_t)(1024 >> 4) << 32;          // bits 32-45: stride byte offset / 16 (8-row groups)
  d |= (uint64_t)1 << 46;                    // bits 46-47: descriptor version 1
  d |= (uint64_t)2 << 61;                    // bits 61-63: 128-byte swizzle
  return d;
}
// instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D, M x N
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int m, int n) {
  return (1u << 4)                         // D format: F32
         | (1u << 7)                       // A format: BF16
         | (1u << 10)                      // B format: BF16
         | ((uint32_t)(n >> 3) << 17)      // N / 8
         | ((uint32_t)(m >> 4) << 24);     // M / 16
}
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on the mbarrier once every MMA issued so far by this thread completed
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// whole warp: allocate ncols tensor-memory columns, address written to *slot
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// whole warp: 32 consecutive 32-bit columns of the warp's 32 lanes (lane l gets row l)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Epilogue of 32 accumulator columns c0 .. c0 + 31 of tile column n0 for the
// calling lane's row (r: the lane's 32 FP32 values from tcgen05.ld): FP32
// store, or BF16 act(D + bias) with the optional transposed copy.
template <int EPI>
__device__ __forceinline__ void epi_store(const Epilogue& ep, const uint32_t (&r)[32], int row, int n0, int c0,
                                          int M, int N) {
  const int nc = N - (n0 + c0) < 32 ? N - (n0 + c0) : 32;
  if (EPI == EPI_F32) {
    if (row < M) {
      float* out = ep.D + (int64_t)row * ep.ldd + n0 + c0;
      if (nc == 32 && (((uintptr_t)out & 15) == 0)) {
#pragma unroll
        for (int i = 0; i < 32; i += 4)
          *reinterpret_cast<float4*>(out + i) = make_float4(__uint_as_float(r[i]), __uint_as_float(r[i + 1]),
                                                            __uint_as_float(r[i + 2]), __uint_as_float(r[i + 3]));
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (i < nc) out[i] = __uint_as_float(r[i]);
      }
    }
  } else {
    uint32_t h[16];
#pragma unroll
    for (int i = 0; i < 32; i += 2) {
      float v0 = __uint_as_float(r[i]) + (i < nc ? __ldg(&ep.bias[n0 + c0 + i]) : 0.0f);
      float v1 = __uint_as_float(r[i + 1]) + (i + 1 < nc ? __ldg(&ep.bias[n0 + c0 + i + 1]) : 0.0f);
      if (ep.relu) {
        v0 = v0 > 0.0f ? v0 : 0.0f;
        v1 = v1 > 0.0f ? v1 : 0.0f;
      }
      h[i / 2] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v0)) |
                 ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v1)) << 16);
    }
    if (row < M) {
      uint16_t* out = ep.H + (int64_t)row * ep.ldh + n0 + c0;
      if (nc == 32 && (((uintptr_t)out & 15) == 0)) {
#pragma unroll
        for (int i = 0; i < 16; i += 4)
          *reinterpret_cast<uint4*>(out + 2 * i) = make_uint4(h[i], h[i + 1], h[i + 2], h[i + 3]);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (i < nc) out[i] = (uint16_t)(h[i / 2] >> (16 * (i & 1)));
      }
      if (ep.HT) {
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (i < nc) ep.HT[(int64_t)(n0 + c0 + i) * ep.ldt + row] = (uint16_t)(h[i / 2] >> (16 * (i & 1)));
      }
    }
  }
}

// ------------------------------------------------------------------ persistent form
// One CTA per SM walks the output tiles t = blockIdx.x, + gridDim.x, ... with
// six warps: warp 4 (one thread) issues the TMA loads of every tile's K chunks
// into the stage ring, warp 5 (one thread) issues the MMAs into one of two
// tensor-memory accumulators (2 x BN columns) and owns the tensor memory, and
// warps 0-3 (accumulator lanes 32w .. 32w + 31) run the epilogue of the other
// accumulator, so one tile's stores overlap the next tile's loads and MMAs.
// Barriers: full/empty per stage (TMA bytes / MMA commit), acc_full per
// accumulator (MMA commit) and acc_empty (one arrival per epilogue warp).
// Every wait is bounded; a wait that gives up sets ERR_MMA_TIMEOUT and a
// shared flag that stops all roles, which then drain their own loads and MMAs
// (bounded) before the tensor memory is freed.
constexpr int kPThreads = 192;
// tensor-memory columns (two FP32 accumulators of BN columns: 512 at BN = 256)
// and dynamic shared memory (1024-byte aligned stages + barriers)
template <int BN>
struct PTile {
  static constexpr uint32_t kTmemCols = 2 * BN;
  static constexpr size_t kSmemBytes = 1024 + (size_t)kStages * (kTileABytes + Tile<BN>::kTileBBytes) + 256;
};

template <int BN, int EPI>
__global__ void __launch_bounds__(kPThreads, 1)
    k_gemm_bf16_tn_p(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const Epilogue ep, int M, int N, int K, unsigned* err) {
  constexpr uint32_t kTileBBytes = Tile<BN>::kTileBBytes;
  constexpr uint32_t kTmemCols = PTile<BN>::kTmemCols;
  extern __shared__ __align__(16) unsigned char tcp_smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tcp_smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = base;
  unsigned char* sB = base + (size_t)kStages * kTileABytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + (size_t)kStages * kTileBBytes);
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;      // [2]
  uint64_t* acc_empty = acc_full + 2;        // [2]
  uint64_t* done = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ volatile int s_fail;

  const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
  const int nk = (K + kBK - 1) / kBK;
  const int tn_count = (N + BN - 1) / BN, tm_count = (M + kBM - 1) / kBM;
  const int ntiles = tn_count * tm_count;

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 4);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 5) tmem_alloc(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  auto fail = [&]() {
    s_fail = 1;
    atomicOr(err, ERR_MMA_TIMEOUT);
  };

  if (warp == 4) {
    if (lane == 0) {   // producer
      int64_t fill = 0;   // chunk loads issued over all tiles
      int64_t landed = 0;
      for (int t = (int)blockIdx.x; t < ntiles && !s_fail; t += (int)gridDim.x) {
        const int m0 = (t / tn_count) * kBM, n0 = (t % tn_count) * BN;
        for (int kc = 0; kc < nk && !s_fail; ++kc, ++fill) {
          const int st = (int)(fill % kStages);
          const uint32_t ph = (uint32_t)((fill / kStages) & 1);
          if (!mbar_wait(&empty[st], ph ^ 1u)) {
            fail();
            break;
          }
          mbar_expect_tx(&full[st], kTileABytes + kTileBBytes);
          tma_load_2d(sA + (size_t)st * kTileABytes, &tmA, &full[st], kc * kBK, m0);
          tma_load_2d(sB + (size_t)st * kTileBBytes, &tmB, &full[st], kc * kBK, n0);
        }
      }
      if (s_fail) {   // let this thread's loads in flight land before the CTA exits (bounded)
        for (landed = fill - kStages > 0 ? fill - kStages : 0; landed < fill; ++landed)
          mbar_wait(&full[landed % kStages], (uint32_t)((landed / kStages) & 1));
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {   // MMA issuer
      const uint32_t idesc = idesc_bf16_f32(kBM, BN);
      int64_t use = 0;   // chunk consumptions over all tiles
      int i = 0;         // tiles of this CTA
      for (int t = (int)blockIdx.x; t < ntiles && !s_fail; t += (int)gridDim.x, ++i) {
        const int a = i & 1;
        if (!mbar_wait(&acc_empty[a], (uint32_t)(((i >> 1) & 1) ^ 1))) {
          fail();
          break;
        }
        tc_fence_after();
        const uint32_t dcol = tmem + (uint32_t)(a * BN);
        for (int kc = 0; kc < nk; ++kc, ++use) {
          const int st = (int)(use % kStages);
          if (!mbar_wait(&full[st], (uint32_t)((use / kStages) & 1))) {
            fail();
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sA + (size_t)st * kTileABytes);
          const uint32_t b0 = smem_u32(sB + (size_t)st * kTileBBytes);
#pragma unroll
          for (int j = 0; j < kBK / kMmaK; ++j)
            tc_mma(dcol, sw128_kmajor_desc(a0 + 32u * j), sw128_kmajor_desc(b0 + 32u * j), idesc,
                   (kc > 0 || j > 0) ? 1u : 0u);
          tc_commit(&empty[st]);
        }
        if (s_fail) break;
        tc_commit(&acc_full[a]);
      }
      tc_commit(done);   // completes once every MMA issued above has completed
      if (!mbar_wait(done, 0)) fail();
    }
  } else {   // epilogue warps 0-3
    const int lrow = warp * 32 + lane;
    int i = 0;
    for (int t = (int)blockIdx.x; t < ntiles && !s_fail; t += (int)gridDim.x, ++i) {
      const int m0 = (t / tn_count) * kBM, n0 = (t % tn_count) * BN;
      const int a = i & 1;
      const bool ok = mbar_wait(&acc_full[a], (uint32_t)((i >> 1) & 1));
      if (!__all_sync(0xffffffffu, ok)) {   // warp-uniform (the accumulator reads are warp-collective)
        if (lane == 0) fail();
        break;
      }
      tc_fence_after();
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        if (n0 + c0 >= N) break;
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(a * BN + c0), r);
        epi_store<EPI>(ep, r, m0 + lrow, n0, c0, M, N);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[a]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) tmem_free(tmem, kTmemCols);
}

}  // namespace tc
}  // namespace hande
