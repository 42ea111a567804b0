// mlp.cu -- tensor-core GEMM entry point and (below) the learned excitation
// proposal built on it.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/hande.h"
#include "tc_gemm.cuh"

namespace hande {
namespace tc {
namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_mu;
EncodeTiledFn g_encode = nullptr;

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda)
EncodeTiledFn encoder() {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<EncodeTiledFn>(fn);
    else
      cudaGetLastError();
  }
  return g_encode;
}

}  // namespace

// 2D BF16 tensor {inner, outer} with row stride ld (elements), box {64, box_outer},
// 128-byte swizzle, zero fill outside
bool make_map(CUtensorMap* map, const void* ptr, uint64_t inner, uint64_t outer, uint64_t ld, uint32_t box_outer) {
  EncodeTiledFn enc = encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// persistent launch: one CTA per SM (at most one per output tile)
template <int BN, int EPI>
bool launch_shape(const CUtensorMap& ma, const CUtensorMap& mb, const Epilogue& ep, int M, int N, int K,
                  unsigned* err, cudaStream_t s, int dev, const char** why) {
  static bool attr_set[256] = {};
  static int nsm[256] = {};
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!attr_set[dev]) {
      if (cudaFuncSetAttribute(k_gemm_bf16_tn_p<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)PTile<BN>::kSmemBytes) != cudaSuccess ||
          cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        *why = "cannot reserve the GEMM's shared memory";
        return false;
      }
      attr_set[dev] = true;
    }
  }
  const int64_t tiles = (int64_t)((N + BN - 1) / BN) * ((M + kBM - 1) / kBM);
  const unsigned grid = (unsigned)(tiles < nsm[dev] ? tiles : nsm[dev]);
  k_gemm_bf16_tn_p<BN, EPI><<<grid, kPThreads, PTile<BN>::kSmemBytes, s>>>(ma, mb, ep, M, N, K, err);
  if (cudaGetLastError() != cudaSuccess) {
    *why = "GEMM launch failed";
    return false;
  }
  return true;
}

// Validated launch of D = A B^T with the given epilogue (see tc_gemm.cuh);
// 256-column tiles when N > 128; false with a message on bad input
bool launch_gemm_ep(const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb, const Epilogue& ep, int epi,
                    int M, int N, int K, unsigned* err, cudaStream_t s, const char** why) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !err || (epi == EPI_F32 ? !ep.D : (!ep.H || !ep.bias))) {
    *why = "bad GEMM sizes or pointers";
    return false;
  }
  if (lda < K || ldb < K || (lda & 7) || (ldb & 7) || ((uintptr_t)A & 15) || ((uintptr_t)B & 15) ||
      (epi == EPI_F32 ? ep.ldd < N : ep.ldh < N)) {
    *why = "GEMM operands need 16-byte aligned rows (leading dimensions multiples of 8, >= K)";
    return false;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    cudaGetLastError();
    *why = "no current CUDA device";
    return false;
  }
  const int bn = N > 128 ? 256 : 128;
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, (uint64_t)K, (uint64_t)M, (uint64_t)lda, kBM) ||
      !make_map(&mb, B, (uint64_t)K, (uint64_t)N, (uint64_t)ldb, (uint32_t)bn)) {
    *why = "cuTensorMapEncodeTiled failed";
    return false;
  }
  if (epi == EPI_F32)
    return bn == 256 ? launch_shape<256, EPI_F32>(ma, mb, ep, M, N, K, err, s, dev, why)
                     : launch_shape<128, EPI_F32>(ma, mb, ep, M, N, K, err, s, dev, why);
  return bn == 256 ? launch_shape<256, EPI_BF16_BIAS>(ma, mb, ep, M, N, K, err, s, dev, why)
                   : launch_shape<128, EPI_BF16_BIAS>(ma, mb, ep, M, N, K, err, s, dev, why);
}

bool launch_gemm(const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb, float* D, int64_t ldd, int M,
                 int N, int K, unsigned* err, cudaStream_t s, const char** why) {
  Epilogue ep{};
  ep.D = D;
  ep.ldd = ldd;
  return launch_gemm_ep(A, lda, B, ldb, ep, EPI_F32, M, N, K, err, s, why);
}

namespace {
__device__ unsigned g_gemm_err;   // error word of hande_gemm_bf16 calls
}

}  // namespace tc
}  // namespace hande

using namespace hande;

extern "C" hande_status hande_gemm_bf16(const uint16_t* d_a, int64_t lda, const uint16_t* d_b, int64_t ldb,
                                        float* d_d, int64_t ldd, int m, int n, int k, unsigned* d_status,
                                        void* cuda_stream) {
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (m < 1 || n < 1 || k < 1 || lda < k || ldb < k || ldd < n || (lda & 7) || (ldb & 7) || !d_a || !d_b || !d_d ||
      ((uintptr_t)d_a & 15) || ((uintptr_t)d_b & 15))
    return HANDE_ERR_INVALID;
  const char* why = "";
  if (d_status) {   // asynchronous: a wait that gives up is ORed into the caller's word
    return tc::launch_gemm(d_a, lda, d_b, ldb, d_d, ldd, m, n, k, d_status, s, &why) ? HANDE_OK : HANDE_ERR_CUDA;
  }
  unsigned* err = nullptr;
  if (cudaGetSymbolAddress((void**)&err, tc::g_gemm_err) != cudaSuccess) {
    cudaGetLastError();
    return HANDE_ERR_CUDA;
  }
  const unsigned zero = 0;
  if (cudaMemcpyAsync(err, &zero, sizeof zero, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return HANDE_ERR_CUDA;
  }
  if (!tc::launch_gemm(d_a, lda, d_b, ldb, d_d, ldd, m, n, k, err, s, &why)) return HANDE_ERR_CUDA;
  unsigned e = 0;
  if (cudaMemcpyAsync(&e, err, sizeof e, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return HANDE_ERR_CUDA;
  }
  return e ? HANDE_ERR_TIMEOUT : HANDE_OK;
}
