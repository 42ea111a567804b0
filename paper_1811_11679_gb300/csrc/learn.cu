// learn.cu -- the learned excitation proposal for the uniform electron gas.
//
// The paper's UEG generator draws the particle orbital of a double excitation
// uniformly (Sec. 2.1, Sec. 4.2); this proposal draws it from a table of
// integer weights per row r = (I, J, same spin) of the occupied pair, so p_gen
// stays exact (see system.cuh).  The table is the output of a small MLP
//   x(r) = [one-hot I, one-hot J, same]  ->  relu(W1 x + b1)  ->  relu(W2 . + b2)
//   ->  z = W3 . + b3,   p(A | r) = masked softmax over the drawable A,
//   q_r(A) = max(1, floor(p(A | r) 2^24)) on drawable A, 0 elsewhere,
// whose dense layers run on the tensor cores (tc_gemm.cuh: BF16 operands, FP32
// accumulation).  It is trained online on the spawning attempts the run draws:
// the spawning kernel records (row, A, w = |H| / p_draw) for a strided subset
// of attempts, and every `period` iterations one Adam step minimises
//   L = - sum_n c_n log p(A_n | r_n),   c_n = w_n / sum_m w_m,
// a self-normalised estimate of the cross-entropy to the distribution
// proportional to |H| (the heat-bath choice), after which the table is
// recomputed from the network.  The estimator stays unbiased whatever the
// network outputs, because the spawn weight uses the table's exact p_gen.
//
// BF16 rounding points (the oracle's FP64 MLP mirrors them): the weights, the
// hidden activations (rounded in the GEMM epilogue after bias and ReLU), and
// the backward signals of the logits and hidden layers; accumulation, biases,
// logits, softmax and Adam are FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "engine.h"
#include "host_util.h"
#include "tc_gemm.cuh"

namespace hande {
namespace tc {
// the tensor-core GEMM D = A B^T (tc_gemm.cuh, launched from mlp.cu): FP32
// output, or BF16 act(D + bias) with an optional transposed copy
bool launch_gemm(const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb, float* D, int64_t ldd, int M, int N,
                 int K, unsigned* err, cudaStream_t s, const char** why);
bool launch_gemm_ep(const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb, const Epilogue& ep, int epi,
                    int M, int N, int K, unsigned* err, cudaStream_t s, const char** why);
}

struct Learner {
  int M = 0, din = 0, kin = 0, H = 0, R = 0, Rp = 0, S = 0, M8 = 0, rows_cap = 0;
  int period = 0;
  float lr = 1e-3f, beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  int64_t nparam = 0;
  size_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
  float *param = nullptr, *mom1 = nullptr, *mom2 = nullptr, *grad = nullptr;
  int64_t* tstep = nullptr;
  uint16_t *W1b = nullptr, *W2b = nullptr, *W2bT = nullptr, *W3b = nullptr, *W3bT = nullptr;
  uint16_t *X = nullptr, *XT = nullptr, *Xtab = nullptr;
  uint16_t *H1 = nullptr, *H2 = nullptr, *H1T = nullptr, *H2T = nullptr;
  uint16_t *G3 = nullptr, *G3T = nullptr, *dZ2 = nullptr, *dZ2T = nullptr, *dZ1 = nullptr, *dZ1T = nullptr;
  float *Z3 = nullptr, *dH = nullptr;
  float* wsum = nullptr;
  double* loss = nullptr;
  unsigned* err = nullptr;
  // rows/targets/weights of a batch given through the C ABI (tests)
  int32_t *in_rows = nullptr, *in_tgt = nullptr;
  float* in_w = nullptr;
  float* probs = nullptr;
  cudaGraphExec_t graph = nullptr;
};

namespace {

constexpr int kLt = 256;

__device__ __forceinline__ uint16_t f2bf(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf2f(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

// features x(r) of rows[0 .. S) (rows with w == 0, or beyond count, are zero):
// X [S][kin] and, if XT, its transpose [kin][S]
__global__ void k_lr_features(const int32_t* rows, const float* w, int count, int S, int M, int kin, uint16_t* X,
                              uint16_t* XT) {
  const int64_t total = (int64_t)S * kin;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(i / kin), k = (int)(i % kin);
    uint16_t v = 0;
    if (n < count && (!w || w[n] > 0.0f)) {
      const int r = rows[n], same = r & 1, IJ = r >> 1, I = IJ / M, J = IJ % M;
      if (k == I || k == M + J || (k == 2 * M && same)) v = 0x3F80;   // BF16 1.0
    }
    X[i] = v;
    if (XT) XT[(int64_t)k * S + n] = v;
  }
}

// dZ = (h > 0) ? dH : 0 in BF16 [n][Hd] and transposed [Hd][ldT], h the layer's
// BF16 ReLU output (positive exactly where the pre-activation is)
__global__ void k_lr_relu_back(const float* dH, const uint16_t* Hact, int n, int Hd, uint16_t* dZ, uint16_t* dZT,
                               int ldT) {
  const int64_t total = (int64_t)n * Hd;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / Hd), j = (int)(i % Hd);
    const uint16_t g = (Hact[i] != 0 && !(Hact[i] & 0x8000)) ? f2bf(dH[i]) : (uint16_t)0;
    dZ[i] = g;
    dZT[(int64_t)j * ldT + r] = g;
  }
}

// *wsum = sum of the sample weights (one block, fixed order)
__global__ void k_lr_wsum(const float* w, int n, float* wsum) {
  __shared__ float sh[kLt];
  float s = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += w[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *wsum = sh[0];
}

// masked softmax of one logits row held by a warp: p[A] for A = lane + 32 k
template <int PER>
__device__ __forceinline__ void warp_softmax(const float* z, const float* b3, const uint8_t* mrow, int M, float (&p)[PER],
                                             bool (&ok)[PER]) {
  const int lane = (int)(threadIdx.x & 31);
  float mx = -INFINITY;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int A = lane + 32 * k;
    ok[k] = A < M && mrow[A];
    p[k] = ok[k] ? z[A] + b3[A] : -INFINITY;
    mx = fmaxf(mx, p[k]);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  float sum = 0.0f;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    p[k] = ok[k] ? expf(p[k] - mx) : 0.0f;
    sum += p[k];
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  const float inv = sum > 0.0f ? 1.0f / sum : 0.0f;
#pragma unroll
  for (int k = 0; k < PER; ++k) p[k] *= inv;
}

constexpr int kMaxPer = 8;   // M <= 256 particle orbitals

// loss and logits gradient, one warp per sample n: G = c_n (p - onehot(A_n)) on
// drawable A (BF16 [S][M8], zero padding; transposed [M][S])
__global__ void k_lr_softmax_grad(const float* Z3, const float* b3, const int32_t* rows, const int32_t* tgt,
                                  const float* w, const float* wsum, int S, int M, int M8, const uint8_t* mask,
                                  uint16_t* G3, uint16_t* G3T, double* loss) {
  const int n = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = (int)(threadIdx.x & 31);
  if (n >= S) return;
  const float c = (w[n] > 0.0f && *wsum > 0.0f) ? w[n] / *wsum : 0.0f;
  float p[kMaxPer];
  bool ok[kMaxPer];
  const int r = rows[n];
  warp_softmax<kMaxPer>(Z3 + (int64_t)n * M, b3, mask + (int64_t)r * M, M, p, ok);
  const int t = tgt[n];
  float lt = 0.0f;
#pragma unroll
  for (int k = 0; k < kMaxPer; ++k) {
    const int A = lane + 32 * k;
    if (A >= M8) continue;
    float g = 0.0f;
    if (A < M && ok[k] && c > 0.0f) {
      g = c * (p[k] - (A == t ? 1.0f : 0.0f));
      if (A == t) lt = -c * logf(p[k]);
    }
    const uint16_t gb = f2bf(g);
    G3[(int64_t)n * M8 + A] = gb;
    if (A < M) G3T[(int64_t)A * S + n] = gb;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) lt += __shfl_xor_sync(0xffffffffu, lt, o);
  if (lane == 0 && lt != 0.0f) atomicAdd(loss, (double)lt);
}

// out[j] = sum_i G[i][j] (BF16 values, FP32 sum in row order), j < ncol
__global__ void k_lr_colsum(const uint16_t* G, int n, int ncol, int ld, float* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncol) return;
  float s = 0.0f;
  for (int i = 0; i < n; ++i) s += bf2f(G[(int64_t)i * ld + j]);
  out[j] = s;
}

__global__ void k_lr_count_step(int64_t* t) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *t += 1;
}

// Adam (Kingma and Ba) with bias correction at step *t
__global__ void k_lr_adam(float* p, float* m, float* v, const float* g, int64_t np, float lr, float b1, float b2,
                          float eps, const int64_t* t) {
  const float tt = (float)*t;
  const float c1 = 1.0f / (1.0f - powf(b1, tt)), c2 = 1.0f / (1.0f - powf(b2, tt));
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// BF16 copies of the weights: W1 [H][kin] (zero-padded from din), W2 [H][H]
// and W2^T, W3 [M][H] and W3^T [H][M8] (zero-padded)
__global__ void k_lr_weights(const float* p, int H, int din, int kin, int M, int M8, size_t oW1, size_t oW2, size_t oW3,
                             uint16_t* W1b, uint16_t* W2b, uint16_t* W2bT, uint16_t* W3b, uint16_t* W3bT) {
  const int64_t n1 = (int64_t)H * kin, n2 = (int64_t)H * H, n3 = (int64_t)H * M8;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n1 + n2 + n3;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n1) {
      const int o = (int)(i / kin), k = (int)(i % kin);
      W1b[i] = k < din ? f2bf(p[oW1 + (size_t)o * din + k]) : (uint16_t)0;
    } else if (i < n1 + n2) {
      const int64_t e = i - n1;
      const int o = (int)(e / H), k = (int)(e % H);
      const uint16_t v = f2bf(p[oW2 + (size_t)e]);
      W2b[e] = v;
      W2bT[(int64_t)k * H + o] = v;
    } else {
      const int64_t e = i - n1 - n2;
      const int h = (int)(e / M8), A = (int)(e % M8);
      const uint16_t v = A < M ? f2bf(p[oW3 + (size_t)A * H + h]) : (uint16_t)0;
      W3bT[e] = v;
      if (A < M) W3b[(int64_t)A * H + h] = v;
    }
  }
}

// proposal table from the logits of every row, one warp per row: masked
// softmax, q = max(1, floor(p 2^24)) on drawable A, cumulative sums
__global__ void k_lr_table(const float* Z3, const float* b3, int R, int M, const uint8_t* mask, uint32_t* cum) {
  const int r = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = (int)(threadIdx.x & 31);
  if (r >= R) return;
  float p[kMaxPer];
  bool ok[kMaxPer];
  warp_softmax<kMaxPer>(Z3 + (int64_t)r * M, b3, mask + (int64_t)r * M, M, p, ok);
  // lane l holds A = l + 32 k; cumulative sums in A order: k-major passes
  uint32_t carry = 0;
#pragma unroll
  for (int k = 0; k < kMaxPer; ++k) {
    const int A = lane + 32 * k;
    uint32_t q = 0;
    if (ok[k]) {
      const float f = floorf(p[k] * 16777216.0f);
      q = f < 1.0f ? 1u : (uint32_t)f;
    }
    uint32_t x = q;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (A < M) cum[(int64_t)r * M + A] = carry + x;
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
}

// masked softmax probabilities of given rows (tests), one warp per row
__global__ void k_lr_probs(const float* Z3, const float* b3, const int32_t* rows, int n, int M, const uint8_t* mask,
                           float* out) {
  const int i = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = (int)(threadIdx.x & 31);
  if (i >= n) return;
  float p[kMaxPer];
  bool ok[kMaxPer];
  warp_softmax<kMaxPer>(Z3 + (int64_t)i * M, b3, mask + (int64_t)rows[i] * M, M, p, ok);
#pragma unroll
  for (int k = 0; k < kMaxPer; ++k) {
    const int A = lane + 32 * k;
    if (A < M) out[(int64_t)i * M + A] = p[k];
  }
}

__global__ void k_lr_fold_err(const unsigned* lerr, DevState* st) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && *lerr) atomicOr(&st->error, ERR_TIMEOUT);
}

inline int grid_for(int64_t n) {
  int64_t g = (n + kLt - 1) / kLt;
  if (g > 4 * 152) g = 4 * 152;
  return g < 1 ? 1 : (int)g;
}

void gemm(Learner& L, const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb, float* D, int64_t ldd, int m,
          int n, int k, cudaStream_t s) {
  const char* why = "";
  if (!tc::launch_gemm(A, lda, B, ldb, D, ldd, m, n, k, L.err, s, &why)) throw Fail{HANDE_ERR_CUDA, why};
}

// forward of `nrows` feature rows X [nrows][kin] to the logits Z3 [nrows][M]
// (activations H1, H2; transposes only for a training batch)
void gemm_act(Learner& L, const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb, const float* bias,
              uint16_t* Hout, uint16_t* HT, int m, int n, int k, cudaStream_t s) {
  tc::Epilogue ep{};
  ep.H = Hout;
  ep.ldh = n;
  ep.HT = HT;
  ep.ldt = L.S;
  ep.bias = bias;
  ep.relu = 1;
  const char* why = "";
  if (!tc::launch_gemm_ep(A, lda, B, ldb, ep, tc::EPI_BF16_BIAS, m, n, k, L.err, s, &why))
    throw Fail{HANDE_ERR_CUDA, why};
}

// hidden layers: BF16 relu(x W^T + b) straight from the GEMM epilogue (and
// their transposes for a training batch); logits in FP32
void forward(Learner& L, const uint16_t* X, int nrows, bool train, cudaStream_t s) {
  const int H = L.H;
  gemm_act(L, X, L.kin, L.W1b, L.kin, L.param + L.ob1, L.H1, train ? L.H1T : nullptr, nrows, H, L.kin, s);
  gemm_act(L, L.H1, H, L.W2b, H, L.param + L.ob2, L.H2, train ? L.H2T : nullptr, nrows, H, H, s);
  gemm(L, L.H2, H, L.W3b, H, L.Z3, L.M, nrows, L.M, H, s);
}

// gradients of the loss of the batch (rows, tgt, w) [S] into L.grad and L.loss
void backward(Engine& E, Learner& L, const int32_t* rows, const int32_t* tgt, const float* w, cudaStream_t s) {
  const int H = L.H, S = L.S, M = L.M;
  k_lr_wsum<<<1, kLt, 0, s>>>(w, S, L.wsum);
  k_lr_features<<<grid_for((int64_t)S * L.kin), kLt, 0, s>>>(rows, w, S, S, M, L.kin, L.X, L.XT);
  forward(L, L.X, S, true, s);
  CK(cudaMemsetAsync(L.loss, 0, sizeof(double), s));
  k_lr_softmax_grad<<<(S * 32 + kLt - 1) / kLt, kLt, 0, s>>>(L.Z3, L.param + L.ob3, rows, tgt, w, L.wsum, S, M, L.M8,
                                                              E.pmask_dev, L.G3, L.G3T, L.loss);
  float* g = L.grad;
  gemm(L, L.G3T, S, L.H2T, S, g + L.oW3, H, M, H, S, s);                 // dW3 = G3^T H2
  k_lr_colsum<<<(M + kLt - 1) / kLt, kLt, 0, s>>>(L.G3, S, M, L.M8, g + L.ob3);
  gemm(L, L.G3, L.M8, L.W3bT, L.M8, L.dH, H, S, H, M, s);                // dH2 = G3 W3
  k_lr_relu_back<<<grid_for((int64_t)S * H), kLt, 0, s>>>(L.dH, L.H2, S, H, L.dZ2, L.dZ2T, S);
  k_lr_colsum<<<(H + kLt - 1) / kLt, kLt, 0, s>>>(L.dZ2, S, H, H, g + L.ob2);
  gemm(L, L.dZ2T, S, L.H1T, S, g + L.oW2, H, H, H, S, s);                // dW2 = dZ2^T H1
  gemm(L, L.dZ2, H, L.W2bT, H, L.dH, H, S, H, H, s);                     // dH1 = dZ2 W2
  k_lr_relu_back<<<grid_for((int64_t)S * H), kLt, 0, s>>>(L.dH, L.H1, S, H, L.dZ1, L.dZ1T, S);
  k_lr_colsum<<<(H + kLt - 1) / kLt, kLt, 0, s>>>(L.dZ1, S, H, H, g + L.ob1);
  gemm(L, L.dZ1T, S, L.XT, S, g + L.oW1, L.din, H, L.din, S, s);         // dW1 = dZ1^T X
}

void to_bf16(Learner& L, cudaStream_t s) {
  const int64_t n = (int64_t)L.H * L.kin + (int64_t)L.H * L.H + (int64_t)L.H * L.M8;
  k_lr_weights<<<grid_for(n), kLt, 0, s>>>(L.param, L.H, L.din, L.kin, L.M, L.M8, L.oW1, L.oW2, L.oW3, L.W1b, L.W2b,
                                           L.W2bT, L.W3b, L.W3bT);
}

void refresh_table(Engine& E, Learner& L, cudaStream_t s) {
  forward(L, L.Xtab, L.Rp, false, s);
  k_lr_table<<<(L.R * 32 + kLt - 1) / kLt, kLt, 0, s>>>(L.Z3, L.param + L.ob3, L.R, L.M, E.pmask_dev, E.ptab);
}

// one training step on the samples the spawning kernel recorded, then the table
void enqueue_step(Engine& E, Learner& L, cudaStream_t s) {
  backward(E, L, E.P.smp_row, E.P.smp_A, E.P.smp_w, s);
  k_lr_count_step<<<1, 32, 0, s>>>(L.tstep);
  k_lr_adam<<<grid_for(L.nparam), kLt, 0, s>>>(L.param, L.mom1, L.mom2, L.grad, L.nparam, L.lr, L.beta1, L.beta2,
                                                L.eps, L.tstep);
  to_bf16(L, s);
  refresh_table(E, L, s);
  CK(cudaMemsetAsync(E.P.smp_w, 0, sizeof(float) * (size_t)L.S, s));
  k_lr_fold_err<<<1, 32, 0, s>>>(L.err, E.P.st);
}

uint64_t splitmix(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

// ------------------------------------------------------------------ host entry points
// drawable mask of the proposal table and its initial weights (1 on every
// drawable particle orbital), built when excit_gen = 1 is chosen
void proposal_init(Engine& E, const int4* kvec, const int16_t* klookup, int nmax, int side) {
  const int M = E.P.sys.norb;
  const size_t R = (size_t)M * M * 2;
  E.pmask.assign(R * M, 0);
  std::vector<uint32_t> cum(R * M, 0);
  for (int I = 0; I < M; ++I)
    for (int J = 0; J < M; ++J)
      for (int same = 0; same < 2; ++same) {
        const size_t r = ((size_t)I * M + J) * 2 + same;
        uint32_t c = 0;
        for (int A = 0; A < M; ++A) {
          const int bx = kvec[I].x + kvec[J].x - kvec[A].x, by = kvec[I].y + kvec[J].y - kvec[A].y,
                    bz = kvec[I].z + kvec[J].z - kvec[A].z;
          int B = -1;
          if (bx >= -nmax && bx <= nmax && by >= -nmax && by <= nmax && bz >= -nmax && bz <= nmax)
            B = klookup[((size_t)(bx + nmax) * side + (by + nmax)) * side + (bz + nmax)];
          const bool ok = B >= 0 && !(same && B == A);
          E.pmask[r * M + A] = ok ? 1 : 0;
          c += ok ? 1u : 0u;
          cum[r * M + A] = c;
        }
      }
  E.ptab = dalloc<uint32_t>(E, R * M);
  E.pmask_dev = dalloc<uint8_t>(E, R * M);
  CK(cudaMemcpyAsync(E.ptab, cum.data(), cum.size() * 4, cudaMemcpyHostToDevice, E.stream));
  CK(cudaMemcpyAsync(E.pmask_dev, E.pmask.data(), E.pmask.size(), cudaMemcpyHostToDevice, E.stream));
  CK(cudaStreamSynchronize(E.stream));
  E.P.sys.ptab_cum = E.ptab;
}

void proposal_set(Engine& E, const uint32_t* q) {
  const int M = E.P.sys.norb;
  const size_t R = (size_t)M * M * 2;
  std::vector<uint32_t> cum(R * M);
  for (size_t r = 0; r < R; ++r) {
    uint32_t c = 0;
    for (int A = 0; A < M; ++A) {
      const uint32_t v = q[r * M + A];
      const bool ok = E.pmask[r * M + A] != 0;
      if (ok ? (v < 1 || v > (1u << 24)) : v != 0)
        throw Fail{HANDE_ERR_INVALID, "proposal weights must be in [1, 2^24] exactly on the drawable orbitals"};
      c += v;
      cum[r * M + A] = c;
    }
  }
  CK(cudaMemcpyAsync(E.ptab, cum.data(), cum.size() * 4, cudaMemcpyHostToDevice, E.stream));
  CK(cudaStreamSynchronize(E.stream));
}

void proposal_get(Engine& E, uint32_t* q) {
  const int M = E.P.sys.norb;
  const size_t R = (size_t)M * M * 2;
  std::vector<uint32_t> cum(R * M);
  CK(cudaMemcpyAsync(cum.data(), E.ptab, cum.size() * 4, cudaMemcpyDeviceToHost, E.stream));
  CK(cudaStreamSynchronize(E.stream));
  for (size_t r = 0; r < R; ++r)
    for (int A = 0; A < M; ++A) q[r * M + A] = cum[r * M + A] - (A > 0 ? cum[r * M + A - 1] : 0u);
}

void learner_attach(Engine& E, const hande_learning& in) {
  if (!E.ptab) throw Fail{HANDE_ERR_INVALID, "the learned proposal needs a UEG context with excit_gen = 1"};
  if (E.learn) throw Fail{HANDE_ERR_INVALID, "a learned proposal is already attached"};
  const int M = E.P.sys.norb;
  if (M > 32 * kMaxPer) throw Fail{HANDE_ERR_INVALID, "the learned proposal supports at most 256 orbitals"};
  Learner* Lp = new Learner();
  E.learn = Lp;
  Learner& L = *Lp;
  L.M = M;
  L.din = 2 * M + 1;
  L.kin = (L.din + 63) / 64 * 64;
  L.H = in.width > 0 ? in.width : 256;
  L.S = in.batch > 0 ? in.batch : 4096;
  if (L.H % 64 || L.H > 512 || L.S % 128) throw Fail{HANDE_ERR_INVALID, "width: multiple of 64 up to 512; batch: multiple of 128"};
  L.period = in.period;
  L.lr = in.learning_rate > 0.0 ? (float)in.learning_rate : 1e-3f;
  L.R = 2 * M * M;
  L.Rp = (L.R + 127) / 128 * 128;
  L.M8 = (M + 7) / 8 * 8;
  L.rows_cap = L.S > L.Rp ? L.S : L.Rp;
  const int H = L.H;
  L.oW1 = 0;
  L.ob1 = L.oW1 + (size_t)H * L.din;
  L.oW2 = L.ob1 + H;
  L.ob2 = L.oW2 + (size_t)H * H;
  L.oW3 = L.ob2 + H;
  L.ob3 = L.oW3 + (size_t)M * H;
  L.nparam = (int64_t)(L.ob3 + M);
  L.param = dalloc<float>(E, L.nparam);
  L.mom1 = dalloc<float>(E, L.nparam);
  L.mom2 = dalloc<float>(E, L.nparam);
  L.grad = dalloc<float>(E, L.nparam);
  L.tstep = dalloc<int64_t>(E, 1);
  L.W1b = dalloc<uint16_t>(E, (size_t)H * L.kin);
  L.W2b = dalloc<uint16_t>(E, (size_t)H * H);
  L.W2bT = dalloc<uint16_t>(E, (size_t)H * H);
  L.W3b = dalloc<uint16_t>(E, (size_t)M * H);
  L.W3bT = dalloc<uint16_t>(E, (size_t)H * L.M8);
  L.X = dalloc<uint16_t>(E, (size_t)L.S * L.kin);
  L.XT = dalloc<uint16_t>(E, (size_t)L.kin * L.S);
  L.Xtab = dalloc<uint16_t>(E, (size_t)L.Rp * L.kin);
  L.H1 = dalloc<uint16_t>(E, (size_t)L.rows_cap * H);
  L.H2 = dalloc<uint16_t>(E, (size_t)L.rows_cap * H);
  L.H1T = dalloc<uint16_t>(E, (size_t)H * L.S);
  L.H2T = dalloc<uint16_t>(E, (size_t)H * L.S);
  L.G3 = dalloc<uint16_t>(E, (size_t)L.S * L.M8);
  L.G3T = dalloc<uint16_t>(E, (size_t)M * L.S);
  L.dZ2 = dalloc<uint16_t>(E, (size_t)L.S * H);
  L.dZ2T = dalloc<uint16_t>(E, (size_t)H * L.S);
  L.dZ1 = dalloc<uint16_t>(E, (size_t)L.S * H);
  L.dZ1T = dalloc<uint16_t>(E, (size_t)H * L.S);
  L.Z3 = dalloc<float>(E, (size_t)L.rows_cap * M);
  L.dH = dalloc<float>(E, (size_t)L.S * H);
  L.wsum = dalloc<float>(E, 1);
  L.loss = dalloc<double>(E, 1);
  L.err = dalloc<unsigned>(E, 1);
  L.in_rows = dalloc<int32_t>(E, L.S);
  L.in_tgt = dalloc<int32_t>(E, L.S);
  L.in_w = dalloc<float>(E, L.S);
  L.probs = dalloc<float>(E, (size_t)L.S * M);
  // sample buffers of the spawning kernel
  E.P.smp_row = dalloc<int32_t>(E, L.S);
  E.P.smp_A = dalloc<int32_t>(E, L.S);
  E.P.smp_w = dalloc<float>(E, L.S);
  cudaStream_t s = E.stream;
  CK(cudaMemsetAsync(E.P.smp_row, 0, sizeof(int32_t) * L.S, s));
  CK(cudaMemsetAsync(E.P.smp_A, 0, sizeof(int32_t) * L.S, s));
  CK(cudaMemsetAsync(E.P.smp_w, 0, sizeof(float) * L.S, s));
  CK(cudaMemsetAsync(L.mom1, 0, sizeof(float) * L.nparam, s));
  CK(cudaMemsetAsync(L.mom2, 0, sizeof(float) * L.nparam, s));
  CK(cudaMemsetAsync(L.tstep, 0, sizeof(int64_t), s));
  CK(cudaMemsetAsync(L.err, 0, sizeof(unsigned), s));
  CK(cudaMemsetAsync(L.G3, 0, sizeof(uint16_t) * (size_t)L.S * L.M8, s));
  // the table rows' features
  std::vector<int32_t> rows(L.Rp);
  for (int i = 0; i < L.Rp; ++i) rows[i] = i < L.R ? i : 0;
  int32_t* drows = dalloc<int32_t>(E, L.Rp);
  CK(cudaMemcpyAsync(drows, rows.data(), rows.size() * 4, cudaMemcpyHostToDevice, s));
  k_lr_features<<<grid_for((int64_t)L.Rp * L.kin), kLt, 0, s>>>(drows, nullptr, L.R, L.Rp, M, L.kin, L.Xtab, nullptr);
  CK(cudaGetLastError());
  // seeded initial weights: uniform in +-sqrt(6 / fan_in), zero biases
  std::vector<float> p((size_t)L.nparam, 0.0f);
  uint64_t st = in.seed ^ 0x6A09E667F3BCC909ull;
  auto uni = [&](double lim) { return (float)(lim * (2.0 * ((double)(splitmix(st) >> 11) * 0x1p-53) - 1.0)); };
  for (size_t i = 0; i < (size_t)H * L.din; ++i) p[L.oW1 + i] = uni(std::sqrt(6.0 / L.din));
  for (size_t i = 0; i < (size_t)H * H; ++i) p[L.oW2 + i] = uni(std::sqrt(6.0 / H));
  for (size_t i = 0; i < (size_t)M * H; ++i) p[L.oW3 + i] = uni(std::sqrt(6.0 / H));
  CK(cudaMemcpyAsync(L.param, p.data(), p.size() * 4, cudaMemcpyHostToDevice, s));
  to_bf16(L, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  E.P.smp_cap = L.S;
}

void learner_release(Engine& E) {
  if (!E.learn) return;
  if (E.learn->graph) cudaGraphExecDestroy(E.learn->graph);
  delete E.learn;
  E.learn = nullptr;
}

int64_t learner_nparam(const Engine& E) { return E.learn ? E.learn->nparam : 0; }

void learner_params(Engine& E, float* get, const float* set) {
  Learner& L = *E.learn;
  if (set) {
    CK(cudaMemcpyAsync(L.param, set, sizeof(float) * L.nparam, cudaMemcpyHostToDevice, E.stream));
    CK(cudaMemsetAsync(L.mom1, 0, sizeof(float) * L.nparam, E.stream));
    CK(cudaMemsetAsync(L.mom2, 0, sizeof(float) * L.nparam, E.stream));
    CK(cudaMemsetAsync(L.tstep, 0, sizeof(int64_t), E.stream));
    to_bf16(L, E.stream);
    CK(cudaGetLastError());
  }
  if (get) CK(cudaMemcpyAsync(get, L.param, sizeof(float) * L.nparam, cudaMemcpyDeviceToHost, E.stream));
  CK(cudaStreamSynchronize(E.stream));
}

// upload a batch of n <= S samples (rows, targets, weights; the rest weight 0)
static void upload_batch(Engine& E, Learner& L, const int32_t* rows, const int32_t* tgt, const float* w, int n) {
  const int R = L.R, M = L.M;
  std::vector<int32_t> r(L.S, 0), t(L.S, 0);
  std::vector<float> ww(L.S, 0.0f);
  for (int i = 0; i < n; ++i) {
    if (rows[i] < 0 || rows[i] >= R || (tgt && (tgt[i] < 0 || tgt[i] >= M)))
      throw Fail{HANDE_ERR_INVALID, "row or target orbital out of range"};
    if (tgt && !E.pmask[(size_t)rows[i] * M + tgt[i]]) throw Fail{HANDE_ERR_INVALID, "target orbital not drawable"};
    r[i] = rows[i];
    t[i] = tgt ? tgt[i] : 0;
    ww[i] = w ? w[i] : 1.0f;
    if (!(ww[i] >= 0.0f)) throw Fail{HANDE_ERR_INVALID, "sample weights must be >= 0"};
  }
  CK(cudaMemcpyAsync(L.in_rows, r.data(), 4 * (size_t)L.S, cudaMemcpyHostToDevice, E.stream));
  CK(cudaMemcpyAsync(L.in_tgt, t.data(), 4 * (size_t)L.S, cudaMemcpyHostToDevice, E.stream));
  CK(cudaMemcpyAsync(L.in_w, ww.data(), 4 * (size_t)L.S, cudaMemcpyHostToDevice, E.stream));
}

void learner_gradients(Engine& E, const int32_t* rows, const int32_t* tgt, const float* w, int n, float* grads,
                       double* loss) {
  Learner& L = *E.learn;
  if (n < 1 || n > L.S) throw Fail{HANDE_ERR_INVALID, "batch size must be in [1, batch]"};
  upload_batch(E, L, rows, tgt, w, n);
  CK(cudaMemsetAsync(L.err, 0, sizeof(unsigned), E.stream));
  backward(E, L, L.in_rows, L.in_tgt, L.in_w, E.stream);
  CK(cudaGetLastError());
  unsigned e = 0;
  CK(cudaMemcpyAsync(grads, L.grad, sizeof(float) * L.nparam, cudaMemcpyDeviceToHost, E.stream));
  CK(cudaMemcpyAsync(loss, L.loss, sizeof(double), cudaMemcpyDeviceToHost, E.stream));
  CK(cudaMemcpyAsync(&e, L.err, sizeof e, cudaMemcpyDeviceToHost, E.stream));
  CK(cudaStreamSynchronize(E.stream));
  if (e) throw Fail{HANDE_ERR_TIMEOUT, "a tensor-core GEMM wait timed out"};
}

void learner_probabilities(Engine& E, const int32_t* rows, int n, float* probs) {
  Learner& L = *E.learn;
  if (n < 1 || n > L.S) throw Fail{HANDE_ERR_INVALID, "row count must be in [1, batch]"};
  upload_batch(E, L, rows, nullptr, nullptr, n);
  CK(cudaMemsetAsync(L.err, 0, sizeof(unsigned), E.stream));
  k_lr_features<<<grid_for((int64_t)L.S * L.kin), kLt, 0, E.stream>>>(L.in_rows, nullptr, n, L.S, L.M, L.kin, L.X,
                                                                       nullptr);
  forward(L, L.X, L.S, false, E.stream);
  k_lr_probs<<<(n * 32 + kLt - 1) / kLt, kLt, 0, E.stream>>>(L.Z3, L.param + L.ob3, L.in_rows, n, L.M, E.pmask_dev,
                                                              L.probs);
  CK(cudaGetLastError());
  unsigned e = 0;
  CK(cudaMemcpyAsync(probs, L.probs, sizeof(float) * (size_t)n * L.M, cudaMemcpyDeviceToHost, E.stream));
  CK(cudaMemcpyAsync(&e, L.err, sizeof e, cudaMemcpyDeviceToHost, E.stream));
  CK(cudaStreamSynchronize(E.stream));
  if (e) throw Fail{HANDE_ERR_TIMEOUT, "a tensor-core GEMM wait timed out"};
}

void learner_refresh(Engine& E) {
  Learner& L = *E.learn;
  refresh_table(E, L, E.stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(E.stream));
}

// one training step (and table refresh) on the recorded samples, as a CUDA
// graph captured on first use; stream-ordered on the context's stream
void learner_step(Engine& E) {
  Learner& L = *E.learn;
  if (!L.graph) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(E.cap_stream, cudaStreamCaptureModeThreadLocal));
    try {
      enqueue_step(E, L, E.cap_stream);
    } catch (...) {
      cudaStreamEndCapture(E.cap_stream, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    cudaError_t le = cudaGetLastError();
    CK(cudaStreamEndCapture(E.cap_stream, &g));
    if (le != cudaSuccess) {
      cudaGraphDestroy(g);
      throw CudaError{le, "kernel launch during capture of the training step"};
    }
    cudaGraphExec_t ex = nullptr;
    cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    CK(ie);
    L.graph = ex;
  }
  CK(cudaGraphLaunch(L.graph, E.stream));
}

bool learner_due(const Engine& E) {
  return E.learn && E.learn->period > 0 && E.host_iter % E.learn->period == 0;
}

}  // namespace hande
