// kernels.cuh -- one FCIQMC iteration as a fixed sequence of kernels
// (HANDE-QMC paper, Sec. 2.1 Eq. (fciqmc) and Sec. 2.4; annihilation as in App. B:
// sort the spawned array and merge it into the sorted main list).
//
//   det_pass      per determinant: projected-energy terms (App. A.1), initiator
//                 flag (Sec. 2.1), spawning-attempt count, death/cloning
//   scan          exclusive scan of attempt counts (attempt space)
//   split         bucket geometry + splitter keys taken from the sorted main list
//   core_*        semi-stochastic exact projection inside the deterministic space
//   attempt       per attempt: Philox draw, excitation, H_ij, spawn amount, bucket id
//   scan          exclusive scan of bucket counts
//   scatter       spawns -> bucket-contiguous layout (one read + one write)
//   merge         per bucket: on-chip sort + reduce of its spawns, merge with the
//                 bucket's main-list segment, initiator rule, real-weight rounding,
//                 new diagonal elements, decoupled look-back compaction
//   finalize      shift update (Sec. 2.1) and the per-iteration estimator record
#pragma once
#include "system.cuh"

namespace hande {

constexpr int kMaxW = 8;
constexpr int kScanBlocks = 608;      // 4 x 152 SMs
constexpr int kScanThreads = 256;

// flags byte of a main-list entry
enum : uint8_t { F_CORE = 1, F_INIT = 2, F_NEG = 4, F_REF = 8, F_NEWDET = 16 };

struct Record {
  int64_t iter;
  double shift;
  int64_t nw_pre, n0, nw_post, ndet, natt, nspawn;
  int64_t num_hi;
  uint64_t num_lo;
  double num;
  double tau;
};

struct DevState {
  int64_t iter;
  int64_t ndet[2];
  int64_t natt;
  int64_t nspawn;
  int64_t nbuckets;
  int64_t sb;
  int64_t nw_pre;
  int64_t n0;
  unsigned long long num[2];   // int128 lo, hi
  int64_t nw_post;
  double shift;
  int64_t nw_ref;
  double e_ref;
  int vary;
  int64_t scan_total;
  int64_t nspawn_prev;   // spawns of the previous iteration (bucket sizing)
  int64_t nnew;          // new determinants written by the merge
  int64_t nuniq;         // distinct spawned keys the warp merge found off the list
  int64_t nuniq_prev;    // the same count of the previous iteration (bucket sizing)
  unsigned error;
  unsigned merge_ticket;
  unsigned defer_ticket;   // block-kernel tickets over the deferred buckets
  unsigned big_ticket;     // block-kernel tickets over all buckets (large-bucket pass)
  int64_t nbig;            // large buckets taken by block tiles
  int64_t ndefer;          // buckets the warp annihilation left to the block kernel
  unsigned long long rmax_bits;   // time-step search: largest |H| / p_gen so far (bits of a double >= 0)
};

struct Params {
  // run
  double tau, cutoff, zeta;
  uint64_t cutoff_fixed;   // spawn cutoff in walker fixed point
  int real_amp, initiator, period, W;
  int tau_search;          // record the largest |H| / p_gen of the attempts
  int64_t init_thr, target_fixed;
  uint64_t seed, replica;
  uint64_t d0[kMaxW];
  // capacities
  int64_t cap, scap;
  int tile_cap, seg_max, rec_cap;
  int bucket_spawns;   // expected spawns per annihilation bucket (sizes the buckets)
  int bucket_new;      // expected distinct new keys per bucket (0 = not used)
  int warp_cap;        // new keys one warp stages (warp annihilation)
  // main list (two buffers)
  uint64_t* key[2];
  int64_t* pop[2];
  double* hdiag[2];
  uint8_t* flags[2];
  // attempt space
  int64_t* natt;
  int64_t* att_begin;
  int64_t* part;         // scan partials, kScanBlocks + 1
  // spawns
  uint64_t* s_key;
  int64_t* s_amt;
  uint64_t* s_meta;
  uint64_t* b_key;
  int64_t* b_amt;
  uint8_t* b_flag;
  uint32_t* bcount;
  uint32_t* boff;
  unsigned long long* tile_state;
  // warp annihilation: kept entries of bucket b in tile_state[b], their output
  // offset in tile_inc[b]; the buckets' merged lists staged (key, N, H_ii,
  // flags) at the upper-bound offset b sb + boff[b] of arrays of mcap entries
  unsigned long long* tile_inc;
  uint64_t* m_key;
  int64_t* m_pop;
  double* m_hd;
  uint8_t* m_flg;
  int64_t mcap;
  uint64_t* split_key;
  // deterministic space
  int ncore;
  const uint64_t* core_key;
  const uint32_t* core_hash;   // open-addressing table of core indices + 1 (0 = empty)
  uint32_t core_hmask;         // table size - 1 (a power of two >= 4 ncore)
  int64_t* core_pos;
  const int64_t* core_rowptr;
  const int32_t* core_col;
  const double* core_val;
  int64_t* core_delta;
  int64_t* core_x;      // the core determinants' populations N(t-1), gathered by k_core_locate
  // training samples of the learned proposal (UEG table generator): attempts
  // g with g % stride == 0 (stride = ceil(natt / smp_cap)) write slot g / stride:
  // row, drawn particle orbital and w = |H| / p(A | row) (0 = no sample)
  int smp_cap;
  int32_t* smp_row;
  int32_t* smp_A;
  float* smp_w;
  // state
  DevState* st;
  Record* rec;
  SysDev sys;
};

// The block index and grid size a kernel body partitions its work by: the
// launch's own for a single run and for per-replica grids, a replica's share
// of a load-balanced batched launch otherwise.
struct VGrid {
  int b, n;
};

// a batched launch's parameter block: replica blockIdx.y's copied to shared
// memory by the whole block (before any thread may leave the kernel)
__device__ __forceinline__ void load_params(Params& sP, const Params* PP) {
  const uint64_t* src = reinterpret_cast<const uint64_t*>(PP + blockIdx.y);
  uint64_t* dst = reinterpret_cast<uint64_t*>(&sP);
  static_assert(sizeof(Params) % 8 == 0, "parameter block copied in 8-byte words");
  for (int i = threadIdx.x; i < (int)(sizeof(Params) / 8); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// A block of a load-balanced batched launch: replica r owns the blocks
// [off[r], off[r + 1]) (offsets written by the planner), this block is block
// blockIdx.x - off[r] of them.  Loads r's parameter block; false (for the whole
// block) when the block belongs to no replica.
__device__ __forceinline__ bool batch_block(const Params* PP, const int* off, int R, Params& sP, VGrid& vg) {
  __shared__ int s_r;
  if (threadIdx.x == 0) {
    const int b = (int)blockIdx.x;
    int lo = 0, hi = R;   // the last r with off[r] <= b
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= b) lo = mid;
      else hi = mid - 1;
    }
    const bool in = lo < R && b < off[lo + 1];
    s_r = in ? lo : -1;
    if (in) vg = VGrid{b - off[lo], off[lo + 1] - off[lo]};
  }
  __syncthreads();
  const int r = s_r;
  if (r < 0) return false;
  const uint64_t* src = reinterpret_cast<const uint64_t*>(PP + r);
  uint64_t* dst = reinterpret_cast<uint64_t*>(&sP);
  for (int i = threadIdx.x; i < (int)(sizeof(Params) / 8); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  return true;
}

// Load-balanced batched launch shape: for each phase p, the grid's blocks
// (budget[p]) are divided among the R replicas in proportion to their work
// (determinants for the list passes, the last iteration's attempts for the
// spawning phases), at least one block each and at most cap[p]; off[p][r] =
// first block of replica r.  One block; runs first in a batched iteration.
constexpr int kPlanPhases = 7;   // list pass, spawning, scatter, warp merge, block merge, copy, diagonals
struct Plan {
  int budget[kPlanPhases];
  int cap[kPlanPhases];
  int by_attempts[kPlanPhases];
};
static __global__ void kb_plan(const Params* PP, int R, int cur, Plan plan, int* off) {
  __shared__ double wsum[2];
  if (threadIdx.x == 0) {
    double a = 0.0, d = 0.0;
    for (int r = 0; r < R; ++r) {
      const DevState* st = PP[r].st;
      const int64_t nd = st->ndet[cur];
      const int64_t na = st->natt > 0 ? st->natt : nd;
      d += (double)(nd > 0 ? nd : 1);
      a += (double)(na > 0 ? na : 1);
    }
    wsum[0] = d;
    wsum[1] = a;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < kPlanPhases; p += blockDim.x) {
    int o = 0;
    for (int r = 0; r < R; ++r) {
      const DevState* st = PP[r].st;
      const int64_t nd = st->ndet[cur];
      const int64_t na = st->natt > 0 ? st->natt : nd;
      const double w = (double)(plan.by_attempts[p] ? (na > 0 ? na : 1) : (nd > 0 ? nd : 1));
      int c = 1 + (int)((double)plan.budget[p] * w / wsum[plan.by_attempts[p] ? 1 : 0]);
      if (c > plan.cap[p]) c = plan.cap[p];
      off[p * (R + 1) + r] = o;
      o += c;
    }
    off[p * (R + 1) + R] = o;
  }
}

template <int W>
__device__ __forceinline__ Key<W> ref_key(const Params& P) {
  Key<W> k;
#pragma unroll
  for (int j = 0; j < W; ++j) k.w[j] = P.d0[j];
  return k;
}

// ------------------------------------------------------------------ block helpers
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ T block_sum(T v, T* sh) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T r = 0;
  if (wid == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : T(0);
    r = warp_sum(r);
  }
  return r;  // valid in thread 0
}
static __device__ I128 block_sum_i128(I128 v, I128* sh) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    I128 x = shfl_xor_i128(v, o);
    i128_add(v, x);
  }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  I128 r{0, 0};
  if (wid == 0) {
    if (lane < (int)(blockDim.x >> 5)) r = sh[lane];
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      I128 x = shfl_xor_i128(r, o);
      i128_add(r, x);
    }
  }
  return r;
}
// exclusive scan over a shared array a[0..n) in place; returns the total (all threads)
template <typename T>
__device__ T block_scan_excl(T* a, int n, T* wsum) {
  const int T_ = blockDim.x;
  const int per = (n + T_ - 1) / T_;
  const int beg = threadIdx.x * per;
  const int end = min(beg + per, n);
  T s = 0;
  for (int i = beg; i < end; ++i) s += a[i];
  // warp inclusive scan of s
  T x = s;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int nw = T_ >> 5;
    T v = lane < nw ? wsum[lane] : T(0);
    T inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane < nw) wsum[lane] = inc - v;  // exclusive warp offsets
    if (lane == nw - 1) wsum[32] = inc;   // total
  }
  __syncthreads();
  T run = wsum[wid] + x - s;
  for (int i = beg; i < end; ++i) {
    T v = a[i];
    a[i] = run;
    run += v;
  }
  T total = wsum[32];
  __syncthreads();
  return total;
}

__device__ __forceinline__ void set_error(DevState* st, unsigned bit) { atomicOr(&st->error, bit); }

// chunk of a block-partitioned range [0, n) for block vg.b of vg.n
__device__ __forceinline__ void block_chunk(int64_t n, int64_t& beg, int64_t& end, const VGrid vg) {
  int64_t per = (n + vg.n - 1) / vg.n;
  beg = (int64_t)vg.b * per;
  end = beg + per < n ? beg + per : n;
  if (beg > n) beg = n;
}

// ------------------------------------------------------------------ det pass
template <int W, int SYS>
__device__ __forceinline__ void d_det_pass(const Params& P, int cur, const VGrid vg) {
  DevState* st = P.st;
  if (st->error) return;
  __shared__ int64_t sh64[32];
  __shared__ I128 sh128[32];
  const int64_t n = st->ndet[cur];
  const int64_t t = st->iter + 1;
  const double S = st->shift;
  const Key<W> d0 = ref_key<W>(P);
  int64_t beg, end;
  block_chunk(n, beg, end, vg);
  uint64_t* key = P.key[cur];
  int64_t* pop = P.pop[cur];
  const double* hd = P.hdiag[cur];
  uint8_t* fl = P.flags[cur];
  int64_t nw = 0, attsum = 0;
  I128 num{0, 0};
  for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
    Key<W> k = load_key<W>(key, P.cap, i);
    int64_t p = pop[i];
    uint8_t f = fl[i] & F_CORE;
    bool core = f != 0;
    bool is0 = key_eq<W>(k, d0);
    int64_t mag = iabs64(p);
    nw += mag;
    if (is0) {
      st->n0 = p;
    } else if (p != 0 && key_popc_xor<W>(k, d0) <= 4) {
      double h0j = h_elem<W, SYS>(P.sys, k, d0);
      i128_add(num, fixed_term(p, h0j));
    }
    bool init = !P.initiator || mag > P.init_thr || is0 || core;
    int64_t na = 0;
    int64_t np = p;
    if (p != 0) {
      Words4 w = draw<W>(P.seed, P.replica, t, kDetDraw, k);
      na = (int64_t)((uint64_t)mag >> 32);
      if (P.real_amp && (w.x >> 32) < ((uint64_t)mag & 0xffffffffull)) na += 1;
      if (!core) {
        double d = __dmul_rn(P.tau, __dsub_rn(__ldg(&hd[i]), S));
        if (P.real_amp) {
          np = p - __double2ll_rn(__dmul_rn(d, (double)p));
        } else {
          int64_t nwk = mag >> 32;
          double x = __dmul_rn(fabs(d), (double)nwk);
          double flo = floor(x);
          int64_t kk = (int64_t)flo;
          if (draw_unit(w.y) < __dsub_rn(x, flo)) kk += 1;
          int64_t nn = d > 0.0 ? nwk - kk : nwk + kk;
          np = (p < 0 ? -nn : nn) * kOne;
        }
        if (iabs64(np) >= (int64_t(1) << 62)) set_error(st, ERR_OVERFLOW);
        if (np != p) pop[i] = np;
      }
    }
    fl[i] = f | (init ? F_INIT : 0) | (p < 0 ? F_NEG : 0) | (is0 ? F_REF : 0);
    P.natt[i] = na;
    attsum += na;
  }
  int64_t a = block_sum<int64_t>(attsum, sh64);
  if (threadIdx.x == 0) P.part[vg.b] = a;
  int64_t b = block_sum<int64_t>(nw, sh64);
  if (threadIdx.x == 0 && b) atomicAdd((unsigned long long*)&st->nw_pre, (unsigned long long)b);
  I128 c = block_sum_i128(num, sh128);
  if (threadIdx.x == 0 && (c.lo | (uint64_t)c.hi)) atomic_add_i128(st->num, c);
}
template <int W, int SYS>
__global__ void __launch_bounds__(kScanThreads) k_det_pass(Params P, int cur) { d_det_pass<W, SYS>(P, cur, VGrid{(int)blockIdx.x, (int)gridDim.x}); }
// the same for replica blockIdx.y of a batch (parameter blocks PP[replica])
template <int W, int SYS>
__global__ void __launch_bounds__(kScanThreads) kb_det_pass(const Params* PP, const int* off, int R, int cur) {
  __shared__ Params sP;
  __shared__ VGrid vg;
  if (!batch_block(PP, off, R, sP, vg)) return;
  d_det_pass<W, SYS>(sP, cur, vg);
}

// ------------------------------------------------------------------ generic scans
// partials scanned by one block; total written to *total
__device__ __forceinline__ void d_scan_partials_i64(int64_t* part, int nparts, int64_t* total, DevState* st) {
  if (st->error) return;
  __shared__ int64_t buf[kScanBlocks];
  __shared__ int64_t wsum[33];
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) buf[i] = part[i];
  __syncthreads();
  int64_t tot = block_scan_excl<int64_t>(buf, nparts, wsum);
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) part[i] = buf[i];
  if (threadIdx.x == 0) *total = tot;
}
static __global__ void k_scan_partials_i64(int64_t* part, int nparts, int64_t* total, DevState* st) {
  d_scan_partials_i64(part, nparts, total, st);
}
// Exclusive scan of in[0, *n_ptr) into out by one block of 1024 threads, for
// short arrays (bucket counts): chunks of 4096 loaded coalesced into shared
// memory, 4 contiguous values per thread, block scan of the thread sums.  The
// total goes to *total; above cap_check (if >= 0) it sets the state-capacity
// error.  With total_hi the values are two packed 32-bit counts, the totals of
// the low and high halves go to *total and *total_hi.
template <typename Tin, typename Tout>
__device__ __forceinline__ void d_scan_one(const Tin* in, Tout* out, const int64_t* n_ptr, int64_t* total,
                                           int64_t cap_check, DevState* st, int64_t* total_hi) {
  if (st->error) return;
  constexpr int kPer = 4, kChunk = 1024 * kPer;
  __shared__ unsigned long long buf[kChunk];
  __shared__ unsigned long long wsum[32];
  const int64_t n = *n_ptr;
  const int tid = (int)threadIdx.x, lane = tid & 31, wid = tid >> 5;
  unsigned long long carry = 0;
  for (int64_t base = 0; base < n; base += kChunk) {
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int64_t i = base + k * 1024 + tid;
      buf[k * 1024 + tid] = i < n ? (unsigned long long)in[i] : 0ull;
    }
    __syncthreads();
    unsigned long long v[kPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      v[k] = buf[tid * kPer + k];
      sum += v[k];
    }
    unsigned long long x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      const unsigned long long w0 = wsum[lane];
      unsigned long long inc = w0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      wsum[lane] = inc - w0;
    }
    __syncthreads();
    unsigned long long run = carry + wsum[wid] + x - sum;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      buf[tid * kPer + k] = run;
      run += v[k];
    }
    __syncthreads();
    if (wid == 31 && lane == 31) wsum[0] = run;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int64_t i = base + k * 1024 + tid;
      if (i < n) out[i] = (Tout)buf[k * 1024 + tid];
    }
    __syncthreads();
    carry = wsum[0];
    __syncthreads();
  }
  if (tid == 0) {
    // total_hi: the values are two packed 32-bit counts (sums stay below 2^32)
    const int64_t lo = total_hi ? (int64_t)(carry & 0xffffffffull) : (int64_t)carry;
    if (total_hi) *total_hi = (int64_t)(carry >> 32);
    *total = lo;
    if (cap_check >= 0 && lo > cap_check) set_error(st, ERR_STATE_CAPACITY);
  }
}
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(1024) k_scan_one(const Tin* in, Tout* out, const int64_t* n_ptr, int64_t* total,
                                                    int64_t cap_check, DevState* st, int64_t* total_hi = nullptr) {
  d_scan_one<Tin, Tout>(in, out, n_ptr, total, cap_check, st, total_hi);
}

// out[i] = exclusive prefix of in over the block's chunk + part[block]; each
// round takes 4 consecutive values per thread (4 x blockDim per round)
template <typename T>
__device__ __forceinline__ void d_scan_apply(const T* in, T* out, const int64_t* n_ptr, const int64_t* part,
                                             DevState* st, const VGrid vg) {
  if (st->error) return;
  constexpr int kItems = 4;
  __shared__ T wsum[33];
  int64_t beg, end;
  block_chunk(*n_ptr, beg, end, vg);
  const int lane = (int)(threadIdx.x & 31), wid = (int)(threadIdx.x >> 5), nw = (int)(blockDim.x >> 5);
  T carry = (T)part[vg.b];
  for (int64_t base = beg; base < end; base += (int64_t)blockDim.x * kItems) {
    const int64_t i0 = base + (int64_t)threadIdx.x * kItems;
    T v[kItems], sum = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      v[k] = i0 + k < end ? in[i0 + k] : T(0);
      sum += v[k];
    }
    T x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      const T w0 = lane < nw ? wsum[lane] : T(0);
      T inc = w0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      if (lane < nw) wsum[lane] = inc - w0;
      if (lane == 31) wsum[32] = inc;
    }
    __syncthreads();
    T run = carry + wsum[wid] + x - sum;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
      if (i0 + k < end) out[i0 + k] = run;
      run += v[k];
    }
    carry += wsum[32];
    __syncthreads();
  }
}
template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const T* in, T* out, const int64_t* n_ptr,
                                                             const int64_t* part, DevState* st) {
  d_scan_apply<T>(in, out, n_ptr, part, st, VGrid{(int)blockIdx.x, (int)gridDim.x});
}
template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const T* in, const int64_t* n_ptr, int64_t* part,
                                                              DevState* st) {
  if (st->error) return;
  __shared__ int64_t sh[32];
  int64_t beg, end;
  block_chunk(*n_ptr, beg, end, VGrid{(int)blockIdx.x, (int)gridDim.x});
  int64_t s = 0;
  for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) s += (int64_t)in[i];
  s = block_sum<int64_t>(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// batched forms of the scans, pointers taken from replica blockIdx.y's block
static __global__ void kb_scan_natt(const Params* PP, const int* off, int R) {
  const Params& P = PP[blockIdx.y];
  d_scan_partials_i64(P.part, off[blockIdx.y + 1] - off[blockIdx.y], &P.st->natt, P.st);
}
static __global__ void __launch_bounds__(kScanThreads) kb_scan_att(const Params* PP, const int* off, int R, int cur) {
  __shared__ Params sP;
  __shared__ VGrid vg;
  if (!batch_block(PP, off, R, sP, vg)) return;
  d_scan_apply<int64_t>(sP.natt, sP.att_begin, &sP.st->ndet[cur], sP.part, sP.st, vg);
}
static __global__ void __launch_bounds__(1024) kb_scan_buckets(const Params* PP) {
  const Params& P = PP[blockIdx.y];
  d_scan_one<uint32_t, uint32_t>(P.bcount, P.boff, &P.st->nbuckets, &P.st->scan_total, -1, P.st, nullptr);
}
static __global__ void __launch_bounds__(1024) kb_scan_kept(const Params* PP, int cur) {
  const Params& P = PP[blockIdx.y];
  d_scan_one<unsigned long long, unsigned long long>(P.tile_state, P.tile_inc, &P.st->nbuckets,
                                                     &P.st->ndet[cur ^ 1], P.cap, P.st, &P.st->nnew);
}

// ------------------------------------------------------------------ buckets
// Bucket b holds the main-list segment [b*sb, (b+1)*sb) and every spawn whose key
// lies in [key[b*sb], key[(b+1)*sb]); sb is chosen so a bucket expects at most
// half a tile of spawns (even if every one went to a new determinant).
template <int W>
__device__ __forceinline__ void d_split(const Params& P, int cur, const VGrid vg) {
  DevState* st = P.st;
  if (st->error) return;
  const int64_t n = st->ndet[cur];
  // expected spawns: the previous iteration's count with 25% headroom (twice
  // the determinants before the first iteration; this kernel may run beside the
  // det pass and the attempt scan, so it reads nothing they write)
  const int64_t na = st->nspawn_prev > 0 ? st->nspawn_prev + st->nspawn_prev / 4 : 2 * n;
  int64_t sb = (int64_t)P.seg_max;
  const int64_t per = P.bucket_spawns;   // expected spawns per bucket
  if (na > 0) {
    int64_t want = (int64_t)(((double)per * (double)n) / (double)na);
    if (want < sb) sb = want;
  }
  // lists whose spawns mostly land off the list (many new keys per bucket)
  // get smaller buckets, so that the warp staging rarely overflows
  const int64_t nu = st->nuniq_prev;
  if (P.bucket_new > 0 && nu > 0) {
    int64_t want = (int64_t)(((double)P.bucket_new * (double)n) / (double)nu);
    if (want < sb) sb = want;
  }
  if (sb < 1) sb = 1;
  int64_t nb = (n + sb - 1) / sb;
  if (nb < 1) nb = 1;
  if (vg.b == 0 && threadIdx.x == 0) {
    st->nbuckets = nb;
    st->sb = sb;
    st->nspawn = 0;
    st->nnew = 0;
    st->nuniq = 0;
    st->merge_ticket = 0;
    st->defer_ticket = 0;
    st->big_ticket = 0;
    st->nbig = 0;
    st->ndefer = 0;
    if (nb > P.cap) set_error(st, ERR_BUCKET_CAPACITY);
  }
  if (nb > P.cap) return;
  for (int64_t b = vg.b * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)vg.n * blockDim.x) {
    P.bcount[b] = 0;
    P.tile_state[b] = 0ull;

    int64_t src = b * sb;
#pragma unroll
    for (int j = 0; j < W; ++j) P.split_key[j * P.cap + b] = src < n ? P.key[cur][j * P.cap + src] : 0ull;
  }
}
template <int W>
__global__ void k_split(Params P, int cur) { d_split<W>(P, cur, VGrid{(int)blockIdx.x, (int)gridDim.x}); }
// the same for replica blockIdx.y of a batch (parameter blocks PP[replica])
template <int W>
__global__ void kb_split(const Params* PP, const int* off, int R, int cur) {
  __shared__ Params sP;
  __shared__ VGrid vg;
  if (!batch_block(PP, off, R, sP, vg)) return;
  d_split<W>(sP, cur, vg);
}

// ------------------------------------------------------------------ deterministic space
template <int W>
__device__ __forceinline__ int64_t lower_bound_main(const uint64_t* key, int64_t stride, int64_t n, const Key<W>& k) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    Key<W> m = load_key<W>(key, stride, mid);
    if (key_lt<W>(m, k)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
// Fibonacci hash of the XOR-folded key words
template <int W>
__device__ __forceinline__ uint32_t key_hash(const Key<W>& k) {
  uint64_t x = k.w[0];
#pragma unroll
  for (int j = 1; j < W; ++j) x ^= k.w[j] * 0xC2B2AE3D27D4EB4Full + (uint64_t)j;
  return (uint32_t)((x * 0x9E3779B97F4A7C15ull) >> 32);
}
// membership in the deterministic space: linear probing of the core hash table
template <int W>
__device__ __forceinline__ bool in_core(const Params& P, const Key<W>& k) {
  uint32_t h = key_hash<W>(k) & P.core_hmask;
  for (uint32_t probe = 0; probe <= P.core_hmask; ++probe) {
    const uint32_t v = __ldg(&P.core_hash[h]);
    if (v == 0) return false;
    if (key_eq<W>(load_key<W>(P.core_key, P.ncore, (int64_t)v - 1), k)) return true;
    h = (h + 1) & P.core_hmask;
  }
  return false;
}
// insert every core key (table zeroed, at most a quarter full)
template <int W>
__global__ void k_core_hash(Params P, uint32_t* table) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= P.ncore) return;
  uint32_t h = key_hash<W>(load_key<W>(P.core_key, P.ncore, r)) & P.core_hmask;
  for (uint32_t probe = 0; probe <= P.core_hmask; ++probe) {
    if (atomicCAS(&table[h], 0u, (uint32_t)r + 1u) == 0u) return;
    h = (h + 1) & P.core_hmask;
  }
}
template <int W>
__device__ __forceinline__ void d_core_locate(const Params& P, int cur) {
  DevState* st = P.st;
  if (st->error) return;
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= P.ncore) return;
  Key<W> k = load_key<W>(P.core_key, P.ncore, r);
  const int64_t n = st->ndet[cur];
  int64_t pos = lower_bound_main<W>(P.key[cur], P.cap, n, k);
  if (pos >= n || !key_eq<W>(load_key<W>(P.key[cur], P.cap, pos), k)) {
    set_error(st, ERR_STATE_CAPACITY);   // a deterministic-space determinant left the list
    pos = 0;
  }
  P.core_pos[r] = pos;
  P.core_x[r] = P.pop[cur][pos];
}
template <int W>
__global__ void k_core_locate(Params P, int cur) { d_core_locate<W>(P, cur); }
// the same for replica blockIdx.y of a batch (parameter blocks PP[replica])
template <int W>
__global__ void kb_core_locate(const Params* PP, int cur) {
  __shared__ Params sP;
  load_params(sP, PP);
  d_core_locate<W>(sP, cur);
}
// one warp per core row: y_r = sum_c H'_rc N_c exactly, dN_r = -rint(tau (y_r - S N_r))
__device__ __forceinline__ void d_core_spmv(const Params& P, int cur) {
  DevState* st = P.st;
  if (st->error) return;
  int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (r >= P.ncore) return;
  I128 acc{0, 0};
  for (int64_t e = P.core_rowptr[r] + lane; e < P.core_rowptr[r + 1]; e += 32) {
    int64_t pc = P.core_x[P.core_col[e]];
    i128_add(acc, fixed_term(pc, P.core_val[e]));
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    I128 x = shfl_xor_i128(acc, o);
    i128_add(acc, x);
  }
  if (lane == 0) {
    double y = fixed_to_double(acc);
    int64_t pr = P.core_x[r];
    double v = __dsub_rn(y, __dmul_rn(st->shift, (double)pr));
    double x = __dmul_rn(P.tau, v);
    P.core_delta[r] = -__double2ll_rn(x);
  }
}
static __global__ void k_core_spmv(Params P, int cur) { d_core_spmv(P, cur); }
// the same for replica blockIdx.y of a batch (parameter blocks PP[replica])
static __global__ void kb_core_spmv(const Params* PP, int cur) {
  __shared__ Params sP;
  load_params(sP, PP);
  d_core_spmv(sP, cur);
}
__device__ __forceinline__ void d_core_apply(const Params& P, int cur) {
  DevState* st = P.st;
  if (st->error) return;
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= P.ncore) return;
  P.pop[cur][P.core_pos[r]] += P.core_delta[r];
}
static __global__ void k_core_apply(Params P, int cur) { d_core_apply(P, cur); }
// the same for replica blockIdx.y of a batch (parameter blocks PP[replica])
static __global__ void kb_core_apply(const Params* PP, int cur) {
  __shared__ Params sP;
  load_params(sP, PP);
  d_core_apply(sP, cur);
}

// ------------------------------------------------------------------ attempts
// ------------------------------------------------------------------ attempts
// Attempts are processed 32 per warp.  Lanes diverge on what an attempt
// produces (nothing, a spawn, a molecular single needing an O(N) matrix
// element), so the rare outcomes go through per-warp shared-memory queues and
// are finished 32 at a time by full warps: singles (select the orbitals,
// evaluate H_ia, weight, rounding) and spawns (bucket search, append to the
// staging arrays).  Two CTAs share an SM: the shared memory below stays
// under half of an SM's 228 KB for every key width and system.
constexpr int kAttemptThreads = 512;
constexpr int kAttemptWarps = kAttemptThreads / 32;
constexpr int kQueue = 64;   // per-warp queue capacity (holds 31 + 32 entries)

template <int W, int SYS>
__host__ __device__ constexpr int attempt_split_smem() {
  return W == 8 ? (SYS == SYS_MOLECULE ? 128 : 256) : (W == 2 ? 2048 : 4096);
}
// molecular generator tables copied to shared memory for 64-bit keys (at most
// 64 spin orbitals): the pair records (int4) and the pair unranking table
constexpr int kStagePairs = 64 * 63 / 2;
template <int W, int SYS>
__host__ __device__ constexpr size_t attempt_stage_bytes() {
  return (SYS == SYS_MOLECULE && W == 1) ? (size_t)kStagePairs * (16 + 2) : 0;
}
// per-warp queue bytes per entry: spawns (key, amount, flag) and, for
// molecules, singles (parent, words w and z, occupied rank)
template <int W, int SYS>
__host__ __device__ constexpr size_t attempt_queue_entry() {
  return (size_t)(8 * W + 8 + 1) + (SYS == SYS_MOLECULE ? (size_t)(8 + 8 + 8 + 1) : 0);
}
template <int W, int SYS>
__host__ __device__ inline size_t attempt_smem_bytes() {
  return (size_t)attempt_split_smem<W, SYS>() * 8 * W + attempt_stage_bytes<W, SYS>() +
         (size_t)kAttemptWarps * kQueue * attempt_queue_entry<W, SYS>() + 256;
}

struct AttemptQueues {
  int64_t* sq_par;     // pending singles: parent index
  uint64_t* sq_word;   // their Philox word w (rounding)
  uint64_t* sq_wz;     // word z (empty orbital)
  uint8_t* sq_ri;      // rank of the occupied orbital, draw_index(w.y, N)
  uint64_t* pq_key;    // finished spawns: key words [W][kQueue]
  int64_t* pq_amt;
  uint8_t* pq_flg;
};

// time-step search: the warp's largest |H| / p_gen into the running maximum
// (bits of non-negative doubles order like the doubles); whole warp
__device__ __forceinline__ void ratio_max(const Params& P, double r) {
  unsigned long long b = (unsigned long long)__double_as_longlong(r);
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long x = __shfl_xor_sync(0xffffffffu, b, o);
    b = x > b ? x : b;
  }
  if (warp_lane() == 0 && b) atomicMax(&P.st->rmax_bits, b);
}

// signed spawn amount (0 = nothing) from the fixed-point amount famt of the
// weight tau |H| / p_gen (floored for integer walkers, rounded for real
// weights), Philox word u and parent flags pf; sign -sign(H) sign(N_parent)
__device__ __forceinline__ int64_t spawn_amount(const Params& P, uint64_t famt, bool hneg, uint64_t u, uint8_t pf) {
  uint64_t q;
  if (!P.real_amp) {   // floor(m) walkers, one more with probability frac(m)
    uint64_t k = famt >> 32;
    if ((u >> 32) < (famt & 0xffffffffull)) k += 1;
    q = k >= (1ull << 30) ? kAmountMax : k << 32;
  } else {             // below the cutoff: kept, as the cutoff, with probability m / cutoff
    q = famt;
    if (q < P.cutoff_fixed) q = __umul64hi(u, P.cutoff_fixed) < q ? P.cutoff_fixed : 0;
  }
  if (q == 0) return 0;
  const bool neg = hneg == ((pf & F_NEG) != 0);
  return neg ? -(int64_t)q : (int64_t)q;
}

// Bucket search of the spawning kernel: every r-th splitter (coarse, in shared
// memory when the kernel stages them) then at most r - 1 splitters in global
// memory.  bucket(k) = number of splitters s_j (1 <= j < nb) with s_j <= k.
struct SplitIdx {
  const uint64_t* coarse;   // coarse[c] = s_{c r}, c < nc
  int64_t cstride, nc, r;
  const uint64_t* fine;     // all splitters
  int64_t fstride, nb;
};

template <int W>
__device__ __forceinline__ uint32_t find_bucket(const SplitIdx& sx, const Key<W>& k) {
  int64_t lo = 1, hi = sx.nc;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (key_le<W>(load_key<W>(sx.coarse, sx.cstride, mid), k)) lo = mid + 1;
    else hi = mid;
  }
  const int64_t c = lo - 1;   // s_{c r} <= k < s_{(c+1) r}
  int64_t blo = c * sx.r + 1, bhi = c * sx.r + sx.r < sx.nb ? c * sx.r + sx.r : sx.nb;
  while (blo < bhi) {
    const int64_t mid = (blo + bhi) >> 1;
    if (key_le<W>(load_key<W>(sx.fine, sx.fstride, mid), k)) blo = mid + 1;
    else bhi = mid;
  }
  return (uint32_t)(blo - 1);
}

// the top `take` queued spawns of this warp: bucket, rank, staging slot
template <int W>
__device__ void flush_spawns(const Params& P, const AttemptQueues& Q, int& pq_n, int take, const SplitIdx& sx) {
  DevState* st = P.st;
  const int lane = (int)warp_lane();
  const bool have = lane < take;
  Key<W> child;
  int64_t amt = 0;
  uint8_t initf = 0;
  uint32_t bkt = 0;
  if (have) {
    const int e = pq_n - take + lane;
#pragma unroll
    for (int j = 0; j < W; ++j) child.w[j] = Q.pq_key[j * kQueue + e];
    amt = Q.pq_amt[e];
    initf = Q.pq_flg[e];
    bkt = find_bucket<W>(sx, child);
  }
  const unsigned want = __ballot_sync(0xffffffffu, have);
  int64_t base = 0;
  if (want && lane == 0)
    base = (int64_t)atomicAdd((unsigned long long*)&st->nspawn, (unsigned long long)__popc(want));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (have) {
    const int64_t slot = base + lane;
    const uint32_t rank = atomicAdd(&P.bcount[bkt], 1u);
    if (slot < P.scap) {
      store_key<W>(P.s_key, P.scap, slot, child);
      P.s_amt[slot] = amt;
      P.s_meta[slot] = ((uint64_t)bkt << 32) | ((uint64_t)rank << 1) | initf;
    } else {
      set_error(st, ERR_SPAWN_CAPACITY);
    }
  }
  pq_n -= take;
  __syncwarp();
}

template <int W>
__device__ __forceinline__ void push_spawn(const Params& P, const AttemptQueues& Q, int& pq_n, bool have,
                                           const Key<W>& child, int64_t amt, uint8_t initf, const SplitIdx& sx) {
  const unsigned m = __ballot_sync(0xffffffffu, have);
  if (have) {
    const int e = pq_n + __popc(m & ((1u << warp_lane()) - 1u));
#pragma unroll
    for (int j = 0; j < W; ++j) Q.pq_key[j * kQueue + e] = child.w[j];
    Q.pq_amt[e] = amt;
    Q.pq_flg[e] = initf;
  }
  pq_n += __popc(m);
  __syncwarp();
  if (pq_n >= 32) flush_spawns<W>(P, Q, pq_n, 32, sx);
}

// the top `take` queued molecular singles: orbitals, H_ia, core test, weight,
// rounding
template <int W, int SYS>
__device__ void flush_singles(const Params& P, const AttemptQueues& Q, int& sq_n, int& pq_n, int take,
                              const uint64_t* key, const uint8_t* fl, const SplitIdx& sx) {
  const int lane = (int)warp_lane();
  bool have = false;
  Key<W> child;
  int64_t amt = 0;
  uint8_t initf = 0;
  double rmax = 0.0;
  if (lane < take) {
    const int e = sq_n - take + lane;
    const int64_t par = Q.sq_par[e];
    const uint64_t u = Q.sq_word[e];
    const Key<W> k = load_key<W>(key, P.cap, par);
    const uint8_t f = fl[par];
    int i = 0, a = 0;
    const bool drawn = single_orbitals<W>(P.sys, k, Q.sq_ri[e], Q.sq_wz[e], i, a);
    child = k;
    key_flip<W>(child, i);
    key_flip<W>(child, a);
    const double hij = drawn ? h_single<W, SYS>(P.sys, k, i, a) : 0.0;
    if (drawn && nonzero(hij) && !((f & F_CORE) && P.ncore > 0 && in_core<W>(P, child))) {
      if (P.tau_search) rmax = __dmul_rn(fabs(hij), P.sys.inv_single[i & 1]);
      const uint64_t famt = fixed_amount(abs_bits(hij), dbl_bits(P.sys.c_single[i & 1]), P.sys.half);
      amt = spawn_amount(P, famt, sign_bit(hij), u, f);
      initf = (f & F_INIT) ? 1 : 0;
      have = amt != 0;
    }
  }
  sq_n -= take;
  __syncwarp();
  if (P.tau_search) ratio_max(P, rmax);
  push_spawn<W>(P, Q, pq_n, have, child, amt, initf, sx);
}

// largest i < n with a[i] <= x, given a[known] <= x (a non-decreasing):
// doubling steps from `known`, then bisection
__device__ __forceinline__ int64_t gallop_last_le(const int64_t* a, int64_t known, int64_t n, int64_t x) {
  int64_t lo = known, hi, step = 1;
  for (;;) {
    hi = lo + step;
    if (hi >= n) {
      hi = n;
      break;
    }
    if (a[hi] > x) break;
    lo = hi;
    step <<= 1;
  }
  while (hi - lo > 1) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (a[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}
// lane l of a warp: av = a[base + l]; lane 31 also av32 = a[base + 32]
// (INT64_MAX past n).  No lane waits for the loads here.
__device__ __forceinline__ void load_window(const int64_t* a, int64_t n, int64_t base, int lane, int64_t& av,
                                            int64_t& av32) {
  const int64_t wi = base + lane;
  av = wi < n ? a[wi] : INT64_MAX;
  av32 = (lane == 31 && wi + 1 < n) ? a[wi + 1] : INT64_MAX;
}

// Training sample of the learned proposal from a proposal-table draw (also a
// rejected one: the UEG matrix element depends only on the four momenta):
// w = |H| / p(A | row) with |H| = |v(k_I - k_A) - [same spin] v(k_I - k_B)|,
// v(q) = 4 pi / (Omega |q|^2), q = 0 terms omitted.
template <int W>
__device__ __forceinline__ void record_sample(const Params& P, int64_t natt, int64_t g, const Excitation<W>& ex) {
  const int64_t stride = (natt + P.smp_cap - 1) / P.smp_cap;
  if (stride < 1 || g % stride != 0) return;
  const int64_t slot = g / stride;
  if (slot >= P.smp_cap) return;
  float wv = 0.0f;
  int row = 0, A = 0;
  if (ex.prow >= 0) {
    const SysDev& s = P.sys;
    const int M = s.norb, same = ex.prow & 1, IJ = ex.prow >> 1, I = IJ / M, J = IJ % M;
    A = ex.pA;
    row = ex.prow;
    const int4 ki = __ldg(&s.kvec[I]), kj = __ldg(&s.kvec[J]), ka = __ldg(&s.kvec[A]);
    const int bx = ki.x + kj.x - ka.x, by = ki.y + kj.y - ka.y, bz = ki.z + kj.z - ka.z;
    const int B = __ldg(&s.klookup[((bx + s.nmax) * s.side + (by + s.nmax)) * s.side + (bz + s.nmax)]);
    const int dA = (ki.x - ka.x) * (ki.x - ka.x) + (ki.y - ka.y) * (ki.y - ka.y) + (ki.z - ka.z) * (ki.z - ka.z);
    const int4 kb = __ldg(&s.kvec[B]);
    const int dB = (ki.x - kb.x) * (ki.x - kb.x) + (ki.y - kb.y) * (ki.y - kb.y) + (ki.z - kb.z) * (ki.z - kb.z);
    const double direct = dA > 0 ? s.vfac / (double)dA : 0.0;
    const double exch = (same && dB > 0) ? s.vfac / (double)dB : 0.0;
    const double h = fabs(direct - exch);
    wv = (float)(h * ((double)ex.pQ / (double)ex.pqa));
  }
  P.smp_row[slot] = row;
  P.smp_A[slot] = A;
  P.smp_w[slot] = wv;
}

template <int W, int SYS>
__device__ __forceinline__ void d_attempt(const Params& P, int cur, const VGrid vg) {
  DevState* st = P.st;
  if (st->error) return;
  constexpr int KS = attempt_split_smem<W, SYS>();
  extern __shared__ __align__(16) unsigned char att_smem[];
  uint64_t* ssplit = reinterpret_cast<uint64_t*>(att_smem);
  const int wid = threadIdx.x >> 5;
  AttemptQueues Q;
  {
    unsigned char* p = att_smem + (size_t)KS * 8 * W + attempt_stage_bytes<W, SYS>();
    const size_t per = kQueue;
    Q.pq_key = reinterpret_cast<uint64_t*>(p) + wid * per * W;
    p += kAttemptWarps * per * 8 * W;
    Q.pq_amt = reinterpret_cast<int64_t*>(p) + wid * per;
    p += kAttemptWarps * per * 8;
    Q.pq_flg = reinterpret_cast<uint8_t*>(p) + wid * per;
    p += kAttemptWarps * per;   // a multiple of 8 bytes
    Q.sq_par = nullptr;
    Q.sq_word = Q.sq_wz = nullptr;
    Q.sq_ri = nullptr;
    if (SYS == SYS_MOLECULE) {
      Q.sq_par = reinterpret_cast<int64_t*>(p) + wid * per;
      p += kAttemptWarps * per * 8;
      Q.sq_word = reinterpret_cast<uint64_t*>(p) + wid * per;
      p += kAttemptWarps * per * 8;
      Q.sq_wz = reinterpret_cast<uint64_t*>(p) + wid * per;
      p += kAttemptWarps * per * 8;
      Q.sq_ri = reinterpret_cast<uint8_t*>(p) + wid * per;
    }
  }
  const int64_t natt = st->natt;
  const int64_t n = st->ndet[cur];
  const int64_t nb = st->nbuckets;
  const int64_t t = st->iter + 1;
  const uint64_t* key = P.key[cur];
  const uint8_t* fl = P.flags[cur];
  // every r-th splitter staged in shared memory (all of them when nb <= KS)
  SplitIdx sx;
  sx.r = (nb + KS - 1) / KS;
  sx.nc = (nb + sx.r - 1) / sx.r;
  sx.fine = P.split_key;
  sx.fstride = P.cap;
  sx.nb = nb;
  sx.coarse = ssplit;
  sx.cstride = KS;
  for (int64_t c = threadIdx.x; c < sx.nc; c += blockDim.x) {
#pragma unroll
    for (int j = 0; j < W; ++j) ssplit[j * KS + c] = P.split_key[j * P.cap + c * sx.r];
  }
  GenTabs gt{P.sys.hb_pair, P.sys.pair_ij};
  if (attempt_stage_bytes<W, SYS>() > 0) {
    int4* sp = reinterpret_cast<int4*>(att_smem + (size_t)KS * 8 * W);
    uint16_t* sij = reinterpret_cast<uint16_t*>(att_smem + (size_t)KS * 8 * W + (size_t)kStagePairs * 16);
    const int npp = P.sys.nspin * (P.sys.nspin - 1) / 2, nij = P.sys.nel * (P.sys.nel - 1) / 2;
    for (int i = threadIdx.x; i < npp; i += blockDim.x) sp[i] = P.sys.hb_pair[i];
    for (int i = threadIdx.x; i < nij; i += blockDim.x) sij[i] = P.sys.pair_ij[i];
    gt.hb_pair = sp;
    gt.pair_ij = sij;
  }
  __syncthreads();
  const int lane = (int)warp_lane();
  const int64_t total_warps = (int64_t)vg.n * kAttemptWarps;
  int sq_n = 0, pq_n = 0;   // warp-uniform queue lengths
  // each warp owns one contiguous span of attempts, taken in chunks of 32.
  // Parents are monotone in the attempt index: with base = the parent of a
  // chunk's first attempt, the chunk's parents lie in base .. base + 31 unless
  // determinants without attempts lie in between (then a galloping search).
  // The offsets att_begin[base .. base + 32] of the next chunk are loaded while
  // the current chunk is processed.
  const int64_t span = (((natt + total_warps - 1) / total_warps) + 31) & ~(int64_t)31;
  const int64_t gbeg = ((int64_t)vg.b * kAttemptWarps + wid) * span;
  const int64_t gend = gbeg + span < natt ? gbeg + span : natt;
  int64_t base = 0, av = INT64_MAX, av32_l = INT64_MAX;
  if (gbeg < gend) {
    if (lane == 0) {
      int64_t lo = 0, hi = n - 1;
      while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (P.att_begin[mid] <= gbeg) lo = mid;
        else hi = mid - 1;
      }
      base = lo;
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    load_window(P.att_begin, n, base, lane, av, av32_l);
  }
  for (int64_t gw = gbeg; gw < gend; gw += 32) {
    const int64_t g = gw + lane;
    const int64_t av32 = __shfl_sync(0xffffffffu, av32_l, 31);
    // number of window entries <= g (binary search over the lanes' values)
    int cnt = 0;
#pragma unroll
    for (int step = 16; step; step >>= 1) {
      const int64_t probe = __shfl_sync(0xffffffffu, av, cnt + step - 1);
      if (probe <= g) cnt += step;
    }
    const int64_t w_at = __shfl_sync(0xffffffffu, av, cnt == 0 ? 0 : (cnt < 32 ? cnt : 31));
    if (w_at <= g && cnt == 31) cnt = 32;
    int64_t par = base + cnt - 1;
    int64_t abeg = __shfl_sync(0xffffffffu, av, (cnt - 1) & 31);
    const bool beyond = g < gend && cnt == 32 && g >= av32;   // past att_begin[base + 32]
    // next chunk: its base, and its window in flight during this chunk
    const int64_t X = gw + 32;
    if (X < gend) {
      const int c = __popc(__ballot_sync(0xffffffffu, av <= X));
      int64_t nbase;
      if (c < 32) nbase = base + c - 1;
      else if (X < av32) nbase = base + 31;
      else nbase = gallop_last_le(P.att_begin, base + 31, n, X);
      load_window(P.att_begin, n, nbase, lane, av, av32_l);
      if (beyond) {
        par = gallop_last_le(P.att_begin, base + 31, n, g);
        abeg = P.att_begin[par];
      }
      base = nbase;
    } else if (beyond) {
      par = gallop_last_le(P.att_begin, base + 31, n, g);
      abeg = P.att_begin[par];
    }
    bool have = false, single = false;
    Key<W> child;
    int64_t amt = 0;
    uint8_t initf = 0;
    uint64_t word = 0, wz = 0;
    uint8_t ri = 0;
    double rmax = 0.0;
    if (g < gend) {
      const uint64_t a = (uint64_t)(g - abeg);
      const Key<W> k = load_key<W>(key, P.cap, par);
      const uint8_t f = fl[par];
      const Words4 w = draw<W>(P.seed, P.replica, t, a, k);
      const Excitation<W> ex = generate<W, SYS>(P.sys, gt, k, w);
      if (SYS == SYS_UEG && P.smp_cap > 0) record_sample(P, natt, g, ex);
      if (ex.single) {
        single = true;
        word = w.w;
        wz = w.z;
        ri = (uint8_t)draw_index(w.y, (uint64_t)P.sys.nel);
      } else if (ex.ok && !((f & F_CORE) && P.ncore > 0 && in_core<W>(P, ex.child))) {
        rmax = fmax(rmax, ex.rval);
        amt = spawn_amount(P, ex.famt, ex.hneg, w.w, f);
        child = ex.child;
        initf = (f & F_INIT) ? 1 : 0;
        have = amt != 0;
      }
    }
    if (SYS == SYS_MOLECULE) {
      const unsigned sm = __ballot_sync(0xffffffffu, single);
      if (single) {
        const int e = sq_n + __popc(sm & ((1u << lane) - 1u));
        Q.sq_par[e] = par;
        Q.sq_word[e] = word;
        Q.sq_wz[e] = wz;
        Q.sq_ri[e] = ri;
      }
      sq_n += __popc(sm);
      __syncwarp();
    }
    if (P.tau_search) ratio_max(P, rmax);
    push_spawn<W>(P, Q, pq_n, have, child, amt, initf, sx);
    if (SYS == SYS_MOLECULE && sq_n >= 32)
      flush_singles<W, SYS>(P, Q, sq_n, pq_n, 32, key, fl, sx);
  }
  if (SYS == SYS_MOLECULE && sq_n > 0)
    flush_singles<W, SYS>(P, Q, sq_n, pq_n, sq_n, key, fl, sx);
  if (pq_n > 0) flush_spawns<W>(P, Q, pq_n, pq_n, sx);
}
template <int W, int SYS>
__global__ void __launch_bounds__(kAttemptThreads) k_attempt(Params P, int cur) { d_attempt<W, SYS>(P, cur, VGrid{(int)blockIdx.x, (int)gridDim.x}); }
// the same for replica blockIdx.y of a batch (parameter blocks PP[replica])
// (two blocks per SM as for the single-run kernel: the shared-memory parameter
// block would otherwise raise the register count past that)
template <int W, int SYS>
__global__ void __launch_bounds__(kAttemptThreads, 2) kb_attempt(const Params* PP, const int* off, int R, int cur) {
  __shared__ Params sP;
  __shared__ VGrid vg;
  if (!batch_block(PP, off, R, sP, vg)) return;
  d_attempt<W, SYS>(sP, cur, vg);
}

template <int W>
__device__ __forceinline__ void d_scatter(const Params& P, const VGrid vg) {
  DevState* st = P.st;
  if (st->error) return;
  const int64_t ns = st->nspawn < P.scap ? st->nspawn : P.scap;
  for (int64_t s = (int64_t)vg.b * blockDim.x + threadIdx.x; s < ns; s += (int64_t)vg.n * blockDim.x) {
    uint64_t m = P.s_meta[s];
    uint32_t b = (uint32_t)(m >> 32);
    uint32_t rank = (uint32_t)(m & 0xffffffffu) >> 1;
    int64_t dst = (int64_t)P.boff[b] + rank;
    Key<W> k = load_key<W>(P.s_key, P.scap, s);
    store_key<W>(P.b_key, P.scap, dst, k);
    P.b_amt[dst] = P.s_amt[s];
    P.b_flag[dst] = (uint8_t)(m & 1u);
  }
}
template <int W>
__global__ void __launch_bounds__(256) k_scatter(Params P) { d_scatter<W>(P, VGrid{(int)blockIdx.x, (int)gridDim.x}); }
// the same for replica blockIdx.y of a batch (parameter blocks PP[replica])
template <int W>
__global__ void __launch_bounds__(256) kb_scatter(const Params* PP, const int* off, int R) {
  __shared__ Params sP;
  __shared__ VGrid vg;
  if (!batch_block(PP, off, R, sP, vg)) return;
  d_scatter<W>(sP, vg);
}

// ------------------------------------------------------------------ merge (annihilation)
template <int W>
struct MergeSmem {
  // tile arrays are carved from dynamic shared memory
  uint64_t* skey;    // [W][TC]  spawned keys, sorted unique after sort_reduce
  int64_t* samt;     // [TC]
  uint32_t* sflg;    // [TC]     bit0 initiator parent, bit31 padding
  int32_t* uid;      // [TC]
  int64_t* uamt;     // [TC]
  uint32_t* uflg;    // [TC]
  uint64_t* mkey;    // [W][SM]  main-list keys of the bucket's segment
  int32_t* mmatch;   // [SM]     unique index matching a main entry, or -1
  int32_t* mlb;      // [SM]     unique keys below the main key
  int32_t* ulb;      // [TC]     main keys below the unique key (-1 if matched)
  uint32_t* mscan;   // [TC+1]   exclusive prefix of matched flags over the unique list
  uint32_t* keep;    // [TC+SM]  keep flags by merged rank, scanned in place
  int64_t* macc;     // [SM]     spawned amounts added to each main entry (then the final N)
  uint64_t* skey2;   // [W][kCountMax] unique keys of the counting reduction
  uint64_t* spl;     // [W][RMAX] sub-range splitters of an oversized bucket
  int32_t* rcnt;     // [RMAX+1] spawns per sub-range
  int32_t* roff;     // [RMAX+1]
  int32_t* rcur;     // [RMAX+1]
  int32_t* runiq;    // [RMAX+1] unique keys per sub-range
  int32_t* rkeep;    // [RMAX+1] surviving entries per sub-range
};

constexpr int kSubRanges = 256;   // RMAX: sub-ranges of one oversized bucket
constexpr int kCountMax = 128;    // new-key sets up to this size are reduced by counting

template <int W>
__host__ __device__ inline size_t merge_smem_bytes(int TC, int SM) {
  return (size_t)TC * (8 * W + 8 + 4 + 4 + 8 + 4 + 4 + 4) + 4 + (size_t)SM * (8 * W + 4 + 4 + 8) + (size_t)kCountMax * 8 * W +
         (size_t)(TC + SM) * 4 + (size_t)kSubRanges * 8 * W + (size_t)(kSubRanges + 1) * 4 * 5 + 1024;
}

template <int W>
__device__ __forceinline__ Key<W> skey_at(const MergeSmem<W>& m, int TC, int i) {
  Key<W> k;
#pragma unroll
  for (int j = 0; j < W; ++j) k.w[j] = m.skey[j * TC + i];
  return k;
}
template <int W>
__device__ __forceinline__ Key<W> mkey_at(const MergeSmem<W>& m, int SM, int i) {
  Key<W> k;
#pragma unroll
  for (int j = 0; j < W; ++j) k.w[j] = m.mkey[j * SM + i];
  return k;
}
template <int W>
__device__ __forceinline__ Key<W> spl_at(const MergeSmem<W>& m, int i) {
  Key<W> k;
#pragma unroll
  for (int j = 0; j < W; ++j) k.w[j] = m.spl[j * kSubRanges + i];
  return k;
}
template <int W>
__device__ __forceinline__ bool rec_lt(const MergeSmem<W>& m, int TC, int a, int b) {
  bool pa = m.sflg[a] >> 31, pb = m.sflg[b] >> 31;
  if (pa != pb) return pb;
  if (pa) return false;
  return key_lt<W>(skey_at<W>(m, TC, a), skey_at<W>(m, TC, b));
}
template <int W>
__device__ __forceinline__ void rec_swap(MergeSmem<W>& m, int TC, int a, int b) {
#pragma unroll
  for (int j = 0; j < W; ++j) {
    uint64_t x = m.skey[j * TC + a];
    m.skey[j * TC + a] = m.skey[j * TC + b];
    m.skey[j * TC + b] = x;
  }
  int64_t y = m.samt[a];
  m.samt[a] = m.samt[b];
  m.samt[b] = y;
  uint32_t z = m.sflg[a];
  m.sflg[a] = m.sflg[b];
  m.sflg[b] = z;
}

// Sort records [0, n) in place (bitonic, padded to a power of two), then combine
// equal keys: on return records [0, u) are the sorted unique keys with summed
// amounts and OR-ed initiator bits.  Returns u.
template <int W>
__device__ int sort_reduce(MergeSmem<W>& m, int TC, int n, uint32_t* wsum) {
  int n2 = 64;
  while (n2 < n) n2 <<= 1;
  for (int i = n + threadIdx.x; i < n2; i += blockDim.x) m.sflg[i] = 0x80000000u;
  __syncthreads();
  // bitonic network over n2 keys; compare-swap pair p joins elements
  // i = 2p - (p mod j) and i + j, so for strides j <= 32 the 32 pairs of a warp
  // stay inside its own 64-element segment and a warp barrier suffices
  const int npairs = n2 >> 1;
  const bool warp_local_ok = npairs <= (int)blockDim.x;
  int prev_j = 64;
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      // a block barrier separates two stages unless both stay inside warps
      if (!warp_local_ok || j > 32 || prev_j > 32) __syncthreads();
      else __syncwarp();
      prev_j = j;
      for (int pbase = 0; pbase < npairs; pbase += blockDim.x) {
        const int p = pbase + threadIdx.x;
        if (p < npairs) {
          const int i = 2 * p - (p & (j - 1));
          const int l = i + j;
          const bool up = (i & k) == 0;
          const bool sw = up ? rec_lt<W>(m, TC, l, i) : rec_lt<W>(m, TC, i, l);
          if (sw) rec_swap<W>(m, TC, i, l);
        }
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    bool head = (i == 0) || !key_eq<W>(skey_at<W>(m, TC, i), skey_at<W>(m, TC, i - 1));
    m.uid[i] = head ? 1 : 0;
    m.uamt[i] = 0;
    m.uflg[i] = 0;
  }
  __syncthreads();
  uint32_t* u32 = reinterpret_cast<uint32_t*>(m.uid);
  uint32_t total = block_scan_excl<uint32_t>(u32, n, wsum);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    bool head = (i == 0) || !key_eq<W>(skey_at<W>(m, TC, i), skey_at<W>(m, TC, i - 1));
    int id = (int)u32[i] + (head ? 1 : 0) - 1;
    atomicAdd((unsigned long long*)&m.uamt[id], (unsigned long long)m.samt[i]);
    if (m.sflg[i] & 1u) atomicOr(&m.uflg[id], 1u);
    m.uid[i] = head ? id : -1;
  }
  __syncthreads();
  // compact heads forward in rounds (a head at i moves to id <= i)
  for (int base = 0; base < n; base += blockDim.x) {
    int i = base + threadIdx.x;
    int id = -1;
    Key<W> k;
    if (i < n) {
      id = m.uid[i];
      if (id >= 0) k = skey_at<W>(m, TC, i);
    }
    __syncthreads();
    if (id >= 0) {
#pragma unroll
      for (int j = 0; j < W; ++j) m.skey[j * TC + id] = k.w[j];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < (int)total; i += blockDim.x) {
    m.samt[i] = m.uamt[i];
    m.sflg[i] = m.uflg[i];
  }
  __syncthreads();
  return (int)total;
}

// The same result as sort_reduce for n <= kCountMax (<= blockDim) records, by
// counting: each record finds the first record with its key, each first record
// counts the first records with smaller keys (its position), and amounts and
// initiator bits are added into that position.  O(n^2) compares, four barriers.
template <int W>
__device__ int count_reduce(MergeSmem<W>& m, int TC, int n) {
  const int i = threadIdx.x;
  Key<W> ki;
  int rep = i;
  if (i < n) {
    ki = skey_at<W>(m, TC, i);
    for (int j = 0; j < i; ++j)
      if (key_eq<W>(skey_at<W>(m, TC, j), ki)) {
        rep = j;
        break;
      }
    m.uid[i] = rep;
    m.uamt[i] = 0;
    m.uflg[i] = 0;
  }
  __syncthreads();
  if (i < n && rep == i) {
    int r = 0;
    for (int j = 0; j < n; ++j)
      if (m.uid[j] == j && key_lt<W>(skey_at<W>(m, TC, j), ki)) ++r;
    m.ulb[i] = r;
  }
  const int u = __syncthreads_count(i < n && rep == i);
  if (i < n) {
    const int r = m.ulb[rep];
    atomicAdd((unsigned long long*)&m.uamt[r], (unsigned long long)m.samt[i]);
    if (m.sflg[i] & 1u) atomicOr(&m.uflg[r], 1u);
    if (rep == i) {
#pragma unroll
      for (int j = 0; j < W; ++j) m.skey2[j * kCountMax + r] = ki.w[j];
    }
  }
  __syncthreads();
  if (i < u) {
#pragma unroll
    for (int j = 0; j < W; ++j) m.skey[j * TC + i] = m.skey2[j * kCountMax + i];
    m.samt[i] = m.uamt[i];
    m.sflg[i] = m.uflg[i];
  }
  __syncthreads();
  return u;
}

// Load spawns [beg, end) of (key, amt, flag) arrays into the tile and reduce
// them; chunks are appended to the unique keys kept so far, so repeated keys
// (many spawns onto one determinant) collapse as they arrive.  Returns the
// number of unique keys, or -1 if more than TC distinct keys arrive.
template <int W>
__device__ int load_reduce(MergeSmem<W>& m, int TC, const uint64_t* key, int64_t kstride, const int64_t* amt,
                           const uint8_t* flg8, const uint64_t* flg64, int64_t beg, int64_t end, uint32_t* wsum) {
  int nu = 0;
  for (int64_t pos = beg; pos < end;) {
    int take = TC - nu;
    if (take <= 0) return -1;
    if ((int64_t)take > end - pos) take = (int)(end - pos);
    for (int i = threadIdx.x; i < take; i += blockDim.x) {
      int64_t src = pos + i;
#pragma unroll
      for (int j = 0; j < W; ++j) m.skey[j * TC + nu + i] = key[j * kstride + src];
      m.samt[nu + i] = amt[src];
      m.sflg[nu + i] = flg8 ? (uint32_t)flg8[src] : (uint32_t)(flg64[src] & 1u);
    }
    __syncthreads();
    nu = sort_reduce<W>(m, TC, nu + take, wsum);
    pos += take;
  }
  return nu;
}

template <int W>
__device__ __forceinline__ int lb_smem_main(const MergeSmem<W>& m, int SM, int lo, int hi, const Key<W>& k) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (key_lt<W>(mkey_at<W>(m, SM, mid), k)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
template <int W>
__device__ __forceinline__ int lb_smem_uniq(const MergeSmem<W>& m, int TC, int nu, const Key<W>& k) {
  int lo = 0, hi = nu;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (key_lt<W>(skey_at<W>(m, TC, mid), k)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Real-weight occupation rounding of 0 < |N| < 1 walker to 0 or +-1 walker
// with probability |N| (per-determinant Philox word z).
template <int W>
__device__ __forceinline__ int64_t round_small(const Params& P, int64_t t, const Key<W>& k, int64_t p) {
  int64_t mag = iabs64(p);
  if (P.real_amp && mag > 0 && mag < kOne) {
    Words4 w = draw<W>(P.seed, P.replica, t, kDetDraw, k);
    int64_t r = ((w.z >> 32) < (uint64_t)mag) ? kOne : 0;
    return p < 0 ? -r : r;
  }
  return p;
}

// Context of one merge: the bucket's main segment and the list buffers.
struct MergeCtx {
  int64_t m0;           // first main-list index of the bucket segment
  int64_t t;            // iteration number
  const int64_t* pop;
  const double* hd;
  const uint8_t* fl;
  uint64_t* okey;
  int64_t* opop;
  double* ohd;
  uint8_t* ofl;
  int64_t ostride;      // key-word stride of the output arrays
  int staged;           // output is the warp annihilation's staging list
  int64_t bucket;       // staged: the bucket (its count word gets the new determinants)
};

// Merge the sorted unique spawns [0, nu) with the main segment entries [ml, mh)
// (segment-local indices, keys in m.mkey): candidates in key order, the keep
// decision of each written to m.keep[rank] and scanned.  Main entries keep their
// slot if core or reference, otherwise they survive with a nonzero population
// after the real-weight occupation rounding.  New determinants need an
// initiator parent (Sec. 2.1) and a nonzero amount.  Returns the number kept.
template <int W>
__device__ uint32_t tile_decide(const Params& P, MergeSmem<W>& m, const MergeCtx& c, int TC, int SM, int nu,
                                int ml, int mh, uint32_t* wsum, int& nc_out) {
  const int nm = mh - ml;
  for (int j = threadIdx.x; j < nu; j += blockDim.x) {
    Key<W> k = skey_at<W>(m, TC, j);
    int lb = lb_smem_main<W>(m, SM, ml, mh, k);
    bool match = lb < mh && key_eq<W>(mkey_at<W>(m, SM, lb), k);
    m.ulb[j] = match ? -1 : lb - ml;
    m.mscan[j] = match ? 1u : 0u;
  }
  for (int i = threadIdx.x; i < nm; i += blockDim.x) {
    Key<W> k = mkey_at<W>(m, SM, ml + i);
    int lb = lb_smem_uniq<W>(m, TC, nu, k);
    m.mlb[i] = lb;
    m.mmatch[i] = (lb < nu && key_eq<W>(skey_at<W>(m, TC, lb), k)) ? lb : -1;
  }
  __syncthreads();
  if (threadIdx.x == 0) m.mscan[nu] = 0;
  __syncthreads();
  uint32_t nmatched = block_scan_excl<uint32_t>(m.mscan, nu + 1, wsum);
  const int nc = nm + nu - (int)nmatched;
  for (int i = threadIdx.x; i < nm; i += blockDim.x) {
    int rank = i + m.mlb[i] - (int)m.mscan[m.mlb[i]];
    int64_t gi = c.m0 + ml + i;
    int64_t p = c.pop[gi];
    if (m.mmatch[i] >= 0) p += m.samt[m.mmatch[i]];
    uint8_t f = c.fl[gi];
    bool always = (f & (F_CORE | F_REF)) != 0;
    if (!always) p = round_small<W>(P, c.t, mkey_at<W>(m, SM, ml + i), p);
    m.keep[rank] = (always || p != 0) ? 1u : 0u;
  }
  for (int j = threadIdx.x; j < nu; j += blockDim.x) {
    int lb = m.ulb[j];
    if (lb < 0) continue;
    int rank = lb + (j - (int)m.mscan[j]);
    int64_t p = m.samt[j];
    bool ok = (!P.initiator || (m.sflg[j] & 1u)) && p != 0;
    if (ok) p = round_small<W>(P, c.t, skey_at<W>(m, TC, j), p);
    m.keep[rank] = (ok && p != 0) ? 1u : 0u;
  }
  __syncthreads();
  nc_out = nc;
  return block_scan_excl<uint32_t>(m.keep, nc, wsum);
}

// Write the entries kept by tile_decide at out + (their rank among the kept).
template <int W, int SYS>
__device__ int64_t tile_write(const Params& P, MergeSmem<W>& m, const MergeCtx& c, int TC, int SM, int nu, int ml,
                              int mh, int nc, uint32_t nkeep, int64_t out) {
  DevState* st = P.st;
  const int nm = mh - ml;
  int64_t nwsum = 0;
  for (int i = threadIdx.x; i < nm; i += blockDim.x) {
    int rank = i + m.mlb[i] - (int)m.mscan[m.mlb[i]];
    uint32_t pos = m.keep[rank];
    uint32_t nx = (rank + 1 < nc) ? m.keep[rank + 1] : nkeep;
    if (nx == pos) continue;
    int64_t gi = c.m0 + ml + i;
    int64_t p = c.pop[gi];
    if (m.mmatch[i] >= 0) p += m.samt[m.mmatch[i]];
    uint8_t f = c.fl[gi];
    Key<W> k = mkey_at<W>(m, SM, ml + i);
    bool always = (f & (F_CORE | F_REF)) != 0;
    if (!always) p = round_small<W>(P, c.t, k, p);
    if (iabs64(p) >= (int64_t(1) << 62)) set_error(st, ERR_OVERFLOW);
    int64_t o = out + pos;
    store_key<W>(c.okey, c.ostride, o, k);
    c.opop[o] = p;
    c.ohd[o] = c.hd[gi];
    c.ofl[o] = f & F_CORE;
    nwsum += iabs64(p);
  }
  for (int j = threadIdx.x; j < nu; j += blockDim.x) {
    int lb = m.ulb[j];
    if (lb < 0) continue;
    int rank = lb + (j - (int)m.mscan[j]);
    uint32_t pos = m.keep[rank];
    uint32_t nx = (rank + 1 < nc) ? m.keep[rank + 1] : nkeep;
    if (nx == pos) continue;
    Key<W> k = skey_at<W>(m, TC, j);
    int64_t p = round_small<W>(P, c.t, k, m.samt[j]);
    if (iabs64(p) >= (int64_t(1) << 62)) set_error(st, ERR_OVERFLOW);
    int64_t o = out + pos;
    store_key<W>(c.okey, c.ostride, o, k);
    c.opop[o] = p;
    c.ohd[o] = 0.0;   // H_ii - E_ref follows in k_new_hdiag
    if (c.staged) {
      c.ofl[o] = F_NEWDET;
      atomicAdd(&P.tile_state[c.bucket], 1ull << 32);
    } else {
      c.ofl[o] = 0;
      P.natt[atomicAdd((unsigned long long*)&st->nnew, 1ull)] = o;
    }
    nwsum += iabs64(p);
  }
  __syncthreads();
  return nwsum;
}

// Common-path merge: spawns onto segment entries were added into m.macc,
// spawns onto new determinants are the sorted unique keys [0, nu); no key is
// in both.  Keep flags by merged rank, scanned; returns the number kept.
template <int W>
__device__ uint32_t acc_decide(const Params& P, MergeSmem<W>& m, const MergeCtx& c, int TC, int SM, int nu,
                               int nm, uint32_t* wsum) {
  for (int j = threadIdx.x; j < nu; j += blockDim.x)
    m.ulb[j] = lb_smem_main<W>(m, SM, 0, nm, skey_at<W>(m, TC, j));
  for (int i = threadIdx.x; i < nm; i += blockDim.x) m.mlb[i] = lb_smem_uniq<W>(m, TC, nu, mkey_at<W>(m, SM, i));
  __syncthreads();
  // the final population of every candidate is kept on chip for acc_write:
  // main entries in macc (flags in mmatch), new determinants in samt
  for (int i = threadIdx.x; i < nm; i += blockDim.x) {
    int64_t gi = c.m0 + i;
    int64_t p = c.pop[gi] + m.macc[i];
    const uint8_t f = c.fl[gi];
    bool always = (f & (F_CORE | F_REF)) != 0;
    if (!always) p = round_small<W>(P, c.t, mkey_at<W>(m, SM, i), p);
    m.macc[i] = p;
    m.mmatch[i] = f;
    m.keep[i + m.mlb[i]] = (always || p != 0) ? 1u : 0u;
  }
  for (int j = threadIdx.x; j < nu; j += blockDim.x) {
    int64_t p = m.samt[j];
    bool ok = (!P.initiator || (m.sflg[j] & 1u)) && p != 0;
    if (ok) p = round_small<W>(P, c.t, skey_at<W>(m, TC, j), p);
    m.samt[j] = p;
    m.keep[m.ulb[j] + j] = (ok && p != 0) ? 1u : 0u;
  }
  __syncthreads();
  return block_scan_excl<uint32_t>(m.keep, nm + nu, wsum);
}

template <int W, int SYS>
__device__ int64_t acc_write(const Params& P, MergeSmem<W>& m, const MergeCtx& c, int TC, int SM, int nu, int nm,
                             uint32_t nkeep, int64_t out) {
  DevState* st = P.st;
  const int nc = nm + nu;
  int64_t nwsum = 0;
  for (int i = threadIdx.x; i < nm; i += blockDim.x) {
    int rank = i + m.mlb[i];
    uint32_t pos = m.keep[rank];
    uint32_t nx = (rank + 1 < nc) ? m.keep[rank + 1] : nkeep;
    if (nx == pos) continue;
    const int64_t gi = c.m0 + i;
    const int64_t p = m.macc[i];
    const uint8_t f = (uint8_t)m.mmatch[i];
    const Key<W> k = mkey_at<W>(m, SM, i);
    if (iabs64(p) >= (int64_t(1) << 62)) set_error(st, ERR_OVERFLOW);
    int64_t o = out + pos;
    store_key<W>(c.okey, c.ostride, o, k);
    c.opop[o] = p;
    c.ohd[o] = c.hd[gi];
    c.ofl[o] = f & F_CORE;
    nwsum += iabs64(p);
  }
  for (int j = threadIdx.x; j < nu; j += blockDim.x) {
    int rank = m.ulb[j] + j;
    uint32_t pos = m.keep[rank];
    uint32_t nx = (rank + 1 < nc) ? m.keep[rank + 1] : nkeep;
    if (nx == pos) continue;
    Key<W> k = skey_at<W>(m, TC, j);
    const int64_t p = m.samt[j];
    if (iabs64(p) >= (int64_t(1) << 62)) set_error(st, ERR_OVERFLOW);
    int64_t o = out + pos;
    store_key<W>(c.okey, c.ostride, o, k);
    c.opop[o] = p;
    c.ohd[o] = 0.0;   // H_ii - E_ref follows in k_new_hdiag
    if (c.staged) {
      c.ofl[o] = F_NEWDET;
      atomicAdd(&P.tile_state[c.bucket], 1ull << 32);
    } else {
      c.ofl[o] = 0;
      P.natt[atomicAdd((unsigned long long*)&st->nnew, 1ull)] = o;
    }
    nwsum += iabs64(p);
  }
  __syncthreads();
  return nwsum;
}

// Decoupled look-back (single-pass chained scan) over bucket output counts,
// run by one warp: each step reads 32 predecessor states at once.  Buckets are
// taken in ticket order, so every predecessor is owned by a running CTA and
// publishes its count without waiting: the spin always ends, and is bounded
// anyway.  Returns the exclusive prefix (all lanes); sets *abort on failure.
__device__ __forceinline__ unsigned long long lookback_warp(const Params& P, int64_t b, uint32_t count, int* abort) {
  DevState* st = P.st;
  const unsigned long long AGG = 1ull << 62, INC = 2ull << 62, MASK = (1ull << 62) - 1;
  const int lane = (int)warp_lane();
  if (b == 0) {
    if (lane == 0) atomicExch(&P.tile_state[0], INC | (unsigned long long)count);
    return 0;
  }
  if (lane == 0) atomicExch(&P.tile_state[b], AGG | (unsigned long long)count);
  unsigned long long excl = 0;
  int64_t p = b - 1;
  long long spins = 0;
  for (;;) {
    const int64_t idx = p - lane;
    const unsigned long long v = idx >= 0 ? *(volatile const unsigned long long*)&P.tile_state[idx] : INC;
    const unsigned long long s = v >> 62;
    const unsigned inc = __ballot_sync(0xffffffffu, s == 2);
    const unsigned none = __ballot_sync(0xffffffffu, s == 0);
    const int first = inc ? __ffs(inc) - 1 : 31;
    const unsigned need = first == 31 ? 0xffffffffu : ((2u << first) - 1u);
    if (none & need) {   // a state we need is not published yet
      ++spins;
      __nanosleep(64);
      if ((spins & 255) == 0 && *(volatile unsigned*)&st->error) {
        *abort = 1;   // another tile failed: give up without adding an error
        return 0;
      }
      if (spins > (1ll << 20)) {
        if (lane == 0) set_error(st, ERR_TIMEOUT);
        *abort = 1;
        return 0;
      }
      continue;
    }
    unsigned long long add = (lane <= first) ? (v & MASK) : 0ull;
#pragma unroll
    for (int o = 16; o; o >>= 1) add += __shfl_xor_sync(0xffffffffu, add, o);
    excl += add;
    if (inc) break;
    p -= 32;
  }
  if (lane == 0) atomicExch(&P.tile_state[b], INC | (excl + count));
  return excl;
}

constexpr int kMergeThreads = 256;

template <int W, int SYS>
__device__ __forceinline__ void d_merge(const Params& P, int cur, int staged, const VGrid vg) {
  DevState* st = P.st;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t wsum[33];
  __shared__ int64_t sh64[32];
  __shared__ int tile_id;
  __shared__ unsigned long long s_base;
  __shared__ int s_abort;
  __shared__ int s_nsub;
  __shared__ int s_nnew;
  const int TC = P.tile_cap, SM = P.seg_max;
  MergeSmem<W> m;
  {
    unsigned char* p = smem_raw;
    auto carve = [&](size_t bytes) {
      unsigned char* r = p;
      p += (bytes + 15) & ~size_t(15);
      return r;
    };
    m.skey = (uint64_t*)carve(sizeof(uint64_t) * W * TC);
    m.samt = (int64_t*)carve(sizeof(int64_t) * TC);
    m.uamt = (int64_t*)carve(sizeof(int64_t) * TC);
    m.mkey = (uint64_t*)carve(sizeof(uint64_t) * W * SM);
    m.spl = (uint64_t*)carve(sizeof(uint64_t) * W * kSubRanges);
    m.sflg = (uint32_t*)carve(4 * TC);
    m.uid = (int32_t*)carve(4 * TC);
    m.uflg = (uint32_t*)carve(4 * TC);
    m.ulb = (int32_t*)carve(4 * TC);
    m.mscan = (uint32_t*)carve(4 * (TC + 1));
    m.mmatch = (int32_t*)carve(4 * SM);
    m.mlb = (int32_t*)carve(4 * SM);
    m.keep = (uint32_t*)carve(4 * (TC + SM));
    m.rcnt = (int32_t*)carve(4 * (kSubRanges + 1));
    m.roff = (int32_t*)carve(4 * (kSubRanges + 1));
    m.rcur = (int32_t*)carve(4 * (kSubRanges + 1));
    m.runiq = (int32_t*)carve(4 * (kSubRanges + 1));
    m.rkeep = (int32_t*)carve(4 * (kSubRanges + 1));
    m.macc = (int64_t*)carve(8 * SM);
    m.skey2 = (uint64_t*)carve(8 * W * kCountMax);
  }
  const int64_t n = st->ndet[cur];
  const int64_t nb = st->nbuckets;
  const int64_t sb = st->sb;
  const int nxt = cur ^ 1;
  MergeCtx c;
  c.t = st->iter + 1;
  c.pop = P.pop[cur];
  c.hd = P.hdiag[cur];
  c.fl = P.flags[cur];
  // staged: only the buckets the warp annihilation deferred, written to its
  // staging list at their upper-bound offsets (no look-back)
  c.okey = staged ? P.m_key : P.key[nxt];
  c.opop = staged ? P.m_pop : P.pop[nxt];
  c.ohd = staged ? P.m_hd : P.hdiag[nxt];
  c.ofl = staged ? P.m_flg : P.flags[nxt];
  c.ostride = staged ? P.mcap : P.cap;
  c.staged = staged;
  const uint64_t* key = P.key[cur];
  int64_t nwsum = 0;
  // large-bucket pass: blocks claim chunks of blockDim.x buckets (one ticket
  // each) and list the chunk's large buckets (more spawns than a warp takes)
  __shared__ int s_big[kMergeThreads];
  __shared__ int s_nbig, s_pbig;
  __shared__ int64_t s_chunk;
  if (threadIdx.x == 0) s_nbig = s_pbig = 0;
  __syncthreads();
  for (;;) {
    if (staged == 2) {
      const int64_t lim = 8 * (int64_t)P.warp_cap;
      for (;;) {
        if (s_pbig < s_nbig) break;   // block-uniform (read after a barrier)
        __syncthreads();
        if (threadIdx.x == 0) {
          s_nbig = s_pbig = 0;
          s_chunk = st->error ? nb : (int64_t)atomicAdd(&st->big_ticket, (unsigned)blockDim.x);
        }
        __syncthreads();
        const int64_t c0 = s_chunk;
        if (c0 >= nb) break;
        const int64_t bb = c0 + threadIdx.x;
        if (bb < nb && (int64_t)P.bcount[bb] > lim) s_big[atomicAdd(&s_nbig, 1)] = (int)bb;
        __syncthreads();
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      s_abort = 0;
      if (st->error) {
        tile_id = -1;
      } else if (staged == 2) {
        tile_id = s_pbig < s_nbig ? s_big[s_pbig++] : -1;
        if (tile_id >= 0) atomicAdd((unsigned long long*)&st->nbig, 1ull);
      } else if (staged) {        // the buckets the warp kernel deferred
        const int64_t tk = (int64_t)atomicAdd(&st->defer_ticket, 1u);
        tile_id = tk < st->ndefer ? (int)P.att_begin[tk] : -1;
      } else {
        tile_id = (int)atomicAdd(&st->merge_ticket, 1u);
      }
    }
    __syncthreads();
    const int64_t b = tile_id;
    if (b < 0 || b >= nb) break;
    const int64_t s0 = P.boff[b];
    const int64_t ns = P.bcount[b];
    c.m0 = b * sb;
    c.bucket = b;
    const int nm = (int)((c.m0 + sb < n ? c.m0 + sb : n) - c.m0);
    for (int i = threadIdx.x; i < nm; i += blockDim.x) {
#pragma unroll
      for (int j = 0; j < W; ++j) m.mkey[j * SM + i] = key[j * P.cap + c.m0 + i];
    }
    __syncthreads();
    {
      // ---- common path: spawns onto entries of the segment are added into
      // per-entry accumulators (integer sums: order-free); spawns onto new
      // determinants are collected and, whenever the collection fills up,
      // sorted and reduced on chip so repeated keys collapse.
      for (int i = threadIdx.x; i < nm; i += blockDim.x) m.macc[i] = 0;
      if (threadIdx.x == 0) s_nnew = 0;
      __syncthreads();
      int nnew = 0;
      bool over = false;
      for (int64_t base = 0; base < ns; base += blockDim.x) {
        if (nnew + (int)blockDim.x > TC) {
          nnew = sort_reduce<W>(m, TC, nnew, wsum);
          if (nnew + (int)blockDim.x > TC) {
            over = true;   // block-uniform: too many distinct new keys for one tile
            break;
          }
          if (threadIdx.x == 0) s_nnew = nnew;
          __syncthreads();
        }
        const int64_t i = base + threadIdx.x;
        const bool have = i < ns;
        Key<W> k;
        int64_t a = 0;
        uint32_t f = 0;
        bool match = false;
        int idx = 0;
        if (have) {
          k = load_key<W>(P.b_key, P.scap, s0 + i);
          a = P.b_amt[s0 + i];
          f = P.b_flag[s0 + i];
          idx = lb_smem_main<W>(m, SM, 0, nm, k);
          match = idx < nm && key_eq<W>(mkey_at<W>(m, SM, idx), k);
        }
        if (have && match) atomicAdd((unsigned long long*)&m.macc[idx], (unsigned long long)a);
        const unsigned nmask = __ballot_sync(0xffffffffu, have && !match);
        int wbase = 0;
        if (nmask) {
          const int lead = __ffs(nmask) - 1;
          if ((int)warp_lane() == lead) wbase = atomicAdd(&s_nnew, __popc(nmask));
          wbase = __shfl_sync(0xffffffffu, wbase, lead);
        }
        if (have && !match) {
          const int slot = wbase + __popc(nmask & ((1u << warp_lane()) - 1u));
#pragma unroll
          for (int j = 0; j < W; ++j) m.skey[j * TC + slot] = k.w[j];
          m.samt[slot] = a;
          m.sflg[slot] = f;
        }
        __syncthreads();
        nnew = s_nnew;
        __syncthreads();
      }
      if (!over) {
        const int nu = (nnew <= kCountMax && nnew <= (int)blockDim.x) ? count_reduce<W>(m, TC, nnew)
                                                                         : sort_reduce<W>(m, TC, nnew, wsum);
        const uint32_t nkeep = acc_decide<W>(P, m, c, TC, SM, nu, nm, wsum);
        if (staged) {
          if (threadIdx.x == 0) atomicAdd(&P.tile_state[b], (unsigned long long)nkeep);
          nwsum += acc_write<W, SYS>(P, m, c, TC, SM, nu, nm, nkeep, c.m0 + (int64_t)s0);
          continue;
        }
        if (threadIdx.x < 32) {
          int ab = 0;
          const unsigned long long base = lookback_warp(P, b, nkeep, &ab);
          if (threadIdx.x == 0) {
            s_base = base;
            s_abort = ab;
            if (!ab && (int64_t)(base + nkeep) > P.cap) {
              set_error(st, ERR_STATE_CAPACITY);
              s_abort = 1;
            }
            if (!s_abort && b == nb - 1) st->ndet[nxt] = (int64_t)(base + nkeep);
          }
        }
        __syncthreads();
        if (s_abort) break;
        nwsum += acc_write<W, SYS>(P, m, c, TC, SM, nu, nm, nkeep, (int64_t)s_base);
        continue;
      }
      // too many distinct new determinants for one tile: the sub-range path
      // below starts again from the bucket's spawns
    }
    // ---- oversized bucket: split its spawns into key sub-ranges with splitters
    // sampled from the spawns themselves, partition them into the staging
    // arrays, reduce each sub-range on chip, keep the unique runs in the
    // bucket's own region, then merge each run with its share of the segment.
    {
      int R = (int)((ns + TC / 4 - 1) / (TC / 4));
      if (R > kSubRanges) R = kSubRanges;
      int nsamp = R * 8 < TC ? R * 8 : TC;
      int64_t stride = ns / nsamp;
      for (int i = threadIdx.x; i < nsamp; i += blockDim.x) {
        int64_t src = s0 + (int64_t)i * stride;
#pragma unroll
        for (int j = 0; j < W; ++j) m.skey[j * TC + i] = P.b_key[j * P.scap + src];
        m.samt[i] = 0;
        m.sflg[i] = 0;
      }
      __syncthreads();
      int nuq = sort_reduce<W>(m, TC, nsamp, wsum);
      int nsub = R < nuq ? R : nuq;   // sub-ranges; splitters = nsub - 1 evenly spaced samples
      for (int r = threadIdx.x; r < nsub - 1; r += blockDim.x) {
        int at = (int)(((int64_t)(r + 1) * nuq) / nsub);
        Key<W> k = skey_at<W>(m, TC, at);
#pragma unroll
        for (int j = 0; j < W; ++j) m.spl[j * kSubRanges + r] = k.w[j];
      }
      for (int r = threadIdx.x; r <= kSubRanges; r += blockDim.x) {
        m.rcnt[r] = 0;
        m.rcur[r] = 0;
      }
      if (threadIdx.x == 0) s_nsub = nsub;
      __syncthreads();
      // histogram of sub-ranges: r = number of splitters <= key
      for (int64_t i = threadIdx.x; i < ns; i += blockDim.x) {
        Key<W> k = load_key<W>(P.b_key, P.scap, s0 + i);
        int lo = 0, hi = nsub - 1;
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (key_le<W>(spl_at<W>(m, mid), k)) lo = mid + 1;
          else hi = mid;
        }
        atomicAdd(&m.rcnt[lo], 1);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        int acc = 0;
        for (int r = 0; r < nsub; ++r) {
          m.roff[r] = acc;
          acc += m.rcnt[r];
        }
      }
      __syncthreads();
      // partition into the staging arrays (free after the scatter)
      for (int64_t i = threadIdx.x; i < ns; i += blockDim.x) {
        Key<W> k = load_key<W>(P.b_key, P.scap, s0 + i);
        int lo = 0, hi = nsub - 1;
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (key_le<W>(spl_at<W>(m, mid), k)) lo = mid + 1;
          else hi = mid;
        }
        int64_t dst = s0 + m.roff[lo] + atomicAdd(&m.rcur[lo], 1);
        store_key<W>(P.s_key, P.scap, dst, k);
        P.s_amt[dst] = P.b_amt[s0 + i];
        P.s_meta[dst] = P.b_flag[s0 + i];
      }
      __syncthreads();
      // pass 1: reduce each sub-range, store its unique run, count survivors
      int64_t uoff = 0;
      uint32_t total = 0;
      for (int r = 0; r < nsub; ++r) {
        int64_t beg = s0 + m.roff[r];
        int nu = load_reduce<W>(m, TC, P.s_key, P.scap, P.s_amt, nullptr, P.s_meta, beg, beg + m.rcnt[r], wsum);
        if (nu < 0) {
          if (threadIdx.x == 0) {
            set_error(st, ERR_TILE_CAPACITY);
            s_abort = 1;
          }
          __syncthreads();
          break;
        }
        for (int i = threadIdx.x; i < nu; i += blockDim.x) {
          int64_t dst = s0 + uoff + i;
#pragma unroll
          for (int j = 0; j < W; ++j) P.b_key[j * P.scap + dst] = m.skey[j * TC + i];
          P.b_amt[dst] = m.samt[i];
          P.b_flag[dst] = (uint8_t)(m.sflg[i] & 1u);
        }
        int ml = r == 0 ? 0 : lb_smem_main<W>(m, SM, 0, nm, spl_at<W>(m, r - 1));
        int mh = r == nsub - 1 ? nm : lb_smem_main<W>(m, SM, 0, nm, spl_at<W>(m, r));
        int nc = 0;
        uint32_t k = tile_decide<W>(P, m, c, TC, SM, nu, ml, mh, wsum, nc);
        if (threadIdx.x == 0) {
          m.runiq[r] = nu;
          m.rkeep[r] = (int)k;
        }
        uoff += nu;
        total += k;
        __syncthreads();
      }
      if (s_abort) break;
      if (staged) {
        if (threadIdx.x == 0) {
          atomicAdd(&P.tile_state[b], (unsigned long long)total);
          s_base = (unsigned long long)(c.m0 + s0);
        }
      } else if (threadIdx.x < 32) {
        int ab = 0;
        const unsigned long long base = lookback_warp(P, b, total, &ab);
        if (threadIdx.x == 0) {
          s_base = base;
          s_abort = ab;
          if (!ab && (int64_t)(base + total) > P.cap) {
            set_error(st, ERR_STATE_CAPACITY);
            s_abort = 1;
          }
          if (!s_abort && b == nb - 1) st->ndet[nxt] = (int64_t)(base + total);
        }
      }
      __syncthreads();
      if (s_abort) break;
      // pass 2: reload each unique run, decide again (same result), write
      int64_t out = (int64_t)s_base;
      uoff = 0;
      for (int r = 0; r < s_nsub; ++r) {
        int nu = m.runiq[r];
        for (int i = threadIdx.x; i < nu; i += blockDim.x) {
          int64_t src = s0 + uoff + i;
#pragma unroll
          for (int j = 0; j < W; ++j) m.skey[j * TC + i] = P.b_key[j * P.scap + src];
          m.samt[i] = P.b_amt[src];
          m.sflg[i] = P.b_flag[src];
        }
        __syncthreads();
        int ml = r == 0 ? 0 : lb_smem_main<W>(m, SM, 0, nm, spl_at<W>(m, r - 1));
        int mh = r == s_nsub - 1 ? nm : lb_smem_main<W>(m, SM, 0, nm, spl_at<W>(m, r));
        int nc = 0;
        uint32_t k = tile_decide<W>(P, m, c, TC, SM, nu, ml, mh, wsum, nc);
        nwsum += tile_write<W, SYS>(P, m, c, TC, SM, nu, ml, mh, nc, k, out);
        out += k;
        uoff += nu;
      }
    }
  }
  int64_t tot = block_sum<int64_t>(nwsum, sh64);
  if (threadIdx.x == 0 && tot) atomicAdd((unsigned long long*)&st->nw_post, (unsigned long long)tot);
}
template <int W, int SYS>
__global__ void __launch_bounds__(kMergeThreads, (W == 8 ? 2 : 4)) k_merge(Params P, int cur, int staged) { d_merge<W, SYS>(P, cur, staged, VGrid{(int)blockIdx.x, (int)gridDim.x}); }
// the same for replica blockIdx.y of a batch (parameter blocks PP[replica])
template <int W, int SYS>
__global__ void __launch_bounds__(kMergeThreads, (W == 8 ? 2 : 4)) kb_merge(const Params* PP, const int* off, int R, int cur, int staged) {
  __shared__ Params sP;
  __shared__ VGrid vg;
  if (!batch_block(PP, off, R, sP, vg)) return;
  d_merge<W, SYS>(sP, cur, staged, vg);
}

// ------------------------------------------------------------------ finalize
__device__ __forceinline__ void d_finalize(const Params& P, int cur) {
  DevState* st = P.st;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (st->error) return;
  const int64_t t = st->iter + 1;
  const int64_t nw = st->nw_post;
  if (st->vary) {
    if (t % P.period == 0) {
      double ratio = __ddiv_rn((double)nw, (double)st->nw_ref);
      double coef = __ddiv_rn(P.zeta, __dmul_rn((double)P.period, P.tau));
      st->shift = __dsub_rn(st->shift, __dmul_rn(coef, log_series(ratio)));
      st->nw_ref = nw;
    }
  } else if (nw > P.target_fixed) {
    st->vary = 1;
    st->nw_ref = nw;
  }
  Record r;
  r.iter = t;
  r.shift = st->shift;
  r.nw_pre = st->nw_pre;
  r.n0 = st->n0;
  r.nw_post = nw;
  r.ndet = st->ndet[cur ^ 1];
  r.natt = st->natt;
  r.nspawn = st->nspawn;
  r.tau = P.tau;
  st->nspawn_prev = st->nspawn;
  st->nuniq_prev = st->nuniq;
  I128 num{(uint64_t)st->num[0], (int64_t)st->num[1]};
  r.num_lo = num.lo;
  r.num_hi = num.hi;
  r.num = fixed_to_double(num);
  P.rec[(t - 1) % P.rec_cap] = r;
  st->iter = t;
  st->nw_pre = 0;
  st->n0 = 0;
  st->num[0] = 0;
  st->num[1] = 0;
  st->nw_post = 0;
}
static __global__ void k_finalize(Params P, int cur) { d_finalize(P, cur); }
// the same for replica blockIdx.y of a batch (parameter blocks PP[replica])
static __global__ void kb_finalize(const Params* PP, int cur) {
  __shared__ Params sP;
  load_params(sP, PP);
  d_finalize(sP, cur);
}

// diagonal elements of the determinants the merge created (list in natt[])
template <int W, int SYS>
__device__ __forceinline__ void d_new_hdiag(const Params& P, int cur, const VGrid vg) {
  DevState* st = P.st;
  if (st->error) return;
  const int nxt = cur ^ 1;
  const int64_t nn = st->nnew;
  for (int64_t i = (int64_t)vg.b * blockDim.x + threadIdx.x; i < nn; i += (int64_t)vg.n * blockDim.x) {
    int64_t o = P.natt[i];
    Key<W> k = load_key<W>(P.key[nxt], P.cap, o);
    P.hdiag[nxt][o] = __dsub_rn(h_diag<W, SYS>(P.sys, k), st->e_ref);
  }
}
template <int W, int SYS>
__global__ void __launch_bounds__(256) k_new_hdiag(Params P, int cur) { d_new_hdiag<W, SYS>(P, cur, VGrid{(int)blockIdx.x, (int)gridDim.x}); }
// the same for replica blockIdx.y of a batch (parameter blocks PP[replica])
template <int W, int SYS>
__global__ void __launch_bounds__(256) kb_new_hdiag(const Params* PP, const int* off, int R, int cur) {
  __shared__ Params sP;
  __shared__ VGrid vg;
  if (!batch_block(PP, off, R, sP, vg)) return;
  d_new_hdiag<W, SYS>(sP, cur, vg);
}

// ------------------------------------------------------------------ utilities
inline int64_t* st_field_i64(DevState* st, size_t off) { return (int64_t*)((char*)st + off); }

// single-block exclusive scan of int32 counts into int64 offsets (n+1 entries)
static __global__ void k_scan_small(const int32_t* in, int64_t* out, int n) {
  __shared__ int64_t tile[1024];
  __shared__ int64_t wsum[33];
  int64_t carry = 0;
  for (int base = 0; base < n; base += blockDim.x) {
    int i = base + threadIdx.x;
    tile[threadIdx.x] = i < n ? in[i] : 0;
    __syncthreads();
    int64_t tot = block_scan_excl<int64_t>(tile, blockDim.x, wsum);
    if (i < n) out[i] = carry + tile[threadIdx.x];
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}


template <int W, int SYS>
__global__ void k_hdiag(Params P, int cur, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    Key<W> k = load_key<W>(P.key[cur], P.cap, i);
    P.hdiag[cur][i] = __dsub_rn(h_diag<W, SYS>(P.sys, k), P.st->e_ref);
  }
}
template <int W, int SYS>
__global__ void k_eref(Params P) {
  if (threadIdx.x || blockIdx.x) return;
  P.st->e_ref = h_diag<W, SYS>(P.sys, ref_key<W>(P));
}

}  // namespace hande

#include "merge_warp.cuh"
