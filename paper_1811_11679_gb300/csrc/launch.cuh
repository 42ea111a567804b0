// launch.cuh -- per-(key width, system) launchers: the iteration sequence, the
// deterministic-space selection ("high" space, HANDE-QMC paper App. A.2) and
// the CSR build of the deterministic-space Hamiltonian.  Included once per key
// width by inst_w{1,2,8}.cu so the three widths compile in parallel.
#pragma once
#include <cstddef>

#include "engine.h"

namespace hande {

// ------------------------------------------------------------------ CSR of H' inside the core
// H'_rc = <D_r|H|D_c> off the diagonal, H_rr - E_ref on it, for every pair that
// differs in at most two spin orbitals (an element that is exactly zero is kept:
// it adds nothing to the exact product).
template <int W, int SYS>
__device__ __forceinline__ double core_elem(const Params& P, int r, int c, const Key<W>& kr, const Key<W>& kc) {
  if (r == c) return __dsub_rn(h_diag<W, SYS>(P.sys, kr), P.st->e_ref);
  return h_elem<W, SYS>(P.sys, kc, kr);
}
template <int W>
__global__ void k_csr_count(Params P, int32_t* rowcnt) {
  int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (r >= P.ncore) return;
  Key<W> kr = load_key<W>(P.core_key, P.ncore, r);
  int cnt = 0;
  for (int c0 = 0; c0 < P.ncore; c0 += 32) {
    int c = c0 + lane;
    bool nz = false;
    if (c < P.ncore) nz = key_popc_xor<W>(kr, load_key<W>(P.core_key, P.ncore, c)) <= 4;
    cnt += __popc(__ballot_sync(0xffffffffu, nz));
  }
  if (lane == 0) rowcnt[r] = cnt;
}
template <int W, int SYS>
__global__ void k_csr_fill(Params P, int64_t* rowptr, int32_t* col, double* val) {
  int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (r >= P.ncore) return;
  Key<W> kr = load_key<W>(P.core_key, P.ncore, r);
  int64_t o = rowptr[r];
  for (int c0 = 0; c0 < P.ncore; c0 += 32) {
    int c = c0 + lane;
    bool conn = false;
    Key<W> kc;
    if (c < P.ncore) {
      kc = load_key<W>(P.core_key, P.ncore, c);
      conn = key_popc_xor<W>(kr, kc) <= 4;
    }
    unsigned m = __ballot_sync(0xffffffffu, conn);
    if (conn) {
      int64_t e = o + __popc(m & ((1u << lane) - 1u));
      col[e] = c;
      val[e] = core_elem<W, SYS>(P, r, c, kr, kc);
    }
    o += __popc(m);
  }
}
// ------------------------------------------------------------------ selection of the core
template <int W>
__global__ void k_sel_hist(Params P, int cur, int shift, uint64_t mask, uint64_t prefix, unsigned long long* hist) {
  __shared__ unsigned h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const int64_t n = P.st->ndet[cur];
  const Key<W> d0 = ref_key<W>(P);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    Key<W> k = load_key<W>(P.key[cur], P.cap, i);
    if (key_eq<W>(k, d0)) continue;
    uint64_t v = (uint64_t)iabs64(P.pop[cur][i]);
    if ((v & mask) == prefix) atomicAdd(&h[(v >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}
// stage 0: natt[i] = 1 for non-reference entries with |N| == vstar
// stage 1: natt[i] = 1 for the selected entries (att_begin holds the tie ranks)
template <int W>
__global__ void k_sel_flags(Params P, int cur, uint64_t vstar, int64_t need_eq, int stage) {
  const int64_t n = P.st->ndet[cur];
  const Key<W> d0 = ref_key<W>(P);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    Key<W> k = load_key<W>(P.key[cur], P.cap, i);
    bool is0 = key_eq<W>(k, d0);
    uint64_t v = (uint64_t)iabs64(P.pop[cur][i]);
    int64_t r;
    if (stage == 0) {
      r = (!is0 && v == vstar) ? 1 : 0;
    } else {
      r = is0 || v > vstar || (v == vstar && P.att_begin[i] < need_eq);
    }
    P.natt[i] = r;
  }
}
template <int W>
__global__ void k_sel_gather(Params P, int cur, uint64_t* core_key, int64_t ncore) {
  const int64_t n = P.st->ndet[cur];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint8_t f = P.flags[cur][i] & (uint8_t)~F_CORE;
    if (P.natt[i]) {
      Key<W> k = load_key<W>(P.key[cur], P.cap, i);
      store_key<W>(core_key, ncore, P.att_begin[i], k);
      f |= F_CORE;
    }
    P.flags[cur][i] = f;
  }
}

// ------------------------------------------------------------------ launchers
// One iteration.  With `ev` non-null, ev[k] is recorded before phase k and
// ev[kPhases] after the last one (phases: det pass, attempt scan, split, core,
// attempts, bucket scan, scatter, merge, new diagonals, finalize).
template <int W, int SYS>
void enqueue_iteration(Engine& E, int cur, bool core, cudaStream_t s, cudaEvent_t* ev) {
  Params& P = E.P;
  DevState* st = P.st;
  auto mark = [&](int k) {
    if (ev) cudaEventRecord(ev[k], s);
  };
  const bool with_core = core && P.ncore > 0;
  const int ncb = (P.ncore + 255) / 256;
  if (!ev && E.aux_stream) {
    // captured iteration: the bucket split and the deterministic-space product
    // (they read only keys, the core populations and the CSR) run on a second
    // branch beside the det pass and the attempt scan; the core update waits
    // for both (the det pass reads the core populations).  A failing record or
    // wait invalidates the capture, which ending the capture reports.
    (void)(cudaEventRecord(E.ev_fork, s));
    (void)(cudaStreamWaitEvent(E.aux_stream, E.ev_fork, 0));
    k_split<W><<<kScanBlocks, 256, 0, E.aux_stream>>>(P, cur);
    if (with_core) {
      k_core_locate<W><<<ncb, 256, 0, E.aux_stream>>>(P, cur);
      k_core_spmv<<<(int)(((int64_t)P.ncore * 32 + 255) / 256), 256, 0, E.aux_stream>>>(P, cur);
    }
    (void)(cudaEventRecord(E.ev_join, E.aux_stream));
    k_det_pass<W, SYS><<<kScanBlocks, kScanThreads, 0, s>>>(P, cur);
    k_scan_partials_i64<<<1, 1024, 0, s>>>(P.part, kScanBlocks, st_field_i64(st, offsetof(DevState, natt)), st);
    k_scan_apply<int64_t><<<kScanBlocks, kScanThreads, 0, s>>>(
        P.natt, P.att_begin, st_field_i64(st, offsetof(DevState, ndet) + 8 * cur), P.part, st);
    (void)(cudaStreamWaitEvent(s, E.ev_join, 0));
    if (with_core) k_core_apply<<<ncb, 256, 0, s>>>(P, cur);
  } else {
    mark(0);
    k_det_pass<W, SYS><<<kScanBlocks, kScanThreads, 0, s>>>(P, cur);
    mark(1);
    k_scan_partials_i64<<<1, 1024, 0, s>>>(P.part, kScanBlocks, st_field_i64(st, offsetof(DevState, natt)), st);
    k_scan_apply<int64_t><<<kScanBlocks, kScanThreads, 0, s>>>(
        P.natt, P.att_begin, st_field_i64(st, offsetof(DevState, ndet) + 8 * cur), P.part, st);
    mark(2);
    k_split<W><<<kScanBlocks, 256, 0, s>>>(P, cur);
    mark(3);
    if (with_core) {
      k_core_locate<W><<<ncb, 256, 0, s>>>(P, cur);
      k_core_spmv<<<(int)(((int64_t)P.ncore * 32 + 255) / 256), 256, 0, s>>>(P, cur);
      k_core_apply<<<ncb, 256, 0, s>>>(P, cur);
    }
  }
  mark(4);
  k_attempt<W, SYS><<<E.attempt_grid, kAttemptThreads, attempt_smem_bytes<W, SYS>(), s>>>(P, cur);
  mark(5);
  int64_t* nbk = st_field_i64(st, offsetof(DevState, nbuckets));
  k_scan_one<uint32_t, uint32_t><<<1, 1024, 0, s>>>(P.bcount, P.boff, nbk,
                                                    st_field_i64(st, offsetof(DevState, scan_total)), -1, st);
  mark(6);
  k_scatter<W><<<E.attempt_grid * 4, 256, 0, s>>>(P);
  mark(7);
  if (E.merge_warp) {
    if (!ev && E.aux_stream) {   // large buckets on block tiles beside the warp kernel
      (void)cudaEventRecord(E.ev_fork, s);
      (void)cudaStreamWaitEvent(E.aux_stream, E.ev_fork, 0);
      k_merge<W, SYS><<<E.merge_grid, kMergeThreads, E.merge_smem_bytes, E.aux_stream>>>(P, cur, 2);
      (void)cudaEventRecord(E.ev_join, E.aux_stream);
      k_merge_warp<W, SYS><<<E.merge_warp_grid, kMwThreads, E.ops.merge_warp_smem, s>>>(P, cur);
      k_merge<W, SYS><<<E.merge_grid, kMergeThreads, E.merge_smem_bytes, s>>>(P, cur, 1);
      (void)cudaStreamWaitEvent(s, E.ev_join, 0);
    } else {
      k_merge_warp<W, SYS><<<E.merge_warp_grid, kMwThreads, E.ops.merge_warp_smem, s>>>(P, cur);
      k_merge<W, SYS><<<E.merge_grid, kMergeThreads, E.merge_smem_bytes, s>>>(P, cur, 2);
      k_merge<W, SYS><<<E.merge_grid, kMergeThreads, E.merge_smem_bytes, s>>>(P, cur, 1);
    }
    k_scan_one<unsigned long long, unsigned long long><<<1, 1024, 0, s>>>(
        P.tile_state, P.tile_inc, nbk, st_field_i64(st, offsetof(DevState, ndet) + 8 * (cur ^ 1)), P.cap, st,
        st_field_i64(st, offsetof(DevState, nnew)));
    k_merge_copy<W><<<E.attempt_grid * 2, 256, 0, s>>>(P, cur);
  } else {
    k_merge<W, SYS><<<E.merge_grid, kMergeThreads, E.merge_smem_bytes, s>>>(P, cur, 0);
  }
  mark(8);
  k_new_hdiag<W, SYS><<<E.attempt_grid, 256, 0, s>>>(P, cur);
  mark(9);
  k_finalize<<<1, 32, 0, s>>>(P, cur);
  mark(10);
}

// One iteration of every replica of a batch group: the same phases and graph
// branches as enqueue_iteration (captured form).  A planner kernel first
// divides each phase's block budget among the replicas in proportion to their
// work; each phase is then one launch of budget + R blocks in which replica r
// owns the blocks [off[r], off[r + 1]) and reads its parameter block
// G.d_params[r].  Single-block steps (scans, shift update) and the
// deterministic-space kernels run on (blocks, replicas) grids.
template <int W, int SYS>
void enqueue_iteration_batch(BatchGroup& G, int cur, cudaStream_t s, cudaStream_t aux, cudaEvent_t fork,
                             cudaEvent_t join) {
  const Params* PP = G.d_params;
  const int R = G.R;
  const Engine& E0 = *G.eng[0];
  const int ncb = (G.max_ncore + 255) / 256;
  auto off = [&](int p) { return G.d_off + (size_t)p * (R + 1); };
  auto blocks = [&](int p) { return (unsigned)(G.plan.budget[p] + R); };
  kb_plan<<<1, 32, 0, s>>>(PP, R, cur, G.plan, G.d_off);
  (void)cudaEventRecord(fork, s);
  (void)cudaStreamWaitEvent(aux, fork, 0);
  kb_split<W><<<blocks(0), 256, 0, aux>>>(PP, off(0), R, cur);
  if (G.max_ncore > 0) {
    kb_core_locate<W><<<dim3(ncb, R), 256, 0, aux>>>(PP, cur);
    kb_core_spmv<<<dim3((unsigned)(((int64_t)G.max_ncore * 32 + 255) / 256), R), 256, 0, aux>>>(PP, cur);
  }
  (void)cudaEventRecord(join, aux);
  kb_det_pass<W, SYS><<<blocks(0), kScanThreads, 0, s>>>(PP, off(0), R, cur);
  kb_scan_natt<<<dim3(1, R), 1024, 0, s>>>(PP, off(0), R);
  kb_scan_att<<<blocks(0), kScanThreads, 0, s>>>(PP, off(0), R, cur);
  (void)cudaStreamWaitEvent(s, join, 0);
  if (G.max_ncore > 0) kb_core_apply<<<dim3(ncb, R), 256, 0, s>>>(PP, cur);
  kb_attempt<W, SYS><<<blocks(1), kAttemptThreads, attempt_smem_bytes<W, SYS>(), s>>>(PP, off(1), R, cur);
  kb_scan_buckets<<<dim3(1, R), 1024, 0, s>>>(PP);
  kb_scatter<W><<<blocks(2), 256, 0, s>>>(PP, off(2), R);
  if (E0.merge_warp) {
    (void)cudaEventRecord(fork, s);
    (void)cudaStreamWaitEvent(aux, fork, 0);
    kb_merge<W, SYS><<<blocks(4), kMergeThreads, E0.merge_smem_bytes, aux>>>(PP, off(4), R, cur, 2);
    (void)cudaEventRecord(join, aux);
    kb_merge_warp<W, SYS><<<blocks(3), kMwThreads, E0.ops.merge_warp_smem, s>>>(PP, off(3), R, cur);
    kb_merge<W, SYS><<<blocks(4), kMergeThreads, E0.merge_smem_bytes, s>>>(PP, off(4), R, cur, 1);
    (void)cudaStreamWaitEvent(s, join, 0);
    kb_scan_kept<<<dim3(1, R), 1024, 0, s>>>(PP, cur);
    kb_merge_copy<W><<<blocks(5), 256, 0, s>>>(PP, off(5), R, cur);
  } else {
    kb_merge<W, SYS><<<blocks(4), kMergeThreads, E0.merge_smem_bytes, s>>>(PP, off(4), R, cur, 0);
  }
  kb_new_hdiag<W, SYS><<<blocks(6), 256, 0, s>>>(PP, off(6), R, cur);
  kb_finalize<<<dim3(1, R), 32, 0, s>>>(PP, cur);
}

template <int W, int SYS>
void enqueue_hdiag(Engine& E, int cur, int64_t n, cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_hdiag<W, SYS><<<blocks, 256, 0, s>>>(E.P, cur, n);
}
template <int W, int SYS>
void enqueue_eref(Engine& E, cudaStream_t s) {
  k_eref<W, SYS><<<1, 32, 0, s>>>(E.P);
}
template <int W, int SYS>
void enqueue_csr_count(Engine& E, int32_t* rowcnt, cudaStream_t s) {
  int blocks = (int)(((int64_t)E.P.ncore * 32 + 255) / 256);
  k_csr_count<W><<<blocks, 256, 0, s>>>(E.P, rowcnt);
}
template <int W, int SYS>
void enqueue_csr_fill(Engine& E, cudaStream_t s) {
  int blocks = (int)(((int64_t)E.P.ncore * 32 + 255) / 256);
  k_csr_fill<W, SYS><<<blocks, 256, 0, s>>>(E.P, E.core_rowptr, E.core_col, E.core_val);
}
template <int W>
void enqueue_sel_hist(Engine& E, int cur, int shift, uint64_t mask, uint64_t prefix, unsigned long long* hist,
                      cudaStream_t s) {
  k_sel_hist<W><<<4 * 152, 256, 0, s>>>(E.P, cur, shift, mask, prefix, hist);
}
template <int W>
void enqueue_sel_flags(Engine& E, int cur, uint64_t vstar, int64_t need_eq, int stage, cudaStream_t s) {
  k_sel_flags<W><<<4 * 152, 256, 0, s>>>(E.P, cur, vstar, need_eq, stage);
}
template <int W>
void enqueue_core_hash(Engine& E, uint32_t* table, cudaStream_t s) {
  k_core_hash<W><<<(E.P.ncore + 255) / 256, 256, 0, s>>>(E.P, table);
}
template <int W>
void enqueue_sel_gather(Engine& E, int cur, uint64_t* core_key, int64_t ncore, cudaStream_t s) {
  k_sel_gather<W><<<4 * 152, 256, 0, s>>>(E.P, cur, core_key, ncore);
}

// ------------------------------------------------------------------ walker-list transfer
// keys of a host-supplied list (array of structures, word j of key i at i W + j):
// bit 0 a bit beyond the spin orbitals, bit 1 wrong electron numbers, bit 2 not
// strictly ascending, bit 3 the reference present
template <int W>
__global__ void k_check_keys(const uint64_t* aos, int64_t n, int nspin, int nalpha, int nbeta, Key<W> d0,
                             unsigned* out) {
  unsigned bits = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    Key<W> k;
    int na = 0, nb = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
      k.w[j] = aos[i * W + j];
      const int lo = 64 * j;
      if (nspin - lo < 64 && (nspin - lo <= 0 ? k.w[j] != 0 : (k.w[j] >> (nspin - lo)) != 0)) bits |= 1u;
      na += __popcll(k.w[j] & 0x5555555555555555ull);
      nb += __popcll(k.w[j] & 0xAAAAAAAAAAAAAAAAull);
    }
    if (na != nalpha || nb != nbeta) bits |= 2u;
    if (key_eq<W>(k, d0)) bits |= 8u;
    if (i > 0) {
      Key<W> pk;
#pragma unroll
      for (int j = 0; j < W; ++j) pk.w[j] = aos[(i - 1) * W + j];
      if (!key_lt<W>(pk, k)) bits |= 4u;
    }
  }
  if (bits) atomicOr(out, bits);
}
// array of structures <-> the list's structure of arrays (key word j at j cap + i)
template <int W>
__global__ void k_keys_to_soa(const uint64_t* aos, uint64_t* soa, int64_t n, int64_t cap) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int j = 0; j < W; ++j) soa[(size_t)j * cap + i] = aos[i * W + j];
  }
}
template <int W>
__global__ void k_keys_to_aos(const uint64_t* soa, uint64_t* aos, int64_t n, int64_t cap) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int j = 0; j < W; ++j) aos[i * W + j] = soa[(size_t)j * cap + i];
  }
}
template <int W>
void enqueue_check_keys(Engine& E, const uint64_t* aos, int64_t n, unsigned* out, cudaStream_t s) {
  Key<W> d0;
#pragma unroll
  for (int j = 0; j < W; ++j) d0.w[j] = E.P.d0[j];
  k_check_keys<W><<<4 * 152, 256, 0, s>>>(aos, n, E.P.sys.nspin, E.nalpha, E.nbeta, d0, out);
}
template <int W>
void enqueue_keys_to_soa(Engine& E, const uint64_t* aos, uint64_t* soa, int64_t n, int64_t stride, cudaStream_t s) {
  k_keys_to_soa<W><<<4 * 152, 256, 0, s>>>(aos, soa, n, stride);
}
template <int W>
void enqueue_keys_to_aos(Engine& E, const uint64_t* soa, uint64_t* aos, int64_t n, int64_t stride, cudaStream_t s) {
  k_keys_to_aos<W><<<4 * 152, 256, 0, s>>>(soa, aos, n, stride);
}
// core flags from given core keys (restart): every list entry's core bit is
// cleared, then each core key is found by binary search and flagged
template <int W>
__global__ void k_core_clear(Params P, int cur) {
  const int64_t n = P.st->ndet[cur];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    P.flags[cur][i] &= (uint8_t)~F_CORE;
}
template <int W>
__global__ void k_core_mark(Params P, int cur, unsigned* missing) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= P.ncore) return;
  const int64_t n = P.st->ndet[cur];
  const Key<W> k = load_key<W>(P.core_key, P.ncore, r);
  const int64_t pos = lower_bound_main<W>(P.key[cur], P.cap, n, k);
  if (pos < n && key_eq<W>(load_key<W>(P.key[cur], P.cap, pos), k)) P.flags[cur][pos] |= F_CORE;
  else atomicOr(missing, 1u);
}
template <int W>
void enqueue_core_mark(Engine& E, int cur, unsigned* missing, cudaStream_t s) {
  k_core_clear<W><<<4 * 152, 256, 0, s>>>(E.P, cur);
  if (E.P.ncore > 0) k_core_mark<W><<<(E.P.ncore + 255) / 256, 256, 0, s>>>(E.P, cur, missing);
}

template <int W>
size_t merge_smem_w(int tc, int sm) {
  return merge_smem_bytes<W>(tc, sm);
}

template <int W, int SYS>
Ops make_ops() {
  Ops o;
  o.iteration = &enqueue_iteration<W, SYS>;
  o.iteration_batch = &enqueue_iteration_batch<W, SYS>;
  o.batch_attempt_kernel = (const void*)&kb_attempt<W, SYS>;
  o.batch_merge_kernel = (const void*)&kb_merge<W, SYS>;
  o.batch_merge_warp_kernel = (const void*)&kb_merge_warp<W, SYS>;
  o.hdiag = &enqueue_hdiag<W, SYS>;
  o.eref = &enqueue_eref<W, SYS>;
  o.csr_count = &enqueue_csr_count<W, SYS>;
  o.csr_fill = &enqueue_csr_fill<W, SYS>;
  o.sel_gather = &enqueue_sel_gather<W>;
  o.check_keys = &enqueue_check_keys<W>;
  o.keys_to_soa = &enqueue_keys_to_soa<W>;
  o.keys_to_aos = &enqueue_keys_to_aos<W>;
  o.core_mark = &enqueue_core_mark<W>;
  o.core_hash = &enqueue_core_hash<W>;
  o.sel_hist = &enqueue_sel_hist<W>;
  o.sel_flags = &enqueue_sel_flags<W>;
  o.merge_smem = &merge_smem_w<W>;
  o.merge_kernel = (const void*)&k_merge<W, SYS>;
  o.merge_warp_kernel = (const void*)&k_merge_warp<W, SYS>;
  o.merge_warp_smem = merge_warp_smem_bytes<W>();
  o.merge_warp_main = MwDims<W>::kMain;
  o.merge_warp_new = MwDims<W>::kNew;
  o.attempt_kernel = (const void*)&k_attempt<W, SYS>;
  o.attempt_smem = attempt_smem_bytes<W, SYS>();
  return o;
}

template <int W>
Ops ops_for(int kind) {
  if (kind == SYS_HUBBARD) return make_ops<W, SYS_HUBBARD>();
  if (kind == SYS_UEG) return make_ops<W, SYS_UEG>();
  return make_ops<W, SYS_MOLECULE>();
}

}  // namespace hande
