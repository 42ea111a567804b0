// merge_warp.cuh -- annihilation with one warp per bucket (every key width).
//
// The annihilation step (HANDE-QMC paper Sec. 2.4 and App. B: combine the
// spawned particles on each determinant, merge them into the sorted main list,
// apply the initiator rule to new determinants) for one bucket: the main-list
// segment [b sb, (b+1) sb) and the spawns whose keys fall in its splitter range.
// A warp owns the whole bucket, so no step needs a block barrier:
//   1. the segment's keys go to the warp's shared-memory tile;
//   2. each spawn finds its key in the segment (binary search): spawns onto
//      listed determinants are added into per-entry integer accumulators (order-
//      free), spawns onto new determinants are staged;
//   3. the staged spawns are sorted in registers (bitonic network over the
//      warp, shuffles across lanes) and equal keys combined (amounts summed,
//      initiator bits OR-ed);
//   4. every candidate gets its merged rank (own index + keys of the other list
//      below it), its final population (spawns added, real-weight occupation
//      rounding) and a keep bit; kept entries are counted;
//   5. the kept entries are written, in merged order, to a staging list at an
//      upper bound of the bucket's output offset (b sb + the spawns of the
//      buckets before b), so no bucket waits for another.
// A bucket with more spawns than a warp should take (8 x the staging) goes to
// the block kernel (k_merge in staged mode 2: 256 threads, sub-ranges for very
// large buckets), which runs beside this kernel; a bucket whose distinct new
// keys overflow the staging is deferred to a second block-kernel pass after it
// (staged mode 1).  Both write to the same staging list.  A one-block scan of the kept counts
// (k_scan_one) then gives every bucket its output offset, and a coalesced copy
// compacts the staging list into the new main list.
#pragma once

namespace hande {

constexpr int kMwThreads = 256;   // 8 warps per CTA
constexpr int kMwWarps = kMwThreads / 32;

// Tile shape per key width: main-list entries per bucket (segment length cap)
// and staged spawns onto new determinants per warp.  512-bit keys take half of
// each, so that two CTAs (16 warps) fit on an SM as for the narrower keys.
template <int W>
struct MwDims {
  static constexpr int kMain = W == 8 ? 96 : 192;
  static constexpr int kNew = W == 8 ? 64 : 128;
  static constexpr int kKeepWords = (kMain + kNew + 31) / 32;
  static constexpr int kMinBlocks = W == 8 ? 2 : 3;   // CTAs per SM the registers are sized for
  static_assert(kKeepWords <= 32, "keep words are scanned by one warp");
  static_assert(kNew <= 128, "the register sort takes at most 128 staged keys");
};

template <int W>
struct WarpTile {
  static constexpr int kMain = MwDims<W>::kMain;
  static constexpr int kNew = MwDims<W>::kNew;
  uint64_t mkey[W][kMain];     // segment keys
  int64_t macc[kMain];         // population plus the spawns onto the entry, then its final value
  double mhd[kMain];           // segment entries' H_ii - E_ref
  uint64_t nkey[W][kNew];      // staged keys of new determinants (sorted unique after dedupe)
  int64_t namt[kNew];
  uint32_t nflg[kNew];         // bit 0: an initiator parent
  int16_t mrank[kMain];        // merged rank of a segment entry
  int16_t nrank[kNew];         // merged rank of a new key
  uint8_t mflg[kMain];         // segment entry flags
  uint32_t keep[MwDims<W>::kKeepWords];  // keep bits by merged rank
  uint32_t kpre[MwDims<W>::kKeepWords];  // kept entries before each word
  int16_t rq[kMain + kNew];    // entries awaiting their occupation-rounding draw
};

template <int W>
__host__ __device__ constexpr size_t merge_warp_tile_bytes() {
  return (sizeof(WarpTile<W>) + 15) & ~(size_t)15;
}
template <int W>
__host__ __device__ constexpr size_t merge_warp_smem_bytes() {
  return (size_t)kMwWarps * merge_warp_tile_bytes<W>();
}

template <int W>
__device__ __forceinline__ Key<W> wt_mkey(const WarpTile<W>& t, int i) {
  Key<W> k;
#pragma unroll
  for (int j = 0; j < W; ++j) k.w[j] = t.mkey[j][i];
  return k;
}
template <int W>
__device__ __forceinline__ Key<W> wt_nkey(const WarpTile<W>& t, int i) {
  Key<W> k;
#pragma unroll
  for (int j = 0; j < W; ++j) k.w[j] = t.nkey[j][i];
  return k;
}
// first index in [lo, hi) whose segment key is >= k
template <int W>
__device__ __forceinline__ int wt_lb_main(const WarpTile<W>& t, int lo, int hi, const Key<W>& k) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (key_lt<W>(wt_mkey<W>(t, mid), k)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
// number of the first u (sorted) new keys below k
template <int W>
__device__ __forceinline__ int wt_lb_new(const WarpTile<W>& t, int u, const Key<W>& k) {
  int lo = 0, hi = u;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (key_lt<W>(wt_nkey<W>(t, mid), k)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// strict order of (key, slot) pairs with the padding slots (-1) after all keys
template <int W>
__device__ __forceinline__ bool sd_less(const Key<W>& a, int ai, const Key<W>& b, int bi) {
  if (ai < 0) return false;
  if (bi < 0) return true;
  return key_lt<W>(a, b);
}

// Sort the n <= 32 E staged entries by key (bitonic network over 32 E slots,
// slot i = lane E + e held by the lane in registers) and combine equal keys.
// On return entries [0, u) are the sorted unique keys; returns u.
template <int W, int E>
__device__ int wt_sort_dedupe_e(WarpTile<W>& t, int n, int lane) {
  Key<W> k[E];
  int ix[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = lane * E + e;
    ix[e] = i < n ? i : -1;
#pragma unroll
    for (int j = 0; j < W; ++j) k[e].w[j] = i < n ? t.nkey[j][i] : 0ull;
  }
  constexpr int N2 = 32 * E;
#pragma unroll
  for (int kk = 2; kk <= N2; kk <<= 1) {
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
      if (j >= E) {   // partner slot i ^ j lives in lane ^ (j / E), same e
        const int lm = j / E;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          Key<W> pk;
#pragma unroll
          for (int w = 0; w < W; ++w) pk.w[w] = __shfl_xor_sync(0xffffffffu, k[e].w[w], lm);
          const int pi = __shfl_xor_sync(0xffffffffu, ix[e], lm);
          const int i = lane * E + e;
          const bool keep_min = ((i & j) == 0) == ((i & kk) == 0);
          const bool take = keep_min ? sd_less<W>(pk, pi, k[e], ix[e]) : sd_less<W>(k[e], ix[e], pk, pi);
          if (take) {
            k[e] = pk;
            ix[e] = pi;
          }
        }
      } else {        // partner slot in the same lane
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if (e & j) continue;
          const int e2 = e | j;
          const int i = lane * E + e;
          const bool asc = (i & kk) == 0;
          const bool sw = asc ? sd_less<W>(k[e2], ix[e2], k[e], ix[e]) : sd_less<W>(k[e], ix[e], k[e2], ix[e2]);
          if (sw) {
            const Key<W> tk = k[e];
            k[e] = k[e2];
            k[e2] = tk;
            const int ti = ix[e];
            ix[e] = ix[e2];
            ix[e2] = ti;
          }
        }
      }
    }
  }
  // heads of equal-key runs, their exclusive count over the warp
  Key<W> up;
#pragma unroll
  for (int w = 0; w < W; ++w) up.w[w] = __shfl_up_sync(0xffffffffu, k[E - 1].w[w], 1);
  bool head[E];
  int nh = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const bool first = lane == 0 && e == 0;
    const Key<W>& pk = e ? k[e - 1] : up;
    head[e] = ix[e] >= 0 && (first || !key_eq<W>(pk, k[e]));
    nh += head[e] ? 1 : 0;
  }
  int incl = nh;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int u = __shfl_sync(0xffffffffu, incl, 31);
  int run = incl - nh;
  int64_t a[E];
  uint32_t f[E];
  int uid[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    a[e] = 0;
    f[e] = 0;
    if (ix[e] >= 0) {
      a[e] = t.namt[ix[e]];
      f[e] = t.nflg[ix[e]];
    }
    run += head[e] ? 1 : 0;
    uid[e] = run - 1;
  }
  __syncwarp();
  for (int i = lane; i < u; i += 32) {
    t.namt[i] = 0;
    t.nflg[i] = 0;
  }
  __syncwarp();
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (ix[e] < 0) continue;
    if (head[e]) {
#pragma unroll
      for (int w = 0; w < W; ++w) t.nkey[w][uid[e]] = k[e].w[w];
    }
    atomicAdd((unsigned long long*)&t.namt[uid[e]], (unsigned long long)a[e]);
    if (f[e] & 1u) atomicOr(&t.nflg[uid[e]], 1u);
  }
  __syncwarp();
  return u;
}

template <int W>
__device__ __forceinline__ int wt_sort_dedupe(WarpTile<W>& t, int n, int lane) {
  if (n <= 1) return n;
  if (n <= 32) return wt_sort_dedupe_e<W, 1>(t, n, lane);
  if (MwDims<W>::kNew <= 64 || n <= 64) return wt_sort_dedupe_e<W, 2>(t, n, lane);   // n <= kNew
  if constexpr (MwDims<W>::kNew > 64) return wt_sort_dedupe_e<W, 4>(t, n, lane);
  return n;
}

// Decide one merge segment: the segment entries [mi, mh) and the unique new
// keys [0, u) (all between the same neighbours).  Merged ranks, final
// populations, keep bits and their per-word prefix.  Segment entries keep their
// slot if core or reference, otherwise they survive with a nonzero population
// after the occupation rounding; new determinants need an initiator parent
// (Sec. 2.1) and a nonzero amount.  Entries that need the rounding draw
// (0 < |N| < 1 walker, real weights) are queued and drawn 32 at a time, so the
// Philox rounds run on full warps.  Returns the number kept.
template <int W>
__device__ uint32_t wt_decide(const Params& P, WarpTile<W>& t, const MergeCtx& c, int mi, int mh, int u, int lane) {
  const int nc = (mh - mi) + u;
  const int nw = (nc + 31) >> 5;
  for (int w = lane; w < nw; w += 32) t.keep[w] = 0;
  __syncwarp();
  const unsigned below = (1u << lane) - 1u;
  int qn = 0;
  for (int i0 = mi; i0 < mh; i0 += 32) {
    const int i = i0 + lane;
    bool need = false;
    if (i < mh) {
      const int r = (i - mi) + wt_lb_new<W>(t, u, wt_mkey<W>(t, i));
      const int64_t p = t.macc[i];
      const bool always = (t.mflg[i] & (F_CORE | F_REF)) != 0;
      need = !always && P.real_amp && p != 0 && iabs64(p) < kOne;
      t.mrank[i] = (int16_t)r;
      if (always || (p != 0 && !need)) atomicOr(&t.keep[r >> 5], 1u << (r & 31));
    }
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (need) t.rq[qn + __popc(m & below)] = (int16_t)i;
    qn += __popc(m);
  }
  for (int j0 = 0; j0 < u; j0 += 32) {
    const int j = j0 + lane;
    bool need = false;
    if (j < u) {
      const int r = j + (wt_lb_main<W>(t, mi, mh, wt_nkey<W>(t, j)) - mi);
      const int64_t p = t.namt[j];
      const bool ok = (!P.initiator || (t.nflg[j] & 1u)) && p != 0;
      need = ok && P.real_amp && iabs64(p) < kOne;
      t.nrank[j] = (int16_t)r;
      if (ok && !need) atomicOr(&t.keep[r >> 5], 1u << (r & 31));
      if (!ok) t.namt[j] = 0;
    }
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (need) t.rq[qn + __popc(m & below)] = (int16_t)(WarpTile<W>::kMain + j);
    qn += __popc(m);
  }
  __syncwarp();
  // occupation rounding (R-13) of the queued entries, full warps
  for (int q0 = 0; q0 < qn; q0 += 32) {
    if (q0 + lane < qn) {
      const int x = t.rq[q0 + lane];
      const bool isnew = x >= WarpTile<W>::kMain;
      const int idx = isnew ? x - WarpTile<W>::kMain : x;
      const Key<W> k = isnew ? wt_nkey<W>(t, idx) : wt_mkey<W>(t, idx);
      const int64_t p = round_small<W>(P, c.t, k, isnew ? t.namt[idx] : t.macc[idx]);
      if (isnew) t.namt[idx] = p;
      else t.macc[idx] = p;
      const int r = isnew ? t.nrank[idx] : t.mrank[idx];
      if (p != 0) atomicOr(&t.keep[r >> 5], 1u << (r & 31));
    }
  }
  __syncwarp();
  const int cnt = lane < nw ? __popc(t.keep[lane]) : 0;
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane < nw) t.kpre[lane] = (uint32_t)(incl - cnt);
  __syncwarp();
  return (uint32_t)__shfl_sync(0xffffffffu, incl, 31);
}

// Write the entries wt_decide kept to the staging list at out + their rank
// among the kept (new determinants flagged F_NEWDET, counted in *nnew_out, all lanes).
// Returns the sum of |N|.
template <int W>
__device__ int64_t wt_write(const Params& P, WarpTile<W>& t, int mi, int mh, int u, int64_t out, int lane,
                            uint32_t* nnew_out) {
  uint32_t nn = 0;
  DevState* st = P.st;
  int64_t nws = 0;
  for (int i = mi + lane; i < mh; i += 32) {
    const int r = t.mrank[i];
    const uint32_t wv = t.keep[r >> 5];
    if (!((wv >> (r & 31)) & 1u)) continue;
    const int64_t o = out + t.kpre[r >> 5] + __popc(wv & ((1u << (r & 31)) - 1u));
    const int64_t p = t.macc[i];
    if (iabs64(p) >= (int64_t(1) << 62)) set_error(st, ERR_OVERFLOW);
    store_key<W>(P.m_key, P.mcap, o, wt_mkey<W>(t, i));
    P.m_pop[o] = p;
    P.m_hd[o] = t.mhd[i];
    P.m_flg[o] = t.mflg[i] & F_CORE;
    nws += iabs64(p);
  }
  for (int j = lane; j < u; j += 32) {
    const int r = t.nrank[j];
    const uint32_t wv = t.keep[r >> 5];
    if (!((wv >> (r & 31)) & 1u)) continue;
    const int64_t o = out + t.kpre[r >> 5] + __popc(wv & ((1u << (r & 31)) - 1u));
    const int64_t p = t.namt[j];
    if (iabs64(p) >= (int64_t(1) << 62)) set_error(st, ERR_OVERFLOW);
    store_key<W>(P.m_key, P.mcap, o, wt_nkey<W>(t, j));
    P.m_pop[o] = p;
    P.m_hd[o] = 0.0;   // H_ii - E_ref follows in k_new_hdiag
    P.m_flg[o] = F_NEWDET;
    nws += iabs64(p);
    ++nn;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
  *nnew_out = nn;
  return nws;
}

// One warp per bucket, buckets taken from a ticket counter (see the file comment).
template <int W, int SYS>
__device__ __forceinline__ void d_merge_warp(const Params& P, int cur, const VGrid vg) {
  DevState* st = P.st;
  extern __shared__ __align__(16) unsigned char mw_smem[];
  const int lane = (int)(threadIdx.x & 31), wid = (int)(threadIdx.x >> 5);
  WarpTile<W>& t = *reinterpret_cast<WarpTile<W>*>(mw_smem + (size_t)wid * merge_warp_tile_bytes<W>());
  const int cap = P.warp_cap;
  const int64_t n = st->ndet[cur];
  const int64_t nb = st->nbuckets;
  const int64_t sb = st->sb;
  MergeCtx c{};   // output fields unused: the buckets go to the staging list
  c.t = st->iter + 1;
  c.pop = P.pop[cur];
  c.hd = P.hdiag[cur];
  c.fl = P.flags[cur];
  const uint64_t* key = P.key[cur];
  int64_t nwsum = 0;
  for (;;) {
    int64_t b = 0;
    if (lane == 0) b = st->error ? -1 : (int64_t)atomicAdd(&st->merge_ticket, 1u);
    b = __shfl_sync(0xffffffffu, b, 0);
    if (b < 0 || b >= nb) break;
    const int64_t s0 = P.boff[b];
    const int64_t ns = P.bcount[b];
    if (ns > 8 * (int64_t)cap) continue;   // large bucket: block tiles take it (k_merge, staged 2)
    c.m0 = b * sb;
    const int nm = (int)((c.m0 + sb < n ? c.m0 + sb : n) - c.m0);
#pragma unroll 2
    for (int i = lane; i < nm; i += 32) {
      const int64_t gi = c.m0 + i;
#pragma unroll
      for (int j = 0; j < W; ++j) t.mkey[j][i] = key[j * P.cap + gi];
      t.macc[i] = c.pop[gi];
      t.mflg[i] = c.fl[gi];
      t.mhd[i] = c.hd[gi];
    }
    __syncwarp();
    // spawns onto segment entries into the accumulators, the others staged
    int nnew = 0;
    bool over = false;
    for (int64_t c0 = 0; c0 < ns; c0 += 32) {
      const int64_t i = c0 + lane;
      const bool have = i < ns;
      Key<W> k;
#pragma unroll
      for (int j = 0; j < W; ++j) k.w[j] = 0;
      int64_t a = 0;
      uint32_t f = 0;
      bool match = false;
      if (have) {
        k = load_key<W>(P.b_key, P.scap, s0 + i);
        a = P.b_amt[s0 + i];
        f = P.b_flag[s0 + i];
        const int j = wt_lb_main<W>(t, 0, nm, k);
        match = j < nm && key_eq<W>(wt_mkey<W>(t, j), k);
        if (match) atomicAdd((unsigned long long*)&t.macc[j], (unsigned long long)a);
      }
      const unsigned mask = __ballot_sync(0xffffffffu, have && !match);
      if (nnew + __popc(mask) > cap) {
        nnew = wt_sort_dedupe<W>(t, nnew, lane);
        if (nnew + __popc(mask) > cap) {
          over = true;
          break;
        }
      }
      if (have && !match) {
        const int s = nnew + __popc(mask & ((1u << lane) - 1u));
#pragma unroll
        for (int j = 0; j < W; ++j) t.nkey[j][s] = k.w[j];
        t.namt[s] = a;
        t.nflg[s] = f;
      }
      nnew += __popc(mask);
      __syncwarp();
    }
    const int64_t out = c.m0 + (int64_t)P.boff[b];   // upper bound of the bucket's offset
    if (over) {   // too many distinct new keys for the staging: the block kernel takes it
      if (lane == 0) {
        P.att_begin[atomicAdd((unsigned long long*)&st->ndefer, 1ull)] = b;
        atomicAdd((unsigned long long*)&st->nuniq, (unsigned long long)(cap + 1));   // at least
      }
      continue;
    }
    const int u = wt_sort_dedupe<W>(t, nnew, lane);
    if (lane == 0) atomicAdd((unsigned long long*)&st->nuniq, (unsigned long long)u);
    const uint32_t nkeep = wt_decide<W>(P, t, c, 0, nm, u, lane);
    uint32_t nnw = 0;
    nwsum += wt_write<W>(P, t, 0, nm, u, out, lane, &nnw);
    if (lane == 0) P.tile_state[b] = (unsigned long long)nkeep | ((unsigned long long)nnw << 32);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) nwsum += __shfl_xor_sync(0xffffffffu, nwsum, o);
  if (lane == 0 && nwsum) atomicAdd((unsigned long long*)&st->nw_post, (unsigned long long)nwsum);
}
template <int W, int SYS>
__global__ void __launch_bounds__(kMwThreads, MwDims<W>::kMinBlocks) k_merge_warp(Params P, int cur) { d_merge_warp<W, SYS>(P, cur, VGrid{(int)blockIdx.x, (int)gridDim.x}); }
// the same for replica blockIdx.y of a batch (parameter blocks PP[replica])
template <int W, int SYS>
__global__ void __launch_bounds__(kMwThreads, MwDims<W>::kMinBlocks) kb_merge_warp(const Params* PP, const int* off, int R, int cur) {
  __shared__ Params sP;
  __shared__ VGrid vg;
  if (!batch_block(PP, off, R, sP, vg)) return;
  d_merge_warp<W, SYS>(sP, cur, vg);
}

// Compact the staged bucket lists into the new main list (one warp per bucket,
// coalesced) and list the new determinants (natt[]) for their diagonals.  The
// bucket's packed scan result gives both its output offset (low 32 bits) and
// its offset in the new-determinant list (high 32 bits).
template <int W>
__device__ __forceinline__ void d_merge_copy(const Params& P, int cur, const VGrid vg) {
  DevState* st = P.st;
  if (st->error) return;
  const int nxt = cur ^ 1;
  const int64_t nb = st->nbuckets, sb = st->sb;
  const int lane = (int)(threadIdx.x & 31);
  const int64_t nwarps = ((int64_t)vg.n * blockDim.x) >> 5;
  uint64_t* okey = P.key[nxt];
  for (int64_t b = ((int64_t)vg.b * blockDim.x + threadIdx.x) >> 5; b < nb; b += nwarps) {
    const int64_t src = b * sb + (int64_t)P.boff[b];
    const int64_t dst = (int64_t)(P.tile_inc[b] & 0xffffffffull);   // output offset
    int64_t nslot = (int64_t)(P.tile_inc[b] >> 32);                  // offset in the new-determinant list
    const int64_t cnt = (int64_t)(P.tile_state[b] & 0xffffffffull);
    // four groups of 32 entries per step: all loads first, then the stores
    for (int64_t i0 = 0; i0 < cnt; i0 += 128) {
      Key<W> kk[4];
      int64_t pp[4];
      double hh[4];
      uint8_t ff[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + u * 32 + lane;
        if (i < cnt) {
          kk[u] = load_key<W>(P.m_key, P.mcap, src + i);
          pp[u] = P.m_pop[src + i];
          hh[u] = P.m_hd[src + i];
          ff[u] = P.m_flg[src + i];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + u * 32 + lane;
        const int64_t o = dst + i;
        bool isnew = false;
        if (i < cnt) {
          store_key<W>(okey, P.cap, o, kk[u]);
          P.pop[nxt][o] = pp[u];
          P.hdiag[nxt][o] = hh[u];
          P.flags[nxt][o] = ff[u] & F_CORE;
          isnew = (ff[u] & F_NEWDET) != 0;
        }
        const unsigned m = __ballot_sync(0xffffffffu, isnew);
        if (isnew) P.natt[nslot + __popc(m & ((1u << lane) - 1u))] = o;
        nslot += __popc(m);
      }
    }
  }
}
template <int W>
__global__ void __launch_bounds__(256) k_merge_copy(Params P, int cur) { d_merge_copy<W>(P, cur, VGrid{(int)blockIdx.x, (int)gridDim.x}); }
// the same for replica blockIdx.y of a batch (parameter blocks PP[replica])
template <int W>
__global__ void __launch_bounds__(256) kb_merge_copy(const Params* PP, const int* off, int R, int cur) {
  __shared__ Params sP;
  __shared__ VGrid vg;
  if (!batch_block(PP, off, R, sP, vg)) return;
  d_merge_copy<W>(sP, cur, vg);
}

}  // namespace hande
