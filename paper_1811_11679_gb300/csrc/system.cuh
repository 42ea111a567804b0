// system.cuh -- Hamiltonians, Slater-Condon matrix elements and excitation
// generators on the device, templated on key width W and system kind.
//
// Matrix elements follow the Slater-Condon rules for the Hamiltonian of the
// FCIQMC propagation (HANDE-QMC paper, Sec. 2.1 Eq. (fciqmc)):
//   diagonal  sum_k h_kk + sum_{k<l} [(kk|ll) - (kl|lk)]
//   single    sign * (h_ia + sum_{k in D, k != i} [(ia|kk) - (ik|ka)])
//   double    sign * [(ia|jb) - (ib|ja)]          (i<j -> a<b)
// with sign = (-1)^(occupied orbitals strictly between i and a), then the
// same for j -> b on the updated string.  Every sum runs in ascending orbital
// order with round-to-nearest intrinsics, so each element has one defined value.
//
// Generators (Sec. 2.4 "spawning": random selection of a connected state with
// its generation probability) return the child and the factor tau / p_gen:
//   Hubbard   : uniform electron, uniform direction, p = 1/(2N)
//   UEG       : uniform pair (i<j), uniform a of spin(i), b fixed by momentum,
//               p = (2 if same spin else 1) / (C(N,2) M)
//   molecule  : single with probability p_s (uniform i, uniform empty a of
//               spin(i)), else uniform pair + heat-bath cumulative table over
//               (a<b) weighted by |<ij||ab>|, with rejection of occupied a, b.
#pragma once
#include "common.cuh"

namespace hande {

enum { SYS_HUBBARD = 0, SYS_UEG = 1, SYS_MOLECULE = 2 };

struct SysDev {
  int norb, nspin, nel;
  // Hubbard
  int L, periodic;
  double t, U;
  // UEG: per spatial orbital (nx, ny, nz, |n|^2) packed in int4; momentum cube
  double vfac, kfac;
  int nmax, side;
  const int4* kvec;
  const int16_t* klookup;
  // molecule: h1 dense norb^2, eri packed with 8-fold symmetry
  const double* h1;
  const double* eri;
  double ecore;
  // heat-bath tables per occupied pair index q(q-1)/2 + p
  const int* hb_start;
  const int* hb_len;
  const uint16_t* hb_ab;   // a | b << 8
  const uint64_t* hb_cum;
  uint32_t psingle_thr;
  double p_single, p_double;
  // diagonal tables: orb_diag[k] = h_kk (molecule, spin orbitals) or |k|^2/2
  // (UEG, spatial); pair_diag = (kk|ll) - (kl|lk) (molecule, nspin^2) or the
  // exchange kernel 4 pi / (Omega |k_k - k_l|^2) (UEG, norb^2)
  const double* orb_diag;
  const double* pair_diag;
  // spawn-weight factors ct = (tau inv_a) inv_b with 1/p_gen = inv_a inv_b, so that
  // tau |H| / p_gen = |H| ct; inv_a: 2N (Hubbard), C(N,2) M / {2, 1} (UEG, same /
  // opposite spins), N n_empty(spin) / p_s (molecular singles), C(N,2) / p_d
  // (heat-bath doubles); inv_b: 2^64 / width per heat-bath entry (1 for a
  // one-entry table), else 1.  Evaluated once on the host.
  double c_hub;
  double c_ueg[2];
  double c_single[2];
  const double* hb_c;
  // pair index P = j(j-1)/2 + i -> (i | j << 8), i < j < nel
  const uint16_t* pair_ij;
  // molecule: single-excitation terms G[(i*nspin + a)*nspin + k] = (ia|kk) - (ik|ka)
  // over spin orbitals (each the same one-rounding difference the sum adds)
  const double* single_g;
  // heat-bath guide: for table t and g = 0..64, the first entry whose threshold
  // exceeds g * 2^58 (clamped to len - 1): the search for word w starts in
  // [guide[w >> 58], guide[(w >> 58) + 1]]
  const uint16_t* hb_guide;
};

__device__ __forceinline__ int tri(int p, int q) { return p >= q ? p * (p + 1) / 2 + q : q * (q + 1) / 2 + p; }

// spatial chemist integral (PQ|RS)
__device__ __forceinline__ double eri_sp(const SysDev& s, int P, int Q, int R, int S) {
  return __ldg(&s.eri[tri(tri(P, Q), tri(R, S))]);
}
// spin-orbital (pq|rs): zero unless spin(p)=spin(q) and spin(r)=spin(s)
__device__ __forceinline__ double eri_so(const SysDev& s, int p, int q, int r, int t) {
  if (((p ^ q) & 1) || ((r ^ t) & 1)) return 0.0;
  return eri_sp(s, p >> 1, q >> 1, r >> 1, t >> 1);
}
__device__ __forceinline__ double h1_so(const SysDev& s, int p, int q) {
  if ((p ^ q) & 1) return 0.0;
  return __ldg(&s.h1[(p >> 1) * s.norb + (q >> 1)]);
}
__device__ __forceinline__ int ueg_dist2(const SysDev& s, int P, int Q) {
  int4 a = __ldg(&s.kvec[P]), b = __ldg(&s.kvec[Q]);
  int dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  return dx * dx + dy * dy + dz * dz;
}
__device__ __forceinline__ double ueg_v(const SysDev& s, int m) { return __ddiv_rn(s.vfac, (double)m); }

// iterate occupied spin orbitals of k in ascending order
#define HANDE_FOR_OCC(W, key, p, body)                 \
  _Pragma("unroll") for (int _j = 0; _j < W; ++_j) {   \
    uint64_t _m = (key).w[_j];                         \
    while (_m) {                                       \
      int p = _j * 64 + __ffsll((long long)_m) - 1;    \
      _m &= _m - 1;                                    \
      body                                             \
    }                                                  \
  }

template <int W, int SYS>
__device__ double h_diag(const SysDev& s, const Key<W>& d) {
  if (SYS == SYS_HUBBARD) {
    int dbl = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) dbl += __popcll(d.w[j] & (d.w[j] >> 1) & 0x5555555555555555ull);
    return __dmul_rn(s.U, (double)dbl);
  } else if (SYS == SYS_UEG) {
    double e = 0.0;
    HANDE_FOR_OCC(W, d, p, { e = __dadd_rn(e, __ldg(&s.orb_diag[p >> 1])); })
    HANDE_FOR_OCC(W, d, p, {
      // partners l > p with the same spin
      Key<W> rest = d;
#pragma unroll
      for (int jj = 0; jj < W; ++jj) {
        int lo = p + 1 - jj * 64;
        if (lo >= 64) rest.w[jj] = 0;
        else if (lo > 0) rest.w[jj] &= ~((1ull << lo) - 1);
        rest.w[jj] &= (p & 1) ? 0xAAAAAAAAAAAAAAAAull : 0x5555555555555555ull;
      }
      const double* row = s.pair_diag + (size_t)(p >> 1) * s.norb;
      HANDE_FOR_OCC(W, rest, l, { e = __dsub_rn(e, __ldg(&row[l >> 1])); })
    })
    return e;
  } else {
    double e1 = 0.0, e2 = 0.0;
    HANDE_FOR_OCC(W, d, p, { e1 = __dadd_rn(e1, __ldg(&s.orb_diag[p])); })
    HANDE_FOR_OCC(W, d, p, {
      Key<W> rest = d;
#pragma unroll
      for (int jj = 0; jj < W; ++jj) {
        int lo = p + 1 - jj * 64;
        if (lo >= 64) rest.w[jj] = 0;
        else if (lo > 0) rest.w[jj] &= ~((1ull << lo) - 1);
      }
      const double* row = s.pair_diag + (size_t)p * s.nspin;
      HANDE_FOR_OCC(W, rest, q, { e2 = __dadd_rn(e2, __ldg(&row[q])); })
    })
    return __dadd_rn(__dadd_rn(e1, e2), s.ecore);
  }
}

// <D'|H|D>, D' = D with i -> a
template <int W, int SYS>
__device__ double h_single(const SysDev& s, const Key<W>& d, int i, int a) {
  double v;
  if (SYS == SYS_HUBBARD) {
    if ((i ^ a) & 1) return 0.0;
    int si = i >> 1, sa = a >> 1;
    int diff = si > sa ? si - sa : sa - si;
    bool bond = (diff == 1) || (s.periodic && s.L > 2 && diff == s.L - 1);
    if (!bond) return 0.0;
    v = -s.t;
  } else if (SYS == SYS_UEG) {
    return 0.0;
  } else {
    double acc = 0.0;
    const double* row = s.single_g + ((size_t)i * s.nspin + a) * s.nspin;
    HANDE_FOR_OCC(W, d, k, {
      if (k != i) acc = __dadd_rn(acc, __ldg(&row[k]));
    })
    v = __dadd_rn(h1_so(s, i, a), acc);
  }
  return (key_between<W>(d, i, a) & 1) ? -v : v;
}

// <D'|H|D>, D' = D with i -> a, j -> b (i < j, a < b)
template <int W, int SYS>
__device__ double h_double(const SysDev& s, const Key<W>& d, int i, int j, int a, int b) {
  if (SYS == SYS_HUBBARD) return 0.0;
  Key<W> tmp = d;
  int n1 = key_between<W>(tmp, i, a);
  key_flip<W>(tmp, i);
  key_flip<W>(tmp, a);
  int n2 = key_between<W>(tmp, j, b);
  double v;
  if (SYS == SYS_UEG) {
    int I = i >> 1, J = j >> 1, A = a >> 1, B = b >> 1;
    int4 ki = __ldg(&s.kvec[I]), kj = __ldg(&s.kvec[J]), ka = __ldg(&s.kvec[A]), kb = __ldg(&s.kvec[B]);
    if (ki.x + kj.x != ka.x + kb.x || ki.y + kj.y != ka.y + kb.y || ki.z + kj.z != ka.z + kb.z) return 0.0;
    double direct = 0.0, exch = 0.0;
    if (!((i ^ a) & 1) && !((j ^ b) & 1)) direct = ueg_v(s, ueg_dist2(s, I, A));
    if (!((i ^ b) & 1) && !((j ^ a) & 1)) exch = ueg_v(s, ueg_dist2(s, I, B));
    v = __dsub_rn(direct, exch);
  } else {
    v = __dsub_rn(eri_so(s, i, a, j, b), eri_so(s, i, b, j, a));
  }
  return ((n1 + n2) & 1) ? -v : v;
}

// <target|H|source>
template <int W, int SYS>
__device__ double h_elem(const SysDev& s, const Key<W>& src, const Key<W>& tgt) {
  int nd = key_popc_xor<W>(src, tgt);
  if (nd == 0) return h_diag<W, SYS>(s, src);
  if (nd != 2 && nd != 4) return 0.0;
  Key<W> from, to;
#pragma unroll
  for (int j = 0; j < W; ++j) {
    uint64_t x = src.w[j] ^ tgt.w[j];
    from.w[j] = x & src.w[j];
    to.w[j] = x & tgt.w[j];
  }
  if (nd == 2) return h_single<W, SYS>(s, src, select_bit<W>(from, 0), select_bit<W>(to, 0));
  return h_double<W, SYS>(s, src, select_bit<W>(from, 0), select_bit<W>(from, 1), select_bit<W>(to, 0),
                          select_bit<W>(to, 1));
}

template <int W>
struct Excitation {
  bool ok;
  Key<W> child;
  double hij;
  double ct;             // tau / p_gen as (tau inv_a) inv_b
  bool single;           // a molecular single selected but not evaluated (DEFER)
  int si, sa;            // its hole and particle
};

// pair index P = j(j-1)/2 + i  ->  (i, j), i < j (tabulated)
__device__ __forceinline__ void unrank_pair(const SysDev& s, uint64_t P, int& i, int& j) {
  uint16_t v = __ldg(&s.pair_ij[P]);
  i = v & 0xff;
  j = v >> 8;
}

template <int W>
__device__ __forceinline__ Key<W> spin_mask(int spin, int nspin) {
  Key<W> m;
#pragma unroll
  for (int j = 0; j < W; ++j) {
    uint64_t x = spin ? 0xAAAAAAAAAAAAAAAAull : 0x5555555555555555ull;
    int hi = nspin - j * 64;
    if (hi <= 0) x = 0;
    else if (hi < 64) x &= (1ull << hi) - 1;
    m.w[j] = x;
  }
  return m;
}

// DEFER: a molecular single excitation is only selected (e.single, e.si, e.sa);
// its matrix element is left to the caller (evaluated later by full warps).
template <int W, int SYS, bool DEFER = false>
__device__ Excitation<W> generate(const SysDev& s, const Key<W>& d, const Words4& w) {
  Excitation<W> e;
  e.ok = false;
  e.single = false;
  const int n = s.nel;
  if (SYS == SYS_HUBBARD) {
    int p = select_bit<W>(d, (int)draw_index(w.x, (uint64_t)n));
    int site = p >> 1, spin = p & 1;
    int ns = (w.y >> 63) == 0 ? site + 1 : site - 1;
    if (s.periodic) {
      ns = (ns + s.L) % s.L;
    } else if (ns < 0 || ns >= s.L) {
      return e;
    }
    int q = 2 * ns + spin;
    if (key_bit<W>(d, q)) return e;
    e.ct = s.c_hub;
    e.hij = h_single<W, SYS>(s, d, p, q);
    e.child = d;
    key_flip<W>(e.child, p);
    key_flip<W>(e.child, q);
    e.ok = true;
    return e;
  } else if (SYS == SYS_UEG) {
    uint64_t npairs = (uint64_t)n * (n - 1) / 2;
    int ii, jj;
    unrank_pair(s, draw_index(w.y, npairs), ii, jj);
    int p = select_bit<W>(d, ii), q = select_bit<W>(d, jj);
    int A = (int)draw_index(w.z, (uint64_t)s.norb);
    int a = 2 * A + (p & 1);
    int4 kp = __ldg(&s.kvec[p >> 1]), kq = __ldg(&s.kvec[q >> 1]), ka = __ldg(&s.kvec[A]);
    int bx = kp.x + kq.x - ka.x, by = kp.y + kq.y - ka.y, bz = kp.z + kq.z - ka.z;
    if (bx < -s.nmax || bx > s.nmax || by < -s.nmax || by > s.nmax || bz < -s.nmax || bz > s.nmax) return e;
    int B = __ldg(&s.klookup[((bx + s.nmax) * s.side + (by + s.nmax)) * s.side + (bz + s.nmax)]);
    if (B < 0) return e;
    int b = 2 * B + (q & 1);
    if (a == b || key_bit<W>(d, a) || key_bit<W>(d, b)) return e;
    e.ct = s.c_ueg[(p ^ q) & 1];
    int lo = a < b ? a : b, hi = a < b ? b : a;
    e.hij = h_double<W, SYS>(s, d, p, q, lo, hi);
    e.child = d;
    key_flip<W>(e.child, p);
    key_flip<W>(e.child, q);
    key_flip<W>(e.child, a);
    key_flip<W>(e.child, b);
    e.ok = true;
    return e;
  } else {
    if ((uint32_t)(w.x >> 32) < s.psingle_thr) {
      int i = select_bit<W>(d, (int)draw_index(w.y, (uint64_t)n));
      Key<W> empty = spin_mask<W>(i & 1, s.nspin);
#pragma unroll
      for (int j = 0; j < W; ++j) empty.w[j] &= ~d.w[j];
      int ne = 0;
#pragma unroll
      for (int j = 0; j < W; ++j) ne += __popcll(empty.w[j]);
      if (ne == 0) return e;
      int a = select_bit<W>(empty, (int)draw_index(w.z, (uint64_t)ne));
      if (DEFER) {
        e.single = true;
        e.si = i;
        e.sa = a;
        return e;
      }
      e.ct = s.c_single[i & 1];
      e.hij = h_single<W, SYS>(s, d, i, a);
      e.child = d;
      key_flip<W>(e.child, i);
      key_flip<W>(e.child, a);
      e.ok = true;
      return e;
    }
    uint64_t npairs = (uint64_t)n * (n - 1) / 2;
    int ii, jj;
    unrank_pair(s, draw_index(w.y, npairs), ii, jj);
    int p = select_bit<W>(d, ii), q = select_bit<W>(d, jj);
    int pidx = q * (q - 1) / 2 + p;
    int len = __ldg(&s.hb_len[pidx]);
    if (len == 0) return e;
    int start = __ldg(&s.hb_start[pidx]);
    // smallest k with w.z < cum[k] among the first len-1 entries, else the last
    const uint16_t* gd = s.hb_guide + (size_t)pidx * 65;
    const int gt = (int)(w.z >> 58);
    int lo = __ldg(&gd[gt]), hi = __ldg(&gd[gt + 1]);
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (__ldg(&s.hb_cum[start + mid]) <= w.z) lo = mid + 1;
      else hi = mid;
    }
    int k = lo;
    uint16_t ab = __ldg(&s.hb_ab[start + k]);
    int a = ab & 0xff, b = ab >> 8;
    if (key_bit<W>(d, a) || key_bit<W>(d, b)) return e;
    e.ct = __ldg(&s.hb_c[start + k]);
    e.hij = h_double<W, SYS>(s, d, p, q, a, b);
    e.child = d;
    key_flip<W>(e.child, p);
    key_flip<W>(e.child, q);
    key_flip<W>(e.child, a);
    key_flip<W>(e.child, b);
    e.ok = true;
    return e;
  }
}

}  // namespace hande
