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
  // Hubbard: L sites, z hops per site, nbr[site * z + k] the site hop k reaches (-1: none)
  int L, periodic, z;
  const int16_t* nbr;
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
  // heat-bath tables, per occupied spin-orbital pair index q(q-1)/2 + p (p < q):
  // hb_pair = {first entry, entry count, guide offset, guide bits g}; per entry
  // the cumulative threshold hb_cum (strictly increasing, the last 2^64 - 1) and
  // hb_ent = {fixed-point spawn amount of |<pq||ab>| tau / p_gen,
  // a | b << 8 | (<pq||ab> < 0) << 16}.  Guide: for t = 0 .. 2^g, the first
  // entry whose threshold exceeds t 2^(64-g) (clamped to the last), so the entry
  // drawn by word w lies in [guide[w >> (64-g)], guide[(w >> (64-g)) + 1]].
  const int4* hb_pair;
  const uint64_t* hb_cum;
  const ulonglong2* hb_ent;
  const uint16_t* hb_guide;
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
  // (heat-bath doubles, folded into hb_ent); inv_b: 2^64 / width per heat-bath
  // entry (1 for a one-entry table), else 1.  Evaluated once on the host.
  double c_hub;
  double c_ueg[2];
  double c_single[2];
  int half;   // spawn amounts rounded to nearest (real weights) or floored (integer walkers)
  // UEG proposal table (the learned proposal's selection table; null = the
  // uniform generator): for row r = (I M + J) 2 + [spin i == spin j], M
  // cumulative integer weights over the particle orbital A; c_tab = tau C(N,2)
  const uint32_t* ptab_cum;
  double c_tab;
  // time-step search: the inv_a factors without tau (inv_b = 1 unless stated)
  // and |<pq||ab>| inv_a inv_b per heat-bath entry; want_r = 1 while searching
  int want_r;
  double inv_hub, inv_ueg[2], inv_single[2], inv_tab;
  const double* hb_R;
  // pair index P = j(j-1)/2 + i -> (i | j << 8), i < j < nel
  const uint16_t* pair_ij;
  // molecule: single-excitation terms G[(i*nspin + a)*nspin + k] = (ia|kk) - (ik|ka)
  // over spin orbitals (each the same one-rounding difference the sum adds)
  const double* single_g;
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
    bool bond = false;
    for (int k = 0; k < s.z; ++k) bond = bond || __ldg(&s.nbr[si * s.z + k]) == sa;
    if (!bond) return 0.0;
    v = -s.t;
  } else if (SYS == SYS_UEG) {
    return 0.0;
  } else {
    // sum over occupied k != i in ascending order; the row entries are loaded
    // four at a time ahead of the (ordered) additions
    double acc = 0.0;
    const double* row = s.single_g + ((size_t)i * s.nspin + a) * s.nspin;
#pragma unroll
    for (int j = 0; j < W; ++j) {
      uint64_t m = d.w[j];
      if ((i >> 6) == j) m &= ~(1ull << (i & 63));
      while (m) {
        double v4[4];
        int cnt = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (m) {
            const int k = j * 64 + __ffsll((long long)m) - 1;
            m &= m - 1;
            v4[u] = __ldg(&row[k]);
            cnt = u + 1;
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (u < cnt) acc = __dadd_rn(acc, v4[u]);
      }
    }
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
  bool ok;               // a connected child with H != 0 was drawn
  bool single;           // a molecular single: chosen only, its orbitals and H_ia left to the caller
  bool hneg;             // H_child,parent < 0
  int prow, pA;          // proposal table: the row and particle orbital drawn (prow < 0: none)
  uint32_t pqa, pQ;      //   the drawn weight q_A and the row total Q
  double rval;           // |H| / p_gen = (|H| inv_a) inv_b when the system's want_r is set
  uint64_t famt;         // fixed-point amount of |H| tau / p_gen (floored or rounded)
  Key<W> child;
};

// tables of the molecular generator read on every attempt; the kernel points
// them at shared-memory copies when they fit
struct GenTabs {
  const int4* hb_pair;
  const uint16_t* pair_ij;
};

// pair index P = j(j-1)/2 + i  ->  (i, j), i < j (tabulated)
__device__ __forceinline__ void unrank_pair(const uint16_t* pair_ij, uint64_t P, int& i, int& j) {
  uint16_t v = pair_ij[P];
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

// orbitals of a molecular single: i the ri-th occupied spin orbital of d
// (ri = draw_index(w.y, N), uniform), a uniform among the empty orbitals of
// i's spin by Philox word wz; false when that spin has no empty orbital
// (nothing is spawned)
template <int W>
__device__ __forceinline__ bool single_orbitals(const SysDev& s, const Key<W>& d, int ri, uint64_t wz, int& i,
                                               int& a) {
  i = select_bit<W>(d, ri);
  Key<W> empty = spin_mask<W>(i & 1, s.nspin);
#pragma unroll
  for (int j = 0; j < W; ++j) empty.w[j] &= ~d.w[j];
  int ne = 0;
#pragma unroll
  for (int j = 0; j < W; ++j) ne += __popcll(empty.w[j]);
  if (ne == 0) return false;
  a = select_bit<W>(empty, (int)draw_index(wz, (uint64_t)ne));
  return true;
}

template <int W>
__device__ __forceinline__ void finish(Excitation<W>& e, const SysDev& s, double hij, double ct, double inv_a,
                                       double inv_b) {
  if (!nonzero(hij)) return;
  if (s.want_r) e.rval = __dmul_rn(__dmul_rn(fabs(hij), inv_a), inv_b);
  e.famt = fixed_amount(abs_bits(hij), dbl_bits(ct), s.half);
  e.hneg = sign_bit(hij);
  e.ok = true;
}

// One excitation drawn from Philox words w (Sec. 2.4 spawning): the child, the
// sign of its matrix element and the fixed-point amount of |H| tau / p_gen.
// A molecular single is only selected (e.single, e.si, e.sa); its O(N) matrix
// element is left to the caller.
template <int W, int SYS>
__device__ Excitation<W> generate(const SysDev& s, const GenTabs& gt, const Key<W>& d, const Words4& w) {
  Excitation<W> e;
  e.ok = false;
  e.single = false;
  e.hneg = false;
  e.famt = 0;
  e.prow = -1;
  e.rval = 0.0;
  const int n = s.nel;
  if (SYS == SYS_HUBBARD) {
    int p = select_bit<W>(d, (int)draw_index(w.x, (uint64_t)n));
    int site = p >> 1, spin = p & 1;
    // hop k uniform among the z of the site (chain: 0 right, 1 left)
    int ns = __ldg(&s.nbr[site * s.z + (int)draw_index(w.y, (uint64_t)s.z)]);
    if (ns < 0) return e;
    int q = 2 * ns + spin;
    if (key_bit<W>(d, q)) return e;
    e.child = d;
    key_flip<W>(e.child, p);
    key_flip<W>(e.child, q);
    finish<W>(e, s, h_single<W, SYS>(s, d, p, q), s.c_hub, s.inv_hub, 1.0);
    return e;
  } else if (SYS == SYS_UEG) {
    uint64_t npairs = (uint64_t)n * (n - 1) / 2;
    int ii, jj;
    unrank_pair(gt.pair_ij, draw_index(w.y, npairs), ii, jj);
    int p = select_bit<W>(d, ii), q = select_bit<W>(d, jj);
    if (s.ptab_cum) {
      // proposal table: A by inverse CDF over the integer weights of row
      // (I, J, same spin); p_gen = (q_A + [same] q_B) / (Q C(N,2)), exact
      const int M = s.norb, I = p >> 1, J = q >> 1, same = ((p ^ q) & 1) ? 0 : 1;
      const int row = (I * M + J) * 2 + same;
      const uint32_t* cum = s.ptab_cum + (size_t)row * M;
      const uint32_t Q = __ldg(&cum[M - 1]);
      if (Q == 0) return e;
      const uint64_t x = draw_index(w.z, (uint64_t)Q);
      int lo = 0, hi = M - 1;   // the first A whose cumulative weight exceeds x
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((uint64_t)__ldg(&cum[mid]) > x) hi = mid;
        else lo = mid + 1;
      }
      const int A = lo;
      int4 kp = __ldg(&s.kvec[I]), kq = __ldg(&s.kvec[J]), ka = __ldg(&s.kvec[A]);
      int bx = kp.x + kq.x - ka.x, by = kp.y + kq.y - ka.y, bz = kp.z + kq.z - ka.z;
      if (bx < -s.nmax || bx > s.nmax || by < -s.nmax || by > s.nmax || bz < -s.nmax || bz > s.nmax) return e;
      const int B = __ldg(&s.klookup[((bx + s.nmax) * s.side + (by + s.nmax)) * s.side + (bz + s.nmax)]);
      if (B < 0) return e;   // weight 0: not drawn
      const uint32_t qa = __ldg(&cum[A]) - (A > 0 ? __ldg(&cum[A - 1]) : 0u);
      const uint32_t qb = same ? __ldg(&cum[B]) - (B > 0 ? __ldg(&cum[B - 1]) : 0u) : 0u;
      e.prow = row;
      e.pA = A;
      e.pqa = qa;
      e.pQ = Q;
      const int a = 2 * A + (p & 1), b = 2 * B + (q & 1);
      if (a == b || key_bit<W>(d, a) || key_bit<W>(d, b)) return e;
      const int lo2 = a < b ? a : b, hi2 = a < b ? b : a;
      e.child = d;
      key_flip<W>(e.child, p);
      key_flip<W>(e.child, q);
      key_flip<W>(e.child, a);
      key_flip<W>(e.child, b);
      const double inv_b = __ddiv_rn((double)Q, (double)(qa + qb));
      finish<W>(e, s, h_double<W, SYS>(s, d, p, q, lo2, hi2), __dmul_rn(s.c_tab, inv_b), s.inv_tab, inv_b);
      return e;
    }
    int A = (int)draw_index(w.z, (uint64_t)s.norb);
    int a = 2 * A + (p & 1);
    int4 kp = __ldg(&s.kvec[p >> 1]), kq = __ldg(&s.kvec[q >> 1]), ka = __ldg(&s.kvec[A]);
    int bx = kp.x + kq.x - ka.x, by = kp.y + kq.y - ka.y, bz = kp.z + kq.z - ka.z;
    if (bx < -s.nmax || bx > s.nmax || by < -s.nmax || by > s.nmax || bz < -s.nmax || bz > s.nmax) return e;
    int B = __ldg(&s.klookup[((bx + s.nmax) * s.side + (by + s.nmax)) * s.side + (bz + s.nmax)]);
    if (B < 0) return e;
    int b = 2 * B + (q & 1);
    if (a == b || key_bit<W>(d, a) || key_bit<W>(d, b)) return e;
    int lo = a < b ? a : b, hi = a < b ? b : a;
    e.child = d;
    key_flip<W>(e.child, p);
    key_flip<W>(e.child, q);
    key_flip<W>(e.child, a);
    key_flip<W>(e.child, b);
    finish<W>(e, s, h_double<W, SYS>(s, d, p, q, lo, hi), s.c_ueg[(p ^ q) & 1], s.inv_ueg[(p ^ q) & 1], 1.0);
    return e;
  } else {
    if ((uint32_t)(w.x >> 32) < s.psingle_thr) {
      // a single: its orbitals (i from w.y, a from w.z) are selected by
      // single_orbitals when the caller evaluates the queued singles
      e.single = true;
      return e;
    }
    uint64_t npairs = (uint64_t)n * (n - 1) / 2;
    int ii, jj;
    unrank_pair(gt.pair_ij, draw_index(w.y, npairs), ii, jj);
    int p = select_bit<W>(d, ii), q = select_bit<W>(d, jj);
    const int4 pr = gt.hb_pair[q * (q - 1) / 2 + p];   // {start, len, guide offset, guide bits}
    if (pr.y == 0) return e;
    // smallest k with w.z < cum[k] among the first len - 1 entries, else the last
    const uint64_t t = w.z >> (64 - pr.w);
    int lo = __ldg(&s.hb_guide[pr.z + t]), hi = __ldg(&s.hb_guide[pr.z + t + 1]);
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (__ldg(&s.hb_cum[pr.x + mid]) <= w.z) lo = mid + 1;
      else hi = mid;
    }
    const ulonglong2 ent = __ldg(&s.hb_ent[pr.x + lo]);
    const int meta = (int)ent.y;
    const int a = meta & 0xff, b = (meta >> 8) & 0xff;
    if (key_bit<W>(d, a) || key_bit<W>(d, b)) return e;
    // Slater-Condon sign of p -> a, then q -> b on the updated string
    Key<W> tmp = d;
    const int n1 = key_between<W>(tmp, p, a);
    key_flip<W>(tmp, p);
    key_flip<W>(tmp, a);
    const int n2 = key_between<W>(tmp, q, b);
    key_flip<W>(tmp, q);
    key_flip<W>(tmp, b);
    e.child = tmp;
    e.famt = ent.x;
    e.hneg = (((meta >> 16) ^ n1 ^ n2) & 1) != 0;
    e.ok = true;
    if (s.want_r) e.rval = __ldg(&s.hb_R[pr.x + lo]);
    return e;
  }
}

}  // namespace hande
