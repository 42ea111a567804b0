// common.cuh -- device-side building blocks of the GPU FCIQMC iteration.
//
// Arithmetic that decides the walker list is exact and order-independent:
// populations are int64 fixed point (one walker = 2^32), sums of FP64 terms
// are accumulated exactly in 128-bit fixed point (2^-16 resolution), and
// every FP64 expression is written with explicit round-to-nearest intrinsics
// (__dadd_rn, __dmul_rn, ...) so the compiler cannot contract or reorder it.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hande {

constexpr int64_t kOne = int64_t(1) << 32;            // one walker
constexpr uint64_t kDetDraw = ~0ull;                   // attempt index of per-determinant draws
constexpr uint64_t kAmountMax = 1ull << 62;            // saturation of one spawned amount

// x != 0.0 (either sign) from the bits, without the FP64 pipe
__host__ __device__ __forceinline__ bool nonzero(double x) {
#ifdef __CUDA_ARCH__
  return ((uint64_t)__double_as_longlong(x) << 1) != 0;
#else
  return x != 0.0;
#endif
}

// error bits (reported through the C ABI as hande_status codes)
enum : unsigned {
  ERR_SPAWN_CAPACITY = 1u,
  ERR_STATE_CAPACITY = 2u,
  ERR_OVERFLOW = 4u,
  ERR_TIMEOUT = 8u,
  ERR_TILE_CAPACITY = 16u,
  ERR_BUCKET_CAPACITY = 32u,
};

// ------------------------------------------------------------------ keys
// A determinant: W 64-bit words, bit p = spin orbital p (p = 2*spatial + spin).
// Order: unsigned big integer, word W-1 most significant.
template <int W>
struct Key {
  uint64_t w[W];
};

template <int W>
__device__ __forceinline__ bool key_lt(const Key<W>& a, const Key<W>& b) {
#pragma unroll
  for (int i = W - 1; i >= 0; --i) {
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i];
  }
  return false;
}
template <int W>
__device__ __forceinline__ bool key_eq(const Key<W>& a, const Key<W>& b) {
  bool e = true;
#pragma unroll
  for (int i = 0; i < W; ++i) e &= (a.w[i] == b.w[i]);
  return e;
}
template <int W>
__device__ __forceinline__ bool key_le(const Key<W>& a, const Key<W>& b) {
  return !key_lt<W>(b, a);
}
// load / store from a structure-of-arrays key block: word k of entry i at p[k*stride + i]
template <int W>
__device__ __forceinline__ Key<W> load_key(const uint64_t* __restrict__ p, int64_t stride, int64_t i) {
  Key<W> k;
#pragma unroll
  for (int j = 0; j < W; ++j) k.w[j] = p[j * stride + i];
  return k;
}
template <int W>
__device__ __forceinline__ void store_key(uint64_t* __restrict__ p, int64_t stride, int64_t i, const Key<W>& k) {
#pragma unroll
  for (int j = 0; j < W; ++j) p[j * stride + i] = k.w[j];
}
template <int W>
__device__ __forceinline__ int key_popc_xor(const Key<W>& a, const Key<W>& b) {
  int n = 0;
#pragma unroll
  for (int j = 0; j < W; ++j) n += __popcll(a.w[j] ^ b.w[j]);
  return n;
}
template <int W>
__device__ __forceinline__ bool key_bit(const Key<W>& k, int p) {
  return (k.w[p >> 6] >> (p & 63)) & 1ull;
}
template <int W>
__device__ __forceinline__ void key_flip(Key<W>& k, int p) {
  k.w[p >> 6] ^= 1ull << (p & 63);
}
// number of set bits strictly between spin orbitals p and q (fermionic sign)
template <int W>
__device__ __forceinline__ int key_between(const Key<W>& k, int p, int q) {
  int lo = p < q ? p : q, hi = p < q ? q : p;
  int n = 0;
#pragma unroll
  for (int j = 0; j < W; ++j) {
    int b0 = j * 64;
    // bits (lo, hi) restricted to this word
    int s = lo + 1 - b0, e = hi - b0;  // [s, e)
    if (s < 0) s = 0;
    if (e > 64) e = 64;
    if (e > s) {
      uint64_t m = (e == 64 ? ~0ull : ((1ull << e) - 1)) & ~((s == 0) ? 0ull : ((1ull << s) - 1));
      n += __popcll(k.w[j] & m);
    }
  }
  return n;
}
// position of the r-th (0-based) set bit of x (r < popcount(x)): bisection of
// the word with popcounts of its lower halves, 32 down to 1 bit
__device__ __forceinline__ int select64(uint64_t x, int r) {
  int pos = 0;
  int c = __popc((unsigned)x);
  if (r >= c) {
    r -= c;
    x >>= 32;
    pos = 32;
  }
  unsigned w = (unsigned)x;
#pragma unroll
  for (int width = 16; width; width >>= 1) {
    c = __popc(w & ((1u << width) - 1u));
    if (r >= c) {
      r -= c;
      w >>= width;
      pos += width;
    }
  }
  return pos;
}
// position of the r-th set bit of a multiword mask
template <int W>
__device__ __forceinline__ int select_bit(const Key<W>& k, int r) {
#pragma unroll
  for (int j = 0; j < W; ++j) {
    int c = __popcll(k.w[j]);
    if (r < c) return j * 64 + select64(k.w[j], r);
    r -= c;
  }
  return -1;
}

// floor(|h| ct 2^32) (half = false) or floor(|h| ct 2^32 + 1/2) (half = true)
// of the exact product of two positive finite doubles given by their bits,
// saturated at 2^62: 53x53-bit significand product on the integer pipe, one
// rounding.  |h| ct 2^32 = m_h m_c 2^(e_h + e_c - 2 * 1075 + 32).
__device__ __forceinline__ uint64_t fixed_amount(uint64_t hb, uint64_t cb, bool half) {
  constexpr uint64_t kFrac = (1ull << 52) - 1;
  int eh = (int)(hb >> 52), ec = (int)(cb >> 52);
  uint64_t mh = hb & kFrac, mc = cb & kFrac;
  if (eh) mh |= 1ull << 52;
  else eh = 1;
  if (ec) mc |= 1ull << 52;
  else ec = 1;
  const uint64_t lo = mh * mc, hi = __umul64hi(mh, mc);
  const int e = eh + ec - 2118;
  if (e >= 0) {
    if (e >= 62 || hi != 0 || (lo >> (62 - e)) != 0) return kAmountMax;
    return lo << e;
  }
  int sh = -e;
  if (sh >= 120) return 0;
  if (half) sh -= 1;   // floor(x + 1/2) = ceil(floor(2x) / 2)
  uint64_t t, over;
  if (sh >= 64) {
    t = hi >> (sh - 64);
    over = 0;
  } else if (sh == 0) {
    t = lo;
    over = hi;
  } else {
    t = (lo >> sh) | (hi << (64 - sh));
    over = hi >> sh;
  }
  if (over) return kAmountMax;
  if (half) t = (t >> 1) + (t & 1);
  return t >= kAmountMax ? kAmountMax : t;
}

__device__ __forceinline__ uint64_t dbl_bits(double x) { return (uint64_t)__double_as_longlong(x); }
__device__ __forceinline__ uint64_t abs_bits(double x) { return dbl_bits(x) & ~(1ull << 63); }
__device__ __forceinline__ bool sign_bit(double x) { return (dbl_bits(x) >> 63) != 0; }

// ------------------------------------------------------------------ Philox4x64-10
// Counter-based generator of Salmon et al. (SC'11): 10 rounds of two 64x64->128
// multiplies with Weyl key increments.
struct Words4 {
  uint64_t x, y, z, w;
};
__device__ __forceinline__ Words4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                                                uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B97F4A7C15ull;
      k1 += 0xBB67AE8584CAA73Bull;
    }
    uint64_t lo0 = M0 * c0, hi0 = __umul64hi(M0, c0);
    uint64_t lo1 = M1 * c2, hi1 = __umul64hi(M1, c2);
    uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return {c0, c1, c2, c3};
}
__device__ __forceinline__ uint64_t splitmix_fold(uint64_t z) {
  z ^= z >> 30;
  z *= 0xbf58476d1ce4e5b9ull;
  z ^= z >> 27;
  z *= 0x94d049bb133111ebull;
  z ^= z >> 31;
  return z;
}
// stream of determinant D at iteration t, attempt a: counter (t, a, h0(D), h1(D)),
// key (seed, replica); h = the key words for W <= 2, a SplitMix64 fold above.
template <int W>
__device__ __forceinline__ Words4 draw(uint64_t seed, uint64_t replica, int64_t t, uint64_t a, const Key<W>& d) {
  uint64_t h0, h1;
  if (W <= 2) {
    h0 = d.w[0];
    h1 = (W == 2) ? d.w[W - 1] : 0ull;
  } else {
    uint64_t p = 0x243F6A8885A308D3ull, q = 0x13198A2E03707344ull;
#pragma unroll
    for (int j = 0; j < W; ++j) {
      p = splitmix_fold(p ^ d.w[j]);
      q = splitmix_fold(q ^ d.w[j]);
    }
    h0 = p;
    h1 = q;
  }
  return philox4x64_10((uint64_t)t, a, h0, h1, seed, replica);
}
__device__ __forceinline__ uint64_t draw_index(uint64_t w, uint64_t n) { return __umul64hi(w, n); }
__device__ __forceinline__ double draw_unit(uint64_t w) { return __dmul_rn((double)(w >> 11), 0x1p-53); }

// ------------------------------------------------------------------ natural log
// atanh series: x = m 2^e with m in [sqrt(1/2), sqrt(2)), s = (m-1)/(m+1),
// ln x = e ln2 + 2 s sum_{k=0..11} s^(2k) / (2k+1); Horner in s^2.
__device__ __forceinline__ double log_series(double x) {
  if (!(x > 0.0)) return __longlong_as_double((long long)0xfff0000000000000ull);  // -inf
  uint64_t bits = (uint64_t)__double_as_longlong(x);
  int e = (int)((bits >> 52) & 0x7ff);
  if (e == 0) {
    double y = __dmul_rn(x, 18446744073709551616.0);
    bits = (uint64_t)__double_as_longlong(y);
    e = (int)((bits >> 52) & 0x7ff) - 64;
  }
  e -= 1023;
  double m = __longlong_as_double((long long)((bits & 0x000fffffffffffffull) | 0x3ff0000000000000ull));
  if (m > 1.4142135623730951) {
    m = __dmul_rn(m, 0.5);
    e += 1;
  }
  double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  double z = __dmul_rn(s, s);
  double p = __ddiv_rn(1.0, 23.0);
  for (int k = 10; k >= 0; --k) {
    p = __dmul_rn(p, z);
    p = __dadd_rn(p, __ddiv_rn(1.0, (double)(2 * k + 1)));
  }
  double lnm = __dmul_rn(__dmul_rn(2.0, s), p);
  return __dadd_rn(__dmul_rn((double)e, 0.69314718055994530942), lnm);
}

// ------------------------------------------------------------------ exact sums
// round_half_even(n h 2^16) of the exact product of an int64 population n and
// a double h, as a signed 128-bit integer (lo, hi words): the 53-bit
// significand times |n| on the integer pipe, one rounding; magnitudes at or
// above 2^126 saturate.  Sums of these terms are exact and order-free.
struct I128 {
  uint64_t lo;
  int64_t hi;
};
__device__ __forceinline__ I128 fixed_term(int64_t n, double h) {
  const uint64_t hb = (uint64_t)__double_as_longlong(h);
  if (n == 0 || (hb << 1) == 0) return {0ull, 0ll};
  int e = (int)((hb >> 52) & 0x7ff);
  uint64_t m = hb & ((1ull << 52) - 1);
  if (e) m |= 1ull << 52;
  else e = 1;
  const uint64_t a = n < 0 ? 0ull - (uint64_t)n : (uint64_t)n;
  const uint64_t lo = a * m, hi = __umul64hi(a, m);   // |n h| 2^16 = (hi:lo) 2^(e - 1059)
  const int sh = e - 1059;
  uint64_t qlo, qhi;
  if (sh >= 0) {
    bool sat;
    if (sh >= 126) {
      sat = true;
    } else {
      const int k = 126 - sh;   // (hi:lo) >> k != 0 ?
      sat = k >= 64 ? (hi >> (k - 64)) != 0 : (hi != 0 || (lo >> k) != 0);
    }
    if (sat) {
      qhi = 1ull << 62;
      qlo = 0;
    } else if (sh == 0) {
      qhi = hi;
      qlo = lo;
    } else if (sh >= 64) {
      qhi = lo << (sh - 64);
      qlo = 0;
    } else {
      qhi = (hi << sh) | (lo >> (64 - sh));
      qlo = lo << sh;
    }
  } else if (-sh >= 128) {
    qhi = 0;
    qlo = 0;
  } else {
    const int s = -sh;
    if (s >= 64) {
      qlo = hi >> (s - 64);
      qhi = 0;
    } else {
      qlo = (lo >> s) | (hi << (64 - s));
      qhi = hi >> s;
    }
    // half to even: round bit (bit s-1) and any lower bit
    const int rb = s - 1;
    const uint64_t rbit = rb >= 64 ? (hi >> (rb - 64)) & 1ull : (lo >> rb) & 1ull;
    bool sticky;
    if (rb >= 64) sticky = lo != 0 || (rb > 64 && (hi & ((1ull << (rb - 64)) - 1)) != 0);
    else sticky = rb > 0 && (lo & ((1ull << rb) - 1)) != 0;
    if (rbit && (sticky || (qlo & 1ull))) {
      qlo += 1;
      if (qlo == 0) qhi += 1;
    }
  }
  if ((n < 0) != ((hb >> 63) != 0)) {   // two's complement negate
    qlo = ~qlo;
    qhi = ~qhi;
    qlo += 1;
    if (qlo == 0) qhi += 1;
  }
  return {qlo, (int64_t)qhi};
}
__device__ __forceinline__ void i128_add(I128& a, const I128& b) {
  uint64_t lo = a.lo + b.lo;
  uint64_t c = lo < a.lo ? 1 : 0;
  a.hi = (int64_t)((uint64_t)a.hi + (uint64_t)b.hi + c);
  a.lo = lo;
}
__device__ __forceinline__ double fixed_to_double(I128 s) {
  double d = __dadd_rn(__dmul_rn((double)s.hi, 18446744073709551616.0), __ull2double_rn(s.lo));
  return __dmul_rn(d, 0x1p-16);
}
__device__ __forceinline__ I128 shfl_xor_i128(I128 v, int m) {
  I128 r;
  r.lo = __shfl_xor_sync(0xffffffffu, v.lo, m);
  r.hi = __shfl_xor_sync(0xffffffffu, v.hi, m);
  return r;
}
__device__ __forceinline__ void atomic_add_i128(unsigned long long* lo_hi, I128 v) {
  unsigned long long old = atomicAdd(lo_hi, (unsigned long long)v.lo);
  unsigned long long c = (old + v.lo < old) ? 1ull : 0ull;
  atomicAdd(lo_hi + 1, (unsigned long long)v.hi + c);
}

// ------------------------------------------------------------------ misc
__device__ __forceinline__ int64_t iabs64(int64_t x) { return x < 0 ? -x : x; }
__device__ __forceinline__ unsigned warp_lane() { return threadIdx.x & 31u; }

}  // namespace hande
