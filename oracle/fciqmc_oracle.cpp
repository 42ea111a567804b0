/*
 * fciqmc_oracle.cpp -- plain, slow, single-threaded CPU FCIQMC.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The GPU
 * product path never links, imports or calls it; it shares no source, header,
 * table builder or constant with the CUDA path.
 *
 * What it follows (HANDE-QMC paper, arXiv:1811.11679):
 *   - Sec. 2.1, Eq. (fciqmc): c_i(t+dt) = c_i(t) - dt sum_j H_ij c_j(t), applied
 *     stochastically with signed particles; shift S as a diagonal energy offset.
 *   - Sec. 2.4: one iteration = spawning (random excitation + H_ij), death
 *     (diagonal), annihilation (combine particles on one state).
 *   - Sec. 2.1: initiator rule (new particles on unoccupied determinants only
 *     from parents above a threshold); real weights; semi-stochastic exact
 *     projection inside a deterministic space ("high" space, App. A.2).
 *   - App. A.1: projected energy  E = E_HF + sum_{i!=0} C_i H_0i / C_0.
 *   - App. B: sorted main list, spawned array, sort + merge annihilation.
 *
 * Where the paper is silent the oracle takes these readings: weights as int64
 * fixed point with F = 2^32; counter-based Philox4x64-10 keyed by (seed,
 * replica) with counter (t, attempt, det); the Slater-Condon sign of moving an
 * electron = (-1)^(occupied spin orbitals strictly between); UEG plane waves
 * ordered by (|n|^2, nx, ny, nz); a heat-bath-with-rejection generator over
 * cumulative integer thresholds; the shift held until the target population
 * and then updated every A iterations; exact 128-bit fixed-point accumulation
 * of the estimator numerator and of the deterministic-space product.  Each is
 * stated again where the code takes it.
 *
 * Parity status: Philox, the logarithm, Slater-Condon, generators and the
 * full iteration are pinned by tests/test_oracle_*.py against numpy,
 * brute-force second quantisation, dense exact diagonalisation and closed
 * forms.  The large-system energies (UEG 14e/38, 28-orbital molecule) are
 * "parity unpinned" against exact results (FCI not computable); they are
 * pinned only through the same code paths on small instances.
 *
 * Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared (see build.py).
 */
#include <stdint.h>
#include <string.h>
#include <math.h>
#include <vector>
#include <algorithm>
#include <string>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

typedef unsigned __int128 u128;
typedef __int128 i128;

const int MAXW = 8;
const uint64_t FIXED_ONE = 1ull << 32;          /* F: one walker */
const uint64_t SENTINEL_DET = ~0ull;            /* attempt index of per-det draws */

struct Det {
    uint64_t w[MAXW];
};

/* ------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its */
/* published definition: 10 rounds, multipliers M0, M1, Weyl key bump. */
/* ------------------------------------------------------------------ */
void philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        u128 p0 = (u128)M0 * c0;
        u128 p1 = (u128)M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform integer in [0, n): high word of w*n (Lemire's multiply-high) */
inline uint64_t draw_index(uint64_t w, uint64_t n) {
    return (uint64_t)(((u128)w * n) >> 64);
}
/* uniform double in [0, 1) with 53 random bits */
inline double draw_unit(uint64_t w) {
    return (double)(w >> 11) * 0x1p-53;
}

/* SplitMix64 finaliser (Steele, Lea, Flood 2014) -- used only to fold keys
 * wider than 128 bits into the two Philox counter words. */
inline uint64_t mix64(uint64_t z) {
    z ^= z >> 30; z *= 0xbf58476d1ce4e5b9ull;
    z ^= z >> 27; z *= 0x94d049bb133111ebull;
    z ^= z >> 31;
    return z;
}

/* ------------------------------------------------------------------ */
/* Natural logarithm written from the atanh series:                    */
/*   x = m 2^e, m in [sqrt(1/2), sqrt(2)), s = (m-1)/(m+1),            */
/*   ln m = 2 s (1 + s^2/3 + s^4/5 + ... + s^22/23),  ln x = e ln2 + ln m */
/* Every operation is one IEEE double op, so the CUDA side can produce */
/* the same bits.  Used in the shift update (Sec. 2.1).                */
/* ------------------------------------------------------------------ */
double own_log(double x) {
    if (!(x > 0.0)) return -INFINITY;          /* the shift never asks for this */
    uint64_t bits;
    memcpy(&bits, &x, 8);
    int e = (int)((bits >> 52) & 0x7ff);
    if (e == 0) {                               /* subnormal: rescale by 2^64 */
        double y = x * 18446744073709551616.0;
        memcpy(&bits, &y, 8);
        e = (int)((bits >> 52) & 0x7ff) - 64;
    }
    e -= 1023;
    uint64_t mbits = (bits & 0x000fffffffffffffull) | 0x3ff0000000000000ull;  /* m in [1,2) */
    double m;
    memcpy(&m, &mbits, 8);
    if (m > 1.4142135623730951) {               /* fold into [sqrt(1/2), sqrt(2)) */
        m = m * 0.5;
        e += 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    double p = 1.0 / 23.0;
    for (int k = 10; k >= 0; --k) {
        p = p * z;
        p = p + 1.0 / (double)(2 * k + 1);
    }
    double lnm = (2.0 * s) * p;
    return (double)e * 0.69314718055994530942 + lnm;
}

/* ------------------------------------------------------------------ */
/* 128-bit fixed point: value * 2^16, used so that sums of products   */
/* N h (population times matrix element) are exact and independent of  */
/* summation order.  Each term is the exact product rounded once,       */
/* half to even, to a multiple of 2^-16; magnitudes at or above 2^126   */
/* saturate (matrix elements that large do not occur).                 */
/* ------------------------------------------------------------------ */
const double FX_UNSCALE = 0x1p-16;

i128 fixed_term(int64_t n, double h) {
    if (n == 0 || h == 0.0) return 0;
    int e;
    double f = frexp(fabs(h), &e);                   /* |h| = f 2^e, f in [1/2, 1) */
    u128 m = (u128)(uint64_t)ldexp(f, 53);           /* exact 53-bit integer */
    u128 a = (u128)(n < 0 ? (uint64_t)0 - (uint64_t)n : (uint64_t)n);
    u128 p = m * a;                                  /* |n h| 2^16 = p 2^(e - 37) */
    const u128 cap = (u128)1 << 126;
    u128 q;
    int sh = e - 37;
    if (sh >= 0) {
        q = (sh >= 126 || (p >> (126 - sh)) != 0) ? cap : p << sh;
    } else if (-sh >= 128) {
        q = 0;                                       /* p < 2^117 < half a unit */
    } else {
        int r = -sh;
        q = p >> r;
        u128 rem = p & (((u128)1 << r) - 1);
        u128 half = (u128)1 << (r - 1);
        if (rem > half || (rem == half && (q & 1))) q += 1;
    }
    i128 v = (i128)q;
    return ((n < 0) != (h < 0.0)) ? -v : v;
}

double from_fixed(i128 s) {
    int64_t hi = (int64_t)(s >> 64);
    uint64_t lo = (uint64_t)s;
    double d = (double)hi * 18446744073709551616.0 + (double)lo;
    return d * FX_UNSCALE;
}

/* ------------------------------------------------------------------ */
/* Spawned amount in walker fixed point (units of 2^-32 walkers) from  */
/* the exact product of two non-negative finite doubles:               */
/*   round = 0: floor(a * b * 2^32)                                    */
/*   round = 1: floor(a * b * 2^32 + 1/2)                              */
/* One rounding of the exact product, no intermediate double rounding; */
/* results at or above 2^62 saturate to 2^62.                          */
/* ------------------------------------------------------------------ */
const uint64_t AMOUNT_MAX = 1ull << 62;

uint64_t fixed_product(double a, double b, int round) {
    if (a == 0.0 || b == 0.0) return 0;
    int ea, eb;
    double fa = frexp(a, &ea), fb = frexp(b, &eb);   /* a = fa 2^ea, fa in [1/2, 1) */
    uint64_t ma = (uint64_t)ldexp(fa, 53);           /* exact 53-bit integers */
    uint64_t mb = (uint64_t)ldexp(fb, 53);
    u128 p = (u128)ma * mb;                          /* a b 2^32 = p 2^(ea+eb-106+32) */
    int e = ea + eb - 74;
    if (e >= 0) {
        if (e >= 62 || (p >> (62 - e)) != 0) return AMOUNT_MAX;
        return (uint64_t)(p << e);
    }
    int s = -e;
    if (s >= 120) return 0;                          /* p < 2^106: below 2^-14 */
    u128 r = round ? ((p >> (s - 1)) + 1) >> 1 : p >> s;
    return r >= (u128)AMOUNT_MAX ? AMOUNT_MAX : (uint64_t)r;
}

/* ------------------------------------------------------------------ */
/* Determinant helpers.  Spin orbital p = 2*spatial + spin (alpha = 0), */
/* bit p lives in word p/64.  Keys order as unsigned big integers       */
/* (most significant word = word W-1).                                  */
/* ------------------------------------------------------------------ */
struct Ctx;

inline bool occ_bit(const Det& d, int p) { return (d.w[p >> 6] >> (p & 63)) & 1ull; }
inline void flip_bit(Det& d, int p) { d.w[p >> 6] ^= 1ull << (p & 63); }

int det_cmp(const Det& a, const Det& b, int W) {
    for (int i = W - 1; i >= 0; --i) {
        if (a.w[i] < b.w[i]) return -1;
        if (a.w[i] > b.w[i]) return 1;
    }
    return 0;
}

std::vector<int> occ_list(const Det& d, int nspin) {
    std::vector<int> o;
    for (int p = 0; p < nspin; ++p)
        if (occ_bit(d, p)) o.push_back(p);
    return o;
}

/* number of occupied spin orbitals strictly between p and q */
int count_between(const Det& d, int p, int q) {
    int lo = p < q ? p : q, hi = p < q ? q : p;
    int c = 0;
    for (int r = lo + 1; r < hi; ++r) c += occ_bit(d, r);
    return c;
}

/* ------------------------------------------------------------------ */
/* System definitions                                                   */
/* ------------------------------------------------------------------ */
enum { SYS_HUBBARD = 0, SYS_UEG = 1, SYS_MOLECULE = 2 };

struct HBEntry {
    int a, b;          /* spin orbitals, a < b */
    uint64_t cum;      /* cumulative threshold: entry chosen if w < cum (last: catch-all) */
};

struct Walker {
    Det key;
    int64_t pop;
    double hdiag;      /* H_ii - E_ref */
    int core;          /* member of the deterministic space */
};

struct Spawn {
    Det key;
    int64_t amount;
    int init;          /* parent was an initiator */
};

struct Record {
    int64_t iter;
    double shift;
    int64_t nw_pre, n0, nw_post, ndet, natt, nspawn;
    int64_t num_hi;
    uint64_t num_lo;
    double num;
    double tau;        /* the time step iteration t used */
};

struct Ctx {
    /* system */
    int kind, W, norb, nalpha, nbeta, nel, nspin;
    int L, periodic;
    int z;                          /* Hubbard: hopping directions per site */
    std::vector<int> nbr;           /* Hubbard: nbr[site * z + k], -1 = none */
    double t_hop, U;
    /* UEG */
    double rs, box, vfac, kfac;
    std::vector<int> kvec;          /* 3 per spatial orbital */
    int nmax, side;
    std::vector<int> klookup;       /* cube -> spatial orbital or -1 */
    /* molecule */
    std::vector<double> h1, eri;
    double ecore;
    uint32_t psingle_thr;
    double p_single, p_double;
    std::vector<std::vector<HBEntry>> hb;   /* per pair index of (p<q) */
    /* proposal-table generator (UEG): per row r = (I M + J) 2 + same-spin,
     * cumulative integer weights over the particle orbital A (empty = off) */
    int excit_gen;
    std::vector<uint32_t> ptab_cum;
    /* time-step search: the largest |H_ij| / p_gen of any attempt so far */
    int tau_search;
    double rmax;
    /* qmc */
    double tau, target, zeta, cutoff, init_pop, n_a;
    int period, initiator, real_amp, core_size, core_start;
    uint64_t seed, replica;
    int64_t target_fixed, init_thr;
    uint64_t cutoff_fixed;   /* spawn cutoff in walker fixed point */
    /* state */
    Det d0;
    double e_ref;
    std::vector<Walker> main;
    double shift;
    int vary;
    int64_t nw_ref;
    int64_t iter;
    std::vector<Det> core;                 /* sorted by key */
    std::vector<std::vector<std::pair<int, double>>> core_rows;  /* (col, H') */
    std::vector<Record> recs;
    std::string err;
};

/* ---------------- spin-orbital integrals (molecule) ---------------- */
inline double mol_h(const Ctx& c, int p, int q) {
    if ((p & 1) != (q & 1)) return 0.0;
    return c.h1[(size_t)(p >> 1) * c.norb + (q >> 1)];
}
/* chemist notation (pq|rs) over spin orbitals */
inline double mol_g(const Ctx& c, int p, int q, int r, int s) {
    if ((p & 1) != (q & 1) || (r & 1) != (s & 1)) return 0.0;
    size_t n = (size_t)c.norb;
    return c.eri[(((size_t)(p >> 1) * n + (q >> 1)) * n + (r >> 1)) * n + (s >> 1)];
}

/* ---------------- UEG ---------------- */
int ueg_orb_of(const Ctx& c, int nx, int ny, int nz) {
    if (nx < -c.nmax || nx > c.nmax || ny < -c.nmax || ny > c.nmax || nz < -c.nmax || nz > c.nmax)
        return -1;
    int s = c.side;
    return c.klookup[((size_t)(nx + c.nmax) * s + (ny + c.nmax)) * s + (nz + c.nmax)];
}
/* Coulomb kernel 4 pi / (Omega |q|^2) with |q|^2 = (2 pi / L)^2 m  ==  vfac / m */
inline double ueg_v(const Ctx& c, int m) { return c.vfac / (double)m; }
inline int ueg_dist2(const Ctx& c, int P, int Q) {
    int dx = c.kvec[3 * P] - c.kvec[3 * Q];
    int dy = c.kvec[3 * P + 1] - c.kvec[3 * Q + 1];
    int dz = c.kvec[3 * P + 2] - c.kvec[3 * Q + 2];
    return dx * dx + dy * dy + dz * dz;
}
inline int ueg_n2(const Ctx& c, int P) {
    return c.kvec[3 * P] * c.kvec[3 * P] + c.kvec[3 * P + 1] * c.kvec[3 * P + 1] +
           c.kvec[3 * P + 2] * c.kvec[3 * P + 2];
}

/* ------------------------------------------------------------------ */
/* Hamiltonian matrix elements (Slater-Condon rules).                  */
/*   diagonal: sum_k h_kk + sum_{k<l} [(kk|ll) - (kl|lk)]              */
/*   single i->a: sign * (h_ia + sum_{k in D, k != i} [(ia|kk)-(ik|ka)]) */
/*   double i<j -> a<b: sign * [(ia|jb) - (ib|ja)]                     */
/* sign: (-1)^(occupied strictly between i and a in D), then the same  */
/* for j->b on the updated string.  Summations run in ascending order. */
/* ------------------------------------------------------------------ */
double h_diag(const Ctx& c, const Det& d) {
    std::vector<int> o = occ_list(d, c.nspin);
    if (c.kind == SYS_HUBBARD) {
        int dbl = 0;
        for (int s = 0; s < c.L; ++s)
            if (occ_bit(d, 2 * s) && occ_bit(d, 2 * s + 1)) ++dbl;
        return c.U * (double)dbl;
    }
    if (c.kind == SYS_UEG) {
        double e = 0.0;
        for (size_t k = 0; k < o.size(); ++k) e = e + c.kfac * (double)ueg_n2(c, o[k] >> 1);
        for (size_t k = 0; k < o.size(); ++k)
            for (size_t l = k + 1; l < o.size(); ++l)
                if ((o[k] & 1) == (o[l] & 1)) e = e - ueg_v(c, ueg_dist2(c, o[k] >> 1, o[l] >> 1));
        return e;
    }
    double e1 = 0.0, e2 = 0.0;
    for (size_t k = 0; k < o.size(); ++k) e1 = e1 + mol_h(c, o[k], o[k]);
    for (size_t k = 0; k < o.size(); ++k)
        for (size_t l = k + 1; l < o.size(); ++l) {
            int p = o[k], q = o[l];
            e2 = e2 + (mol_g(c, p, p, q, q) - mol_g(c, p, q, q, p));
        }
    return (e1 + e2) + c.ecore;
}

/* <D'|H|D> for D' = D with i->a (i occupied, a empty) */
double h_single(const Ctx& c, const Det& d, int i, int a) {
    Det tmp = d;
    int sgn = (count_between(d, i, a) & 1) ? -1 : 1;
    double v;
    if (c.kind == SYS_HUBBARD) {
        /* hopping -t between nearest-neighbour sites with the same spin */
        if ((i & 1) != (a & 1)) return 0.0;
        int si = i >> 1, sa = a >> 1;
        bool bond = false;
        for (int k = 0; k < c.z; ++k)
            if (c.nbr[(size_t)si * c.z + k] == sa) bond = true;
        if (!bond) return 0.0;
        v = -c.t_hop;
    } else if (c.kind == SYS_UEG) {
        return 0.0;     /* momentum conservation forbids single excitations */
    } else {
        double s = 0.0;
        for (int k = 0; k < c.nspin; ++k) {
            if (k == i || !occ_bit(d, k)) continue;
            s = s + (mol_g(c, i, a, k, k) - mol_g(c, i, k, k, a));
        }
        v = mol_h(c, i, a) + s;
    }
    (void)tmp;
    return sgn < 0 ? -v : v;
}

/* <D'|H|D> for D' = D with i->a, j->b (i<j occupied, a<b empty) */
double h_double(const Ctx& c, const Det& d, int i, int j, int a, int b) {
    Det tmp = d;
    int n1 = count_between(tmp, i, a);
    flip_bit(tmp, i); flip_bit(tmp, a);
    int n2 = count_between(tmp, j, b);
    int sgn = ((n1 + n2) & 1) ? -1 : 1;
    double v;
    if (c.kind == SYS_HUBBARD) {
        return 0.0;
    } else if (c.kind == SYS_UEG) {
        int I = i >> 1, J = j >> 1, A = a >> 1, B = b >> 1;
        /* momentum conservation */
        for (int x = 0; x < 3; ++x)
            if (c.kvec[3 * I + x] + c.kvec[3 * J + x] != c.kvec[3 * A + x] + c.kvec[3 * B + x])
                return 0.0;
        double direct = 0.0, exch = 0.0;
        if ((i & 1) == (a & 1) && (j & 1) == (b & 1)) direct = ueg_v(c, ueg_dist2(c, I, A));
        if ((i & 1) == (b & 1) && (j & 1) == (a & 1)) exch = ueg_v(c, ueg_dist2(c, I, B));
        v = direct - exch;
    } else {
        v = mol_g(c, i, a, j, b) - mol_g(c, i, b, j, a);
    }
    return sgn < 0 ? -v : v;
}

/* general <dt|H|ds>, ds = source (parent), dt = target */
double h_elem(const Ctx& c, const Det& ds, const Det& dt) {
    int nd = 0;
    int from[2], to[2], nf = 0, nt = 0;
    for (int wi = 0; wi < c.W; ++wi) nd += __builtin_popcountll(ds.w[wi] ^ dt.w[wi]);
    if (nd == 0) return h_diag(c, ds);
    if (nd != 2 && nd != 4) return 0.0;
    for (int p = 0; p < c.nspin; ++p) {
        bool x = occ_bit(ds, p), y = occ_bit(dt, p);
        if (x && !y) from[nf++] = p;
        if (!x && y) to[nt++] = p;
    }
    if (nd == 2) return h_single(c, ds, from[0], to[0]);
    return h_double(c, ds, from[0], from[1], to[0], to[1]);
}

/* ------------------------------------------------------------------ */
/* Excitation generators.  Each consumes Philox words w[0..2] and       */
/* returns the child determinant and its exact generation probability. */
/* ------------------------------------------------------------------ */
struct Excit {
    bool null;
    Det child;
    double pgen;
    double hij;
    /* 1/p_gen as two factors inv_a * inv_b, each exact or one rounding of a
     * ratio of the generator's counts and table widths */
    double inv_a, inv_b;
};

/* pair index -> (i, j), i < j, with P = j(j-1)/2 + i */
void unrank_pair(uint64_t P, int& i, int& j) {
    int jj = 1;
    while ((uint64_t)(jj + 1) * jj / 2 <= P) ++jj;
    j = jj;
    i = (int)(P - (uint64_t)jj * (jj - 1) / 2);
}

Excit gen_hubbard(const Ctx& c, const Det& d, const uint64_t w[4]) {
    Excit e;
    e.null = true;
    std::vector<int> o = occ_list(d, c.nspin);
    int n = (int)o.size();
    int p = o[draw_index(w[0], (uint64_t)n)];
    int site = p >> 1, spin = p & 1;
    /* direction k uniform among the z hops (chain: k = 0 right, 1 left) */
    int k = (int)draw_index(w[1], (uint64_t)c.z);
    int ns = c.nbr[(size_t)site * c.z + k];
    if (ns < 0) return e;
    int q = 2 * ns + spin;
    if (occ_bit(d, q)) return e;
    e.pgen = 1.0 / ((double)c.z * (double)n);
    e.inv_a = (double)c.z * (double)n;
    e.inv_b = 1.0;
    e.hij = h_single(c, d, p, q);
    e.child = d;
    flip_bit(e.child, p);
    flip_bit(e.child, q);
    e.null = false;
    return e;
}

Excit gen_ueg(const Ctx& c, const Det& d, const uint64_t w[4]) {
    Excit e;
    e.null = true;
    std::vector<int> o = occ_list(d, c.nspin);
    int n = (int)o.size();
    uint64_t npairs = (uint64_t)n * (n - 1) / 2;
    int ii, jj;
    unrank_pair(draw_index(w[1], npairs), ii, jj);
    int p = o[ii], q = o[jj];
    int A = (int)draw_index(w[2], (uint64_t)c.norb);
    int a = 2 * A + (p & 1);
    int P = p >> 1, Q = q >> 1;
    int B = ueg_orb_of(c, c.kvec[3 * P] + c.kvec[3 * Q] - c.kvec[3 * A],
                       c.kvec[3 * P + 1] + c.kvec[3 * Q + 1] - c.kvec[3 * A + 1],
                       c.kvec[3 * P + 2] + c.kvec[3 * Q + 2] - c.kvec[3 * A + 2]);
    if (B < 0) return e;
    int b = 2 * B + (q & 1);
    if (a == b || occ_bit(d, a) || occ_bit(d, b)) return e;
    double ways = ((p & 1) == (q & 1)) ? 2.0 : 1.0;
    e.pgen = ways / ((double)npairs * (double)c.norb);
    e.inv_a = ((double)npairs * (double)c.norb) / ways;
    e.inv_b = 1.0;
    int lo = a < b ? a : b, hi = a < b ? b : a;
    e.hij = h_double(c, d, p, q, lo, hi);
    e.child = d;
    flip_bit(e.child, p); flip_bit(e.child, q);
    flip_bit(e.child, a); flip_bit(e.child, b);
    e.null = false;
    return e;
}

int pair_index(int p, int q) { return q * (q - 1) / 2 + p; }   /* p < q */

Excit gen_heat_bath(const Ctx& c, const Det& d, const uint64_t w[4]) {
    Excit e;
    e.null = true;
    std::vector<int> o = occ_list(d, c.nspin);
    int n = (int)o.size();
    if ((uint32_t)(w[0] >> 32) < c.psingle_thr) {
        /* single: i uniform over electrons, a uniform over empty orbitals of i's spin */
        int i = o[draw_index(w[1], (uint64_t)n)];
        int spin = i & 1;
        std::vector<int> empty;
        for (int A = 0; A < c.norb; ++A)
            if (!occ_bit(d, 2 * A + spin)) empty.push_back(2 * A + spin);
        if (empty.empty()) return e;
        int a = empty[draw_index(w[2], (uint64_t)empty.size())];
        e.pgen = c.p_single / ((double)n * (double)empty.size());
        e.inv_a = ((double)n * (double)empty.size()) / c.p_single;
        e.inv_b = 1.0;
        e.hij = h_single(c, d, i, a);
        e.child = d;
        flip_bit(e.child, i); flip_bit(e.child, a);
        e.null = false;
        return e;
    }
    uint64_t npairs = (uint64_t)n * (n - 1) / 2;
    int ii, jj;
    unrank_pair(draw_index(w[1], npairs), ii, jj);
    int p = o[ii], q = o[jj];
    const std::vector<HBEntry>& tab = c.hb[pair_index(p, q)];
    if (tab.empty()) return e;
    size_t k = 0;
    while (k + 1 < tab.size() && !(w[2] < tab[k].cum)) ++k;
    int a = tab[k].a, b = tab[k].b;
    if (occ_bit(d, a) || occ_bit(d, b)) return e;
    double pk, inv_pk;
    if (tab.size() == 1) {
        pk = 1.0;
        inv_pk = 1.0;
    } else {
        uint64_t prev = k == 0 ? 0 : tab[k - 1].cum;
        uint64_t width = (k + 1 == tab.size()) ? (0 - prev) : (tab[k].cum - prev);
        pk = (double)width * 0x1p-64;
        inv_pk = 18446744073709551616.0 / (double)width;
    }
    double pg = c.p_double / (double)npairs;
    e.pgen = pg * pk;
    e.inv_a = (double)npairs / c.p_double;
    e.inv_b = inv_pk;
    e.hij = h_double(c, d, p, q, a, b);
    e.child = d;
    flip_bit(e.child, p); flip_bit(e.child, q);
    flip_bit(e.child, a); flip_bit(e.child, b);
    e.null = false;
    return e;
}

/* UEG doubles from a proposal table (the learned proposal's selection table).
 * The occupied pair (i < j) is drawn uniformly as in gen_ueg; the particle
 * orbital A (spin of i) is drawn from the integer weights q_r[A] of the row
 * r = (I M + J) 2 + [spin i == spin j] by inverse CDF over their cumulative
 * sums (Q_r = the row total, x = floor(w2 Q_r / 2^64), A = the first index whose
 * cumulative sum exceeds x); b follows from momentum conservation.  The child
 * {a, b} of a same-spin pair is also drawn through A' = B, so
 *   p_gen = [1 / C(N,2)] (q_A + [same spin] q_B) / Q_r,
 * exact in the integers; 1/p_gen = inv_a inv_b with inv_a = C(N,2) and
 * inv_b = Q_r / (q_A + [same] q_B) (one rounding).  Null when a or b is
 * occupied. */
inline uint32_t ptab_weight(const Ctx& c, size_t row, int A) {
    const uint32_t* cum = &c.ptab_cum[row * (size_t)c.norb];
    return cum[A] - (A > 0 ? cum[A - 1] : 0u);
}

Excit gen_ueg_table(const Ctx& c, const Det& d, const uint64_t w[4]) {
    Excit e;
    e.null = true;
    std::vector<int> o = occ_list(d, c.nspin);
    int n = (int)o.size();
    uint64_t npairs = (uint64_t)n * (n - 1) / 2;
    int ii, jj;
    unrank_pair(draw_index(w[1], npairs), ii, jj);
    int p = o[ii], q = o[jj];
    int I = p >> 1, J = q >> 1, same = (p & 1) == (q & 1) ? 1 : 0;
    size_t row = ((size_t)I * c.norb + J) * 2 + same;
    const uint32_t* cum = &c.ptab_cum[row * (size_t)c.norb];
    uint32_t Q = cum[c.norb - 1];
    if (Q == 0) return e;
    uint64_t x = draw_index(w[2], (uint64_t)Q);
    int A = 0;
    while (!((uint64_t)cum[A] > x)) ++A;
    int B = ueg_orb_of(c, c.kvec[3 * I] + c.kvec[3 * J] - c.kvec[3 * A],
                       c.kvec[3 * I + 1] + c.kvec[3 * J + 1] - c.kvec[3 * A + 1],
                       c.kvec[3 * I + 2] + c.kvec[3 * J + 2] - c.kvec[3 * A + 2]);
    if (B < 0) return e;   /* not drawn: such entries have weight 0 */
    int a = 2 * A + (p & 1), b = 2 * B + (q & 1);
    if (a == b || occ_bit(d, a) || occ_bit(d, b)) return e;
    uint32_t qab = ptab_weight(c, row, A) + (same ? ptab_weight(c, row, B) : 0u);
    e.pgen = ((double)qab / (double)Q) / (double)npairs;
    e.inv_a = (double)npairs;
    e.inv_b = (double)Q / (double)qab;
    int lo = a < b ? a : b, hi = a < b ? b : a;
    e.hij = h_double(c, d, p, q, lo, hi);
    e.child = d;
    flip_bit(e.child, p); flip_bit(e.child, q);
    flip_bit(e.child, a); flip_bit(e.child, b);
    e.null = false;
    return e;
}

Excit generate(const Ctx& c, const Det& d, const uint64_t w[4]) {
    if (c.kind == SYS_HUBBARD) return gen_hubbard(c, d, w);
    if (c.kind == SYS_UEG) return c.excit_gen == 1 ? gen_ueg_table(c, d, w) : gen_ueg(c, d, w);
    return gen_heat_bath(c, d, w);
}

/* Heat-bath tables: for each occupied pair (p<q), all spin-allowed (a<b)
 * with a,b not in {p,q} and weight |(pa|qb) - (pb|qa)| > 0, in ascending
 * (a, b) order; cum_k = floor(2^64 * S_k / S_total), forced strictly
 * increasing, last entry catches the remainder. */
void build_heat_bath(Ctx& c) {
    int ns = c.nspin;
    c.hb.assign((size_t)ns * (ns - 1) / 2, std::vector<HBEntry>());
    for (int q = 1; q < ns; ++q)
        for (int p = 0; p < q; ++p) {
            std::vector<HBEntry> tab;
            std::vector<double> wts;
            for (int a = 0; a < ns; ++a)
                for (int b = a + 1; b < ns; ++b) {
                    if (a == p || a == q || b == p || b == q) continue;
                    int sp = p & 1, sq = q & 1, sa = a & 1, sb = b & 1;
                    if (!((sa == sp && sb == sq) || (sa == sq && sb == sp))) continue;
                    double v = mol_g(c, p, a, q, b) - mol_g(c, p, b, q, a);
                    double wgt = fabs(v);
                    if (!(wgt > 0.0)) continue;
                    HBEntry h;
                    h.a = a; h.b = b; h.cum = 0;
                    tab.push_back(h);
                    wts.push_back(wgt);
                }
            if (!tab.empty()) {
                std::vector<double> cs(wts.size());
                double s = 0.0;
                for (size_t k = 0; k < wts.size(); ++k) { s = s + wts[k]; cs[k] = s; }
                double total = s;
                uint64_t prev = 0;
                for (size_t k = 0; k + 1 < tab.size(); ++k) {
                    double r = cs[k] / total;
                    uint64_t v = r >= 1.0 ? ~0ull : (uint64_t)(r * 18446744073709551616.0);
                    if (v <= prev) v = prev + 1;
                    tab[k].cum = v;
                    prev = v;
                }
                tab.back().cum = ~0ull;    /* catch-all; never compared */
            }
            c.hb[pair_index(p, q)] = tab;
        }
}

/* ------------------------------------------------------------------ */
/* RNG streams: key = (seed, replica); counter = (t, attempt, h0, h1)   */
/* with (h0, h1) the key words for W <= 2 and a SplitMix64 fold above. */
/* ------------------------------------------------------------------ */
void det_hash(const Ctx& c, const Det& d, uint64_t& h0, uint64_t& h1) {
    if (c.W <= 2) {
        h0 = d.w[0];
        h1 = c.W == 2 ? d.w[1] : 0;
        return;
    }
    uint64_t a = 0x243F6A8885A308D3ull, b = 0x13198A2E03707344ull;
    for (int i = 0; i < c.W; ++i) {
        a = mix64(a ^ d.w[i]);
        b = mix64(b ^ d.w[i]);
    }
    h0 = a; h1 = b;
}

void draw(const Ctx& c, int64_t t, uint64_t attempt, const Det& d, uint64_t out[4]) {
    uint64_t ctr[4], key[2];
    uint64_t h0, h1;
    det_hash(c, d, h0, h1);
    ctr[0] = (uint64_t)t; ctr[1] = attempt; ctr[2] = h0; ctr[3] = h1;
    key[0] = c.seed; key[1] = c.replica;
    philox4x64_10(ctr, key, out);
}

/* ------------------------------------------------------------------ */
/* One FCIQMC iteration (Sec. 2.1 / 2.4, App. B)                        */
/* ------------------------------------------------------------------ */
bool is_d0(const Ctx& c, const Det& d) { return det_cmp(d, c.d0, c.W) == 0; }

int exc_level(const Ctx& c, const Det& a, const Det& b) {
    int n = 0;
    for (int i = 0; i < c.W; ++i) n += __builtin_popcountll(a.w[i] ^ b.w[i]);
    return n / 2;
}

bool in_core(const Ctx& c, const Det& d) {
    size_t lo = 0, hi = c.core.size();
    while (lo < hi) {
        size_t mid = (lo + hi) / 2;
        int r = det_cmp(c.core[mid], d, c.W);
        if (r == 0) return true;
        if (r < 0) lo = mid + 1; else hi = mid;
    }
    return false;
}

inline int64_t iabs64(int64_t x) { return x < 0 ? -x : x; }

void select_core(Ctx& c);
void install_core(Ctx& c, std::vector<Det> keys);

/* (1) estimator terms of one entry of M(t-1): N_w, N_0 and the numerator
 * sum_{j != 0} N_j H_0j (App. A.1) */
void estimator_terms(const Ctx& c, const Walker& wk, int64_t& nw, int64_t& n0, i128& num) {
    nw += iabs64(wk.pop);
    if (is_d0(c, wk.key)) {
        n0 = wk.pop;
        return;
    }
    if (wk.pop == 0 || exc_level(c, c.d0, wk.key) > 2) return;
    double h0j = h_elem(c, wk.key, c.d0);
    num += fixed_term(wk.pop, h0j);
}

/* (2) initiator flag (Sec. 2.1) */
int initiator_flag(const Ctx& c, const Walker& wk) {
    if (!c.initiator) return 1;
    return (iabs64(wk.pop) > c.init_thr) || is_d0(c, wk.key) || wk.core;
}

/* (3) the spawning attempts of one determinant (Sec. 2.4); appends its spawns */
void spawn_from(const Ctx& c, int64_t t, const Walker& wk, int init, std::vector<Spawn>& spawned, int64_t& natt_tot,
                double& rmax) {
    if (wk.pop == 0) return;
    uint64_t mag = (uint64_t)iabs64(wk.pop);
    uint64_t wdet[4];
    draw(c, t, SENTINEL_DET, wk.key, wdet);
    uint64_t natt = mag >> 32;
    if (c.real_amp) {
        uint64_t frac = mag & 0xffffffffull;
        if ((wdet[0] >> 32) < frac) natt += 1;
    }
    natt_tot += (int64_t)natt;
    int psign = wk.pop < 0 ? -1 : 1;
    for (uint64_t a = 0; a < natt; ++a) {
        uint64_t w[4];
        draw(c, t, a, wk.key, w);
        Excit ex = generate(c, wk.key, w);
        if (ex.null) continue;
        if (ex.hij == 0.0) continue;
        if (wk.core && in_core(c, ex.child)) continue;   /* exact inside the core */
        /* |H_ij| / p_gen of the attempt, (|H| inv_a) inv_b, while the time-step
         * search runs (until the population first exceeded the target) */
        if (c.tau_search && !c.vary) {
            double ratio = (fabs(ex.hij) * ex.inv_a) * ex.inv_b;
            if (ratio > rmax) rmax = ratio;
        }
        /* spawn weight tau |H_ij| / p_gen = |H_ij| * ct, ct = (tau inv_a) inv_b,
         * taken exactly in walker fixed point (one rounding of the product) */
        double ct = (c.tau * ex.inv_a) * ex.inv_b;
        int64_t q;
        if (!c.real_amp) {
            /* floor(m) walkers, one more with probability frac(m) (frac to 2^-32) */
            uint64_t f = fixed_product(fabs(ex.hij), ct, 0);
            uint64_t k = f >> 32;
            if ((w[3] >> 32) < (f & 0xffffffffull)) k += 1;
            if (k == 0) continue;
            q = k >= (1ull << 30) ? (int64_t)AMOUNT_MAX : (int64_t)(k << 32);
        } else {
            uint64_t r = fixed_product(fabs(ex.hij), ct, 1);
            if (r < c.cutoff_fixed) {   /* kept, as the cutoff, with probability r / cutoff */
                if (draw_index(w[3], c.cutoff_fixed) < r) r = c.cutoff_fixed;
                else continue;
            }
            if (r == 0) continue;
            q = (int64_t)r;
        }
        int hs = ex.hij < 0.0 ? -1 : 1;
        Spawn sp;
        sp.key = ex.child;
        sp.amount = (-hs * psign) < 0 ? -q : q;
        sp.init = init;
        spawned.push_back(sp);
    }
}

/* (4) death / cloning of a non-core determinant from N(t-1): its new population */
int64_t after_death(const Ctx& c, int64_t t, const Walker& wk) {
    if (wk.core || wk.pop == 0) return wk.pop;
    double d = c.tau * (wk.hdiag - c.shift);
    if (c.real_amp) {
        double x = d * (double)wk.pop;
        return wk.pop - llrint(x);
    }
    uint64_t wdet[4];
    draw(c, t, SENTINEL_DET, wk.key, wdet);
    int64_t n = iabs64(wk.pop) >> 32;
    double x = fabs(d) * (double)n;
    double fl = floor(x);
    int64_t k = (int64_t)fl;
    if (draw_unit(wdet[1]) < x - fl) k += 1;
    int64_t nn = d > 0.0 ? n - k : n + k;
    return (wk.pop < 0 ? -nn : nn) * (int64_t)FIXED_ONE;
}

/* positions of the core determinants in the sorted main list */
std::vector<size_t> core_positions(const Ctx& c) {
    std::vector<size_t> pos(c.core.size());
    for (size_t r = 0; r < c.core.size(); ++r) {
        size_t lo = 0, hi = c.main.size();
        while (lo < hi) {
            size_t mid = (lo + hi) / 2;
            if (det_cmp(c.main[mid].key, c.core[r], c.W) < 0) lo = mid + 1; else hi = mid;
        }
        pos[r] = lo;
    }
    return pos;
}

/* (5) semi-stochastic: exact projection of core row r (App. A.2), its new population */
int64_t after_projection(const Ctx& c, size_t r, const std::vector<size_t>& pos) {
    i128 acc = 0;
    for (size_t k = 0; k < c.core_rows[r].size(); ++k) {
        int col = c.core_rows[r][k].first;
        double h = c.core_rows[r][k].second;
        acc += fixed_term(c.main[pos[col]].pop, h);
    }
    double y = from_fixed(acc);
    int64_t pr = c.main[pos[r]].pop;
    double v = y - c.shift * (double)pr;
    double x = c.tau * v;
    return pr - llrint(x);
}

/* (6) annihilation: sort the spawns, combine equal keys, merge them into the
 * sorted main entries main[mine[0]], main[mine[1]], ... (new populations in
 * newpop), initiator rule for new determinants; appends the surviving
 * entries in key order */
void annihilate(const Ctx& c, int64_t t, std::vector<Spawn>& spawned, const std::vector<size_t>& mine,
                const std::vector<int64_t>& newpop, std::vector<Walker>& out) {
    const int W = c.W;
    std::sort(spawned.begin(), spawned.end(), [W](const Spawn& x, const Spawn& y) {
        return det_cmp(x.key, y.key, W) < 0;
    });
    std::vector<Spawn> merged;
    for (size_t k = 0; k < spawned.size(); ++k) {
        if (!merged.empty() && det_cmp(merged.back().key, spawned[k].key, W) == 0) {
            merged.back().amount += spawned[k].amount;
            merged.back().init |= spawned[k].init;
        } else {
            merged.push_back(spawned[k]);
        }
    }
    size_t im = 0, is = 0;
    while (im < mine.size() || is < merged.size()) {
        int r;
        if (im == mine.size()) r = 1;
        else if (is == merged.size()) r = -1;
        else r = det_cmp(c.main[mine[im]].key, merged[is].key, W);
        Walker nw;
        if (r < 0) {
            nw = c.main[mine[im]];
            nw.pop = newpop[mine[im]];
            ++im;
        } else if (r == 0) {
            nw = c.main[mine[im]];
            nw.pop = newpop[mine[im]] + merged[is].amount;
            ++im; ++is;
        } else {
            const Spawn& sp = merged[is];
            ++is;
            if (c.initiator && !sp.init) continue;
            if (sp.amount == 0) continue;
            nw.key = sp.key;
            nw.pop = sp.amount;
            nw.hdiag = h_diag(c, sp.key) - c.e_ref;
            nw.core = 0;
        }
        bool keep_always = nw.core || is_d0(c, nw.key);
        if (!keep_always && c.real_amp) {
            int64_t mag = iabs64(nw.pop);
            if (mag > 0 && mag < (int64_t)FIXED_ONE) {
                uint64_t wdet[4];
                draw(c, t, SENTINEL_DET, nw.key, wdet);
                int64_t rounded = ((wdet[2] >> 32) < (uint64_t)mag) ? (int64_t)FIXED_ONE : 0;
                nw.pop = nw.pop < 0 ? -rounded : rounded;
            }
        }
        if (nw.pop == 0 && !keep_always) continue;
        out.push_back(nw);
    }
}

/* (7) shift update (Sec. 2.1): S <- S - zeta/(A tau) ln(N_w(t)/N_w(t-A)), the
 * record, and (8) the deterministic space "high", chosen once at start_iteration */
void finish_iteration(Ctx& c, Record& rec, int64_t t) {
    int64_t nw_post = 0;
    for (size_t i = 0; i < c.main.size(); ++i) nw_post += iabs64(c.main[i].pop);
    if (c.vary) {
        if (t % c.period == 0) {
            double ratio = (double)nw_post / (double)c.nw_ref;
            double coef = c.zeta / ((double)c.period * c.tau);
            c.shift = c.shift - coef * own_log(ratio);
            c.nw_ref = nw_post;
        }
    } else if (nw_post > c.target_fixed) {
        c.vary = 1;
        c.nw_ref = nw_post;
    }
    rec.shift = c.shift;
    rec.nw_post = nw_post;
    rec.ndet = (int64_t)c.main.size();
    rec.tau = c.tau;
    c.recs.push_back(rec);
    /* time-step search (the tutorial's tau_search): until the population first
     * exceeds the target, the next iteration's time step is the largest that
     * keeps every spawn seen so far at or below one walker, never larger than now */
    if (c.tau_search && !c.vary && c.rmax > 0.0) {
        double cand = 1.0 / c.rmax;
        if (cand < c.tau) c.tau = cand;
    }
    if (c.core_size > 0 && t == c.core_start) select_core(c);
}

/* One FCIQMC iteration (Sec. 2.1 / 2.4, App. B), steps (1)-(8) in order. */
void iterate_once(Ctx& c) {
    const int64_t t = ++c.iter;
    Record rec;
    memset(&rec, 0, sizeof rec);
    rec.iter = t;
    i128 num = 0;
    for (size_t i = 0; i < c.main.size(); ++i) estimator_terms(c, c.main[i], rec.nw_pre, rec.n0, num);
    rec.num_hi = (int64_t)(num >> 64);
    rec.num_lo = (uint64_t)num;
    rec.num = from_fixed(num);
    std::vector<int> init(c.main.size());
    for (size_t i = 0; i < c.main.size(); ++i) init[i] = initiator_flag(c, c.main[i]);
    std::vector<Spawn> spawned;
    for (size_t i = 0; i < c.main.size(); ++i) spawn_from(c, t, c.main[i], init[i], spawned, rec.natt, c.rmax);
    rec.nspawn = (int64_t)spawned.size();
    std::vector<int64_t> newpop(c.main.size());
    for (size_t i = 0; i < c.main.size(); ++i) newpop[i] = after_death(c, t, c.main[i]);
    if (!c.core.empty()) {
        std::vector<size_t> pos = core_positions(c);
        for (size_t r = 0; r < c.core.size(); ++r) newpop[pos[r]] = after_projection(c, r, pos);
    }
    std::vector<size_t> all(c.main.size());
    for (size_t i = 0; i < all.size(); ++i) all[i] = i;
    std::vector<Walker> out;
    out.reserve(c.main.size() + spawned.size());
    annihilate(c, t, spawned, all, newpop, out);
    c.main.swap(out);
    finish_iteration(c, rec, t);
}

#ifdef _OPENMP
/* The same iteration on P threads, partitioned like the paper's parallel code
 * (App. B, Parallelization): determinant D belongs to owner(D) = h(D) mod P
 * (a SplitMix64 fold of its key words; the paper uses MurmurHash2).  Each
 * thread takes one contiguous block of the list for the estimator terms,
 * spawning, death and projection, and sends every spawn to its child's owner
 * (the all-to-all exchange); each owner then sorts the spawns it received and
 * merges them into its own determinants; the owners' sorted lists are merged.
 * Random numbers are counter-based and all sums exact integers, so the result
 * is the serial iteration's bit for bit. */
int owner_of(const Ctx& c, const Det& d, int P) {
    uint64_t x = 0x243F6A8885A308D3ull;
    for (int i = 0; i < c.W; ++i) x = mix64(x ^ d.w[i]);
    return (int)(x % (uint64_t)P);
}

void iterate_once_parallel(Ctx& c, int P) {
    const int64_t t = ++c.iter;
    Record rec;
    memset(&rec, 0, sizeof rec);
    rec.iter = t;
    const size_t n = c.main.size();
    std::vector<int64_t> nw(P, 0), n0(P, 0), natt(P, 0);
    std::vector<double> rmx(P, 0.0);
    std::vector<i128> num(P, 0);
    std::vector<int> has0(P, 0);
    std::vector<int64_t> newpop(n);
    std::vector<std::vector<std::vector<Spawn>>> outbox(P, std::vector<std::vector<Spawn>>(P));
    std::vector<std::vector<size_t>> mine(P);
    std::vector<size_t> pos;
    if (!c.core.empty()) pos = core_positions(c);
#pragma omp parallel num_threads(P)
    {
        const int p = omp_get_thread_num();
        const size_t beg = n * (size_t)p / (size_t)P, end = n * (size_t)(p + 1) / (size_t)P;
        for (size_t i = beg; i < end; ++i) {
            int64_t z = 0;
            estimator_terms(c, c.main[i], nw[p], z, num[p]);
            if (is_d0(c, c.main[i].key)) { n0[p] = z; has0[p] = 1; }
        }
        std::vector<Spawn> local;
        for (size_t i = beg; i < end; ++i) {
            local.clear();
            spawn_from(c, t, c.main[i], initiator_flag(c, c.main[i]), local, natt[p], rmx[p]);
            for (size_t k = 0; k < local.size(); ++k) outbox[p][owner_of(c, local[k].key, P)].push_back(local[k]);
            newpop[i] = after_death(c, t, c.main[i]);
        }
#pragma omp barrier
#pragma omp for schedule(static)
        for (long r = 0; r < (long)c.core.size(); ++r) newpop[pos[r]] = after_projection(c, (size_t)r, pos);
        /* annihilation by owner */
        for (size_t i = 0; i < n; ++i)
            if (owner_of(c, c.main[i].key, P) == p) mine[p].push_back(i);
    }
    for (int p = 0; p < P; ++p) {
        if (rmx[p] > c.rmax) c.rmax = rmx[p];
        rec.nw_pre += nw[p];
        if (has0[p]) rec.n0 = n0[p];
        rec.natt += natt[p];
        for (int q = 0; q < P; ++q) rec.nspawn += (int64_t)outbox[p][q].size();
    }
    i128 tot = 0;
    for (int p = 0; p < P; ++p) tot += num[p];
    rec.num_hi = (int64_t)(tot >> 64);
    rec.num_lo = (uint64_t)tot;
    rec.num = from_fixed(tot);
    std::vector<std::vector<Walker>> part(P);
#pragma omp parallel num_threads(P)
    {
        const int p = omp_get_thread_num();
        std::vector<Spawn> recv;
        for (int q = 0; q < P; ++q) recv.insert(recv.end(), outbox[q][p].begin(), outbox[q][p].end());
        annihilate(c, t, recv, mine[p], newpop, part[p]);
    }
    /* merge the owners' sorted lists */
    const int W = c.W;
    std::vector<Walker> out;
    for (int p = 0; p < P; ++p) out.insert(out.end(), part[p].begin(), part[p].end());
    std::sort(out.begin(), out.end(), [W](const Walker& x, const Walker& y) { return det_cmp(x.key, y.key, W) < 0; });
    c.main.swap(out);
    finish_iteration(c, rec, t);
}
#endif

/* core = D0 plus the (size-1) other determinants of largest |N|, ties by key */
void select_core(Ctx& c) {
    std::vector<size_t> idx;
    for (size_t i = 0; i < c.main.size(); ++i)
        if (!is_d0(c, c.main[i].key)) idx.push_back(i);
    const Ctx& cc = c;
    std::stable_sort(idx.begin(), idx.end(), [&cc](size_t x, size_t y) {
        int64_t ax = iabs64(cc.main[x].pop), ay = iabs64(cc.main[y].pop);
        if (ax != ay) return ax > ay;
        return det_cmp(cc.main[x].key, cc.main[y].key, cc.W) < 0;
    });
    size_t ntake = (size_t)c.core_size - 1;
    if (ntake > idx.size()) ntake = idx.size();
    std::vector<Det> keys;
    keys.push_back(c.d0);
    for (size_t k = 0; k < ntake; ++k) keys.push_back(c.main[idx[k]].key);
    install_core(c, keys);
}

/* make `keys` the deterministic space: sorted, members flagged in the list,
 * H' in rows and columns of key order */
void install_core(Ctx& c, std::vector<Det> keys) {
    const int W = c.W;
    std::sort(keys.begin(), keys.end(), [W](const Det& x, const Det& y) { return det_cmp(x, y, W) < 0; });
    c.core = keys;
    for (size_t i = 0; i < c.main.size(); ++i) c.main[i].core = in_core(c, c.main[i].key) ? 1 : 0;
    /* H' = H - E_ref on the diagonal; rows and columns in key order */
    c.core_rows.assign(c.core.size(), std::vector<std::pair<int, double>>());
    for (size_t r = 0; r < c.core.size(); ++r)
        for (size_t k = 0; k < c.core.size(); ++k) {
            if (exc_level(c, c.core[r], c.core[k]) > 2) continue;
            double h;
            if (r == k) h = h_diag(c, c.core[r]) - c.e_ref;
            else h = h_elem(c, c.core[k], c.core[r]);
            if (h == 0.0) continue;                 /* zero elements add nothing */
            c.core_rows[r].push_back(std::make_pair((int)k, h));
        }
}

}  /* namespace */

/* ======================= C interface for the tests ======================= */
extern "C" {

typedef struct {
    int kind, key_words, norb, nalpha, nbeta, periodic;
    double t, U, rs;
    const double* h1;
    const double* eri;
    double ecore;
    int ndim;           /* Hubbard lattice: 0 = 1D chain of norb sites, else lattice vectors */
    int lattice[9];     /* row k = vector a_k (ndim x ndim, row-major in a 3 x 3 array) */
} orc_system;

/* Hubbard sites and hops.  ndim = 0: a chain of L sites, hops to s + 1 (k = 0)
 * and s - 1 (k = 1), wrapped when periodic (L >= 3), else none past the ends.
 * ndim = d >= 1: the real-space lattice spanned by the integer rows a_k of the
 * paper's `lattice` input, periodic in each: the sites are the integer points
 * r whose fractional coordinates f = r A^-1 lie in [0, 1)^d, in lexicographic
 * order of r (sublattice-interleaved for a bipartite cell, see below); hop k
 * goes to r + e_{k/2} (k even) or r - e_{k/2} (k odd),
 * reduced into the cell by lattice vectors.  The 2d hops of a site must reach
 * 2d distinct other sites.  Returns false for an invalid lattice. */
static bool build_hubbard_sites(Ctx& c, int ndim, const int* lat) {
    if (ndim == 0) {
        c.z = 2;
        c.nbr.assign((size_t)c.L * 2, -1);
        for (int s = 0; s < c.L; ++s) {
            int r = s + 1, l = s - 1;
            if (c.periodic) { r %= c.L; l = (l + c.L) % c.L; }
            c.nbr[(size_t)s * 2] = (r >= 0 && r < c.L) ? r : -1;
            c.nbr[(size_t)s * 2 + 1] = (l >= 0 && l < c.L) ? l : -1;
        }
        return true;
    }
    if (ndim > 3) return false;
    const int d = ndim;
    long long A[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) A[i][j] = lat[3 * i + j];
    /* adjugate and determinant of the d x d block (identity elsewhere) */
    long long adj[3][3], det;
    adj[0][0] = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    adj[0][1] = A[0][2] * A[2][1] - A[0][1] * A[2][2];
    adj[0][2] = A[0][1] * A[1][2] - A[0][2] * A[1][1];
    adj[1][0] = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    adj[1][1] = A[0][0] * A[2][2] - A[0][2] * A[2][0];
    adj[1][2] = A[0][2] * A[1][0] - A[0][0] * A[1][2];
    adj[2][0] = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    adj[2][1] = A[0][1] * A[2][0] - A[0][0] * A[2][1];
    adj[2][2] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    det = A[0][0] * adj[0][0] + A[0][1] * adj[1][0] + A[0][2] * adj[2][0];
    if (det == 0) return false;
    long long D = det < 0 ? -det : det, sg = det < 0 ? -1 : 1;
    if (D != c.L) return false;
    /* f = r adj / det: r is in the cell iff 0 <= (r adj sg)_k < D */
    auto frac = [&](const long long r[3], long long g[3]) {
        for (int k = 0; k < 3; ++k) g[k] = sg * (r[0] * adj[0][k] + r[1] * adj[1][k] + r[2] * adj[2][k]);
    };
    long long lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int m = 0; m < (1 << d); ++m) {
        long long v[3] = {0, 0, 0};
        for (int i = 0; i < d; ++i)
            if (m >> i & 1)
                for (int j = 0; j < d; ++j) v[j] += A[i][j];
        for (int j = 0; j < d; ++j) { if (v[j] < lo[j]) lo[j] = v[j]; if (v[j] > hi[j]) hi[j] = v[j]; }
    }
    std::vector<std::vector<long long>> sites;
    long long r[3] = {0, 0, 0};
    for (r[0] = lo[0]; r[0] <= hi[0]; ++r[0])
        for (r[1] = d > 1 ? lo[1] : 0; r[1] <= (d > 1 ? hi[1] : 0); ++r[1])
            for (r[2] = d > 2 ? lo[2] : 0; r[2] <= (d > 2 ? hi[2] : 0); ++r[2]) {
                long long g[3];
                frac(r, g);
                bool in = true;
                for (int k = 0; k < d; ++k) in = in && g[k] >= 0 && g[k] < D;
                if (in) sites.push_back({r[0], r[1], r[2]});
            }
    if ((long long)sites.size() != D) return false;
    /* a cell whose lattice vectors all have even coordinate sums is bipartite
     * (checkerboard by the parity of x + y + z) with equal halves: order it
     * sublattice-interleaved (even-parity site, odd-parity site, ...), each half
     * in lexicographic order, so that the reference (alpha on even indices,
     * beta on odd) is the Neel state */
    bool bip = D % 2 == 0;
    for (int i = 0; i < d; ++i) {
        long long sum = 0;
        for (int j = 0; j < d; ++j) sum += A[i][j];
        if (sum % 2 != 0) bip = false;
    }
    if (bip) {
        std::vector<std::vector<long long>> ev, od;
        for (size_t i = 0; i < sites.size(); ++i) {
            long long par = sites[i][0] + sites[i][1] + sites[i][2];
            if (((par % 2) + 2) % 2 == 0) ev.push_back(sites[i]); else od.push_back(sites[i]);
        }
        if (ev.size() == od.size()) {
            sites.clear();
            for (size_t i = 0; i < ev.size(); ++i) { sites.push_back(ev[i]); sites.push_back(od[i]); }
        }
    }
    auto index_of = [&](long long x[3]) -> int {
        for (size_t i = 0; i < sites.size(); ++i)
            if (sites[i][0] == x[0] && sites[i][1] == x[1] && sites[i][2] == x[2]) return (int)i;
        return -1;
    };
    c.z = 2 * d;
    c.nbr.assign((size_t)c.L * c.z, -1);
    for (int s = 0; s < c.L; ++s)
        for (int k = 0; k < c.z; ++k) {
            long long x[3] = {sites[s][0], sites[s][1], sites[s][2]};
            x[k / 2] += (k & 1) ? -1 : 1;
            long long g[3];
            frac(x, g);
            for (int i = 0; i < d; ++i) {      /* n_i = floor(g_i / D), x -= n A */
                long long n = g[i] >= 0 ? g[i] / D : -((-g[i] + D - 1) / D);
                for (int j = 0; j < d; ++j) x[j] -= n * A[i][j];
            }
            int t = index_of(x);
            if (t < 0 || t == s) return false;
            for (int k2 = 0; k2 < k; ++k2)
                if (c.nbr[(size_t)s * c.z + k2] == t) return false;
            c.nbr[(size_t)s * c.z + k] = t;
        }
    return true;
}

typedef struct {
    double tau, target_population, shift_damping, spawn_cutoff, init_pop, initiator_threshold;
    double p_single;
    int shift_period, initiator, real_amplitudes, semi_stoch_size, semi_stoch_start;
    uint64_t seed, replica;
    int excit_gen;      /* 0: the system's generator; 1: proposal table (UEG) */
    int tau_search;     /* 1: time-step search until the population exceeds the target */
} orc_qmc;

void orc_philox(const uint64_t* ctr, const uint64_t* key, uint64_t* out) { philox4x64_10(ctr, key, out); }
double orc_log(double x) { return own_log(x); }
uint64_t orc_fixed_product(double a, double b, int round) { return fixed_product(a, b, round); }
void orc_fixed_term(int64_t n, double h, int64_t* hi, uint64_t* lo) {
    i128 v = fixed_term(n, h);
    *hi = (int64_t)(v >> 64);
    *lo = (uint64_t)v;
}

/* a particle orbital A is drawable in row (I, J, same) when its momentum
 * partner B = k_I + k_J - k_A is in the basis and, for a same-spin pair, B != A */
static bool ptab_valid(const Ctx& c, int I, int J, int same, int A) {
    int B = ueg_orb_of(c, c.kvec[3 * I] + c.kvec[3 * J] - c.kvec[3 * A],
                       c.kvec[3 * I + 1] + c.kvec[3 * J + 1] - c.kvec[3 * A + 1],
                       c.kvec[3 * I + 2] + c.kvec[3 * J + 2] - c.kvec[3 * A + 2]);
    return B >= 0 && !(same && B == A);
}

/* install integer weights q[rows][M] (rows = 2 M^2) as cumulative sums */
static void set_ptab(Ctx& c, const uint32_t* q) {
    size_t rows = (size_t)c.norb * c.norb * 2;
    c.ptab_cum.assign(rows * (size_t)c.norb, 0u);
    for (size_t r = 0; r < rows; ++r) {
        uint32_t s = 0;
        for (int A = 0; A < c.norb; ++A) {
            s += q[r * (size_t)c.norb + A];
            c.ptab_cum[r * (size_t)c.norb + A] = s;
        }
    }
}

static bool setup_ueg(Ctx& c) {
    const double PI = 3.14159265358979323846;
    /* basis: plane waves k = 2 pi n / L sorted by (|n|^2, nx, ny, nz) */
    int R = 1;
    for (;;) {
        int cnt = 0;
        for (int x = -R; x <= R; ++x)
            for (int y = -R; y <= R; ++y)
                for (int z = -R; z <= R; ++z)
                    if (x * x + y * y + z * z <= R * R) ++cnt;
        if (cnt > c.norb) break;
        ++R;
    }
    std::vector<std::vector<int>> pts;
    for (int x = -R; x <= R; ++x)
        for (int y = -R; y <= R; ++y)
            for (int z = -R; z <= R; ++z)
                if (x * x + y * y + z * z <= R * R) pts.push_back({x * x + y * y + z * z, x, y, z});
    std::sort(pts.begin(), pts.end());
    c.kvec.clear();
    c.nmax = 0;
    for (int i = 0; i < c.norb; ++i) {
        for (int k = 1; k <= 3; ++k) {
            c.kvec.push_back(pts[i][k]);
            int a = pts[i][k] < 0 ? -pts[i][k] : pts[i][k];
            if (a > c.nmax) c.nmax = a;
        }
    }
    c.side = 2 * c.nmax + 1;
    c.klookup.assign((size_t)c.side * c.side * c.side, -1);
    for (int i = 0; i < c.norb; ++i)
        c.klookup[((size_t)(c.kvec[3 * i] + c.nmax) * c.side + (c.kvec[3 * i + 1] + c.nmax)) * c.side +
                  (c.kvec[3 * i + 2] + c.nmax)] = i;
    /* Wigner-Seitz radius: Omega = (4 pi / 3) r_s^3 N, L = Omega^(1/3) */
    c.box = c.rs * cbrt(4.0 * PI * (double)c.nel / 3.0);
    c.vfac = 1.0 / (PI * c.box);                     /* 4pi/(Omega (2pi/L)^2) */
    double kf = 2.0 * PI / c.box;
    c.kfac = 0.5 * (kf * kf);                         /* |k|^2/2 = kfac |n|^2 */
    return true;
}

void* orc_create(const orc_system* s, const orc_qmc* q) {
    Ctx* c = new Ctx();
    c->kind = s->kind;
    c->W = s->key_words;
    c->norb = s->norb;
    c->nalpha = s->nalpha;
    c->nbeta = s->nbeta;
    c->nel = s->nalpha + s->nbeta;
    c->nspin = 2 * s->norb;
    c->L = s->norb;
    c->periodic = s->periodic;
    c->t_hop = s->t;
    c->U = s->U;
    c->rs = s->rs;
    c->ecore = s->ecore;
    if (c->W < 1 || c->W > MAXW || c->nspin > 64 * c->W) { delete c; return nullptr; }
    if (c->kind == SYS_HUBBARD && s->ndim == 0 && c->periodic && c->L < 3) { delete c; return nullptr; }
    if (c->kind == SYS_HUBBARD && !build_hubbard_sites(*c, s->ndim, s->lattice)) { delete c; return nullptr; }
    if (c->kind == SYS_MOLECULE) {
        size_t n = (size_t)c->norb;
        c->h1.assign(s->h1, s->h1 + n * n);
        c->eri.assign(s->eri, s->eri + n * n * n * n);
    }
    c->tau = q->tau;
    c->target = q->target_population;
    c->zeta = q->shift_damping;
    c->cutoff = q->spawn_cutoff;
    c->init_pop = q->init_pop;
    c->n_a = q->initiator_threshold;
    c->period = q->shift_period > 0 ? q->shift_period : 1;
    c->initiator = q->initiator;
    c->real_amp = q->real_amplitudes;
    c->core_size = q->semi_stoch_size;
    c->core_start = q->semi_stoch_start;
    c->seed = q->seed;
    c->replica = q->replica;
    c->excit_gen = q->excit_gen;
    c->tau_search = q->tau_search;
    c->rmax = 0.0;
    if (c->excit_gen != 0 && !(c->excit_gen == 1 && c->kind == SYS_UEG)) { delete c; return nullptr; }
    /* thresholds in fixed point, saturated at the int64 range */
    c->target_fixed = c->target * 4294967296.0 >= 9223372036854775807.0
                          ? INT64_MAX : llrint(c->target * 4294967296.0);
    c->init_thr = c->n_a * 4294967296.0 >= 9223372036854775807.0
                      ? INT64_MAX : llrint(c->n_a * 4294967296.0);
    c->cutoff_fixed = c->cutoff * 4294967296.0 >= 4611686018427387904.0
                          ? AMOUNT_MAX : (uint64_t)llrint(c->cutoff * 4294967296.0);
    /* p_single as an exact dyadic: threshold on the top 32 bits of a word */
    c->psingle_thr = (uint32_t)llrint(q->p_single * 4294967296.0);
    c->p_single = (double)c->psingle_thr * 0x1p-32;
    c->p_double = (double)(4294967296ull - c->psingle_thr) * 0x1p-32;

    memset(&c->d0, 0, sizeof c->d0);
    if (c->kind == SYS_HUBBARD) {
        /* Neel reference: alpha on even sites, beta on odd sites */
        if (c->nalpha > (c->L + 1) / 2 || c->nbeta > c->L / 2) { delete c; return nullptr; }
        for (int k = 0; k < c->nalpha; ++k) flip_bit(c->d0, 2 * (2 * k) + 0);
        for (int k = 0; k < c->nbeta; ++k) flip_bit(c->d0, 2 * (2 * k + 1) + 1);
    } else {
        if (c->kind == SYS_UEG) {
            setup_ueg(*c);
            if (c->excit_gen == 1) {
                /* until a table is given: weight 1 on every valid particle orbital */
                std::vector<uint32_t> q((size_t)c->norb * c->norb * 2 * c->norb, 0u);
                for (int I = 0; I < c->norb; ++I)
                    for (int J = 0; J < c->norb; ++J)
                        for (int same = 0; same < 2; ++same)
                            for (int A = 0; A < c->norb; ++A)
                                if (ptab_valid(*c, I, J, same, A))
                                    q[(((size_t)I * c->norb + J) * 2 + same) * c->norb + A] = 1;
                set_ptab(*c, q.data());
            }
        }
        for (int k = 0; k < c->nalpha; ++k) flip_bit(c->d0, 2 * k);
        for (int k = 0; k < c->nbeta; ++k) flip_bit(c->d0, 2 * k + 1);
        if (c->kind == SYS_MOLECULE) build_heat_bath(*c);
    }
    c->e_ref = h_diag(*c, c->d0);
    Walker w0;
    w0.key = c->d0;
    w0.pop = llrint(c->init_pop * 4294967296.0);
    w0.hdiag = 0.0;
    w0.core = 0;
    c->main.push_back(w0);
    c->shift = 0.0;
    c->vary = 0;
    c->nw_ref = 0;
    c->iter = 0;
    return c;
}

void orc_destroy(void* h) { delete (Ctx*)h; }

void orc_iterate(void* h, int n) {
    Ctx* c = (Ctx*)h;
    for (int i = 0; i < n; ++i) iterate_once(*c);
}

/* n iterations on `threads` threads (the hash-partitioned form; bit-identical
 * to orc_iterate).  Returns 0, or -1 in a build without OpenMP. */
int orc_iterate_parallel(void* h, int n, int threads) {
#ifdef _OPENMP
    Ctx* c = (Ctx*)h;
    if (threads < 1) threads = omp_get_max_threads();
    for (int i = 0; i < n; ++i) iterate_once_parallel(*c, threads);
    return 0;
#else
    (void)h; (void)n; (void)threads;
    return -1;
#endif
}

int64_t orc_nrec(void* h) { return (int64_t)((Ctx*)h)->recs.size(); }
int64_t orc_ndet(void* h) { return (int64_t)((Ctx*)h)->main.size(); }
double orc_eref(void* h) { return ((Ctx*)h)->e_ref; }
double orc_shift(void* h) { return ((Ctx*)h)->shift; }

/* keys: W words per walker (word 0 first); flags bit0 = core */
int64_t orc_get_walkers(void* h, uint64_t* keys, int64_t* pops, double* hdiag, uint8_t* flags, int64_t cap) {
    Ctx* c = (Ctx*)h;
    int64_t n = (int64_t)c->main.size();
    if (n > cap) return -n;
    for (int64_t i = 0; i < n; ++i) {
        const Walker& wk = c->main[(size_t)i];
        for (int k = 0; k < c->W; ++k) keys[i * c->W + k] = wk.key.w[k];
        pops[i] = wk.pop;
        hdiag[i] = wk.hdiag;
        flags[i] = (uint8_t)(wk.core ? 1 : 0);
    }
    return n;
}

/* replace the walker list (sorted by key is required) -- test hook */
int orc_set_walkers(void* h, const uint64_t* keys, const int64_t* pops, int64_t n) {
    Ctx* c = (Ctx*)h;
    c->main.clear();
    for (int64_t i = 0; i < n; ++i) {
        Walker wk;
        memset(&wk.key, 0, sizeof wk.key);
        for (int k = 0; k < c->W; ++k) wk.key.w[k] = keys[i * c->W + k];
        wk.pop = pops[i];
        wk.hdiag = h_diag(*c, wk.key) - c->e_ref;
        wk.core = 0;
        if (!c->main.empty() && det_cmp(c->main.back().key, wk.key, c->W) >= 0) return -1;
        c->main.push_back(wk);
    }
    /* start_iteration 0: the deterministic space is taken from the list as
     * given before the first iteration; later a chosen space is kept and its
     * members flagged in the new list, which must hold all of them */
    if (c->core_size > 0 && c->core_start == 0 && c->iter == 0) {
        select_core(*c);
    } else if (!c->core.empty()) {
        int64_t found = 0;
        for (size_t i = 0; i < c->main.size(); ++i) {
            c->main[i].core = in_core(*c, c->main[i].key) ? 1 : 0;
            found += c->main[i].core;
        }
        if (found != (int64_t)c->core.size()) return -2;
    }
    return 0;
}

/* records: 11 int64/double slots per iteration, see Record */
int64_t orc_records(void* h, int64_t* iter, double* shift, int64_t* nw_pre, int64_t* n0, double* num,
                    int64_t* num_hi, uint64_t* num_lo, int64_t* nw_post, int64_t* ndet, int64_t* natt,
                    int64_t* nspawn, double* tau, int64_t cap) {
    Ctx* c = (Ctx*)h;
    int64_t n = (int64_t)c->recs.size();
    if (n > cap) n = cap;
    for (int64_t i = 0; i < n; ++i) {
        const Record& r = c->recs[(size_t)i];
        iter[i] = r.iter; shift[i] = r.shift; nw_pre[i] = r.nw_pre; n0[i] = r.n0;
        num[i] = r.num; num_hi[i] = r.num_hi; num_lo[i] = r.num_lo; nw_post[i] = r.nw_post;
        ndet[i] = r.ndet; natt[i] = r.natt; nspawn[i] = r.nspawn; tau[i] = r.tau;
    }
    return n;
}

void orc_reference(void* h, uint64_t* key) {
    Ctx* c = (Ctx*)h;
    for (int k = 0; k < c->W; ++k) key[k] = c->d0.w[k];
}

double orc_hdiag(void* h, const uint64_t* key) {
    Ctx* c = (Ctx*)h;
    Det d;
    memset(&d, 0, sizeof d);
    for (int k = 0; k < c->W; ++k) d.w[k] = key[k];
    return h_diag(*c, d);
}

/* <target|H|source> */
double orc_hij(void* h, const uint64_t* source, const uint64_t* target) {
    Ctx* c = (Ctx*)h;
    Det s, t;
    memset(&s, 0, sizeof s);
    memset(&t, 0, sizeof t);
    for (int k = 0; k < c->W; ++k) { s.w[k] = source[k]; t.w[k] = target[k]; }
    return h_elem(*c, s, t);
}

/* one excitation from the Philox words w[4]; returns 0 if null */
int orc_generate(void* h, const uint64_t* key, const uint64_t* w, uint64_t* child, double* pgen, double* hij,
                 double* inv) {
    Ctx* c = (Ctx*)h;
    Det d;
    memset(&d, 0, sizeof d);
    for (int k = 0; k < c->W; ++k) d.w[k] = key[k];
    Excit e = generate(*c, d, w);
    if (e.null) return 0;
    for (int k = 0; k < c->W; ++k) child[k] = e.child.w[k];
    *pgen = e.pgen;
    *hij = e.hij;
    if (inv) {
        inv[0] = e.inv_a;
        inv[1] = e.inv_b;
    }
    return 1;
}

/* Every selection path of the generator from `key` with its probability.
 * Returns the number of paths (children[k] all-zero words = null path). */
int64_t orc_enumerate(void* h, const uint64_t* key, uint64_t* children, double* probs, int64_t cap) {
    Ctx* c = (Ctx*)h;
    Det d;
    memset(&d, 0, sizeof d);
    for (int k = 0; k < c->W; ++k) d.w[k] = key[k];
    std::vector<int> o = occ_list(d, c->nspin);
    int n = (int)o.size();
    std::vector<std::pair<Det, double>> paths;
    Det zero;
    memset(&zero, 0, sizeof zero);
    auto add = [&](const Det* ch, double p) { paths.push_back(std::make_pair(ch ? *ch : zero, p)); };
    if (c->kind == SYS_HUBBARD) {
        for (int k = 0; k < n; ++k)
            for (int dir = 0; dir < c->z; ++dir) {
                uint64_t w[4] = {0, 0, 0, 0};
                /* smallest words mapping to electron k and direction dir */
                w[0] = (uint64_t)((((u128)k << 64) + (uint64_t)n - 1) / (uint64_t)n);
                w[1] = (uint64_t)((((u128)(uint64_t)dir << 64) + (uint64_t)c->z - 1) / (uint64_t)c->z);
                Excit e = generate(*c, d, w);
                add(e.null ? nullptr : &e.child, 1.0 / ((double)c->z * n));
            }
    } else if (c->kind == SYS_UEG && c->excit_gen == 1) {
        uint64_t npairs = (uint64_t)n * (n - 1) / 2;
        for (uint64_t P = 0; P < npairs; ++P) {
            int ii, jj;
            unrank_pair(P, ii, jj);
            int p = o[ii], q = o[jj];
            size_t row = (((size_t)(p >> 1)) * c->norb + (q >> 1)) * 2 + ((p & 1) == (q & 1) ? 1 : 0);
            uint32_t Q = c->ptab_cum[row * (size_t)c->norb + c->norb - 1];
            for (int A = 0; A < c->norb; ++A) {
                uint32_t qa = ptab_weight(*c, row, A);
                if (qa == 0) continue;
                /* the smallest word drawing x = cum[A] - qa, i.e. orbital A */
                uint64_t xlo = (uint64_t)c->ptab_cum[row * (size_t)c->norb + A] - qa;
                uint64_t w[4] = {0, 0, 0, 0};
                w[1] = (uint64_t)((((u128)P << 64) + npairs - 1) / npairs);
                w[2] = (uint64_t)((((u128)xlo << 64) + (uint64_t)Q - 1) / (uint64_t)Q);
                Excit e = generate(*c, d, w);
                add(e.null ? nullptr : &e.child, ((double)qa / (double)Q) / (double)npairs);
            }
        }
    } else if (c->kind == SYS_UEG) {
        uint64_t npairs = (uint64_t)n * (n - 1) / 2;
        for (uint64_t P = 0; P < npairs; ++P)
            for (int A = 0; A < c->norb; ++A) {
                uint64_t w[4] = {0, 0, 0, 0};
                w[1] = (uint64_t)((((u128)P << 64) + npairs - 1) / npairs);
                w[2] = (uint64_t)((((u128)(uint64_t)A << 64) + (uint64_t)c->norb - 1) / (uint64_t)c->norb);
                Excit e = generate(*c, d, w);
                add(e.null ? nullptr : &e.child, 1.0 / ((double)npairs * c->norb));
            }
    } else {
        for (int k = 0; k < n; ++k) {
            int i = o[k];
            int spin = i & 1;
            std::vector<int> empty;
            for (int A = 0; A < c->norb; ++A)
                if (!occ_bit(d, 2 * A + spin)) empty.push_back(2 * A + spin);
            for (size_t r = 0; r < empty.size(); ++r) {
                Det ch = d;
                flip_bit(ch, i); flip_bit(ch, empty[r]);
                add(&ch, c->p_single / ((double)n * (double)empty.size()));
            }
        }
        uint64_t npairs = (uint64_t)n * (n - 1) / 2;
        for (uint64_t P = 0; P < npairs; ++P) {
            int ii, jj;
            unrank_pair(P, ii, jj);
            int p = o[ii], q = o[jj];
            const std::vector<HBEntry>& tab = c->hb[pair_index(p, q)];
            if (tab.empty()) { add(nullptr, c->p_double / (double)npairs); continue; }
            uint64_t prev = 0;
            for (size_t k = 0; k < tab.size(); ++k) {
                double pk;
                if (tab.size() == 1) pk = 1.0;
                else if (k + 1 == tab.size()) pk = (double)(0 - prev) * 0x1p-64;
                else pk = (double)(tab[k].cum - prev) * 0x1p-64;
                prev = tab[k].cum;
                double pp = (c->p_double / (double)npairs) * pk;
                if (occ_bit(d, tab[k].a) || occ_bit(d, tab[k].b)) { add(nullptr, pp); continue; }
                Det ch = d;
                flip_bit(ch, p); flip_bit(ch, q); flip_bit(ch, tab[k].a); flip_bit(ch, tab[k].b);
                add(&ch, pp);
            }
        }
    }
    int64_t m = (int64_t)paths.size();
    if (m > cap) return -m;
    for (int64_t i = 0; i < m; ++i) {
        for (int k = 0; k < c->W; ++k) children[i * c->W + k] = paths[(size_t)i].first.w[k];
        probs[i] = paths[(size_t)i].second;
    }
    return m;
}

/* UEG basis vectors (3 ints per spatial orbital) and box length */
int orc_ueg_basis(void* h, int* kvec, double* box) {
    Ctx* c = (Ctx*)h;
    if (c->kind != SYS_UEG) return -1;
    for (int i = 0; i < 3 * c->norb; ++i) kvec[i] = c->kvec[(size_t)i];
    *box = c->box;
    return c->norb;
}

/* Proposal table of the UEG table generator: q[2 M^2][M] integer weights,
 * row r = (I M + J) 2 + same-spin.  A weight must be >= 1 exactly where the
 * particle orbital is drawable (ptab_valid) and 0 elsewhere, each <= 2^24.
 * Returns 0, or -1 for a system without the table generator or a bad table. */
int orc_set_proposal(void* h, const uint32_t* q) {
    Ctx* c = (Ctx*)h;
    if (c->kind != SYS_UEG || c->excit_gen != 1) return -1;
    for (int I = 0; I < c->norb; ++I)
        for (int J = 0; J < c->norb; ++J)
            for (int same = 0; same < 2; ++same)
                for (int A = 0; A < c->norb; ++A) {
                    uint32_t v = q[(((size_t)I * c->norb + J) * 2 + same) * c->norb + A];
                    bool ok = ptab_valid(*c, I, J, same, A);
                    if (ok ? (v < 1 || v > (1u << 24)) : v != 0) return -1;
                }
    set_ptab(*c, q);
    return 0;
}

/* drawable particle orbitals: mask[2 M^2][M] (1 = drawable) */
int orc_proposal_mask(void* h, uint8_t* mask) {
    Ctx* c = (Ctx*)h;
    if (c->kind != SYS_UEG) return -1;
    for (int I = 0; I < c->norb; ++I)
        for (int J = 0; J < c->norb; ++J)
            for (int same = 0; same < 2; ++same)
                for (int A = 0; A < c->norb; ++A)
                    mask[(((size_t)I * c->norb + J) * 2 + same) * c->norb + A] =
                        ptab_valid(*c, I, J, same, A) ? 1 : 0;
    return 0;
}

/* Restart (Sec. 3.1: a restarted calculation follows the same Markov chain).
 * With counter-based random numbers the generator state is the iteration
 * number; the rest is the shift, its latch and reference population, and the
 * deterministic space. */
void orc_get_state(void* h, int64_t* iter, double* shift, int64_t* nw_ref, int* vary, double* tau, double* rmax) {
    Ctx* c = (Ctx*)h;
    *iter = c->iter;
    *shift = c->shift;
    *nw_ref = c->nw_ref;
    *vary = c->vary;
    *tau = c->tau;
    *rmax = c->rmax;
}

/* after orc_set_walkers: restore the counters and the deterministic space
 * (ncore keys, all in the list; ncore = 0: none).  Returns 0, or -1 if a core
 * key is not in the list. */
int orc_set_state(void* h, int64_t iter, double shift, int64_t nw_ref, int vary, double tau, double rmax,
                  const uint64_t* core_keys, int64_t ncore) {
    Ctx* c = (Ctx*)h;
    c->tau = tau;
    c->rmax = rmax;
    std::vector<Det> keys;
    for (int64_t i = 0; i < ncore; ++i) {
        Det d;
        memset(&d, 0, sizeof d);
        for (int k = 0; k < c->W; ++k) d.w[k] = core_keys[i * c->W + k];
        keys.push_back(d);
    }
    c->iter = iter;
    c->shift = shift;
    c->nw_ref = nw_ref;
    c->vary = vary;
    c->recs.clear();
    if (ncore == 0) {
        c->core.clear();
        c->core_rows.clear();
        for (size_t i = 0; i < c->main.size(); ++i) c->main[i].core = 0;
        return 0;
    }
    install_core(*c, keys);
    int64_t found = 0;
    for (size_t i = 0; i < c->main.size(); ++i) found += c->main[i].core;
    return found == ncore ? 0 : -1;
}

/* The heat-bath table of the occupied pair (p < q): entries (a, b) in table
 * order with their cumulative thresholds.  Returns the entry count, -1 for a
 * system without tables or a bad pair, -count if cap is too small. */
int64_t orc_heat_bath(void* h, int p, int q, int* a, int* b, uint64_t* cum, int64_t cap) {
    Ctx* c = (Ctx*)h;
    if (c->kind != SYS_MOLECULE || p < 0 || q <= p || q >= c->nspin) return -1;
    const std::vector<HBEntry>& tab = c->hb[pair_index(p, q)];
    int64_t n = (int64_t)tab.size();
    if (n > cap) return -n;
    for (int64_t k = 0; k < n; ++k) {
        a[k] = tab[(size_t)k].a;
        b[k] = tab[(size_t)k].b;
        cum[k] = tab[(size_t)k].cum;
    }
    return n;
}

int64_t orc_core(void* h, uint64_t* keys, int64_t cap) {
    Ctx* c = (Ctx*)h;
    int64_t n = (int64_t)c->core.size();
    if (n > cap) return -n;
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < c->W; ++k) keys[i * c->W + k] = c->core[(size_t)i].w[k];
    return n;
}

}  /* extern "C" */
