"""Brute-force second quantisation on explicit occupation-number vectors.

Independent of the oracle's Slater-Condon rules: every matrix element is
obtained by applying creation/annihilation operators one at a time with the
Jordan-Wigner sign (-1)^(number of occupied spin orbitals below p), to the
Hamiltonian written as
    H = sum_pq h_pq a+_p a_q + 1/2 sum_pqrs <pq|rs> a+_p a+_q a_s a_r,
with <pq|rs> = (pr|qs) in chemist notation.  Spin orbital p = 2*spatial + spin.
"""
from __future__ import annotations

import itertools

import numpy as np


def _annihilate(bits: int, p: int):
    if not (bits >> p) & 1:
        return 0, 0
    sign = -1 if bin(bits & ((1 << p) - 1)).count("1") & 1 else 1
    return sign, bits ^ (1 << p)


def _create(bits: int, p: int):
    if (bits >> p) & 1:
        return 0, 0
    sign = -1 if bin(bits & ((1 << p) - 1)).count("1") & 1 else 1
    return sign, bits | (1 << p)


def determinants(norb: int, nalpha: int, nbeta: int):
    """All determinants (int bit strings) with the given spin populations, ascending."""
    out = []
    for a in itertools.combinations(range(norb), nalpha):
        for b in itertools.combinations(range(norb), nbeta):
            bits = 0
            for x in a:
                bits |= 1 << (2 * x)
            for x in b:
                bits |= 1 << (2 * x + 1)
            out.append(bits)
    return sorted(out)


def hamiltonian(dets, nspin, one_body, two_body):
    """Dense H in the basis `dets`.  one_body(p, q) -> h_pq over spin orbitals;
    two_body(p, q, r, s) -> <pq|rs> (physicist) over spin orbitals (only
    called with r, s occupied and p, q arbitrary)."""
    index = {d: i for i, d in enumerate(dets)}
    n = len(dets)
    H = np.zeros((n, n))
    for j, d in enumerate(dets):
        occ = [p for p in range(nspin) if (d >> p) & 1]
        for q in occ:
            s1, d1 = _annihilate(d, q)
            for p in range(nspin):
                v = one_body(p, q)
                if v == 0.0:
                    continue
                s2, d2 = _create(d1, p)
                if s2 == 0:
                    continue
                H[index[d2], j] += s1 * s2 * v
        for r in occ:
            for s in occ:
                if s == r:
                    continue
                s1, d1 = _annihilate(d, r)
                s2, d2 = _annihilate(d1, s)
                for q in range(nspin):
                    s3, d3 = _create(d2, q)
                    if s3 == 0:
                        continue
                    for p in range(nspin):
                        v = two_body(p, q, r, s)
                        if v == 0.0:
                            continue
                        s4, d4 = _create(d3, p)
                        if s4 == 0:
                            continue
                        H[index[d4], j] += 0.5 * s1 * s2 * s3 * s4 * v
    return H


def hubbard_hamiltonian(L, nalpha, nbeta, t, U, periodic):
    dets = determinants(L, nalpha, nbeta)
    nspin = 2 * L
    bonds = set()
    for s in range(L - 1):
        bonds.add((s, s + 1))
    if periodic and L > 2:
        bonds.add((0, L - 1))

    def one(p, q):
        if (p & 1) != (q & 1):
            return 0.0
        a, b = sorted((p >> 1, q >> 1))
        return -t if (a, b) in bonds else 0.0

    def two(p, q, r, s):
        # U n_up n_down on each site: <pq|rs> = U if p=r, q=s on one site with opposite spins
        if p == r and q == s and (p >> 1) == (q >> 1) and (p & 1) != (q & 1):
            return U
        return 0.0

    return dets, hamiltonian(dets, nspin, one, two)


def molecule_hamiltonian(h1, eri, nalpha, nbeta, ecore=0.0):
    norb = h1.shape[0]
    dets = determinants(norb, nalpha, nbeta)
    nspin = 2 * norb

    def one(p, q):
        return h1[p >> 1, q >> 1] if (p & 1) == (q & 1) else 0.0

    def two(p, q, r, s):
        # <pq|rs> = (pr|qs)
        if (p & 1) != (r & 1) or (q & 1) != (s & 1):
            return 0.0
        return eri[p >> 1, r >> 1, q >> 1, s >> 1]

    H = hamiltonian(dets, nspin, one, two)
    H += ecore * np.eye(len(dets))
    return dets, H


def ueg_basis(norb):
    """Plane-wave vectors n sorted by (|n|^2, nx, ny, nz), first norb."""
    R = 1
    while True:
        pts = [(x * x + y * y + z * z, x, y, z) for x in range(-R, R + 1) for y in range(-R, R + 1)
               for z in range(-R, R + 1) if x * x + y * y + z * z <= R * R]
        if len(pts) > norb:
            break
        R += 1
    pts.sort()
    return np.array([p[1:] for p in pts[:norb]], dtype=np.int64)


def ueg_hamiltonian(norb, nalpha, nbeta, rs):
    """Zero-temperature UEG in a plane-wave basis, Madelung term omitted:
    h_pq = delta_pq |k_p|^2 / 2;  <pq|rs> = delta(k_p + k_q = k_r + k_s)
    4 pi / (Omega |k_p - k_r|^2) for k_p != k_r (spin-conserving)."""
    nel = nalpha + nbeta
    kv = ueg_basis(norb)
    omega = (4.0 * np.pi / 3.0) * rs ** 3 * nel
    L = omega ** (1.0 / 3.0)
    kf = 2.0 * np.pi / L
    dets = determinants(norb, nalpha, nbeta)
    nspin = 2 * norb

    def one(p, q):
        if p != q:
            return 0.0
        n = kv[p >> 1]
        return 0.5 * kf * kf * float(n @ n)

    def two(p, q, r, s):
        if (p & 1) != (r & 1) or (q & 1) != (s & 1):
            return 0.0
        P, Q, Rr, S = p >> 1, q >> 1, r >> 1, s >> 1
        if not np.array_equal(kv[P] + kv[Q], kv[Rr] + kv[S]):
            return 0.0
        d = kv[P] - kv[Rr]
        m = float(d @ d)
        if m == 0.0:
            return 0.0
        return 4.0 * np.pi / (omega * kf * kf * m)

    return dets, hamiltonian(dets, nspin, one, two), kv, L


def bits_to_words(bits: int, W: int):
    return np.array([(bits >> (64 * k)) & ((1 << 64) - 1) for k in range(W)], dtype=np.uint64)


def words_to_bits(words) -> int:
    return sum(int(w) << (64 * k) for k, w in enumerate(words))
