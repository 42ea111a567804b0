"""Seeded synthetic inputs shared by the GPU path, the tests and bench.py.

This module holds no FCIQMC arithmetic: it only states problem definitions
(system and run parameters) and draws the synthetic molecular integrals that
stand in for the integral files the paper reads (Sec. 3.1, FCIDUMP/HDF5; the
water, NO and diamond integrals are not available here).  Both the CPU oracle
and the CUDA library receive these values as plain inputs.

Workloads (sizes as in the HANDE-QMC paper's tutorial and examples):
  * hubbard8     -- 1D real-space Hubbard ring, 8 sites, 4 up + 4 down, t=1, U=4,
                    integer walkers, tau=0.01, target 1e4, 2000 iterations.
  * ueg14        -- uniform electron gas, 14 electrons, 38 plane-wave spatial
                    orbitals (76 spin orbitals, 128-bit keys), r_s = 1,
                    initiator real-weight FCIQMC, tau=0.002.
  * hubbard18_2d -- 2D Hubbard model, tilted 18-site square cluster (lattice
                    vectors (3, 3), (3, -3)), 9 up + 9 down, U/t = 1.3,
                    initiator real-weight FCIQMC, deterministic space 1e4.
  * molecule28   -- synthetic molecule, 28 spatial orbitals (56 spin orbitals,
                    64-bit keys), 15 electrons (8 up, 7 down), heat-bath
                    generator, initiator, real weights, semi-stochastic core,
                    1e7 walkers.
"""
from __future__ import annotations

import numpy as np


def molecule_integrals(norb: int, seed: int = 11):
    """Seeded one- and two-electron integrals with 8-fold symmetry.

    Orbitals behave like localised functions on a line: products p*q decay
    with |p-q| and interactions between products with their separation.
    h_pq  : diagonal -2 + 0.15 p (Fock-like ordering), off-diagonal
            g exp(-|p-q|/4), g ~ U(-0.1, 0.1), symmetric.
    (pq|rs): Coulomb (pp|rr) = 0.25 exp(-|p-r|/8) + 0.05 u, u ~ U(0, 1) (> 0);
            exchange-like (pq|pq) = |g| exp(-|p-q|/2), g ~ U(-0.1, 0.1) (> 0);
            everything else g exp(-(|p-q| + |r-s|)/2 - |p+q-r-s|/4),
            g ~ U(-0.05, 0.05).
    Returns (h1[norb, norb], eri[norb, norb, norb, norb]) in chemist order.
    """
    rng = np.random.Generator(np.random.Philox(seed))
    n = norb
    h1 = np.zeros((n, n))
    for p in range(n):
        h1[p, p] = -2.0 + 0.15 * p
        for q in range(p):
            g = rng.uniform(-0.1, 0.1)
            h1[p, q] = h1[q, p] = g * np.exp(-abs(p - q) / 4.0)
    eri = np.zeros((n, n, n, n))
    pairs = [(p, q) for p in range(n) for q in range(p + 1)]
    for ia, (p, q) in enumerate(pairs):
        for (r, s) in pairs[: ia + 1]:
            if p == q and r == s:
                v = 0.25 * np.exp(-abs(p - r) / 8.0) + 0.05 * rng.uniform(0.0, 1.0)
            elif (p, q) == (r, s):
                v = abs(rng.uniform(-0.1, 0.1)) * np.exp(-abs(p - q) / 2.0)
            else:
                v = rng.uniform(-0.05, 0.05) * np.exp(-(abs(p - q) + abs(r - s)) / 2.0
                                                      - abs(p + q - r - s) / 4.0)
            for (a, b) in ((p, q), (q, p)):
                for (c, d) in ((r, s), (s, r)):
                    eri[a, b, c, d] = v
                    eri[c, d, a, b] = v
    return h1, eri


def hubbard_system(L=8, nalpha=4, nbeta=4, t=1.0, U=4.0, periodic=True):
    return {"kind": "hubbard", "key_words": 1 if 2 * L <= 64 else 2, "norb": L,
            "nalpha": nalpha, "nbeta": nbeta, "t": t, "U": U, "periodic": int(periodic)}


def hubbard_lattice_system(lattice, nalpha, nbeta, t=1.0, U=4.0):
    """Real-space Hubbard model on the periodic lattice spanned by the integer
    rows of `lattice` (the paper's `lattice` input); |det| sites."""
    lat = np.asarray(lattice, dtype=np.int64)
    L = int(round(abs(np.linalg.det(lat.astype(np.float64)))))
    return {"kind": "hubbard", "key_words": 1 if 2 * L <= 64 else (2 if 2 * L <= 128 else 8), "norb": L,
            "nalpha": nalpha, "nbeta": nbeta, "t": t, "U": U, "periodic": 1, "lattice": lat.tolist()}


def ueg_system(nel=14, norb=38, rs=1.0, key_words=None):
    nspin = 2 * norb
    if key_words is None:
        key_words = 1 if nspin <= 64 else (2 if nspin <= 128 else 8)
    return {"kind": "ueg", "key_words": key_words, "norb": norb, "nalpha": nel // 2,
            "nbeta": nel - nel // 2, "rs": rs}


def molecule_system(norb=28, nalpha=8, nbeta=7, seed=11, key_words=1):
    h1, eri = molecule_integrals(norb, seed)
    return {"kind": "molecule", "key_words": key_words, "norb": norb, "nalpha": nalpha,
            "nbeta": nbeta, "h1": h1, "eri": eri, "ecore": 0.0}


def qmc_params(**kw):
    """Run parameters; defaults follow the paper's tutorial input (Sec. S1:
    tau 0.01, rng_seed 8, init_pop 500, target 1e4, spawn_cutoff 0.1)."""
    q = {"tau": 0.01, "target_population": 1e4, "shift_damping": 0.05, "spawn_cutoff": 0.1,
         "init_pop": 500.0, "initiator_threshold": 3.0, "p_single": 0.1, "shift_period": 1,
         "initiator": 0, "real_amplitudes": 0, "semi_stoch_size": 0, "semi_stoch_start": 0,
         "seed": 8, "replica": 0}
    q.update(kw)
    return q


WORKLOADS = {
    # 1D Hubbard ring, integer walkers, no initiator (checked against dense ED)
    "hubbard8": (lambda: hubbard_system(),
                 lambda: qmc_params(tau=0.01, target_population=1e4, seed=8)),
    # UEG 14e / 38 spatial orbitals, initiator real-weight FCIQMC
    "ueg14": (lambda: ueg_system(14, 38, 1.0),
              lambda: qmc_params(tau=0.002, target_population=1e6, initiator=1,
                                 real_amplitudes=1, spawn_cutoff=0.1, seed=7)),
    # half-filled 2D Hubbard model on the tilted 18-site square cluster, U/t = 1.3,
    # semi-stochastic with a 1e4 deterministic space (the paper's Fig. semistoch b)
    "hubbard18_2d": (lambda: hubbard_lattice_system([[3, 3], [3, -3]], 9, 9, t=1.0, U=1.3),
                     lambda: qmc_params(tau=0.002, target_population=1e6, initiator=1, real_amplitudes=1,
                                        spawn_cutoff=0.01, init_pop=100, semi_stoch_size=10000,
                                        semi_stoch_start=500, seed=8, state_capacity=12_000_000,
                                        spawn_capacity=24_000_000)),
    # synthetic 28-orbital molecule, heat-bath, initiator, real weights, core 1e4
    "molecule28": (lambda: molecule_system(),
                   lambda: qmc_params(tau=0.01, target_population=1e7, initiator=1,
                                      real_amplitudes=1, spawn_cutoff=0.1,
                                      semi_stoch_size=10000, semi_stoch_start=2000, seed=8)),
}


def batched_replicas(n: int = 256, seed: int = 13, lo: float = 1e4, hi: float = 1e6):
    """(systems, qmcs) of n independent replicas: UEG 14 electrons in 38 or 66
    spatial orbitals (128- or 512-bit keys), r_s in {0.5, 1, 2, 5}, 32 seeds per
    (basis, r_s) pair for n = 256, cycled for other n; initiator real-weight
    FCIQMC at tau = 0.002; target populations log-uniform in [lo, hi] (default
    [1e4, 1e6]) drawn from numpy's Philox generator with the given seed.  Each
    replica starts with half its target on the reference determinant, so the
    population reaches the target within a few hundred iterations."""
    rng = np.random.Generator(np.random.Philox(seed))
    targets = np.exp(rng.uniform(np.log(lo), np.log(hi), n))
    systems, qmcs = [], []
    for r in range(n):
        norb = (38, 66)[r % 2]
        rs = (0.5, 1.0, 2.0, 5.0)[(r // 2) % 4]
        tgt = float(targets[r])
        systems.append(ueg_system(14, norb, rs))
        qmcs.append(qmc_params(tau=0.002, target_population=tgt, initiator=1, real_amplitudes=1,
                               spawn_cutoff=0.1, init_pop=0.5 * tgt, seed=100 + r // 8, replica=r,
                               state_capacity=int(1.5 * tgt) + (1 << 16),
                               spawn_capacity=int(3 * tgt) + (1 << 17)))
    return systems, qmcs


def workload(name: str, **overrides):
    """(system, qmc) dicts for a named workload, qmc keys overridable."""
    sysf, qf = WORKLOADS[name]
    q = qf()
    q.update(overrides)
    return sysf(), q


def reference_key(system: dict) -> np.ndarray:
    """Reference determinant as key words: Neel (alpha on even sites, beta on odd
    sites) for the real-space Hubbard model, aufbau otherwise."""
    W = int(system["key_words"])
    bits = 0
    na, nb = int(system["nalpha"]), int(system["nbeta"])
    if system["kind"] == "hubbard":
        for k in range(na):
            bits |= 1 << (2 * (2 * k))
        for k in range(nb):
            bits |= 1 << (2 * (2 * k + 1) + 1)
    else:
        for k in range(na):
            bits |= 1 << (2 * k)
        for k in range(nb):
            bits |= 1 << (2 * k + 1)
    return np.array([(bits >> (64 * j)) & ((1 << 64) - 1) for j in range(W)], dtype=np.uint64)


def _choose(rng, m: int, pool: np.ndarray, k: int) -> np.ndarray:
    """k distinct entries of `pool` per row (m rows), uniformly at random."""
    if k == 0:
        return np.zeros((m, 0), dtype=np.int64)
    r = rng.random((m, len(pool)), dtype=np.float32)
    if k >= len(pool):
        return np.broadcast_to(pool, (m, len(pool))).copy()
    return pool[np.argpartition(r, k - 1, axis=1)[:, :k]]


def synthetic_walkers(system: dict, n_det: int, n_walkers: float, seed: int = 21,
                      ref_fraction: float = 0.1, levels=(0.05, 0.45, 0.3, 0.2)):
    """A seeded walker list with the shape of a converged large run: the reference
    holds `ref_fraction` of the walkers; the other n_det - 1 determinants are
    random spin-conserving 1-4-fold excitations of it (level probabilities
    `levels`), with heavy-tailed (Pareto, shape 1.2) populations of at least one
    walker and random signs.  Returns (keys[n, W] ascending, pops int64 fixed point).
    Only random numbers and bit patterns: no Hamiltonian is evaluated."""
    W = int(system["key_words"])
    nspin = 2 * int(system["norb"])
    rng = np.random.Generator(np.random.Philox(seed))
    d0 = reference_key(system)
    bit = lambda p: (int(d0[p // 64]) >> (p % 64)) & 1
    occ = [np.array([p for p in range(s, nspin, 2) if bit(p)], dtype=np.int64) for s in (0, 1)]
    vir = [np.array([p for p in range(s, nspin, 2) if not bit(p)], dtype=np.int64) for s in (0, 1)]
    cap = [min(len(occ[s]), len(vir[s])) for s in (0, 1)]
    lv = np.asarray(levels, dtype=np.float64)
    lv = lv / lv.sum()
    want = n_det - 1
    found = np.zeros((0, W), dtype=np.uint64)
    while len(found) < want:
        m = int(min(2_000_000, (want - len(found)) * 1.3 + 1000))
        level = rng.choice(np.arange(1, len(lv) + 1), size=m, p=lv)
        lo = np.maximum(0, level - cap[1])
        hi = np.minimum(level, cap[0])
        ok = hi >= lo
        na = lo + np.floor(rng.random(m) * (hi - lo + 1)).astype(np.int64)
        nb = level - na
        keys = np.tile(d0, (m, 1))
        for a in range(cap[0] + 1):
            for b in range(cap[1] + 1):
                rows = np.nonzero(ok & (na == a) & (nb == b))[0]
                if len(rows) == 0:
                    continue
                flips = [_choose(rng, len(rows), occ[0], a), _choose(rng, len(rows), vir[0], a),
                         _choose(rng, len(rows), occ[1], b), _choose(rng, len(rows), vir[1], b)]
                pos = np.concatenate(flips, axis=1)
                sub = keys[rows]
                for c in range(pos.shape[1]):
                    word = pos[:, c] // 64
                    mask = np.left_shift(np.uint64(1), (pos[:, c] % 64).astype(np.uint64))
                    for j in range(W):
                        sub[:, j] ^= np.where(word == j, mask, np.uint64(0))
                keys[rows] = sub
        keys = np.concatenate([found, keys[ok]])
        order = np.lexsort([keys[:, j] for j in range(W)])
        keys = keys[order]
        fresh = np.ones(len(keys), dtype=bool)
        fresh[1:] = np.any(keys[1:] != keys[:-1], axis=1)
        found = keys[fresh]
        found = found[~np.all(found == d0[None, :], axis=1)]
    pick = np.sort(rng.choice(len(found), size=want, replace=False))
    allk = np.concatenate([found[pick], d0[None, :]])
    allk = allk[np.lexsort([allk[:, j] for j in range(W)])]   # last key = most significant word
    F = float(1 << 32)
    is0 = np.all(allk == d0[None, :], axis=1)
    extra = rng.pareto(1.2, size=len(allk))
    extra[is0] = 0.0
    spare = max((1.0 - ref_fraction) * n_walkers - (len(allk) - 1), 0.0)
    mag = 1.0 + extra * (spare / extra.sum())
    pops = np.rint(mag * F).astype(np.int64)
    pops *= rng.choice(np.array([-1, 1], dtype=np.int64), size=len(pops))
    pops[is0] = int(round(ref_fraction * n_walkers * F))
    return allk, pops


def random_proposal(mask, seed: int = 17) -> np.ndarray:
    """Seeded integer weights in [1, 2^24] on the drawable entries of a UEG
    proposal-table mask (bool[2 M^2, M]), 0 elsewhere."""
    rng = np.random.Generator(np.random.Philox(seed))
    q = rng.integers(1, 1 << 24, size=mask.shape, endpoint=True).astype(np.uint32)
    return np.where(mask, q, 0).astype(np.uint32)
