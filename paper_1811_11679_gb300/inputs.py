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
  * molecule28   -- synthetic molecule, 28 spatial orbitals (56 spin orbitals,
                    64-bit keys), 15 electrons (8 up, 7 down), heat-bath
                    generator, initiator, real weights, semi-stochastic core,
                    1e7 walkers.
"""
from __future__ import annotations

import numpy as np


def molecule_integrals(norb: int, seed: int = 11):
    """Seeded one- and two-electron integrals with 8-fold symmetry.

    h_pq  : diagonal -2 + 0.15 p (Fock-like ordering), off-diagonal
            g exp(-|p-q|/4), g ~ U(-0.1, 0.1), symmetric.
    (pq|rs): Coulomb (pp|rr) = 0.5 exp(-|p-r|/8) + 0.05 u, u ~ U(0, 1) (> 0);
            exchange-like (pq|pq) = |g| exp(-|p-q|/2) (> 0);
            everything else g exp(-(|p-q| + |r-s|)/4), g ~ U(-0.1, 0.1).
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
                v = 0.5 * np.exp(-abs(p - r) / 8.0) + 0.05 * rng.uniform(0.0, 1.0)
            elif (p, q) == (r, s):
                v = abs(rng.uniform(-0.1, 0.1)) * np.exp(-abs(p - q) / 2.0)
            else:
                v = rng.uniform(-0.1, 0.1) * np.exp(-(abs(p - q) + abs(r - s)) / 4.0)
            for (a, b) in ((p, q), (q, p)):
                for (c, d) in ((r, s), (s, r)):
                    eri[a, b, c, d] = v
                    eri[c, d, a, b] = v
    return h1, eri


def hubbard_system(L=8, nalpha=4, nbeta=4, t=1.0, U=4.0, periodic=True):
    return {"kind": "hubbard", "key_words": 1 if 2 * L <= 64 else 2, "norb": L,
            "nalpha": nalpha, "nbeta": nbeta, "t": t, "U": U, "periodic": int(periodic)}


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
    # synthetic 28-orbital molecule, heat-bath, initiator, real weights, core 1e4
    "molecule28": (lambda: molecule_system(),
                   lambda: qmc_params(tau=0.01, target_population=1e7, initiator=1,
                                      real_amplitudes=1, spawn_cutoff=0.1,
                                      semi_stoch_size=10000, semi_stoch_start=2000, seed=8)),
}


def workload(name: str, **overrides):
    """(system, qmc) dicts for a named workload, qmc keys overridable."""
    sysf, qf = WORKLOADS[name]
    q = qf()
    q.update(overrides)
    return sysf(), q
