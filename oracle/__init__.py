"""CPU FCIQMC oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded C++ implementation of one FCIQMC iteration
(HANDE-QMC paper, Sec. 2.1 Eq. (fciqmc), Sec. 2.4, App. A.1, App. A.2, App. B),
loaded through ctypes.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of bench.py may import this
package.  It shares no code with the GPU path (``paper_1811_11679_gb300``),
and neither imports the other.

Everything it needs is passed in as plain numbers and numpy arrays; seeded
synthetic inputs come from ``paper_1811_11679_gb300.inputs``, a module that
holds no FCIQMC arithmetic.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fciqmc_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}

SYS_HUBBARD, SYS_UEG, SYS_MOLECULE = 0, 1, 2


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile liboracle.so (g++, -O2, FMA contraction off) if it is stale; with
    openmp=True the same source as liboracle_omp.so (-fopenmp), whose
    orc_iterate_parallel runs the hash-partitioned form of the iteration."""
    os.makedirs(_BUILD, exist_ok=True)
    lib = _LIB_OMP if openmp else _LIB
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(_SRC)):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


class _System(C.Structure):
    _fields_ = [("kind", C.c_int), ("key_words", C.c_int), ("norb", C.c_int),
                ("nalpha", C.c_int), ("nbeta", C.c_int), ("periodic", C.c_int),
                ("t", C.c_double), ("U", C.c_double), ("rs", C.c_double),
                ("h1", C.POINTER(C.c_double)), ("eri", C.POINTER(C.c_double)),
                ("ecore", C.c_double), ("ndim", C.c_int), ("lattice", C.c_int * 9)]


class _Qmc(C.Structure):
    _fields_ = [("tau", C.c_double), ("target_population", C.c_double),
                ("shift_damping", C.c_double), ("spawn_cutoff", C.c_double),
                ("init_pop", C.c_double), ("initiator_threshold", C.c_double),
                ("p_single", C.c_double),
                ("shift_period", C.c_int), ("initiator", C.c_int),
                ("real_amplitudes", C.c_int), ("semi_stoch_size", C.c_int),
                ("semi_stoch_start", C.c_int),
                ("seed", C.c_uint64), ("replica", C.c_uint64), ("excit_gen", C.c_int), ("tau_search", C.c_int)]


def _load(openmp: bool = False):
    with _lock:
        if openmp in _libs:
            return _libs[openmp]
        lib = C.CDLL(build(openmp=openmp))
        P = C.c_void_p
        u64p, i64p, dp = C.POINTER(C.c_uint64), C.POINTER(C.c_int64), C.POINTER(C.c_double)
        lib.orc_philox.argtypes = [u64p, u64p, u64p]
        lib.orc_log.argtypes = [C.c_double]
        lib.orc_log.restype = C.c_double
        lib.orc_fixed_term.argtypes = [C.c_int64, C.c_double, i64p, u64p]
        lib.orc_fixed_product.argtypes = [C.c_double, C.c_double, C.c_int]
        lib.orc_fixed_product.restype = C.c_uint64
        lib.orc_create.argtypes = [C.POINTER(_System), C.POINTER(_Qmc)]
        lib.orc_create.restype = P
        lib.orc_destroy.argtypes = [P]
        lib.orc_iterate.argtypes = [P, C.c_int]
        lib.orc_nrec.argtypes = [P]
        lib.orc_nrec.restype = C.c_int64
        lib.orc_ndet.argtypes = [P]
        lib.orc_ndet.restype = C.c_int64
        lib.orc_eref.argtypes = [P]
        lib.orc_eref.restype = C.c_double
        lib.orc_shift.argtypes = [P]
        lib.orc_shift.restype = C.c_double
        lib.orc_get_walkers.argtypes = [P, u64p, i64p, dp, C.POINTER(C.c_uint8), C.c_int64]
        lib.orc_get_walkers.restype = C.c_int64
        lib.orc_set_walkers.argtypes = [P, u64p, i64p, C.c_int64]
        lib.orc_set_walkers.restype = C.c_int
        lib.orc_records.argtypes = [P, i64p, dp, i64p, i64p, dp, i64p, u64p, i64p, i64p, i64p,
                                    i64p, dp, C.c_int64]
        lib.orc_records.restype = C.c_int64
        lib.orc_reference.argtypes = [P, u64p]
        lib.orc_hdiag.argtypes = [P, u64p]
        lib.orc_hdiag.restype = C.c_double
        lib.orc_hij.argtypes = [P, u64p, u64p]
        lib.orc_hij.restype = C.c_double
        lib.orc_generate.argtypes = [P, u64p, u64p, u64p, dp, dp, dp]
        lib.orc_generate.restype = C.c_int
        lib.orc_enumerate.argtypes = [P, u64p, u64p, dp, C.c_int64]
        lib.orc_enumerate.restype = C.c_int64
        lib.orc_ueg_basis.argtypes = [P, C.POINTER(C.c_int), dp]
        lib.orc_ueg_basis.restype = C.c_int
        lib.orc_core.argtypes = [P, u64p, C.c_int64]
        lib.orc_core.restype = C.c_int64
        lib.orc_set_proposal.argtypes = [P, C.POINTER(C.c_uint32)]
        lib.orc_set_proposal.restype = C.c_int
        lib.orc_proposal_mask.argtypes = [P, C.POINTER(C.c_uint8)]
        lib.orc_proposal_mask.restype = C.c_int
        lib.orc_get_state.argtypes = [P, i64p, dp, i64p, C.POINTER(C.c_int), dp, dp]
        lib.orc_get_state.restype = None
        lib.orc_set_state.argtypes = [P, C.c_int64, C.c_double, C.c_int64, C.c_int, C.c_double, C.c_double, u64p,
                                      C.c_int64]
        lib.orc_set_state.restype = C.c_int
        lib.orc_heat_bath.argtypes = [P, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), u64p,
                                      C.c_int64]
        lib.orc_heat_bath.restype = C.c_int64
        lib.orc_iterate_parallel.argtypes = [P, C.c_int, C.c_int]
        lib.orc_iterate_parallel.restype = C.c_int
        _libs[openmp] = lib
        return lib


def _u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.ctypes.data_as(C.POINTER(C.c_uint64))


def philox(ctr, key):
    """Philox4x64-10 block for counter (4 words) and key (2 words)."""
    lib = _load()
    c, cp = _u64(ctr)
    k, kp = _u64(key)
    out = np.zeros(4, dtype=np.uint64)
    lib.orc_philox(cp, kp, out.ctypes.data_as(C.POINTER(C.c_uint64)))
    return out


def log(x: float) -> float:
    """The oracle's own natural logarithm (atanh series)."""
    return _load().orc_log(float(x))


def fixed_term(n: int, h: float) -> int:
    """round_half_even(n h 2^16) of the exact product, as a Python int (the 128-bit term)."""
    hi, lo = C.c_int64(), C.c_uint64()
    _load().orc_fixed_term(int(n), float(h), C.byref(hi), C.byref(lo))
    return (hi.value << 64) | lo.value


def fixed_product(a: float, b: float, round_half: bool) -> int:
    """floor(a b 2^32) (or floor(a b 2^32 + 1/2)) of the exact product, saturated at 2^62."""
    return int(_load().orc_fixed_product(float(a), float(b), 1 if round_half else 0))


class Oracle:
    """One FCIQMC run on the CPU.  ``system``/``qmc`` are plain dicts (see
    paper_1811_11679_gb300.inputs for the keys).  With ``threads`` the run uses
    the OpenMP build and iterates in the hash-partitioned form on that many
    threads (0 = all cores); the results are the serial ones bit for bit."""

    def __init__(self, system: dict, qmc: dict, threads: int | None = None):
        self.threads = threads
        lib = _load(openmp=threads is not None)
        self._lib = lib
        s = _System()
        kind = {"hubbard": SYS_HUBBARD, "ueg": SYS_UEG, "molecule": SYS_MOLECULE}[system["kind"]]
        s.kind = kind
        s.key_words = int(system["key_words"])
        s.norb = int(system["norb"])
        s.nalpha = int(system["nalpha"])
        s.nbeta = int(system["nbeta"])
        s.periodic = int(system.get("periodic", 0))
        s.t = float(system.get("t", 0.0))
        s.U = float(system.get("U", 0.0))
        s.rs = float(system.get("rs", 0.0))
        s.ecore = float(system.get("ecore", 0.0))
        lat = system.get("lattice")
        if lat is not None:
            lat = np.asarray(lat, dtype=np.int64)
            s.ndim = lat.shape[0]
            for i in range(s.ndim):
                for j in range(s.ndim):
                    s.lattice[3 * i + j] = int(lat[i, j])
        self._keep = []
        if kind == SYS_MOLECULE:
            h1 = np.ascontiguousarray(system["h1"], dtype=np.float64)
            eri = np.ascontiguousarray(system["eri"], dtype=np.float64)
            self._keep += [h1, eri]
            s.h1 = h1.ctypes.data_as(C.POINTER(C.c_double))
            s.eri = eri.ctypes.data_as(C.POINTER(C.c_double))
        q = _Qmc()
        q.tau = float(qmc["tau"])
        q.target_population = float(qmc["target_population"])
        q.shift_damping = float(qmc.get("shift_damping", 0.05))
        q.spawn_cutoff = float(qmc.get("spawn_cutoff", 0.0))
        q.init_pop = float(qmc["init_pop"])
        q.initiator_threshold = float(qmc.get("initiator_threshold", 3.0))
        q.p_single = float(qmc.get("p_single", 0.1))
        q.shift_period = int(qmc.get("shift_period", 1))
        q.initiator = int(qmc.get("initiator", 0))
        q.real_amplitudes = int(qmc.get("real_amplitudes", 0))
        q.semi_stoch_size = int(qmc.get("semi_stoch_size", 0))
        q.semi_stoch_start = int(qmc.get("semi_stoch_start", 0))
        q.seed = int(qmc["seed"])
        q.replica = int(qmc.get("replica", 0))
        q.excit_gen = int(qmc.get("excit_gen", 0))
        q.tau_search = int(qmc.get("tau_search", 0))
        h = lib.orc_create(C.byref(s), C.byref(q))
        if not h:
            raise ValueError("oracle rejected the system/qmc parameters")
        self._h = h
        self.W = s.key_words
        self._norb = s.norb

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    def iterate(self, n: int = 1) -> None:
        if self.threads is None:
            self._lib.orc_iterate(self._h, int(n))
        elif self._lib.orc_iterate_parallel(self._h, int(n), int(self.threads)) != 0:
            raise RuntimeError("the oracle was built without OpenMP")

    @property
    def e_ref(self) -> float:
        return self._lib.orc_eref(self._h)

    @property
    def shift(self) -> float:
        return self._lib.orc_shift(self._h)

    def reference(self) -> np.ndarray:
        k = np.zeros(self.W, dtype=np.uint64)
        self._lib.orc_reference(self._h, k.ctypes.data_as(C.POINTER(C.c_uint64)))
        return k

    def walkers(self):
        """(keys[n, W] uint64, pops int64, hdiag f64, flags u8) sorted by key."""
        n = self._lib.orc_ndet(self._h)
        keys = np.zeros((n, self.W), dtype=np.uint64)
        pops = np.zeros(n, dtype=np.int64)
        hd = np.zeros(n, dtype=np.float64)
        fl = np.zeros(n, dtype=np.uint8)
        got = self._lib.orc_get_walkers(self._h, keys.ctypes.data_as(C.POINTER(C.c_uint64)),
                                        pops.ctypes.data_as(C.POINTER(C.c_int64)),
                                        hd.ctypes.data_as(C.POINTER(C.c_double)),
                                        fl.ctypes.data_as(C.POINTER(C.c_uint8)), n)
        assert got == n
        return keys, pops, hd, fl

    def set_walkers(self, keys, pops) -> None:
        k, kp = _u64(np.asarray(keys).reshape(-1, self.W))
        p = np.ascontiguousarray(pops, dtype=np.int64)
        rc = self._lib.orc_set_walkers(self._h, kp, p.ctypes.data_as(C.POINTER(C.c_int64)), len(p))
        if rc == -2:
            raise ValueError("the list lacks a determinant of the deterministic space")
        if rc != 0:
            raise ValueError("walker keys must be strictly ascending")

    def records(self) -> dict:
        cols = {}
        names = ["iter", "shift", "nw_pre", "n0", "num", "num_hi", "num_lo", "nw_post", "ndet",
                 "natt", "nspawn", "tau"]
        types = [np.int64, np.float64, np.int64, np.int64, np.float64, np.int64, np.uint64,
                 np.int64, np.int64, np.int64, np.int64, np.float64]
        n = max(1, self._lib.orc_nrec(self._h))
        arrs = [np.zeros(n, dtype=t) for t in types]
        ptrs = []
        for a, t in zip(arrs, types):
            ct = {np.int64: C.c_int64, np.float64: C.c_double, np.uint64: C.c_uint64}[t]
            ptrs.append(a.ctypes.data_as(C.POINTER(ct)))
        got = self._lib.orc_records(self._h, *ptrs, n)
        for name, a in zip(names, arrs):
            cols[name] = a[:got].copy()
        return cols

    def hdiag(self, key) -> float:
        k, kp = _u64(np.asarray(key).reshape(self.W))
        return self._lib.orc_hdiag(self._h, kp)

    def hij(self, source, target) -> float:
        s, sp = _u64(np.asarray(source).reshape(self.W))
        t, tp = _u64(np.asarray(target).reshape(self.W))
        return self._lib.orc_hij(self._h, sp, tp)

    def generate(self, key, words):
        k, kp = _u64(np.asarray(key).reshape(self.W))
        w, wp = _u64(np.asarray(words).reshape(4))
        child = np.zeros(self.W, dtype=np.uint64)
        pg, hv = C.c_double(), C.c_double()
        inv = np.zeros(2, dtype=np.float64)
        ok = self._lib.orc_generate(self._h, kp, wp, child.ctypes.data_as(C.POINTER(C.c_uint64)),
                                    C.byref(pg), C.byref(hv), inv.ctypes.data_as(C.POINTER(C.c_double)))
        if not ok:
            return None
        self.last_inv = (float(inv[0]), float(inv[1]))
        return child, pg.value, hv.value

    def enumerate(self, key):
        """All generator selection paths from `key`: (children[m, W], probs[m]);
        an all-zero child marks a null path."""
        k, kp = _u64(np.asarray(key).reshape(self.W))
        cap = 1 << 22
        ch = np.zeros((cap, self.W), dtype=np.uint64)
        pr = np.zeros(cap, dtype=np.float64)
        m = self._lib.orc_enumerate(self._h, kp, ch.ctypes.data_as(C.POINTER(C.c_uint64)),
                                    pr.ctypes.data_as(C.POINTER(C.c_double)), cap)
        assert m >= 0
        return ch[:m].copy(), pr[:m].copy()

    def ueg_basis(self):
        kv = np.zeros(3 * 4096, dtype=np.int32)
        box = C.c_double()
        n = self._lib.orc_ueg_basis(self._h, kv.ctypes.data_as(C.POINTER(C.c_int)), C.byref(box))
        return kv[:3 * n].reshape(n, 3).copy(), box.value

    def core(self) -> np.ndarray:
        cap = 1 << 20
        k = np.zeros((cap, self.W), dtype=np.uint64)
        n = self._lib.orc_core(self._h, k.ctypes.data_as(C.POINTER(C.c_uint64)), cap)
        return k[:n].copy()

    def heat_bath_table(self, p: int, q: int):
        """The heat-bath table of the occupied spin-orbital pair p < q:
        (a[m], b[m], cum[m]) in table order (cumulative 64-bit thresholds)."""
        cap = 1 << 16
        a = np.zeros(cap, dtype=np.int32)
        b = np.zeros(cap, dtype=np.int32)
        cum = np.zeros(cap, dtype=np.uint64)
        m = self._lib.orc_heat_bath(self._h, int(p), int(q), a.ctypes.data_as(C.POINTER(C.c_int)),
                                    b.ctypes.data_as(C.POINTER(C.c_int)),
                                    cum.ctypes.data_as(C.POINTER(C.c_uint64)), cap)
        if m < 0:
            raise ValueError("no heat-bath table for this system or pair")
        return a[:m].copy(), b[:m].copy(), cum[:m].copy()

    def state(self):
        """Restart snapshot beyond the walker list: (dict with iter, shift,
        nw_ref, vary, core_active, ncore; deterministic-space keys[ncore, W])."""
        it, sh, nw, va = C.c_int64(), C.c_double(), C.c_int64(), C.c_int()
        tau, rmax = C.c_double(), C.c_double()
        self._lib.orc_get_state(self._h, C.byref(it), C.byref(sh), C.byref(nw), C.byref(va), C.byref(tau),
                                C.byref(rmax))
        core = self.core()
        return ({"iter": it.value, "shift": sh.value, "nw_ref": nw.value, "vary": va.value,
                 "core_active": int(len(core) > 0), "ncore": len(core), "tau": tau.value,
                 "rmax": rmax.value}, core)

    def set_state(self, state: dict, core_keys=None) -> None:
        """Restore a snapshot (after set_walkers of its list)."""
        n = int(state["ncore"]) if state.get("core_active") else 0
        k, kp = _u64(np.zeros((1, self.W)) if n == 0 else np.asarray(core_keys).reshape(-1, self.W))
        rc = self._lib.orc_set_state(self._h, int(state["iter"]), float(state["shift"]), int(state["nw_ref"]),
                                     int(state["vary"]), float(state["tau"]), float(state["rmax"]), kp, n)
        if rc != 0:
            raise ValueError("a deterministic-space key is not in the walker list")

    def proposal_mask(self) -> np.ndarray:
        """UEG: drawable particle orbitals of the proposal table, bool[2 M^2, M]
        (row r = (I M + J) 2 + same-spin)."""
        M = int(self._norb)
        m = np.zeros((2 * M * M, M), dtype=np.uint8)
        if self._lib.orc_proposal_mask(self._h, m.ctypes.data_as(C.POINTER(C.c_uint8))) != 0:
            raise ValueError("no proposal table for this system")
        return m.astype(bool)

    def set_proposal(self, q) -> None:
        """Install the integer weights q[2 M^2, M] of the proposal-table generator."""
        a = np.ascontiguousarray(q, dtype=np.uint32)
        if self._lib.orc_set_proposal(self._h, a.ctypes.data_as(C.POINTER(C.c_uint32))) != 0:
            raise ValueError("proposal table rejected (weights >= 1 exactly where drawable, <= 2^24)")
