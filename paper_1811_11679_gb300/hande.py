"""Python binding of libhande.so (include/hande.h), argument marshalling only.

Every step of an FCIQMC iteration runs in the library's CUDA kernels; this
module converts dicts and numpy arrays to the C structs, passes PyTorch's
current CUDA stream and routes the library's device allocations through
PyTorch's caching allocator.  There is no CPU fallback: if the shared library
is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

ONE_WALKER = 1 << 32
_KIND = {"hubbard": 0, "ueg": 1, "molecule": 2}

STATUS = {0: "HANDE_OK", -1: "HANDE_ERR_INVALID", -2: "HANDE_ERR_NOMEM", -3: "HANDE_ERR_CAPACITY",
          -4: "HANDE_ERR_OVERFLOW", -5: "HANDE_ERR_CUDA", -6: "HANDE_ERR_TIMEOUT", -7: "HANDE_ERR_STATE"}


def _pinned_array(shape, dtype):
    """A numpy array over page-locked host memory (allocated through PyTorch)."""
    import torch
    dt = np.dtype(dtype)
    count = int(np.prod(shape))
    buf = torch.empty(max(count * dt.itemsize, 1), dtype=torch.uint8, pin_memory=True)
    arr = buf.numpy()[:count * dt.itemsize].view(dt).reshape(shape)
    return arr


class HandeError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class _System(C.Structure):
    _fields_ = [("kind", C.c_int), ("key_words", C.c_int), ("norb", C.c_int), ("nalpha", C.c_int),
                ("nbeta", C.c_int), ("periodic", C.c_int), ("t", C.c_double), ("U", C.c_double),
                ("rs", C.c_double), ("h1", C.POINTER(C.c_double)), ("eri", C.POINTER(C.c_double)),
                ("ecore", C.c_double), ("ndim", C.c_int), ("lattice", C.c_int * 9)]


class _Qmc(C.Structure):
    _fields_ = [("tau", C.c_double), ("target_population", C.c_double), ("shift_damping", C.c_double),
                ("spawn_cutoff", C.c_double), ("init_pop", C.c_double), ("initiator_threshold", C.c_double),
                ("p_single", C.c_double), ("shift_period", C.c_int), ("initiator", C.c_int),
                ("real_amplitudes", C.c_int), ("semi_stoch_size", C.c_int), ("semi_stoch_start", C.c_int),
                ("seed", C.c_uint64), ("replica", C.c_uint64), ("state_capacity", C.c_int64),
                ("spawn_capacity", C.c_int64), ("record_capacity", C.c_int), ("tile_capacity", C.c_int),
                ("annihilation", C.c_int), ("excit_gen", C.c_int), ("tau_search", C.c_int)]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class _Allocator(C.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", C.c_void_p)]


class _Estimate(C.Structure):
    _fields_ = [("iter", C.c_int64), ("shift", C.c_double), ("nw_pre", C.c_int64), ("n0", C.c_int64),
                ("num_hi", C.c_int64), ("num_lo", C.c_uint64), ("num", C.c_double), ("nw_post", C.c_int64),
                ("ndet", C.c_int64), ("natt", C.c_int64), ("nspawn", C.c_int64), ("tau", C.c_double)]


class _Learning(C.Structure):
    _fields_ = [("width", C.c_int), ("batch", C.c_int), ("period", C.c_int), ("learning_rate", C.c_double),
                ("seed", C.c_uint64)]


class _Tuning(C.Structure):
    _fields_ = [("bucket_spawns", C.c_int), ("bucket_new", C.c_int), ("attempt_blocks", C.c_int),
                ("ms_per_iteration", C.c_double)]


class _State(C.Structure):
    _fields_ = [("iter", C.c_int64), ("shift", C.c_double), ("nw_ref", C.c_int64), ("vary", C.c_int),
                ("core_active", C.c_int), ("ncore", C.c_int64), ("tau", C.c_double), ("rmax", C.c_double)]


class _Diag(C.Structure):
    _fields_ = [("error_bits", C.c_uint32), ("ndet", C.c_int64), ("natt", C.c_int64), ("nspawn", C.c_int64),
                ("nbuckets", C.c_int64), ("bucket_main", C.c_int64), ("max_bucket_spawns", C.c_int64),
                ("tile_capacity", C.c_int64), ("ncore", C.c_int64),
                ("launches_per_iteration", C.c_int64), ("deferred_buckets", C.c_int64)]


# names declared in include/hande.h, in order
EXPORTS = ["hande_init_system", "hande_iterate", "hande_iterate_timed", "hande_synchronize", "hande_estimators", "hande_get_walkers",
           "hande_set_walkers", "hande_autotune", "hande_diagnostics", "hande_estimate_noalloc", "hande_get_state", "hande_set_state",
           "hande_reference", "hande_iterations", "hande_destroy", "hande_last_error",
           "hande_batch_init", "hande_batch_iterate", "hande_batch_failed_replica", "hande_batch_autotune",
           "hande_batch_size", "hande_batch_layout", "hande_batch_replica", "hande_batch_synchronize", "hande_batch_destroy", "hande_set_proposal", "hande_get_proposal", "hande_learn_proposal",
           "hande_learn_params", "hande_learn_gradients", "hande_learn_probabilities", "hande_learn_refresh",
           "hande_gemm_bf16"]

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libhande.so (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_needed:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build the CUDA extension first")
        lib = C.CDLL(path)
        P = C.c_void_p
        u64p, i64p, dp = C.POINTER(C.c_uint64), C.POINTER(C.c_int64), C.POINTER(C.c_double)
        lib.hande_init_system.argtypes = [C.POINTER(_System), C.POINTER(_Qmc), C.POINTER(_Allocator), P,
                                          C.POINTER(P)]
        lib.hande_iterate.argtypes = [P, C.c_int]
        lib.hande_iterate_timed.argtypes = [P, C.c_int, C.POINTER(C.c_float), C.c_int]
        lib.hande_synchronize.argtypes = [P]
        lib.hande_estimators.argtypes = [P, C.POINTER(_Estimate), C.c_int, C.POINTER(C.c_int)]
        lib.hande_get_walkers.argtypes = [P, u64p, i64p, dp, C.POINTER(C.c_uint8), C.c_int64, i64p]
        lib.hande_set_walkers.argtypes = [P, u64p, i64p, dp, C.c_int64]
        lib.hande_reference.argtypes = [P, dp, u64p]
        lib.hande_iterations.argtypes = [P]
        lib.hande_iterations.restype = C.c_int64
        lib.hande_destroy.argtypes = [P]
        lib.hande_destroy.restype = None
        lib.hande_last_error.argtypes = [P]
        lib.hande_last_error.restype = C.c_char_p
        lib.hande_diagnostics.argtypes = [P, C.POINTER(_Diag)]
        lib.hande_estimate_noalloc.argtypes = [P, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]
        lib.hande_autotune.argtypes = [P, C.c_int, C.POINTER(_Tuning)]
        lib.hande_autotune.restype = C.c_int
        lib.hande_get_state.argtypes = [P, C.POINTER(_State), u64p, C.c_int64]
        lib.hande_set_state.argtypes = [P, C.POINTER(_State), u64p]
        for name in EXPORTS[:12]:
            getattr(lib, name).restype = C.c_int
        lib.hande_batch_init.argtypes = [C.POINTER(_System), C.POINTER(_Qmc), C.c_int, C.POINTER(_Allocator), P,
                                         C.POINTER(P), C.POINTER(C.c_int)]
        lib.hande_batch_iterate.argtypes = [P, C.c_int]
        lib.hande_batch_size.argtypes = [P]
        lib.hande_batch_layout.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        lib.hande_batch_layout.restype = C.c_int
        lib.hande_batch_replica.argtypes = [P, C.c_int]
        lib.hande_batch_replica.restype = P
        lib.hande_batch_synchronize.argtypes = [P]
        lib.hande_batch_destroy.argtypes = [P]
        lib.hande_batch_destroy.restype = None
        lib.hande_batch_failed_replica.argtypes = [P]
        lib.hande_batch_failed_replica.restype = C.c_int
        lib.hande_batch_autotune.argtypes = [P, C.c_int, dp, dp]
        lib.hande_batch_autotune.restype = C.c_int
        for name in ("hande_batch_init", "hande_batch_iterate", "hande_batch_size", "hande_batch_synchronize"):
            getattr(lib, name).restype = C.c_int
        lib.hande_gemm_bf16.argtypes = [P, C.c_int64, P, C.c_int64, P, C.c_int64, C.c_int, C.c_int, C.c_int, P, P]
        lib.hande_gemm_bf16.restype = C.c_int
        u32p, i32p, fp = C.POINTER(C.c_uint32), C.POINTER(C.c_int32), C.POINTER(C.c_float)
        lib.hande_set_proposal.argtypes = [P, u32p]
        lib.hande_get_proposal.argtypes = [P, u32p]
        lib.hande_learn_proposal.argtypes = [P, C.POINTER(_Learning)]
        lib.hande_learn_params.argtypes = [P, fp, fp, C.c_int64, i64p]
        lib.hande_learn_gradients.argtypes = [P, i32p, i32p, fp, C.c_int, fp, dp]
        lib.hande_learn_probabilities.argtypes = [P, i32p, C.c_int, fp]
        lib.hande_learn_refresh.argtypes = [P]
        for name in ("hande_set_proposal", "hande_get_proposal", "hande_learn_proposal", "hande_learn_params",
                     "hande_learn_gradients", "hande_learn_probabilities", "hande_learn_refresh"):
            getattr(lib, name).restype = C.c_int
        _lib = lib
        return lib


def _torch_allocator(device):
    import torch

    stream = torch.cuda.current_stream(device)

    def alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream)
        except Exception:  # out of memory: the library reports HANDE_ERR_NOMEM
            return None

    def free(ptr, nbytes, user):
        torch.cuda.caching_allocator_delete(ptr)

    return _ALLOC_FN(alloc), _FREE_FN(free)


def _structs(system: dict, qmc: dict):
    """The C structs of one run (and the arrays they point into, to keep alive)."""
    s = _System()
    s.kind = _KIND[system["kind"]]
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
    keep = []
    if s.kind == 2:
        h1 = np.ascontiguousarray(system["h1"], dtype=np.float64)
        eri = np.ascontiguousarray(system["eri"], dtype=np.float64)
        keep += [h1, eri]
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
    q.state_capacity = int(qmc.get("state_capacity", 0))
    q.spawn_capacity = int(qmc.get("spawn_capacity", 0))
    q.record_capacity = int(qmc.get("record_capacity", 0))
    q.tile_capacity = int(qmc.get("tile_capacity", 0))
    q.annihilation = int(qmc.get("annihilation", 0))
    q.excit_gen = int(qmc.get("excit_gen", 0))
    q.tau_search = int(qmc.get("tau_search", 0))
    return s, q, keep


def _stream_and_allocator(stream, torch_memory):
    """The CUDA stream handle (PyTorch's current stream by default) and the
    allocator struct routing device memory through PyTorch (or None)."""
    alloc, fns = None, None
    if stream is None or torch_memory:
        import torch
        dev = torch.cuda.current_device()
        if stream is None:
            stream = torch.cuda.current_stream(dev).cuda_stream
        if torch_memory:
            fns = _torch_allocator(dev)
            alloc = _Allocator(fns[0], fns[1], None)
    return int(stream), alloc, fns


class Hande:
    """One FCIQMC run on the current CUDA device (see include/hande.h)."""

    def __init__(self, system: dict, qmc: dict, stream: int | None = None, torch_memory: bool = True):
        lib = load()
        self._lib = lib
        self._h = C.c_void_p()
        self._batch = None
        s, q, self._keep = _structs(system, qmc)
        self.W = s.key_words
        self._system_norb = s.norb
        self.stream, self._alloc, self._alloc_fns = _stream_and_allocator(stream, torch_memory)
        alloc_p = C.byref(self._alloc) if self._alloc is not None else None
        rc = lib.hande_init_system(C.byref(s), C.byref(q), alloc_p, C.c_void_p(self.stream), C.byref(self._h))
        if rc != 0:
            raise HandeError(rc, "hande_init_system failed")

    # ------------------------------------------------------------------ calls
    def _check(self, rc: int, what: str):
        if rc != 0:
            msg = self._lib.hande_last_error(self._h).decode()
            raise HandeError(rc, f"{what}: {msg}")

    def iterate(self, n: int = 1) -> None:
        self._check(self._lib.hande_iterate(self._h, int(n)), "hande_iterate")

    PHASES = ("det_pass", "attempt_scan", "split", "core", "attempt", "bucket_scan", "scatter", "merge",
              "new_hdiag", "finalize")

    def iterate_timed(self, n: int = 1) -> dict:
        """n iterations launched kernel by kernel with CUDA events between the
        phases; returns summed device milliseconds per phase."""
        buf = (C.c_float * len(self.PHASES))()
        self._check(self._lib.hande_iterate_timed(self._h, int(n), buf, len(self.PHASES)), "hande_iterate_timed")
        return {k: float(v) for k, v in zip(self.PHASES, buf)}

    def estimate_noalloc(self, d_keys: int, d_pops: int, n: int, d_out: int) -> None:
        """Projected-energy sums of a walker list in device memory (pointers as
        ints), written to d_out[4] on the context's stream; allocates nothing."""
        self._check(self._lib.hande_estimate_noalloc(self._h, C.c_void_p(d_keys), C.c_void_p(d_pops), int(n),
                                                     C.c_void_p(d_out)), "hande_estimate_noalloc")

    def diagnostics(self) -> dict:
        d = _Diag()
        self._check(self._lib.hande_diagnostics(self._h, C.byref(d)), "hande_diagnostics")
        return {name: getattr(d, name) for name, _ in _Diag._fields_}

    def autotune(self, iterations: int = 5) -> dict:
        """Choose bucket sizes and the spawning grid by timing (include/hande.h,
        hande_autotune); the run advances, its walker lists do not change."""
        t = _Tuning()
        self._check(self._lib.hande_autotune(self._h, int(iterations), C.byref(t)), "hande_autotune")
        return {name: getattr(t, name) for name, _ in _Tuning._fields_}

    def launches_per_iteration(self) -> int:
        """Kernels one iteration launches with the current settings."""
        return int(self.diagnostics()["launches_per_iteration"])

    def synchronize(self) -> None:
        self._check(self._lib.hande_synchronize(self._h), "hande_synchronize")

    @property
    def iterations(self) -> int:
        return int(self._lib.hande_iterations(self._h))

    def reference(self):
        e = C.c_double()
        k = np.zeros(self.W, dtype=np.uint64)
        self._check(self._lib.hande_reference(self._h, C.byref(e), k.ctypes.data_as(C.POINTER(C.c_uint64))),
                    "hande_reference")
        return e.value, k

    def estimators(self, max_records: int = 1 << 20) -> dict:
        """Records of the iterations since the last call (at most max_records),
        fetched through one reused 4096-record buffer."""
        if getattr(self, "_est_buf", None) is None:
            self._est_buf = (_Estimate * 4096)()
        buf, parts, left = self._est_buf, [], int(max_records)
        while left > 0:
            n = C.c_int()
            want = min(left, len(buf))
            self._check(self._lib.hande_estimators(self._h, buf, want, C.byref(n)), "hande_estimators")
            if n.value:
                parts.append(np.ctypeslib.as_array(buf)[: n.value].copy())
            left -= n.value
            if n.value < want:
                break
        arr = np.concatenate(parts) if parts else np.ctypeslib.as_array(buf)[:0]
        return {name: np.array(arr[name]) for name, _ in _Estimate._fields_}

    def host_buffers(self, capacity: int, pinned: bool = True):
        """Host arrays (keys, populations, H_ii - E_ref, flags) for `capacity`
        determinants, page-locked by default, for reuse with walkers(out=...)."""
        alloc = _pinned_array if pinned else (lambda shape, dt: np.zeros(shape, dtype=dt))
        return (alloc((capacity, self.W), np.uint64), alloc((capacity,), np.int64),
                alloc((capacity,), np.float64), alloc((capacity,), np.uint8))

    def walkers(self, out=None):
        """The walker list (keys, populations, H_ii - E_ref, core flags) in host
        memory: new arrays, or views of the given host_buffers(...) when they are
        large enough (page-locked buffers make the copies direct DMA)."""
        n = C.c_int64()
        rc = self._lib.hande_get_walkers(self._h, None, None, None, None, 0, C.byref(n))
        if rc not in (0, -3):
            self._check(rc, "hande_get_walkers")
        cap = n.value
        if out is not None and len(out[1]) >= cap:
            keys, pops, hd, fl = out
            cap = len(pops)
        else:
            keys = np.zeros((cap, self.W), dtype=np.uint64)
            pops = np.zeros(cap, dtype=np.int64)
            hd = np.zeros(cap, dtype=np.float64)
            fl = np.zeros(cap, dtype=np.uint8)
        self._check(self._lib.hande_get_walkers(self._h, keys.ctypes.data_as(C.POINTER(C.c_uint64)),
                                                pops.ctypes.data_as(C.POINTER(C.c_int64)),
                                                hd.ctypes.data_as(C.POINTER(C.c_double)),
                                                fl.ctypes.data_as(C.POINTER(C.c_uint8)), cap, C.byref(n)),
                    "hande_get_walkers")
        m = n.value
        return keys[:m], pops[:m], hd[:m], fl[:m]

    def set_walkers(self, keys, pops, hdiag=None) -> None:
        k = np.ascontiguousarray(np.asarray(keys, dtype=np.uint64).reshape(-1, self.W))
        p = np.ascontiguousarray(pops, dtype=np.int64)
        hp = None
        if hdiag is not None:
            h = np.ascontiguousarray(hdiag, dtype=np.float64)
            self._hd_keep = h
            hp = h.ctypes.data_as(C.POINTER(C.c_double))
        self._check(self._lib.hande_set_walkers(self._h, k.ctypes.data_as(C.POINTER(C.c_uint64)),
                                                p.ctypes.data_as(C.POINTER(C.c_int64)), hp, len(p)),
                    "hande_set_walkers")

    def state(self):
        """Restart snapshot beyond the walker list: (dict of the run state,
        deterministic-space keys[ncore, W] ascending)."""
        st = _State()
        self._check(self._lib.hande_get_state(self._h, C.byref(st), None, 0), "hande_get_state")
        keys = np.zeros((max(int(st.ncore), 1), self.W), dtype=np.uint64)
        self._check(self._lib.hande_get_state(self._h, C.byref(st), keys.ctypes.data_as(C.POINTER(C.c_uint64)),
                                              len(keys)), "hande_get_state")
        d = {name: getattr(st, name) for name, _ in _State._fields_}
        return d, keys[:int(st.ncore)].copy()

    def set_state(self, state: dict, core_keys=None) -> None:
        """Restore a snapshot taken by state() (after set_walkers of its list)."""
        st = _State()
        for name, _ in _State._fields_:
            setattr(st, name, state[name])
        kp = None
        if core_keys is not None and len(core_keys):
            k = np.ascontiguousarray(np.asarray(core_keys, dtype=np.uint64).reshape(-1, self.W))
            self._core_keep = k
            kp = k.ctypes.data_as(C.POINTER(C.c_uint64))
        self._check(self._lib.hande_set_state(self._h, C.byref(st), kp), "hande_set_state")

    # ------------------------------------------------------------ learned proposal
    def _norb(self):
        return int(self._system_norb)

    def set_proposal(self, q) -> None:
        """Integer weights q[2 M^2, M] of the UEG proposal table (excit_gen = 1)."""
        a = np.ascontiguousarray(q, dtype=np.uint32)
        self._check(self._lib.hande_set_proposal(self._h, a.ctypes.data_as(C.POINTER(C.c_uint32))),
                    "hande_set_proposal")

    def proposal(self) -> np.ndarray:
        M = self._norb()
        q = np.zeros((2 * M * M, M), dtype=np.uint32)
        self._check(self._lib.hande_get_proposal(self._h, q.ctypes.data_as(C.POINTER(C.c_uint32))),
                    "hande_get_proposal")
        return q

    def learn_proposal(self, width=256, batch=4096, period=10, learning_rate=1e-3, seed=1) -> None:
        """Attach the learned proposal (include/hande.h, hande_learn_proposal)."""
        L = _Learning(int(width), int(batch), int(period), float(learning_rate), int(seed))
        self._check(self._lib.hande_learn_proposal(self._h, C.byref(L)), "hande_learn_proposal")

    def learn_params(self, set_params=None) -> np.ndarray:
        """The network's parameters as one float32 vector (optionally replaced first)."""
        n = C.c_int64()
        self._check(self._lib.hande_learn_params(self._h, None, None, 0, C.byref(n)), "hande_learn_params")
        out = np.zeros(n.value, dtype=np.float32)
        sp = None
        if set_params is not None:
            src = np.ascontiguousarray(set_params, dtype=np.float32)
            if src.size != n.value:
                raise ValueError(f"expected {n.value} parameters")
            self._params_keep = src
            sp = src.ctypes.data_as(C.POINTER(C.c_float))
        self._check(self._lib.hande_learn_params(self._h, out.ctypes.data_as(C.POINTER(C.c_float)), sp, n.value,
                                                 None), "hande_learn_params")
        return out

    def learn_gradients(self, rows, targets, weights):
        """(loss, gradient vector) of a sample batch through the BF16 tensor-core kernels."""
        r = np.ascontiguousarray(rows, dtype=np.int32)
        t = np.ascontiguousarray(targets, dtype=np.int32)
        w = np.ascontiguousarray(weights, dtype=np.float32)
        n = C.c_int64()
        self._check(self._lib.hande_learn_params(self._h, None, None, 0, C.byref(n)), "hande_learn_params")
        g = np.zeros(n.value, dtype=np.float32)
        loss = C.c_double()
        self._check(self._lib.hande_learn_gradients(self._h, r.ctypes.data_as(C.POINTER(C.c_int32)),
                                                    t.ctypes.data_as(C.POINTER(C.c_int32)),
                                                    w.ctypes.data_as(C.POINTER(C.c_float)), len(r),
                                                    g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss)),
                    "hande_learn_gradients")
        return loss.value, g

    def learn_probabilities(self, rows) -> np.ndarray:
        r = np.ascontiguousarray(rows, dtype=np.int32)
        M = self._norb()
        p = np.zeros((len(r), M), dtype=np.float32)
        self._check(self._lib.hande_learn_probabilities(self._h, r.ctypes.data_as(C.POINTER(C.c_int32)), len(r),
                                                        p.ctypes.data_as(C.POINTER(C.c_float))),
                    "hande_learn_probabilities")
        return p

    def learn_refresh(self) -> None:
        self._check(self._lib.hande_learn_refresh(self._h), "hande_learn_refresh")

    def close(self) -> None:
        if self._h and self._batch is None:   # a batch's replica is freed with its batch
            self._lib.hande_destroy(self._h)
        self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def gemm_bf16(a, b, out=None, stream=None, status=None):
    """D = A B^T on the tensor cores (include/hande.h, hande_gemm_bf16) for
    CUDA tensors: a (m x k) and b (n x k) bfloat16, row-major with unit column
    stride; returns (or fills) a float32 (m x n) tensor.  With `status` (an
    int32 CUDA tensor) the call is asynchronous and a device-side timeout is
    ORed into status[0]; without it the call synchronises."""
    import torch
    lib = load()
    m, k = a.shape
    n, k2 = b.shape
    if k2 != k or a.dtype != torch.bfloat16 or b.dtype != torch.bfloat16 or a.stride(1) != 1 or b.stride(1) != 1:
        raise ValueError("a (m x k) and b (n x k) must be bfloat16 with unit column stride")
    if out is None:
        out = torch.empty((m, n), dtype=torch.float32, device=a.device)
    if stream is None:
        stream = torch.cuda.current_stream(a.device).cuda_stream
    sp = C.c_void_p(status.data_ptr()) if status is not None else None
    rc = lib.hande_gemm_bf16(C.c_void_p(a.data_ptr()), a.stride(0), C.c_void_p(b.data_ptr()), b.stride(0),
                             C.c_void_p(out.data_ptr()), out.stride(0), m, n, k, sp, C.c_void_p(int(stream)))
    if rc != 0:
        raise HandeError(rc, "hande_gemm_bf16")
    return out


class HandeBatch:
    """Independent replicas advanced together on the current CUDA device
    (include/hande.h, batches).  `replicas[r]` is a Hande view of replica r
    (owned by the batch): walkers, estimators and diagnostics as for one run."""

    def __init__(self, systems, qmcs, stream: int | None = None, torch_memory: bool = True):
        systems, qmcs = list(systems), list(qmcs)
        if len(systems) != len(qmcs) or not systems:
            raise ValueError("one system and one qmc dict per replica")
        lib = load()
        self._lib = lib
        self._h = C.c_void_p()
        n = len(systems)
        S, Q, self._keep = (_System * n)(), (_Qmc * n)(), []
        for r in range(n):
            s, q, keep = _structs(systems[r], qmcs[r])
            S[r], Q[r] = s, q
            self._keep += keep
        self.stream, self._alloc, self._alloc_fns = _stream_and_allocator(stream, torch_memory)
        alloc_p = C.byref(self._alloc) if self._alloc is not None else None
        bad = C.c_int(-1)
        rc = lib.hande_batch_init(S, Q, n, alloc_p, C.c_void_p(self.stream), C.byref(self._h), C.byref(bad))
        if rc != 0:
            raise HandeError(rc, f"hande_batch_init failed (replica {bad.value})")
        self.replicas = []
        for r in range(n):
            v = object.__new__(Hande)
            v._lib, v._batch, v._keep = lib, self, []
            v._h = C.c_void_p(lib.hande_batch_replica(self._h, r))
            v.W = int(systems[r]["key_words"])
            v._system_norb = int(systems[r]["norb"])
            v.stream, v._alloc, v._alloc_fns = None, None, None
            self.replicas.append(v)

    def __len__(self) -> int:
        return int(self._lib.hande_batch_size(self._h))

    def _raise(self, rc, what):
        r = int(self._lib.hande_batch_failed_replica(self._h))
        msg = self._lib.hande_last_error(self.replicas[r]._h).decode() if r >= 0 else ""
        err = HandeError(rc, f"{what}: replica {r}: {msg}")
        err.replica = r
        raise err

    def iterate(self, n: int = 1) -> None:
        rc = self._lib.hande_batch_iterate(self._h, int(n))
        if rc != 0:
            self._raise(rc, "hande_batch_iterate")

    def synchronize(self) -> None:
        rc = self._lib.hande_batch_synchronize(self._h)
        if rc != 0:
            self._raise(rc, "hande_batch_synchronize")

    def autotune(self, iterations: int = 5):
        """Choose the batched launch shape by timing (include/hande.h,
        hande_batch_autotune); returns (scale, ms per batched iteration)."""
        f, ms = C.c_double(), C.c_double()
        rc = self._lib.hande_batch_autotune(self._h, int(iterations), C.byref(f), C.byref(ms))
        if rc != 0:
            self._raise(rc, "hande_batch_autotune")
        return f.value, ms.value

    def layout(self):
        """(launch groups of a batched iteration, most replicas per group; 0 =
        no limit) as now in use (include/hande.h, hande_batch_layout)."""
        g, cap = C.c_int(), C.c_int()
        rc = self._lib.hande_batch_layout(self._h, C.byref(g), C.byref(cap))
        if rc != 0:
            self._raise(rc, "hande_batch_layout")
        return g.value, cap.value

    def close(self) -> None:
        if self._h:
            for v in self.replicas:
                v._h = C.c_void_p()
            self._lib.hande_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
