"""The C-ABI library loads and exports every entry point include/hande.h
declares; argument validation runs without a GPU."""
from __future__ import annotations

import ctypes as C
import os
import re

import pytest

from paper_1811_11679_gb300 import hande, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "hande.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hande_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = hande.load()
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(hande.EXPORTS) == names


def test_invalid_arguments_rejected_before_any_device_call():
    lib = hande.load()
    out = C.c_void_p()
    assert lib.hande_init_system(None, None, None, None, C.byref(out)) == -1
    s = hande._System()
    q = hande._Qmc()
    s.kind, s.key_words, s.norb, s.nalpha, s.nbeta = 1, 3, 19, 7, 7   # key_words must be 1, 2 or 8
    q.tau, q.init_pop = 0.01, 10.0
    assert lib.hande_init_system(C.byref(s), C.byref(q), None, None, C.byref(out)) == -1
    s.key_words, s.rs = 1, 1.0
    q.tau = -1.0
    assert lib.hande_init_system(C.byref(s), C.byref(q), None, None, C.byref(out)) == -1
    q.tau = 0.01
    q.semi_stoch_size, q.real_amplitudes = 10, 0   # semi-stochastic needs real weights
    assert lib.hande_init_system(C.byref(s), C.byref(q), None, None, C.byref(out)) == -1
    s.kind, s.norb, s.nalpha, s.nbeta, s.periodic = 0, 2, 1, 1, 1   # periodic 2-site ring
    q.semi_stoch_size = 0
    assert lib.hande_init_system(C.byref(s), C.byref(q), None, None, C.byref(out)) == -1
    assert lib.hande_iterate(None, 1) == -1
    assert lib.hande_last_error(None) == b"no context"
    lib.hande_destroy(None)


def test_python_binding_has_no_cpu_fallback(monkeypatch, tmp_path):
    """With the shared library missing, the binding raises instead of computing."""
    monkeypatch.setattr(hande, "_lib", None)
    monkeypatch.setattr(hande._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        hande.load(build_if_needed=False)


def test_batch_arguments_rejected_before_any_device_call():
    lib = hande.load()
    out = C.c_void_p()
    bad = C.c_int(7)
    s, q = hande._System(), hande._Qmc()
    assert lib.hande_batch_init(None, None, 1, None, None, C.byref(out), C.byref(bad)) == -1
    assert bad.value == -1
    assert lib.hande_batch_init(C.byref(s), C.byref(q), 0, None, None, C.byref(out), None) == -1
    assert lib.hande_batch_iterate(None, 1) == -1
    assert lib.hande_batch_synchronize(None) == -1
    assert lib.hande_batch_size(None) == 0
    assert lib.hande_batch_layout(None, None, None) == -1
    assert lib.hande_batch_replica(None, 0) is None
    lib.hande_batch_destroy(None)


def test_batch_binding_marshalling_and_errors(monkeypatch):
    """HandeBatch passes one (system, qmc) struct pair per replica, names the
    failing replica (hande_batch_failed_replica) and its message on an error,
    and frees the batch once (its replica views never free their contexts)."""
    seen = {"destroy": 0}

    class FakeLib:
        def hande_batch_init(self, S, Q, n, alloc, stream, out, bad):
            seen["n"], seen["stream"], seen["alloc"] = n, stream.value, alloc
            seen["sys"] = [(S[r].kind, S[r].key_words, S[r].norb, S[r].rs) for r in range(n)]
            seen["qmc"] = [(Q[r].seed, Q[r].replica, Q[r].target_population) for r in range(n)]
            out._obj.value = 77
            return 0

        def hande_batch_replica(self, h, r):
            return 1000 + r

        def hande_batch_size(self, h):
            return seen["n"]

        def hande_batch_iterate(self, h, k):
            return -3

        def hande_batch_failed_replica(self, h):
            return 1

        def hande_last_error(self, h):
            return b"spawn capacity exceeded" if h.value == 1001 else b""

        def hande_batch_destroy(self, h):
            seen["destroy"] += 1

        def hande_destroy(self, h):
            raise AssertionError("a replica view must not free its context")

    monkeypatch.setattr(hande, "load", lambda build_if_needed=True: FakeLib())
    s1, q1 = inputs.workload("hubbard8")
    s2, q2 = inputs.workload("ueg14")
    b = hande.HandeBatch([s1, s2], [q1, dict(q2, replica=5)], stream=99, torch_memory=False)
    assert len(b) == 2 and seen["stream"] == 99 and seen["alloc"] is None
    assert seen["sys"] == [(0, 1, 8, 0.0), (1, 2, 38, 1.0)]
    assert seen["qmc"] == [(8, 0, 1e4), (7, 5, 1e6)]
    assert [v.W for v in b.replicas] == [1, 2]
    with pytest.raises(hande.HandeError, match=r"replica 1: spawn capacity exceeded"):
        b.iterate(3)
    b.replicas[0].close()
    b.close()
    b.close()
    assert seen["destroy"] == 1
    assert all(not v._h for v in b.replicas)
