"""FP64 CPU oracle for the psi-score (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It shares no code with the CUDA path.

* ``psi_oracle.c`` (wrapped here): the matrices A, B, c, d built entry by entry from their
  definitions (Sec. II, after Eqs. 6-7); Power-psi as Algorithm 2; Power-NF as
  Algorithm 1; PageRank's power method (Eq. 22); the newsfeed mass used by the sum
  identity; the ranking.
* ``dense.py``: dense linear-algebra routes for small N -- the N per-origin systems
  (Eqs. 10-11, 7, 9), the one-system form (Eq. 12) and the scalar balance equations
  (Eqs. 1-5).

Parity status: every routine here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed forms, brute force over all 4-user graphs, PageRank
special cases, the sum identity, residual certificates).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psi_oracle.c")
_LIB = os.path.join(_HERE, "libpsi_oracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_ID, ERR_SELF_LOOP, ERR_RATE, ERR_NOMEM, NOT_CONVERGED = 0, 1, 2, 3, 4, 5, 7
TOL_PSI, TOL_S_ABS = 0, 1
BNORM_NONE, BNORM_INF = 0, 1


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle status {code}")
        self.code = code


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("gap_s", ctypes.c_double), ("gap", ctypes.c_double),
                ("bnorm", ctypes.c_double), ("converged", ctypes.c_int32), ("threads", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile ``libpsi_oracle.so`` (gcc, FP contraction off, OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11", _SRC, "-o", _LIB + ".tmp"]
    try:
        subprocess.run(base[:5] + ["-fopenmp"] + base[5:] + ["-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-lm"], check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, dbl, p = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
            lib.orc_num_threads.restype = i32
            lib.orc_set_threads.argtypes = [i32]
            lib.orc_canonical_edges.restype = i32
            lib.orc_canonical_edges.argtypes = [i64, i64, p, p, i32, p, p, ctypes.POINTER(i64)]
            lib.orc_model_create.restype = p
            lib.orc_model_create.argtypes = [i64, i64, p, p, p, p, i32, ctypes.POINTER(i32)]
            lib.orc_model_destroy.argtypes = [p]
            lib.orc_model_dims.argtypes = [p, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(dbl)]
            lib.orc_model_vectors.argtypes = [p, p, p, p]
            lib.orc_model_edges.argtypes = [p, p, p]
            lib.orc_apply_AB.argtypes = [p, p, p, p]
            lib.orc_psi_from_s.argtypes = [p, p, p]
            lib.orc_power_psi.restype = i32
            lib.orc_power_psi.argtypes = [p, dbl, i32, i32, i64, i32, p, p, p, p, ctypes.POINTER(Info)]
            lib.orc_power_nf.restype = i32
            lib.orc_power_nf.argtypes = [p, dbl, i64, p, ctypes.POINTER(i64)]
            lib.orc_power_nf_origins.restype = i32
            lib.orc_power_nf_origins.argtypes = [p, dbl, i64, p, i64, p, ctypes.POINTER(i64)]
            lib.orc_newsfeed_mass.restype = i64
            lib.orc_newsfeed_mass.argtypes = [p, i64, p]
            lib.orc_pagerank.restype = i64
            lib.orc_pagerank.argtypes = [i64, i64, p, p, dbl, i64, p]
            lib.orc_topk.restype = i32
            lib.orc_topk.argtypes = [i64, p, i64, p, p]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_threads(t: int) -> None:
    _load().orc_set_threads(int(t))


def canonical_edges(n, follower, leader, drop_self_loops=False):
    """Validated, sorted (follower, leader) pairs with duplicates merged."""
    f, l = _i32(follower), _i32(leader)
    fo = np.empty(max(f.size, 1), np.int32)
    lo = np.empty(max(f.size, 1), np.int32)
    m = ctypes.c_int64(0)
    st = _load().orc_canonical_edges(n, f.size, _p(f), _p(l), int(drop_self_loops), _p(fo), _p(lo), ctypes.byref(m))
    if st != OK:
        raise OracleError(st)
    return fo[: m.value].copy(), lo[: m.value].copy()


class Model:
    """A, B, c, d of one graph, built from their definitions (explicit per-edge values)."""

    def __init__(self, n, follower, leader, lam, mu, drop_self_loops=False):
        self._lib = _load()
        f, l = _i32(follower), _i32(leader)
        self._lam, self._mu = _f64(lam), _f64(mu)
        st = ctypes.c_int32(0)
        h = self._lib.orc_model_create(int(n), f.size, _p(f), _p(l), _p(self._lam), _p(self._mu),
                                       int(drop_self_loops), ctypes.byref(st))
        if not h:
            raise OracleError(st.value)
        self._h = h
        nn, mm, bn = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        self._lib.orc_model_dims(h, ctypes.byref(nn), ctypes.byref(mm), ctypes.byref(bn))
        self.n, self.m, self.bnorm_inf = nn.value, mm.value, bn.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_model_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def lam(self):
        return self._lam

    @property
    def mu(self):
        return self._mu

    def vectors(self):
        """(c, d, sigma)"""
        c, d, s = (np.empty(self.n) for _ in range(3))
        self._lib.orc_model_vectors(self._h, _p(c), _p(d), _p(s))
        return c, d, s

    def edges(self):
        f = np.empty(max(self.m, 1), np.int32)
        l = np.empty(max(self.m, 1), np.int32)
        self._lib.orc_model_edges(self._h, _p(f), _p(l))
        return f[: self.m], l[: self.m]

    def apply(self, s):
        """(s^T A, s^T B)"""
        s = _f64(s)
        a, b = np.empty(self.n), np.empty(self.n)
        self._lib.orc_apply_AB(self._h, _p(s), _p(a), _p(b))
        return a, b

    def psi_from_s(self, s):
        s = _f64(s)
        out = np.empty(self.n)
        self._lib.orc_psi_from_s(self._h, _p(s), _p(out))
        return out

    def power_psi(self, eps=0.0, tol_mode=TOL_PSI, bnorm_mode=BNORM_NONE, max_iter=100000,
                  to_floor=False, s_init=None, history=False):
        """Algorithm 2.  Returns dict(psi, s, iters, gap_s, gap, converged[, gaps])."""
        s = np.empty(self.n)
        psi = np.empty(self.n)
        hist = np.empty(max(int(max_iter), 1)) if history else None
        info = Info()
        si = None if s_init is None else _f64(s_init)
        st = self._lib.orc_power_psi(self._h, float(eps), int(tol_mode), int(bnorm_mode), int(max_iter),
                                     int(to_floor), _p(si), _p(s), _p(psi), _p(hist), ctypes.byref(info))
        if st not in (OK, NOT_CONVERGED):
            raise OracleError(st)
        out = dict(psi=psi, s=s, iters=info.iters, gap_s=info.gap_s, gap=info.gap,
                   converged=bool(info.converged), bnorm=info.bnorm, threads=info.threads)
        if history:
            out["gaps"] = hist[: info.iters].copy()
        return out

    def power_nf(self, eps, max_iter=100000, origins=None):
        """Algorithm 1 for every origin, or for the listed origins (input ids) only: each
        origin is its own problem, so a subset gives the same values.  Returns (psi,
        matvecs), psi[q] the score of the q-th origin."""
        mv = ctypes.c_int64(0)
        if origins is None:
            psi = np.empty(self.n)
            self._lib.orc_power_nf(self._h, float(eps), int(max_iter), _p(psi), ctypes.byref(mv))
            return psi, mv.value
        ids = np.ascontiguousarray(origins, np.int64)
        psi = np.empty(ids.size)
        st = self._lib.orc_power_nf_origins(self._h, float(eps), int(max_iter), _p(ids), ids.size, _p(psi),
                                            ctypes.byref(mv))
        if st not in (0, 7):  # OK, or not converged within max_iter
            raise OracleError(st)
        return psi, mv.value

    def newsfeed_mass(self, max_iter=100000):
        m = np.empty(self.n)
        self._lib.orc_newsfeed_mass(self._h, int(max_iter), _p(m))
        return m


def pagerank(n, follower, leader, alpha, max_iter=100000):
    """Eq. 22 on canonical edges (no dangling redistribution), to the FP64 floor."""
    f, l = canonical_edges(n, follower, leader)
    pi = np.empty(n)
    _load().orc_pagerank(n, f.size, _p(f), _p(l), float(alpha), int(max_iter), _p(pi))
    return pi


def topk(psi, k):
    """Ranking by psi descending, ties by id ascending."""
    psi = _f64(psi)
    k = min(int(k), psi.size)
    ids = np.empty(max(k, 1), np.int32)
    vals = np.empty(max(k, 1))
    _load().orc_topk(psi.size, _p(psi), k, _p(ids), _p(vals))
    return ids[:k], vals[:k]


def solve(n, follower, leader, lam, mu, eps=1e-8, tol_mode=TOL_PSI, bnorm_mode=BNORM_NONE,
          max_iter=100000, to_floor=False, drop_self_loops=False):
    """One call: model + Algorithm 2.  Returns the power_psi dict plus m_unique."""
    with Model(n, follower, leader, lam, mu, drop_self_loops) as g:
        out = g.power_psi(eps, tol_mode, bnorm_mode, max_iter, to_floor)
        out["m_unique"] = g.m
        out["bnorm_inf"] = g.bnorm_inf
        return out
