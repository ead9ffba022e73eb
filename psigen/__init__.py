"""Seeded synthetic inputs for the psi-score solver (shared by the CUDA path's tests and
benchmark and by the CPU oracle).

This module draws follower graphs and activity rates only; it holds none of the method's
arithmetic.  The C code in ``psigen.c`` does the drawing; this file compiles it on demand
with gcc and wraps it with ctypes.

Edge convention (paper Sec. II): edge k means ``follower[k]`` follows ``leader[k]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psigen.c")
_LIB = os.path.join(_HERE, "libpsigen.so")
_lock = threading.Lock()
_lib = None

# stream ids used for rates (graph streams live inside psigen.c)
STREAM_LAMBDA = 101
STREAM_MU = 102
STREAM_SIZES = 103


def build(force: bool = False) -> str:
    """Compile ``libpsigen.so`` next to this file (gcc, OpenMP when available)."""
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
            i64, u64, i32, dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double
            p = ctypes.c_void_p
            lib.psigen_splitmix64_at.restype = u64
            lib.psigen_splitmix64_at.argtypes = [u64, u64]
            lib.psigen_stream_state.restype = u64
            lib.psigen_stream_state.argtypes = [u64, u64]
            lib.psigen_uniform.argtypes = [u64, u64, i64, p]
            lib.psigen_rates_uniform.argtypes = [i64, dbl, dbl, u64, u64, p]
            lib.psigen_rates_lognormal.argtypes = [i64, dbl, dbl, dbl, dbl, u64, u64, p]
            lib.psigen_permutation.argtypes = [i64, u64, u64, p]
            lib.psigen_poisson_uniform.restype = i64
            lib.psigen_poisson_uniform.argtypes = [i64, dbl, u64, p, p]
            lib.psigen_rmat.restype = i64
            lib.psigen_rmat.argtypes = [i32, i64, dbl, dbl, dbl, u64, i32, p, p]
            lib.psigen_chung_lu.restype = i64
            lib.psigen_chung_lu.argtypes = [i64, dbl, i64, u64, p, p]
            lib.psigen_num_threads.restype = i32
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def splitmix64_at(state: int, i: int) -> int:
    """Output ``i`` (0-based) of the SplitMix64 sequence with initial state ``state``."""
    return int(_load().psigen_splitmix64_at(state, i))


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    out = np.empty(n, np.float64)
    _load().psigen_uniform(seed, stream, n, _ptr(out))
    return out


def permutation(n: int, seed: int, stream: int) -> np.ndarray:
    out = np.empty(n, np.int32)
    _load().psigen_permutation(n, seed, stream, _ptr(out))
    return out


def uniform_rates(n: int, lo: float, hi: float, seed: int, stream: int) -> np.ndarray:
    out = np.empty(n, np.float64)
    _load().psigen_rates_uniform(n, lo, hi, seed, stream, _ptr(out))
    return out


def lognormal_rates(n: int, m: float, s: float, lo: float, hi: float, seed: int, stream: int) -> np.ndarray:
    out = np.empty(n, np.float64)
    _load().psigen_rates_lognormal(n, m, s, lo, hi, seed, stream, _ptr(out))
    return out


def poisson_uniform_graph(n: int, mean: float, seed: int):
    lib = _load()
    m = lib.psigen_poisson_uniform(n, mean, seed, None, None)
    f = np.empty(m, np.int32)
    l = np.empty(m, np.int32)
    lib.psigen_poisson_uniform(n, mean, seed, _ptr(f), _ptr(l))
    return f, l


def rmat_graph(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int,
               relabel: bool = True, out=None):
    """R-MAT draws (duplicates kept, self-loops redrawn).  ``out`` may be a pair of
    preallocated int32 arrays (e.g. pinned host memory) of length edge_factor*2^scale."""
    m = edge_factor << scale
    if out is None:
        f = np.empty(m, np.int32)
        l = np.empty(m, np.int32)
    else:
        f, l = out
        assert f.dtype == np.int32 and l.dtype == np.int32 and f.size >= m and l.size >= m
    got = _load().psigen_rmat(scale, edge_factor, a, b, c, seed, 1 if relabel else 0, _ptr(f), _ptr(l))
    if got != m:
        raise RuntimeError("psigen_rmat failed")
    return f[:m], l[:m]


def chung_lu_graph(n: int, gamma: float, draws: int, seed: int):
    f = np.empty(draws, np.int32)
    l = np.empty(draws, np.int32)
    got = _load().psigen_chung_lu(n, gamma, draws, seed, _ptr(f), _ptr(l))
    if got != draws:
        raise RuntimeError("psigen_chung_lu failed")
    return f, l


def num_threads() -> int:
    return int(_load().psigen_num_threads())


# --------------------------------------------------------------------------- workloads
#
# The three single-graph workloads of the evaluation (sizes, degree law and rate law);
# they stand in for the paper's Konect datasets (Table II), which are not available.

RMAT_ABC = (0.57, 0.19, 0.19)


def workload(name: str, seed: int = 0, scale: int | None = None):
    """Return a dict with n, follower, leader, lam, mu and the solve settings.

    * ``poisson1000``: N=1000, k~Poisson(10) leaders uniform without replacement,
      lambda, mu ~ U(0.1, 1.0); FP64, absolute s-tolerance 1e-12.
    * ``chunglu``: Chung-Lu N=2^20 (or 2^scale), 2e7 draws (scaled as 19.07 per user),
      exponent 2.1, lambda, mu ~ LogNormal(0,1) clipped to [1e-3, 1e3]; eps 1e-8.
    * ``rmat``: R-MAT scale 25 (or ``scale``), edge factor 16, (a,b,c)=(.57,.19,.19),
      random relabel, lambda, mu ~ LogNormal(0,1.5) clipped to [1e-3, 1e3]; eps 1e-8.
    """
    if name == "poisson1000":
        n = 1000 if scale is None else int(scale)
        f, l = poisson_uniform_graph(n, 10.0, seed)
        lam = uniform_rates(n, 0.1, 1.0, seed, STREAM_LAMBDA)
        mu = uniform_rates(n, 0.1, 1.0, seed, STREAM_MU)
        return dict(name=name, n=n, follower=f, leader=l, lam=lam, mu=mu, eps=1e-12,
                    precision="fp64", tol_mode="s_abs")
    if name == "chunglu":
        sc = 20 if scale is None else int(scale)
        n = 1 << sc
        draws = int(round(20_000_000 * n / (1 << 20)))
        f, l = chung_lu_graph(n, 2.1, draws, seed)
        lam = lognormal_rates(n, 0.0, 1.0, 1e-3, 1e3, seed, STREAM_LAMBDA)
        mu = lognormal_rates(n, 0.0, 1.0, 1e-3, 1e3, seed, STREAM_MU)
        return dict(name=name, n=n, follower=f, leader=l, lam=lam, mu=mu, eps=1e-8,
                    precision="fp32_refine", tol_mode="psi")
    if name == "rmat":
        sc = 25 if scale is None else int(scale)
        n = 1 << sc
        f, l = rmat_graph(sc, 16, *RMAT_ABC, seed, relabel=True)
        lam = lognormal_rates(n, 0.0, 1.5, 1e-3, 1e3, seed, STREAM_LAMBDA)
        mu = lognormal_rates(n, 0.0, 1.5, 1e-3, 1e3, seed, STREAM_MU)
        return dict(name=name, n=n, follower=f, leader=l, lam=lam, mu=mu, eps=1e-8,
                    precision="fp32_refine", tol_mode="psi")
    raise ValueError(f"unknown workload {name!r}")


def multi_workload(G: int, seed: int = 0, n_lo: int = 1000, n_hi: int = 100_000, mean_degree: float = 12.0,
                   gamma: float = 2.1):
    """G independent Chung-Lu graphs: N_q ~ U{n_lo..n_hi}, round(mean_degree * N_q) draws
    with exponent ``gamma`` (duplicates kept), lambda, mu ~ LogNormal(0, 1) clipped to
    [1e-3, 1e3].  Graph q uses the seed ``seed * 65536 + q``.  Edge lists (ids local to each
    graph) and rates are concatenated graph by graph."""
    u = uniform(seed, STREAM_SIZES, G)
    n_g = np.minimum(n_lo + np.floor(u * (n_hi - n_lo + 1)).astype(np.int64), n_hi)
    fs, ls, lams, mus, m_g = [], [], [], [], []
    for q in range(G):
        n = int(n_g[q])
        sq = seed * 65536 + q
        f, l = chung_lu_graph(n, gamma, int(round(mean_degree * n)), sq)
        fs.append(f)
        ls.append(l)
        m_g.append(len(f))
        lams.append(lognormal_rates(n, 0.0, 1.0, 1e-3, 1e3, sq, STREAM_LAMBDA))
        mus.append(lognormal_rates(n, 0.0, 1.0, 1e-3, 1e3, sq, STREAM_MU))
    return dict(name="multi", G=G, n_g=n_g, m_g=np.asarray(m_g, np.int64),
                follower=np.concatenate(fs).astype(np.int32), leader=np.concatenate(ls).astype(np.int32),
                lam=np.concatenate(lams), mu=np.concatenate(mus), eps=1e-8, tol_mode="psi")
