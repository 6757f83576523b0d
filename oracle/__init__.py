"""FP64 CPU oracle of the paper's definitions -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
library path never does, and nothing here imports the library.

The arithmetic lives in ``pastila_oracle.c`` (plain C, FP64, OpenMP over
independent segments or cells); this module compiles it with gcc on first use
and marshals arguments through ctypes.  ``select_length`` composes the C
functions in the order Section 4.2 gives (profiles per m, greedy snippets,
eq. 18), with no arithmetic of its own beyond an argmax.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pastila_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.ora_window_stats.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int, _f64p, _f64p, _i32p]
        lib.ora_zdist.argtypes = [_f64p, _f64p, ctypes.c_int]
        lib.ora_zdist.restype = ctypes.c_double
        lib.ora_mpdist_pair.argtypes = [_f64p, _f64p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.ora_mpdist_pair.restype = ctypes.c_double
        lib.ora_profile_cells.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, _i32p, _i64p, ctypes.c_int64, _f64p]
        lib.ora_profiles_psf.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, _i32p, ctypes.c_int, _f64p]
        lib.ora_profiles_psf_range.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, _i32p, ctypes.c_int, ctypes.c_int64,
                                               ctypes.c_int64, _f64p]
        lib.ora_greedy.argtypes = [_f64p, ctypes.c_int, ctypes.c_int64, ctypes.c_int, _i32p, _f64p]
        lib.ora_neighbors.argtypes = [_f64p, ctypes.c_int64, _i32p, ctypes.c_int, _i32p, _f64p,
                                      _i32p]
        lib.ora_criterion.argtypes = [_f64p, ctypes.c_int, ctypes.c_int64, _i32p, ctypes.c_int]
        lib.ora_criterion.restype = ctypes.c_double
        _lib = lib
    return _lib


def _p64(a):
    return a.ctypes.data_as(_f64p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def set_threads(n: int) -> None:
    """Thread count of the OpenMP loops (segments or cells)."""
    os.environ["OMP_NUM_THREADS"] = str(int(n))


def window_stats(T, ell):
    T = _f64(T)
    C = T.shape[0] - ell + 1
    mu, sig, flat = np.empty(C), np.empty(C), np.empty(C, dtype=np.int32)
    _load().ora_window_stats(_p64(T), T.shape[0], ell, _p64(mu), _p64(sig),
                             flat.ctypes.data_as(_i32p))
    return mu, sig, flat.astype(bool)


def zdist(x, y):
    x, y = _f64(x), _f64(y)
    assert x.shape == y.shape
    return _load().ora_zdist(_p64(x), _p64(y), x.shape[0])


def mpdist(A, B, ell, k):
    """MPdist of two equal-length series (pair definition)."""
    A, B = _f64(A), _f64(B)
    assert A.shape == B.shape
    return _load().ora_mpdist_pair(_p64(A), _p64(B), A.shape[0], ell, k)


def profile_cells(T, m, ell, k, segs, pos):
    """D_s(p) for the listed (segment, position) pairs (pair definition)."""
    T = _f64(T)
    segs = _i32(segs)
    pos = np.ascontiguousarray(pos, dtype=np.int64)
    out = np.empty(segs.shape[0])
    _load().ora_profile_cells(_p64(T), T.shape[0], m, ell, k, segs.ctypes.data_as(_i32p),
                              pos.ctypes.data_as(_i64p), segs.shape[0], _p64(out))
    return out


def profiles(T, m, ell, k, segs=None):
    """Full profiles of the listed segments (all of them by default), S' x P,
    by the PSF steps (eqs. 9-13)."""
    T = _f64(T)
    n = T.shape[0]
    S = n // m
    segs = np.arange(S, dtype=np.int32) if segs is None else _i32(segs)
    P = n - m + 1
    D = np.empty((segs.shape[0], P))
    _load().ora_profiles_psf(_p64(T), n, m, ell, k, segs.ctypes.data_as(_i32p), segs.shape[0],
                             _p64(D))
    return D


def profiles_range(T, m, ell, k, segs, p_lo, p_hi):
    """Profiles of the listed segments at positions p_lo .. p_hi-1 (PSF steps)."""
    T = _f64(T)
    segs = _i32(segs)
    D = np.empty((segs.shape[0], p_hi - p_lo))
    _load().ora_profiles_psf_range(_p64(T), T.shape[0], m, ell, k, segs.ctypes.data_as(_i32p),
                                   segs.shape[0], p_lo, p_hi, _p64(D))
    return D


def greedy(D, K):
    D = _f64(D)
    S, P = D.shape
    chosen = np.empty(K, dtype=np.int32)
    area = np.empty(K)
    _load().ora_greedy(_p64(D), S, P, K, chosen.ctypes.data_as(_i32p), _p64(area))
    return chosen, area


def neighbors(D, chosen):
    D = _f64(D)
    chosen = _i32(chosen)
    S, P = D.shape
    K = chosen.shape[0]
    labels = np.empty(P, dtype=np.int32)
    frac = np.empty(K)
    order = np.empty(K, dtype=np.int32)
    _load().ora_neighbors(_p64(D), P, chosen.ctypes.data_as(_i32p), K,
                          labels.ctypes.data_as(_i32p), _p64(frac), order.ctypes.data_as(_i32p))
    return labels, frac, order


def criterion(D, chosen):
    D = _f64(D)
    chosen = _i32(chosen)
    S, P = D.shape
    return _load().ora_criterion(_p64(D), S, P, chosen.ctypes.data_as(_i32p), chosen.shape[0])


def snippets(T, m, ell, k, K, D=None):
    """Snippets of one length m: (chosen in greedy order, area_after, labels,
    frac per chosen, eq. 8 order, D)."""
    if D is None:
        D = profiles(T, m, ell, k)
    chosen, area = greedy(D, K)
    labels, frac, order = neighbors(D, chosen)
    return chosen, area, labels, frac, order, D


def select_length(T, ms, K, ell_of, k_of):
    """Section 4.2 end to end on the CPU: eq. 18 for every m of the sweep, then
    the argmax (smallest m on ties).  Returns (m_best, crit per m, {m: chosen})."""
    crit = []
    chosen_by_m = {}
    for m in ms:
        D = profiles(T, m, ell_of(m), k_of(m))
        chosen, _ = greedy(D, K)
        chosen_by_m[m] = chosen
        crit.append(criterion(D, chosen))
    crit = np.asarray(crit)
    top = crit.max()
    m_best = min(m for m, c in zip(ms, crit) if c == top)  # smallest m on ties
    return m_best, crit, chosen_by_m
