"""The oracle: plain, slow, obviously correct CPU reference for the percolation hot path.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It shares no code with the
CUDA library (``paper_2607_18991_b300``) and neither side imports the other.

Contents and the passages they follow:

* ``zone_offsets`` / ``mask_offsets`` / ``mask_z_zeta`` -- coordination zones, eq. (z) and
  eq. (zeta), Table I.
* ``philox4x32_10`` / ``site_keys`` / ``rank`` -- the random site-addition order of the
  Newman--Ziff method (Methods, "Computational methods"), keyed by Philox4x32-10 (Salmon et al.,
  SC'11) and ordered by (key, site index).
* ``nz`` -- the sequential Newman--Ziff sweep: n* (first n with a cluster touching x1 = 0 and
  x1 = L-1) and S_max(n) (eq. Pmax).
* ``nstar_span`` -- the same sweep's n* under another spanning rule: both borders of axis a
  (x_{a+1} = 0 and x_{a+1} = L-1, a = 0..4) or of any axis (``SPAN_ANY``), with ten border flags.
* ``bfs`` and ``minimax_nstar`` -- independent brute-force cross-checks (flood fill at fixed n;
  bottleneck-path identity) used only to pin ``nz`` and ``nstar_span``.
* ``nz_periodic`` / ``bfs_periodic`` -- the periodic-boundary variant (offsets wrap modulo L): the
  first n at which a cluster wraps around the torus along one axis, and S_max(n); the sweep keeps
  an unwrapped coordinate per cluster, the flood fill checks it without union-find.
* ``smax_prefix`` -- the same sweep stopped after n_stop sites: S_max(n) for n = 0..n_stop.
* ``binomial_weights`` / ``binomial_convolve`` / ``pmax`` -- S_max(n) -> S_max(p) (Methods,
  "Computational methods") and P_max(p) = S_max(p) / L^5 (eq. Pmax).
* ``oracle.mlp`` -- FP64 numpy forward/backward/Adam of the bracket network.

The C part is compiled on first use with gcc into ``oracle/liboracle.so`` (``build()``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

NEVER = 0xFFFFFFFF
SPAN_ANY = 5  # spanning rule: both borders of some axis
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "perc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/liboracle.so`` (gcc, -O2, no vendor code)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u32, u64, i32, i64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_int64
        P = ctypes.POINTER
        L.orc_zone_offsets.argtypes = [i32, P(ctypes.c_int8)]
        L.orc_zone_offsets.restype = i32
        L.orc_mask_offsets.argtypes = [i32, P(ctypes.c_int8)]
        L.orc_mask_offsets.restype = i32
        L.orc_mask_z_zeta.argtypes = [i32, P(i32), P(ctypes.c_double)]
        L.orc_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
        L.orc_site_key.argtypes = [u64, u32]
        L.orc_site_key.restype = u32
        L.orc_rank.argtypes = [u32, u64, P(u32), P(u32)]
        L.orc_rank.restype = i32
        L.orc_nz.argtypes = [u32, u32, P(u32), P(u32), P(u64), u32, P(i64), P(u32), P(i64)]
        L.orc_nz.restype = i32
        L.orc_bfs.argtypes = [u32, u32, P(u32), u64, P(i32), P(i64)]
        L.orc_bfs.restype = i32
        L.orc_bfs_span.argtypes = [u32, u32, u32, P(u32), u64, P(i32), P(i64)]
        L.orc_bfs_span.restype = i32
        L.orc_minimax_nstar.argtypes = [u32, u32, P(u32)]
        L.orc_minimax_nstar.restype = u32
        L.orc_minimax_nstar_axis.argtypes = [u32, u32, u32, P(u32)]
        L.orc_minimax_nstar_axis.restype = u32
        L.orc_nstar_span.argtypes = [u32, u32, u32, P(u32), P(u32), P(u32)]
        L.orc_nstar_span.restype = i32
        L.orc_nz_periodic.argtypes = [u32, u32, u32, P(u32), P(u32), P(u64), u32, P(i64), P(u32)]
        L.orc_nz_periodic.restype = i32
        L.orc_bfs_periodic.argtypes = [u32, u32, u32, P(u32), u64, P(i32), P(i64)]
        L.orc_bfs_periodic.restype = i32
        L.orc_smax_prefix.argtypes = [u32, u32, P(u32), P(u32), u64, P(i64)]
        L.orc_smax_prefix.restype = i32
        L.orc_binomial_weights.argtypes = [u64, ctypes.c_double, P(ctypes.c_double)]
        L.orc_binomial_weights.restype = i32
        L.orc_binomial_convolve.argtypes = [u64, P(ctypes.c_double), ctypes.c_double]
        L.orc_binomial_convolve.restype = ctypes.c_double
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def zone_offsets(zone: int) -> np.ndarray:
    """Offsets v in {-2..2}^5 with |v|^2 = zone, as an int8 array [z_zone, 5] (eq. z)."""
    n = lib().orc_zone_offsets(zone, None)
    out = np.zeros((n, 5), dtype=np.int8)
    lib().orc_zone_offsets(zone, _ptr(out, ctypes.c_int8))
    return out


def mask_offsets(mask: int) -> np.ndarray:
    """Offsets of the neighborhood that unites the zones whose bits are set in ``mask``."""
    n = lib().orc_mask_offsets(mask, None)
    out = np.zeros((n, 5), dtype=np.int8)
    lib().orc_mask_offsets(mask, _ptr(out, ctypes.c_int8))
    return out


def mask_z_zeta(mask: int) -> tuple[int, float]:
    """(z, zeta) of a neighborhood, eq. (z) and eq. (zeta) with r_i = sqrt(i)."""
    z = ctypes.c_int()
    zeta = ctypes.c_double()
    lib().orc_mask_z_zeta(mask, ctypes.byref(z), ctypes.byref(zeta))
    return z.value, zeta.value


def philox4x32_10(ctr, key) -> tuple[int, int, int, int]:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(o, ctypes.c_uint32))
    return tuple(int(x) for x in o)


def site_key(seed: int, i: int) -> int:
    return int(lib().orc_site_key(seed, i))


def num_sites(L: int) -> int:
    return L ** 5


def rank(L: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """(perm, rank) of one sample: sites sorted ascending by (Philox key, index)."""
    N = num_sites(L)
    perm = np.zeros(N, dtype=np.uint32)
    rk = np.zeros(N, dtype=np.uint32)
    if lib().orc_rank(L, seed, _ptr(perm, ctypes.c_uint32), _ptr(rk, ctypes.c_uint32)) != 0:
        raise ValueError(f"orc_rank failed for L={L}")
    return perm, rk


def nz(L: int, mask: int, perm: np.ndarray, rk: np.ndarray, nq=(), smax_all: bool = False):
    """Newman--Ziff sweep.  Returns (nstar, smax_at[len(nq)] int64, smax_all or None)."""
    nq = np.ascontiguousarray(np.asarray(nq, dtype=np.uint64).reshape(-1))
    smax_at = np.zeros(len(nq), dtype=np.int64)
    nstar = ctypes.c_uint32()
    N = num_sites(L)
    all_arr = np.zeros(N + 1, dtype=np.int64) if smax_all else None
    perm = np.ascontiguousarray(perm, dtype=np.uint32)
    rk = np.ascontiguousarray(rk, dtype=np.uint32)
    rc = lib().orc_nz(L, mask, _ptr(perm, ctypes.c_uint32), _ptr(rk, ctypes.c_uint32),
                      _ptr(nq, ctypes.c_uint64), len(nq), _ptr(smax_at, ctypes.c_int64),
                      ctypes.byref(nstar), _ptr(all_arr, ctypes.c_int64) if smax_all else None)
    if rc != 0:
        raise ValueError(f"orc_nz failed for L={L} mask={mask}")
    return nstar.value, smax_at, all_arr


def smax_prefix(L: int, mask: int, perm: np.ndarray, rk: np.ndarray, n_stop: int) -> np.ndarray:
    """S_max(n) for n = 0..n_stop (int64[n_stop + 1]) from the sweep stopped after n_stop sites."""
    out = np.zeros(n_stop + 1, dtype=np.int64)
    perm = np.ascontiguousarray(perm, dtype=np.uint32)
    rk = np.ascontiguousarray(rk, dtype=np.uint32)
    if lib().orc_smax_prefix(L, mask, _ptr(perm, ctypes.c_uint32), _ptr(rk, ctypes.c_uint32), n_stop,
                             _ptr(out, ctypes.c_int64)) != 0:
        raise ValueError(f"orc_smax_prefix failed for L={L} mask={mask} n_stop={n_stop}")
    return out


def nstar_span(L: int, mask: int, span: int, perm: np.ndarray, rk: np.ndarray) -> int:
    """n* of the sweep under spanning rule ``span``: 0..4 = both borders of axis x_{span+1},
    SPAN_ANY = both borders of some axis."""
    out = ctypes.c_uint32()
    perm = np.ascontiguousarray(perm, dtype=np.uint32)
    rk = np.ascontiguousarray(rk, dtype=np.uint32)
    if lib().orc_nstar_span(L, mask, span, _ptr(perm, ctypes.c_uint32), _ptr(rk, ctypes.c_uint32),
                            ctypes.byref(out)) != 0:
        raise ValueError(f"orc_nstar_span failed for L={L} mask={mask} span={span}")
    return out.value


def nz_periodic(L: int, mask: int, perm: np.ndarray, rk: np.ndarray, nq=(), axis: int = 0):
    """Sweep with periodic boundaries: (first n at which a cluster wraps along axis ``axis``,
    S_max after nq[q] sites as int64[len(nq)])."""
    nq = np.ascontiguousarray(np.asarray(nq, dtype=np.uint64).reshape(-1))
    smax_at = np.zeros(len(nq), dtype=np.int64)
    out = ctypes.c_uint32()
    perm = np.ascontiguousarray(perm, dtype=np.uint32)
    rk = np.ascontiguousarray(rk, dtype=np.uint32)
    if lib().orc_nz_periodic(L, mask, axis, _ptr(perm, ctypes.c_uint32), _ptr(rk, ctypes.c_uint32),
                             _ptr(nq, ctypes.c_uint64), len(nq), _ptr(smax_at, ctypes.c_int64),
                             ctypes.byref(out)) != 0:
        raise ValueError(f"orc_nz_periodic failed for L={L} mask={mask} axis={axis}")
    return out.value, smax_at


def bfs_periodic(L: int, mask: int, rk: np.ndarray, n: int, axis: int = 0) -> tuple[bool, int]:
    """Flood fill of the sites with rank < n on the torus: (some cluster wraps along ``axis``, S_max)."""
    w = ctypes.c_int()
    sm = ctypes.c_int64()
    rk = np.ascontiguousarray(rk, dtype=np.uint32)
    if lib().orc_bfs_periodic(L, mask, axis, _ptr(rk, ctypes.c_uint32), n, ctypes.byref(w),
                              ctypes.byref(sm)) != 0:
        raise ValueError("orc_bfs_periodic failed")
    return bool(w.value), sm.value


def bfs(L: int, mask: int, rk: np.ndarray, n: int, span: int = 0) -> tuple[bool, int]:
    """Flood fill of the sites with rank < n: (some cluster spans under rule ``span``, S_max)."""
    sp = ctypes.c_int()
    sm = ctypes.c_int64()
    rk = np.ascontiguousarray(rk, dtype=np.uint32)
    if lib().orc_bfs_span(L, mask, span, _ptr(rk, ctypes.c_uint32), n, ctypes.byref(sp),
                          ctypes.byref(sm)) != 0:
        raise ValueError("orc_bfs_span failed")
    return bool(sp.value), sm.value


def minimax_nstar(L: int, mask: int, rk: np.ndarray, axis: int = 0) -> int:
    """n* from the bottleneck-path identity between the faces x_{axis+1} = 0 and = L-1
    (Dijkstra with max as path cost)."""
    rk = np.ascontiguousarray(rk, dtype=np.uint32)
    return int(lib().orc_minimax_nstar_axis(L, mask, axis, _ptr(rk, ctypes.c_uint32)))


def binomial_convolve(q_of_n: np.ndarray, p: float) -> float:
    """sum_n C(N,n) p^n (1-p)^(N-n) q(n) for q given at n = 0..N."""
    q = np.ascontiguousarray(q_of_n, dtype=np.float64)
    return float(lib().orc_binomial_convolve(len(q) - 1, _ptr(q, ctypes.c_double), p))


def binomial_weights(N: int, p: float) -> np.ndarray:
    """B(N, n, p) for n = 0..N (float64[N + 1]), built by the ratio recursion and normalised."""
    w = np.zeros(N + 1, dtype=np.float64)
    if lib().orc_binomial_weights(N, p, _ptr(w, ctypes.c_double)) != 0:
        raise ValueError(f"orc_binomial_weights failed for N={N} p={p}")
    return w


def pmax(smax_all: np.ndarray, L: int, p: float) -> float:
    """P_max(p) = S_max(p) / L^5 from S_max(n), n = 0..N (eq. Pmax with the binomial convolution)."""
    N = num_sites(L)
    assert len(smax_all) == N + 1
    return binomial_convolve(np.asarray(smax_all, dtype=np.float64), p) / N


def nstar_batch(L: int, seeds, masks, span: int = 0) -> np.ndarray:
    """n*[len(masks), len(seeds)] by one ranking per seed and one sweep per (mask, seed), under
    spanning rule ``span`` (0 = the x1 axis)."""
    out = np.zeros((len(masks), len(seeds)), dtype=np.uint32)
    for s_i, seed in enumerate(seeds):
        perm, rk = rank(L, int(seed))
        for m_i, m in enumerate(masks):
            out[m_i, s_i] = nz(L, int(m), perm, rk)[0] if span == 0 else nstar_span(L, int(m), span, perm, rk)
    return out
