"""CPU reference oracle for minimum-distance certification over F_p.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path (the
CUDA library in ``paper_2603_29942_gb300``) never imports this package, and
this package imports nothing from the product.

The arithmetic lives in ``bz_oracle.c`` (plain mod-p on byte arrays); this
module compiles it with gcc and marshals arguments through ctypes.

Functions (each cites the passage it follows in its C docstring):
  brute_force(code)      definition of d, Sec. 3 (all p^k messages)
  info_sets(code)        systematic generator matrices on disjoint
                         information sets, Sec. 3.1 (leftmost greedy reading)
  bz(code, ...)          Brouwer-Zimmermann, Sec. 3.1 Alg. 6, with the
                         normalisation of Sec. 4.2 and early termination of
                         Sec. 4.4
  pass_size(p, k, g)     C(k, g) (p-1)^(g-1), codewords of one pass
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bz_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

MAX_N = 256
MAX_K = 64
MAX_M = 256
MAX_PASSES = 1024

OK, EINVAL, ENOMEM, EBUDGET, ETOOBIG = 0, 1, 2, 3, 4


class _Opts(ctypes.Structure):
    _fields_ = [
        ("per_round_check", ctypes.c_int),
        ("defer", ctypes.c_int),
        ("threads", ctypes.c_int),
        ("reserved", ctypes.c_int),
        ("budget", ctypes.c_uint64),
    ]


class _Result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("d", ctypes.c_int),
        ("L", ctypes.c_int),
        ("U", ctypes.c_int),
        ("m", ctypes.c_int),
        ("npasses", ctypes.c_int),
        ("exhausted", ctypes.c_int),
        ("reserved", ctypes.c_int),
        ("evaluated", ctypes.c_uint64),
        ("counts", ctypes.c_uint64 * (MAX_K + 1)),
        ("kj", ctypes.c_int * MAX_M),
        ("pass_g", ctypes.c_int * MAX_PASSES),
        ("pass_j", ctypes.c_int * MAX_PASSES),
        ("pass_best", ctypes.c_int * MAX_PASSES),
        ("pass_L", ctypes.c_int * MAX_PASSES),
    ]


def build(force: bool = False, extra_flags: tuple[str, ...] = (), out: str | None = None) -> str:
    """Compile ``bz_oracle.c`` into a shared library (gcc -O2).  Returns its path."""
    path = out or _LIB_PATH
    if not force and os.path.exists(path) and os.path.getmtime(path) >= os.path.getmtime(_SRC):
        return path
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-shared", "-fPIC", "-pthread", *extra_flags, _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


_lib = None


def _load(path: str | None = None):
    global _lib
    if path is not None:
        lib = ctypes.CDLL(path)
    else:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
    u8p = ctypes.POINTER(ctypes.c_uint8)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.oracle_brute_force.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u8p, ip,
                                       ctypes.POINTER(ctypes.c_uint64), u8p]
    lib.oracle_brute_force.restype = ctypes.c_int
    lib.oracle_info_sets.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u8p, ctypes.c_int, ip, ip,
                                     u8p, ip]
    lib.oracle_info_sets.restype = ctypes.c_int
    lib.oracle_bz.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u8p, ctypes.POINTER(_Opts),
                              ctypes.POINTER(_Result), u8p]
    lib.oracle_bz.restype = ctypes.c_int
    lib.oracle_pass_size.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.oracle_pass_size.restype = ctypes.c_uint64
    if path is None:
        _lib = lib
    return lib


def _u8(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _matrix(code) -> tuple[int, int, int, np.ndarray]:
    G = np.ascontiguousarray(code.G, dtype=np.uint8)
    return int(code.p), int(code.n), int(code.k), G


@dataclass
class BruteForce:
    d: int
    dist: np.ndarray  # dist[w] = number of codewords of weight w (all p^k)
    witness: np.ndarray


def brute_force(code, lib_path: str | None = None) -> BruteForce:
    """Minimum distance by the definition (Sec. 3): every message m, codeword m G."""
    lib = _load(lib_path)
    p, n, k, G = _matrix(code)
    d = ctypes.c_int(0)
    dist = np.zeros(n + 1, dtype=np.uint64)
    wit = np.zeros(n, dtype=np.uint8)
    st = lib.oracle_brute_force(p, n, k, _u8(G), ctypes.byref(d),
                                dist.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _u8(wit))
    if st != OK:
        raise ValueError(f"oracle_brute_force status {st}")
    return BruteForce(d.value, dist, wit)


@dataclass
class InfoSets:
    m: int
    kj: list[int]
    gammas: np.ndarray  # m x k x n
    pivots: np.ndarray  # m x k


def info_sets(code, lib_path: str | None = None) -> InfoSets:
    """Gamma_1..Gamma_m on disjoint information sets (Sec. 3.1; greedy reading)."""
    lib = _load(lib_path)
    p, n, k, G = _matrix(code)
    gam = np.zeros((MAX_M, k, n), dtype=np.uint8)
    piv = np.zeros((MAX_M, k), dtype=np.int32)
    kj = np.zeros(MAX_M, dtype=np.int32)
    m = ctypes.c_int(0)
    ip = ctypes.POINTER(ctypes.c_int)
    st = lib.oracle_info_sets(p, n, k, _u8(G), MAX_M, ctypes.byref(m), kj.ctypes.data_as(ip), _u8(gam),
                              piv.ctypes.data_as(ip))
    if st != OK:
        raise ValueError(f"oracle_info_sets status {st}")
    mm = m.value
    return InfoSets(mm, [int(x) for x in kj[:mm]], gam[:mm].copy(), piv[:mm].copy())


@dataclass
class BZResult:
    status: int
    d: int
    L: int
    U: int
    m: int
    kj: list[int]
    evaluated: int
    counts: list[int]  # counts[g] for g = 0..k
    passes: list[tuple[int, int, int, int]] = field(default_factory=list)  # (g, j, best, L_after)
    exhausted: bool = False
    witness: np.ndarray | None = None


def bz(code, per_round_check: bool = False, defer: bool = True, threads: int = 1, budget: int = 0,
       lib_path: str | None = None) -> BZResult:
    """Brouwer-Zimmermann minimum distance (Sec. 3.1, Alg. 6) on byte arrays mod p."""
    lib = _load(lib_path)
    p, n, k, G = _matrix(code)
    o = _Opts(int(per_round_check), int(defer), int(threads), 0, int(budget))
    r = _Result()
    wit = np.zeros(n, dtype=np.uint8)
    lib.oracle_bz(p, n, k, _u8(G), ctypes.byref(o), ctypes.byref(r), _u8(wit))
    if r.status not in (OK, EBUDGET):
        raise ValueError(f"oracle_bz status {r.status}")
    passes = [(r.pass_g[i], r.pass_j[i], r.pass_best[i], r.pass_L[i]) for i in range(r.npasses)]
    return BZResult(r.status, r.d, r.L, r.U, r.m, [int(x) for x in r.kj[:r.m]], int(r.evaluated),
                    [int(x) for x in r.counts[:k + 1]], passes, bool(r.exhausted), wit)


def pass_size(p: int, k: int, g: int) -> int:
    """C(k, g) (p-1)^(g-1): normalised codewords with exactly g nonzero coefficients."""
    return int(_load().oracle_pass_size(p, k, g))
