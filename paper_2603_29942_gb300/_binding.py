"""ctypes binding of libfpcode (include/fpcode.h, include/fpcode_testing.h).

Argument marshalling only: every step of the search runs in the CUDA
library.  Functions keep the C names.  Matrices are numpy uint8 arrays;
``stream`` is a cudaStream_t handle as an int (0: default stream), e.g.
``torch.cuda.current_stream().cuda_stream``.  Loading fails loudly if the
compiled library is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

from collections.abc import Sequence

import numpy as np

from . import build as _build

MAX_K = 64
MAX_N = 255
MAX_M = 255

OK, EINVAL, ENOMEM, ECUDA, EBUDGET, ETIMEOUT, EBUSY, ENOTREADY = range(8)
STATUS_NAMES = {OK: "OK", EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", EBUDGET: "EBUDGET",
                ETIMEOUT: "ETIMEOUT", EBUSY: "EBUSY", ENOTREADY: "ENOTREADY"}

OP_ADD, OP_NZ_SUB, OP_NZ_ADD, OP_NEG, OP_MUL2 = range(5)


class fpcode_opts(ctypes.Structure):
    _fields_ = [
        ("per_round_check", ctypes.c_int),
        ("defer", ctypes.c_int),
        ("mid_pass_exit", ctypes.c_int),
        ("ctas_per_sm", ctypes.c_int),
        ("prefixes_per_lane", ctypes.c_int),
        ("lookahead", ctypes.c_int),
        ("budget", ctypes.c_uint64),
        ("timeout_s", ctypes.c_double),
        ("wait_limit_s", ctypes.c_double),
        ("pair_leaves", ctypes.c_int),
        ("min_steps", ctypes.c_int),
        ("task_work", ctypes.c_int),
        ("task_share", ctypes.c_int),
        ("batch_words", ctypes.c_int),
    ]


class fpcode_tuning(ctypes.Structure):
    _fields_ = [
        ("ctas_per_sm", ctypes.c_int),
        ("min_steps", ctypes.c_int),
        ("batch_words", ctypes.c_int),
        ("evaluated", ctypes.c_int),
        ("ms", ctypes.c_double),
        ("ms_default", ctypes.c_double),
        ("workload_class", ctypes.c_char * 96),
    ]


class fpcode_result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("d", ctypes.c_int),
        ("L", ctypes.c_int),
        ("U", ctypes.c_int),
        ("m", ctypes.c_int),
        ("npasses", ctypes.c_int),
        ("launch", ctypes.c_int),
        ("reserved1", ctypes.c_int),
        ("enumerated", ctypes.c_uint64),
        ("counts", ctypes.c_uint64 * (MAX_K + 1)),
        ("kj", ctypes.c_int * MAX_M),
        ("reserved2", ctypes.c_int),
        ("t_prepare_ms", ctypes.c_double),
        ("t_h2d_ms", ctypes.c_double),
        ("t_kernel_ms", ctypes.c_double),
        ("t_d2h_ms", ctypes.c_double),
        ("t_total_ms", ctypes.c_double),
        ("best_key", ctypes.c_uint64),
    ]


class fpcode_desc(ctypes.Structure):
    _fields_ = [
        ("p", ctypes.c_int),
        ("n", ctypes.c_int),
        ("k", ctypes.c_int),
        ("reserved", ctypes.c_int),
        ("G", ctypes.POINTER(ctypes.c_uint8)),
        ("budget", ctypes.c_uint64),
    ]


class fpcode_checkpoint(ctypes.Structure):
    _fields_ = [
        ("p", ctypes.c_int),
        ("n", ctypes.c_int),
        ("k", ctypes.c_int),
        ("passes_done", ctypes.c_int),
        ("best_key", ctypes.c_uint64),
        ("code_hash", ctypes.c_uint64),
    ]


class fpcode_serve_opts(ctypes.Structure):
    _fields_ = [
        ("slots", ctypes.c_int),
        ("ctas_per_sm", ctypes.c_int),
        ("device_bytes", ctypes.c_size_t),
        ("idle_exit_s", ctypes.c_double),
        ("max_words", ctypes.c_int),
        ("reserved", ctypes.c_int),
        ("search", fpcode_opts),
    ]


class fpcode_pass_info(ctypes.Structure):
    _fields_ = [
        ("g", ctypes.c_int),
        ("j", ctypes.c_int),
        ("L_before", ctypes.c_int),
        ("L_after", ctypes.c_int),
        ("round_end", ctypes.c_int),
        ("ntasks", ctypes.c_int),
        ("size", ctypes.c_uint64),
        ("nprefix", ctypes.c_uint64),
    ]


_lib = None
_U8P = ctypes.POINTER(ctypes.c_uint8)
_U32P = ctypes.POINTER(ctypes.c_uint32)
_IP = ctypes.POINTER(ctypes.c_int)
_VP = ctypes.c_void_p


def _declare(lib):
    sig = {
        "fpcode_opts_default": (None, [ctypes.POINTER(fpcode_opts)]),
        "fpcode_last_error": (ctypes.c_char_p, []),
        "fpcode_prepare": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _U8P,
                                          ctypes.POINTER(fpcode_opts), ctypes.POINTER(_VP)]),
        "fpcode_prepared_free": (None, [_VP]),
        "fpcode_prepared_upload": (ctypes.c_int, [_VP, _VP]),
        "fpcode_search_enqueue": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(fpcode_opts)]),
        "fpcode_search_finish": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(fpcode_result), _U8P]),
        "fpcode_min_distance_ex": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(fpcode_opts),
                                                  ctypes.POINTER(fpcode_result), _U8P]),
        "fpcode_min_distance": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _U8P, _VP, _IP, _U8P]),
        "fpcode_min_distance_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _U8P, _VP, _IP,
                                                       _U8P]),
        "fpcode_min_distance_batch": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(fpcode_desc), _VP,
                                                     ctypes.POINTER(fpcode_opts), ctypes.POINTER(fpcode_result),
                                                     _U8P]),
        "fpcode_serve_opts_default": (None, [ctypes.POINTER(fpcode_serve_opts)]),
        "fpcode_serve_create": (ctypes.c_int, [ctypes.POINTER(fpcode_serve_opts), _VP, ctypes.POINTER(_VP)]),
        "fpcode_serve_submit": (ctypes.c_int, [_VP, ctypes.POINTER(fpcode_desc), ctypes.POINTER(ctypes.c_uint64)]),
        "fpcode_serve_poll": (ctypes.c_int, [_VP, ctypes.POINTER(fpcode_result), ctypes.POINTER(ctypes.c_uint64),
                                             _U8P, ctypes.c_int, _IP]),
        "fpcode_serve_drain": (ctypes.c_int, [_VP, ctypes.c_int]),
        "fpcode_serve_launches": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint64)]),
        "fpcode_serve_destroy": (None, [_VP]),
        "fpcode_int_peaks": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double)]),
        "fpcode_test_bitslice_host": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _U32P, _U32P, _U32P]),
        "fpcode_test_bitslice_device": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _U32P, _U32P,
                                                       _U32P]),
        "fpcode_test_rd_unrank": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_int, ctypes.c_int]),
        "fpcode_test_rd_rank": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_int, ctypes.c_int]),
        "fpcode_test_rd_next": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_uint64)]),
        "fpcode_test_prefix_unrank": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int, _IP,
                                                     ctypes.POINTER(ctypes.c_uint64), _IP]),
        "fpcode_test_prefix_walk": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_int, _IP, ctypes.POINTER(ctypes.c_uint64), _IP]),
        "fpcode_prepared_shape": (ctypes.c_int, [_VP, _IP, _IP, _IP, _IP]),
        "fpcode_prepared_gamma": (ctypes.c_int, [_VP, ctypes.c_int, _U8P, _IP]),
        "fpcode_prepared_passes": (ctypes.c_int, [_VP, ctypes.POINTER(fpcode_pass_info), ctypes.c_int]),
        "fpcode_test_prepared_row": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                    ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)]),
        "fpcode_test_task_ranges": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                                   ctypes.c_int]),
        "fpcode_test_pass_times": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
        "fpcode_prepared_bytes": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
        "fpcode_prepared_single_pass": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_VP)]),
        "fpcode_search_checkpoint": (ctypes.c_int, [_VP, ctypes.POINTER(fpcode_checkpoint)]),
        "fpcode_bench_additions": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, _U8P, _U8P, _U8P, _VP,
                                                  ctypes.POINTER(ctypes.c_double)]),
        "fpcode_search_resume": (ctypes.c_int, [_VP, ctypes.POINTER(fpcode_checkpoint), _VP,
                                                ctypes.POINTER(fpcode_opts)]),
        "fpcode_test_pair_mode": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint32)]),
        "fpcode_test_key_coefficients": (ctypes.c_int, [_VP, ctypes.c_uint64, _IP, _IP, _IP]),
        "fpcode_test_pair_entry": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]),
        "fpcode_test_lane_ranges": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                                   ctypes.c_int]),
        "fpcode_test_pair_table_device": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]),
        "fpcode_prepared_pass_slice": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                                      ctypes.POINTER(_VP)]),
        "fpcode_prepared_set_bound": (ctypes.c_int, [_VP, ctypes.c_int]),
        "fpcode_prepared_codeword": (ctypes.c_int, [_VP, ctypes.c_uint64, _U8P, _IP]),
        "fpcode_autotune_batch": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(fpcode_desc), _VP,
                                                 ctypes.POINTER(fpcode_opts), ctypes.c_int,
                                                 ctypes.POINTER(fpcode_tuning)]),
        "fpcode_tuning_apply": (None, [ctypes.POINTER(fpcode_tuning), ctypes.POINTER(fpcode_opts)]),
        "fpcode_test_tune_search": (ctypes.c_int, [ctypes.c_int, _IP, _IP, ctypes.POINTER(ctypes.c_double), _IP, _IP]),
    }
    found = []
    for name, (res, args) in sig.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
        found.append(name)
    return found


# Every entry point the headers declare (checked by the tests).
EXPORTS: list[str] = []


def lib():
    """Load (building first if needed) libfpcode.so."""
    global _lib, EXPORTS
    if _lib is None:
        path = _build.LIB if _build.up_to_date() else _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libfpcode.so is missing; run paper_2603_29942_gb300.build.build()")
        _lib = ctypes.CDLL(path)
        EXPORTS = sorted(_declare(_lib))
    return _lib


def last_error() -> str:
    return (lib().fpcode_last_error() or b"").decode()


class FpcodeError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)} ({last_error()})")
        self.status = status


def _check(status: int, what: str, ok=(OK,)):
    if status not in ok:
        raise FpcodeError(status, what)
    return status


def _stream(stream) -> int | None:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _matrix(G) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(G, dtype=np.uint8))


def fpcode_opts_default(**over) -> fpcode_opts:
    o = fpcode_opts()
    lib().fpcode_opts_default(ctypes.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


@dataclass
class Result:
    """Python view of fpcode_result."""

    status: int
    d: int
    L: int
    U: int
    m: int
    npasses: int
    enumerated: int
    counts: list[int]
    kj: list[int]
    t_prepare_ms: float
    t_kernel_ms: float
    t_total_ms: float
    witness: np.ndarray | None = field(default=None, repr=False)
    launch: int = 0
    best_key: int = (1 << 64) - 1

    @classmethod
    def of(cls, r: fpcode_result, k: int, witness=None) -> "Result":
        return cls(r.status, r.d, r.L, r.U, r.m, r.npasses, int(r.enumerated), [int(x) for x in r.counts[:k + 1]],
                   [int(x) for x in r.kj[:r.m]], r.t_prepare_ms, r.t_kernel_ms, r.t_total_ms, witness, r.launch,
                   int(r.best_key))


class Prepared:
    """Owns an fpcode_prepared handle."""

    def __init__(self, handle: int, p: int, n: int, k: int):
        self.handle = handle
        self.p, self.n, self.k = p, n, k

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.fpcode_prepared_free(self.handle)
            self.handle = None


def fpcode_prepare(p: int, n: int, k: int, G, opts: fpcode_opts | None = None) -> Prepared:
    G = _matrix(G)
    h = _VP()
    _check(lib().fpcode_prepare(p, n, k, G.ctypes.data_as(_U8P), ctypes.byref(opts) if opts else None,
                                ctypes.byref(h)), "fpcode_prepare")
    return Prepared(h.value, p, n, k)


def fpcode_prepared_upload(prep: Prepared, stream=None) -> None:
    _check(lib().fpcode_prepared_upload(prep.handle, _stream(stream)), "fpcode_prepared_upload")


def fpcode_search_enqueue(prep: Prepared, stream=None, opts: fpcode_opts | None = None) -> None:
    _check(lib().fpcode_search_enqueue(prep.handle, _stream(stream), ctypes.byref(opts) if opts else None),
           "fpcode_search_enqueue")


def fpcode_search_finish(prep: Prepared, stream=None, want_witness: bool = True) -> Result:
    r = fpcode_result()
    w = np.zeros(prep.n, dtype=np.uint8)
    _check(lib().fpcode_search_finish(prep.handle, _stream(stream), ctypes.byref(r),
                                      w.ctypes.data_as(_U8P) if want_witness else None),
           "fpcode_search_finish", ok=(OK, EBUDGET, ETIMEOUT))
    return Result.of(r, prep.k, w if (want_witness and r.U <= prep.n) else None)


def fpcode_search_checkpoint(prep: Prepared) -> fpcode_checkpoint:
    """State after a search that stopped at its budget (status EBUDGET)."""
    ck = fpcode_checkpoint()
    _check(lib().fpcode_search_checkpoint(prep.handle, ctypes.byref(ck)), "fpcode_search_checkpoint")
    return ck


def fpcode_search_resume(prep: Prepared, ck: fpcode_checkpoint, stream=None,
                         opts: fpcode_opts | None = None) -> None:
    """Enqueue a search that continues after checkpoint `ck` (pair with
    fpcode_search_finish)."""
    _check(lib().fpcode_search_resume(prep.handle, ctypes.byref(ck), _stream(stream),
                                      ctypes.byref(opts) if opts else None), "fpcode_search_resume")


def fpcode_bench_additions(p: int, a, b, reps: int, sliced: bool, stream=None):
    """Additions benchmark: (a + reps * b mod p, kernel ms) for nvec x nsym
    symbol arrays a, b."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint8))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.uint8))
    if a.shape != b.shape or a.ndim != 2:
        raise ValueError("a and b must be nvec x nsym arrays of the same shape")
    out = np.zeros_like(a)
    ms = ctypes.c_double(0.0)
    _check(lib().fpcode_bench_additions(int(p), int(bool(sliced)), a.shape[0], a.shape[1], int(reps),
                                        a.ctypes.data_as(_U8P), b.ctypes.data_as(_U8P), out.ctypes.data_as(_U8P),
                                        _stream(stream), ctypes.byref(ms)), "fpcode_bench_additions")
    return out, ms.value


def fpcode_min_distance_ex(prep: Prepared, stream=None, opts: fpcode_opts | None = None) -> Result:
    r = fpcode_result()
    w = np.zeros(prep.n, dtype=np.uint8)
    _check(lib().fpcode_min_distance_ex(prep.handle, _stream(stream), ctypes.byref(opts) if opts else None,
                                        ctypes.byref(r), w.ctypes.data_as(_U8P)),
           "fpcode_min_distance_ex", ok=(OK, EBUDGET, ETIMEOUT))
    return Result.of(r, prep.k, w)


def fpcode_min_distance(p: int, n: int, k: int, G, stream=None) -> tuple[int, np.ndarray]:
    """Certified minimum distance and a witness codeword of that weight."""
    G = _matrix(G)
    d = ctypes.c_int(0)
    w = np.zeros(n, dtype=np.uint8)
    _check(lib().fpcode_min_distance(p, n, k, G.ctypes.data_as(_U8P), _stream(stream), ctypes.byref(d),
                                     w.ctypes.data_as(_U8P)), "fpcode_min_distance")
    return d.value, w


def fpcode_min_distance_noalloc(p: int, n: int, k: int, G, stream=None) -> tuple[int, np.ndarray]:
    """fpcode_min_distance without device allocation (fixed in-library scratch)."""
    G = _matrix(G)
    d = ctypes.c_int(0)
    w = np.zeros(n, dtype=np.uint8)
    _check(lib().fpcode_min_distance_noalloc(p, n, k, G.ctypes.data_as(_U8P), _stream(stream), ctypes.byref(d),
                                             w.ctypes.data_as(_U8P)), "fpcode_min_distance_noalloc")
    return d.value, w


_DESC_DT = np.dtype([("p", "<i4"), ("n", "<i4"), ("k", "<i4"), ("reserved", "<i4"), ("G", "<u8"), ("budget", "<u8")])
_RESULT_DT = np.dtype(fpcode_result)


def _results_of(res: np.ndarray, ks, ns, wit) -> list[Result]:
    """Result objects from a structured array of fpcode_result (field by
    field, vectorised, so that a large batch costs little Python)."""
    cols = {f: res[f].tolist() for f in ("status", "d", "L", "U", "m", "npasses", "enumerated", "t_prepare_ms",
                                         "t_kernel_ms", "t_total_ms", "launch", "best_key")}
    counts, kj = res["counts"], res["kj"]
    out = []
    off = 0
    for i, (k, n) in enumerate(zip(ks, ns)):
        w = wit[off:off + n] if wit is not None else None
        off += n
        m = cols["m"][i]
        out.append(Result(cols["status"][i], cols["d"][i], cols["L"][i], cols["U"][i], m, cols["npasses"][i],
                          cols["enumerated"][i], counts[i, :k + 1].tolist(), kj[i, :max(m, 0)].tolist(),
                          cols["t_prepare_ms"][i], cols["t_kernel_ms"][i], cols["t_total_ms"][i], w,
                          cols["launch"][i], int(cols["best_key"][i])))
    return out


class BatchResults(Sequence):
    """Results of a batch call, as a sequence of Result: a view over the
    arrays the call filled (fpcode_result records and the witnesses), whose
    Result objects are built on first access.  Building all of them at once
    cost more than a millisecond per 512 codes, a sixth of a batch's time."""

    def __init__(self, res: np.ndarray, ks, ns, wit):
        self._res, self._ks, self._ns, self._wit = res, list(ks), list(ns), wit
        self._off = [0]
        for n in self._ns:
            self._off.append(self._off[-1] + n)
        self._memo: list[Result | None] = [None] * len(self._ks)

    def __len__(self) -> int:
        return len(self._ks)

    def __getitem__(self, i):
        if isinstance(i, slice):
            return [self[j] for j in range(*i.indices(len(self)))]
        if i < 0:
            i += len(self)
        if not 0 <= i < len(self):
            raise IndexError(i)
        r = self._memo[i]
        if r is None:
            r = self._memo[i] = _result_at(self._res, i, self._ks[i], self._ns[i],
                                           self._wit[self._off[i]:self._off[i + 1]] if self._wit is not None else None)
        return r

    def field(self, name: str) -> np.ndarray:
        """One field of every result at once (e.g. "d", "status", "enumerated")."""
        return self._res[name]


def _result_at(res: np.ndarray, i: int, k: int, n: int, w) -> Result:
    r = res[i]
    m = int(r["m"])
    return Result(int(r["status"]), int(r["d"]), int(r["L"]), int(r["U"]), m, int(r["npasses"]),
                  int(r["enumerated"]), r["counts"][:k + 1].tolist(), r["kj"][:max(m, 0)].tolist(),
                  float(r["t_prepare_ms"]), float(r["t_kernel_ms"]), float(r["t_total_ms"]), w, int(r["launch"]),
                  int(r["best_key"]))


def fpcode_min_distance_batch(codes, stream=None, opts: fpcode_opts | None = None, budgets=None,
                              want_witness: bool = True) -> BatchResults:
    """codes: objects with p, n, k, G (e.g. inputs.Code).  The codes'
    matrices are packed into one buffer and the descriptors and results are
    numpy structured arrays with the C layouts, so the call's Python cost
    stays small next to the search."""
    num = len(codes)
    ps = [int(c.p) for c in codes]
    ns = [int(c.n) for c in codes]
    ks = [int(c.k) for c in codes]
    mats = [np.asarray(c.G, dtype=np.uint8).reshape(-1) for c in codes]
    for G, n, k in zip(mats, ns, ks):
        if G.size != n * k:
            raise ValueError("a generator matrix is not k x n")
    buf = np.concatenate(mats) if num else np.zeros(1, dtype=np.uint8)
    offs = np.zeros(num + 1, dtype=np.uint64)
    np.cumsum(np.asarray([n * k for n, k in zip(ns, ks)], dtype=np.uint64), out=offs[1:])
    descs = np.zeros(max(num, 1), dtype=_DESC_DT)
    descs["p"][:num], descs["n"][:num], descs["k"][:num] = ps, ns, ks
    descs["G"][:num] = np.uint64(buf.ctypes.data) + offs[:-1]
    if budgets is not None:
        descs["budget"][:num] = np.asarray(budgets, dtype=np.uint64)
    res = np.zeros(max(num, 1), dtype=_RESULT_DT)
    wit = np.zeros(max(sum(ns), 1), dtype=np.uint8) if want_witness else None
    _check(lib().fpcode_min_distance_batch(num, ctypes.cast(descs.ctypes.data, ctypes.POINTER(fpcode_desc)),
                                           _stream(stream), ctypes.byref(opts) if opts else None,
                                           ctypes.cast(res.ctypes.data, ctypes.POINTER(fpcode_result)),
                                           wit.ctypes.data_as(_U8P) if want_witness else None),
           "fpcode_min_distance_batch")
    return BatchResults(res[:num], ks, ns, wit)


def _descs(codes, budgets=None):
    """Packed matrices and a descriptor array (the buffer must outlive the call)."""
    num = len(codes)
    mats = [np.asarray(c.G, dtype=np.uint8).reshape(-1) for c in codes]
    buf = np.concatenate(mats) if num else np.zeros(1, dtype=np.uint8)
    offs = np.zeros(num + 1, dtype=np.uint64)
    np.cumsum(np.asarray([int(c.n) * int(c.k) for c in codes], dtype=np.uint64), out=offs[1:])
    descs = np.zeros(max(num, 1), dtype=_DESC_DT)
    descs["p"][:num] = [int(c.p) for c in codes]
    descs["n"][:num] = [int(c.n) for c in codes]
    descs["k"][:num] = [int(c.k) for c in codes]
    descs["G"][:num] = np.uint64(buf.ctypes.data) + offs[:-1]
    if budgets is not None:
        descs["budget"][:num] = np.asarray(budgets, dtype=np.uint64)
    return buf, descs


def fpcode_autotune_batch(codes, stream=None, opts: fpcode_opts | None = None, budgets=None, reps: int = 2) -> dict:
    """Measured choice of the batch launch settings for these codes (cached
    per GPU and workload class); returns the tuning as a dict, and the
    options with it applied under key "opts"."""
    buf, descs = _descs(codes, budgets)
    t = fpcode_tuning()
    _check(lib().fpcode_autotune_batch(len(codes), ctypes.cast(descs.ctypes.data, ctypes.POINTER(fpcode_desc)),
                                       _stream(stream), ctypes.byref(opts) if opts else None, int(reps),
                                       ctypes.byref(t)), "fpcode_autotune_batch")
    del buf
    o = fpcode_opts()
    if opts is not None:
        ctypes.memmove(ctypes.byref(o), ctypes.byref(opts), ctypes.sizeof(o))
    else:
        lib().fpcode_opts_default(ctypes.byref(o))
    lib().fpcode_tuning_apply(ctypes.byref(t), ctypes.byref(o))
    return {"ctas_per_sm": t.ctas_per_sm, "min_steps": t.min_steps, "batch_words": t.batch_words,
            "evaluated": t.evaluated, "ms": t.ms, "ms_default": t.ms_default,
            "workload_class": t.workload_class.decode(), "opts": o}


def fpcode_test_tune_search(sizes, start, cost):
    """The tuner's coordinate search over a synthetic cost table (row-major)."""
    nd = len(sizes)
    sz = (ctypes.c_int * nd)(*sizes)
    st = (ctypes.c_int * nd)(*start)
    c = np.ascontiguousarray(np.asarray(cost, dtype=np.float64).reshape(-1))
    best = (ctypes.c_int * nd)()
    ev = ctypes.c_int(0)
    rc = lib().fpcode_test_tune_search(nd, sz, st, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), best,
                                       ctypes.byref(ev))
    if rc < 0:
        raise FpcodeError(-rc, "fpcode_test_tune_search")
    return [int(x) for x in best], int(ev.value)


def fpcode_int_peaks(stream=None) -> dict:
    r = (ctypes.c_double * 6)()
    _check(lib().fpcode_int_peaks(_stream(stream), r), "fpcode_int_peaks")
    return {"lop3_per_clk_sm": r[0], "popc_per_clk_sm": r[1], "iadd_per_clk_sm": r[2], "lop3_per_s": r[3],
            "popc_per_s": r[4], "sm_mhz": r[5]}


# ----------------------------------------------------------- test hooks ----

def fpcode_test_bitslice_host(op: int, p: int, a, b) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint32)
    b = np.ascontiguousarray(b, dtype=np.uint32)
    out = np.zeros(max(len(a), 1), dtype=np.uint32)
    _check(lib().fpcode_test_bitslice_host(op, p, a.ctypes.data_as(_U32P), b.ctypes.data_as(_U32P),
                                           out.ctypes.data_as(_U32P)), "fpcode_test_bitslice_host")
    return out


def fpcode_test_bitslice_device(op: int, p: int, a: np.ndarray, b: np.ndarray, r: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint32).ravel()
    b = np.ascontiguousarray(b, dtype=np.uint32).ravel()
    count = len(a) // r
    out = np.zeros(len(a), dtype=np.uint32)
    _check(lib().fpcode_test_bitslice_device(op, p, count, a.ctypes.data_as(_U32P), b.ctypes.data_as(_U32P),
                                             out.ctypes.data_as(_U32P)), "fpcode_test_bitslice_device")
    return out if op not in (OP_NZ_SUB, OP_NZ_ADD) else out[:count]


def fpcode_test_rd_unrank(rank: int, n: int, t: int) -> int:
    return int(lib().fpcode_test_rd_unrank(rank, n, t))


def fpcode_test_rd_rank(subset: int, n: int, t: int) -> int:
    return int(lib().fpcode_test_rd_rank(subset, n, t))


def fpcode_test_rd_next(subset: int, n: int, t: int) -> int | None:
    nxt = ctypes.c_uint64(0)
    ok = lib().fpcode_test_rd_next(subset, n, t, ctypes.byref(nxt))
    return int(nxt.value) if ok else None


def _prefix(fn, *args, g):
    m = ctypes.c_int(0)
    Q = ctypes.c_uint64(0)
    coefs = (ctypes.c_int * max(g - 2, 1))()
    _check(fn(*args, ctypes.byref(m), ctypes.byref(Q), coefs), fn.__name__)
    return m.value, int(Q.value), [coefs[i] for i in range(g - 2)]


def fpcode_test_prefix_unrank(I: int, k: int, g: int, p: int):
    return _prefix(lib().fpcode_test_prefix_unrank, I, k, g, p, g=g)


def fpcode_test_prefix_walk(I: int, steps: int, k: int, g: int, p: int):
    return _prefix(lib().fpcode_test_prefix_walk, I, steps, k, g, p, g=g)


def fpcode_prepared_shape(prep: Prepared):
    m = ctypes.c_int(0)
    kj = (ctypes.c_int * MAX_M)()
    npasses = ctypes.c_int(0)
    complete = ctypes.c_int(0)
    _check(lib().fpcode_prepared_shape(prep.handle, ctypes.byref(m), kj, ctypes.byref(npasses),
                                       ctypes.byref(complete)), "fpcode_prepared_shape")
    return m.value, [kj[i] for i in range(m.value)], npasses.value, bool(complete.value)


def fpcode_prepared_gamma(prep: Prepared, j: int):
    gam = np.zeros((prep.k, prep.n), dtype=np.uint8)
    piv = (ctypes.c_int * prep.k)()
    _check(lib().fpcode_prepared_gamma(prep.handle, j, gam.ctypes.data_as(_U8P), piv), "fpcode_prepared_gamma")
    return gam, [piv[i] for i in range(prep.k)]


def fpcode_test_prepared_row(prep: Prepared, j: int, t: int, v: int):
    """(slices, signature words) stored for v * A_j[t]."""
    r = max(1, int(prep.p).bit_length())
    W = max(1, -(-(prep.n - prep.k) // 32))
    sl = (ctypes.c_uint32 * (r * W))()
    sg = (ctypes.c_uint32 * 64)()
    nsig = lib().fpcode_test_prepared_row(prep.handle, j, t, v, sl, sg)
    if nsig < 0:
        raise FpcodeError(nsig, "fpcode_test_prepared_row")
    return [int(x) for x in sl], [int(sg[i]) for i in range(nsig)]


def fpcode_prepared_passes(prep: Prepared):
    arr = (fpcode_pass_info * 256)()
    n = lib().fpcode_prepared_passes(prep.handle, arr, 256)
    return [(arr[i].g, arr[i].j, arr[i].L_before, arr[i].L_after, arr[i].round_end, int(arr[i].size),
             int(arr[i].nprefix)) for i in range(n)]


def fpcode_prepared_single_pass(prep: Prepared, pass_index: int, u_init: int = 0) -> Prepared:
    """Probe: pass `pass_index` of prep's schedule alone, termination off."""
    h = _VP()
    _check(lib().fpcode_prepared_single_pass(prep.handle, int(pass_index), int(u_init), ctypes.byref(h)),
           "fpcode_prepared_single_pass")
    return Prepared(h.value, prep.p, prep.n, prep.k)


def fpcode_prepared_schedule(prep: Prepared) -> list[dict]:
    """The passes of the schedule with their bounds, sizes and (after an
    upload) the tasks of each under the plan."""
    arr = (fpcode_pass_info * 256)()
    n = lib().fpcode_prepared_passes(prep.handle, arr, 256)
    return [{"g": arr[i].g, "j": arr[i].j, "L_before": arr[i].L_before, "L_after": arr[i].L_after,
             "round_end": arr[i].round_end, "ntasks": arr[i].ntasks, "size": int(arr[i].size)} for i in range(n)]


def fpcode_prepared_pass_slice(prep: Prepared, pass_index: int, task_lo: int, task_hi: int, u_init: int) -> Prepared:
    """Tasks [task_lo, task_hi) of one pass of the uploaded prep, alone, with
    the first bound u_init (multi-GPU split of one search)."""
    h = _VP()
    _check(lib().fpcode_prepared_pass_slice(prep.handle, int(pass_index), int(task_lo), int(task_hi), int(u_init),
                                            ctypes.byref(h)), "fpcode_prepared_pass_slice")
    return Prepared(h.value, prep.p, prep.n, prep.k)


def fpcode_prepared_set_bound(slice_prep: Prepared, u_init: int) -> None:
    """The first bound (0: none) of the next searches of a pass slice."""
    _check(lib().fpcode_prepared_set_bound(slice_prep.handle, int(u_init)), "fpcode_prepared_set_bound")


def fpcode_prepared_codeword(prep: Prepared, key: int):
    """(codeword, weight) of a packed key of prep's schedule."""
    cw = np.zeros(prep.n, dtype=np.uint8)
    w = ctypes.c_int(0)
    _check(lib().fpcode_prepared_codeword(prep.handle, ctypes.c_uint64(key), cw.ctypes.data_as(_U8P), ctypes.byref(w)),
           "fpcode_prepared_codeword")
    return cw, int(w.value)


def fpcode_prepared_bytes(prep: Prepared) -> tuple[int, int]:
    h2d = ctypes.c_uint64(0)
    d2h = ctypes.c_uint64(0)
    _check(lib().fpcode_prepared_bytes(prep.handle, ctypes.byref(h2d), ctypes.byref(d2h)), "fpcode_prepared_bytes")
    return int(h2d.value), int(d2h.value)


# --------------------------------------------------------------- serving ----

def fpcode_serve_opts_default(**over) -> fpcode_serve_opts:
    o = fpcode_serve_opts()
    lib().fpcode_serve_opts_default(ctypes.byref(o))
    for k, v in over.items():
        if k == "search":
            o.search = v
        else:
            setattr(o, k, v)
    return o


class Server:
    """Owns an fpcode_server handle (fpcode_serve_*)."""

    def __init__(self, handle: int):
        self.handle = handle
        self.ks: dict[int, int] = {}
        self.bufs: dict[int, tuple] = {}  # poll buffers by capacity, made once

    def poll_buffers(self, cap: int):
        b = self.bufs.get(cap)
        if b is None:
            b = ((fpcode_result * cap)(), (ctypes.c_uint64 * cap)())
            self.bufs[cap] = b
        return b

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.fpcode_serve_destroy(self.handle)
            self.handle = None


def fpcode_serve_create(opts: fpcode_serve_opts | None = None, stream=None) -> Server:
    h = _VP()
    _check(lib().fpcode_serve_create(ctypes.byref(opts) if opts else None, _stream(stream), ctypes.byref(h)),
           "fpcode_serve_create")
    return Server(h.value)


def fpcode_serve_submit(server: Server, code, budget: int = 0) -> int | None:
    """Ticket, or None if the server is busy (no slot or memory free)."""
    G = _matrix(code.G)
    desc = fpcode_desc(int(code.p), int(code.n), int(code.k), 0, G.ctypes.data_as(_U8P), int(budget))
    t = ctypes.c_uint64(0)
    st = lib().fpcode_serve_submit(server.handle, ctypes.byref(desc), ctypes.byref(t))
    if st == EBUSY:
        return None
    _check(st, "fpcode_serve_submit")
    server.ks[int(t.value)] = int(code.k)
    return int(t.value)


def fpcode_serve_poll(server: Server, max_results: int = 256, want_witness: bool = True):
    """List of (ticket, Result) for codes that finished since the last poll."""
    res, tickets = server.poll_buffers(max_results)
    wit = np.zeros(max_results * MAX_N, dtype=np.uint8) if want_witness else None
    n = ctypes.c_int(0)
    _check(lib().fpcode_serve_poll(server.handle, res, tickets, wit.ctypes.data_as(_U8P) if want_witness else None,
                                   max_results, ctypes.byref(n)), "fpcode_serve_poll")
    out = []
    for i in range(n.value):
        t = int(tickets[i])
        k = server.ks.pop(t, MAX_K)
        w = wit[i * MAX_N:(i + 1) * MAX_N].copy() if want_witness else None
        out.append((t, Result.of(res[i], k, w)))
    return out


def fpcode_serve_drain(server: Server, timeout_ms: int = 60000) -> None:
    _check(lib().fpcode_serve_drain(server.handle, timeout_ms), "fpcode_serve_drain")


def fpcode_serve_launches(server: Server) -> int:
    """Kernel launches the server has made so far."""
    n = ctypes.c_uint64(0)
    _check(lib().fpcode_serve_launches(server.handle, ctypes.byref(n)), "fpcode_serve_launches")
    return int(n.value)


def fpcode_serve_destroy(server: Server) -> None:
    if server.handle:
        lib().fpcode_serve_destroy(server.handle)
        server.handle = None


def fpcode_test_task_ranges(prep: Prepared, pass_index: int, ctas: int, fixed_pl: int = 0, min_steps: int = 8):
    cap = 1 << 16
    lo = (ctypes.c_uint64 * cap)()
    hi = (ctypes.c_uint64 * cap)()
    n = lib().fpcode_test_task_ranges(prep.handle, pass_index, ctas, fixed_pl, min_steps, lo, hi, cap)
    if n < 0:
        raise FpcodeError(EINVAL, "fpcode_test_task_ranges")
    return [(int(lo[i]), int(hi[i])) for i in range(min(n, cap))]


def fpcode_test_lane_ranges(prep: Prepared, pass_index: int, ctas: int, fixed_pl: int = 0, min_steps: int = 8):
    """[(lo, hi)] of every lane of every task of a one-row pass, task-major."""
    cap = 1 << 22
    lo = np.zeros(cap, dtype=np.uint64)
    hi = np.zeros(cap, dtype=np.uint64)
    n = lib().fpcode_test_lane_ranges(prep.handle, pass_index, ctas, fixed_pl, min_steps,
                                      lo.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                      hi.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), cap)
    if n < 0:
        raise FpcodeError(EINVAL, "fpcode_test_lane_ranges")
    return lo[:min(n, cap)], hi[:min(n, cap)]


def fpcode_test_pair_mode(prep: Prepared, pass_index: int = -1, J: int = 0):
    """Words per pair-table entry (0: one-row leaves); with a pass and a
    stem J of it, also the number of pair entries the stem is evaluated
    against."""
    e = ctypes.c_uint32(0)
    w = lib().fpcode_test_pair_mode(prep.handle, int(pass_index), int(J), ctypes.byref(e))
    if w < 0:
        raise FpcodeError(-w, "fpcode_test_pair_mode")
    return w if pass_index < 0 else (w, int(e.value))


def fpcode_test_pair_entry(prep: Prepared, j: int, e: int) -> list[int]:
    """The words of pair-table entry e of information set j, computed on
    the host: its signature (pair_sigp words), then slice 0 of B (W words)."""
    sig = (ctypes.c_uint32 * 16)()
    n = lib().fpcode_test_pair_entry(prep.handle, int(j), int(e), sig)
    if n < 0:
        raise FpcodeError(-n, "fpcode_test_pair_entry")
    return [int(sig[i]) for i in range(n)]


def fpcode_test_pair_table_device(prep: Prepared, j: int) -> np.ndarray:
    """The pair table of information set j as the kernels build it in shared
    memory (u32 words: signatures of all entries, padded, then slice 0)."""
    cap = 1 << 16
    out = np.zeros(cap, dtype=np.uint32)
    n = lib().fpcode_test_pair_table_device(prep.handle, int(j), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                            cap)
    if n < 0:
        raise FpcodeError(-n, "fpcode_test_pair_table_device")
    return out[:n].copy()


def fpcode_test_key_coefficients(prep: Prepared, key: int):
    """(g, j, coefficients) of the codeword a packed key stands for, or None."""
    g = ctypes.c_int(0)
    j = ctypes.c_int(0)
    coef = (ctypes.c_int * prep.k)()
    if lib().fpcode_test_key_coefficients(prep.handle, ctypes.c_uint64(key), ctypes.byref(g), ctypes.byref(j), coef):
        return None
    return g.value, j.value, [int(x) for x in coef]


def fpcode_test_pass_times(prep: Prepared, stream=None) -> list[float]:
    """Microseconds from the last search's start to the end of each pass."""
    us = (ctypes.c_double * 256)()
    n = lib().fpcode_test_pass_times(prep.handle, _stream(stream), us, 256)
    if n < 0:
        raise FpcodeError(EINVAL, "fpcode_test_pass_times")
    return [us[i] for i in range(n)]
