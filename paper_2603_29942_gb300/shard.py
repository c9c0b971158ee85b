"""One certified search split over several GPUs, one process per GPU.

The paper runs its Brouwer-Zimmermann search on several CPU cores by
splitting the work of each level among them (Sec. 5.2, Table 4).  Here the
unit of work is a task of the device plan: every rank prepares and uploads
the same code (the same GPU type gives every rank the same plan), and for
each pass of the schedule (Alg. 6), in order,

  1. each rank searches its own contiguous range of the pass's tasks on its
     GPU (fpcode_prepared_pass_slice), starting from the best weight the
     ranks have found so far;
  2. the ranks exchange one 8-byte value: the minimum of their packed keys
     (an allreduce; keys order by weight, then pass, then position), and
     the sum of the codewords they evaluated;
  3. every rank applies the same termination test, L_after(pass) >= U, to
     the same reduced values, so all ranks stop after the same pass.

The result -- d, L, U, the per-level counts and the best key (hence the
witness) -- is the one sequential search of Alg. 6 gives: each pass is
enumerated completely before its test, the test of a pass sees the least
weight of the passes up to it, and among equal weights the least key wins
on every rank count.  Nothing here moves data between GPUs but the
per-pass allreduce; the collectives are passed in (NCCL on GPUs, gloo in the
tests on CPU ranks), and this module holds no arithmetic of the search.
"""
from __future__ import annotations

from dataclasses import dataclass, field

NO_KEY = (1 << 64) - 1
_KEY_WEIGHT, _KEY_PASS = 56, 48
OK, EBUDGET = 0, 4


def key_weight(key: int) -> int:
    """Weight field of a packed key."""
    return key >> _KEY_WEIGHT


def with_pass(key: int, pass_index: int) -> int:
    """The key with its pass field set (a slice's keys carry pass 0)."""
    if key == NO_KEY:
        return key
    return (key & ~(0xFF << _KEY_PASS)) | (pass_index << _KEY_PASS)


def rank_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """The contiguous part [lo, hi) of n tasks that rank `rank` of `world`
    takes: n split evenly, the first n % world ranks one more."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


@dataclass
class SplitResult:
    status: int
    d: int
    L: int
    U: int
    npasses: int
    counts: list[int]
    best_key: int
    evaluated: int
    per_pass_keys: list[int] = field(default_factory=list)


def split_search(schedule: list[dict], *, n: int, k: int, per_round_check: bool, complete: bool, rank: int,
                 world: int, search_slice, min_over_ranks, sum_over_ranks, L0: int = 0) -> SplitResult:
    """Alg. 6 with every pass split over `world` ranks.

    schedule: the passes in order, each with g, L_after, round_end, size and
      ntasks (the units a pass is split into; the same on every rank).
    search_slice(pass, lo, hi, u): this rank's best key (pass field set to
      `pass`) and codewords evaluated over units [lo, hi) of the pass, with u
      (0: none) the best weight found so far as the bound.
    min_over_ranks / sum_over_ranks: the exchange (an allreduce of one value).
    """
    best = NO_KEY
    counts = [0] * (k + 1)
    evaluated = 0
    keys = []
    L = L0
    for P, ps in enumerate(schedule):
        lo, hi = rank_range(int(ps["ntasks"]), rank, world)
        u = key_weight(best) if best != NO_KEY else 0
        key, ev = search_slice(P, lo, hi, u) if hi > lo else (NO_KEY, 0)
        key = int(min_over_ranks(key))
        ev = int(sum_over_ranks(ev))
        keys.append(key)
        best = min(best, key)
        evaluated += ev
        counts[ps["g"]] += int(ps["size"])
        L = ps["L_after"]
        useq = key_weight(best) if best != NO_KEY else n - k + 2
        check = (not per_round_check) or bool(ps["round_end"])
        certified = check and ps["L_after"] >= useq
        if certified or P + 1 == len(schedule):
            status = OK if (certified or complete) else EBUDGET
            U = min(key_weight(best), n - k + 1) if best != NO_KEY else n - k + 1
            return SplitResult(status, U if status == OK else -1, L, U, P + 1, counts, best, evaluated, keys)
    U = n - k + 1
    return SplitResult(EBUDGET, -1, L, U, 0, counts, best, evaluated, keys)


class GpuSlices:
    """search_slice on this process's GPU: tasks [lo, hi) of one pass of an
    uploaded code, searched alone (fpcode_prepared_pass_slice).  Each slice
    is prepared and uploaded once and kept: later searches of the split only
    set its first bound (fpcode_prepared_set_bound) and launch it."""

    def __init__(self, B, prep, stream=None):
        self.B = B
        self.prep = prep
        self.stream = stream
        self.slices = {}

    def __call__(self, pass_index: int, lo: int, hi: int, u: int):
        s = self.slices.get((pass_index, lo, hi))
        if s is None:
            s = self.B.fpcode_prepared_pass_slice(self.prep, pass_index, lo, hi, u)
            self.B.fpcode_prepared_upload(s, self.stream)
            self.slices[(pass_index, lo, hi)] = s
        else:
            self.B.fpcode_prepared_set_bound(s, u)
        self.B.fpcode_search_enqueue(s, self.stream)
        r = self.B.fpcode_search_finish(s, self.stream, want_witness=False)
        return with_pass(r.best_key, pass_index), r.enumerated


def torch_reducers(device=None):
    """min / sum of one integer over the ranks of torch.distributed (the
    default group).  Keys are unsigned 64-bit: they are shifted by 2^63 into
    the signed range, which keeps their order."""
    import torch
    import torch.distributed as dist

    def red(x: int, op, shift: bool) -> int:
        v = (x - (1 << 63)) if shift else x
        t = torch.tensor([v], dtype=torch.int64, device=device)
        dist.all_reduce(t, op=op)
        v = int(t.item())
        return (v + (1 << 63)) if shift else v

    return (lambda x: red(x, dist.ReduceOp.MIN, True)), (lambda x: red(x, dist.ReduceOp.SUM, False))


def min_distance_split(B, code, rank: int, world: int, stream=None, opts=None, device=None) -> SplitResult:
    """The certified distance of `code`, its search split over the ranks of
    torch.distributed (one GPU each).  Returns the same result on every
    rank; the witness is B.fpcode_prepared_codeword(prep, result.best_key)."""
    prep = B.fpcode_prepare(code.p, code.n, code.k, code.G, opts)
    B.fpcode_prepared_upload(prep, stream)
    schedule = B.fpcode_prepared_schedule(prep)
    mn, sm = torch_reducers(device)
    o = opts if opts is not None else B.fpcode_opts_default()
    complete = B.fpcode_prepared_shape(prep)[3]
    res = split_search(schedule, n=code.n, k=code.k, per_round_check=bool(o.per_round_check), complete=complete,
                       rank=rank, world=world, search_slice=GpuSlices(B, prep, stream), min_over_ranks=mn,
                       sum_over_ranks=sm)
    res.prep = prep
    return res
