"""Multi-rank host logic of the benchmark on CPU ranks (gloo, two
processes): the independent units (codes) are split among ranks exactly
once, and job times and counts combine as the slowest rank and the sum."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    bench.dist_init(world, 0, backend="gloo")
    mine = list(bench.shard(512, rank, world))
    slowest = bench.max_over_ranks(10.0 + rank, world)
    total = bench.sum_over_ranks(len(mine), world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    out.put((rank, mine, slowest, total, gathered))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_shard_and_reduce_on_cpu_ranks(world):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    results = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mine, slowest, total, gathered in results:
        assert slowest == 10.0 + world - 1
        assert total == 512
        flat = [i for part in gathered for i in part]
        assert sorted(flat) == list(range(512))  # every code exactly once
        assert mine == gathered[rank] and mine == sorted(mine)


def test_shard_single_rank():
    import bench

    assert list(bench.shard(7, 0, 1)) == list(range(7))
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert [len(bench.shard(10, r, 4)) for r in range(4)] == [3, 3, 2, 2]


# ------------------------------------------- one search split over ranks ----
#
# paper_2603_29942_gb300.shard splits every pass of one search over the ranks
# and exchanges the minimum packed key before each termination test.  On CPU
# ranks (gloo) the slices are searched by the tests' own enumeration of a
# pass's codewords (all g-subsets of rows of Gamma_j, lexicographic, the
# first coefficient 1, the others in lexicographic order): a key is
# (weight, pass, index in that order).  The sharded result must equal the
# one-rank result field by field and the oracle's d, L, U and counts.

def _split_codes():
    import numpy as np

    from paper_2603_29942_gb300 import inputs

    rng = np.random.default_rng(21)
    out = []
    for p, n, k in [(3, 14, 6), (5, 12, 5), (7, 11, 4), (3, 16, 7), (7, 12, 5)]:
        A = rng.integers(0, p, size=(k, n - k), dtype=np.uint8)
        out.append(inputs.systematic(p, n, k, A))
    return out


def _cpu_slices(B, prep, code):
    """search_slice over the tests' own enumeration of each pass."""
    import itertools

    import numpy as np

    sched = B.fpcode_prepared_schedule(prep)
    cache = {}

    def words(P):
        if P not in cache:
            g, j = sched[P]["g"], sched[P]["j"]
            gam, _piv = B.fpcode_prepared_gamma(prep, j)
            gam = np.asarray(gam, dtype=np.int64)
            ws = []
            for T in itertools.combinations(range(code.k), g):
                for rest in itertools.product(range(1, code.p), repeat=g - 1):
                    c = np.array((1,) + rest, dtype=np.int64)
                    ws.append(int(np.count_nonzero((c @ gam[list(T)]) % code.p)))
            cache[P] = np.array(ws, dtype=np.int64)
        return cache[P]

    def search_slice(P, lo, hi, u):
        w = words(P)[lo:hi]
        if u:
            keep = np.nonzero(w <= u)[0]
        else:
            keep = np.arange(len(w))
        if not len(keep):
            return (1 << 64) - 1, hi - lo
        i = int(keep[np.argmin(w[keep])])
        return (int(w[i]) << 56) | (P << 48) | (lo + i), hi - lo

    for P, s in enumerate(sched):
        s["ntasks"] = s["size"]  # the units of a pass: its codewords in the tests' order
    return sched, search_slice


def _split_one(code, rank, world, mn, sm):
    from paper_2603_29942_gb300 import _binding as B
    from paper_2603_29942_gb300 import shard

    prep = B.fpcode_prepare(code.p, code.n, code.k, code.G, B.fpcode_opts_default(defer=0))
    sched, search_slice = _cpu_slices(B, prep, code)
    r = shard.split_search(sched, n=code.n, k=code.k, per_round_check=False,
                           complete=B.fpcode_prepared_shape(prep)[3], rank=rank, world=world,
                           search_slice=search_slice, min_over_ranks=mn, sum_over_ranks=sm)
    return (r.status, r.d, r.L, r.U, r.npasses, r.counts, r.best_key, r.evaluated)


def _split_rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2603_29942_gb300 import shard

    mn, sm = shard.torch_reducers()
    res = [_split_one(c, rank, world, mn, sm) for c in _split_codes()]
    out.put((rank, res))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_search_over_cpu_ranks(world):
    """Every rank reaches the same stop pass, d, L, U, counts and best key,
    equal to one rank's search, and d, L, U and the counts equal the oracle's
    (Alg. 6 on the same schedule)."""
    import oracle

    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    results = dict(out.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    one = [_split_one(c, 0, 1, lambda x: x, lambda x: x) for c in _split_codes()]
    for r in range(world):
        assert results[r] == one
    for code, (status, d, L, U, npasses, counts, key, ev) in zip(_split_codes(), one):
        orc = oracle.bz(code, threads=2, defer=0)
        assert status == 0 and d == orc.d and (L, U) == (orc.L, orc.U)
        assert counts == list(orc.counts) and ev == sum(counts)
        assert key >> 56 == d


def test_rank_ranges_tile_a_pass():
    """The units of a pass are split into contiguous, ordered ranges that
    cover every unit once, for any number of ranks."""
    from paper_2603_29942_gb300 import shard

    for n in (0, 1, 5, 17, 1000):
        for world in (1, 2, 3, 8):
            pos = 0
            for r in range(world):
                lo, hi = shard.rank_range(n, r, world)
                assert lo == pos and hi >= lo
                pos = hi
            assert pos == n
