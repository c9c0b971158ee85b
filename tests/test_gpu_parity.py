"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bit-exact on d, on the codewords enumerated per level g (counts of the
passes entered), on L and on the schedule; the witness is a nonzero
codeword of weight d (checked against a parity-check matrix computed by the
tests' own linear algebra).  Where several witnesses are correct they are
verified, not compared.
"""
from __future__ import annotations

import itertools
import json
import math
import os

import numpy as np
import pytest

import gf
import oracle
from paper_2603_29942_gb300 import _binding as B
from paper_2603_29942_gb300 import inputs

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    B.lib()


def golden():
    with open(os.path.join(HERE, "golden", "oracle_single_codes.json")) as f:
        return json.load(f)


def check_witness(code, d, w):
    w = [int(x) for x in w]
    assert any(w) and gf.weight(w) == d
    H = gf.null_space(np.asarray(code.G).tolist(), code.p)  # rows span the dual
    for h in H:
        assert sum(a * b for a, b in zip(h, w)) % code.p == 0


def status_of_oracle(st):
    """The oracle's status numbering mapped onto the library's."""
    return {oracle.OK: B.OK, oracle.EBUDGET: B.EBUDGET}[st]


def run(code, **kw):
    pr = B.fpcode_prepare(code.p, code.n, code.k, code.G, B.fpcode_opts_default(**kw))
    return B.fpcode_min_distance_ex(pr), pr


# --------------------------------------------------- bit-sliced ops ----

@pytest.mark.parametrize("p", [3, 5, 7, 11, 13, 31, 127, 251])
def test_bitslice_ops_on_device(p):
    """The device build of every operation equals mod-p arithmetic on all
    p^2 pairs, spread over random lane positions."""
    r = p.bit_length()
    rng = np.random.default_rng(p)
    pairs = [(a, b) for a in range(p) for b in range(p)]
    reps = max(1, 4096 // len(pairs))
    A = np.zeros((len(pairs) * reps, r), dtype=np.uint32)
    Bm = np.zeros_like(A)
    expect = []
    for i in range(len(pairs) * reps):
        lanes = rng.integers(0, p, size=(32, 2))
        lanes[i % 32] = pairs[i % len(pairs)]
        for q in range(32):
            for s in range(r):
                A[i, s] |= np.uint32(((int(lanes[q, 0]) >> s) & 1) << q)
                Bm[i, s] |= np.uint32(((int(lanes[q, 1]) >> s) & 1) << q)
        expect.append(lanes)
    out = B.fpcode_test_bitslice_device(B.OP_ADD, p, A, Bm, r).reshape(-1, r)
    nz = B.fpcode_test_bitslice_device(B.OP_NZ_SUB, p, A, Bm, r)
    for i, lanes in enumerate(expect):
        for q in range(32):
            s = sum(((int(out[i, b]) >> q) & 1) << b for b in range(r))
            assert s == (int(lanes[q, 0]) + int(lanes[q, 1])) % p
            assert ((int(nz[i]) >> q) & 1) == int(lanes[q, 0] != lanes[q, 1])


# ------------------------------------------------- single workloads ----

@pytest.mark.parametrize("pair", [1, 0])
@pytest.mark.parametrize("name", ["f3_n30_k15", "f7_n40_k20", "f3_n80_k40"])
def test_single_code_parity(name, pair):
    """Both leaf forms (pair leaves: the last two rows from the pair table;
    one-row leaves) against the oracle's stored values."""
    code = inputs.single(name)
    g = golden()[name]
    assert code.digest() == g["sha256"]
    for mode, kw in (("default", {}), ("paper_literal", {"per_round_check": 1, "defer": 0})):
        exp = g[mode]
        for mid in (1, 0):
            res, pr = run(code, mid_pass_exit=mid, pair_leaves=pair, **kw)
            assert (B.fpcode_test_pair_mode(pr) > 0) == bool(pair)
            assert res.status == B.OK
            assert (res.d, res.L, res.U, res.m, res.kj) == (exp["d"], exp["L"], exp["U"], exp["m"], exp["kj"])
            assert res.counts == exp["counts"]
            assert res.npasses == len(exp["passes"])
            if mid == 0:  # every pass entered is fully enumerated
                assert res.enumerated == exp["evaluated"]
            else:
                assert res.enumerated <= exp["evaluated"]
            check_witness(code, res.d, res.witness)


@pytest.mark.parametrize("pair", [1, 0])
def test_parity_mode_witness_is_deterministic(pair):
    code = inputs.single("f7_n40_k20")
    ws = []
    for _ in range(3):
        res, _ = run(code, mid_pass_exit=0, pair_leaves=pair)
        ws.append(res.witness.tobytes())
    assert len(set(ws)) == 1


@pytest.mark.parametrize("pl", [1, 3, 64])
def test_task_shape_does_not_change_result(pl):
    code = inputs.single("f3_n80_k40")
    exp = golden()["f3_n80_k40"]["default"]
    res, _ = run(code, prefixes_per_lane=pl, mid_pass_exit=0, ctas_per_sm=1)
    assert (res.d, res.counts, res.enumerated) == (exp["d"], exp["counts"], exp["evaluated"])


def _random_codes(seed, count):
    rng = np.random.default_rng(seed)
    shapes = [(3, 20, 8), (5, 18, 7), (7, 16, 6), (11, 12, 5), (13, 12, 4), (3, 50, 12), (7, 45, 8),
              (3, 90, 20), (5, 100, 10), (3, 140, 12), (3, 24, 24), (7, 9, 1), (3, 40, 39), (17, 10, 4),
              (31, 9, 3), (127, 7, 2), (251, 6, 2)]
    for i in range(count):
        p, n, k = shapes[i % len(shapes)]
        G = rng.integers(0, p, size=(k, n), dtype=np.uint8)
        if i % 4 == 0:
            G[:, rng.integers(0, n)] = 0
        if i % 5 == 0:
            G[:, :k] = np.eye(k, dtype=np.uint8)
        if gf.rank(G.tolist(), p) < k:
            continue
        yield inputs.Code(p, n, k, G)


@pytest.mark.parametrize("p,n,k,budget", [(31, 24, 6, 5 * 10 ** 7), (31, 50, 6, 5 * 10 ** 7), (31, 70, 10, 5 * 10 ** 7),
                                          (127, 30, 5, 5 * 10 ** 7), (127, 80, 4, 5 * 10 ** 7),
                                          (127, 110, 6, 5 * 10 ** 7)])
def test_mersenne_prime_kernels_parity(p, n, k, budget):
    """p = 31 and 127 run their own kernels (the end-around-carry exact add):
    the same status, d, counts, L and U as the oracle, W = 1..4, certified
    and budget-limited searches, and a valid witness."""
    code = inputs.single_code(500 + n, p, n, k)
    r = oracle.bz(code, threads=4, budget=budget)
    res, _ = run(code, budget=budget)
    assert res.status == status_of_oracle(r.status)
    assert res.counts == r.counts and (res.L, res.U) == (r.L, r.U)
    if r.status == oracle.OK:
        assert res.d == r.d
        check_witness(code, res.d, res.witness)


@pytest.mark.parametrize("seed", range(6))
def test_random_codes_parity(seed):
    """Random codes over several primes, word counts W = 1..4, rank-deficient
    last information sets, zero columns, k = 1 and k = n: same d, counts, L,
    schedule as the oracle; a valid witness.  Pair leaves for p = 3, 7 on
    even seeds, one-row leaves on odd ones."""
    for code in _random_codes(1000 + seed, 17):
        r = oracle.bz(code, threads=4, budget=5 * 10 ** 7)
        res, _ = run(code, mid_pass_exit=seed % 2, budget=5 * 10 ** 7, pair_leaves=1 - seed % 2)
        assert res.status == status_of_oracle(r.status), (code.p, code.n, code.k)
        assert res.counts == r.counts
        assert (res.L, res.U) == (r.L, r.U)
        if r.status == oracle.OK:
            assert res.d == r.d
            check_witness(code, res.d, res.witness)


def test_budget_interval():
    code = inputs.single("f7_n40_k20")
    r = oracle.bz(code, budget=100000)
    res, _ = run(code, budget=100000)
    assert res.status == B.EBUDGET == status_of_oracle(r.status)
    assert (res.L, res.U, res.counts) == (r.L, r.U, r.counts)


def test_one_shot_call():
    code = inputs.single("f3_n30_k15")
    d, w = B.fpcode_min_distance(code.p, code.n, code.k, code.G)
    assert d == 6
    check_witness(code, d, w)


def test_batch_equals_alone():
    codes = inputs.batch_codes(48)
    budgets = [2 * 10 ** 6] * len(codes)
    res = B.fpcode_min_distance_batch(codes, budgets=budgets)
    for c, rb in zip(codes, res):
        ra, _ = run(c, budget=2 * 10 ** 6)
        assert (rb.status, rb.d, rb.L, rb.U, rb.counts) == (ra.status, ra.d, ra.L, ra.U, ra.counts)
        if rb.status == B.OK:
            check_witness(c, rb.d, rb.witness)


def test_random_small_codes_against_oracle():
    """A seeded sweep of small random codes (p in {3, 5, 7, 11, 31, 127},
    n <= 34, both leaf forms where they apply, both schedule modes, with
    and without a budget): status, d, L, U and the per-level counts equal
    the oracle's, and every certified search's witness has weight d and
    lies in the code."""
    import random
    rng = random.Random(20261203)
    seen = 0
    for i in range(150):
        p = rng.choice([3, 3, 5, 7, 7, 11, 31, 127])
        n = rng.randint(6, 34)
        k = rng.randint(1, min(n, 14 if p <= 7 else 8))
        unlimited_ok = p == 3 or (p <= 7 and k <= 10)
        budget = rng.choice([0, 10 ** 5, 10 ** 6] if unlimited_ok else [10 ** 5, 10 ** 6])
        prc = rng.choice([0, 1])
        c = inputs.single_code(12000 + i, p, n, k)
        r = oracle.bz(c, budget=budget, per_round_check=bool(prc), threads=1)
        for pair in ((0, 1) if p in (3, 7) and k >= 3 else (0,)):
            g, _ = run(c, budget=budget, per_round_check=prc, pair_leaves=pair)
            case = (i, p, n, k, budget, prc, pair)
            assert (g.status, g.L, g.U, g.counts) == (status_of_oracle(r.status), r.L, r.U, r.counts), case
            if r.status == oracle.OK:
                assert g.d == r.d, case
                check_witness(c, g.d, g.witness)
            seen += 1
    assert seen >= 150


def test_batch_against_oracle_mixed_primes():
    rng = np.random.default_rng(77)
    codes = []
    for i in range(30):
        p = [3, 5, 7, 11, 13][i % 5]
        n = int(rng.integers(12, 40))
        k = int(rng.integers(3, min(n, 14)))
        codes.append(inputs.single_code(500 + i, p, n, k))
    res = B.fpcode_min_distance_batch(codes, budgets=[10 ** 7] * len(codes))
    for c, rb in zip(codes, res):
        r = oracle.bz(c, budget=10 ** 7, threads=4)
        assert (rb.status, rb.counts, rb.L, rb.U) == (status_of_oracle(r.status), r.counts, r.L, r.U)
        if r.status == oracle.OK:
            assert rb.d == r.d
            check_witness(c, rb.d, rb.witness)


@pytest.mark.parametrize("words", [2, 1])
def test_batch512_sample_against_oracle(words):
    """The batched workload at its bench size (512 codes, budget 10^8
    codewords per code): a fixed sample spread over the batch matches the
    oracle run alone at the same budget (status, d, per-level counts, L, U)
    with a valid witness, in one batched launch (batch_words 2) and in one
    launch per kernel variant with pair leaves for the codes that take
    them (batch_words 1)."""
    codes = inputs.batch_codes(512)
    budget = 10 ** 8
    res = B.fpcode_min_distance_batch(codes, opts=B.fpcode_opts_default(batch_words=words),
                                      budgets=[budget] * len(codes))
    for i in range(0, 512, 51):
        c, rb = codes[i], res[i]
        r = oracle.bz(c, budget=budget, threads=os.cpu_count() or 4)
        assert (rb.status, rb.counts, rb.L, rb.U) == (status_of_oracle(r.status), r.counts, r.L, r.U), i
        if r.status == oracle.OK:
            assert rb.d == r.d
            check_witness(c, rb.d, rb.witness)


@pytest.mark.parametrize("words", [2, 4, 1])
def test_batch_mixed_widths_against_oracle(words):
    """Codes of one, two and three words per slice in one batch run in the
    narrow and the wide batched kernels, or one launch per variant with pair
    leaves forced on for p = 3, 7 (batch_words 1); each matches the oracle."""
    shapes = [(3, 70, 5), (3, 40, 6), (3, 30, 6), (7, 75, 4), (5, 100, 4), (7, 50, 8), (5, 36, 7), (3, 98, 6),
              (3, 60, 20), (7, 44, 14), (3, 48, 16)]
    codes = [inputs.single_code(700 + i, p, n, k) for i, (p, n, k) in enumerate(shapes)]
    o = B.fpcode_opts_default(batch_words=words, pair_leaves=1 if words == 1 else 2)
    res = B.fpcode_min_distance_batch(codes, opts=o, budgets=[10 ** 7] * len(codes))
    for c, rb in zip(codes, res):
        r = oracle.bz(c, budget=10 ** 7, threads=4)
        assert (rb.status, rb.counts, rb.L, rb.U) == (status_of_oracle(r.status), r.counts, r.L, r.U)
        if r.status == oracle.OK:
            assert rb.d == r.d
            check_witness(c, rb.d, rb.witness)


def _pass_minimum(gamma, p, g):
    """Least weight over every codeword that combines exactly g rows of
    gamma with nonzero coefficients (brute force, numpy)."""
    k, n = gamma.shape
    coefs = np.array(list(itertools.product(range(1, p), repeat=g)), dtype=np.int64)
    best = n + 1
    for rows in itertools.combinations(range(k), g):
        cw = (coefs @ gamma[list(rows)].astype(np.int64)) % p
        best = min(best, int((cw != 0).sum(axis=1).min()))
    return best


@pytest.mark.parametrize("name", ["f7_n40_k20", "f3_n80_k40", "f3_n30_k15"])
def test_split_search_gpu_slices(name):
    """One search split over ranks (paper_2603_29942_gb300.shard), each rank's
    slice of every pass searched on the GPU (fpcode_prepared_pass_slice): with
    the ranks emulated one after another on this GPU, 2 and 3 ranks give the
    d, L, U, stop pass and per-level counts of the one-launch search, every
    codeword counted once, and a best key whose codeword has weight d and lies
    in the code."""
    from paper_2603_29942_gb300 import shard

    code = inputs.single(name)
    ref, _ = run(code, mid_pass_exit=0)
    prep = B.fpcode_prepare(code.p, code.n, code.k, code.G)
    B.fpcode_prepared_upload(prep)
    sched = B.fpcode_prepared_schedule(prep)
    assert all(s["ntasks"] >= 1 for s in sched)
    gpu = shard.GpuSlices(B, prep)
    for world in (2, 3):
        def search_slice(P, lo, hi, u):
            best, ev = shard.NO_KEY, 0
            for r in range(world):  # the ranks, one after another
                a, b = shard.rank_range(hi - lo, r, world)
                if b > a:
                    key, e = gpu(P, lo + a, lo + b, u)
                    best, ev = min(best, key), ev + e
            return best, ev
        res = shard.split_search(sched, n=code.n, k=code.k, per_round_check=False, complete=True, rank=0, world=1,
                                 search_slice=search_slice, min_over_ranks=lambda x: x, sum_over_ranks=lambda x: x)
        assert (res.status, res.d, res.L, res.U, res.npasses) == (B.OK, ref.d, ref.L, ref.U, ref.npasses)
        assert res.counts == ref.counts and res.evaluated == sum(ref.counts)
        cw, wt = B.fpcode_prepared_codeword(prep, res.best_key)
        assert wt == ref.d
        check_witness(code, ref.d, cw)


def test_batch_autotune_keeps_results_and_caches():
    """The batch autotuner picks settings from its grid by measurement; a second
    call for the same workload class comes from the cache (nothing measured);
    and the batch searched with the tuned settings gives every code the same
    status, d, [L, U] and per-level counts as with the defaults."""
    codes = inputs.batch_codes(64, seed=7)
    budgets = [10 ** 6] * len(codes)
    t = B.fpcode_autotune_batch(codes, budgets=budgets, reps=1)
    assert t["ctas_per_sm"] in (0, 2, 3) and t["min_steps"] in (8, 16, 32, 64, 128) and t["batch_words"] in (2, 4, 1)
    assert t["evaluated"] >= 1 and t["ms"] > 0 and t["ms_default"] > 0 and "k" in t["workload_class"]
    again = B.fpcode_autotune_batch(codes, budgets=budgets, reps=1)
    assert again["evaluated"] == 0
    assert (again["ctas_per_sm"], again["min_steps"], again["batch_words"]) == (
        t["ctas_per_sm"], t["min_steps"], t["batch_words"])
    ref = B.fpcode_min_distance_batch(codes, budgets=budgets, want_witness=False)
    for wide in (2, 4, 1):  # also the other groupings, whichever was chosen
        o = t["opts"]
        o.batch_words = wide
        got = B.fpcode_min_distance_batch(codes, opts=o, budgets=budgets, want_witness=False)
        for r, q in zip(ref, got):
            assert (r.status, r.d, r.L, r.U, r.counts) == (q.status, q.d, q.L, q.U, q.counts)


@pytest.mark.parametrize("name,g", [("f3_n30_k15", 3), ("f7_n40_k20", 3), ("f3_n80_k40", 2)])
def test_single_pass_probe(name, g):
    """One pass alone (termination off): every codeword of the pass is
    evaluated (count = closed-form size), the least weight found equals the
    brute-force minimum over the pass, a seeded bound at that minimum keeps
    it, and a seeded bound below it is returned unchanged with no witness."""
    code = inputs.single(name)
    pr = B.fpcode_prepare(code.p, code.n, code.k, code.G, B.fpcode_opts_default(budget=0))
    passes = B.fpcode_prepared_passes(pr)
    idx = next(i for i, x in enumerate(passes) if x[0] == g and x[1] == 0)
    gamma, _ = B.fpcode_prepared_gamma(pr, 0)
    want = _pass_minimum(gamma, code.p, g)
    for u_init, expect_u, witness in ((0, want, True), (want, want, True), (want - 1, want - 1, False)):
        q = B.fpcode_prepared_single_pass(pr, idx, u_init)
        B.fpcode_prepared_upload(q)
        B.fpcode_search_enqueue(q)
        r = B.fpcode_search_finish(q)
        assert r.status == B.EBUDGET
        assert r.counts[g] == passes[idx][5] == math.comb(code.k, g) * (code.p - 1) ** (g - 1)
        assert sum(r.counts) == passes[idx][5]
        assert r.U == expect_u
        if witness:
            check_witness(code, want, r.witness)


@pytest.mark.parametrize("name", ["f7_n40_k20", "f3_n80_k40"])
def test_checkpoint_resume_equals_one_search(name):
    """A search stopped at a small budget, checkpointed and resumed twice
    with larger budgets ends exactly as one unbounded search: status, d,
    L, U and per-level counts; a valid witness."""
    code = inputs.single(name)
    ref, _ = run(code)
    pr = B.fpcode_prepare(code.p, code.n, code.k, code.G, B.fpcode_opts_default(budget=10 ** 5))
    B.fpcode_prepared_upload(pr)
    B.fpcode_search_enqueue(pr)
    r = B.fpcode_search_finish(pr)
    assert r.status == B.EBUDGET
    ck = B.fpcode_search_checkpoint(pr)
    for budget in (3 * 10 ** 6, 0):
        pr = B.fpcode_prepare(code.p, code.n, code.k, code.G, B.fpcode_opts_default(budget=budget))
        B.fpcode_prepared_upload(pr)
        B.fpcode_search_resume(pr, ck)
        r = B.fpcode_search_finish(pr)
        if r.status == B.EBUDGET:
            ck = B.fpcode_search_checkpoint(pr)
    assert r.status == B.OK
    assert (r.d, r.L, r.U, r.counts, r.m, r.kj) == (ref.d, ref.L, ref.U, ref.counts, ref.m, ref.kj)
    check_witness(code, r.d, r.witness)


@pytest.mark.parametrize("p,sliced", [(3, True), (7, True), (3, False), (7, False), (5, False), (127, False)])
def test_additions_benchmark_kernels(p, sliced):
    """The additions benchmark's kernels give a + reps * b (mod p) on every
    symbol, with ragged vector lengths (not a multiple of 32 or 4)."""
    rng = np.random.default_rng(p + 100 * sliced)
    a = rng.integers(0, p, size=(37, 517), dtype=np.uint8)
    b = rng.integers(0, p, size=(37, 517), dtype=np.uint8)
    for reps in (0, 1, 7, 100):
        out, ms = B.fpcode_bench_additions(p, a, b, reps, sliced)
        want = (a.astype(np.int64) + reps * b.astype(np.int64)) % p
        assert np.array_equal(out, want.astype(np.uint8)), reps
        assert ms >= 0


def test_bounded_wait_reports_timeout():
    """A hand-off wait limit far below a task's duration makes the waiting
    CTAs give up and the kernel return; the host reports ETIMEOUT and the
    context stays usable."""
    code = inputs.single("f3_n80_k40")
    res, _ = run(code, wait_limit_s=1e-7)
    assert res.status in (B.ETIMEOUT, B.OK)
    res2, _ = run(code, timeout_s=1e-6)
    assert res2.status == B.ETIMEOUT
    assert res2.L <= 14
    ok, _ = run(code)
    assert ok.status == B.OK and ok.d == 14


@pytest.mark.parametrize("lookahead", [0, 1])
@pytest.mark.parametrize("name", ["f3_n30_k15", "f7_n40_k20", "f3_n80_k40"])
def test_lookahead_keeps_the_schedule(name, lookahead):
    """Taking tasks of later passes while earlier ones drain leaves d, L,
    the passes entered and their counts exactly as the sequential schedule
    has them."""
    code = inputs.single(name)
    exp = golden()[name]["default"]
    for mid in (0, 1):
        res, _ = run(code, lookahead=lookahead, mid_pass_exit=mid)
        assert res.status == B.OK
        assert (res.d, res.L, res.U, res.counts, res.npasses) == (
            exp["d"], exp["L"], exp["U"], exp["counts"], len(exp["passes"]))
        if mid == 0:
            assert res.enumerated == exp["evaluated"]
        check_witness(code, res.d, res.witness)


@pytest.mark.gpu
@pytest.mark.parametrize("p,n,k", [(3, 80, 40), (7, 40, 20), (3, 150, 30), (7, 90, 12), (3, 20, 3)])
def test_device_pair_table_matches_definition(p, n, k):
    """The pair table the kernels build in shared memory from the staged
    multiples equals, entry by entry, the host's computation of its
    definition (the signature words and slice 0 of B = A[y] + c A[x])."""
    code = inputs.single_code(11 + n, p, n, k)
    pr = B.fpcode_prepare(code.p, code.n, code.k, code.G, B.fpcode_opts_default(pair_leaves=1))
    sigp = B.fpcode_test_pair_mode(pr)
    assert sigp > 0
    m = B.fpcode_prepared_shape(pr)[0]
    W = -(-(n - k) // 32)
    ne = (p - 1) * (k * (k - 1) // 2)
    off0 = (ne * sigp + 3) & ~3
    for j in range(m):
        dev = B.fpcode_test_pair_table_device(pr, j)
        assert len(dev) == off0 + ((ne * W + 3) & ~3)
        for e in range(ne):
            host = B.fpcode_test_pair_entry(pr, j, e)
            assert list(dev[e * sigp:(e + 1) * sigp]) == host[:sigp], (j, e)
            assert list(dev[off0 + e * W:off0 + (e + 1) * W]) == host[sigp:], (j, e)


def test_int_peaks_are_measured():
    """The roofline's denominator comes from fpcode_int_peaks: positive issue
    rates, POPC no faster than LOP3, no unit above one warp instruction per
    SM sub-partition per clock (4 x 32 lanes), and the per-second rates equal
    to lanes per clock x SMs x the measured clock."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    r = B.fpcode_int_peaks()
    for key in ("lop3_per_clk_sm", "popc_per_clk_sm", "iadd_per_clk_sm", "sm_mhz"):
        assert r[key] > 0, key
    assert r["popc_per_clk_sm"] <= r["lop3_per_clk_sm"] * 1.05
    for key in ("lop3_per_clk_sm", "popc_per_clk_sm", "iadd_per_clk_sm"):
        assert r[key] <= 128 * 1.05, key
    for per_clk, per_s in (("lop3_per_clk_sm", "lop3_per_s"), ("popc_per_clk_sm", "popc_per_s")):
        want = r[per_clk] * sms * r["sm_mhz"] * 1e6
        assert abs(r[per_s] - want) <= 0.10 * want, (per_s, r[per_s], want)
