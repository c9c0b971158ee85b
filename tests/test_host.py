"""CPU tests of libfpcode's host logic (no GPU needed).

- the library loads and exports every function include/*.h declares;
- bit-sliced F_p operations, exhaustively over all p^2 operand pairs for
  every odd prime p < 256, against plain mod-p arithmetic;
- the paper's worked examples (tests/golden/paper_examples.json);
- revolving-door order and the prefix walk against their definitions;
- information sets and pass schedule against the oracle.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2603_29942_gb300 import _binding as B
from paper_2603_29942_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PRIMES = [p for p in range(3, 256, 2) if all(p % q for q in range(3, int(p ** 0.5) + 1, 2))]


@pytest.fixture(scope="module")
def lib():
    return B.lib()


def r_bits(p):
    return p.bit_length()


def slices(vals, r):
    """Sliced-bit storage (Sec. 2): slice i holds bit i of every symbol."""
    out = np.zeros(r, dtype=np.uint32)
    for q, v in enumerate(vals):
        for i in range(r):
            if (v >> i) & 1:
                out[i] |= np.uint32(1 << q)
    return out


def unslice(words, r, count):
    return [sum(((int(words[i]) >> q) & 1) << i for i in range(r)) for q in range(count)]


def test_exports_match_headers(lib):
    declared = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            declared |= set(re.findall(r"\b(fpcode_[a-z0-9_]+)\s*\(", src))
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"
    assert declared <= set(B.EXPORTS) | {"fpcode_last_error"} | set(B.EXPORTS)


# ------------------------------------------------------- bit-sliced ops ----

def _pairs(p):
    """All p^2 pairs, 32 per word batch."""
    pairs = list(itertools.product(range(p), repeat=2))
    for i in range(0, len(pairs), 32):
        yield pairs[i:i + 32]


@pytest.mark.parametrize("p", PRIMES)
def test_exact_add_exhaustive(p, lib):
    r = r_bits(p)
    for chunk in _pairs(p):
        a = slices([x for x, _ in chunk], r)
        b = slices([y for _, y in chunk], r)
        out = B.fpcode_test_bitslice_host(B.OP_ADD, p, a, b)
        assert unslice(out, r, len(chunk)) == [(x + y) % p for x, y in chunk]
        # padding lanes (beyond the chunk) stay zero
        if len(chunk) < 32:
            assert all((int(w) >> len(chunk)) == 0 for w in out[:r])


@pytest.mark.parametrize("p", PRIMES)
def test_iso_sub_exhaustive(p, lib):
    r = r_bits(p)
    for chunk in _pairs(p):
        a = slices([x for x, _ in chunk], r)
        b = slices([y for _, y in chunk], r)
        m = int(B.fpcode_test_bitslice_host(B.OP_NZ_SUB, p, a, b)[0])
        assert [(m >> q) & 1 for q in range(len(chunk))] == [int((x - y) % p != 0) for x, y in chunk]


@pytest.mark.parametrize("p", [3, 7, 31, 127])
def test_mersenne_ops_exhaustive(p, lib):
    """Isometric addition (Sec. 4.3), negation by complement and doubling by
    slice rotation (Sec. 4.2) for p = 2^r - 1."""
    r = r_bits(p)
    for chunk in _pairs(p):
        a = slices([x for x, _ in chunk], r)
        b = slices([y for _, y in chunk], r)
        m = int(B.fpcode_test_bitslice_host(B.OP_NZ_ADD, p, a, b)[0])
        assert [(m >> q) & 1 for q in range(len(chunk))] == [int((x + y) % p != 0) for x, y in chunk]
        neg = B.fpcode_test_bitslice_host(B.OP_NEG, p, a, b)
        assert unslice(neg, r, len(chunk)) == [(-x) % p for x, _ in chunk]
        dbl = B.fpcode_test_bitslice_host(B.OP_MUL2, p, a, b)
        assert unslice(dbl, r, len(chunk)) == [(2 * x) % p for x, _ in chunk]


# ----------------------------------------------------- worked examples ----

def golden():
    with open(os.path.join(HERE, "golden", "paper_examples.json")) as f:
        return json.load(f)


def test_paper_encodings_and_storage():
    g = golden()
    for key in ("natural_encoding_f3", "natural_encoding_f7"):
        p = g[key]["p"]
        for v, bits in g[key]["table"].items():
            assert [(int(v) >> i) & 1 for i in range(r_bits(p))] == bits
    st = g["sliced_storage"]
    s = slices(st["vector"], 2)
    assert [[(int(s[i]) >> q) & 1 for q in range(3)] for i in range(2)] == st["slices"]


@pytest.mark.parametrize("name", ["example1", "example2", "example3"])
def test_paper_addition_examples(name, lib):
    ex = golden()[name]
    p, r = ex["p"], r_bits(ex["p"])
    a = slices([ex["V"]], r)
    b = slices([ex["W"]], r)
    assert [int(a[i]) & 1 for i in range(r)] == ex["v"]
    out = B.fpcode_test_bitslice_host(B.OP_ADD, p, a, b)
    assert [int(out[i]) & 1 for i in range(r)] == ex["c"]
    assert unslice(out, r, 1) == [ex["sum"]]


def test_paper_shift_and_rewrites(lib):
    g = golden()
    sh = g["shift_multiplication"]
    w = sum(b << i for i, b in enumerate(sh["w"]))
    a = slices([w], 3)
    two = B.fpcode_test_bitslice_host(B.OP_MUL2, 7, a, a)
    four = B.fpcode_test_bitslice_host(B.OP_MUL2, 7, two, two)
    assert [int(two[i]) & 1 for i in range(3)] == sh["times2"]
    assert [int(four[i]) & 1 for i in range(3)] == sh["times4"]
    for key in ("f7_rewrites", "f3_rewrite"):
        p = g[key]["p"]
        for _s1, h, s2, h2 in g[key]["rows"]:
            for v in range(p):
                for wv in range(p):
                    rhs = (v + h2 * wv) % p if s2 == "+" else (v - h2 * wv) % p
                    assert (v + h * wv) % p == rhs


def test_alg3_reading():
    """Alg. 3 as printed (its update s0 = s0 and carry_1) is wrong on 5 of the 9
    pairs of F_3; read as xor it is right on all 9 (natural encoding)."""
    def alg3(a, b, sixth):
        a0, a1, b0, b1 = a & 1, a >> 1, b & 1, b >> 1
        s0 = a0 ^ b0
        c0 = a0 & b0
        s1 = a1 ^ b1 ^ c0
        c1 = a1 & b1
        s0 = sixth(s0, c1)
        t = s0 & s1
        return (s0 ^ t) | ((s1 ^ t) << 1)
    lit = sum(alg3(a, b, lambda x, y: x & y) != (a + b) % 3 for a in range(3) for b in range(3))
    fix = sum(alg3(a, b, lambda x, y: x ^ y) != (a + b) % 3 for a in range(3) for b in range(3))
    assert (lit, fix) == (5, 0)


def test_alg5_as_printed_is_not_canonical():
    """Alg. 5 (p != 2^r - 1) as printed leaves some sums in [p+1, 2^r); the
    library therefore uses ripple add + conditional subtract.  Ex. 3 is one
    of the cases it gets right."""
    def alg5(p, v, w):
        r = r_bits(p)
        f = (1 << r) - p
        d, e = v ^ w, v & w
        while e:
            eps = (e >> (r - 1)) & 1
            v, w = d, (e << 1) & ((1 << r) - 1)
            ef = f if eps else 0
            d, e = v ^ w ^ ef, (v & w) | (v & ef) | (w & ef)
        t = all((d >> i) & 1 for i in range(r) if (p >> i) & 1)
        return d ^ (p if t else 0)
    assert alg5(11, 10, 9) == 8
    bad = {p: sum(alg5(p, a, b) != (a + b) % p for a in range(p) for b in range(p)) for p in (5, 11, 13)}
    assert all(v > 0 for v in bad.values())


# ---------------------------------------------------- enumeration order ----

def revolving_door(n, t):
    """R(n,t) from its recursive definition, subsets of {0..n-1}."""
    if t == 0:
        return [frozenset()]
    if t == n:
        return [frozenset(range(n))]
    return revolving_door(n - 1, t) + [s | {n - 1} for s in reversed(revolving_door(n - 1, t - 1))]


def mask(s):
    return sum(1 << x for x in s)


def test_revolving_door(lib):
    for n in range(1, 13):
        for t in range(0, n + 1):
            seq = revolving_door(n, t)
            assert len(seq) == math.comb(n, t)
            for r, s in enumerate(seq):
                assert B.fpcode_test_rd_unrank(r, n, t) == mask(s)
                assert B.fpcode_test_rd_rank(mask(s), n, t) == r
                nxt = B.fpcode_test_rd_next(mask(s), n, t)
                if r + 1 < len(seq):
                    assert nxt == mask(seq[r + 1])
                    assert len(s ^ seq[r + 1]) == 2  # one exchange
                else:
                    assert nxt is None


def test_revolving_door_large_n(lib):
    """Unranking at the kernel's sizes (n up to 64, t up to 23) inverts the
    ranking, which walks the definition's recursion from the top."""
    rng = np.random.default_rng(11)
    for n in (20, 33, 40, 63, 64):
        for t in (1, 2, 5, 12, 23):
            if t > n:
                continue
            total = math.comb(n, t)
            ranks = {0, total - 1, total // 2} | {int(x) for x in rng.integers(0, total, size=40, dtype=np.uint64)
                                                 if int(x) < total}
            for r in sorted(ranks):
                T = B.fpcode_test_rd_unrank(r, n, t)
                assert bin(T).count("1") == t and T < (1 << n)
                assert B.fpcode_test_rd_rank(T, n, t) == r


def _codeword_coeffs(k, g, p, I, x, c):
    m, Q, coefs = B.fpcode_test_prefix_unrank(I, k, g, p)
    v = [0] * k
    v[m] = 1
    for s, q in enumerate(sorted(b for b in range(64) if (Q >> b) & 1)):
        v[q] = coefs[s]
    assert x > m
    v[x] = c
    return v


@pytest.mark.parametrize("k,g,p", [(6, 2, 3), (7, 3, 3), (7, 4, 5), (6, 3, 7), (8, 5, 3), (6, 4, 11), (9, 3, 7)])
def test_pass_enumerates_each_class_once(k, g, p, lib):
    """Prefixes x leaves of pass g visit every vector of F_p^k with exactly
    g nonzeros exactly once up to scaling (Sec. 4.2)."""
    NC = (p - 1) ** (g - 2)
    nprefix = math.comb(k - 1, g - 1) * NC
    seen = set()
    count = 0
    for I in range(nprefix):
        m, _Q, _c = B.fpcode_test_prefix_unrank(I, k, g, p)
        for x in range(m + 1, k):
            for c in range(1, p):
                v = _codeword_coeffs(k, g, p, I, x, c)
                assert sum(1 for a in v if a) == g
                lead = next(a for a in v if a)
                inv = pow(lead, p - 2, p)
                seen.add(tuple((a * inv) % p for a in v))
                count += 1
    assert count == math.comb(k, g) * (p - 1) ** (g - 1) == len(seen)


@pytest.mark.parametrize("k,g,p", [(9, 4, 3), (8, 3, 7), (10, 5, 5), (12, 6, 3), (7, 4, 13)])
def test_prefix_walk_matches_unrank(k, g, p, lib):
    """The kernel's walk from prefix I reaches the prefix of index I + s, and
    each Gray step changes exactly one coefficient by +-1."""
    NC = (p - 1) ** (g - 2)
    nprefix = math.comb(k - 1, g - 1) * NC
    rng = np.random.default_rng(5)
    starts = sorted(set(int(x) for x in rng.integers(0, nprefix, size=12)) | {0})
    for I in starts:
        steps = min(40, nprefix - 1 - I)
        prev = B.fpcode_test_prefix_unrank(I, k, g, p)
        for s in range(1, steps + 1):
            walked = B.fpcode_test_prefix_walk(I, s, k, g, p)
            assert walked == B.fpcode_test_prefix_unrank(I + s, k, g, p)
            if walked[0] == prev[0] and walked[1] == prev[1]:
                diff = [(a - b) % p for a, b in zip(walked[2], prev[2])]
                assert sum(1 for d in diff if d) == 1 and all(d in (0, 1, p - 1) for d in diff)
            prev = walked


# ------------------------------------------------ preparation + schedule ----

@pytest.mark.parametrize("p,n,k", [(3, 80, 40), (3, 30, 15), (7, 40, 20), (5, 70, 20), (7, 150, 30), (11, 40, 12),
                                   (3, 140, 12), (31, 60, 10), (127, 40, 6), (251, 20, 4)])
def test_stored_rows_are_the_sliced_multiples(p, n, k, lib):
    """Every stored table row is v * A_j[t] (the non-pivot part of row t of
    Gamma_j, times v, mod p) in the bit-sliced natural encoding: word w,
    slice i holds bit i of symbols 32w .. 32w + 31; for p = 3, 7 the pair
    signature of representative c holds bits y_i xor y_{i+1} of y = c A_j[t]."""
    code = inputs.single_code(77 + n, p, n, k)
    pr = _prep(code, pair_leaves=0)  # the one-row-leaf tables (pair tables: test_stored_pair_table)
    m, _kj, _np, _c = B.fpcode_prepared_shape(pr)
    r = p.bit_length()
    W = -(-(n - k) // 32)
    reps = {3: [1], 7: [1, 2, 4]}.get(p, [])

    def sliced(vals, nbits):
        out = []
        for w in range(W):
            for i in range(nbits):
                out.append(sum(((int(vals[32 * w + b]) >> i) & 1) << b
                               for b in range(32) if 32 * w + b < len(vals)))
        return out

    for j in range(m):
        gam, piv = B.fpcode_prepared_gamma(pr, j)
        red = [c for c in range(n) if c not in set(piv)]
        for t in range(k):
            a = [int(gam[t, c]) for c in red]
            for v in range(1, p):
                slices, sig = B.fpcode_test_prepared_row(pr, j, t, v)
                assert slices == sliced([(v * x) % p for x in a], r), (j, t, v)
            want = []
            for c in reps:
                y = [(c * x) % p for x in a]
                want += sliced([(q ^ (q >> 1)) & ((1 << (r - 1)) - 1) for q in y], r - 1)
            assert sig[:len(want)] == want and not any(sig[len(want):]), (j, t)

def _prep(code, **kw):
    return B.fpcode_prepare(code.p, code.n, code.k, code.G, B.fpcode_opts_default(**kw))


@pytest.mark.parametrize("seed", range(12))
def test_info_sets_and_schedule_match_oracle(seed, lib):
    rng = np.random.default_rng(100 + seed)
    shapes = [(3, 11, 4), (7, 13, 5), (5, 10, 3), (3, 17, 6), (11, 9, 4), (3, 30, 15)]
    p, n, k = shapes[seed % len(shapes)]
    G = rng.integers(0, p, size=(k, n), dtype=np.uint8)
    if seed % 3 == 0:
        G[:, 1] = 0
    code = inputs.Code(p, n, k, G)
    try:
        info = oracle.info_sets(code)
    except ValueError:
        with pytest.raises(B.FpcodeError):
            _prep(code)
        return
    pr = _prep(code)
    m, kj, npasses, complete = B.fpcode_prepared_shape(pr)
    assert (m, kj) == (info.m, info.kj)
    for j in range(m):
        gam, piv = B.fpcode_prepared_gamma(pr, j)
        assert np.array_equal(gam, info.gammas[j]) and piv == list(info.pivots[j])
    for per_round, defer in ((0, 1), (1, 0), (0, 0)):
        pr2 = _prep(code, per_round_check=per_round, defer=defer)
        passes = B.fpcode_prepared_passes(pr2)
        r = oracle.bz(code, per_round_check=bool(per_round), defer=bool(defer))
        # the oracle's passes are a prefix of the full schedule
        assert [(g, j) for g, j, *_ in passes[:len(r.passes)]] == [(g, j) for g, j, _b, _L in r.passes]
        assert [La for _g, _j, _Lb, La, *_ in passes[:len(r.passes)]] == [L for *_x, L in r.passes]
        for g, _j, _Lb, _La, _re, size, _np in passes:
            assert size == math.comb(k, g) * (p - 1) ** (g - 1)


def test_budget_truncates_schedule(lib):
    code = inputs.single("f7_n40_k20")
    pr = _prep(code, budget=100000)
    _m, _kj, npasses, complete = B.fpcode_prepared_shape(pr)
    passes = B.fpcode_prepared_passes(pr)
    assert not complete and sum(x[5] for x in passes) <= 100000
    r = oracle.bz(code, budget=100000)
    assert [(g, j) for g, j, *_ in passes] == [(g, j) for g, j, _b, _L in r.passes]


def test_prepare_rejects_bad_input(lib):
    G = np.eye(3, 5, dtype=np.uint8)
    for p, n, k, M in ((4, 5, 3, G), (3, 5, 3, G + 3), (3, 5, 0, G[:0]), (257, 5, 3, G)):
        with pytest.raises(B.FpcodeError) as e:
            B.fpcode_prepare(p, n, k, M)
        assert e.value.status == B.EINVAL
    rank_def = np.zeros((2, 5), dtype=np.uint8)
    rank_def[0, 0] = rank_def[1, 0] = 1
    with pytest.raises(B.FpcodeError):
        B.fpcode_prepare(3, 5, 2, rank_def)


@pytest.mark.parametrize("ctas,fixed_pl,min_steps", [(760, 0, 8), (608, 0, 8), (608, 0, 1), (608, 0, 32), (152, 0, 8),
                                                     (7, 0, 8), (760, 3, 8), (1, 0, 8)])
def test_task_ranges_tile_each_pass(ctas, fixed_pl, min_steps, lib):
    """Guided (shrinking) and fixed task ranges cover every prefix of a pass
    exactly once, in order; a pass too small to give every lane of the grid
    min_steps prefixes gets fewer tasks than CTAs, each (but the last)
    giving every lane at least min_steps prefixes."""
    code = inputs.single("f3_n80_k40")
    pr = _prep(code, pair_leaves=0)  # one-row leaves (pair-leaf plans: test_pair_tasks_tile_each_pass)
    passes = B.fpcode_prepared_passes(pr)
    for i, (g, _j, _Lb, _La, _re, _size, nprefix) in enumerate(passes[:14]):
        if fixed_pl and nprefix > 256 * fixed_pl * 60000:
            continue  # more tasks than the hook returns
        ranges = B.fpcode_test_task_ranges(pr, i, ctas, fixed_pl, min_steps)
        if not fixed_pl and g > 1 and nprefix < 256 * ctas * min_steps:
            assert len(ranges) <= ctas
            if min_steps <= 8 and nprefix <= 256 * ctas:  # single code: a tiny pass is spread wide
                assert all(hi - lo <= 256 * 256 for lo, hi in ranges)
            else:
                assert all(hi - lo >= 256 * min_steps for lo, hi in ranges[:-1])
        if g == 1:
            assert ranges == [(0, nprefix)]
            continue
        pos = 0
        for lo, hi in ranges:
            assert lo == pos and hi >= lo
            pos = hi
        assert pos == nprefix
        if fixed_pl == 0 and nprefix > 2 * 256 * ctas:
            sizes = [hi - lo for lo, hi in ranges]
            assert sizes[0] + 256 >= sizes[-1]  # tasks shrink as the pass drains (up to one unit)


@pytest.mark.parametrize("name,ctas,fixed_pl,min_steps", [("f3_n80_k40", 608, 0, 8), ("f7_n40_k20", 608, 0, 8),
                                                          ("f7_n40_k20", 152, 0, 32), ("f3_n30_k15", 7, 0, 8),
                                                          ("f7_n40_k20", 608, 3, 8), ("f3_n80_k40", 100, 0, 32)])
def test_lanes_tile_each_pass(name, ctas, fixed_pl, min_steps, lib):
    """Every prefix of a one-row pass is walked by exactly one lane of one
    task, for guided and fixed task plans."""
    pr = _prep(inputs.single(name), pair_leaves=0)
    passes = B.fpcode_prepared_passes(pr)
    for i, (g, _j, _Lb, _La, _re, _size, nprefix) in enumerate(passes[:12]):
        if g < 2 or nprefix > 1 << 21:
            continue
        lo, hi = B.fpcode_test_lane_ranges(pr, i, ctas, fixed_pl, min_steps)
        lo, hi = lo.astype(np.int64), hi.astype(np.int64)
        keep = hi > lo
        order = np.argsort(lo[keep], kind="stable")
        a, b = lo[keep][order], hi[keep][order]
        assert a[0] == 0 and b[-1] == nprefix, i
        assert (a[1:] == b[:-1]).all(), i  # no gap, no overlap


def test_guided_tasks_are_whole_rows_and_shrink(lib):
    """A guided pass is cut into rows of one prefix unit per lane (256
    units): every task but the pass's last holds whole rows, and task sizes
    never grow along the pass, ending on one-row tasks."""
    code = inputs.single("f3_n80_k40")
    pr = _prep(code, pair_leaves=0)
    passes = B.fpcode_prepared_passes(pr)
    seen = 0
    for i, (g, _j, _Lb, _La, _re, _size, nprefix) in enumerate(passes[:14]):
        if g < 2:
            continue
        for ctas in (608, 152):
            ranges = B.fpcode_test_task_ranges(pr, i, ctas, 0, 8)
            sizes = [hi - lo for lo, hi in ranges]
            if nprefix < 256 * ctas * 8:
                continue  # fixed tasks of a small pass
            seen += 1
            unit = sizes[-2] // 256  # a one-row task
            assert all(sz % (256 * unit) == 0 for sz in sizes[:-1]), (i, ctas)
            assert all(a >= b for a, b in zip(sizes[:-1], sizes[1:-1])), (i, ctas)
            assert sizes[-2] == 256 * unit and sizes[-1] <= 256 * unit
    assert seen >= 4


def test_schedule_stays_within_staged_binomial_columns():
    """A level g needs binomial columns up to g - 1 in shared memory (24 are
    staged).  k = 24 over F_3 schedules every level up to g = 24; for larger
    k the prefix-index limit ends the schedule earlier, so no schedule holds
    a level past the staged columns."""
    rng = np.random.default_rng(5)
    for k, complete in ((24, True), (26, False), (40, False)):
        A = rng.integers(0, 3, size=(k, k), dtype=np.uint8)
        code = inputs.systematic(3, 2 * k, k, A)
        pr = B.fpcode_prepare(code.p, code.n, code.k, code.G, B.fpcode_opts_default(budget=0))
        gmax = max(x[0] for x in B.fpcode_prepared_passes(pr))
        assert gmax <= 24
        assert B.fpcode_prepared_shape(pr)[3] is complete
        if complete:
            assert gmax == 24


def test_checkpoint_and_resume_validation(lib):
    """Checkpoints exist only after a search that stopped at its budget, and
    a resume refuses a checkpoint of another code, of other schedule
    options, or one the schedule does not reach past (all before any
    device work)."""
    code = inputs.single("f7_n40_k20")
    pr = B.fpcode_prepare(code.p, code.n, code.k, code.G, B.fpcode_opts_default(budget=10 ** 6))
    with pytest.raises(B.FpcodeError) as e:
        B.fpcode_search_checkpoint(pr)
    assert e.value.status == B.EINVAL
    npasses = len(B.fpcode_prepared_passes(pr))
    other = inputs.single_code(5, code.p, code.n, code.k)
    pr_other = B.fpcode_prepare(other.p, other.n, other.k, other.G, B.fpcode_opts_default(budget=10 ** 6))
    pr_lit = B.fpcode_prepare(code.p, code.n, code.k, code.G,
                              B.fpcode_opts_default(budget=10 ** 6, per_round_check=1))
    ck = B.fpcode_checkpoint(code.p, code.n, code.k, 2, ~0 & 0xFFFFFFFFFFFFFFFF, 0)
    for target in (pr, pr_other, pr_lit):  # wrong hash for all three (0)
        with pytest.raises(B.FpcodeError, match="another code"):
            B.fpcode_search_resume(target, ck)
    # a checkpoint of this code taken at the end of a shorter schedule ...
    short = B.fpcode_prepare(code.p, code.n, code.k, code.G, B.fpcode_opts_default(budget=10 ** 5))
    h = _code_hash(short)
    ck = B.fpcode_checkpoint(code.p, code.n, code.k, npasses, ~0 & 0xFFFFFFFFFFFFFFFF, h)
    with pytest.raises(B.FpcodeError, match="no pass after"):
        B.fpcode_search_resume(pr, ck)
    ck.passes_done = 2
    with pytest.raises(B.FpcodeError, match="not uploaded"):
        B.fpcode_search_resume(pr, ck)  # valid checkpoint, but nothing on the device yet


def _code_hash(prep):
    """The code identity the library stores (a 64-bit hash of p, n, k, the
    two schedule options, whether pair leaves are taken, and G, eight bytes
    of G per step), recomputed here from its definition."""
    M = (1 << 64) - 1
    h = 1469598103934665603

    def mix(w):
        nonlocal h
        h = ((h ^ w) * 0x9E3779B97F4A7C15) & M
        h ^= h >> 32
    code = inputs.single("f7_n40_k20")
    pair = 1 if B.fpcode_test_pair_mode(prep) > 0 else 0
    mix(code.p | code.n << 16 | code.k << 32)
    mix(0 | 1 << 8 | pair << 16)  # per_round_check 0, defer 1 (defaults), the leaf form
    g = np.asarray(code.G, dtype=np.uint8).reshape(-1).tobytes()
    i = 0
    while i + 8 <= len(g):
        mix(int.from_bytes(g[i:i + 8], "little"))
        i += 8
    tail = (len(g) << 56) & M
    for b, byte in enumerate(g[i:]):
        tail |= byte << (8 * b)
    mix(tail)
    return h


# ------------------------------------------------------------ pair leaves ----

def _pair_key(pass_index, J, e, sign):
    """The packed key of a pair-leaf codeword at weight 0 (its layout: pass
    at bit 48, stem at bit 15, entry at bit 1, sign at bit 0)."""
    return (pass_index << 48) | (J << 15) | (e << 1) | sign


@pytest.mark.parametrize("p,n,k", [(3, 80, 40), (3, 30, 15), (7, 40, 20), (3, 50, 10), (7, 80, 20), (3, 140, 12)])
def test_stored_pair_table(p, n, k, lib):
    """Pair leaves: entry e of an information set's table holds the pair
    signature (bits y_i xor y_{i+1} of every symbol) of B = A[y] + c A[x]
    mod p, where the pairs run y = k-2 down to 0, x = y+1 up to k-1, and c
    = 1 .. p-1 innermost; the words after the signature are zero; and
    slice 0 (bit 0 of every symbol) of B."""
    code = inputs.single_code(5 + n, p, n, k)
    pr = _prep(code, pair_leaves=1)
    sigp = B.fpcode_test_pair_mode(pr)
    assert sigp > 0
    m, _kj, _np, _c = B.fpcode_prepared_shape(pr)
    r = p.bit_length()
    W = -(-(n - k) // 32)

    def sliced(vals, nbits):
        out = []
        for w in range(W):
            for i in range(nbits):
                out.append(sum(((int(vals[32 * w + bb]) >> i) & 1) << bb
                               for bb in range(32) if 32 * w + bb < len(vals)))
        return out

    rng = np.random.default_rng(k)
    for j in range(m):
        gam, piv = B.fpcode_prepared_gamma(pr, j)
        red = [c for c in range(n) if c not in set(piv)]
        A = [[int(gam[t, c]) for c in red] for t in range(k)]
        order = [(y, x, c) for y in range(k - 2, -1, -1) for x in range(y + 1, k) for c in range(1, p)]
        picks = range(len(order)) if len(order) <= 400 else rng.choice(len(order), 400, replace=False)
        for e in picks:
            y, x, c = order[e]
            Bv = [(A[y][i] + c * A[x][i]) % p for i in range(n - k)]
            want = sliced([(q ^ (q >> 1)) & ((1 << (r - 1)) - 1) for q in Bv], r - 1)
            got = B.fpcode_test_pair_entry(pr, j, int(e))
            assert len(got) == sigp + W
            assert got[:len(want)] == want and not any(got[len(want):sigp]), (j, e)
            assert got[sigp:] == sliced([q & 1 for q in Bv], 1), (j, e)


def test_pair_mode_selection(lib):
    """Pair leaves (pair_leaves = 1) are taken for p = 3, 7 with k >= 3 when a
    set's pair table fits 40 KiB, and never when switched off, for other
    primes, or for k < 3.  The default (2) takes them only for searches
    expected to need 10^8 codewords or more."""
    def mode(p, n, k, **kw):
        return B.fpcode_test_pair_mode(_prep(inputs.single_code(9, p, n, k), **kw))
    assert mode(3, 80, 40, pair_leaves=1) == 2 and mode(7, 40, 20, pair_leaves=1) == 2
    assert mode(3, 30, 15, pair_leaves=1) == 1
    assert mode(3, 80, 40, pair_leaves=0) == 0
    assert mode(5, 40, 20, pair_leaves=1) == 0 and mode(11, 30, 10, pair_leaves=1) == 0
    assert mode(31, 40, 8, pair_leaves=1) == 0 and mode(3, 10, 2, pair_leaves=1) == 0
    assert mode(7, 100, 40, pair_leaves=1) == 0  # 6 C(40,2) entries of 2 + 4 words: 112 KiB
    assert mode(3, 160, 64, pair_leaves=1) == 0  # 2 C(64,2) entries of 4 + 4 words: 126 KiB
    # default: the large F_3 [80,40] search (2.7e8 codewords) takes them, the
    # small ones (F_3 [30,15]: 450; F_7 [40,20]: 4.2e7) do not
    assert mode(3, 80, 40) == 2 and mode(3, 30, 15) == 0 and mode(7, 40, 20) == 0


@pytest.mark.parametrize("p,k", [(3, 5), (3, 7), (7, 5), (7, 6)])
def test_pair_pass_enumerates_each_class_once(p, k, lib):
    """Every pass of a pair-leaf schedule visits each projective class of
    codewords with exactly g nonzero coefficients once: over the stems J of
    the pass, the entries the stem is evaluated against (hook: those with y
    above the stem's largest row), and both signs (one for g = 2), the keys
    decode to coefficient vectors that are pairwise inequivalent and number
    C(k, g) (p-1)^(g-1)."""
    rng = np.random.default_rng(k)
    A = rng.integers(0, p, size=(k, k), dtype=np.uint8)
    code = inputs.systematic(p, 2 * k, k, A)
    pr = _prep(code, budget=0, defer=0, pair_leaves=1)
    assert B.fpcode_test_pair_mode(pr) > 0
    inv = {a: pow(a, p - 2, p) for a in range(1, p)}
    for i, (g, j, _Lb, _La, _re, size, nstems) in enumerate(B.fpcode_prepared_passes(pr)):
        if g < 2:
            continue
        seen = set()
        for J in range(nstems):
            _w, E = B.fpcode_test_pair_mode(pr, i, J)
            for e in range(E):
                for sign in ((0, 1) if g >= 3 else (0,)):
                    got = B.fpcode_test_key_coefficients(pr, _pair_key(i, J, e, sign))
                    assert got is not None and got[0] == g and got[1] == j
                    coef = got[2]
                    assert sum(1 for c in coef if c) == g
                    lead = next(c for c in coef if c)
                    cls = tuple(c * inv[lead] % p for c in coef)  # first nonzero coefficient 1
                    assert cls not in seen, (i, J, e, sign)
                    seen.add(cls)
        assert len(seen) == size == math.comb(k, g) * (p - 1) ** (g - 1)


@pytest.mark.parametrize("name", ["f3_n80_k40", "f7_n40_k20", "f3_n30_k15"])
@pytest.mark.parametrize("ctas", [608, 152, 7, 1])
def test_pair_tasks_tile_each_pass(name, ctas, lib):
    """The pair-leaf plan's tasks cover every stem of a pass exactly once and
    in order, and the work per task shrinks toward the end of the pass
    (guided by work): the last task is no larger than the first."""
    pr = _prep(inputs.single(name), pair_leaves=1)
    assert B.fpcode_test_pair_mode(pr) > 0
    passes = B.fpcode_prepared_passes(pr)
    for i, (g, _j, _Lb, _La, _re, _size, nstems) in enumerate(passes[:14]):
        if g < 2:
            continue
        ranges = B.fpcode_test_task_ranges(pr, i, ctas, 0, 8)
        assert 0 < len(ranges) < 1 << 16
        pos = 0
        for lo, hi in ranges:
            assert lo == pos and hi > lo, (i, lo, hi, pos)
            pos = hi
        assert pos == nstems


@pytest.mark.parametrize("ctas", [1, 7, 32])
def test_pair_plan_of_deep_passes_on_small_grids(ctas, lib):
    """The deepest passes of a p = 7 code on a small grid want more stems per
    group than a segment holds: the plan caps them (whole units of the
    coefficient counter, at least one), so every pass still tiles its stems
    with non-empty tasks.  (Choosing the unit before the cap once left zero
    stems per group, and counting the segment's tasks divided by zero.)"""
    code = inputs.single_code(11, 7, 30, 15)
    pr = _prep(code, pair_leaves=1)
    assert B.fpcode_test_pair_mode(pr) > 0
    passes = B.fpcode_prepared_passes(pr)
    assert max(g for g, *_ in passes) >= 10
    for i, (g, _j, _Lb, _La, _re, _size, nstems) in enumerate(passes):
        if g < 2:
            continue
        ranges = B.fpcode_test_task_ranges(pr, i, ctas, 0, 8)
        assert ranges and all(hi > lo for lo, hi in ranges), i
        if len(ranges) < 1 << 16:  # the whole pass came back: it tiles the stems
            assert ranges[0][0] == 0 and ranges[-1][1] == nstems, i
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:])), i


@pytest.mark.parametrize("name", ["f3_n80_k40", "f7_n40_k20"])
def test_pass_slices_keep_the_schedule_plan(name, lib):
    """A slice of a pass (one rank's part of a split search) is planned as
    the pass is in the full schedule: the same tasks over the same stems,
    whether the pass has passes after it (larger tasks) or is the last."""
    pr = _prep(inputs.single(name), pair_leaves=1)
    passes = B.fpcode_prepared_passes(pr)
    for i in (2, 5, len(passes) - 1):
        if passes[i][0] < 2:
            continue
        full = B.fpcode_test_task_ranges(pr, i, 608, 0, 8)
        sl = B.fpcode_prepared_pass_slice(pr, i, 0, len(full), 0)
        assert B.fpcode_test_task_ranges(sl, 0, 608, 0, 8) == full, i


# ------------------------------------------------------------- autotuner ----

def test_tune_search_finds_the_minimum_of_separable_costs(lib):
    """The batch autotuner's coordinate search (fpcode_autotune_batch) on
    synthetic cost tables: on a separable cost it reaches the global minimum
    from any start in one round plus a confirming round, evaluating each grid
    point at most once."""
    sizes = [3, 5, 2]
    rng = np.random.default_rng(11)
    for _ in range(20):
        parts = [rng.uniform(1, 10, size=s) for s in sizes]
        cost = parts[0][:, None, None] + parts[1][None, :, None] + parts[2][None, None, :]
        start = [int(rng.integers(0, s)) for s in sizes]
        best, evals = B.fpcode_test_tune_search(sizes, start, cost)
        assert tuple(best) == np.unravel_index(int(np.argmin(cost)), cost.shape)
        assert evals <= cost.size


def test_tune_search_moves_until_a_round_finds_nothing(lib):
    """A cost whose best value along one setting depends on another: the search
    keeps sweeping until no setting improves, ends at a point no single-setting
    change improves (a coordinate-wise minimum), and never returns a point
    marked as unable to run (negative cost)."""
    sizes = [4, 4]
    cost = np.array([[9, 8, 7, 6],
                     [8, 7, 6, 5],
                     [7, 6, 5, 4],
                     [6, 5, 4, 1]], dtype=float)
    best, _ = B.fpcode_test_tune_search(sizes, [0, 0], cost)
    assert best == [3, 3]
    cost2 = cost.copy()
    cost2[3, 3] = -1.0  # cannot run
    best, _ = B.fpcode_test_tune_search(sizes, [0, 0], cost2)
    b0, b1 = best
    assert cost2[b0, b1] >= 0
    for v in range(4):  # a coordinate-wise minimum over the runnable points
        assert cost2[v, b1] < 0 or cost2[v, b1] >= cost2[b0, b1]
        assert cost2[b0, v] < 0 or cost2[b0, v] >= cost2[b0, b1]


def test_batch_results_view_equals_eager_results():
    """The batch call's results view builds each Result on first access from
    the returned arrays: every field, the witness slices, negative indices
    and slices equal the eagerly built list."""
    codes = inputs.batch_codes(64)
    ns, ks = [c.n for c in codes], [c.k for c in codes]
    rng = np.random.default_rng(1)
    res = np.zeros(len(codes), dtype=B._RESULT_DT)
    for f in ("status", "d", "L", "U", "m", "npasses", "launch"):
        res[f] = rng.integers(0, 20, len(codes))
    res["enumerated"] = rng.integers(0, 10 ** 9, len(codes))
    res["best_key"] = rng.integers(0, 2 ** 62, len(codes), dtype=np.int64).astype(np.uint64)
    res["counts"] = rng.integers(0, 1000, (len(codes), 65))
    res["kj"] = rng.integers(0, 60, (len(codes), 255))
    res["t_kernel_ms"] = rng.random(len(codes))
    wit = rng.integers(0, 7, sum(ns)).astype(np.uint8)
    eager = B._results_of(res, ks, ns, wit)
    view = B.BatchResults(res, ks, ns, wit)
    assert len(view) == len(eager)

    def fields(r):
        return (r.status, r.d, r.L, r.U, r.m, r.npasses, r.enumerated, r.counts, r.kj, r.t_prepare_ms, r.t_kernel_ms,
                r.t_total_ms, r.launch, r.best_key, r.witness.tolist())
    assert [fields(r) for r in view] == [fields(r) for r in eager]
    assert fields(view[-1]) == fields(eager[-1]) and [fields(r) for r in view[3:9]] == [fields(r) for r in eager[3:9]]
    assert (view.field("d") == np.array([r.d for r in eager])).all()
    with pytest.raises(IndexError):
        view[len(codes)]
