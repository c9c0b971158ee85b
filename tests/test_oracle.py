"""Pins for the CPU oracle, independent of the oracle itself.

Each pin checks the oracle against something fixed outside it: textbook codes
built from their definitions with published weight distributions,
MacWilliams identities, closed forms, the bounds of Alg. 6 and hand-checkable
tiny codes.  ``PINS`` lists the pin functions; ``test_oracle_mutants`` plants
mistakes in a copy of the oracle source and checks that at least one pin
fails for each.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import gf
import oracle
from paper_2603_29942_gb300 import inputs

# Weight distributions of the ternary Golay codes (MacWilliams & Sloane,
# "The Theory of Error-Correcting Codes", Ch. 20): nonzero weights only.
GOLAY_11 = {5: 132, 6: 132, 8: 330, 9: 110, 11: 24}
GOLAY_12 = {6: 264, 9: 440, 12: 24}


def _code(p, G):
    G = np.ascontiguousarray(np.asarray(G, dtype=np.uint8))
    return inputs.Code(int(p), int(G.shape[1]), int(G.shape[0]), G)


def _dist_dict(dist):
    return {w: int(c) for w, c in enumerate(dist) if w > 0 and c}


# ---------------------------------------------------------------- pins ----

def pin_golay(lib_path=None):
    """Brute force and BZ on the [11,6,5] and [12,6,6] ternary Golay codes."""
    G11 = gf.ternary_golay()
    G12 = gf.extend_parity(G11, 3)
    bf11 = oracle.brute_force(_code(3, G11), lib_path=lib_path)
    bf12 = oracle.brute_force(_code(3, G12), lib_path=lib_path)
    assert _dist_dict(bf11.dist) == GOLAY_11
    assert _dist_dict(bf12.dist) == GOLAY_12
    assert bf11.d == 5 and bf12.d == 6
    assert oracle.bz(_code(3, G11), lib_path=lib_path).d == 5
    assert oracle.bz(_code(3, G12), lib_path=lib_path).d == 6


def pin_hamming(lib_path=None):
    """Ternary [13,10,3] and heptary [8,6,3] Hamming codes: d = 3, and the
    weight distribution is the MacWilliams transform of the simplex code's
    (every nonzero simplex codeword has weight q^(r-1))."""
    for q, r in ((3, 3), (7, 2)):
        G, H = gf.hamming_code(q, r)
        N = G.shape[1]
        c = _code(q, G)
        assert c.k == N - r
        bf = oracle.brute_force(c, lib_path=lib_path)
        simplex = [0] * (N + 1)
        simplex[0] = 1
        simplex[q ** (r - 1)] = q ** r - 1
        assert [int(x) for x in bf.dist] == gf.macwilliams(simplex, N, q, q ** r)
        assert bf.d == 3
        assert oracle.bz(c, lib_path=lib_path).d == 3
        # the dual (simplex) code itself: constant weight q^(r-1)
        bfs = oracle.brute_force(_code(q, H), lib_path=lib_path)
        assert [int(x) for x in bfs.dist] == simplex


def pin_tiny_by_hand(lib_path=None):
    """Repetition [n,1,n], its dual [n,n-1,2], the full space [n,n,1] and a
    hand-worked [4,2] code over F_5 with d = 3."""
    for p in (3, 5, 7, 11):
        for n in (1, 2, 5, 9):
            rep = _code(p, np.ones((1, n), dtype=np.uint8))
            assert oracle.brute_force(rep, lib_path=lib_path).d == n
            assert oracle.bz(rep, lib_path=lib_path).d == n
            if n >= 2:
                dual = np.hstack([np.eye(n - 1, dtype=np.uint8), np.full((n - 1, 1), p - 1, dtype=np.uint8)])
                assert oracle.bz(_code(p, dual), lib_path=lib_path).d == 2
                assert oracle.brute_force(_code(p, dual), lib_path=lib_path).d == 2
            full = _code(p, np.eye(n, dtype=np.uint8))
            assert oracle.bz(full, lib_path=lib_path).d == 1
    # rows (1,0,1,1), (0,1,1,2) over F_5: a(1,0,1,1) + b(0,1,1,2) = (a, b, a+b, a+2b);
    # with a, b != 0 at most one of a+b, a+2b vanishes, so d = 3 (e.g. a=1,b=4).
    G = np.array([[1, 0, 1, 1], [0, 1, 1, 2]], dtype=np.uint8)
    bf = oracle.brute_force(_code(5, G), lib_path=lib_path)
    assert bf.d == 3
    assert oracle.bz(_code(5, G), lib_path=lib_path).d == 3
    # slow pure-Python enumeration for the same tiny code
    assert [int(x) for x in bf.dist] == gf.weight_distribution_slow(G.tolist(), 5)


def pin_macwilliams_random(lib_path=None):
    """Random small codes: brute-force distributions of C and of its dual
    (null space computed by the tests' own linear algebra) satisfy the
    MacWilliams identity."""
    rng = np.random.default_rng(11)
    for p, n, k in ((3, 10, 4), (5, 7, 3), (7, 6, 2), (11, 5, 2), (3, 9, 5)):
        for _ in range(3):
            G = rng.integers(0, p, size=(k, n), dtype=np.uint8)
            if gf.rank(G.tolist(), p) < k:
                continue
            Hd = np.array(gf.null_space(G.tolist(), p), dtype=np.uint8)
            a = oracle.brute_force(_code(p, G), lib_path=lib_path)
            b = oracle.brute_force(_code(p, Hd), lib_path=lib_path)
            assert [int(x) for x in b.dist] == gf.macwilliams(a.dist, n, p, p ** k)
            assert int(a.dist.sum()) == p ** k


def pin_bz_equals_brute_force(lib_path=None, seeds=60):
    """BZ oracle = brute force on random codes, including rank-deficient
    last information sets, zero and repeated columns; the BZ witness is a
    nonzero codeword of weight d."""
    rng = np.random.default_rng(12)
    shapes = [(3, 11, 4), (3, 14, 6), (5, 9, 4), (7, 10, 4), (11, 7, 3), (3, 16, 5), (5, 12, 3), (7, 9, 5)]
    for s in range(seeds):
        p, n, k = shapes[s % len(shapes)]
        G = rng.integers(0, p, size=(k, n), dtype=np.uint8)
        if s % 5 == 0:
            G[:, rng.integers(0, n)] = 0  # a zero column
        if s % 7 == 0:
            G[:, 0] = G[:, n - 1]  # a repeated column
        if gf.rank(G.tolist(), p) < k:
            continue
        c = _code(p, G)
        bf = oracle.brute_force(c, lib_path=lib_path)
        for per_round, defer in ((False, True), (True, False), (False, False)):
            r = oracle.bz(c, per_round_check=per_round, defer=defer, lib_path=lib_path)
            assert r.status == oracle.OK
            assert r.d == bf.d, (s, p, n, k, per_round, defer)
            w = [int(x) for x in r.witness]
            assert gf.weight(w) == r.d and any(w)
            assert gf.in_rowspace(G.tolist(), w, p)
    # low-rate codes (three or four information sets, d near 0.3 n) whose
    # search reaches g >= 3 while p^k stays small enough for brute force
    deepest = 0
    for p, n, k in ((3, 33, 11), (3, 36, 12), (5, 24, 8), (7, 21, 7), (11, 18, 6)):
        G = np.hstack([np.eye(k, dtype=np.uint8), rng.integers(0, p, size=(k, n - k), dtype=np.uint8)])
        c = _code(p, G)
        bf = oracle.brute_force(c, lib_path=lib_path)
        r = oracle.bz(c, lib_path=lib_path)
        assert r.d == bf.d, (p, n, k)
        deepest = max(deepest, max(g for g, *_ in r.passes))
    assert deepest >= 3


def pin_counts_closed_form(lib_path=None):
    """Per-level counts equal (passes entered at level g) * C(k,g)(p-1)^(g-1),
    and they add up to the evaluated total."""
    rng = np.random.default_rng(13)
    deepest = 0
    for p, n, k in ((3, 20, 8), (7, 14, 6), (5, 17, 6), (3, 13, 5), (3, 40, 20), (5, 30, 15), (7, 30, 15)):
        G = rng.integers(0, p, size=(k, n), dtype=np.uint8)
        if gf.rank(G.tolist(), p) < k:
            continue
        r = oracle.bz(_code(p, G), lib_path=lib_path)
        per_level = {}
        for g, _j, _b, _L in r.passes:
            per_level[g] = per_level.get(g, 0) + 1
        for g in range(1, k + 1):
            expect = per_level.get(g, 0) * math.comb(k, g) * (p - 1) ** (g - 1)
            assert r.counts[g] == expect
        assert sum(r.counts) == r.evaluated
        for g in range(1, k + 1):
            assert oracle.pass_size(p, k, g) == math.comb(k, g) * (p - 1) ** (g - 1)
        deepest = max(deepest, max(g for g, *_ in r.passes))
    assert deepest >= 4


def pin_bounds_alg6(lib_path=None):
    """With full-rank Gamma_1..Gamma_(m-1) and the per-round check, the bound
    after round g is (m-1)(g+1) + max(0, g+1-k+k_m) (the bound of Alg. 6); every
    pass's best weight is >= d; the search stops at L >= U = d; Singleton
    and Griesmer hold."""
    rng = np.random.default_rng(14)
    closed_form_checked = 0
    for p, n, k in ((3, 22, 8), (7, 15, 5), (3, 25, 10), (5, 14, 5), (3, 20, 8), (7, 17, 6)):
        G = np.hstack([np.eye(k, dtype=np.uint8), rng.integers(0, p, size=(k, n - k), dtype=np.uint8)])
        c = _code(p, G)
        r = oracle.bz(c, per_round_check=True, defer=False, lib_path=lib_path)
        m, kj = r.m, r.kj
        e = [0] * m
        for g, j, best, L in r.passes:
            assert best >= r.d
            e[j] = g
            # bound from the levels completed: fresh positions only
            assert L == sum(max(0, e[i] + 1 - (k - kj[i])) for i in range(m))
            if j == m - 1 and all(x == k for x in kj[:-1]):  # end of round g
                assert L == (m - 1) * (g + 1) + max(0, g + 1 - k + kj[-1])
                closed_form_checked += 1
        assert r.L >= r.U == r.d
        assert r.d <= n - k + 1
        assert n >= gf.griesmer(k, r.d, p)
    assert closed_form_checked > 0


def pin_metamorphic(lib_path=None):
    """d is invariant under column permutation, nonzero column scaling and
    invertible row operations; [G|G] doubles it; a direct sum takes the
    minimum; deleting a column lowers it by at most one."""
    rng = np.random.default_rng(15)
    for p, n, k in ((3, 14, 5), (7, 10, 4), (5, 11, 4)):
        G = rng.integers(0, p, size=(k, n), dtype=np.uint8)
        if gf.rank(G.tolist(), p) < k:
            continue
        d = oracle.brute_force(_code(p, G), lib_path=lib_path).d
        perm = rng.permutation(n)
        scale = rng.integers(1, p, size=n)
        G2 = (G[:, perm].astype(np.int64) * scale[None, :]) % p
        while True:
            R = rng.integers(0, p, size=(k, k))
            if gf.rank(R.tolist(), p) == k:
                break
        G3 = (R @ G2) % p
        assert oracle.bz(_code(p, G3.astype(np.uint8)), lib_path=lib_path).d == d
        GG = np.hstack([G, G])
        assert oracle.bz(_code(p, GG), lib_path=lib_path).d == 2 * d
        H = rng.integers(0, p, size=(3, 7), dtype=np.uint8)
        if gf.rank(H.tolist(), p) == 3:
            dH = oracle.brute_force(_code(p, H), lib_path=lib_path).d
            S = np.zeros((k + 3, n + 7), dtype=np.uint8)
            S[:k, :n] = G
            S[k:, n:] = H
            assert oracle.bz(_code(p, S), lib_path=lib_path).d == min(d, dH)
        Gp = np.delete(G, int(rng.integers(0, n)), axis=1)
        if gf.rank(Gp.tolist(), p) == k:
            dp = oracle.bz(_code(p, Gp), lib_path=lib_path).d
            assert d - 1 <= dp <= d


def pin_info_sets(lib_path=None):
    """Each Gamma_j generates the same code, is the identity on its pivot
    columns (rows ordered by pivot), fresh pivot sets are disjoint, and the
    greedy choice is maximal: an unused column that was not taken in round
    j lies in the span of that round's fresh pivot columns of G."""
    rng = np.random.default_rng(16)
    for p, n, k in ((3, 11, 4), (7, 13, 5), (5, 10, 3), (3, 17, 6)):
        G = rng.integers(0, p, size=(k, n), dtype=np.uint8)
        G[:, 2] = 0
        if gf.rank(G.tolist(), p) < k:
            continue
        info = oracle.info_sets(_code(p, G), lib_path=lib_path)
        used = set()
        rg = gf.rank(G.tolist(), p)
        for j in range(info.m):
            Gam = info.gammas[j]
            piv = [int(x) for x in info.pivots[j]]
            assert piv == sorted(piv)
            assert np.array_equal(Gam[:, piv], np.eye(k, dtype=np.uint8))
            assert gf.rank(np.vstack([G, Gam]).tolist(), p) == rg == k
            fresh = [c for c in piv if c not in used]
            assert len(fresh) == info.kj[j]
            unused_before = [c for c in range(n) if c not in used]
            # maximality of the greedy scan over unused columns
            for c in unused_before:
                if c not in fresh:
                    cols = G[:, fresh + [c]].T.tolist()
                    assert gf.rank(cols, p) == len(fresh)
            used |= set(fresh)
        assert info.kj[0] == k


def _all_codewords(G, p):
    """Every codeword m G (numpy, test-side), one row per message."""
    k = G.shape[0]
    msgs = np.array(np.meshgrid(*[np.arange(p)] * k, indexing="ij")).reshape(k, -1).T
    return (msgs.astype(np.int64) @ G.astype(np.int64)) % p


def pin_pass_minima_and_bound(lib_path=None):
    """For tiny codes, per pass (g, j): the best weight the search reports is
    the true minimum over codewords with exactly g nonzeros on the pivot
    columns of Gamma_j; each Gamma_j's levels are enumerated as 1..e_j
    without gaps; and every lower bound L reported after a pass is <= the
    weight of every nonzero codeword not yet enumerated (the bound is
    valid).  Computed by numpy over all p^k codewords."""
    rng = np.random.default_rng(17)
    shapes = [(3, 33, 11), (3, 16, 10), (5, 12, 7), (7, 10, 6), (3, 18, 7), (5, 13, 6), (7, 11, 5), (11, 9, 4)]
    for s, (p, n, k) in enumerate(shapes * 2):
        G = rng.integers(0, p, size=(k, n), dtype=np.uint8)
        if s % 3 == 0:
            G[:, : k] = np.eye(k, dtype=np.uint8)
        if gf.rank(G.tolist(), p) < k:
            continue
        code = _code(p, G)
        info = oracle.info_sets(code, lib_path=lib_path)
        C = _all_codewords(G, p)
        wt = (C != 0).sum(axis=1)
        nz = wt > 0
        wt_on = [(C[:, info.pivots[j]] != 0).sum(axis=1) for j in range(info.m)]
        for defer in (True, False):
            r = oracle.bz(code, defer=defer, lib_path=lib_path)
            assert r.m == info.m
            e = [0] * r.m
            for g, j, best, L in r.passes:
                assert g == e[j] + 1, "levels of an information set must be enumerated without gaps"
                e[j] = g
                sel = nz & (wt_on[j] == g)
                assert best == int(wt[sel].min())
                covered = np.zeros_like(nz)
                for i in range(r.m):
                    covered |= wt_on[i] <= e[i]
                rest = nz & ~covered
                if rest.any():
                    assert L <= int(wt[rest].min())
            assert r.d == int(wt[nz].min())


PINS = [pin_golay, pin_hamming, pin_tiny_by_hand, pin_macwilliams_random, pin_bz_equals_brute_force,
        pin_counts_closed_form, pin_bounds_alg6, pin_metamorphic, pin_info_sets, pin_pass_minima_and_bound]


@pytest.mark.parametrize("pin", PINS, ids=[f.__name__ for f in PINS])
def test_pin(pin, oracle_lib):
    pin()


def test_budget_interval(oracle_lib):
    """A budget stops the search at a pass boundary with L <= d <= U."""
    c = inputs.single("f7_n40_k20")
    r = oracle.bz(c, budget=100000)
    assert r.status == oracle.EBUDGET
    assert r.evaluated <= 100000
    full = oracle.bz(c, threads=4)
    assert r.L <= full.d <= r.U
    nxt = oracle.pass_size(7, 20, r.passes[-1][0] + (1 if r.passes[-1][1] == r.m - 1 else 0))
    assert r.evaluated + nxt > 100000 or r.passes[-1][1] != r.m - 1


def test_threads_do_not_change_result(oracle_lib):
    c = inputs.single("f7_n40_k20")
    a = oracle.bz(c, threads=1)
    b = oracle.bz(c, threads=7)
    assert (a.d, a.counts, a.passes) == (b.d, b.counts, b.passes)
    assert np.array_equal(a.witness, b.witness)


def test_config1_against_brute_force(oracle_lib):
    """F_3 [30,15] (3^15 messages): BZ equals brute force; the paper's T5
    reports d = 6 for a 15 x 30 F_3 matrix of the same shape."""
    c = inputs.single("f3_n30_k15")
    bf = oracle.brute_force(c)
    r = oracle.bz(c)
    assert r.d == bf.d == 6
    w = [int(x) for x in r.witness]
    assert gf.weight(w) == 6 and gf.in_rowspace(c.G.tolist(), w, 3)


# ------------------------------------------------------------ mutants ----

MUTANTS = {
    "drop_last_coefficient": ("for (int c = 1; c < p; ++c) {\n      memcpy(part[depth + 1]",
                              "for (int c = 1; c < p - 1; ++c) {\n      memcpy(part[depth + 1]"),
    "elimination_sign": ("if (f) axpy_mod(M + (size_t)q * n, row, p - f, p, n);",
                         "if (f) axpy_mod(M + (size_t)q * n, row, f, p, n);"),
    "bound_off_by_one": ("int v = e[i] + 1 - (k - kj[i]);", "int v = e[i] + 2 - (k - kj[i]);"),
    "weight_counts_ones": ("w += (v[i] != 0);", "w += (v[i] == 1);"),
    "odometer_stops_before_top_digit": ("if (i == k) break; /* back at the zero message",
                                        "if (i == k - 1) break; /* back at the zero message"),
    "row_index_transposed": ("axpy_mod(part[depth + 1], cx->gam + (size_t)t * n, c, p, n);",
                             "axpy_mod(part[depth + 1], cx->gam + (size_t)t, c, p, n);"),
    "skip_deferred_catch_up": ("for (int h = e[j] + 1; h <= g && !stop; ++h) {",
                               "for (int h = g; h <= g && !stop; ++h) {"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_oracle_mutants(name, tmp_path, oracle_lib):
    """Plant a mistake in a copy of the oracle (on the CPU) and check that the
    pins catch it."""
    src = open(oracle._SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    import subprocess

    subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-pthread", str(mut), "-o", str(lib)], check=True)
    caught = []
    for pin in PINS:
        try:
            pin(lib_path=str(lib))
        except (AssertionError, ValueError, IndexError):
            caught.append(pin.__name__)
    assert caught, f"mutant {name} passed every pin"


# ------------------------------------------------------------- golden ----

def _golden():
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_single_codes.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("name", ["f3_n30_k15", "f7_n40_k20", "f3_n80_k40"])
def test_single_code_golden(name, oracle_lib):
    """The stored oracle values for the three single-code workloads still hold
    (inputs identical by SHA-256), under both schedules."""
    import os

    g = _golden()[name]
    code = inputs.single(name)
    assert code.digest() == g["sha256"]
    for mode, kw in (("default", {}), ("paper_literal", {"per_round_check": True, "defer": False})):
        r = oracle.bz(code, threads=os.cpu_count() or 1, **kw)
        exp = g[mode]
        assert (r.d, r.L, r.U, r.m, r.kj, r.evaluated, r.counts) == (
            exp["d"], exp["L"], exp["U"], exp["m"], exp["kj"], exp["evaluated"], exp["counts"])
        assert [list(x) for x in r.passes] == exp["passes"]
        w = [int(x) for x in r.witness]
        assert gf.weight(w) == r.d and gf.in_rowspace(code.G.tolist(), w, code.p)
