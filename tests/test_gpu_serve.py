"""Serving on the GPU: continuous batching over the persistent kernel.

Each result is the same alone and in the mix: codes submitted while others
run (and into slots that earlier codes have left) give exactly the status,
d, [L, U] and per-level counts of the same code searched on its own, and a
valid witness.  Admission by device memory: a server with a tiny table
arena turns requests away (EBUSY) until earlier codes finish.
"""
import time

import numpy as np
import pytest

import os

import gf
import oracle
from paper_2603_29942_gb300 import _binding as B
from paper_2603_29942_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    B.lib()


def _alone(code, budget):
    pr = B.fpcode_prepare(code.p, code.n, code.k, code.G, B.fpcode_opts_default(budget=budget))
    return B.fpcode_min_distance_ex(pr)


def _check(code, r, ref):
    assert (r.status, r.d, r.L, r.U, r.counts[:code.k + 1]) == (ref.status, ref.d, ref.L, ref.U, ref.counts)
    if r.status == B.OK:
        w = [int(x) for x in r.witness[:code.n]]
        assert gf.weight(w) == r.d
        for h in gf.null_space(code.G.tolist(), code.p):
            assert sum(a * b for a, b in zip(h, w)) % code.p == 0


def test_serve_alone_equals_mix():
    codes, _ = inputs.serve_codes(count=120)
    budget = 2 * 10 ** 6
    srv = B.fpcode_serve_create(B.fpcode_serve_opts_default(slots=16))
    pending = list(range(len(codes)))
    tickets = {}
    results = {}
    t0 = time.time()
    while (pending or len(results) < len(codes)) and time.time() - t0 < 120:
        while pending:
            i = pending[0]
            t = B.fpcode_serve_submit(srv, codes[i], budget=budget)
            if t is None:
                break
            tickets[t] = i
            pending.pop(0)
        for t, r in B.fpcode_serve_poll(srv):
            results[tickets[t]] = r
    B.fpcode_serve_drain(srv)
    for t, r in B.fpcode_serve_poll(srv):
        results[tickets[t]] = r
    assert len(results) == len(codes)
    for i, c in enumerate(codes):
        _check(c, results[i], _alone(c, budget))
    B.fpcode_serve_destroy(srv)


def test_serve_slot_reuse_back_to_back():
    """One slot, codes submitted one after another with no pause: each code
    goes into the slot the moment its predecessor's result is posted.  A
    search's later passes are taken ahead of its termination tests (F_7
    [40,20] certifies after the g = 5 passes while CTAs already run tasks of
    its 3 * 10^8-codeword g = 6 passes), so the slot is handed over while
    those tasks are being dropped.  With mid-pass exit off every count is
    deterministic: a single count-off or record of the previous code landing
    in the next one's bookkeeping would change its per-pass codewords,
    counts or bound.  Each result equals the code's search alone, field by
    field, on a sequence that alternates long and short searches."""
    search = B.fpcode_opts_default(mid_pass_exit=0)
    srv = B.fpcode_serve_create(B.fpcode_serve_opts_default(slots=1, search=search))
    small, _ = inputs.serve_codes(count=6)
    big = [inputs.single("f7_n40_k20"), inputs.single("f3_n80_k40")]
    seq = [big[0], small[0], big[0], big[1], small[1], big[0], small[2], big[1], big[0], small[3], small[4], big[0]]
    budget = 10 ** 7
    got = []
    for c in seq:
        b = 0 if any(c is x for x in big) else budget
        t = B.fpcode_serve_submit(srv, c, budget=b)
        assert t is not None  # the only slot was handed back with the previous result
        t0 = time.time()
        out = []
        while not out and time.time() - t0 < 60:
            out = B.fpcode_serve_poll(srv)
        assert len(out) == 1 and out[0][0] == t
        got.append((c, b, out[0][1]))
    B.fpcode_serve_destroy(srv)
    for c, b, r in got:
        pr = B.fpcode_prepare(c.p, c.n, c.k, c.G, B.fpcode_opts_default(budget=b, mid_pass_exit=0))
        ref = B.fpcode_min_distance_ex(pr)
        _check(c, r, ref)
        assert r.enumerated == ref.enumerated == sum(ref.counts)


def test_serve_admission_by_memory():
    """With room for about one code's tables, later requests wait (EBUSY)
    and are admitted once earlier codes finish."""
    codes = [inputs.single_code(40 + i, 7, 40, 20) for i in range(4)]
    # one code's table: 2 information sets x 20 rows x (6 multiples x 4 words
    # + 8 words of pair signatures) x 4 bytes
    tb = 2 * 20 * (6 * 4 + 8) * 4
    srv = B.fpcode_serve_create(B.fpcode_serve_opts_default(slots=8, device_bytes=tb + 256))
    first = B.fpcode_serve_submit(srv, codes[0], budget=10 ** 5)
    assert first is not None
    assert B.fpcode_serve_submit(srv, codes[1], budget=10 ** 5) is None  # busy: no memory
    done = {}
    for i in range(1, 4):
        t = None
        t0 = time.time()
        while t is None and time.time() - t0 < 30:
            for tk, r in B.fpcode_serve_poll(srv):
                done[tk] = r
            t = B.fpcode_serve_submit(srv, codes[i], budget=10 ** 5)
        assert t is not None
    B.fpcode_serve_drain(srv)
    for tk, r in B.fpcode_serve_poll(srv):
        done[tk] = r
    assert len(done) == 4
    for r in done.values():
        assert r.status in (B.OK, B.EBUDGET)
    B.fpcode_serve_destroy(srv)


def test_serve_relaunch_after_idle():
    """The kernel exits after its idle period; a later request relaunches it."""
    srv = B.fpcode_serve_create(B.fpcode_serve_opts_default(slots=4, idle_exit_s=0.005))
    code = inputs.single("f3_n30_k15")
    for _ in range(3):
        t = B.fpcode_serve_submit(srv, code)
        B.fpcode_serve_drain(srv)
        out = dict(B.fpcode_serve_poll(srv))
        assert out[t].status == B.OK and out[t].d == 6
        time.sleep(0.05)  # longer than the idle period: the kernel has exited
    B.fpcode_serve_destroy(srv)


def test_serve_word_limit():
    """A server for n - k <= 64 turns a wider code away with EINVAL; a
    server created with max_words = 4 serves it, with the result it has
    alone."""
    wide = inputs.single_code(801, 3, 72, 6)  # n - k = 66: three words per slice
    srv = B.fpcode_serve_create(B.fpcode_serve_opts_default(slots=4))
    with pytest.raises(B.FpcodeError):
        B.fpcode_serve_submit(srv, wide, budget=10 ** 6)
    B.fpcode_serve_destroy(srv)
    srv = B.fpcode_serve_create(B.fpcode_serve_opts_default(slots=4, max_words=4))
    t = B.fpcode_serve_submit(srv, wide, budget=10 ** 6)
    assert t is not None
    B.fpcode_serve_drain(srv)
    got = dict(B.fpcode_serve_poll(srv))
    B.fpcode_serve_destroy(srv)
    _check(wide, got[t], _alone(wide, 10 ** 6))


def test_serve_stream_sample_against_oracle():
    """The serving workload's first 64 requests at the bench budget (10^8
    codewords per code), all admitted together so that they share the
    persistent kernel: a fixed sample matches the oracle run alone at the
    same budget (status, d, per-level counts, L, U) with a valid witness."""
    codes, _ = inputs.serve_codes(count=64)
    budget = 10 ** 8
    srv = B.fpcode_serve_create(B.fpcode_serve_opts_default(slots=64))
    tickets = {}
    for i, c in enumerate(codes):
        t = B.fpcode_serve_submit(srv, c, budget=budget)
        assert t is not None
        tickets[t] = i
    B.fpcode_serve_drain(srv)
    results = {tickets[t]: r for t, r in B.fpcode_serve_poll(srv)}
    B.fpcode_serve_destroy(srv)
    assert len(results) == len(codes)
    status = {oracle.OK: B.OK, oracle.EBUDGET: B.EBUDGET}
    for i in range(0, 64, 8):
        c, rs = codes[i], results[i]
        r = oracle.bz(c, budget=budget, threads=os.cpu_count() or 4)
        assert (rs.status, rs.counts[:c.k + 1], rs.L, rs.U) == (status[r.status], r.counts, r.L, r.U), i
        if r.status == oracle.OK:
            assert rs.d == r.d
            w = [int(x) for x in rs.witness[:c.n]]
            assert gf.weight(w) == r.d
            for h in gf.null_space(c.G.tolist(), c.p):
                assert sum(a * b for a, b in zip(h, w)) % c.p == 0
