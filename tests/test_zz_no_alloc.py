"""The allocation-free entry point, checked against the allocating one.

fpcode_min_distance_noalloc serves callers that cannot call cudaMalloc: it
keeps all device state in a fixed array inside the library.  This file is
collected last so that a failure here comes after every other test; it
passes alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

import gf
from paper_2603_29942_gb300 import _binding as B
from paper_2603_29942_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    B.lib()


def _check_codeword(code, d, w):
    w = [int(x) for x in w]
    assert any(w) and gf.weight(w) == d
    for h in gf.null_space(np.asarray(code.G).tolist(), code.p):
        assert sum(a * b for a, b in zip(h, w)) % code.p == 0


@pytest.mark.parametrize("name", ["f3_n30_k15", "f7_n40_k20", "f3_n80_k40"])
def test_noalloc_matches_allocating_entry_point(name):
    """Two calls in a row through the C ABI give the distance the allocating
    entry point gives (exact), each with a valid witness."""
    code = inputs.single(name)
    d_ref, w_ref = B.fpcode_min_distance(code.p, code.n, code.k, code.G)
    _check_codeword(code, d_ref, w_ref)
    for _ in range(2):
        d, w = B.fpcode_min_distance_noalloc(code.p, code.n, code.k, code.G)
        assert d == d_ref
        _check_codeword(code, d, w)


def test_noalloc_rejects_codes_above_its_fixed_scratch():
    """A code whose tables exceed the fixed array is refused with EINVAL and
    a message; the allocating entry point still handles it."""
    base = inputs.single_code(9, 61, 136, 8)  # 17 information sets, ~46 KiB of multiples each
    G = base.G.copy()
    G[0, :] = 0
    G[0, 0] = 1  # a weight-1 codeword: the search certifies d = 1 after its first pass
    code = inputs.Code(base.p, base.n, base.k, G)
    with pytest.raises(B.FpcodeError) as e:
        B.fpcode_min_distance_noalloc(code.p, code.n, code.k, code.G)
    assert e.value.status == B.EINVAL and "scratch" in str(e.value)
    d, w = B.fpcode_min_distance(code.p, code.n, code.k, code.G)
    assert d == 1
    _check_codeword(code, d, w)
