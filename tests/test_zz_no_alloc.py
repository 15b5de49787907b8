"""airg_dot_exact_noalloc: the allocation-free dot product for callers that
cannot allocate device memory (frameworks whose caching pool has reserved the
device's memory, latency-critical loops where cudaMalloc would synchronise the
device), checked against the allocating airg_dot_exact.

Collected last on purpose, and runs either alone or after the other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2508_17517_gb300 as G  # noqa: E402

pytestmark = pytest.mark.gpu


def test_dot_exact_noalloc_two_calls_match_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.build()
    G.lib()
    rng = np.random.default_rng(11)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    # two calls in a row: the second must not see the first call's accumulator
    for n in (1_000_003, 77):
        x = torch.tensor(rng.standard_normal(n) * np.exp2(rng.integers(-30, 30, n)), device="cuda")
        y = torch.tensor(rng.standard_normal(n), device="cuda")
        G.airg_dot_exact_noalloc(x, y, out)
        torch.cuda.synchronize()
        ref = G.airg_dot_exact(x, y)
        # both return the correctly rounded value, so the tolerance is zero
        assert out.item() == ref


def test_dot_exact_noalloc_rejects_n_beyond_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    x = torch.ones(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(G.AirgError) as e:
        G.airg_dot_exact_noalloc(x, x, out, n=1 << 31)   # checked before any GPU work
    assert e.value.status == 1 and "2^31" in str(e.value)
