"""airg_dot_exact_noalloc: the correctly rounded dot product for callers that
cannot allocate device memory -- code running inside a framework whose
caching pool has reserved the device's memory (a cudaMalloc behind the
pool's back can fail or fragment it), or a latency-critical loop in which
cudaMalloc / cudaFree would synchronise the device.  Checked through the C
ABI against the allocating airg_dot_exact.

Collected last on purpose; it passes when run alone in a fresh process and
after the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2508_17517_gb300 as G  # noqa: E402

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.build()
    G.lib()


def test_dot_exact_noalloc_two_calls_match_allocating_entry_point():
    _need_gpu()
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


def test_dot_exact_noalloc_nan_then_finite_and_empty():
    """The inf/nan flag word is shared scratch too: a call on a NaN input
    must not leak into the next call.  n = 0 writes +0.0."""
    _need_gpu()
    rng = np.random.default_rng(12)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    x = torch.tensor(rng.standard_normal(4099), device="cuda")
    y = torch.tensor(rng.standard_normal(4099), device="cuda")
    xn = x.clone()
    xn[17] = float("nan")
    G.airg_dot_exact_noalloc(xn, y, out)
    torch.cuda.synchronize()
    assert np.isnan(out.item())
    G.airg_dot_exact_noalloc(x, y, out)
    torch.cuda.synchronize()
    assert out.item() == G.airg_dot_exact(x, y)
    out.fill_(-1.0)
    L = G.lib()
    assert L.airg_dot_exact_noalloc(0, None, None, ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()
    v = out.item()
    assert v == 0.0 and np.copysign(1.0, v) == 1.0


def test_dot_exact_noalloc_allocates_nothing():
    """After a warm-up call, further calls leave both torch's pool and the
    driver's free-memory figure unchanged."""
    _need_gpu()
    rng = np.random.default_rng(13)
    x = torch.tensor(rng.standard_normal(1 << 20), device="cuda")
    y = torch.tensor(rng.standard_normal(1 << 20), device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    G.airg_dot_exact_noalloc(x, y, out)
    torch.cuda.synchronize()
    pool0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(20):
        G.airg_dot_exact_noalloc(x, y, out)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == pool0
    assert torch.cuda.mem_get_info()[0] == free0


def test_dot_exact_noalloc_rejects_bad_tensors():
    _need_gpu()
    x = torch.ones(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        G.airg_dot_exact_noalloc(x.float(), x, out)
    with pytest.raises(ValueError):
        G.airg_dot_exact_noalloc(x, x[:3], out)
    with pytest.raises(ValueError):
        G.airg_dot_exact_noalloc(x, x, out[:0])
    with pytest.raises(ValueError):
        G.airg_dot_exact_noalloc(x, x, out.cpu())
