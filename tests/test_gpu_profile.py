"""Solve-kernel timing and the setup breakdown (through the C ABI).

Timing must not change a result bit; timing one kernel group alone must see
exactly the launches that the per-kernel pass attributes to it; the setup
phases must account for the setup's wall time.
"""
import pytest

torch = pytest.importorskip("torch")

import paper_2508_17517_gb300 as G  # noqa: E402
from synthetic import velocity, workload  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.build()
    G.lib()


@pytest.mark.parametrize("prec", [G.AIRG_FP64, G.AIRG_MIXED_FP32])
def test_group_timing_counts_and_changes_no_bit(prec):
    w = workload("c2", n=384)
    vx, vy = velocity(w["theta"])
    pg = G.airg_problem_advection2d(w["nx"], w["ny"], vx, vy)
    h = G.airg_setup(pg["rowptr"], pg["col"], pg["val"], G.airg_options_default(precision=prec, **w["opts"]))
    info = G.airg_setup_info(h)
    b = G.airg_assemble_rhs_advection2d(pg, torch.tensor(w["g"][0], device="cuda"))
    x0, i0 = G.airg_solve(h, b, rtol=1e-10)
    G.airg_profile(h, True)
    x1, _ = G.airg_solve(h, b, rtol=1e-10)
    per = G.airg_profile_read_level(h, info["levels"])
    G.airg_profile(h, False)
    assert torch.equal(x0, x1)
    L = info["levels"] - 1
    for kind, level in (("coarse_newton", L), ("f_smoother", 0), ("krylov_vectors", 0)):
        G.airg_profile_group(h, kind, level)
        x2, _ = G.airg_solve(h, b, rtol=1e-10)
        got = G.airg_profile_read_level(h, info["levels"])
        G.airg_profile(h, False)
        assert torch.equal(x0, x2), kind
        assert set(got) == {(kind, level)}, (kind, sorted(got))
        ms, nl, nb, nf = got[(kind, level)]
        assert nl == per[(kind, level)][1] and nb == per[(kind, level)][2] and nf == per[(kind, level)][3]
        assert ms > 0
    # a V-cycle group is one event pair per V-cycle: the whole run of its
    # launches, so it cannot take longer than the solve
    G.airg_profile_group(h, "coarse_newton", L)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    G.airg_solve(h, b, rtol=1e-10)
    ev1.record()
    ev1.synchronize()
    ms = G.airg_profile_read_level(h, info["levels"])[("coarse_newton", L)][0]
    G.airg_profile(h, False)
    assert 0 < ms < ev0.elapsed_time(ev1)
    with pytest.raises(G.AirgError):
        G.airg_profile_group(h, 7, 0)
    with pytest.raises(G.AirgError):
        G.airg_profile_group(h, 0, 65)


def test_setup_breakdown_accounts_for_the_setup():
    w = workload("c2", n=512)
    vx, vy = velocity(w["theta"])
    pg = G.airg_problem_advection2d(w["nx"], w["ny"], vx, vy)
    h = G.airg_setup(pg["rowptr"], pg["col"], pg["val"], G.airg_options_default(**w["opts"]))
    info = G.airg_setup_info(h)
    br = info["setup_breakdown_ms"]
    assert list(br) == G.SETUP_PHASES
    assert all(v >= 0 for v in br.values())
    tot = sum(br.values())
    # the phases cover everything but problem copies and validation
    assert 0.6 * info["setup_ms"] <= tot <= info["setup_ms"] * (1 + 1e-9), (tot, info["setup_ms"])
    for k in ("cf_split", "smoother_poly", "restrictor", "rap", "coarse_poly", "solve_layout"):
        assert br[k] > 0, k
    assert info["exact_dots"] > 0
