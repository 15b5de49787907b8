"""airg_operator_layout_info: the storage and row-kernel variant of every
solve-phase operator, as the setup laid it out and its timing picked it,
checked against the hierarchy's own sizes and against the variant that the
AIRG_* overrides force."""
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


def _setup(n, **opts):
    w = workload("c2", n=n)
    vx, vy = velocity(w["theta"])
    pg = G.airg_problem_advection2d(w["nx"], w["ny"], vx, vy)
    o = dict(w["opts"])
    o.update(opts)
    h = G.airg_setup(pg["rowptr"], pg["col"], pg["val"], G.airg_options_default(**o))
    return h, pg


@pytest.mark.parametrize("precision", [G.AIRG_FP64, G.AIRG_MIXED_FP32, G.AIRG_MIXED_FP32_BF16R])
def test_layout_matches_hierarchy(precision):
    h, pg = _setup(512, precision=precision)
    info = G.airg_setup_info(h)
    L = info["levels"] - 1
    vb = 8 if precision == G.AIRG_FP64 else 4
    rows = G.airg_row_kernel_choices(h)
    got = {(lev, name): d for lev, name, d in rows}
    top = got[(0, "top")]
    assert top["n_rows"] == top["n_cols"] == info["n"][0]
    assert top["nnz"] == pg["col"].numel() and top["value_bytes"] == 8 and top["dense_diagonal"] == 1
    co = got[(L, "coarse")]
    assert co["n_rows"] == co["n_cols"] == info["n"][L] and co["nnz"] == info["nnz_a"][L]
    assert co["value_bytes"] == vb
    for lev in range(L):
        nf, nc = info["n_f"][lev], info["n"][lev] - info["n_f"][lev]
        aff, m, z = got[(lev, "A_ff")], got[(lev, "M")], got[(lev, "Z")]
        assert (aff["n_rows"], aff["n_cols"]) == (nf, nf) and aff["dense_diagonal"] == 1
        assert (m["n_rows"], m["n_cols"]) == (nf, nc)
        assert (z["n_rows"], z["n_cols"]) == (nc, nf)
        assert aff["value_bytes"] == m["value_bytes"] == vb
        assert z["value_bytes"] == (2 if precision == G.AIRG_MIXED_FP32_BF16R else vb)
        # nothing but the default F-point smoother's operators is kept
        assert (lev, "Ainv") not in got and (lev, "A_cc") not in got
    for (lev, name), d in got.items():
        k, r = d["warps_per_slice"], d["r"]
        assert k in (1, 2, 4, 8), (lev, name, k)
        assert r in ((1, 2, 4) if k == 1 else (4, 8, 16)), (lev, name, r)
        assert d["resident_grid"] in (0, 1)
        # SELL-32: every slice padded to its longest row
        off = d["nnz"] - (d["n_rows"] if d["dense_diagonal"] else 0)
        assert d["padded"] % 32 == 0 and d["padded"] >= off, (lev, name)
        assert d["index_bytes"] in (2, 4)
        if d["n_cols"] <= 65536 and d["padded"] > 0:
            assert d["index_bytes"] == 2 and d["slice_bases"] == 0, (lev, name)
        else:
            assert d["slice_bases"] == (1 if d["index_bytes"] == 2 else 0), (lev, name)
    # the 512^2 top level has 262,144 columns: some operator needs slice bases
    assert any(d["slice_bases"] for d in got.values())
    G.airg_free(h)


def test_layout_reports_forced_variants(monkeypatch):
    monkeypatch.setenv("AIRG_ROWS_PER_WARP", "2")
    monkeypatch.setenv("AIRG_LOADS_PER_LANE", "8")
    monkeypatch.setenv("AIRG_PERSIST_GRID", "1")
    monkeypatch.setenv("AIRG_COL16", "0")
    h, _ = _setup(256, precision=G.AIRG_MIXED_FP32)
    for lev, name, d in G.airg_row_kernel_choices(h):
        assert d["r"] == (2 if d["warps_per_slice"] == 1 else 8), (lev, name)
        assert d["resident_grid"] == 1 and d["index_bytes"] == 4 and d["slice_bases"] == 0, (lev, name)
    G.airg_free(h)


def test_layout_assembled_and_c_point_operators():
    h, _ = _setup(128, smoother=G.AIRG_SMOOTH_ASSEMBLED, smooth_type=G.AIRG_SMOOTH_FCF)
    info = G.airg_setup_info(h)
    L = info["levels"] - 1
    got = {(lev, name): d for lev, name, d in G.airg_row_kernel_choices(h)}
    for lev in range(L):
        nf, n = info["n_f"][lev], info["n"][lev]
        assert got[(lev, "Ainv")]["n_rows"] == nf
        assert (got[(lev, "C_rows")]["n_rows"], got[(lev, "C_rows")]["n_cols"]) == (n - nf, n)
        assert (got[(lev, "F_rows")]["n_rows"], got[(lev, "F_rows")]["n_cols"]) == (nf, n)
    G.airg_free(h)


def test_layout_rejects_bad_slots():
    h, _ = _setup(64)
    L = G.airg_setup_info(h)["levels"] - 1
    for level, op in [(1, "top"), (0, "coarse"), (L, "A_ff"), (L + 1, "Z"), (-1, "M"), (0, 10), (0, -1)]:
        with pytest.raises(G.AirgError):
            G.airg_operator_layout_info(h, level, op)
    G.airg_free(h)
