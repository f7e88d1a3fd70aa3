"""The autotuner's search, candidate grid and cache (no GPU: the timing
function and the parameter setter are stand-ins)."""
import json

from paper_1703_10440_gb300 import mgsa, tune


def test_bucket_key_groups_nearby_shapes():
    a = tune.bucket_key("GB300", "hp", 262144, 64, 1308672)
    assert a == tune.bucket_key("GB300", "hp", 262000, 63, 1300000)
    assert a != tune.bucket_key("GB300", "hp", 262144 * 4, 64, 1308672 * 4)
    assert a != tune.bucket_key("GB300", "ha", 262144, 64, 1308672)
    assert a != tune.bucket_key("GB300", "hp", 262144, 64, 1308672 * 40)


def test_candidates_skip_what_cannot_matter():
    hp = tune.candidates(tune.SINGLE_SPACE, "hp", rows_per_cta_max=None)
    ha = tune.candidates(tune.SINGLE_SPACE, "ha", rows_per_cta_max=None)
    assert len(hp) == 2 * 2 * 4 * 2 and len(ha) == 2 * 4 * 2  # the panel only matters with a block product
    assert all(c["spmm_panel"] == 8 for c in ha)
    small = tune.candidates(tune.SINGLE_SPACE, "hp", rows_per_cta_max=1024)
    assert all(c["chunk_rows"] == 0 for c in small)  # a slab of <= 1024 rows is one chunk anyway


def test_search_keeps_the_median_fastest_and_caches(tmp_path):
    path = tmp_path / "tune.json"
    t = tune.Tuner(str(path))
    space = tune.candidates(tune.SINGLE_SPACE, "hp")
    calls = []

    def fake_ms(p):  # deterministic cost surface with one outlier repetition
        calls.append(p)
        base = 1.0 + 0.1 * p["row_mode"] + 0.01 * p["spmm_panel"] + abs(p["min_rows"] - 64) / 1000.0
        return base + (5.0 if len(calls) % 7 == 0 else 0.0)

    rec = t.search("k", space, fake_ms, reps=3)
    assert rec["params"] == {"row_mode": 1, "spmm_panel": 4, "min_rows": 64, "chunk_rows": 0}
    assert len(calls) == 3 * len(space)
    t.save()
    again = tune.Tuner(str(path))
    assert again.lookup("k") == rec["params"]
    assert again.lookup("missing") is None
    assert json.loads(path.read_text())["k"]["ms"] == rec["ms"]


def test_apply_and_reset_set_the_library_parameters():
    seen = []
    tune.apply(7, {"row_mode": 2, "spmm_panel": 4, "min_rows": 32}, set_param=lambda h, p, v: seen.append((h, p, v)))
    assert seen == [(7, mgsa.MGSA_PARAM_ROW_MODE, 2), (7, mgsa.MGSA_PARAM_SPMM_PANEL, 4),
                    (7, mgsa.MGSA_PARAM_MIN_ROWS_PER_CTA, 32)]
    seen.clear()
    tune.reset(7, ["chunk_rows", "batch_ctas"], set_param=lambda h, p, v: seen.append((h, p, v)))
    assert seen == [(7, mgsa.MGSA_PARAM_CHUNK_ROWS, 0), (7, mgsa.MGSA_PARAM_BATCH_CTAS, 0)]
