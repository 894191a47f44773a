"""Host-only behaviour of the tuning cache of the combination path: set/get,
validation, removal, the planner honouring the knobs (workspace size follows
rows_per_task) and the save/load round trip of the cache file."""
import pytest

import paper_1303_2285_gb300 as cov


@pytest.fixture(autouse=True)
def _clean_cache():
    cov.tuning_clear()
    yield
    cov.tuning_clear()


def test_defaults_not_cached():
    knobs, cached = cov.tuning_get("c64", 1024, 1024, 16, 16)
    assert not cached
    assert knobs["lag_group"] in (4, 8, 16)
    assert knobs["rows_per_task"] % 8 == 0
    assert 1 <= knobs["reseed_interval"] <= 32


def test_set_get_remove():
    k = {"lag_group": 4, "rows_per_task": 24, "reseed_interval": 4, "kernels": 4, "tile_cols": 32}
    cov.tuning_set("c64", 300, 200, 8, 6, k)
    got, cached = cov.tuning_get("c64", 300, 200, 8, 6)
    assert cached and got == k
    # other dtype / shape unaffected
    assert not cov.tuning_get("c128", 300, 200, 8, 6)[1]
    assert not cov.tuning_get("c64", 300, 201, 8, 6)[1]
    cov.tuning_set("c64", 300, 200, 8, 6, None)
    assert not cov.tuning_get("c64", 300, 200, 8, 6)[1]


@pytest.mark.parametrize("bad", [
    {"lag_group": 5, "rows_per_task": 24, "reseed_interval": 4, "kernels": 4},
    {"lag_group": 8, "rows_per_task": 20, "reseed_interval": 4, "kernels": 4},
    {"lag_group": 8, "rows_per_task": 0, "reseed_interval": 4, "kernels": 4},
    {"lag_group": 8, "rows_per_task": 264, "reseed_interval": 4, "kernels": 4},
    {"lag_group": 8, "rows_per_task": 24, "reseed_interval": 0, "kernels": 4},
    {"lag_group": 8, "rows_per_task": 24, "reseed_interval": 33, "kernels": 4},
    {"lag_group": 8, "rows_per_task": 24, "reseed_interval": 4, "kernels": 4, "tile_cols": 48},
])
def test_invalid_knobs_rejected(bad):
    with pytest.raises(cov.CovError) as e:
        cov.tuning_set("c64", 300, 200, 8, 6, bad)
    assert e.value.code == 1


def test_kernels_knob():
    with pytest.raises(cov.CovError):
        cov.tuning_set("c64", 300, 200, 8, 6,
                       {"lag_group": 8, "rows_per_task": 24, "reseed_interval": 4, "kernels": 2})
    with pytest.raises(cov.CovError):  # the fused kernel is FP32 only
        cov.tuning_set("c128", 300, 200, 8, 6,
                       {"lag_group": 8, "rows_per_task": 24, "reseed_interval": 4, "kernels": 1})
    cov.tuning_set("c64", 300, 200, 8, 6,
                   {"lag_group": 8, "rows_per_task": 24, "reseed_interval": 4, "kernels": 0})
    assert cov.tuning_get("c64", 300, 200, 8, 6)[0]["kernels"] == 1  # default: fused
    assert cov.tuning_get("c64", 2048, 512, 32, 32)[0]["kernels"] == 4  # large reductions
    assert cov.tuning_get("c128", 300, 200, 8, 6)[0]["kernels"] == 4


def test_fp64_lag_group_16_rejected():
    with pytest.raises(cov.CovError):
        cov.tuning_set("c128", 300, 200, 8, 6,
                       {"lag_group": 16, "rows_per_task": 24, "reseed_interval": 4, "kernels": 4})
    cov.tuning_set("c64", 300, 200, 8, 6,
                   {"lag_group": 16, "rows_per_task": 24, "reseed_interval": 4, "kernels": 4})


def test_unsupported_shape():
    # P above 32: the combination path does not take it
    with pytest.raises(cov.CovError) as e:
        cov.tuning_set("c64", 40, 40, 33, 2,
                       {"lag_group": 8, "rows_per_task": 24, "reseed_interval": 4, "kernels": 4})
    assert e.value.code == 5
    # no inner rows or columns: taken
    cov.tuning_set("c64", 10, 10, 8, 8,
                   {"lag_group": 8, "rows_per_task": 24, "reseed_interval": 4, "kernels": 4})
    cov.tuning_clear()


def test_planner_honours_rows_per_task():
    # the per-row-block partial sums scale with the number of row blocks,
    # so fewer rows per task means a larger workspace
    base = cov.workspace_size("c64", 1024, 1024, 16, 16, "recurrence")
    cov.tuning_set("c64", 1024, 1024, 16, 16,
                   {"lag_group": 8, "rows_per_task": 16, "reseed_interval": 8, "kernels": 1})
    small = cov.workspace_size("c64", 1024, 1024, 16, 16, "recurrence")
    assert small > base
    assert cov.tuning_get("c64", 1024, 1024, 16, 16)[0]["rows_per_task"] == 16
    # the planner clamps rows_per_task to what a shared-memory tile holds
    cov.tuning_set("c64", 1024, 1024, 32, 32,
                   {"lag_group": 8, "rows_per_task": 256, "reseed_interval": 8, "kernels": 1})
    assert cov.tuning_get("c64", 1024, 1024, 32, 32)[0]["rows_per_task"] < 256


def test_autotune_workspace_bound():
    need = cov.workspace_size("c64", 1024, 1024, 16, 16, "recurrence")
    lib = cov.load()
    import ctypes
    out = ctypes.c_size_t(0)
    assert lib.cov_autotune_workspace_size(0, 1024, 1024, 16, 16, ctypes.byref(out)) == 0
    assert out.value >= need


def test_save_load_round_trip(tmp_path):
    a = {"lag_group": 4, "rows_per_task": 32, "reseed_interval": 2, "kernels": 1, "tile_cols": 64}
    b = {"lag_group": 8, "rows_per_task": 64, "reseed_interval": 16, "kernels": 4, "tile_cols": 32}
    cov.tuning_set("c64", 512, 256, 12, 10, a)
    cov.tuning_set("c128", 100, 90, 5, 7, b)
    f = tmp_path / "tune.txt"
    cov.tuning_save(str(f))
    cov.tuning_clear()
    assert not cov.tuning_get("c64", 512, 256, 12, 10)[1]
    assert cov.tuning_load(str(f)) == 2
    assert cov.tuning_get("c64", 512, 256, 12, 10) == (a, True)
    assert cov.tuning_get("c128", 100, 90, 5, 7) == (b, True)


def test_load_errors(tmp_path):
    with pytest.raises(cov.CovError):
        cov.tuning_load(str(tmp_path / "missing.txt"))
    bad = tmp_path / "bad.txt"
    bad.write_text("# header\n8 100 100 4 4\n")
    with pytest.raises(cov.CovError):
        cov.tuning_load(str(bad))


def test_tile_cols_knob_and_default():
    # 2048 x 512 with a 32 x 32 window: a 64-column tile holds 87 rows besides
    # its halo, so the default tile is 32 columns (and 128-row tasks fit)
    knobs, cached = cov.tuning_get("c64", 2048, 512, 32, 32)
    assert not cached and knobs["tile_cols"] == 32 and knobs["rows_per_task"] == 128
    # 1024 x 1024 with 16 x 16 keeps 64-column tiles
    assert cov.tuning_get("c64", 1024, 1024, 16, 16)[0]["tile_cols"] == 64
    cov.tuning_set("c64", 2048, 512, 32, 32, {"lag_group": 16, "rows_per_task": 64,
                                              "reseed_interval": 8, "kernels": 4, "tile_cols": 64})
    got = cov.tuning_get("c64", 2048, 512, 32, 32)[0]
    assert got["tile_cols"] == 64 and got["rows_per_task"] == 64


def test_load_reads_four_knob_lines(tmp_path):
    # a file written before the tile_cols knob: the same line without it
    cov.tuning_set("c64", 512, 256, 12, 10, {"lag_group": 4, "rows_per_task": 32,
                                             "reseed_interval": 2, "kernels": 1, "tile_cols": 64})
    f = tmp_path / "old.txt"
    cov.tuning_save(str(f))
    cov.tuning_clear()
    lines = [ln for ln in f.read_text().splitlines() if not ln.startswith("#")]
    assert len(lines) == 1
    f.write_text("# elem N M P Q sms G TRB L K\n" + " ".join(lines[0].split()[:10]) + "\n")
    assert cov.tuning_load(str(f)) == 1
    got, cached = cov.tuning_get("c64", 512, 256, 12, 10)
    assert cached and got["lag_group"] == 4 and got["rows_per_task"] == 32
