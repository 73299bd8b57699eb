"""Host-side logic of the autotuner's size classes (no GPU)."""
from paper_1205_4883_gb300 import autotune


def test_class_keys_cover_the_bands():
    assert autotune.class_key(0, 10) == "0/0"
    assert autotune.class_key(10**12, 10**12 + 10**6) == "3/3"
    assert autotune.class_key(10**14, 10**14 + 10**8) == "4/4"
    assert autotune.class_key(10**14, 10**14 + 10**9) == "4/4"
    assert autotune.class_key(5 * 10**9, 5 * 10**9 + 2 * 10**4) == "1/1"
    keys = {autotune.class_key(10 ** a, 10 ** a + 10 ** b) for a in range(0, 15) for b in range(0, 9)}
    assert keys == {f"{i}/{j}" for i in range(len(autotune.LO_BANDS)) for j in range(len(autotune.W_BANDS))}


def test_plan_lookup_range_params_and_missing_table(tmp_path):
    t = {"classes": {"3/3": {"seg_bytes": 65536, "wheel": 210, "note": "ignored"}}}
    assert autotune.plan_for(t, 10**12, 10**12 + 10**6) == {"seg_bytes": 65536, "wheel": 210, "note": "ignored"}
    assert autotune.plan_for(t, 0, 10) == {}
    assert autotune.range_params(t, [10**12, 0], [10**12 + 10**6, 10]) == [{"seg_bytes": 65536, "wheel": 210}, {}]
    assert autotune.load_table(str(tmp_path / "none.json")) == {"classes": {}}


def test_samples_stay_in_band():
    los, his = autotune.sample_class((6, 10), (3, 5), 50, seed=1, hi_max=10**14)
    for lo, hi in zip(los, his):
        assert 10**6 <= lo < 10**10 and 10**3 <= hi - lo < 10**5


def test_candidates_are_valid_range_parameters():
    for v in autotune.CANDIDATES["seg_bytes"]:
        assert v == 0 or (1024 <= v <= 229376 and v % 32 == 0)
    assert set(autotune.CANDIDATES["wheel"]) <= {0, 30, 210}
    assert all(c[0] == 0 for c in autotune.CANDIDATES.values())  # the defaults are always a candidate
