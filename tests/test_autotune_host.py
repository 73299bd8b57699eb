"""Host-side logic of the autotuner's size classes (no GPU)."""
from paper_1205_4883_gb300 import autotune


def test_class_keys_cover_the_bands():
    assert autotune.class_key(0, 10) == "0/0"
    assert autotune.class_key(10**12, 10**12 + 10**6) == "1/1"
    assert autotune.class_key(10**14, 10**14 + 10**8) == "2/2"
    assert autotune.class_key(10**14, 10**14 + 10**9) == "2/3"
    assert autotune.class_key(5 * 10**9, 5 * 10**9 + 2 * 10**7) == "0/2"


def test_plan_lookup_and_missing_table(tmp_path):
    t = {"classes": {"1/1": {"segment_bytes": 65536}}}
    assert autotune.plan_for(t, 10**12, 10**12 + 10**6) == {"segment_bytes": 65536}
    assert autotune.plan_for(t, 0, 10) == {}
    assert autotune.load_table(str(tmp_path / "none.json")) == {"classes": {}}


def test_samples_stay_in_band():
    los, his = autotune.sample_class((6, 10), (3, 5), 50, seed=1, hi_max=10**14)
    for lo, hi in zip(los, his):
        assert 10**6 <= lo < 10**10 and 10**3 <= hi - lo < 10**5
