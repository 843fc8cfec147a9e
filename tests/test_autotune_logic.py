"""Host logic of the schedule autotuner (no GPU: the timing is faked).

The staged search must keep the best candidate of each stage as the base of
the next, return the overall minimum, put the library's schedule back, and
store / re-apply results per (k, size bucket).
"""
import pytest

from paper_2201_11655_b300 import autotune, vdmc


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2201_11655_b300 import build
    build.build()
    vdmc.load()


def fake_cost():
    s = vdmc.get_schedule()
    return (100.0 + abs(s["hub_min_l"] - 16) + abs(s["a_chunk"] - 4) + (0 if s["hub_warps"] == 32 else 5)
            + (0 if (s["hub_split"], s["hub_split_roots"]) == (2, 32) else 3))


def test_staged_search_picks_minimum_and_restores(monkeypatch):
    monkeypatch.setattr(autotune, "time_count", lambda g, k, reps=1: fake_cost())
    old = vdmc.get_schedule()
    best, ms, timings = autotune.tune(None, 4, log=lambda *a: None)
    assert (best["hub_min_l"], best["a_chunk"], best["hub_warps"], best["hub_split"], best["hub_split_roots"]) == \
        (16, 4, 32, 2, 32)
    assert ms == 100.0 and min(timings.values()) == 100.0
    assert len(timings) == len({*map(str, autotune.STAGE1 + autotune.STAGE2 + autotune.STAGE3)})
    assert vdmc.get_schedule() == old


def test_bucket_names():
    assert autotune.bucket(1_000_000, 9_908_908) == "n2^19_d2^4"
    assert autotune.bucket(1, 0) == "n2^0_d2^0"


def test_save_and_apply_roundtrip(tmp_path):
    old = vdmc.get_schedule()
    try:
        sched = dict(old, hub_min_l=24, hub_warps=32, hub_split=3, hub_split_roots=7)
        path = str(tmp_path / "tuned.json")
        autotune.save_tuned("k4/" + autotune.bucket(5000, 40000), sched, 12.5, {"workload": "w"}, path)
        assert autotune.apply_tuned(3, 5000, 40000, path) is None  # other k: nothing applied
        assert vdmc.get_schedule() == old
        assert autotune.apply_tuned(4, 5000, 40000, path) == sched
        assert vdmc.get_schedule() == sched
    finally:
        vdmc.set_schedule(**old)
