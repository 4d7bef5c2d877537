"""Host logic of the supercell / threads autotuner (no GPU: a fake timer)."""
import pytest

from paper_1606_02862_gb300 import autotune


def test_feasible_keeps_only_dividing_supercells():
    grids = [(16, 16, 16), (24, 24, 24)]
    got = autotune.feasible(autotune.CANDIDATES, grids)
    assert ((4, 4, 4), 128) in got and ((8, 8, 4), 256) in got
    grids = [(12, 12, 12)]
    assert all(sc == (4, 4, 4) for sc, _ in autotune.feasible(autotune.CANDIDATES, grids))


def test_tune_picks_fastest_and_caches(tmp_path):
    cache = str(tmp_path / "cache.json")
    speed = {((4, 4, 4), 128): 3.0, ((8, 8, 4), 256): 1.5, ((8, 4, 4), 128): 2.0}
    calls = []

    def timer(make_ctx, sc, t, steps, warmup):
        calls.append((sc, t))
        if (sc, t) == ((8, 4, 4), 128):
            raise RuntimeError("does not fit")
        return speed[(sc, t)]

    cands = list(speed)
    sc, t, trials = autotune.tune(None, cands, key="k1", cache_path=cache, gpu_name="X", timer=timer)
    assert (sc, t) == ((8, 8, 4), 256)
    assert len(trials) == 3 and sum(not tr.ok for tr in trials) == 1
    # second call: served from the cache, nothing timed
    calls.clear()
    sc2, t2, trials2 = autotune.tune(None, cands, key="k1", cache_path=cache, gpu_name="X", timer=timer)
    assert (sc2, t2) == (sc, t) and trials2 == [] and calls == []
    # another GPU name is another key
    autotune.tune(None, cands, key="k1", cache_path=cache, gpu_name="Y", timer=timer)
    assert len(calls) == 3


def test_tune_raises_when_nothing_runs(tmp_path):
    def timer(*_a):
        raise RuntimeError("no")

    with pytest.raises(RuntimeError, match="no candidate ran"):
        autotune.tune(None, [((4, 4, 4), 128)], timer=timer, cache_path=str(tmp_path / "c.json"))


def test_signature_depends_on_workload():
    a = autotune.signature([(16, 16, 16)], 8, [2], 1)
    b = autotune.signature([(16, 16, 16)], 4, [2], 1)
    c = autotune.signature([(16, 16, 16)], 8, [1], 1)
    assert len({a, b, c}) == 3
    assert a == autotune.signature([(16, 16, 16)], 8.0, [2], 1)
