"""Host logic of the launch-shape autotuner: the search keeps the fastest
candidate, the result is cached under its key and reused without a new
search, and a refresh searches again. The timing function is a fake."""
import json

from paper_2109_13176_gb300 import tune


def fake_run(best):
    calls = []

    def run(c):
        calls.append(c)
        return 1.0 if c == best else 2.0 + 0.01 * c[0]
    return run, calls


def test_search_picks_the_fastest():
    run, calls = fake_run((12, 128, 0, 0))
    best, table = tune.search(run, repeats=2)
    assert best == (12, 128, 0, 0)
    assert len(calls) == 3 * len(tune.CANDIDATES)  # one warm-up + two timed each
    assert table["12/128/0/0"] == 1e6


def test_cache_reuse_and_refresh(tmp_path, monkeypatch):
    monkeypatch.setenv("GVOM_TUNE_CACHE", str(tmp_path / "t.json"))
    run, calls = fake_run((8, 256, 0, 1))
    best, entry = tune.tuned("dev|map|1x1x1@0.2|~1", run, repeats=1)
    assert best == (8, 256, 0, 1) and calls
    stored = json.loads((tmp_path / "t.json").read_text())
    assert stored["dev|map|1x1x1@0.2|~1"]["best"] == [8, 256, 0, 1]
    calls.clear()
    best2, _ = tune.tuned("dev|map|1x1x1@0.2|~1", run, repeats=1)
    assert best2 == (8, 256, 0, 1) and not calls          # from the cache
    run3, calls3 = fake_run((16, 128, 0, 1))
    best3, _ = tune.tuned("dev|map|1x1x1@0.2|~1", run3, repeats=1, refresh=True)
    assert best3 == (16, 128, 0, 1) and calls3           # searched again


def test_unwritable_cache_is_not_an_error(tmp_path, monkeypatch):
    (tmp_path / "afile").write_text("not a directory")
    monkeypatch.setenv("GVOM_TUNE_CACHE", str(tmp_path / "afile" / "t.json"))
    run, _ = fake_run((12, 128, 0, 0))
    best, _ = tune.tuned("k", run, repeats=1)
    assert best == (12, 128, 0, 0)


def test_cached_entry_of_another_shape_is_searched_again(tmp_path, monkeypatch):
    # a table written when candidates had three fields is not reused for
    # four-field candidates (the fused-ingest flag)
    monkeypatch.setenv("GVOM_TUNE_CACHE", str(tmp_path / "t.json"))
    (tmp_path / "t.json").write_text(json.dumps({"k": {"best": [8, 256, 0], "us": {}}}))
    run, calls = fake_run((24, 256, 0, 1))
    best, _ = tune.tuned("k", run, repeats=1)
    assert best == (24, 256, 0, 1) and calls
    run_b, calls_b = fake_run((8, 256, 0))
    best_b, _ = tune.tuned("k", run_b, candidates=tune.WALK_CANDIDATES, repeats=1, refresh=True)
    assert best_b == (8, 256, 0) and len(calls_b) == 2 * len(tune.WALK_CANDIDATES)


def test_apply_walk_passes_the_fused_flag():
    # a three-field candidate (a batch's walk shape) keeps the two-kernel
    # ingest; a four-field one sets the fused-ingest flag it names
    calls = []

    class FakeMap:
        def set_tuning(self, *args, **kw):
            calls.append((args, kw))

    tune.apply_walk(FakeMap(), (16, 256, 0))
    tune.apply_walk(FakeMap(), (48, 128, 0, 1))
    assert calls == [((16, 256, 0), {"fused_ingest": 0}), ((48, 128, 0), {"fused_ingest": 1})]
    assert all(len(c) == 4 for c in tune.CANDIDATES) and all(len(c) == 3 for c in tune.WALK_CANDIDATES)
    assert {c[3] for c in tune.CANDIDATES} == {0, 1}
