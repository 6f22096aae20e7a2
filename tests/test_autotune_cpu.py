"""Host logic of the launch-shape autotuner, on CPU: the batch buckets and
the persistent choice table."""
import json

from paper_2402_14670_gb300 import autotune


def test_bucket_edges():
    # size class from the mean input tracks per event (edges 32, 64, 128, 256)
    assert autotune.bucket_of(1000, 32000) == (0, 9)
    assert autotune.bucket_of(1000, 32001) == (1, 9)
    assert autotune.bucket_of(1000, 256000) == (3, 9)
    assert autotune.bucket_of(1000, 256001) == (4, 9)
    # event-count scale: floor(log2(n_events)); an empty batch is class 0
    assert autotune.bucket_of(1024, 0) == (0, 10)
    assert autotune.bucket_of(1023, 0) == (0, 9)
    assert autotune.bucket_of(0, 0) == (0, 0)


def test_choice_table_round_trip(tmp_path):
    path = tmp_path / "tune.json"
    key = autotune.Autotuner._key(autotune.bucket_of(100_000, 8_000_000))
    choice = dict(queue=0, blocks_per_sm=2)
    path.write_text(json.dumps({key: choice}))
    t = autotune.Autotuner(cache_path=str(path))
    assert t.lookup(100_000, 8_000_000) == choice
    # another bucket is not in the table
    assert t.lookup(100, 100) is None
    # every candidate is a valid tuning (queue 0..2; the stage pipeline first,
    # with its per-stage occupancy knobs)
    assert autotune.CANDIDATES[0] == dict(queue=0)
    assert all(c.get("queue", 0) in (0, 1, 2) for c in autotune.CANDIDATES)
    from paper_2402_14670_gb300 import lf
    names = {f for f, _ in lf.lf_tuning._fields_}
    assert all(set(c) <= names for c in autotune.CANDIDATES)
    assert sum(1 for c in autotune.CANDIDATES if c.get("queue", 0) == 0 and len(c) > 1) >= 4


def test_candidates_applicable_to_the_no_ut_variant():
    """The no-UT variant runs on the stage pipeline without the triplet
    pre-filter; the tuner skips the rest for it, and keeps every candidate
    for VELO-UT input."""
    from paper_2402_14670_gb300 import autotune
    velo_ut = [c for c in autotune.CANDIDATES if autotune.applicable(c, dict(no_ut=0))]
    assert velo_ut == autotune.CANDIDATES
    no_ut = [c for c in autotune.CANDIDATES if autotune.applicable(c, dict(no_ut=1))]
    assert no_ut and all(c.get("queue", 0) == 0 and not c.get("triplet_prefilter", 0) for c in no_ut)
    assert any(c.get("triplet_prefilter", 0) for c in autotune.CANDIDATES)
