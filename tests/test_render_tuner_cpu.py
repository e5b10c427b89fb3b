"""Host logic of the render autotuner (no GPU): classes, `reps` interleaved
trials per class and candidate, the lowest median kept."""
from paper_2405_20067_gb300.render import CANDIDATES, Autotuner, frame_class


def test_frame_classes_round_to_powers_of_two():
    assert frame_class(10, 455626, 1712 * 995) == (10, 19, 21)
    assert frame_class(6, 10000, 256 * 256) == (6, 13, 16)
    assert frame_class(8, 1, 1) == (8, 0, 0)


def test_autotuner_times_each_candidate_reps_times_per_class():
    calls = []
    cost = {("tc", 256): 3.0, ("auto", 256): 2.0, ("tc", 128): 2.5, ("fp32", 256): 9.0}

    def timer(cfg):
        calls.append(cfg)
        return cost[cfg]

    t = Autotuner()
    assert t.reps >= 5
    assert t.choose((6, 13, 16), timer) == ("auto", 256)
    assert len(calls) == t.reps * len(CANDIDATES)
    assert sorted(set(calls)) == sorted(CANDIDATES)
    # interleaved: every pass times each candidate once
    assert calls[:len(CANDIDATES)] == list(CANDIDATES)
    calls.clear()
    assert t.choose((6, 13, 16), timer) == ("auto", 256)  # cached
    assert calls == []
    cost[("tc", 128)] = 1.0
    assert t.choose((10, 19, 21), timer) == ("tc", 128)  # a new class is tuned afresh
    assert len(calls) == t.reps * len(CANDIDATES)
    assert set(t.trials) == {(6, 13, 16), (10, 19, 21)}


def test_autotuner_decides_on_the_median_not_one_outlier():
    # ("tc", 256) is usually fastest but has one slow sample; ("auto", 256)
    # has one lucky fast sample and is otherwise slower
    seq = {("tc", 256): iter([1.0, 9.0, 1.0, 1.1, 1.0]),
           ("auto", 256): iter([0.5, 2.0, 2.0, 2.0, 2.0]),
           ("tc", 128): iter([3.0] * 5), ("fp32", 256): iter([5.0] * 5)}
    t = Autotuner(reps=5)
    assert t.choose((8, 17, 20), lambda cfg: next(seq[cfg])) == ("tc", 256)
    assert t.trials[(8, 17, 20)][("tc", 256)] == [1.0, 9.0, 1.0, 1.1, 1.0]
