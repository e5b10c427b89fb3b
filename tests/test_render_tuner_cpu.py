"""Host logic of the render autotuner (no GPU): classes, one trial per
class and candidate, the fastest kept."""
from paper_2405_20067_gb300.render import CANDIDATES, Autotuner, frame_class


def test_frame_classes_round_to_powers_of_two():
    assert frame_class(10, 455626, 1712 * 995) == (10, 19, 21)
    assert frame_class(6, 10000, 256 * 256) == (6, 13, 16)
    assert frame_class(8, 1, 1) == (8, 0, 0)


def test_autotuner_tries_each_candidate_once_per_class():
    calls = []
    cost = {("tc", 256): 3.0, ("auto", 256): 2.0, ("tc", 128): 2.5, ("fp32", 256): 9.0}

    def timer(cfg):
        calls.append(cfg)
        return cost[cfg]

    t = Autotuner()
    assert t.choose((6, 13, 16), timer) == ("auto", 256)
    assert sorted(calls) == sorted(CANDIDATES)
    calls.clear()
    assert t.choose((6, 13, 16), timer) == ("auto", 256)  # cached
    assert calls == []
    cost[("tc", 128)] = 1.0
    assert t.choose((10, 19, 21), timer) == ("tc", 128)  # a new class is tuned afresh
    assert len(calls) == len(CANDIDATES)
    assert set(t.trials) == {(6, 13, 16), (10, 19, 21)}
