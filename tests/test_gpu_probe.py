"""The pipe-throughput probe behind the benchmark's MUFU and FP32 rooflines
(ndg_probe_pipe): the rates it reports are those of a real pipe, i.e.
positive and below the per-SM lane counts (32 FP32 lanes per SM
sub-partition, four sub-partitions)."""
import pytest

pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible():
    import torch
    from paper_2405_20067_gb300 import build, ndg
    build.build()
    assert torch.cuda.is_available()
    ex2 = ndg.probe_pipe(0, reps=2)
    ffma = ndg.probe_pipe(1, reps=2)
    print(f"ex2 {ex2['per_clk_per_sm']:.1f}/clk/SM ({ex2['per_s']:.3e}/s), "
          f"ffma {ffma['per_clk_per_sm']:.1f}/clk/SM ({ffma['per_s']:.3e}/s)")
    assert 4.0 <= ex2["per_clk_per_sm"] <= 128.5
    assert 32.0 <= ffma["per_clk_per_sm"] <= 128.5
    assert ex2["per_clk_per_sm"] < ffma["per_clk_per_sm"]
