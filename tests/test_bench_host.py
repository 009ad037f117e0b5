"""Host logic of bench.py that runs without a GPU."""
import pytest

import bench


def test_group_measurement_fails_with_an_ordinary_exception():
    """The default run measures the Group-Lasso workload last and records a failure as an
    error entry (an ordinary exception); without a GPU it must fail that way, not end the
    process."""
    with pytest.raises(Exception):
        bench.group_measure(steps=1, warmup=0)


def test_small_fp64_latency_fails_with_an_ordinary_exception():
    with pytest.raises(Exception):
        bench.config1_latency(reps=1, warmup=0)
