"""The mock operator on the device executors (Sec. 5.1): an operator that adds its two inputs
after a spin of a given duration, run along every scan DAG by every executor.  The prefix sums
are exact (integer values), so any scheduling error shows; the durations are the paper's two
configurations, fixed and exponentially distributed (Mersenne Twister seeded 1410)."""
import numpy as np
import pytest
import torch

from paper_2010_12478_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2010_12478_gb300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("schedule", ["sequential", "brent_kung", "dissemination", "ladner_fischer", "blelloch",
                                      "lookback4"])
@pytest.mark.parametrize("exec_", ["plain", "level", "persistent"])
def test_mock_scan_gives_exact_prefix_sums(schedule, exec_):
    n = 300 if schedule == "sequential" else 1000
    rng = np.random.default_rng(7)
    v = rng.integers(-1000, 1000, size=n).astype(np.float64)
    m = B.scan_work(schedule, n)
    us = np.random.RandomState(1410).exponential(5.0, size=m).astype(np.float32)
    ctx = B.Context(B.Config())
    out, ms = ctx.mock_scan(v, us, schedule=schedule, exec=exec_)
    want = np.concatenate([[0.0], np.cumsum(v)[:-1]]) if schedule == "blelloch" else np.cumsum(v)
    assert np.array_equal(out, want)
    assert ms > 0.0


def test_blelloch_work_is_table_1():
    # Table 1: the Blelloch scan applies the operator 2 (n - 1) times, its identity applications included
    for n in (2, 8, 64, 1024, 98304):
        assert B.scan_work("blelloch", n) == 2 * (n - 1)


def test_mock_durations_are_honoured_and_checked():
    ctx = B.Context(B.Config())
    n = 64
    m = B.scan_work("sequential", n)
    _, ms = ctx.mock_scan(np.ones(n), np.full(m, 200.0, np.float32), schedule="sequential", exec="persistent")
    assert ms >= 0.9 * m * 0.2          # a chain of m operators of 200 us each
    with pytest.raises(B.RegError) as e:
        ctx.mock_scan(np.ones(n), np.full(m, 2.0e5, np.float32), schedule="sequential")
    assert e.value.code == B.REG_EINVAL
    with pytest.raises(B.RegError) as e:
        ctx.scan(torch.zeros((3, 32, 32), device="cuda"), schedule="blelloch")
    assert e.value.code == B.REG_EINVAL
