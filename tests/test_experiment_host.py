"""Host-side arithmetic of the Algorithm 1 driver (no GPU): error histories and the
speed-up at equal error, interpolated log-log over the plain orders' error/cost curve."""
import math
import types

import numpy as np
import pytest

pytest.importorskip("torch")
from paper_2207_11571_gb300 import experiment  # noqa: E402


def run_record(err, ms):
    return {"errors": {"dke": err}, "ms": ms}


def test_speedup_interpolates_a_power_law_exactly():
    # plain orders on cost = 0.4 / error: log-log linear, so interpolation is exact
    plain = [run_record(0.4, 1.0), run_record(0.2, 2.0), run_record(0.1, 4.0), run_record(float("inf"), 0.5)]
    s, kind = experiment.speedup_at_equal_error(run_record(0.4 / 2.83, 1.0), plain, "dke")
    assert s == pytest.approx(2.83, rel=1e-12) and kind == "interpolated"
    # below the smallest plain error: no extrapolation, the result is a lower bound
    s, kind = experiment.speedup_at_equal_error(run_record(0.05, 2.0), plain, "dke")
    assert s == pytest.approx(2.0, rel=1e-12) and kind == "lower_bound"
    # above every plain error: the cheapest plain run is already more accurate
    s, kind = experiment.speedup_at_equal_error(run_record(0.8, 4.0), plain, "dke")
    assert s == pytest.approx(0.25, rel=1e-12) and kind == "cheapest_plain_is_more_accurate"
    # a diverged corrected run has no speed-up
    assert experiment.speedup_at_equal_error(run_record(float("inf"), 1.0), plain, "dke") == (None, None)


def test_speedup_with_errors_that_do_not_fall_with_cost_takes_the_cheapest_as_accurate_run():
    # saturated errors: 0.99 at cost 1, 0.78 at 2, 1.13 at 3, 1.03 at 5 (not monotone)
    plain = [run_record(0.99, 1.0), run_record(0.78, 2.0), run_record(1.13, 3.0), run_record(1.03, 5.0)]
    s, kind = experiment.speedup_at_equal_error(run_record(0.9, 2.0), plain, "dke")
    assert s == pytest.approx(1.0, rel=1e-12) and kind == "pareto"   # the cost-2 run (0.78 <= 0.9)


def test_run_errors_of_a_diverged_run_are_infinite_and_exact_run_is_zero():
    t = np.linspace(0.0, 1.0, 11)
    ke = 0.125 * np.exp(-t)
    dke = -0.125 * np.exp(-t)
    einf = [0.5 * (i + 1) for i in range(11)]   # e_n samples: their mean is the einf error
    same = types.SimpleNamespace(diverged_at=None, dke=dke, ke=ke, einf=einf)
    e = experiment.run_errors(same, t, dke, ke, ke)
    assert e == {"dke": 0.0, "ke": 0.0, "dke_filtered": 0.0, "einf": 3.0}
    gone = types.SimpleNamespace(diverged_at=0.3, dke=dke, ke=ke, einf=einf)
    assert all(math.isinf(v) for v in experiment.run_errors(gone, t, dke, ke, ke).values())
    # a 1 % uniform error in the dissipation history is a 1 % relative L2 error
    off = types.SimpleNamespace(diverged_at=None, dke=1.01 * dke, ke=ke, einf=einf)
    assert experiment.run_errors(off, t, dke, ke, ke)["dke"] == pytest.approx(0.01, rel=1e-12)
