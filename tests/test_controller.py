"""Host logic of the adaptive time-step controller (Solver.advance) on a stand-in step that
fails above a step size and reports a change proportional to the step: rejection halves the
step, the step after a rejection or a hard Newton solve does not grow, small changes double
it, the tolerance sets it otherwise, and the run ends exactly on t_end."""
import pytest

from paper_0908_2654_gb300 import _rt
from paper_0908_2654_gb300.solver import Solver


class FakeSolver(Solver):
    """Solver.advance on a stand-in step (no library state, no GPU)."""

    def __init__(self, fail_above, change_per_time, newton=3):
        self.t, self.dt = 0.0, 1.0
        self.fail_above, self.k, self.newton = fail_above, change_per_time, newton
        self.calls = []

    def step(self, fold=True, advect=None):
        self.calls.append(self.dt)
        if self.dt > self.fail_above:
            raise _rt.RTError(_rt.RT_ENOCONV, "stand-in step")
        self.t += self.dt
        return {"change_norm": self.k * self.dt, "newton_iters": self.newton}


def test_rejections_halve_and_block_growth():
    s = FakeSolver(fail_above=0.3, change_per_time=1e-3)
    out = s.advance(1.0, tau_tol=0.1)
    assert s.calls[:3] == [1.0, 0.5, 0.25]          # two rejections, then accepted at 0.25
    assert out[0][1] == 0.25 and out[0][2]["rejected"] == 2
    assert out[1][1] == 0.25                          # no growth right after a rejection
    assert s.t == pytest.approx(1.0, rel=1e-15)


def test_growth_and_tolerance_limits():
    s = FakeSolver(fail_above=1e9, change_per_time=1.0)
    s.dt = 1e-3
    s.advance(0.015, tau_tol=0.01)                     # change 1e-3: below tau/2, so doubling
    dts = [dt for dt in s.calls]
    assert dts[:3] == pytest.approx([1e-3, 2e-3, 4e-3])
    s2 = FakeSolver(fail_above=1e9, change_per_time=1.0)
    s2.dt = 0.008
    out = s2.advance(0.1, tau_tol=0.01)
    assert out[1][1] == pytest.approx(0.01)            # tau / eps = 0.01 / 0.008 -> dt 0.01
    assert s2.t == pytest.approx(0.1, rel=1e-15)       # the last step is cut to end on t_end


def test_hard_newton_solves_stop_growth():
    s = FakeSolver(fail_above=1e9, change_per_time=1e-6, newton=10)
    s.dt = 1.0
    s.advance(3.0, tau_tol=0.1)
    assert s.calls == [1.0, 1.0, 1.0]                  # 10 > 8 Newton iterations: no growth
    s = FakeSolver(fail_above=1e9, change_per_time=1e-6, newton=13)
    s.dt = 1.0
    s.advance(1.7, tau_tol=0.1)
    assert s.calls == pytest.approx([1.0, 0.7])        # 13 > 12: shrink by 0.7


def test_non_retryable_errors_propagate():
    class Broken(FakeSolver):
        def step(self, fold=True, advect=None):
            raise _rt.RTError(_rt.RT_EINVAL, "stand-in step")
    with pytest.raises(_rt.RTError):
        Broken(1.0, 1.0).advance(1.0)
