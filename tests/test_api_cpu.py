"""Host logic of the Python binding that needs no GPU."""
import pytest


def test_richardson_solve_checks_params_before_solving():
    torch = pytest.importorskip("torch")
    from paper_2103_12571_gb300.api import RichardsonSolve

    class StubPlan:
        def params(self):
            return [0.05, 0.7, -0.4]

        def solve(self, *args, **kw):
            raise AssertionError("the solve must not run with mismatched parameters")

    x = torch.zeros(4, dtype=torch.float64)
    with pytest.raises(ValueError):
        RichardsonSolve.apply(x, torch.tensor([0.05, 0.8, -0.4], dtype=torch.float64), StubPlan(), 1e-12)
    with pytest.raises(ValueError):
        RichardsonSolve.apply(x, torch.tensor([0.05, 0.7], dtype=torch.float64), StubPlan(), 1e-12)


def test_host_step_pointer_checks():
    """ac_richardson_step_host takes host arrays: contiguous float64 CPU
    tensors pass, anything else is refused before the library is called."""
    torch = pytest.importorskip("torch")
    from paper_2103_12571_gb300.api import _host_ptr
    t = torch.zeros((2, 3), dtype=torch.float64)
    assert _host_ptr(t).value == t.data_ptr()
    assert _host_ptr(None) is None
    with pytest.raises(ValueError):
        _host_ptr(torch.zeros((2, 3), dtype=torch.float32))
    with pytest.raises(ValueError):
        _host_ptr(torch.zeros((3, 2), dtype=torch.float64).t())


def test_library_declares_the_host_step_and_the_cluster_option():
    """The binding's structures mirror the header: the schedule carries the
    cluster option, the plan record reports the cluster size, and the host
    step has a prototype."""
    from paper_2103_12571_gb300 import _lib
    assert "space_cluster" in [f for f, _ in _lib.Schedule._fields_]
    assert "space_cluster" in [f for f, _ in _lib.PlanInfo._fields_]
    assert "ac_richardson_step_host" in _lib._PROTOS
