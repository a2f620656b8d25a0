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
