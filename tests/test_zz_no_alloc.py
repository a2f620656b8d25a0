"""The allocation-free preconditioner solve (ac_precond_solve_noalloc).

Callers that cannot allocate device memory when they need a solve (their
device memory belongs to another framework's caching allocator, or their
loop must not pay for cudaMalloc's implicit synchronisation) use this entry
point instead of a plan.  Its result must be the one ac_precond_solve gives,
call after call, even though every call reuses the same fixed scratch array.
This file is collected last so that a run stopping at the first failure has
run every other test before it."""
import ctypes

import numpy as np
import pytest

from gpu_common import rel2, to_dev, torch_cuda
from paper_2103_12571_gb300 import workloads

pytestmark = pytest.mark.gpu

CASES = [
    (workloads.problem(1, 512, cx=1.0, order=4, M=3, L=16, T=0.25), "c128"),
    (workloads.problem(2, 128, 128, nu=0.05, order=2, M=3, L=32, T=0.25), "c64"),
    (workloads.problem(2, 128, 256, nu=0.05, cx=0.5, cy=-0.25, order=2, M=3, L=8, T=0.0625), "c128"),
    # mixed-radix solves (sizes that are not powers of two)
    (workloads.problem(1, 700, cx=1.0, order=5, upwind=True, M=3, L=16, T=0.05), "c64"),
    (workloads.problem(2, 45, 28, nu=0.02, cx=0.3, cy=-0.2, order=4, M=2, L=4, T=0.05), "c128"),
]


def call_noalloc(torch, prob, precision, alpha, r, e):
    from paper_2103_12571_gb300 import _lib
    from paper_2103_12571_gb300.api import PRECISION, make_problem
    L = prob["L"]
    rc = _lib.lib().ac_precond_solve_noalloc(
        ctypes.byref(make_problem(prob)), prob["M"], L, prob["T"] / L, float(alpha), PRECISION[precision],
        ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(e.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


@pytest.mark.parametrize("prob,precision", CASES, ids=lambda v: str(v) if isinstance(v, str) else
                         "d%d_%dx%d_L%d" % (v["dim"], v["nx"], v["ny"], v["L"]))
def test_noalloc_matches_plan_solve_twice(prob, precision):
    torch = torch_cuda()
    from paper_2103_12571_gb300.api import Plan
    plan = Plan(prob, precision=precision)
    rng = np.random.default_rng(11)
    N = prob["nx"] * prob["ny"]
    for alpha in (1e-2, 1e-4):  # two calls in a row on the shared scratch
        r = to_dev(torch, rng.standard_normal((prob["L"], prob["M"], N)))
        ref = plan.precond_solve(alpha, r)
        e = torch.full_like(r, float("nan"))
        assert call_noalloc(torch, prob, precision, alpha, r, e) == 0
        torch.cuda.synchronize()
        assert torch.isfinite(e).all()
        # the same launches (ac_setup's tiles and spatial path) on the same
        # tables: the result must be ac_precond_solve's, bit for bit; a call
        # that read tables left over from the previous one would differ
        assert torch.equal(e, ref), rel2(e.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_rejects_problems_beyond_the_scratch():
    torch = torch_cuda()
    from paper_2103_12571_gb300 import _lib
    prob, u0, _ = workloads.config(2)   # 256 x 256, L = 64: 52 MB of complex64 work space
    r = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = call_noalloc(torch, prob, "c64", 1e-3, r, r)
    assert rc == _lib.AC_ERR_INVALID_ARG
    msg = _lib.lib().ac_last_error().decode()
    assert "MiB" in msg and "32" in msg
