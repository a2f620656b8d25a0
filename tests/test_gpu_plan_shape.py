"""The host-side shape query (ac_plan_shape) reports what ac_setup builds on
the GPU: the same spatial path, time-kernel tiles and cluster size."""
import pytest

from gpu_common import torch_cuda
from paper_2103_12571_gb300 import workloads

pytestmark = pytest.mark.gpu

P = workloads.problem
CASES = [
    (P(1, 512, cx=1.0, order=4, M=3, L=16, T=0.25), "c128", "fft", 0),
    (P(2, 64, 64, nu=1e-3, cx=1.0, cy=0.5, order=2, M=3, L=32, T=0.25), "c64", "fft", 0),
    (P(2, 128, 256, nu=0.05, order=2, M=3, L=8, T=0.0625), "c128", "fft", 0),
    (P(2, 128, 256, nu=0.05, order=2, M=3, L=8, T=0.0625), "c64", "fft", 8),
    (P(2, 45, 28, nu=0.02, cx=0.3, cy=-0.2, order=4, M=2, L=4, T=0.05), "c64", "fft", 0),
    (P(1, 97, nu=0.05, cx=0.5, order=2, M=2, L=8, T=0.2), "c128", "bicgstab", 0),
    (P(2, 24, 20, nu=0.02, cx=0.4, cy=-0.3, order=2, M=3, L=8, T=0.1), "c64", "gmres", 0),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dx%d_%s_%s_cl%d" % (c[0]["nx"], c[0]["ny"], c[1], c[2], c[3]))
def test_plan_shape_matches_setup(case):
    torch_cuda()
    from paper_2103_12571_gb300.api import Plan, plan_shape
    prob, precision, inner, cluster = case
    info = Plan(prob, precision=precision, inner=inner, space_cluster=cluster).info()
    shape = plan_shape(prob, precision=precision, inner=inner, space_cluster=cluster)
    for k in ("N", "M", "L", "F", "tile_fwd", "tile_upd", "spatial_path", "space_cluster"):
        assert shape[k] == info[k], (k, shape, info)
