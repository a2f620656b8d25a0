"""Shared set-up for the GPU parity tests: plans from problem dicts and the
oracle's reference objects for the same problem."""
import numpy as np
import pytest

from oracle import collocation, operators


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_12571_gb300 import _lib
    _lib.lib()  # fail loudly if the library is missing
    return torch


def oracle_setup(prob):
    t = collocation.radau_iia_nodes(prob["M"])
    Q = collocation.collocation_matrix(t)
    A = operators.spatial_operator(prob)
    return Q, A, prob["T"] / prob["L"]


def rel2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def to_dev(torch, x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
