"""CPU checks of the host logic of the probe term (LogDetProbes): more probes
than one lockstep solve takes are split into blocks of DCG_MAX_RHS in order,
and the lockstep and one-by-one paths feed the same solutions to the
derivative forms. A stand-in solver replaces the library: A = I / 2, so each
solve returns 2 z, and the forms are plain dot products."""

import numpy as np
import pytest
import torch

from paper_1706_00241_gb300 import autograd as AG
from paper_1706_00241_gb300._lib import DCG_MAX_RHS


class StandInSolver:
    def __init__(self):
        self.multi_sizes = []
        self.single_calls = 0
        self.params = []

    def set_rbf_params(self, *p):
        self.params.append(p)

    def solve_multi(self, B):
        assert B.dim() == 2 and B.is_contiguous()
        self.multi_sizes.append(B.shape[0])
        return (2.0 * B).to(torch.float64), [{"status": 0, "iters": 1}] * B.shape[0]

    def solve(self, b):
        self.single_calls += 1
        return (2.0 * b).to(torch.float64), {"status": 0, "iters": 1}

    def rbf_dtheta(self, U, V):
        # per pair: (u.v, 2 u.v, 3 u.v), as the three forms of the library
        d = (U.double() * V.double()).sum(dim=1).numpy()
        return np.stack([d, 2 * d, 3 * d], axis=1)


@pytest.mark.parametrize("P", [1, DCG_MAX_RHS, DCG_MAX_RHS + 8, 2 * DCG_MAX_RHS + 3])
def test_probe_blocks_and_paths_agree(P):
    n = 7
    g = torch.Generator().manual_seed(P)
    Z = (torch.randint(0, 2, (P, n), generator=g) * 2 - 1).to(torch.float32)
    grads = {}
    for block in (True, False):
        s = StandInSolver()
        theta = torch.tensor([0.5, 1.0, 0.1], dtype=torch.float64, requires_grad=True)
        AG.LogDetProbes.apply(theta, s, Z, block).backward()
        grads[block] = theta.grad.numpy().copy()
        if block:
            full, rest = divmod(P, DCG_MAX_RHS)
            assert s.multi_sizes == [DCG_MAX_RHS] * full + ([rest] if rest else [])
            assert s.single_calls == 0
        else:
            assert s.multi_sizes == [] and s.single_calls == P
        assert len(s.last_probe_infos) == P
    # u_p = 2 z_p, z_p in {-1, 1}^n: u.z = 2 n per probe; grad = 1/2 mean(forms)
    np.testing.assert_array_equal(grads[True], grads[False])
    np.testing.assert_allclose(grads[True], 0.5 * np.array([2 * n, 4 * n, 6 * n]))
