"""Checkpoint and resume through the C ABI: a path propagated in two calls, the second starting from the
amplitudes the first returned at the split node, ends with the same bits as the uninterrupted call.

The kernels have no floating-point atomics and every position's elements, factors and RK4 steps are
computed in a fixed order, so the chunk schedule (which the workspace limit changes) and the split point
move nothing."""
import numpy as np
import pytest

import wpccc_inputs as wi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small2c():
    return wi.make_basis(1.0, 1.0, 2, 1, 2, 2.0, True, Nr=600, Geta=20, Gtau=14)


@pytest.mark.parametrize("solve,precision", [(0, 0), (2, 0), (2, 2)])
def test_resumed_path_is_bit_identical(small2c, solve, precision):
    import paper_2403_04252_gb300 as w
    g = w.Basis(small2c)
    g.set_solve_mode(solve)
    g.set_workspace_limit(64 << 20)
    bs = np.array([0.4, 1.7, 3.0])
    zg = wi.uniform_zgrid(-6.0, 6.0, 0.25)
    whole = g.propagate(bs, 1.3, zg, precision_mode=precision)
    for k in (1, 20, zg.size - 2):
        first = g.propagate(bs, 1.3, zg[:k + 1], precision_mode=precision)
        resumed = g.propagate(bs, 1.3, zg[k:], c=first.clone(), precision_mode=precision)
        assert torch.equal(resumed, whole), (k, (resumed - whole).abs().max().item())
    g.close()
