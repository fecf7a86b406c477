"""RK4 with the vectors in global memory (wpccc_basis_set_rk4_layout, one-centre form) through the C ABI:
the same amplitudes as the shared-memory sweep, the oracle's probabilities at the FP64 bar, and a
one-centre basis beyond the shared-memory limit (N = 3289: n <= 10, l <= 10, 24 packets per l)."""
import numpy as np
import pytest

import wpccc_inputs as wi
from oracle import wpccc_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P_TOL = 1e-10


def _w():
    import paper_2403_04252_gb300 as w
    return w


def _prob_close(Pg, Po):
    bound = P_TOL * np.maximum(Po, 1e-4)
    assert np.all(np.abs(Pg - Po) <= bound), np.abs(Pg - Po).max()


def test_global_layout_matches_shared_one_centre():
    # ragged paths and a workspace limit that forces several chunks (each chunk evaluates its first node
    # again in the global layout)
    w = _w()
    basis, _ = wi.config_inputs("p_H_1c_n3l2")
    g = w.Basis(basis)
    g.set_workspace_limit(64 << 20)
    bs = np.array([0.5, 2.0, 5.5])
    zgs = [wi.uniform_zgrid(-6.0, 6.0, 0.1), wi.uniform_zgrid(-3.0, 4.0, 0.1), wi.uniform_zgrid(-1.0, 1.0, 0.25)]
    out = {}
    for layout in (w.RK4_SHARED, w.RK4_GLOBAL):
        g.set_rk4_layout(layout)
        out[layout] = w.probabilities(g.propagate(bs, 1.0, zgs)).cpu().numpy()
    assert np.abs(out[w.RK4_GLOBAL] - out[w.RK4_SHARED]).max() < 1e-13
    for p in range(3):
        _prob_close(out[w.RK4_GLOBAL][p], O.probabilities(O.propagate(basis, float(bs[p]), 1.0, zgs[p])))
    with pytest.raises(w.WpcccError) as e:
        g.set_rk4_layout(3)
    assert e.value.status == w.EINVAL
    g.close()


def test_global_layout_large_one_centre_basis():
    # N = 3289 > the shared-memory sweep's limit: the default layout switches to global memory
    w = _w()
    basis = wi.make_basis(1.0, 1.0, 10, 10, 24, 2.0, False, Nr=2000)
    assert basis.N == 3289
    g = w.Basis(basis)
    zg = np.array([-0.1, 0.05])
    bs = np.array([1.0, 3.0])
    c = g.propagate(bs, 1.0, zg)
    P = w.probabilities(c).cpu().numpy()
    # S = I and D Hermitian: only RK4's truncation moves the norm, here by ~4e-7 (h = 0.15 against the
    # basis' largest coupling eigenvalues); the oracle comparison below is the parity check
    assert np.abs(P.sum(axis=1) - 1.0).max() < 1e-5
    _prob_close(P[0], O.probabilities(O.propagate(basis, 1.0, 1.0, zg)))
    g.set_rk4_layout(w.RK4_SHARED)
    with pytest.raises(w.WpcccError) as e:
        g.propagate(bs, 1.0, zg)
    assert e.value.status == w.EINVAL
    g.close()


def test_global_layout_is_one_centre_only():
    w = _w()
    two = wi.make_basis(1.0, 1.0, 2, 1, 2, 2.0, True, Nr=600, Geta=16, Gtau=16)
    g = w.Basis(two)
    g.set_rk4_layout(w.RK4_GLOBAL)
    with pytest.raises(w.WpcccError) as e:
        g.propagate(np.array([1.0]), 1.0, [np.array([0.0, 0.1])])
    assert e.value.status == w.EUNSUPPORTED
    g.close()


def test_global_layout_edge_paths():
    # a path without steps keeps its amplitudes; one-step and many-step paths through several chunks
    # (every chunk evaluates its first node again) equal the shared-memory sweep
    w = _w()
    basis, _ = wi.config_inputs("p_H_1c_n3l2")
    g = w.Basis(basis)
    g.set_workspace_limit(64 << 20)
    bs = np.array([0.8, 1.5, 4.0])
    zgs = [np.array([0.3]), np.array([-0.2, 0.1]), wi.uniform_zgrid(-8.0, 8.0, 0.1)]
    c0 = torch.zeros((3, g.N), dtype=torch.complex128, device="cuda")
    c0[:, 0] = 0.6
    c0[:, 1] = 0.8j
    res = {}
    for layout in (w.RK4_SHARED, w.RK4_GLOBAL):
        g.set_rk4_layout(layout)
        res[layout] = g.propagate(bs, 1.0, zgs, c=c0.clone())
    assert torch.equal(res[w.RK4_GLOBAL][0], c0[0])
    assert (res[w.RK4_GLOBAL] - res[w.RK4_SHARED]).abs().max().item() < 1e-13
    g.close()
