"""The (eta, tau) rules of the workloads whose rule the paper leaves open: the overlap matrix S is the
Gram matrix of the basis, so the singular values of its target-projectile block K must stay below 1.
Checked with the oracle's assembly at the smallest impact parameter, where a coarse eta rule fails
first (velocity scan at v = 0.5: 72 eta nodes; the C6+ + H basis with fewer packets: 128 eta nodes)."""
import numpy as np

import wpccc_inputs as wi
from oracle import wpccc_oracle as O


def _sigma_max(basis, b, v, z):
    S, _ = O.assemble(basis, b, v, z)
    NT = basis.T.N
    return np.linalg.svd(S[:NT, NT:], compute_uv=False).max()


def test_velocity_scan_rule_gives_a_gram_overlap():
    v, basis, _ = wi.batch_inputs(n_b=2, speeds=(0.5,))[0]
    assert v == 0.5 and basis.quad.s.size == 72
    s72 = _sigma_max(basis, 0.2, v, 0.0)
    assert s72 < 1.0, s72
    # the 48-node rule of the fixed-speed workload is not enough here: an indefinite S
    _, coarse, _ = wi.batch_inputs(n_b=2, speeds=(0.5,), Geta=48)[0]
    assert _sigma_max(coarse, 0.2, v, 0.0) > 1.0


def test_c6_rule_gives_a_gram_overlap():
    basis, paths = wi.config_inputs("C6_H_2c_n6l5", nbins=4, Nr=1200)
    assert basis.quad.s.size == 128
    assert _sigma_max(basis, 0.5, 2.0, 0.0) < 1.0


def _omega_max(basis, b, v, z):
    """max |lambda| / v of the generalised problem H x = lambda S x: the largest frequency of the
    amplitudes' equation dc/dz = -(i/v) S^-1 H c, whose eigenvalues are imaginary (H Hermitian, S positive
    definite)."""
    import scipy.linalg as sl
    S, H = O.assemble(basis, b, v, z)
    return np.abs(sl.eigh(H, S, eigvals_only=True)).max() / v


def test_c6_zgrid_keeps_rk4_stable_where_the_geometric_grid_does_not():
    # RK4's stability interval on the imaginary axis is |h omega| < 2 sqrt(2); the C6+ + H grid bounds
    # h omega_max by about 2 along the smallest impact parameter, where the basis is stiffest
    basis, paths = wi.config_inputs("C6_H_2c_n6l5")
    zg = paths.z[0]
    assert zg.size - 1 == 3562 and zg[0] == -50.0 and zg[-1] == 50.0
    b, v = float(paths.b[0]), float(paths.v[0])
    assert b == 0.5
    h = np.diff(zg)
    for z in (0.3, 2.0, 4.0, 8.0):
        k = int(np.searchsorted(zg, z))
        om = _omega_max(basis, b, v, z)
        step = max(h[k - 1], h[min(k, h.size - 1)])
        assert step * om < 2.1, (z, step, om)
    # the paper's geometric grid (Sec. II) takes steps of about 0.022 |z|: unstable at |z| = 1 here
    zgeo = wi.geometric_zgrid(1e-3, 50.0, 500)
    k = int(np.searchsorted(zgeo, 1.0))
    assert (zgeo[k] - zgeo[k - 1]) * _omega_max(basis, b, v, 1.0) > 2.0 * np.sqrt(2.0)
