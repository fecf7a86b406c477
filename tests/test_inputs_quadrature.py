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
