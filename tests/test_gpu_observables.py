"""Observables, cross sections, the overlap norms and the state list through the C ABI.

* wpccc_observables: P = sum_i g_i |c_i|^2 against a plain numpy evaluation, and capture + 2p excitation
  of a propagated path against the oracle's probabilities.
* wpccc_cross_sections: the trapezoid rule on the impact parameters plus b = 0 is exact for P = 1
  (b P(b) linear): sigma = pi b_max^2; for other P it equals the workload generator's per-path weights and
  numpy's trapezoid on the nodes (0, b).
* wpccc_overlap_norms: c^+ S c at the start of a path equals 1 (c = e_1, S_11 = 1); along a two-centre path
  its change equals the integral of c^+ (dS/dz) c (the balance law of i v S dc/dz = H c with Hermitian H),
  checked against the oracle's S at the path's nodes.
* wpccc_basis_states: the generator's state list and energies.
"""
import numpy as np
import pytest

import wpccc_inputs as wi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _basis_small():
    return wi.make_basis(1.0, 1.0, 2, 1, 2, 2.0, True, Nr=600, Geta=16, Gtau=12)


def test_observables_and_cross_sections_closed_forms():
    import paper_2403_04252_gb300 as w
    rng = np.random.default_rng(3)
    c = torch.from_numpy(rng.standard_normal((5, 37)) + 1j * rng.standard_normal((5, 37))).cuda()
    g = (rng.random((3, 37)) < 0.4).astype(np.float64)
    P = w.observables_of(c, g).cpu().numpy()
    cn = c.cpu().numpy()
    assert np.allclose(P, (np.abs(cn) ** 2) @ g.T, rtol=1e-14, atol=0)
    b = np.linspace(0.5, 4.0, 8)
    sig = w.cross_sections(b, np.ones((8, 1))).cpu().numpy()
    assert abs(sig[0] - np.pi * 4.0 ** 2) <= 1e-13 * np.pi * 16.0
    b = np.linspace(0.2, 12.0, 32)
    Pb = np.stack([np.exp(-b) * (1 + b), 0.3 * np.exp(-0.5 * (b - 2.0) ** 2)], axis=1)
    sig = w.cross_sections(b, Pb).cpu().numpy()
    assert np.allclose(sig, wi.cross_section_weights(b) @ Pb, rtol=1e-14, atol=0)
    nodes = np.concatenate([[0.0], b])
    ref = [2 * np.pi * np.trapezoid(np.concatenate([[0.0], b * Pb[:, o]]), nodes) for o in range(2)]
    assert np.allclose(sig, ref, rtol=1e-13, atol=0)
    with pytest.raises(w.WpcccError) as e:
        w.cross_sections(b[::-1].copy(), Pb)
    assert e.value.status == w.EINVAL


def test_observables_of_a_propagated_path_against_oracle():
    from oracle import wpccc_oracle as O
    import paper_2403_04252_gb300 as w
    basis = _basis_small()
    g = w.Basis(basis)
    zg = wi.uniform_zgrid(-3.0, 3.0, 0.25)
    c = g.propagate([0.7], 1.2, zg)
    gw = wi.observable_weights(basis)
    P = w.observables_of(c, gw).cpu().numpy()[0]
    Po = gw @ O.probabilities(O.propagate(basis, 0.7, 1.2, zg))
    assert np.allclose(P, Po, rtol=1e-10, atol=1e-14)
    qn, eps = g.states()
    T, Pc = basis.T, basis.P
    assert np.array_equal(qn[:T.N, 0], np.zeros(T.N)) and np.array_equal(qn[T.N:, 0], np.ones(Pc.N))
    assert np.array_equal(qn[:T.N, 1], T.st_rad) and np.array_equal(qn[T.N:, 1], Pc.st_rad)
    assert np.array_equal(qn[:T.N, 2], T.rad_l[T.st_rad]) and np.array_equal(qn[:T.N, 3], T.st_m)
    assert np.array_equal(eps, np.concatenate([T.st_eps, Pc.st_eps]))
    g.close()


def test_overlap_norm_balance_along_a_two_centre_path():
    # i v S dc/dz = H c with H, S Hermitian gives d(c^+ S c)/dz = c^+ (dS/dz) c: the change of c^+ S c over
    # the path equals the integral of c^+ S' c, here with S' from central differences of the oracle's S and
    # Simpson's rule on a fine path (h = 0.02); c^+ S c itself is not conserved under Eq. 1's Q^+ block
    from oracle import wpccc_oracle as O
    import paper_2403_04252_gb300 as w
    basis = _basis_small()
    g = w.Basis(basis)
    b, v = 0.7, 1.2
    zg = wi.uniform_zgrid(-2.0, 2.0, 0.02)
    norms, cs = [], []
    c = torch.zeros((1, g.N), dtype=torch.complex128, device="cuda")
    c[:, 0] = 1.0
    assert abs(g.overlap_norms([b], v, [zg[0]], c).cpu().numpy()[0, 0] - 1.0) < 1e-14
    for k in range(zg.size):
        if k > 0:
            g.propagate([b], v, zg[k - 1:k + 1], c=c)
        norms.append(g.overlap_norms([b], v, [zg[k]], c).cpu().numpy()[0, 0])
        cs.append(c.cpu().numpy()[0].copy())
    norms = np.array(norms)
    dz = 1e-4
    integrand = []
    for k, z in enumerate(zg):
        Sp = (O.assemble(basis, b, v, z + dz)[0] - O.assemble(basis, b, v, z - dz)[0]) / (2 * dz)
        integrand.append(np.real(cs[k].conj() @ Sp @ cs[k]))
    integrand = np.array(integrand)
    h = zg[1] - zg[0]
    simpson = h / 3 * (integrand[0] + integrand[-1] + 4 * integrand[1:-1:2].sum() + 2 * integrand[2:-1:2].sum())
    drift = norms[-1] - norms[0]
    assert abs(drift) > 1e-4                     # not an invariant in the two-centre form
    assert abs(drift - simpson) < 1e-7 * max(1.0, abs(drift)), (drift, simpson)
    g.close()
