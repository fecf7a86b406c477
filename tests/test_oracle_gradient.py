"""Pins of the differentiation form's oracle (CPU): the Li-like model-potential elements against
lab-frame brute-force integrals, the parameter tangents of the basis, S and H against central
differences with the basis regenerated, and the forward-mode gradient of the probabilities against
central differences of the oracle's own propagation."""
import math

import numpy as np
import pytest

import brute_force as BF
import wpccc_inputs as wi
from oracle import wpccc_oracle as O

SMALL = dict(nmax=2, lmax=1, nbins=2, kmax=1.5, Nr=400, rmax=40.0, Geta=16, Gtau=16)
THETA0 = dict(Z_p=1.0, a=3.1, b=1.45)


def _shifted(name, h):
    kw = dict(THETA0)
    kw[name] += h
    return wi.li_basis(**kw, **SMALL)


@pytest.fixture(scope="module")
def small():
    return wi.li_basis(**THETA0, **SMALL)


def test_box_states_reduce_to_hydrogenic_energies():
    # a pure Coulomb potential: the discrete eigenvalues approach -Z^2/(2 n^2); with c = 2, a = b = 0 the
    # model potential is -3/r near and far, so its (valence) 2s/2p levels are those of Z = 3
    g = wi.radial_grid(2000, 100.0)
    zero = lambda r: np.zeros_like(r)
    for Z, skip, V in ((1.0, False, lambda r: -1.0 / r), (3.0, True, wi.li_model_potential(2.0, 0.0, 0.0)[0])):
        c, _ = wi.box_centre(V, [zero], 3, 1, 0, 1.0, g, skip_lowest_s=skip)
        for e, n in zip(c.rad_eps, c.rad_n):
            assert abs(e + Z * Z / (2.0 * n * n)) < 2e-4 * Z * Z


def test_basis_tangents_are_derivatives_of_the_generator():
    base = wi.li_basis(**THETA0, **SMALL)
    for p, name in enumerate(base.theta_names):
        errs = []
        for h in (1e-2, 1e-3):
            bp, bm = _shifted(name, h), _shifted(name, -h)
            for c0, cp, cm, tg in ((base.T, bp.T, bm.T, base.tangent_T), (base.P, bp.P, bm.P, base.tangent_P)):
                assert cp.f.shape == c0.f.shape
                fd = (cp.f - cm.f) / (2 * h)
                errs.append(np.abs(fd - tg.df[p]).max() / max(1e-300, np.abs(tg.df[p]).max() + 1e-3))
                assert np.abs((cp.rad_eps - cm.rad_eps) / (2 * h) - tg.deps[p]).max() < 1e-4 * (h / 1e-2) ** 2 + 1e-9
        # second-order convergence of the central difference towards the tangent
        assert errs[2] < 2e-2 * errs[0] + 1e-7 and errs[3] < 2e-2 * errs[1] + 1e-7


def test_model_potential_elements_brute_force():
    # hydrogenic states on both centres, Li-like potential on the target: D_P's short-range part and Q
    g = wi.radial_grid(1500)
    nl = [(1, 0), (2, 1)]

    def centre(Z):
        f = [wi.hydrogenic_radial(n, l, Z, g.r) for n, l in nl]
        return wi.centre_from_functions(Z, [l for _, l in nl], [n for n, _ in nl], f, np.zeros(len(nl)))
    T, P = centre(1.0), centre(1.0)
    c, a, bb = 2.0, 2.0, 1.2
    basis = wi.Basis(grid=g, T=T, P=P, quad=wi.make_quadrature(48, 48, 0.5), Z_T=1.0, Z_P=1.0,
                     mp_c=c, mp_a=a, mp_b=bb)
    b, z, v = 0.9, 0.6, 0.8
    Vs = lambda r: -c * np.exp(-a * r) * (1.0 + bb * r) / r
    states = lambda C: [(int(C.rad_n[C.st_rad[i]]), int(C.st_l[i]), int(C.st_m[i]), 1.0) for i in range(C.N)]
    th = math.acos(z / math.hypot(b, z))
    DR = O.rotation_matrix(P, th)
    Dsr = DR @ O.sr_direct_mol(basis, b, z) @ DR.T
    Dbf = BF.potential_elements(states(P), Vs, b, z, centre_is_projectile=True, n_u=200, n_tau=120)
    assert np.abs(Dsr - Dbf).max() < 2e-5 * max(1.0, np.abs(Dbf).max())
    assert np.abs(Dbf).max() > 1e-2
    S, H = O.assemble(basis, b, v, z)
    _, Qbf, _ = BF.two_centre_elements(states(T), states(P), 1.0, 1.0, b, z, v,
                                       VT=lambda r: -1.0 / r + Vs(r), n_u=200, n_tau=120)
    NT = T.N
    assert np.abs(H[:NT, NT:] - Qbf).max() < 2e-6 * max(1.0, np.abs(Qbf).max())


@pytest.mark.parametrize("name", ["Z_p", "a", "b"])
def test_element_tangents_match_central_differences(small, name):
    b, v, z = 1.1, 1.5, 0.3
    S, H, dS, dH = O.assemble_with_tangents(small, b, v, z)
    p = small.theta_names.index(name)
    h = 1e-4
    Sp, Hp = O.assemble(_shifted(name, h), b, v, z)
    Sm, Hm = O.assemble(_shifted(name, -h), b, v, z)
    assert np.abs((Sp - Sm) / (2 * h) - dS[p]).max() < 1e-7
    assert np.abs((Hp - Hm) / (2 * h) - dH[p]).max() < 1e-7
    assert np.abs(dH[p]).max() > 1e-2


def test_gradient_matches_central_differences_of_the_oracle(small):
    b, v = 0.9, 1.5
    zg = wi.uniform_zgrid(-3.0, 3.0, 0.5)
    g = wi.observable_weights(small)
    P, dP, X = O.gradient(small, b, v, zg, g)
    assert np.allclose(P, g @ O.probabilities(O.propagate(small, b, v, zg)), rtol=1e-13, atol=0)
    h = 1e-4
    for p, name in enumerate(small.theta_names):
        Pp = g @ O.probabilities(O.propagate(_shifted(name, h), b, v, zg))
        Pm = g @ O.probabilities(O.propagate(_shifted(name, -h), b, v, zg))
        fd = (Pp - Pm) / (2 * h)
        assert np.all(np.abs(fd - dP[:, p]) <= 3e-6 * np.abs(dP[:, p]) + 1e-10), (name, fd, dP[:, p])


def test_gradient_without_phase_derivative_fails(small):
    # a plausible slip planted in the oracle's inputs: differentiating the elements but not their energy
    # phases (energy tangents zeroed) moves the gradient far outside the central-difference tolerance
    import copy
    b, v = 0.9, 1.5
    zg = wi.uniform_zgrid(-3.0, 3.0, 0.5)
    g = wi.observable_weights(small)
    _, dP_ok, _ = O.gradient(small, b, v, zg, g)
    nophase = copy.copy(small)
    nophase.tangent_T = wi.CentreTangent(df=small.tangent_T.df, deps=np.zeros_like(small.tangent_T.deps))
    nophase.tangent_P = wi.CentreTangent(df=small.tangent_P.df, deps=np.zeros_like(small.tangent_P.deps))
    _, dP_bad, _ = O.gradient(nophase, b, v, zg, g)
    assert np.abs(dP_bad - dP_ok).max() > 1e3 * 3e-6 * np.abs(dP_ok).max()
