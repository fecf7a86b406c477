"""Differentiation form on the GPU: the Li-like model-potential target (elements and propagation
against the oracle) and wpccc_propagate_adjoint (gradients against the oracle's forward-mode
gradient, against central differences of the GPU's own propagation, and invariance under the
checkpoint interval), through the C ABI."""
import numpy as np
import pytest

import wpccc_inputs as wi
from oracle import wpccc_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TINY = dict(nmax=2, lmax=1, nbins=2, kmax=1.5, Nr=400, rmax=40.0, Geta=16, Gtau=16)
MED = dict(nmax=3, lmax=2, nbins=3, kmax=2.0, Nr=600, rmax=50.0, Geta=24, Gtau=20)
THETA = (1.0, 3.1, 1.45)


def _basis(theta=THETA, **kw):
    return wi.li_basis(Z_p=theta[0], a=theta[1], b=theta[2], **kw)


def _natural(t):
    return t.transpose(-1, -2).cpu().numpy()


@pytest.fixture(scope="module")
def w():
    import paper_2403_04252_gb300 as w
    return w


@pytest.mark.parametrize("kw", [TINY, MED])
def test_model_potential_elements_match_oracle(w, kw):
    basis = _basis(**kw)
    g = w.Basis(basis)
    zs = np.array([-6.0, -0.4, 0.0, 0.7, 35.0])
    for b, v in ((0.8, 1.5), (3.0, 0.9)):
        S, H = g.matrix_elements(b, v, zs)
        torch.cuda.synchronize()
        Sg, Hg = _natural(S), _natural(H)
        for k, z in enumerate(zs):
            So, Ho = O.assemble(basis, b, v, z)
            assert np.abs(Sg[k] - So).max() < 1e-12
            assert np.abs(Hg[k] - Ho).max() < 1e-12 * max(1.0, np.abs(Ho).max())
    g.close()


def test_model_potential_propagation_matches_oracle(w):
    basis = _basis(**MED)
    g = w.Basis(basis)
    zg = wi.uniform_zgrid(-4.0, 4.0, 0.25)
    bs = [0.6, 2.0]
    c = g.propagate(bs, 1.5, zg)
    P = w.probabilities(c).cpu().numpy()
    for k, b in enumerate(bs):
        Po = O.probabilities(O.propagate(basis, b, 1.5, zg))
        assert np.all(np.abs(P[k] - Po) <= 1e-10 * np.maximum(Po, 1e-4))
    # mode 2 (FP64 elements, FP32 LU + refinement) also takes model potentials; mode 1 does not
    c2 = g.propagate(bs, 1.5, zg, precision_mode=2)
    assert np.abs(w.probabilities(c2).cpu().numpy() - P).max() < 1e-6
    with pytest.raises(w.WpcccError) as e:
        g.propagate(bs, 1.5, zg, precision_mode=1)
    assert e.value.status == w.EUNSUPPORTED
    g.close()


def test_gradient_matches_oracle_forward_mode(w):
    basis = _basis(**TINY)
    g = w.Basis(basis)
    gw = wi.observable_weights(basis)
    zg = wi.uniform_zgrid(-3.0, 3.0, 0.5)          # 12 steps: segments of 5, 5 and 2
    bs = [0.9, 2.2]
    c, P, J = g.propagate_adjoint(bs, 1.5, zg, gw, checkpoint_every=5)
    P, J = P.cpu().numpy(), J.cpu().numpy()
    for k, b in enumerate(bs):
        Po, dPo, Xo = O.gradient(basis, b, 1.5, zg, gw)
        assert np.allclose(P[k], Po, rtol=1e-10, atol=1e-14)
        assert np.all(np.abs(J[k] - dPo) <= 1e-9 * np.abs(dPo) + 1e-12), (J[k], dPo)
        assert np.abs(c[k].cpu().numpy() - Xo).max() < 1e-11
    g.close()


def test_gradient_is_independent_of_the_checkpoint_interval(w):
    basis = _basis(**MED)
    g = w.Basis(basis)
    gw = wi.observable_weights(basis)
    zg = wi.uniform_zgrid(-2.0, 2.0, 0.2)          # 20 steps
    out = [g.propagate_adjoint([1.1], 1.5, zg, gw, checkpoint_every=K)[2].cpu().numpy() for K in (1, 3, 20, 50)]
    for J in out[1:]:
        assert np.abs(J - out[0]).max() <= 1e-12 * np.abs(out[0]).max()
    g.close()


def test_gradient_ragged_paths_equal_single_path_calls(w):
    basis = _basis(**MED)
    g = w.Basis(basis)
    gw = wi.observable_weights(basis)
    zgs = [wi.uniform_zgrid(-2.0, 1.0, 0.25), wi.uniform_zgrid(-1.0, 1.2, 0.2), np.array([0.3])]
    bs, vs = [0.7, 1.9, 1.0], [1.5, 1.2, 1.5]
    _, P, J = g.propagate_adjoint(bs, vs, zgs, gw, checkpoint_every=4)
    P, J = P.cpu().numpy(), J.cpu().numpy()
    for k in range(3):
        _, Pk, Jk = g.propagate_adjoint([bs[k]], [vs[k]], [zgs[k]], gw, checkpoint_every=4)
        assert np.abs(P[k] - Pk.cpu().numpy()[0]).max() < 1e-14
        assert np.abs(J[k] - Jk.cpu().numpy()[0]).max() <= 1e-13 * max(1e-300, np.abs(J[k]).max())
    # a path without steps: observables of the initial state, zero derivative
    assert np.allclose(P[2], gw[:, 0]) and np.all(J[2] == 0.0)
    g.close()


@pytest.mark.parametrize("h, floor", [(1e-5, 5e-8), (1e-4, 5e-9)])
def test_gradient_matches_central_differences(w, h, floor):
    """The derivative of the GPU propagation itself: central differences with the basis regenerated at
    theta +- h.  Their own error has two parts: truncation, O(h^2), and the rounding of the regenerated
    basis (the eigensolver's backward error leaves ~1e-12 noise in the probabilities, ~1e-12/(2h) in
    the difference).  Hence 1e-6 relative plus that floor: ~5e-8 at h = 1e-5, ~5e-9 at h = 1e-4."""
    basis = _basis(**MED)
    g = w.Basis(basis)
    gw = wi.observable_weights(basis)
    zg = wi.uniform_zgrid(-3.0, 3.0, 0.2)
    bs = [0.8, 2.4]
    _, P, J = g.propagate_adjoint(bs, 1.5, zg, gw, checkpoint_every=7)
    J = J.cpu().numpy()
    g.close()
    for p in range(3):
        vals = []
        for sgn in (1.0, -1.0):
            th = list(THETA)
            th[p] += sgn * h
            gp = w.Basis(_basis(tuple(th), **MED))
            c = gp.propagate(bs, 1.5, zg)
            vals.append(w.probabilities(c).cpu().numpy() @ gw.T)
            gp.close()
        fd = (vals[0] - vals[1]) / (2 * h)
        assert np.all(np.abs(fd - J[:, :, p]) <= 1e-6 * np.abs(J[:, :, p]) + floor), (p, fd, J[:, :, p])


def test_autograd_function_backward(w):
    gw = wi.observable_weights(_basis(**TINY))
    zg = wi.uniform_zgrid(-2.0, 2.0, 0.5)
    bs = np.array([0.9, 2.2])
    theta = torch.tensor(THETA, dtype=torch.float64, requires_grad=True)
    make = lambda th: _basis(tuple(th), **TINY)
    P = w.observables(theta, make, bs, 1.5, zg, gw, checkpoint_every=3)
    wts = torch.tensor(wi.cross_section_weights(bs), dtype=torch.float64, device=P.device)
    sigma = (wts[:, None] * P).sum(0)                 # capture and 2p-excitation cross sections
    sigma[0].backward()
    g = w.Basis(make(THETA))
    _, _, J = g.propagate_adjoint(bs, 1.5, zg, gw, checkpoint_every=3)
    g.close()
    ref = (wts[:, None] * J[:, 0, :]).sum(0).cpu()
    assert torch.allclose(theta.grad, ref, rtol=1e-13, atol=0)
    # without a gradient the plain propagation gives the same observables
    with torch.no_grad():
        P2 = w.observables(theta.detach(), make, bs, 1.5, zg, gw)
    assert torch.allclose(P.detach(), P2, rtol=1e-12, atol=1e-15)


def test_adjoint_argument_errors(w):
    basis = _basis(**TINY)
    g = w.Basis(basis)
    gw = wi.observable_weights(basis)
    zg = wi.uniform_zgrid(-1.0, 1.0, 0.5)
    with pytest.raises(w.WpcccError) as e:
        g.propagate_adjoint([1.0], 1.0, zg, np.zeros((5, g.N)))
    assert e.value.status == w.EINVAL
    with pytest.raises(w.WpcccError) as e:
        g.propagate_adjoint([1.0], 1.0, zg, gw, checkpoint_every=0)
    assert e.value.status == w.EINVAL
    g.close()
    bare = wi.make_basis(1.0, 1.0, 2, 1, 2, 1.5, True, Nr=400, rmax=40.0, Geta=16, Gtau=16)
    gb = w.Basis(bare)
    with pytest.raises(w.WpcccError) as e:
        gb.propagate_adjoint([1.0], 1.0, zg, np.zeros((2, gb.N)))
    assert e.value.status == w.EINVAL and "tangents" in str(e.value)
    gb.close()
    one = wi.config_inputs("p_H_1c_n3l2", nbins=2, Nr=400, rmax=40.0)[0]
    g1 = w.Basis(one)
    with pytest.raises(w.WpcccError):
        g1.set_tangents(np.zeros((1, one.T.n_rad, 400)), np.zeros((1, one.T.n_rad)), np.zeros((1, 1, 400)),
                        np.zeros((1, 1)), np.zeros((1, 4)))
    g1.close()
