"""The Python binding refuses, before any call into the library, output and amplitude tensors that the
kernels would write past or misread (wrong dtype, non-contiguous, too short, wrong device).  No GPU is
needed: the checks run on CPU tensors and on a Basis object that holds no device handle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _fake_basis(w, N=6, device=0):
    g = object.__new__(w.Basis)          # no wpccc_basis_create: any library call would fail on a null handle
    g._h = None
    g.N, g.N_T, g.N_P, g.device, g.n_par = N, 3, 3, device, 0
    return g


def test_short_output_is_refused_before_any_launch():
    import paper_2403_04252_gb300 as w
    g = _fake_basis(w)
    z = np.array([0.0, 1.0])
    S = torch.empty((1, 6, 6), dtype=torch.complex128)      # one position, two asked for
    H = torch.empty((2, 6, 6), dtype=torch.complex128)
    for call in (g.matrix_elements_noalloc, g.matrix_elements):
        with pytest.raises(ValueError, match="need 72"):
            call(1.0, 1.0, z, S=S, H=H)
    with pytest.raises(ValueError, match="need 72"):
        g.matrix_elements_precision(1.0, 1.0, z, 3, S=S, H=H)


@pytest.mark.parametrize("bad", ["dtype", "contiguous", "device"])
def test_wrong_output_tensor_is_refused(bad):
    import paper_2403_04252_gb300 as w
    g = _fake_basis(w)
    z = np.array([0.5])
    S = torch.empty((1, 6, 6), dtype=torch.complex128)
    if bad == "dtype":
        S = torch.empty((1, 6, 6), dtype=torch.complex64)
    elif bad == "contiguous":
        S = torch.empty((1, 6, 12), dtype=torch.complex128)[:, :, ::2]
    H = torch.empty((1, 6, 6), dtype=torch.complex128)
    # a CPU tensor of the right dtype, shape and layout still fails: it is not on the basis' device
    msg = {"dtype": "complex128", "contiguous": "contiguous", "device": "cuda:0"}[bad]
    with pytest.raises(ValueError, match=msg):
        g.matrix_elements_noalloc(1.0, 1.0, z, S, H)


def test_wrong_amplitudes_are_refused():
    import paper_2403_04252_gb300 as w
    g = _fake_basis(w)
    zg = np.linspace(-1.0, 1.0, 5)
    with pytest.raises(ValueError, match="need 12"):
        g.propagate([1.0, 2.0], 1.0, zg, c=torch.zeros((1, 6), dtype=torch.complex128))
    with pytest.raises(ValueError, match="complex128"):
        g.propagate([1.0], 1.0, zg, c=torch.zeros((1, 6), dtype=torch.complex64))
    with pytest.raises(ValueError, match="cuda:0"):
        g.propagate_adjoint([1.0], 1.0, zg, np.ones((1, 6)), c=torch.zeros((1, 6), dtype=torch.complex128))
