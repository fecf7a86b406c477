"""wpccc_matrix_elements_noalloc: the element call for callers that cannot let the library allocate
device memory (a framework that reserved the device memory up front, or a latency-critical loop that
cannot take cudaMalloc's device-wide synchronisation).  Its scratch lives in a fixed 64 MiB array
inside the library.

Checked through the C ABI against wpccc_matrix_elements on the same basis, on two calls in a row (the
array keeps the previous call's contents, which must not leak into the next result).  This file is
collected last so that a failure here never hides the other GPU tests.
"""
import numpy as np
import pytest

import wpccc_inputs as wi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _compare(g, w, b, v, zs):
    N = g.N
    S0 = torch.empty((len(zs), N, N), dtype=torch.complex128, device="cuda")
    H0 = torch.empty_like(S0)
    g.matrix_elements(b, v, np.asarray(zs), S0, H0)
    # poison the outputs so that an element the no-alloc call fails to write shows up
    S1 = torch.full_like(S0, complex(float("nan"), 0.0))
    H1 = torch.full_like(S0, complex(float("nan"), 0.0))
    g.matrix_elements_noalloc(b, v, np.asarray(zs), S1, H1)
    torch.cuda.synchronize()
    assert torch.isfinite(torch.view_as_real(S1)).all() and torch.isfinite(torch.view_as_real(H1)).all()
    scale = max(1.0, H0.abs().max().item())
    assert (S1 - S0).abs().max().item() <= TOL
    assert (H1 - H0).abs().max().item() <= TOL * scale


def test_noalloc_matches_matrix_elements_two_calls_in_a_row():
    import paper_2403_04252_gb300 as w
    basis, paths = wi.config_inputs("p_H_2c_n4l3")      # 4.5 MB of scratch per position: 14 per group
    g = w.Basis(basis)
    _compare(g, w, 0.7, 1.5, np.linspace(-3.0, 3.0, 20))      # two groups
    _compare(g, w, 5.0, 1.5, [-50.0, 0.05, 12.5])              # second call, other path
    g.close()


def test_noalloc_one_centre_and_small_two_centre():
    import paper_2403_04252_gb300 as w
    b1, _ = wi.config_inputs("p_H_1c_n3l2")
    g1 = w.Basis(b1)
    _compare(g1, w, 2.0, 1.0, [-4.0, 0.0, 1.5])
    _compare(g1, w, 0.5, 1.0, [7.0])
    g1.close()
    b2 = wi.make_basis(1.0, 6.0, (3, 2), (2, 1), (3, 2), (3.0, 4.0), True, Nr=600, Geta=18, Gtau=16)
    g2 = w.Basis(b2)
    _compare(g2, w, 0.9, 1.3, [-7.3, 0.0, 140.0])
    _compare(g2, w, 2.2, 0.8, [0.4, 0.5])
    g2.close()


def test_noalloc_rejects_a_basis_beyond_the_fixed_scratch():
    import paper_2403_04252_gb300 as w
    # 240 x 240 nodes: one position needs ~75 MB of scratch, more than the 64 MiB array
    basis = wi.make_basis(1.0, 1.0, 4, 3, 10, 3.0, True, Nr=600, Geta=240, Gtau=240)
    g = w.Basis(basis)
    S = torch.empty((1, g.N, g.N), dtype=torch.complex128, device="cuda")
    H = torch.empty_like(S)
    with pytest.raises(w.WpcccError) as e:
        g.matrix_elements_noalloc(1.0, 1.0, [0.0], S, H)
    assert e.value.status == w.EINVAL
    assert "scratch" in str(e.value)
    g.close()
