"""Failure paths on the GPU, made on the host (no fault, trap or endless wait on the device).

* ETIMEOUT: the tensor-core kernels' mbarrier waits are bounded.  With the limit set to one poll the waits
  run out: every CTA records the failure, lets its copies and MMAs in flight complete, frees its tensor
  memory and returns; the call reports ETIMEOUT, and the next call with the default limit gives the same
  elements as before, so the device stayed usable.
* ENONFINITE: amplitudes with a NaN, passed in from the host, are reported after the propagation.
* ENOCONV: the refined forms check the last refinement sweep's correction against the solution; a
  tolerance no correction can meet makes the propagation report non-convergence, the default passes.
"""
import numpy as np
import pytest

import wpccc_inputs as wi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _small():
    # 16 x 16 nodes: a multiple of 128, as the tensor-core layout needs
    return wi.make_basis(1.0, 1.0, 2, 1, 2, 2.0, True, Nr=600, Geta=16, Gtau=16)


@pytest.mark.parametrize("mode", [3, 4])
def test_tensor_core_wait_limit_gives_timeout_and_the_device_recovers(mode):
    import paper_2403_04252_gb300 as w
    g = w.Basis(_small())
    zs = np.array([-1.0, 0.0, 0.7])
    S0, H0 = g.matrix_elements_precision(0.8, 1.2, zs, mode)
    torch.cuda.synchronize()
    g.set_wait_limit(1)
    with pytest.raises(w.WpcccError) as e:
        g.matrix_elements_precision(0.8, 1.2, zs, mode)
    assert e.value.status == w.ETIMEOUT
    with pytest.raises(w.WpcccError) as e:
        g.propagate([0.8], 1.2, wi.uniform_zgrid(-1.0, 1.0, 0.5), precision_mode=mode)
    assert e.value.status == w.ETIMEOUT
    g.set_wait_limit(w.DEFAULT_WAIT_POLLS)
    S1, H1 = g.matrix_elements_precision(0.8, 1.2, zs, mode)
    torch.cuda.synchronize()
    assert torch.equal(S0, S1) and torch.equal(H0, H1)
    c = g.propagate([0.8], 1.2, wi.uniform_zgrid(-1.0, 1.0, 0.5), precision_mode=mode)
    assert torch.isfinite(torch.view_as_real(c)).all()
    g.close()


@pytest.mark.parametrize("mode", [0, 1, 3])
def test_nan_amplitudes_are_reported(mode):
    import paper_2403_04252_gb300 as w
    g = w.Basis(_small())
    c = torch.zeros((2, g.N), dtype=torch.complex128, device="cuda")
    c[:, 0] = 1.0
    c[1, 3] = complex(float("nan"), 0.0)
    with pytest.raises(w.WpcccError) as e:
        g.propagate([0.8, 2.0], 1.2, wi.uniform_zgrid(-1.0, 1.0, 0.25), c=c, precision_mode=mode)
    assert e.value.status == w.ENONFINITE
    ok = g.propagate([0.8, 2.0], 1.2, wi.uniform_zgrid(-1.0, 1.0, 0.25), precision_mode=mode)
    assert torch.isfinite(torch.view_as_real(ok)).all()
    g.close()


@pytest.mark.parametrize("solve", ["stage", "schur"])
def test_refinement_convergence_check(solve):
    import paper_2403_04252_gb300 as w
    g = w.Basis(_small())
    g.set_solve_mode(w.SOLVE_STAGE if solve == "stage" else w.SOLVE_SCHUR)
    zg = wi.uniform_zgrid(-1.0, 1.0, 0.25)
    P64 = w.probabilities(g.propagate([0.8], 1.2, zg, precision_mode=0)).cpu().numpy()
    P2 = w.probabilities(g.propagate([0.8], 1.2, zg, precision_mode=2)).cpu().numpy()   # default 1e-3
    assert np.abs(P2 - P64).max() < 1e-10
    g.set_refine_tolerance(1e-30)
    with pytest.raises(w.WpcccError) as e:
        g.propagate([0.8], 1.2, zg, precision_mode=2)
    assert e.value.status == w.ENOCONV
    g.set_refine_iters(1)            # a single preconditioner solve has no correction to check
    g.propagate([0.8], 1.2, zg, precision_mode=2)
    g.set_refine_iters(2)
    g.set_refine_tolerance(0.0)      # off
    g.propagate([0.8], 1.2, zg, precision_mode=2)
    g.close()
