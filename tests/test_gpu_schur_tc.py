"""The FP32 preconditioner of the mixed Schur forms with the trailing update I - K^+ K formed on the tensor
cores (tcgen05, four fixed-point bf16 slices per operand, exact FP32 level accumulators): the refined
propagation with it reaches the FP64 form within 1e-6 with two refinement sweeps and at the FP64 bar with
four, on bases whose projectile block is not a multiple of the 128 x 64 tiles (uneven centres, N_P = 13,
190 and 286)."""
import numpy as np
import pytest

import wpccc_inputs as wi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bases():
    uneven = wi.make_basis(1.0, 6.0, (3, 2), (2, 1), (3, 2), (3.0, 4.0), True, Nr=600, Geta=16, Gtau=16)
    p_h, _ = wi.config_inputs("p_H_2c_n4l3")
    v4 = [bs for v, bs, _ in wi.batch_inputs(n_b=2, speeds=(4.0,))][0]
    return [("uneven", uneven, 1.3, wi.uniform_zgrid(-2.0, 2.0, 0.1)),
            ("p_H", p_h, 1.5, wi.uniform_zgrid(-0.8, 0.8, 0.1)),
            ("v4", v4, 4.0, wi.uniform_zgrid(-1.2, 1.2, 0.2))]


@pytest.mark.parametrize("name,basis,v,zg", _bases(), ids=lambda x: x if isinstance(x, str) else "")
def test_refined_schur_forms_with_tensor_core_update(name, basis, v, zg):
    import paper_2403_04252_gb300 as w
    g = w.Basis(basis)
    g.set_solve_mode(w.SOLVE_SCHUR)
    g.set_schur_update(w.SCHUR_UPDATE_TENSOR)
    bs = np.array([0.2, 0.9, 3.0])
    P64 = w.probabilities(g.propagate(bs, v, zg, precision_mode=0)).cpu().numpy()
    g.set_refine_iters(2)
    P2 = w.probabilities(g.propagate(bs, v, zg, precision_mode=2)).cpu().numpy()
    assert np.abs(P2 - P64).max() <= 1e-6, np.abs(P2 - P64).max()
    g.set_refine_iters(4)
    P4 = w.probabilities(g.propagate(bs, v, zg, precision_mode=2)).cpu().numpy()
    assert (np.abs(P4 - P64) <= 1e-10 * np.maximum(P64, 1e-4)).all(), np.abs(P4 - P64).max()
    # the CUDA-core update gives the same propagation within the same bars
    g.set_schur_update(w.SCHUR_UPDATE_CUDA_CORES)
    Pc = w.probabilities(g.propagate(bs, v, zg, precision_mode=2)).cpu().numpy()
    assert (np.abs(Pc - P64) <= 1e-10 * np.maximum(P64, 1e-4)).all(), np.abs(Pc - P64).max()
    print(f"{name}: N_T={g.N_T} N_P={g.N_P} two sweeps {np.abs(P2 - P64).max():.2e}, four {np.abs(P4 - P64).max():.2e}")
    g.close()
