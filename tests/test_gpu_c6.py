"""The bare C6+ on H workload (projectile charge 6, N_T = N_P = 811, N = 1622): FP64 parity with the oracle
at sampled positions and steps, and the mixed-precision form against the FP64 form.

The C6+ couplings are strong and the two-centre basis is close to linearly dependent near closest
approach, so M has large eigenvalues and RK4 needs short steps there (h |lambda| < 2.8): the workload's
z-grid bounds the step by the basis' stiffness (h = 2e-3 for |z| < 2); the 6-pseudostate variant uses
h = 0.005."""
import numpy as np
import pytest

import wpccc_inputs as wi
from oracle import wpccc_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c6():
    return wi.config_inputs("C6_H_2c_n6l5")


@pytest.fixture(scope="module")
def gbasis(c6):
    import paper_2403_04252_gb300 as w
    g = w.Basis(c6[0])
    yield g
    g.close()


def test_c6_matrix_elements_sampled(c6, gbasis):
    import paper_2403_04252_gb300 as w
    basis, paths = c6
    S, H = gbasis.matrix_elements(2.0, 2.0, np.array([0.3]))
    torch.cuda.synchronize()
    Sg, Hg = w.natural(S).cpu().numpy()[0], w.natural(H).cpu().numpy()[0]
    So, Ho = O.assemble(basis, 2.0, 2.0, 0.3)
    assert np.abs(Sg - So).max() < 1e-12
    assert np.abs(Hg - Ho).max() < 1e-12 * max(1.0, np.abs(Ho).max())


def test_c6_fp64_steps_against_oracle(c6, gbasis):
    import paper_2403_04252_gb300 as w
    basis, paths = c6
    zg = np.array([-2e-4, 0.0, 2e-4])
    c = gbasis.propagate(np.array([1.0]), 2.0, zg, precision_mode=0)
    Pg = w.probabilities(c).cpu().numpy()[0]
    Po = O.probabilities(O.propagate(basis, 1.0, 2.0, zg))
    bound = 1e-10 * np.maximum(Po, 1e-4)
    assert (np.abs(Pg - Po) <= bound).all(), np.abs(Pg - Po).max()


def _window(zg, z_mid, n_steps):
    k = int(np.searchsorted(zg, z_mid))
    k0 = max(0, k - n_steps // 2)
    return zg[k0:k0 + n_steps + 1]


@pytest.mark.parametrize("z_mid", [0.0, 2.0])
def test_c6_precision_forms_against_fp64_on_the_workload_grid(c6, gbasis, z_mid):
    # 128 RK4 steps of the workload's own z-grid, through closest approach (h = 2e-3) and across the
    # |z| = 2 change of step (2e-3 -> 3.9e-3, the stiffest part of the grid relative to its step), on the
    # smallest, a middle and the largest impact parameter, every path checked:
    # * FP64 elements, four-slice tensor-core elements or FP64-accurate tensor-core elements with FP32
    #   factors and two refinement sweeps (modes 2, 3 and 5) within 1e-6 of the FP64 form; mode 5 with four
    #   sweeps at the FP64 bar;
    # * the FP32 CUDA-core contraction (mode 1) misses 1e-6 at b = 0.5, where cond(S) ~ 1.3e3 amplifies its
    #   ~2^-24 element errors (4.1e-6 here, 5.2e-6 over the whole b = 0.5 path): it is held to the 1e-5 it
    #   reaches and is not this workload's reduced-precision form
    import paper_2403_04252_gb300 as w
    basis, paths = c6
    idx = [0, 8, 15]
    zg = _window(paths.z[0], z_mid, 128)
    assert zg.size == 129
    bs, vs = paths.b[idx], paths.v[idx]
    gbasis.set_solve_mode(w.SOLVE_SCHUR)
    try:
        P64 = w.probabilities(gbasis.propagate(bs, vs, zg, precision_mode=0)).cpu().numpy()
        assert np.isfinite(P64).all()
        for mode, iters in ((2, 2), (5, 2), (5, 4), (1, 2), (3, 2)):
            gbasis.set_refine_iters(iters)
            P = w.probabilities(gbasis.propagate(bs, vs, zg, precision_mode=mode)).cpu().numpy()
            err = np.abs(P - P64).max(axis=1)
            print(f"C6+ (N=1622) z~{z_mid} b={bs} mode {mode} ({iters} sweeps) max |dP| per path: {err}")
            if iters == 4:
                assert (np.abs(P - P64) <= 1e-10 * np.maximum(P64, 1e-4)).all(), err
            elif mode in (2, 3, 5):
                assert err.max() <= 1e-6, (mode, err)
            else:
                assert err.max() <= 1e-5, (mode, err)
    finally:
        gbasis.set_refine_iters(2)
        gbasis.set_solve_mode(w.SOLVE_STAGE)


def test_c6_lu_and_schur_solves_agree_on_the_workload_grid(c6, gbasis):
    import paper_2403_04252_gb300 as w
    basis, paths = c6
    zg = _window(paths.z[0], 0.0, 32)
    P_lu = w.probabilities(gbasis.propagate(paths.b[:1], paths.v[:1], zg, precision_mode=0)).cpu().numpy()
    gbasis.set_solve_mode(w.SOLVE_SCHUR)
    try:
        P_sc = w.probabilities(gbasis.propagate(paths.b[:1], paths.v[:1], zg, precision_mode=0)).cpu().numpy()
    finally:
        gbasis.set_solve_mode(w.SOLVE_STAGE)
    assert (np.abs(P_sc - P_lu) <= 1e-10 * np.maximum(P_lu, 1e-4)).all()


def test_c6_mixed_against_fp64_small_basis_closest_approach():
    import paper_2403_04252_gb300 as w
    basis, paths = wi.config_inputs("C6_H_2c_n6l5", nbins=6)
    g = w.Basis(basis)
    bs = np.array([0.5, 1.5, 3.0, 6.0])
    zg = wi.uniform_zgrid(-1.0, 1.0, 0.005)
    c64 = g.propagate(bs, 2.0, zg, precision_mode=0)
    P64 = w.probabilities(c64).cpu().numpy()
    # (neither sum |c|^2 nor c^+ S c is conserved in the two-centre form: d(c^+ S c)/dz = c^+ (dS/dz) c)
    assert np.isfinite(P64).all()
    for mode in (2, 5, 1):
        cmx = g.propagate(bs, 2.0, zg, precision_mode=mode)
        err = np.abs(w.probabilities(cmx).cpu().numpy() - P64).max(axis=1)
        print(f"C6+ (N=614) b: {bs} mode {mode} max |dP| per path:", err)
        # modes 2 and 5 everywhere; mode 1's FP32 elements reach the 1e-5 level at b = 0.5 (see above)
        assert err.max() <= (1e-6 if mode != 1 else 1e-5)
    g.close()
