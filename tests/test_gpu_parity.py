"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same generated inputs.

Bars: matrix elements and solves agree to FP64 rounding (scaled tolerances
below); probabilities agree to |dP| <= 1e-10 * max(P, 1e-4).
"""
import math

import numpy as np
import pytest

import wpccc_inputs as wi
from oracle import wpccc_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P_TOL = 1e-10


def _w():
    import paper_2403_04252_gb300 as w
    return w


def _prob_close(Pg, Po):
    bound = P_TOL * np.maximum(Po, 1e-4)
    bad = np.abs(Pg - Po) > bound
    assert not bad.any(), f"max |dP| = {np.abs(Pg - Po).max():.3e} at {np.nonzero(bad)}"


@pytest.fixture(scope="module")
def small2c():
    # ragged sizes: 13 states per centre (N = 26) and a 20 x 14 quadrature, neither a multiple of a tile
    return wi.make_basis(1.0, 1.0, 2, 1, 2, 2.0, True, Nr=600, Geta=20, Gtau=14)


@pytest.fixture(scope="module")
def small2c_uneven():
    # different charges and basis sizes on the two centres (C6+ + H like)
    return wi.make_basis(1.0, 6.0, (3, 2), (2, 1), (3, 2), (3.0, 4.0), True, Nr=600, Geta=18, Gtau=16)


@pytest.fixture(scope="module")
def config1():
    return wi.config_inputs("p_H_1c_n3l2")


@pytest.fixture(scope="module")
def config2():
    return wi.config_inputs("p_H_2c_n4l3")


def _elements(basis, b, v, zs):
    w = _w()
    g = w.Basis(basis)
    S, H = g.matrix_elements(b, v, np.asarray(zs))
    torch.cuda.synchronize()
    return w.natural(S).cpu().numpy(), w.natural(H).cpu().numpy()


@pytest.mark.parametrize("fixture", ["small2c", "small2c_uneven"])
def test_matrix_elements_small_two_centre(request, fixture):
    basis = request.getfixturevalue(fixture)
    b, v = 0.9, 1.3
    zs = [-7.3, -0.4, 0.0, 0.25, 3.1, 60.0, 140.0]      # 140: R beyond the grid
    Sg, Hg = _elements(basis, b, v, zs)
    for k, z in enumerate(zs):
        So, Ho = O.assemble(basis, b, v, z)
        scale = max(1.0, np.abs(Ho).max())
        assert np.abs(Sg[k] - So).max() < 1e-12, (z, np.abs(Sg[k] - So).max())
        assert np.abs(Hg[k] - Ho).max() < 1e-12 * scale, (z, np.abs(Hg[k] - Ho).max())


def test_matrix_elements_one_centre(config1):
    basis, paths = config1
    zs = [-40.0, -3.05, 0.0, 0.05, 12.0]
    Sg, Hg = _elements(basis, 2.5, 1.0, zs)
    for k, z in enumerate(zs):
        So, Ho = O.assemble(basis, 2.5, 1.0, z)
        assert np.array_equal(Sg[k], np.eye(basis.N))
        assert np.abs(Hg[k] - Ho).max() < 1e-13 * max(1.0, np.abs(Ho).max())


def test_matrix_elements_full_two_centre_sampled(config2):
    # the full p + H two-centre basis (N = 380, 48 x 48 nodes) at sampled positions
    basis, paths = config2
    b = float(paths.b[3])
    zs = [-50.0, -0.35, 1.05]
    Sg, Hg = _elements(basis, b, 1.5, zs)
    for k, z in enumerate(zs):
        So, Ho = O.assemble(basis, b, 1.5, z)
        assert np.abs(Sg[k] - So).max() < 1e-12
        assert np.abs(Hg[k] - Ho).max() < 1e-12 * max(1.0, np.abs(Ho).max())


@pytest.mark.parametrize("N", [1, 5, 31, 32, 33, 100, 259])
def test_solve_random_systems(N):
    w = _w()
    rng = np.random.default_rng(N)
    batch = 3
    A = rng.standard_normal((batch, N, N)) + 1j * rng.standard_normal((batch, N, N)) + 3 * np.eye(N)
    B = rng.standard_normal((batch, N, N)) + 1j * rng.standard_normal((batch, N, N))
    S = w.colmajor(torch.from_numpy(A).cuda())
    H = w.colmajor(torch.from_numpy(B).cuda())
    ipiv, info = w.solve(S, H)
    torch.cuda.synchronize()
    X = w.natural(H).cpu().numpy()
    LU = w.natural(S).cpu().numpy()
    piv = ipiv.cpu().numpy()
    assert (info.cpu().numpy() == 0).all()
    for k in range(batch):
        Xo = np.linalg.solve(A[k], B[k])
        cond = np.linalg.cond(A[k])
        assert np.abs(X[k] - Xo).max() < 1e-13 * cond * max(1.0, np.abs(Xo).max())
        # P A = L U with LAPACK's 1-based interchanges
        PA = A[k].copy()
        for i in range(N):
            p = piv[k, i] - 1
            assert i <= p < N
            PA[[i, p]] = PA[[p, i]]
        L = np.tril(LU[k], -1) + np.eye(N)
        U = np.triu(LU[k])
        assert np.abs(L @ U - PA).max() < 1e-13 * N * np.abs(A[k]).max()


def test_solve_pivot_matches_partial_pivoting():
    w = _w()
    A = np.array([[1e-3, 2.0, 0.0], [3.0, 1.0, 1.0], [-4.0, 0.5, 2.0]], dtype=complex)
    B = np.eye(3, dtype=complex)[None]
    S = w.colmajor(torch.from_numpy(A[None].copy()).cuda())
    H = w.colmajor(torch.from_numpy(B.copy()).cuda())
    ipiv, info = w.solve(S, H)
    torch.cuda.synchronize()
    assert ipiv.cpu().numpy()[0, 0] == 3        # largest |re|+|im| in column 1 is row 3
    assert np.allclose(w.natural(H).cpu().numpy()[0], np.linalg.inv(A), atol=1e-14)


def test_solve_singular_reports_info():
    w = _w()
    A = np.eye(4, dtype=complex)
    A[:, 2] = 0.0
    S = w.colmajor(torch.from_numpy(A[None].copy()).cuda())
    H = w.colmajor(torch.from_numpy(np.eye(4, dtype=complex)[None].copy()).cuda())
    ipiv, info = w.solve(S, H)
    torch.cuda.synchronize()
    assert info.cpu().numpy()[0] == 3


def test_solve_assembled_overlap(config2):
    # the solve on a real two-centre S(z) (small b: the least well-conditioned case)
    basis, paths = config2
    w = _w()
    g = w.Basis(basis)
    S, H = g.matrix_elements(0.2, 1.5, np.array([0.0, 0.6]))
    So = w.natural(S).cpu().numpy()
    Ho = w.natural(H).cpu().numpy()
    ipiv, info = w.solve(S, H)
    torch.cuda.synchronize()
    X = w.natural(H).cpu().numpy()
    for k in range(2):
        Xo = O.solve(So[k], Ho[k])
        assert np.abs(X[k] - Xo).max() < 1e-11 * np.abs(Xo).max()


def test_propagate_one_centre_full_paths(config1):
    # the one-centre p + H workload, two of its eight paths over all 800 steps
    basis, paths = config1
    w = _w()
    g = w.Basis(basis)
    idx = [0, 5]
    zg = paths.z[0]
    c = g.propagate(paths.b[idx], paths.v[idx], zg)
    Pg = w.probabilities(c).cpu().numpy()
    for n, p in enumerate(idx):
        Po = O.probabilities(O.propagate(basis, float(paths.b[p]), float(paths.v[p]), zg))
        _prob_close(Pg[n], Po)
    # S = I and D Hermitian: only RK4's O((h w)^6) per-step drift moves the norm
    assert abs(Pg.sum(axis=1) - 1.0).max() < 1e-5


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_propagate_two_centre_ragged_paths_and_chunks(small2c, mode):
    # uneven path lengths and a workspace limit that forces several chunks of steps;
    # the three ways of applying S^-1 (LU per RK4 stage, the paper's X = S^-1 H, and the
    # Cholesky factor of the Schur complement I - K^+ K per RK4 stage)
    w = _w()
    g = w.Basis(small2c)
    g.set_solve_mode(mode)
    g.set_workspace_limit(64 << 20)
    bs = np.array([0.4, 1.7, 3.0])
    zgs = [wi.uniform_zgrid(-6.0, 6.0, 0.25), wi.uniform_zgrid(-5.0, 4.0, 0.3), wi.uniform_zgrid(-2.0, -1.0, 0.5)]
    c = g.propagate(bs, 1.3, zgs)
    Pg = w.probabilities(c).cpu().numpy()
    for p in range(3):
        Po = O.probabilities(O.propagate(small2c, float(bs[p]), 1.3, zgs[p]))
        _prob_close(Pg[p], Po)


def test_propagate_zero_steps_leaves_amplitudes(small2c):
    w = _w()
    g = w.Basis(small2c)
    c0 = torch.zeros((1, g.N), dtype=torch.complex128, device="cuda")
    c0[0, 3] = 0.6 + 0.8j
    c = g.propagate(np.array([1.0]), 1.0, [np.array([0.5])], c=c0.clone())
    assert torch.equal(c, c0)


def test_propagate_rejects_bad_paths(small2c):
    w = _w()
    g = w.Basis(small2c)
    with pytest.raises(w.WpcccError) as e:
        g.propagate(np.array([1.0]), 1.0, [np.array([0.0, -1.0])])
    assert e.value.status == w.EINVAL
    with pytest.raises(w.WpcccError) as e:
        g.propagate(np.array([-1.0]), 1.0, [np.array([0.0, 1.0])])
    assert e.value.status == w.EINVAL


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_propagate_full_two_centre_sampled_paths(config2, mode):
    # the bench launch configuration (all 32 paths of the two-centre p + H workload batched),
    # two RK4 steps from z = -0.2; two sampled paths recomputed by the oracle
    basis, paths = config2
    w = _w()
    g = w.Basis(basis)
    g.set_solve_mode(mode)
    zg = np.array([-0.2, -0.1, 0.0])
    c = g.propagate(paths.b, paths.v, zg)
    Pg = w.probabilities(c).cpu().numpy()
    for p in (0, 17):
        Po = O.probabilities(O.propagate(basis, float(paths.b[p]), float(paths.v[p]), zg))
        _prob_close(Pg[p], Po)


def test_schur_solve_mode_uneven_centres(small2c_uneven):
    # N_T != N_P (C6+ + H like): the Schur complement is the projectile block's, of a different size
    # than the target's; against the oracle, and against the pivoted-LU stage form to FP64 rounding
    w = _w()
    g = w.Basis(small2c_uneven)
    assert g.N_T != g.N - g.N_T
    bs = np.array([0.6, 2.5])
    zg = wi.uniform_zgrid(-4.0, 4.0, 0.25)
    out = {}
    for mode in (w.SOLVE_STAGE, w.SOLVE_SCHUR):
        g.set_solve_mode(mode)
        out[mode] = w.probabilities(g.propagate(bs, 2.0, zg)).cpu().numpy()
    for p in range(2):
        Po = O.probabilities(O.propagate(small2c_uneven, float(bs[p]), 2.0, zg))
        _prob_close(out[w.SOLVE_SCHUR][p], Po)
    assert np.abs(out[w.SOLVE_SCHUR] - out[w.SOLVE_STAGE]).max() < 1e-12
    with pytest.raises(w.WpcccError) as e:
        g.set_solve_mode(3)
    assert e.value.status == w.EINVAL
    g.close()


def test_probabilities_kernel():
    w = _w()
    c = torch.randn(4, 37, dtype=torch.complex128, device="cuda")
    P = w.probabilities(c)
    assert torch.allclose(P, (c.conj() * c).real, rtol=0, atol=1e-15)


# ---------------------------------------------------------------- mixed-precision form
MIXED_TOL = 1e-6     # absolute, per probability


def _mixed_errors(basis, bs, v, zgs, workspace=None, mode=1, solve=None):
    w = _w()
    g = w.Basis(basis)
    if solve is not None:
        g.set_solve_mode(solve)
    if workspace:
        g.set_workspace_limit(workspace)
    c = g.propagate(bs, v, zgs, precision_mode=mode)
    Pg = w.probabilities(c).cpu().numpy()
    errs = []
    for p in range(len(bs)):
        zg = zgs[p] if isinstance(zgs, list) else zgs
        Po = O.probabilities(O.propagate(basis, float(bs[p]), float(v), zg))
        errs.append(np.abs(Pg[p] - Po))
    return np.array(errs)


@pytest.mark.parametrize("solve", [0, 2])
def test_mixed_form_small_two_centre(small2c, solve):
    # mode 1 (FP32 elements, FP32 factors of S, FP64 refinement) on a p + H-like basis, against the
    # oracle; the FP32 factors are the pivoted LU of S (solve mode 0) or the Schur factors (2)
    bs = np.array([0.5, 2.0])
    zgs = [wi.uniform_zgrid(-6.0, 6.0, 0.2), wi.uniform_zgrid(-4.0, 5.0, 0.25)]
    err = _mixed_errors(small2c, bs, 1.3, zgs, workspace=64 << 20, mode=1, solve=solve)
    assert err.max() <= MIXED_TOL, err.max()


@pytest.mark.parametrize("solve", [0, 2])
def test_mixed_fp64_elements_small_uneven_two_centre(small2c_uneven, solve):
    # mode 2 (FP64 elements, FP32 factors, FP64 refinement) on a C6+ on H-like basis (stiff near closest
    # approach: h = 0.05), against the oracle
    bs = np.array([0.5, 2.0])
    zgs = [wi.uniform_zgrid(-3.0, 3.0, 0.05), wi.uniform_zgrid(-2.0, 2.5, 0.05)]
    err = _mixed_errors(small2c_uneven, bs, 1.3, zgs, workspace=64 << 20, mode=2, solve=solve)
    assert err.max() <= MIXED_TOL, err.max()


def test_mixed_form_full_two_centre_sampled(config2):
    basis, paths = config2
    w = _w()
    g = w.Basis(basis)
    zg = wi.uniform_zgrid(-0.6, 0.6, 0.1)
    c = g.propagate(paths.b, paths.v, zg, precision_mode=1)
    Pg = w.probabilities(c).cpu().numpy()
    for p in (0, 9):
        Po = O.probabilities(O.propagate(basis, float(paths.b[p]), float(paths.v[p]), zg))
        assert np.abs(Pg[p] - Po).max() <= MIXED_TOL


def test_mixed_form_full_paths_against_fp64(config2):
    # whole paths (1000 RK4 steps, z from -50 to 50) of the two-centre p + H workload: the mixed form
    # (with either FP32 factorisation) against the plain FP64 form on the GPU (itself within 1e-10 of
    # the oracle, tests above)
    basis, paths = config2
    w = _w()
    g = w.Basis(basis)
    idx = [0, 4, 12, 31]          # b = 0.2, 1.72, 4.77, 12
    zg = paths.z[0]
    c64 = g.propagate(paths.b[idx], paths.v[idx], zg, precision_mode=0)
    P64 = w.probabilities(c64).cpu().numpy()
    for solve in (w.SOLVE_STAGE, w.SOLVE_SCHUR):
        g.set_solve_mode(solve)
        cmx = g.propagate(paths.b[idx], paths.v[idx], zg, precision_mode=1)
        Pmx = w.probabilities(cmx).cpu().numpy()
        err = np.abs(Pmx - P64)
        print("mixed-form max |dP| per path, solve mode", solve, ":", err.max(axis=1))
        assert err.max() <= MIXED_TOL


# ---------------------------------------------------------------- batched form
def test_batch_graph_matches_separate_propagation(small2c, small2c_uneven):
    # three sets of uneven size and step count in one graph launch, against separate propagate calls
    w = _w()
    gA, gB = w.Basis(small2c), w.Basis(small2c_uneven)
    sets = [(gA, np.array([0.4, 2.5]), 1.0, wi.uniform_zgrid(-3.0, 3.0, 0.2)),
            (gA, np.array([1.1, 0.7, 5.0]), 2.0, wi.uniform_zgrid(-2.0, 2.0, 0.4)),
            (gB, np.array([1.5]), 1.3, wi.uniform_zgrid(-1.0, 1.0, 0.05))]
    c = []
    for g, b, v, zg in sets:
        t = torch.zeros((b.size, g.N), dtype=torch.complex128, device="cuda")
        t[:, 0] = 1.0
        c.append(t)
    batch = w.Batch(sets, c, precision_mode=0, autotune=True)
    batch.launch()
    batch.status()
    steps, ms = batch.info()
    assert (steps >= 1).all()
    for (g, b, v, zg), cb in zip(sets, c):
        ref = g.propagate(b, v, zg)
        assert torch.equal(cb, ref)
    # a second launch advances the same amplitudes again through the same segments
    before = [t.clone() for t in c]
    batch.launch()
    batch.status()
    for (g, b, v, zg), cb, c0 in zip(sets, c, before):
        ref = g.propagate(b, v, zg, c=c0.clone())
        assert torch.equal(cb, ref)
    batch.close()


def test_tensor_core_elements_match_fp64_as_closely_as_fp32():
    """Precision mode 3 (Eq. 9 contraction on tcgen05 with fixed-point bf16 slices): element errors
    against the FP64 elements at the level of the FP32 CUDA-core contraction, and no bias (the tensor
    core's FP32 accumulation truncates; the sliced main products are integers it holds exactly)."""
    import paper_2403_04252_gb300 as w
    basis, _ = wi.config_inputs("p_H_2c_n4l3")
    g = w.Basis(basis)
    NT = g.N_T
    zs = np.array([-7.0, -0.55, 0.0, 0.35, 12.0])
    for b in (0.2, 3.2, 11.0):
        S0, H0 = g.matrix_elements_precision(b, 1.5, zs, 0)
        S1, H1 = g.matrix_elements_precision(b, 1.5, zs, 1)
        S3, H3 = g.matrix_elements_precision(b, 1.5, zs, 3)
        torch.cuda.synchronize()
        e1 = max((S1 - S0).abs().max().item(), (H1 - H0).abs().max().item())
        e3 = max((S3 - S0).abs().max().item(), (H3 - H0).abs().max().item())
        assert e3 < 1e-7 and e3 < 3.0 * e1 + 1e-9, (b, e1, e3)
        # no systematic shrink of the two-centre blocks
        X0 = torch.cat([S0[:, :NT, NT:], H0[:, :NT, NT:]]).flatten()
        X3 = torch.cat([S3[:, :NT, NT:], H3[:, :NT, NT:]]).flatten()
        m = X0.abs() > 1e-3
        rel = ((X3[m] - X0[m]) / X0[m]).real
        assert abs(rel.mean().item()) < 2e-8
    g.close()


def test_tensor_core_propagation_within_bound():
    import paper_2403_04252_gb300 as w
    basis, paths = wi.config_inputs("p_H_2c_n4l3")
    g = w.Basis(basis)
    zg = paths.z[0]
    k0 = zg.size // 2 - 8
    seg = zg[k0:k0 + 17]
    bs = paths.b[::4]
    P0 = w.probabilities(g.propagate(bs, 1.5, seg, precision_mode=0)).cpu().numpy()
    P3 = w.probabilities(g.propagate(bs, 1.5, seg, precision_mode=3)).cpu().numpy()
    assert np.abs(P3 - P0).max() < 1e-6
    g.close()


def test_tensor_core_small_uneven_basis_and_errors():
    import paper_2403_04252_gb300 as w
    # groups of different sizes, ragged tiles (N_T = 40, n_half = 27), nodes a multiple of 32
    basis = wi.make_basis(1.0, 1.0, (3, 2), (2, 2), (3, 2), (3.0, 4.0), True, Nr=600, Geta=16, Gtau=16)
    g = w.Basis(basis)
    zs = np.array([-2.0, 0.3, 5.0])
    S0, H0 = g.matrix_elements_precision(0.9, 1.3, zs, 0)
    S3, H3 = g.matrix_elements_precision(0.9, 1.3, zs, 3)
    torch.cuda.synchronize()
    assert (S3 - S0).abs().max().item() < 1e-6 and (H3 - H0).abs().max().item() < 1e-6
    with pytest.raises(w.WpcccError) as e:
        g.matrix_elements_precision(0.9, 1.3, zs, 2)
    assert e.value.status == w.EUNSUPPORTED
    g.close()
    odd = wi.make_basis(1.0, 1.0, 2, 1, 2, 2.0, True, Nr=600, Geta=15, Gtau=13)   # 195 nodes
    go = w.Basis(odd)
    with pytest.raises(w.WpcccError) as e:
        go.matrix_elements_precision(0.9, 1.3, zs, 3)
    assert e.value.status == w.EUNSUPPORTED
    go.close()


def test_batch_graph_tensor_core_matches_separate_propagation():
    # the tensor-core form captured into the batch graph (tensor maps as launch parameters)
    w = _w()
    bA = wi.make_basis(1.0, 1.0, 2, 1, 3, 2.0, True, Nr=600, Geta=16, Gtau=16)
    bB = wi.make_basis(1.0, 1.0, (3, 2), (2, 2), (3, 2), (3.0, 4.0), True, Nr=600, Geta=16, Gtau=16)
    gA, gB = w.Basis(bA), w.Basis(bB)
    sets = [(gA, np.array([0.4, 2.5]), 1.0, wi.uniform_zgrid(-3.0, 3.0, 0.2)),
            (gB, np.array([1.5, 0.8, 3.0]), 1.3, wi.uniform_zgrid(-1.0, 1.0, 0.1))]
    c = []
    for g, b, v, zg in sets:
        t = torch.zeros((b.size, g.N), dtype=torch.complex128, device="cuda")
        t[:, 0] = 1.0
        c.append(t)
    batch = w.Batch(sets, c, precision_mode=3, autotune=False)
    batch.launch()
    batch.status()
    for (g, b, v, zg), cb in zip(sets, c):
        ref = g.propagate(b, v, zg, precision_mode=3)
        assert torch.equal(cb, ref)
        P0 = w.probabilities(g.propagate(b, v, zg, precision_mode=0))
        assert (w.probabilities(cb) - P0).abs().max().item() < 1e-6
    batch.close()
