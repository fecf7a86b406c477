"""Whole paths on the GPU, through the C ABI, at the workloads' own sizes.

* p + H (N = 380, 48 x 48 nodes, v = 1.5): all 32 impact parameters over the full z range [-50, 50]
  (1000 RK4 steps each).  The reduced-precision forms (modes 1 and 3, and mode 5 with two refinement
  sweeps) stay within 1e-6 of the plain FP64 form on every probability of every path; the FP64-accurate
  forms (mode 4, and mode 5 with four sweeps) within the FP64 bar 1e-10 max(P, 1e-4).
* One whole 1000-step FP64 path (b = 0.2, the strongest collision) against the oracle at the FP64 bar;
  the oracle's positions are evaluated by a pool of host processes (tests/oracle_parallel.py).
* The velocity scan (six bases, N = 316..572, 72 x 48 nodes): one path per speed, a few RK4 steps through
  closest approach in the batched graph, against the oracle at the FP64 bar (plain FP64 graph and mode 5
  with four sweeps) and within 1e-6 (mode 5 with two sweeps, the batched form's reduced-precision form).
"""
import numpy as np
import pytest

import wpccc_inputs as wi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P_TOL = 1e-10


def _fp64_bar(P, Pref):
    return np.abs(P - Pref) <= P_TOL * np.maximum(Pref, 1e-4)


@pytest.fixture(scope="module")
def config2():
    return wi.config_inputs("p_H_2c_n4l3")


def test_config2_every_form_over_whole_paths(config2):
    import paper_2403_04252_gb300 as w
    basis, paths = config2
    zg = paths.z[0]
    assert zg.size == 1001 and zg[0] == -50.0 and zg[-1] == 50.0 and paths.n_paths == 32
    g = w.Basis(basis)
    g.set_workspace_limit(16 << 30)
    g.set_solve_mode(w.SOLVE_SCHUR)
    P64 = w.probabilities(g.propagate(paths.b, paths.v, zg, precision_mode=0)).cpu().numpy()
    assert np.isfinite(P64).all()
    for mode, iters, bar in ((1, 2, "1e-6"), (3, 2, "1e-6"), (5, 2, "1e-6"), (4, 2, "fp64"), (5, 4, "fp64")):
        g.set_refine_iters(iters)
        P = w.probabilities(g.propagate(paths.b, paths.v, zg, precision_mode=mode)).cpu().numpy()
        err = np.abs(P - P64).max(axis=1)
        print(f"p + H whole paths, mode {mode} ({iters} sweeps): max |dP| {err.max():.3e} (path {err.argmax()})")
        if bar == "fp64":
            assert _fp64_bar(P, P64).all(), err.max()
        else:
            assert err.max() <= 1e-6, err.max()
    g.close()


def test_config2_fp64_whole_path_against_oracle(config2):
    import oracle_parallel as OP
    from oracle import wpccc_oracle as O
    import paper_2403_04252_gb300 as w
    basis, paths = config2
    zg = paths.z[0]
    b, v = float(paths.b[0]), float(paths.v[0])
    assert b == 0.2
    g = w.Basis(basis)
    Pg = w.probabilities(g.propagate([b], v, zg)).cpu().numpy()[0]
    g.close()
    Po = O.probabilities(OP.propagate(basis, b, v, zg))
    assert _fp64_bar(Pg, Po).all(), np.abs(Pg - Po).max()


def test_velocity_scan_bases_against_oracle():
    import oracle_parallel as OP
    from oracle import wpccc_oracle as O
    import paper_2403_04252_gb300 as w
    sets_in = wi.batch_inputs(n_b=64)
    sets, c, ref = [], [], []
    for v, basis, paths in sets_in:
        g = w.Basis(basis)
        g.set_solve_mode(w.SOLVE_SCHUR)
        zg = paths.z[0]
        k = zg.size // 2
        seg = zg[k - 2:k + 3]            # four RK4 steps through closest approach
        b = np.array([paths.b[0]])       # b = 0.2: the smallest impact parameter
        sets.append((g, b, v, seg))
        t = torch.zeros((1, g.N), dtype=torch.complex128, device="cuda")
        t[:, 0] = 1.0
        c.append(t)
        ref.append(O.probabilities(OP.propagate(basis, float(b[0]), v, seg)))
    for mode, iters in ((0, 2), (5, 4), (5, 2)):
        for (g, _, _, _), t in zip(sets, c):
            g.set_refine_iters(iters)
            t.zero_()
            t[:, 0] = 1.0
        batch = w.Batch(sets, c, precision_mode=mode, autotune=False)
        batch.launch()
        batch.status()
        for (g, b, v, seg), t, Po in zip(sets, c, ref):
            P = w.probabilities(t).cpu().numpy()[0]
            if mode == 5 and iters == 2:
                assert np.abs(P - Po).max() <= 1e-6, (v, np.abs(P - Po).max())
            else:
                assert _fp64_bar(P, Po).all(), (v, mode, np.abs(P - Po).max())
        batch.close()
    for g, _, _, _ in sets:
        g.close()
