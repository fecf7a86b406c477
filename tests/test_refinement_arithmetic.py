"""The arithmetic claim behind the mixed-precision solve forms, checked on the CPU with numpy: the
Schur-complement factor of S computed entirely in FP32 (K rounded to complex64, C = I - K^+ K and its
Cholesky factor in complex64, every stage's two K products and two triangles in complex64), used as the
preconditioner of iterative refinement with FP64 residuals b - S x, reaches FP64 accuracy.

The error of the FP32 solve is about kappa(S) u_32, and each sweep multiplies it by about the same factor.
At the best-conditioned workload (p + H, kappa ~ 220 at b = 0.2) and the worst (the velocity scan at
v = 0.5 on its 72-node rule, kappa ~ 2e3), two solves (one correction) reach 4e-11 and 2e-8 relative, and
four reach the FP64 solve's own accuracy (5e-14 and 2e-13). The CUDA kernels are not involved; S comes
from the oracle.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import wpccc_inputs as wi
from oracle import wpccc_oracle as O


def _fp32_schur_solver(S, NT):
    K32 = S[:NT, NT:].astype(np.complex64)
    C32 = np.eye(S.shape[0] - NT, dtype=np.complex64) - K32.conj().T @ K32
    L32 = np.linalg.cholesky(C32)
    assert L32.dtype == np.complex64

    def solve(t):
        t = t.astype(np.complex64)
        tT, tP = t[:NT], t[NT:]
        u = tP - K32.conj().T @ tT
        kP = sla.solve_triangular(L32.conj().T, sla.solve_triangular(L32, u, lower=True), lower=False)
        assert kP.dtype == np.complex64
        return np.concatenate([tT - K32 @ kP, kP]).astype(np.complex128)
    return solve


def _sweeps(basis, b, v, n=4):
    S, H = O.assemble(basis, b, v, 0.0)
    NT = basis.T.N
    sv = np.linalg.svd(S[:NT, NT:], compute_uv=False)
    kappa = (1.0 + sv.max()) / (1.0 - sv.max())
    solve = _fp32_schur_solver(S, NT)
    rng = np.random.default_rng(3)
    rhs = H @ (rng.standard_normal(S.shape[0]) + 1j * rng.standard_normal(S.shape[0]))
    ref = np.linalg.solve(S, rhs)
    x = solve(rhs)
    errs = [np.abs(x - ref).max() / np.abs(ref).max()]
    for _ in range(n - 1):
        x = x + solve(rhs - S @ x)
        errs.append(np.abs(x - ref).max() / np.abs(ref).max())
    return kappa, errs


@pytest.mark.parametrize("case", ["p_H", "velocity_scan_v0.5"])
def test_fp32_schur_preconditioned_refinement_reaches_fp64(case):
    if case == "p_H":
        basis, _ = wi.config_inputs("p_H_2c_n4l3")
        v = 1.5
    else:
        v, basis, _ = wi.batch_inputs(n_b=2, speeds=(0.5,))[0]
    kappa, errs = _sweeps(basis, 0.2, v)
    assert 1e2 < kappa < 1e4
    u32 = 2.0 ** -24
    # the first solve is an FP32 solve: its error is of order kappa u_32 (not FP64 by accident)
    assert 1e-3 * kappa * u32 < errs[0] < 10.0 * kappa * u32
    # one correction contracts the error by about kappa u_32
    assert errs[1] < 10.0 * kappa * u32 * errs[0]
    # four solves: the FP64 solve's own accuracy (kappa u_64 with a margin)
    assert errs[3] < 1e-12
